// Coarse propagator G: one backward-Euler step (I + dT A) x = b (§5.1),
// solved by textbook (Hestenes-Stiefel) conjugate gradients in FP64 as one
// cooperative persistent kernel: every block owns a grid-stride share of the
// points, dot products are warp-shuffle + block reductions followed by one
// grid barrier and a fixed-order sum of the block partials (deterministic:
// every block computes bit-identical scalars, so all take the same branch).
//
// The correction of Algorithm 1 (§4.1) is fused into the epilogue: while the
// solution x is still in the workspace the kernel forms
//     lam_i^{k+1} = (x + v_i) - w_i^k        (this operation order, no FMA)
// its max-norm increment against lam_i^k (Eq. (22)), and stores w_i = x.
#include <cooperative_groups.h>

#include "device.cuh"

namespace cg = cooperative_groups;

namespace pr {

namespace {

constexpr int CG_THREADS = RED_THREADS;

struct CgDev {
  Geom g;
  int var;
  StencilConst k;         // constant coefficients of I + dT A (off-diagonals -R_a)
  StencilVar<double> gv;  // variable coefficients (c0 diagonal, faces positive)
  const double* b;
  const double* x0;
  double* out;
  double* lam;
  const double* v;
  unsigned long long* delta;
  int* iters;
  int mode;
  CgWork ws;
  double rtol;
  int maxit;
};

struct GridBarrier {
  __device__ bool sync() const {
    cg::this_grid().sync();
    return true;
  }
};

// MINB = blocks per SM the register budget must allow.  The CG vectors of a
// grid up to about 2 M points stay in L2 and 2 blocks/SM are best (fewer
// partials and barrier arrivals); beyond that the phases stream from HBM and
// are latency-bound, so a 4-blocks/SM instance (<= 64 registers) keeps twice
// as many loads in flight (measured 707 -> ~550 us per iteration at 256^3).
template <int MINB>
__global__ void __launch_bounds__(CG_THREADS, MINB) cg_kernel(CgDev a) {
  const long long M = a.g.M;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  if (a.mode == CG_CORRECT && t0 == 0) *a.delta = 0ull;
  const int it = cg_core(a.g, a.k, a.var != 0, a.gv, a.b, a.x0, a.rtol, a.maxit, a.ws,
                         GridBarrier{}, gridDim.x, blockIdx.x);
  // epilogue (x is final in the workspace)
  const double* x = a.ws.x;
  if (a.mode == CG_PLAIN) {
    for (long long i = t0; i < M; i += nt) a.out[i] = x[i];
  } else if (a.mode == CG_PREDICTOR) {
    for (long long i = t0; i < M; i += nt) {
      const double xi = x[i];
      a.out[i] = xi;
      a.lam[i] = xi;
    }
  } else {
    unsigned long long dmax = 0ull;
    for (long long i = t0; i < M; i += nt) {
      const double xi = x[i];
      const double wo = a.out[i];
      const double ln = __dsub_rn(__dadd_rn(xi, a.v[i]), wo);
      const unsigned long long d = abs_bits(__dsub_rn(ln, a.lam[i]));
      dmax = d > dmax ? d : dmax;
      a.lam[i] = ln;
      a.out[i] = xi;
    }
    dmax = warp_max_u64(dmax);
    if ((threadIdx.x & 31) == 0 && dmax) atomicMax(a.delta, dmax);
  }
  if (t0 == 0) *a.iters = it;
}

__global__ void correct_kernel(const double* __restrict__ wn, const double* __restrict__ v,
                               const double* __restrict__ wo, double* __restrict__ lam,
                               unsigned long long* delta, long long M) {
  unsigned long long dmax = 0ull;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M;
       i += (long long)gridDim.x * blockDim.x) {
    const double ln = __dsub_rn(__dadd_rn(wn[i], v[i]), wo[i]);
    const unsigned long long d = abs_bits(__dsub_rn(ln, lam[i]));
    dmax = d > dmax ? d : dmax;
    lam[i] = ln;
  }
  dmax = warp_max_u64(dmax);
  if ((threadIdx.x & 31) == 0 && dmax) atomicMax(delta, dmax);
}

__global__ void copy_kernel(double* __restrict__ d, const double* __restrict__ s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = s[i];
}

constexpr long long CG_L2_POINTS = 2LL << 20;  // 5 FP64 vectors of 2 M points = 80 MB

template <int MINB>
int cg_blocks_of(int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_kernel<MINB>, CG_THREADS, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (per_sm > MINB) per_sm = MINB;
  return per_sm * num_sms;
}

}  // namespace

int cg_max_blocks(int num_sms) {
  const int a = cg_blocks_of<2>(num_sms), b = cg_blocks_of<4>(num_sms);
  return a > b ? a : b;
}

cudaError_t cg_solve(pr_ctx* c, const CgArgs& in) {
  CgDev a{};
  a.g = c->g;
  a.var = c->var_kappa ? 1 : 0;
  a.k = c->gst;
  a.gv = c->gvar;
  a.b = in.b;
  a.x0 = in.x0 ? in.x0 : in.b;
  a.out = in.out;
  a.lam = in.lam;
  a.v = in.v;
  a.delta = in.delta;
  a.iters = in.iters;
  a.mode = in.mode;
  a.ws = {c->cg_x, c->cg_r, c->cg_p, c->cg_q, c->cg_part};
  a.rtol = c->prob.g_rtol;
  a.maxit = c->prob.g_maxit;
  const bool big = c->g.M > CG_L2_POINTS;
  int cap = big ? cg_blocks_of<4>(c->num_sms) : cg_blocks_of<2>(c->num_sms);
  // a caller-chosen blocks-per-SM cap leaves room for concurrent kernels
  if (c->opt_cg_bps > 0 && c->opt_cg_bps * c->num_sms < cap) cap = c->opt_cg_bps * c->num_sms;
  long long want = (c->g.M + CG_THREADS * 4 - 1) / (CG_THREADS * 4);
  int blocks = (int)(want < cap ? want : cap);
  if (blocks > c->cg_blocks) blocks = c->cg_blocks;  // partials are sized for cg_blocks
  if (blocks < 1) blocks = 1;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(big ? (void*)cg_kernel<4> : (void*)cg_kernel<2>, dim3(blocks),
                                     dim3(CG_THREADS), args, 0, c->stream);
}

cudaError_t correct(pr_ctx* c, const double* w_new, const double* v, const double* w_old,
                    double* lam, unsigned long long* delta) {
  long long blocks = (c->g.M + 255) / 256;
  if (blocks > c->num_sms * 8) blocks = c->num_sms * 8;
  if (blocks < 1) blocks = 1;
  correct_kernel<<<(int)blocks, 256, 0, c->stream>>>(w_new, v, w_old, lam, delta, c->g.M);
  return cudaGetLastError();
}

cudaError_t vec_copy(pr_ctx* c, double* dst, const double* src, long long n) {
  long long blocks = (n + 255) / 256;
  if (blocks > c->num_sms * 8) blocks = c->num_sms * 8;
  if (blocks < 1) blocks = 1;
  copy_kernel<<<(int)blocks, 256, 0, c->stream>>>(dst, src, n);
  return cudaGetLastError();
}

}  // namespace pr
