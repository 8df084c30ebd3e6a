// Trapezoidal-rule (Crank-Nicolson) fine propagator in 2D and 3D, the fine
// scheme of Table 1 (§5.1):
//   (I + dt/2 A) u' = (I - dt/2 A) u      per fine step, n_f steps per slice.
//
// One cooperative launch applies F to a whole batch of slices.  The grid is
// cut into T teams of C co-resident CTAs; team t takes slices t, t+T, ...
// and, for every fine step of a slice,
//   1. forms the right-hand side b = (I - dt/2 A) u pointwise (the explicit
//      half step, the same stencil as the explicit F with dt/2),
//   2. solves (I + dt/2 A) x = b by the team-local conjugate gradients used by
//      the coarse solver (fixed-order reductions, counter team barrier),
//      started from x0 = u and stopped when ||r||_2 <= f_rtol ||b||_2,
//   3. continues from x (two ping-pong buffers; the last step writes the
//      output slice directly).
// Every barrier wait is bounded by globaltimer (a per-step limit); on expiry
// the team stops and the host reports PR_ETIMEOUT-like failure through the
// error word.  FP64 throughout.
#include "common.cuh"
#include "device.cuh"

namespace pr {

namespace {

constexpr int CN_THREADS = 256;
constexpr unsigned long long CN_STEP_LIMIT_NS = 20ull * 1000 * 1000 * 1000;  // 20 s per step

struct CnArgs {
  Geom g;
  StencilConst ke;           // right-hand side operator I - dt/2 A (explicit-step form)
  StencilConst ks;           // system operator I + dt/2 A (coarse-operator form)
  int var;
  StencilVar<double> ev, sv; // variable-kappa forms of the same two operators
  const double* in;
  double* out;
  int count, steps, maxit, C, T;
  double rtol;
  double* work;              // T x 6 M: two iterates, b, r, p, q
  double* part;              // T x C x 6 reduction partials
  unsigned long long* bar;   // T barrier counters, zero at launch
  int* err;                  // set to 1 when a barrier wait expired
  unsigned long long* iters; // CG iterations of all fine steps (accumulated)
};

__global__ void __launch_bounds__(CN_THREADS, 2) cn_kernel(CnArgs a) {
  const int team = blockIdx.x / a.C;
  const int tb = blockIdx.x % a.C;
  const long long M = a.g.M;
  double* base = a.work + (size_t)team * 6 * M;
  double* X[2] = {base, base + M};
  double* b = base + 2 * M;
  CgWork ws{nullptr, base + 3 * M, base + 4 * M, base + 5 * M,
            a.part + (size_t)team * 6 * a.C};
  unsigned long long total = 0;
  for (int slice = team; slice < a.count; slice += a.T) {
    const double* src = a.in + (size_t)slice * M;
    for (int s = 0; s < a.steps; ++s) {
      const TeamBarrier bar{a.bar + team, a.C, globaltimer() + CN_STEP_LIMIT_NS, a.err};
      for_each_point(a.g, tb, a.C, [&](int x, int y, int z, long long i) {
        b[i] = fstep_xyz<double, double>(a.g, a.ke.c0, a.ke.rx, a.ke.ry, a.ke.rz, a.var != 0,
                                         a.ev, src, x, y, z, i);
      });
      // b complete, and every block done with the previous solve's partials
      if (!bar.sync()) return;
      ws.x = (s == a.steps - 1) ? a.out + (size_t)slice * M : X[s & 1];
      const int it = cg_core(a.g, a.ks, a.var != 0, a.sv, b, src, a.rtol, a.maxit, ws, bar,
                             a.C, tb);
      if (it < 0) return;
      total += (unsigned long long)it;
      src = ws.x;
    }
  }
  if (tb == 0 && threadIdx.x == 0 && total) atomicAdd(a.iters, total);
}

}  // namespace

int cn_capacity(int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cn_kernel, CN_THREADS, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * num_sms;
}

cudaError_t cn_alloc(pr_ctx* c) {
  const long long M = c->g.M;
  c->cn_cap = cn_capacity(c->num_sms);
  int T = c->prob.N < c->cn_cap ? c->prob.N : c->cn_cap;
  cudaError_t e = cudaErrorMemoryAllocation;
  // as many teams as the batch and the device allow; halve on allocation failure
  while (T >= 1) {
    e = cudaMalloc(&c->cn_work, (size_t)T * 6 * M * sizeof(double));
    if (e == cudaSuccess) break;
    cudaGetLastError();
    c->cn_work = nullptr;
    T /= 2;
  }
  if (e != cudaSuccess) return e;
  c->cn_teams = T;
  if ((e = cudaMalloc(&c->cn_part, (size_t)c->cn_cap * 6 * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->cn_bar, (size_t)c->cn_cap * sizeof(unsigned long long) + 64)) !=
      cudaSuccess)
    return e;
  // status word and iteration counter after the barrier counters
  c->cn_err = reinterpret_cast<int*>(c->cn_bar + c->cn_cap);
  c->cn_iters = c->cn_bar + c->cn_cap + 1;
  return cudaMemsetAsync(c->cn_bar, 0, (size_t)c->cn_cap * sizeof(unsigned long long) + 64,
                         c->stream);
}

void cn_free(pr_ctx* c) {
  if (c->cn_work) cudaFree(c->cn_work);
  if (c->cn_part) cudaFree(c->cn_part);
  if (c->cn_bar) cudaFree(c->cn_bar);
  c->cn_work = c->cn_part = nullptr;
  c->cn_bar = nullptr;
  c->cn_err = nullptr;
  c->cn_iters = nullptr;
  c->cn_teams = c->cn_cap = 0;
}

#ifndef PR_CN_L2_FRACTION
#define PR_CN_L2_FRACTION 0.8
#endif

// Teams for a batch of `count` slices: as many as the batch and the workspace
// allow, but no more than keep the teams' six CG vectors within about 80% of
// L2 (beyond that every CG iteration streams its vectors from HBM and the
// kernel is bound by HBM as much as by the FP64 pipe); the slices then run in
// waves, and the team count is evened out over the waves.
int cn_team_count(const pr_ctx* c, int count) {
  int T = count < c->cn_teams ? count : c->cn_teams;
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device) != cudaSuccess || l2 <= 0)
    return T;
  const double per_team = 6.0 * (double)c->g.M * sizeof(double);
  int t_l2 = (int)(PR_CN_L2_FRACTION * l2 / per_team);
  if (t_l2 < 1) t_l2 = 1;
  if (t_l2 < T) {
    const int waves = (count + t_l2 - 1) / t_l2;
    T = (count + waves - 1) / waves;
  }
  return T;
}

cudaError_t cn_fine(pr_ctx* c, const double* in, double* out, int count) {
  if (count <= 0) return cudaSuccess;
  const int T = cn_team_count(c, count);
  const int C = c->cn_cap / T;
  cudaError_t e = cudaMemsetAsync(c->cn_bar, 0, (size_t)T * sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return e;
  CnArgs a{};
  a.g = c->g;
  a.ke = c->fst;
  a.ks = c->fsys;
  a.var = c->var_kappa ? 1 : 0;
  a.ev = c->fvar;
  a.sv = c->fsysvar;
  a.in = in;
  a.out = out;
  a.count = count;
  a.steps = c->prob.f_steps;
  a.maxit = c->prob.f_maxit;
  a.rtol = c->prob.f_rtol;
  a.C = C;
  a.T = T;
  a.work = c->cn_work;
  a.part = c->cn_part;
  a.bar = c->cn_bar;
  a.err = c->cn_err;
  a.iters = c->cn_iters;
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((void*)cn_kernel, dim3(T * C), dim3(CN_THREADS), args, 0,
                                  c->stream);
  if (e != cudaSuccess) return e;
  // the error word is sticky: read it after the batch (one small copy)
  int err = 0;
  e = cudaMemcpyAsync(&err, c->cn_err, sizeof err, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess && err) e = cudaErrorTimeout;
  return e;
}

unsigned long long cn_take_iterations(pr_ctx* c) {
  if (!c->cn_iters) return 0;
  unsigned long long v = 0;
  if (cudaMemcpyAsync(&v, c->cn_iters, sizeof v, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->cn_iters, 0, sizeof v, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return 0;
  return v;
}

}  // namespace pr
