// Batched coarse solves: (I + dT A) x_j = b_j for independent right-hand
// sides j = 0..count-1 (one implicit-Euler step each, §5.1), as one
// cooperative launch.  The grid is cut into T teams of C co-resident CTAs;
// team t solves systems t, t+T, ... with the team-local CG (fixed-order
// reductions, counter team barrier with a bounded wait) writing x_j directly
// into out_j.  Used where many coarse solves are known to be independent (the
// adjoint of a logged asynchronous run: every coarse solve of one slice's
// updates reads versions of the previous slice only).  A sequence of
// single-system cooperative solves pays each iteration's barriers and
// reductions once per system; a batch pays them once per team.
#include "common.cuh"
#include "device.cuh"

namespace pr {

namespace {

constexpr int GB_THREADS = 256;
constexpr unsigned long long GB_SOLVE_LIMIT_NS = 20ull * 1000 * 1000 * 1000;  // 20 s per solve

struct GBatchArgs {
  Geom g;
  StencilConst k;
  int var;
  StencilVar<double> gv;
  const double* const* b;   // count right-hand sides
  const double* const* x0;  // count starting guesses (none may alias its out)
  double* const* out;       // count solutions
  int count, C, T, maxit;
  double rtol;
  double* work;             // T x 3 M: r, p, q of each team
  double* part;             // T x 6 C reduction partials
  unsigned long long* bar;  // T barrier counters, zero at launch
  int* err;                 // 1 when a barrier wait expired
};

__global__ void __launch_bounds__(GB_THREADS, 2) gbatch_kernel(GBatchArgs a) {
  const int team = blockIdx.x / a.C;
  const int tb = blockIdx.x % a.C;
  const long long M = a.g.M;
  double* base = a.work + (size_t)team * 3 * M;
  for (int j = team; j < a.count; j += a.T) {
    const TeamBarrier bar{a.bar + team, a.C, globaltimer() + GB_SOLVE_LIMIT_NS, a.err};
    // every block of the team is done with the previous system's partials
    if (!bar.sync()) return;
    CgWork ws{a.out[j], base, base + M, base + 2 * M, a.part + (size_t)team * 6 * a.C};
    if (cg_core(a.g, a.k, a.var != 0, a.gv, a.b[j], a.x0[j], a.rtol, a.maxit, ws, bar, a.C, tb) < 0)
      return;
  }
}

}  // namespace

cudaError_t gbatch_solve(pr_ctx* c, const double* const* b_dev, const double* const* x0_dev,
                         double* const* out_dev, int count) {
  if (count <= 0) return cudaSuccess;
  cudaError_t e;
  if (!c->gb_work) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gbatch_kernel, GB_THREADS, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    c->gb_cap = per_sm * c->num_sms;
    // teams whose three CG vectors fit in about 80% of L2 (at least one)
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device);
    const double per_team = 3.0 * (double)c->g.M * sizeof(double);
    int t = l2 > 0 ? (int)(0.8 * l2 / per_team) : 1;
    if (t < 1) t = 1;
    if (t > c->gb_cap) t = c->gb_cap;
    c->gb_teams = t;
    e = cudaMalloc(&c->gb_work, (size_t)t * 3 * c->g.M * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->gb_part, (size_t)c->gb_cap * 6 * sizeof(double));
    if (e == cudaSuccess)
      e = cudaMalloc(&c->gb_bar, (size_t)c->gb_cap * sizeof(unsigned long long) + 64);
    if (e == cudaSuccess) {
      c->gb_err = reinterpret_cast<int*>(c->gb_bar + c->gb_cap);
      e = cudaMemsetAsync(c->gb_err, 0, sizeof(int), c->stream);
    }
    if (e != cudaSuccess) {
      // leave no half-built workspace behind: the next call starts over
      gbatch_free(c);
      return e;
    }
  }
  const int T = count < c->gb_teams ? count : c->gb_teams;
  const int C = c->gb_cap / T;
  if ((e = cudaMemsetAsync(c->gb_bar, 0, (size_t)T * sizeof(unsigned long long), c->stream)) !=
      cudaSuccess)
    return e;
  GBatchArgs a{};
  a.g = c->g;
  a.k = c->gst;
  a.var = c->var_kappa ? 1 : 0;
  a.gv = c->gvar;
  a.b = b_dev;
  a.x0 = x0_dev;
  a.out = out_dev;
  a.count = count;
  a.C = C;
  a.T = T;
  a.maxit = c->prob.g_maxit;
  a.rtol = c->prob.g_rtol;
  a.work = c->gb_work;
  a.part = c->gb_part;
  a.bar = c->gb_bar;
  a.err = c->gb_err;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((void*)gbatch_kernel, dim3(T * C), dim3(GB_THREADS), args, 0,
                                     c->stream);
}

// Error word of the batched solves (1 after a bounded wait expired); resets it.
int gbatch_take_error(pr_ctx* c) {
  if (!c->gb_err) return 0;
  int v = 0;
  if (cudaMemcpyAsync(&v, c->gb_err, sizeof v, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->gb_err, 0, sizeof v, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return 1;
  return v;
}

void gbatch_free(pr_ctx* c) {
  if (c->gb_work) cudaFree(c->gb_work);
  if (c->gb_part) cudaFree(c->gb_part);
  if (c->gb_bar) cudaFree(c->gb_bar);
  c->gb_work = c->gb_part = nullptr;
  c->gb_bar = nullptr;
  c->gb_err = nullptr;
  c->gb_teams = c->gb_cap = 0;
}

}  // namespace pr
