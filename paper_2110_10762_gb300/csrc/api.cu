// C ABI entry points (include/parareal.h) and the host side of the
// synchronous driver (Algorithm 1, §4.1).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace pr {

// NVTX range for the duration of a scope (timeline tools show the phases of
// the drivers; without an attached tool the calls are no-ops).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

int fail(pr_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(pr_ctx* c, cudaError_t e, const char* where) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
  // a failed allocation (or launch configuration) leaves a non-sticky "last
  // error" behind; clear it so the next call's launch checks do not report it
  cudaGetLastError();
  return fail(c, e == cudaErrorMemoryAllocation ? PR_ENOMEM : PR_ECUDA, buf);
}

namespace {

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// a coarse solve reports a negative iteration count when a bounded wait of its
// TMA-fed preconditioner steps expired (its result is then not valid)
const char* const kCoarseWaitExpired =
    "coarse solve: a bounded wait of the TMA-fed Chebyshev steps expired";

void free_problem(pr_ctx* c) {
  void* ptrs[] = {c->fcoef, c->fcoef32, c->gcoef, c->fsys0, c->v, c->w, c->tmp, c->f32a, c->f32b,
                  c->tma_err,
                  c->cg_x, c->cg_r, c->cg_p, c->cg_q, c->cg_w, c->cg_part, c->cg_iters_dev,
                  c->delta_dev, c->u0_stage, c->lam_stage, c->async_ws, c->adj_ws};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  c->fcoef = nullptr;
  c->fcoef32 = nullptr;
  c->gcoef = nullptr;
  c->fsys0 = nullptr;
  c->v = c->w = c->tmp = nullptr;
  c->f32a = c->f32b = nullptr;
  c->tma_err = nullptr;
  c->tma_ok = false;
  c->cg_x = c->cg_r = c->cg_p = c->cg_q = c->cg_w = c->cg_part = nullptr;
  c->cg_iters_dev = nullptr;
  c->delta_dev = nullptr;
  c->u0_stage = c->lam_stage = nullptr;
  c->lam_stage_bytes = 0;
  c->async_ws = nullptr;
  c->async_ws_bytes = 0;
  c->adj_ws = nullptr;
  c->adj_ws_bytes = 0;
  tri_free(&c->tri_f);
  tri_free(&c->tri_g);
  cn_free(c);
  cheb_free(c);
  gbatch_free(c);
  pipeline_free(c);
  c->fvar = {};
  c->gvar = {};
  c->fsysvar = {};
  c->fvar32 = {};
  c->has_problem = false;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, (count ? count : 1) * sizeof(T));
}

// Exact largest eigenvalue of the constant-coefficient A: sum_a 4/h_a^2 sin^2(n_a pi h_a / 2).
double lambda_max_const(const Geom& g) {
  double s = 0.0;
  const int n[3] = {g.nx, g.ny, g.nz};
  const double h[3] = {g.hx, g.hy, g.hz};
  for (int a = 0; a < g.dim; ++a) {
    const double sn = sin(n[a] * M_PI * h[a] / 2.0);
    s += 4.0 / (h[a] * h[a]) * sn * sn;
  }
  return s;
}

__global__ void min_kernel(const double* __restrict__ a, long long n, double* out) {
  __shared__ double sh[256];
  double m = 1e300;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    m = fmin(m, a[i]);
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

int check_ready(pr_ctx* c) {
  if (!c) return PR_EINVAL;
  if (!c->has_problem) return fail(c, PR_ESTATE, "no problem set (call parareal_set_problem)");
  return PR_OK;
}

cudaError_t fine_batch(pr_ctx* c, const double* in, double* out, int count) {
  return fine_apply(c, in, out, count);
}

}  // namespace

// F on `count` consecutive states: explicit steps, or implicit / trapezoidal
// steps by the tridiagonal solver (1D) or the batched CG kernel (2D/3D).
cudaError_t fine_apply(pr_ctx* c, const double* in, double* out, int count) {
  // the explicit and FP32 paths ping-pong through N-state workspaces
  if (count < 0 || count > c->prob.N) return cudaErrorInvalidValue;
  if (c->prob.f_scheme == PR_EXPLICIT_EULER)
    return explicit_fine(c, in, out, count, c->prob.f_steps, c->prob.f_prec);
  if (c->prob.f_scheme == PR_CRANK_NICOLSON && c->g.dim > 1) return cn_fine(c, in, out, count);
  return tri_solve_steps(c, &c->tri_f, in, out, count, c->prob.f_steps);
}
}  // namespace pr

using namespace pr;

extern "C" {

const char* parareal_version(void) { return "parareal-gb300 1.0 (sm_103a)"; }

const char* parareal_last_error(const pr_ctx* c) { return c ? c->err.c_str() : "null context"; }

int parareal_create(pr_ctx** out, int device, void* stream) {
  if (!out) return PR_EINVAL;
  *out = nullptr;
  pr_ctx* c = new (std::nothrow) pr_ctx();
  if (!c) return PR_ENOMEM;
  c->device = device;
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  int coop = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreate(&c->ev[i]);
  if (e != cudaSuccess || !coop) {
    delete c;
    return e != cudaSuccess ? PR_ECUDA : PR_EINVAL;
  }
  c->cg_blocks = cg_max_blocks(c->num_sms);
  *out = c;
  return PR_OK;
}

void parareal_destroy(pr_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_problem(c);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  delete c;
}

int parareal_set_problem(pr_ctx* c, const pr_problem* pin) {
  if (!c || !pin) return PR_EINVAL;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_problem(c);
  pr_problem p = *pin;
  if (p.dim < 1 || p.dim > 3) return fail(c, PR_EINVAL, "dim must be 1, 2 or 3");
  // each axis, then the running product, is bounded before the next
  // multiplication, so no product of large axes can overflow past the limits
  long long m_points = 1;
  for (int a = 0; a < 3; ++a) {
    if (a >= p.dim) p.n[a] = 1;
    if (p.n[a] < 1) return fail(c, PR_EINVAL, "every n[a] must be >= 1");
    if (p.n[a] > PR_MAX_POINTS) return fail(c, PR_EINVAL, "n[a] exceeds the point limit");
    m_points *= p.n[a];
    if (m_points > PR_MAX_POINTS)
      return fail(c, PR_EINVAL, "prod(n) exceeds the point limit (2^31 - 1 per state)");
  }
  if (p.N < 1) return fail(c, PR_EINVAL, "N must be >= 1");
  if (p.N > PR_MAX_SLICES) return fail(c, PR_EINVAL, "N exceeds the slice limit (65536)");
  if ((long long)(p.N + 1) > PR_MAX_TRAJ_POINTS / m_points)
    return fail(c, PR_EINVAL, "(N+1) * prod(n) exceeds the trajectory limit (2^40 points)");
  if (!(p.T > p.T0)) return fail(c, PR_EINVAL, "T must exceed T0");
  if (p.f_steps < 1) return fail(c, PR_EINVAL, "f_steps must be >= 1");
  if (p.f_scheme != PR_EXPLICIT_EULER && p.f_scheme != PR_IMPLICIT_EULER &&
      p.f_scheme != PR_CRANK_NICOLSON)
    return fail(c, PR_EINVAL, "unknown f_scheme");
  if (!(p.f_rtol >= 0.0)) return fail(c, PR_EINVAL, "f_rtol must be >= 0");
  if (p.f_rtol == 0.0) p.f_rtol = 1e-12;
  if (p.f_maxit <= 0) p.f_maxit = 10000;
  if (p.f_scheme == PR_IMPLICIT_EULER && p.dim != 1)
    return fail(c, PR_EINVAL, "implicit fine propagator is 1D (Thomas) only");
  if (p.f_prec != 64 && p.f_prec != 32) return fail(c, PR_EINVAL, "f_prec must be 64 or 32");
  if (p.f_prec == 32 && p.f_scheme != PR_EXPLICIT_EULER)
    return fail(c, PR_EINVAL, "FP32 fine steps need the explicit scheme");
  if (p.g_steps <= 0) p.g_steps = 1;
  if (p.g_solver == PR_SOLVER_THOMAS) {
    if (p.dim != 1) return fail(c, PR_EINVAL, "Thomas coarse solver is 1D only");
  } else if (p.g_solver == PR_SOLVER_CG) {
    if (p.g_steps != 1) return fail(c, PR_EINVAL, "CG coarse propagator takes one step");
  } else {
    return fail(c, PR_EINVAL, "unknown g_solver");
  }
  if (!(p.g_rtol >= 0.0)) return fail(c, PR_EINVAL, "g_rtol must be >= 0");
  if (p.g_maxit <= 0) p.g_maxit = 20000;
  if (!(p.tol >= 0.0)) return fail(c, PR_EINVAL, "tol must be >= 0");
  if (p.max_iter <= 0 || p.max_iter > p.N) p.max_iter = p.N;
  if (!p.u0_dev) return fail(c, PR_EINVAL, "u0_dev is NULL");
  if (!aligned16(p.u0_dev) || (p.kappa_dev && !aligned16(p.kappa_dev)))
    return fail(c, PR_EINVAL, "device arrays must be 16-byte aligned");
  if (p.dim == 1 && p.n[0] > 24000 &&
      (p.f_scheme != PR_EXPLICIT_EULER || p.g_solver == PR_SOLVER_THOMAS))
    return fail(c, PR_EINVAL, "1D Thomas path holds the state in shared memory: n <= 24000");

  Geom g{};
  g.dim = p.dim;
  g.nx = p.n[0];
  g.ny = p.n[1];
  g.nz = p.n[2];
  g.M = (long long)g.nx * g.ny * g.nz;
  g.hx = 1.0 / (g.nx + 1);
  g.hy = 1.0 / (g.ny + 1);
  g.hz = 1.0 / (g.nz + 1);
  c->g = g;
  c->prob = p;
  c->dT = (p.T - p.T0) / p.N;
  c->dt = c->dT / p.f_steps;
  c->var_kappa = p.kappa_dev != nullptr;
  const double rx = c->dt / (g.hx * g.hx), ry = p.dim > 1 ? c->dt / (g.hy * g.hy) : 0.0,
               rz = p.dim > 2 ? c->dt / (g.hz * g.hz) : 0.0;
  c->fst = {1.0 - 2.0 * (rx + ry + rz), rx, ry, rz};
  if (p.f_scheme == PR_CRANK_NICOLSON) {
    // half steps: right-hand side I - dt/2 A, system I + dt/2 A
    const double hx = 0.5 * rx, hy = 0.5 * ry, hz = 0.5 * rz;
    c->fst = {1.0 - 2.0 * (hx + hy + hz), hx, hy, hz};
    c->fsys = {1.0 + 2.0 * (hx + hy + hz), hx, hy, hz};
  }
  const double Rx = c->dT / (g.hx * g.hx), Ry = p.dim > 1 ? c->dT / (g.hy * g.hy) : 0.0,
               Rz = p.dim > 2 ? c->dT / (g.hz * g.hz) : 0.0;
  c->gst = {1.0 + 2.0 * (Rx + Ry + Rz), Rx, Ry, Rz};

  const size_t NM = (size_t)p.N * g.M;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  // stop at the first failed allocation (the rest would only be freed again)
  auto alloc = [&](auto** ptr, size_t count) {
    if (e == cudaSuccess) e = dalloc(ptr, count);
  };
  alloc(&c->v, NM);
  alloc(&c->w, NM);
  if (p.f_scheme == PR_EXPLICIT_EULER && p.f_prec == 64) alloc(&c->tmp, NM);
  if (p.f_prec == 32) {
    alloc(&c->f32a, NM);
    alloc(&c->f32b, NM);
  }
  alloc(&c->cg_x, g.M);
  alloc(&c->cg_r, g.M);
  alloc(&c->cg_p, g.M);
  alloc(&c->cg_q, g.M);
  alloc(&c->cg_w, g.M);
  alloc(&c->cg_part, 6 * (size_t)c->cg_blocks);
  alloc(&c->cg_iters_dev, (size_t)p.N + 1);
  alloc(&c->delta_dev, (size_t)p.N);
  if (e != cudaSuccess) {
    free_problem(c);
    return cuda_fail(c, e, "workspace allocation");
  }
  if (c->var_kappa) {
    e = build_var_coefficients(c);
    if (e != cudaSuccess) {
      free_problem(c);
      return cuda_fail(c, e, "variable-kappa coefficients");
    }
  }
  if (p.f_scheme == PR_IMPLICIT_EULER) chk(tri_build(c, &c->tri_f, g.nx, rx, p.kappa_dev));
  if (p.f_scheme == PR_CRANK_NICOLSON && p.dim == 1)
    chk(tri_build(c, &c->tri_f, g.nx, 0.5 * rx, p.kappa_dev, true));
  if (p.f_scheme == PR_CRANK_NICOLSON && p.dim > 1) chk(cn_alloc(c));
  if (p.g_solver == PR_SOLVER_THOMAS)
    chk(tri_build(c, &c->tri_g, g.nx, c->dT / p.g_steps / (g.hx * g.hx), p.kappa_dev));
  if (e != cudaSuccess) {
    free_problem(c);
    return cuda_fail(c, e, "tridiagonal tables");
  }
  tma_prepare(c);  // optional: the TMA-fed FP32 steps when their tensor maps encode
  if (p.g_solver == PR_SOLVER_CG) chk(coarse_bounds(c));
  if (p.g_solver == PR_SOLVER_CG && c->opt_g_cheb) chk(cheb_alloc(c));
  if (e != cudaSuccess) {
    free_problem(c);
    return cuda_fail(c, e, "coarse preconditioner");
  }
  // Stability of the explicit step: dt * lambda_max(A) <= 2 (exact for constant
  // kappa; Gershgorin bound, i.e. every diagonal c0 >= 0, for variable kappa).
  if (p.f_scheme == PR_EXPLICIT_EULER) {
    if (!c->var_kappa) {
      if (c->dt * lambda_max_const(g) > 2.0)
        return free_problem(c), fail(c, PR_EINVAL, "explicit fine step unstable: dt*lambda_max(A) > 2");
    } else {
      const int blocks = 64;
      double* d = c->cg_part;  // scratch
      min_kernel<<<blocks, 256, 0, c->stream>>>(c->fvar.c0, g.M, d);
      std::vector<double> h(blocks);
      chk(cudaMemcpyAsync(h.data(), d, blocks * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      chk(cudaStreamSynchronize(c->stream));
      if (e != cudaSuccess) {
        free_problem(c);
        return cuda_fail(c, e, "stability check");
      }
      if (*std::min_element(h.begin(), h.end()) < -1e-12)
        return free_problem(c),
               fail(c, PR_EINVAL, "explicit fine step unstable: Gershgorin bound dt*lambda_max(A) > 2");
    }
  }
  chk(cudaStreamSynchronize(c->stream));
  if (e != cudaSuccess) {
    free_problem(c);
    return cuda_fail(c, e, "set_problem");
  }
  c->last_k.assign(p.N, 0);
  c->last_delta.assign(p.N, 0.0);
  c->has_problem = true;
  return PR_OK;
}

int parareal_fine(pr_ctx* c, const double* in, double* out, int count) {
  int s = check_ready(c);
  if (s) return s;
  if (count < 0 || count > c->prob.N) return fail(c, PR_EINVAL, "count must be in [0, N]");
  if (!in || !out || !aligned16(in) || !aligned16(out)) return fail(c, PR_EINVAL, "bad pointer");
  const size_t bytes = (size_t)count * c->g.M * sizeof(double);
  if ((const char*)in < (const char*)out + bytes && (const char*)out < (const char*)in + bytes)
    return fail(c, PR_EINVAL, "in and out overlap");
  cudaSetDevice(c->device);
  PR_CUDA(c, fine_batch(c, in, out, count));
  PR_CUDA(c, cudaStreamSynchronize(c->stream));
  return PR_OK;
}

int parareal_coarse(pr_ctx* c, const double* in, const double* x0, double* out, int* iters) {
  int s = check_ready(c);
  if (s) return s;
  if (!in || !out || !aligned16(in) || !aligned16(out) || (x0 && !aligned16(x0)))
    return fail(c, PR_EINVAL, "bad pointer");
  cudaSetDevice(c->device);
  if (c->prob.g_solver == PR_SOLVER_THOMAS) {
    PR_CUDA(c, tri_solve_steps(c, &c->tri_g, in, out, 1, c->prob.g_steps));
    if (iters) *iters = 0;
  } else {
    CgArgs a{};
    a.b = in;
    a.x0 = x0;
    a.out = out;
    a.iters = c->cg_iters_dev;
    a.mode = CG_PLAIN;
    PR_CUDA(c, cg_solve(c, a));
    int it = 0;
    PR_CUDA(c, cudaMemcpyAsync(&it, c->cg_iters_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PR_CUDA(c, cudaStreamSynchronize(c->stream));
    if (it < 0) return fail(c, PR_ECUDA, kCoarseWaitExpired);
    if (iters) *iters = it;
  }
  PR_CUDA(c, cudaStreamSynchronize(c->stream));
  return PR_OK;
}

int parareal_correct(pr_ctx* c, const double* w_new, const double* v, const double* w_old,
                     double* lam, double* delta) {
  int s = check_ready(c);
  if (s) return s;
  if (!w_new || !v || !w_old || !lam) return fail(c, PR_EINVAL, "bad pointer");
  cudaSetDevice(c->device);
  PR_CUDA(c, cudaMemsetAsync(c->delta_dev, 0, sizeof(unsigned long long), c->stream));
  PR_CUDA(c, correct(c, w_new, v, w_old, lam, c->delta_dev));
  unsigned long long bits = 0;
  PR_CUDA(c, cudaMemcpyAsync(&bits, c->delta_dev, sizeof bits, cudaMemcpyDeviceToHost, c->stream));
  PR_CUDA(c, cudaStreamSynchronize(c->stream));
  if (delta) memcpy(delta, &bits, sizeof(double));
  return PR_OK;
}

int parareal_serial_fine(pr_ctx* c, double* lam, pr_stats* st) {
  int s = check_ready(c);
  if (s) return s;
  if (!lam || !aligned16(lam)) return fail(c, PR_EINVAL, "bad pointer");
  cudaSetDevice(c->device);
  const long long M = c->g.M;
  cn_take_iterations(c);
  PR_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
  PR_CUDA(c, cudaMemcpyAsync(lam, c->prob.u0_dev, M * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  for (int i = 1; i <= c->prob.N; ++i) PR_CUDA(c, fine_batch(c, lam + (i - 1) * M, lam + i * M, 1));
  PR_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
  PR_CUDA(c, cudaStreamSynchronize(c->stream));
  if (st) {
    memset(st, 0, sizeof *st);
    float ms = 0;
    cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
    st->t_total_ms = ms;
    st->t_fine_ms = ms;
    st->fine_lups = (long long)c->prob.N * M * c->prob.f_steps;
    st->launches = (long long)c->prob.N * fine_launch_count(c);
    st->fine_cg_iterations = (long long)cn_take_iterations(c);
    st->iterations = 0;
    st->converged = 1;
  }
  return PR_OK;
}

int parareal_set_option(pr_ctx* c, int option, double value) {
  if (!c) return PR_EINVAL;
  switch (option) {
    case PR_OPT_PIPELINE:
      c->opt_pipeline = value != 0.0 ? 1 : 0;
      return PR_OK;
    case PR_OPT_PIPELINE_CHUNKS:
      if (!(value >= 1.0 && value <= 1024.0)) return fail(c, PR_EINVAL, "chunks must be in [1, 1024]");
      c->opt_chunks = (int)value;
      return PR_OK;
    case PR_OPT_CG_BLOCKS_PER_SM:
      if (!(value >= 0.0 && value <= 32.0)) return fail(c, PR_EINVAL, "blocks per SM must be in [0, 32]");
      c->opt_cg_bps = (int)value;
      return PR_OK;
    case PR_OPT_G_CHEBYSHEV:
      if (!(value == 0.0 || (value >= 2.0 && value <= 64.0)))
        return fail(c, PR_EINVAL, "Chebyshev steps must be 0 or in [2, 64]");
      c->opt_g_cheb = (int)value;
      if (c->opt_g_cheb && c->has_problem) {
        cudaSetDevice(c->device);
        cudaError_t e = cheb_alloc(c);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
          c->opt_g_cheb = 0;  // keep the plain solver usable
          return cuda_fail(c, e, "Chebyshev workspaces");
        }
      }
      return PR_OK;
    case PR_OPT_F_STEPS_PER_PASS:
      if (!(value == 1.0 || value == 2.0))
        return fail(c, PR_EINVAL, "fine steps per pass must be 1 or 2");
      c->opt_f_blocking = (int)value;
      return PR_OK;
    case PR_OPT_G_CG:
      if (!(value == 0.0 || value == 1.0 || value == 2.0))
        return fail(c, PR_EINVAL, "coarse CG recurrence must be 0, 1 or 2");
      c->opt_g_cg = (int)value;
      return PR_OK;
    default:
      return fail(c, PR_EINVAL, "unknown option");
  }
}

int parareal_run_sync(pr_ctx* c, double* lam, pr_stats* st) {
  int s = check_ready(c);
  if (s) return s;
  if (!lam || !aligned16(lam)) return fail(c, PR_EINVAL, "bad pointer");
  cudaSetDevice(c->device);
  // the trapezoidal 2D/3D F is itself a cooperative launch over the whole
  // device, so it cannot overlap the coarse sweep: plain schedule
  const bool cn_grid = c->prob.f_scheme == PR_CRANK_NICOLSON && c->g.dim > 1;
  if (c->opt_pipeline && !cn_grid) return run_sync_pipelined(c, lam, st);
  NvtxRange range_all("parareal_run_sync");
  cn_take_iterations(c);
  const pr_problem& p = c->prob;
  const long long M = c->g.M;
  const int N = p.N;
  const bool thomas = p.g_solver == PR_SOLVER_THOMAS;
  pr_stats S{};
  float ms = 0, t_f = 0, t_g = 0;
  std::vector<unsigned long long> dbits(N);
  std::vector<int> iters(N + 1);

  PR_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
  PR_CUDA(c, cudaMemcpyAsync(lam, p.u0_dev, M * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  // Predictor (Algorithm 1, first lines): w_i^0 = G(lam_{i-1}^0), lam_i^0 = w_i^0.
  nvtxRangePushA("predictor");
  PR_CUDA(c, cudaMemsetAsync(c->cg_iters_dev, 0, (N + 1) * sizeof(int), c->stream));
  for (int i = 1; i <= N; ++i) {
    double* wi = c->w + (i - 1) * M;
    double* li = lam + i * M;
    const double* lp = lam + (i - 1) * M;
    if (thomas) {
      PR_CUDA(c, tri_solve_steps(c, &c->tri_g, lp, wi, 1, p.g_steps));
      PR_CUDA(c, vec_copy(c, li, wi, M));
      S.launches += 2;
    } else {
      S.launches += 1;
      CgArgs a{};
      a.b = lp;
      a.x0 = lp;
      a.out = wi;
      a.lam = li;
      a.iters = c->cg_iters_dev + i;
      a.mode = CG_PREDICTOR;
      PR_CUDA(c, cg_solve(c, a));
    }
  }
  PR_CUDA(c, cudaMemcpyAsync(iters.data(), c->cg_iters_dev, (N + 1) * sizeof(int),
                             cudaMemcpyDeviceToHost, c->stream));
  PR_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
  PR_CUDA(c, cudaStreamSynchronize(c->stream));
  nvtxRangePop();
  cudaEventElapsedTime(&t_g, c->ev[0], c->ev[1]);
  S.t_predictor_ms = t_g;
  for (int i = 1; i <= N; ++i) {
    if (iters[i] < 0) return fail(c, PR_ECUDA, kCoarseWaitExpired);
    S.cg_iterations += iters[i];
    S.coarse_solves += 1;
  }
  S.predictor_cg_iterations = S.cg_iterations;

  int k = 0;
  double maxd = 0.0;
  bool conv = false;
  while (k < p.max_iter) {
    const int count = N - k;
    // fine propagation of every active slice at once: v_i = F(lam_{i-1}^k), i = k+1..N
    PR_CUDA(c, cudaEventRecord(c->ev[2], c->stream));
    {
      NvtxRange r("fine batch");
      PR_CUDA(c, fine_batch(c, lam + (size_t)k * M, c->v + (size_t)k * M, count));
    }
    PR_CUDA(c, cudaEventRecord(c->ev[3], c->stream));
    nvtxRangePushA("coarse sweep");
    S.launches += fine_launch_count(c);
    S.fine_lups += (long long)count * M * p.f_steps;
    // sequential coarse sweep with the fused correction and increment
    PR_CUDA(c, cudaMemsetAsync(c->delta_dev, 0, N * sizeof(unsigned long long), c->stream));
    PR_CUDA(c, cudaMemsetAsync(c->cg_iters_dev, 0, (N + 1) * sizeof(int), c->stream));
    for (int i = k + 1; i <= N; ++i) {
      double* wi = c->w + (size_t)(i - 1) * M;
      double* vi = c->v + (size_t)(i - 1) * M;
      double* li = lam + (size_t)i * M;
      unsigned long long* di = c->delta_dev + (i - 1);
      if (i - 1 > k) {
        const double* lp = lam + (size_t)(i - 1) * M;  // lam_{i-1}^{k+1}, already updated
        if (thomas) {
          PR_CUDA(c, tri_solve_steps(c, &c->tri_g, lp, c->cg_x, 1, p.g_steps));
          PR_CUDA(c, correct(c, c->cg_x, vi, wi, li, di));
          PR_CUDA(c, vec_copy(c, wi, c->cg_x, M));
          S.launches += 3;
        } else {
          S.launches += cg_solve_launches(CG_CORRECT);
          CgArgs a{};
          a.b = lp;
          a.x0 = wi;
          a.out = wi;
          a.lam = li;
          a.v = vi;
          a.delta = di;
          a.iters = c->cg_iters_dev + i;
          a.mode = CG_CORRECT;
          PR_CUDA(c, cg_solve(c, a));
        }
      } else {
        // w_i^{k+1} = w_i^k: lam_i^{k+1} = (w_i^k + v_i) - w_i^k
        PR_CUDA(c, correct(c, wi, vi, wi, li, di));
        S.launches += 1;
      }
    }
    nvtxRangePop();
    PR_CUDA(c, cudaEventRecord(c->ev[4], c->stream));
    PR_CUDA(c, cudaMemcpyAsync(dbits.data(), c->delta_dev, N * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, c->stream));
    PR_CUDA(c, cudaMemcpyAsync(iters.data(), c->cg_iters_dev, (N + 1) * sizeof(int),
                               cudaMemcpyDeviceToHost, c->stream));
    PR_CUDA(c, cudaStreamSynchronize(c->stream));
    float a_ms = 0, b_ms = 0;
    cudaEventElapsedTime(&a_ms, c->ev[2], c->ev[3]);
    cudaEventElapsedTime(&b_ms, c->ev[3], c->ev[4]);
    t_f += a_ms;
    t_g += b_ms;
    maxd = 0.0;
    bool nan = false;
    for (int i = 0; i < N; ++i) {
      double d;
      memcpy(&d, &dbits[i], sizeof d);
      if (i >= k) c->last_delta[i] = d;
      if (d != d) nan = true;
      maxd = std::max(maxd, d);
    }
    for (int i = k + 2; i <= N; ++i) {
      if (iters[i] < 0) return fail(c, PR_ECUDA, kCoarseWaitExpired);
      S.cg_iterations += iters[i];
      S.coarse_solves += 1;
    }
    ++k;
    if (nan) maxd = NAN;
    if (maxd < p.tol || k == N) {
      conv = true;
      break;
    }
  }
  PR_CUDA(c, cudaEventRecord(c->ev[5], c->stream));
  PR_CUDA(c, cudaStreamSynchronize(c->stream));
  cudaEventElapsedTime(&ms, c->ev[0], c->ev[5]);
  for (int i = 0; i < N; ++i) c->last_k[i] = k;
  S.iterations = k;
  S.converged = conv ? 1 : 0;
  S.max_delta = maxd;
  S.t_total_ms = ms;
  S.t_fine_ms = t_f;
  S.t_coarse_ms = t_g;
  S.fine_cg_iterations = (long long)cn_take_iterations(c);
  if (st) *st = S;
  if (!conv && p.tol > 0.0) return fail(c, PR_ENOTCONV, "max_iter reached before tol");
  return PR_OK;
}

int parareal_run_sync_host(pr_ctx* c, const double* u0_host, double* lam_host, pr_stats* st) {
  int s = check_ready(c);
  if (s) return s;
  if (!u0_host || !lam_host) return fail(c, PR_EINVAL, "bad pointer");
  cudaSetDevice(c->device);
  const long long M = c->g.M;
  const size_t lam_bytes = (size_t)(c->prob.N + 1) * M * sizeof(double);
  if (!c->u0_stage) PR_CUDA(c, cudaMalloc(&c->u0_stage, M * sizeof(double)));
  if (c->lam_stage_bytes < lam_bytes) {
    if (c->lam_stage) cudaFree(c->lam_stage);
    c->lam_stage = nullptr;
    c->lam_stage_bytes = 0;
    PR_CUDA(c, cudaMalloc(&c->lam_stage, lam_bytes));
    c->lam_stage_bytes = lam_bytes;
  }
  PR_CUDA(c, cudaMemcpyAsync(c->u0_stage, u0_host, M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  const double* saved = c->prob.u0_dev;
  c->prob.u0_dev = c->u0_stage;
  int r = parareal_run_sync(c, c->lam_stage, st);
  c->prob.u0_dev = saved;
  if (r != PR_OK && r != PR_ENOTCONV) return r;
  PR_CUDA(c, cudaMemcpyAsync(lam_host, c->lam_stage, lam_bytes, cudaMemcpyDeviceToHost, c->stream));
  PR_CUDA(c, cudaStreamSynchronize(c->stream));
  return r;
}

int parareal_slice_stats(pr_ctx* c, int* k_host, double* delta_host) {
  int s = check_ready(c);
  if (s) return s;
  for (int i = 0; i < c->prob.N; ++i) {
    if (k_host) k_host[i] = c->last_k[i];
    if (delta_host) delta_host[i] = c->last_delta[i];
  }
  return PR_OK;
}

int parareal_run_async(pr_ctx* c, const pr_async_opts* o, double* lam, pr_stats* st,
                       pr_event* log, size_t log_cap, size_t* log_len) {
  int s = check_ready(c);
  if (s) return s;
  if (!o || !lam || !aligned16(lam)) return fail(c, PR_EINVAL, "bad pointer");
  cudaSetDevice(c->device);
  return pr::run_async(c, o, lam, st, log, log_cap, log_len);
}

int parareal_adjoint(pr_ctx* c, const double* gN, int K, double* grad_u0, double* grad_kappa) {
  int s = check_ready(c);
  if (s) return s;
  if (!gN || !grad_u0) return fail(c, PR_EINVAL, "bad pointer");
  if (K < 0 || K > c->prob.N) return fail(c, PR_EINVAL, "K must be in [0, N]");
  cudaSetDevice(c->device);
  return pr::run_adjoint(c, gN, K, grad_u0, grad_kappa);
}

int parareal_adjoint_async(pr_ctx* c, const pr_event* log, size_t n_events, const double* gN,
                           double* grad_u0, double* grad_kappa, double* lamN) {
  int s = check_ready(c);
  if (s) return s;
  if (!gN || !grad_u0) return fail(c, PR_EINVAL, "bad pointer");
  cudaSetDevice(c->device);
  return pr::run_adjoint_async(c, log, n_events, gN, grad_u0, grad_kappa, lamN);
}

}  // extern "C"
