// Discrete adjoint (reverse mode) of K synchronous Parareal iterations
// (Algorithm 1 of §4.1 with the prefix frozen and no early stop; Eq. (11)),
// for L = L(lambda_N^K): given dL/dlambda_N it returns dL/du0 and dL/dkappa.
//
// Structure (mirrors the forward pass):
//  * forward: predictor and K iterations with every iterate lambda^k and
//    coarse value w^k kept as a checkpoint (slice-boundary states only);
//  * reverse, iteration k = K-1..0:
//      - sequential coarse sweep i = N..k+1: the correction's adjoint
//        (wbar_i^{k+1} += g, wbar_i^k -= g with g = lambar_i^{k+1}), then
//        G^T = G by CG on wbar_i^{k+1} feeding lambar_{i-1}^{k+1}, and the
//        kappa-derivative of the coarse solve;
//      - batched fine adjoint over the active slices: the n_f fine states are
//        recomputed from the checkpoint lambda_{i-1}^k, then the transposed
//        step (S^T = S, the same stencil) runs backward while the
//        kappa-gradient kernel accumulates -dt * facegrad(a_{j+1}, u_j);
//  * reverse predictor.
// kappa-gradient of <a, A_kappa u>: every face (p,q) adds
// (a_p - a_q)(u_p - u_q) / (2 h^2) to both of its nodes (boundary ring
// included); the kernel gathers per node, so it is deterministic and needs
// no atomics.
//
// Adjoint of a logged asynchronous run (Eq. (12), Algorithm 2): the log fixes
// the computation graph.  Version 0 of slice i is the predictor value
// G lambda_{i-1}^0; event (i, k, vF, vG) makes
//   lambda_i^k = G lambda_{i-1}^{vG} + F lambda_{i-1}^{vF} - G lambda_{i-1}^{vF}
// (= F lambda_{i-1}^{vF} when vG = vF), the subtracted value being the stored
// coarse value of the fine input.  The forward pass replays the log slice by
// slice keeping every version; the reverse pass runs slices N..1 (a version
// depends only on versions of the previous slice): per slice, one CG solve
// G g per event with vG > vF, the fine adjoints of all its events batched,
// then the predictor step.
#include <algorithm>
#include <map>

#include "device.cuh"

namespace pr {
namespace {

__global__ void axpy_kernel(double* __restrict__ y, const double* __restrict__ x, double a,
                            long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

__device__ __forceinline__ double padded_val(const Geom& g, const double* u, int xr, int yr, int zr) {
  if (xr < 1 || xr > g.nx) return 0.0;
  if (g.dim > 1 && (yr < 1 || yr > g.ny)) return 0.0;
  if (g.dim > 2 && (zr < 1 || zr > g.nz)) return 0.0;
  const int y = g.dim > 1 ? yr - 1 : 0;
  const int z = g.dim > 2 ? zr - 1 : 0;
  return u[((long long)z * g.ny + y) * g.nx + (xr - 1)];
}

// kbar[node] += scale * sum_{s < count} sum_{faces f of node} (a_s diff)(u_s diff) / (2 h^2)
__global__ void facegrad_kernel(Geom g, double* __restrict__ kbar, const double* __restrict__ a,
                                const double* __restrict__ u, int count, double scale) {
  const int nxr = g.nx + 2;
  const int nyr = g.dim > 1 ? g.ny + 2 : 1;
  const int nzr = g.dim > 2 ? g.nz + 2 : 1;
  const long long total = (long long)nxr * nyr * nzr;
  const double ih[3] = {0.5 / (g.hx * g.hx), 0.5 / (g.hy * g.hy), 0.5 / (g.hz * g.hz)};
  const int n[3] = {g.nx, g.ny, g.nz};
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < total;
       r += (long long)gridDim.x * blockDim.x) {
    int c[3];
    c[0] = r % nxr;
    const long long rest = r / nxr;
    c[1] = g.dim > 1 ? (int)(rest % nyr) : 1;
    c[2] = g.dim > 2 ? (int)(rest / nyr) : 1;
    double acc = 0.0;
    for (int ax = 0; ax < g.dim; ++ax) {
      bool others_inside = true;
      for (int b = 0; b < g.dim; ++b)
        if (b != ax && (c[b] < 1 || c[b] > n[b])) others_inside = false;
      if (!others_inside) continue;
      for (int side = 0; side < 2; ++side) {
        // face between padded positions lo and lo+1 along ax
        const int lo = side == 0 ? c[ax] - 1 : c[ax];
        if (lo < 0 || lo > n[ax]) continue;
        int plo[3] = {c[0], c[1], c[2]}, phi[3] = {c[0], c[1], c[2]};
        plo[ax] = lo;
        phi[ax] = lo + 1;
        for (int s = 0; s < count; ++s) {
          const double* as = a + (long long)s * g.M;
          const double* us = u + (long long)s * g.M;
          const double da = padded_val(g, as, phi[0], phi[1], phi[2]) - padded_val(g, as, plo[0], plo[1], plo[2]);
          const double du = padded_val(g, us, phi[0], phi[1], phi[2]) - padded_val(g, us, plo[0], plo[1], plo[2]);
          acc += ih[ax] * da * du;
        }
      }
    }
    kbar[r] += scale * acc;
  }
}

long long ring_count(const Geom& g) {
  return (long long)(g.nx + 2) * (g.dim > 1 ? g.ny + 2 : 1) * (g.dim > 2 ? g.nz + 2 : 1);
}

}  // namespace

int run_adjoint(pr_ctx* c, const double* gN, int K, double* grad_u0, double* grad_kappa) {
  const pr_problem& p = c->prob;
  // explicit F (any dimension) or implicit F (1D, tridiagonal solves); G by CG
  // or, in 1D, by one Thomas step
  const bool implicit = p.f_scheme == PR_IMPLICIT_EULER;
  const bool thomas = p.g_solver == PR_SOLVER_THOMAS;
  if ((p.f_scheme != PR_EXPLICIT_EULER && !implicit) || p.f_prec != 64 || p.g_steps != 1)
    return fail(c, PR_EINVAL,
                "adjoint needs FP64 explicit or 1D implicit fine steps and one coarse step");
  const Geom& g = c->g;
  const long long M = g.M;
  const int N = p.N, nf = p.f_steps;
  const bool var = c->var_kappa;
  if (grad_kappa && !var) return fail(c, PR_EINVAL, "grad_kappa needs a variable-kappa problem");
  const long long Mr = ring_count(g);
  const size_t traj = (size_t)(K + 1) * (N + 1) * M;
  // recomputed fine states: u_1..u_{nf-1} (explicit) or u_1..u_nf (implicit)
  const size_t nstates = (size_t)std::max(implicit ? nf : nf - 1, 1);
  const size_t words = 4 * traj + nstates * N * M + 2 * (size_t)N * M + M +
                       (var ? (size_t)Mr : 0);
  const size_t bytes = words * sizeof(double);
  if (c->adj_ws_bytes < bytes) {
    if (c->adj_ws) cudaFree(c->adj_ws);
    c->adj_ws = nullptr;
    c->adj_ws_bytes = 0;
    PR_CUDA(c, cudaMalloc(&c->adj_ws, bytes));
    c->adj_ws_bytes = bytes;
  }
  double* base = static_cast<double*>(c->adj_ws);
  double* lam = base;
  double* wv = lam + traj;
  double* lb = wv + traj;
  double* wb = lb + traj;
  double* states = wb + traj;
  double* abuf0 = states + nstates * N * M;
  double* abuf1 = abuf0 + (size_t)N * M;
  double* zbuf = abuf1 + (size_t)N * M;
  double* kbar = var ? zbuf + M : nullptr;
  auto L = [&](double* arr, int k, int i) { return arr + ((size_t)k * (N + 1) + i) * M; };
  const int blocks = c->num_sms * 8;
  auto axpy = [&](double* y, const double* x, double a, long long n) {
    axpy_kernel<<<blocks, 256, 0, c->stream>>>(y, x, a, n);
    return cudaGetLastError();
  };
  auto G = [&](const double* b, double* out) {
    if (thomas) return tri_solve_steps(c, &c->tri_g, b, out, 1, 1);
    CgArgs a{};
    a.b = b;
    a.x0 = b;
    a.out = out;
    a.iters = c->cg_iters_dev;
    a.mode = CG_PLAIN;
    return cg_solve(c, a);
  };
  // one fine step on `count` states: explicit S or the implicit solve S^-1 (both symmetric)
  auto step = [&](const double* in, double* out, int count) {
    return implicit ? tri_solve_steps(c, &c->tri_f, in, out, count, 1)
                    : explicit_step64(c, in, out, count);
  };
  unsigned long long* dscratch = c->delta_dev;

  // ------------------------------------------------ forward with checkpoints
  PR_CUDA(c, cudaMemcpyAsync(L(lam, 0, 0), p.u0_dev, M * sizeof(double), cudaMemcpyDeviceToDevice,
                             c->stream));
  for (int i = 1; i <= N; ++i) {
    if (thomas) {
      PR_CUDA(c, G(L(lam, 0, i - 1), L(wv, 0, i)));
      PR_CUDA(c, vec_copy(c, L(lam, 0, i), L(wv, 0, i), M));
      continue;
    }
    CgArgs a{};
    a.b = L(lam, 0, i - 1);
    a.x0 = a.b;
    a.out = L(wv, 0, i);
    a.lam = L(lam, 0, i);
    a.iters = c->cg_iters_dev;
    a.mode = CG_PREDICTOR;
    PR_CUDA(c, cg_solve(c, a));
  }
  for (int k = 0; k < K; ++k) {
    PR_CUDA(c, cudaMemcpyAsync(L(lam, k + 1, 0), L(lam, k, 0), (size_t)(N + 1) * M * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->stream));
    PR_CUDA(c, cudaMemcpyAsync(L(wv, k + 1, 0), L(wv, k, 0), (size_t)(N + 1) * M * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->stream));
    PR_CUDA(c, fine_apply(c, L(lam, k, k), c->v + (size_t)k * M, N - k));
    for (int i = k + 1; i <= N; ++i) {
      double* vi = c->v + (size_t)(i - 1) * M;
      if (i - 1 > k && thomas) {
        PR_CUDA(c, G(L(lam, k + 1, i - 1), L(wv, k + 1, i)));
        PR_CUDA(c, cudaMemsetAsync(dscratch, 0, sizeof(unsigned long long), c->stream));
        PR_CUDA(c, correct(c, L(wv, k + 1, i), vi, L(wv, k, i), L(lam, k + 1, i), dscratch));
      } else if (i - 1 > k) {
        CgArgs a{};
        a.b = L(lam, k + 1, i - 1);
        a.x0 = L(wv, k + 1, i);
        a.out = L(wv, k + 1, i);
        a.lam = L(lam, k + 1, i);
        a.v = vi;
        a.delta = dscratch;
        a.iters = c->cg_iters_dev;
        a.mode = CG_CORRECT;
        PR_CUDA(c, cg_solve(c, a));
      } else {
        PR_CUDA(c, cudaMemsetAsync(dscratch, 0, sizeof(unsigned long long), c->stream));
        PR_CUDA(c, correct(c, L(wv, k + 1, i), vi, L(wv, k, i), L(lam, k + 1, i), dscratch));
      }
    }
  }

  // ------------------------------------------------------------- reverse
  PR_CUDA(c, cudaMemsetAsync(lb, 0, 2 * traj * sizeof(double), c->stream));  // lb and wb
  if (var) PR_CUDA(c, cudaMemsetAsync(kbar, 0, Mr * sizeof(double), c->stream));
  PR_CUDA(c, cudaMemcpyAsync(L(lb, K, N), gN, M * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  for (int k = K - 1; k >= 0; --k) {
    // coarse sweep in reverse order
    for (int i = N; i >= k + 1; --i) {
      const double* gk = L(lb, k + 1, i);
      PR_CUDA(c, axpy(L(wb, k + 1, i), gk, 1.0, M));
      PR_CUDA(c, axpy(L(wb, k, i), gk, -1.0, M));
      if (i - 1 > k) {
        PR_CUDA(c, G(L(wb, k + 1, i), zbuf));
        PR_CUDA(c, axpy(L(lb, k + 1, i - 1), zbuf, 1.0, M));
        if (var) {
          facegrad_kernel<<<blocks, 256, 0, c->stream>>>(g, kbar, zbuf, L(wv, k + 1, i), 1, -c->dT);
          PR_CUDA(c, cudaGetLastError());
        }
      } else {
        PR_CUDA(c, axpy(L(wb, k, i), L(wb, k + 1, i), 1.0, M));
      }
    }
    // frozen prefix (slices 0..k): lambda_i^{k+1} = lambda_i^k
    PR_CUDA(c, axpy(L(lb, k, 0), L(lb, k + 1, 0), 1.0, (long long)(k + 1) * M));
    PR_CUDA(c, axpy(L(wb, k, 0), L(wb, k + 1, 0), 1.0, (long long)(k + 1) * M));
    // batched fine adjoint for i = k+1..N: inputs lambda_{i-1}^k, vbar_i = lambar_i^{k+1}
    const int count = N - k;
    const double* x0 = L(lam, k, k);
    // states u_j (j >= 1) recomputed from the checkpoint u_0 = lambda_{i-1}^k
    for (int j = 1; j <= (int)nstates && (implicit || j < nf); ++j) {
      const double* src = j == 1 ? x0 : states + (size_t)(j - 2) * N * M;
      PR_CUDA(c, step(src, states + (size_t)(j - 1) * N * M, count));
    }
    PR_CUDA(c, cudaMemcpyAsync(abuf0, L(lb, k + 1, k + 1), (size_t)count * M * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->stream));
    double* a = abuf0;
    double* b = abuf1;
    for (int j = nf - 1; j >= 0; --j) {
      if (!implicit) {
        // explicit: d<a_{j+1}, S u_j> gives -dt facegrad(a_{j+1}, u_j); a_j = S a_{j+1}
        const double* uj = j == 0 ? x0 : states + (size_t)(j - 1) * N * M;
        if (var) {
          facegrad_kernel<<<blocks, 256, 0, c->stream>>>(g, kbar, a, uj, count, -c->dt);
          PR_CUDA(c, cudaGetLastError());
        }
        PR_CUDA(c, step(a, b, count));
      } else {
        // implicit: a_j = S^-1 a_{j+1}, then -dt facegrad(a_j, u_{j+1})
        PR_CUDA(c, step(a, b, count));
        if (var) {
          facegrad_kernel<<<blocks, 256, 0, c->stream>>>(g, kbar, b, states + (size_t)j * N * M,
                                                          count, -c->dt);
          PR_CUDA(c, cudaGetLastError());
        }
      }
      std::swap(a, b);
    }
    PR_CUDA(c, axpy(L(lb, k, k), a, 1.0, (long long)count * M));
  }
  // predictor in reverse
  for (int i = N; i >= 1; --i) {
    PR_CUDA(c, axpy(L(wb, 0, i), L(lb, 0, i), 1.0, M));
    PR_CUDA(c, G(L(wb, 0, i), zbuf));
    PR_CUDA(c, axpy(L(lb, 0, i - 1), zbuf, 1.0, M));
    if (var) {
      facegrad_kernel<<<blocks, 256, 0, c->stream>>>(g, kbar, zbuf, L(wv, 0, i), 1, -c->dT);
      PR_CUDA(c, cudaGetLastError());
    }
  }
  PR_CUDA(c, cudaMemcpyAsync(grad_u0, L(lb, 0, 0), M * sizeof(double), cudaMemcpyDeviceToDevice,
                             c->stream));
  if (grad_kappa)
    PR_CUDA(c, cudaMemcpyAsync(grad_kappa, kbar, Mr * sizeof(double), cudaMemcpyDeviceToDevice,
                               c->stream));
  PR_CUDA(c, cudaStreamSynchronize(c->stream));
  return PR_OK;
}

namespace {

struct AEvent {
  int vF, vG;
};

__global__ void scatter_add_kernel(double* __restrict__ y, const double* __restrict__ x, double a,
                                   long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

}  // namespace

int run_adjoint_async(pr_ctx* c, const pr_event* log, size_t n_events, const double* gN,
                      double* grad_u0, double* grad_kappa, double* lamN) {
  const pr_problem& p = c->prob;
  if (p.f_scheme != PR_EXPLICIT_EULER || p.g_solver != PR_SOLVER_CG || p.f_prec != 64)
    return fail(c, PR_EINVAL, "adjoint needs the FP64 explicit fine scheme and the CG coarse solver");
  const Geom& g = c->g;
  const long long M = g.M;
  const int N = p.N, nf = p.f_steps;
  const bool var = c->var_kappa;
  if (grad_kappa && !var) return fail(c, PR_EINVAL, "grad_kappa needs a variable-kappa problem");
  if (n_events && !log) return fail(c, PR_EINVAL, "log is NULL");

  // ---- the graph: events per slice in version order, validated like a replay
  std::vector<std::vector<AEvent>> ev(N + 1);
  {
    std::vector<std::map<int, AEvent>> bys(N + 1);
    for (size_t e = 0; e < n_events; ++e) {
      const pr_event& x = log[e];
      if (x.slice < 1 || x.slice > N || x.version < 1)
        return fail(c, PR_EINVAL, "log: slice or version out of range");
      if (!bys[x.slice].emplace(x.version, AEvent{x.vF, x.vG}).second)
        return fail(c, PR_EINVAL, "log: duplicate (slice, version)");
    }
    for (int i = 1; i <= N; ++i) {
      int expect = 1, prev_vG = 0;
      for (const auto& kv : bys[i]) {
        if (kv.first != expect++) return fail(c, PR_EINVAL, "log: versions of a slice not consecutive");
        const AEvent& a = kv.second;
        if (a.vF != prev_vG || a.vG < a.vF)
          return fail(c, PR_EINVAL, "log: fine input is not the previous coarse input");
        const int pred_max = i == 1 ? 0 : (int)bys[i - 1].size();
        if (a.vG > pred_max) return fail(c, PR_EINVAL, "log: input version never produced");
        prev_vG = a.vG;
        ev[i].push_back(a);
      }
    }
  }
  // version (i, v) lives at vbase[i] + v; coarse values of events at wbase[i] + k - 1
  std::vector<size_t> vbase(N + 1), wbase(N + 1);
  size_t nver = 1, nw = 0;
  vbase[0] = 0;
  int kmax = 1;
  for (int i = 1; i <= N; ++i) {
    vbase[i] = nver;
    nver += ev[i].size() + 1;
    wbase[i] = nw;
    nw += ev[i].size();
    kmax = std::max(kmax, (int)ev[i].size());
  }
  // events per batch of fine propagations / fine adjoints: all of a slice's
  // updates when the recomputed states fit in about 16 GB, at most 64
  const double per_event = (double)std::max(nf, 2) * M * sizeof(double);
  const int b_mem = std::max(1, (int)(16e9 / per_event));
  // (and at most N: the batched fine propagation ping-pongs through the N-state
  // workspace of the context)
  const int B = std::min(std::min(std::min(kmax, 64), b_mem), N);
  const long long Mr = ring_count(g);
  const size_t ptr_words = 3 * (2 * n_events + 16);  // device pointer triples of the batches
  const size_t words = 2 * nver * M + nw * M + (size_t)std::max(nf - 1, 1) * B * M +
                       3 * (size_t)B * M + M + (var ? (size_t)Mr : 0) + ptr_words;
  const size_t bytes = words * sizeof(double);
  if (c->adj_ws_bytes < bytes) {
    if (c->adj_ws) cudaFree(c->adj_ws);
    c->adj_ws = nullptr;
    c->adj_ws_bytes = 0;
    PR_CUDA(c, cudaMalloc(&c->adj_ws, bytes));
    c->adj_ws_bytes = bytes;
  }
  double* ver = static_cast<double*>(c->adj_ws);
  double* lb = ver + nver * M;
  double* W = lb + nver * M;
  double* states = W + nw * M;
  double* xbuf = states + (size_t)std::max(nf - 1, 1) * B * M;
  double* abuf0 = xbuf + (size_t)B * M;
  double* abuf1 = abuf0 + (size_t)B * M;
  double* zbuf = abuf1 + (size_t)B * M;
  double* kbar = var ? zbuf + M : nullptr;
  auto V = [&](double* arr, int i, int v) { return arr + (vbase[i] + v) * M; };
  const int blocks = c->num_sms * 8;
  auto axpy = [&](double* y, const double* x, double a, long long n) {
    axpy_kernel<<<blocks, 256, 0, c->stream>>>(y, x, a, n);
    return cudaGetLastError();
  };
  auto solve = [&](const double* b, const double* x0, double* out) {
    CgArgs a{};
    a.b = b;
    a.x0 = x0;
    a.out = out;
    a.iters = c->cg_iters_dev;
    a.mode = CG_PLAIN;
    return cg_solve(c, a);
  };
  // coarse value subtracted by event k (1-based) of slice i: the last coarse
  // value produced before it, or the predictor value lambda_i^0
  auto w_before = [&](int i, int k) -> double* {
    for (int j = k - 1; j >= 1; --j)
      if (ev[i][j - 1].vG > ev[i][j - 1].vF) return W + (wbase[i] + j - 1) * M;
    return V(ver, i, 0);
  };
  auto w_after = [&](int i, int k) -> double* {
    return ev[i][k - 1].vG > ev[i][k - 1].vF ? W + (wbase[i] + k - 1) * M : w_before(i, k);
  };

  // pointer triples (b, x0, out) of the batched coarse solves, one segment per
  // batch, kept for the whole call (the copies to the device are asynchronous)
  std::vector<const double*> ptrs;
  ptrs.reserve(3 * (2 * n_events + 16));
  const double** dptr = reinterpret_cast<const double**>(kbar ? kbar + Mr : zbuf + M);
  size_t dpos = 0;
  auto batch = [&](const std::vector<const double*>& bs, const std::vector<const double*>& xs,
                   const std::vector<double*>& outs) -> cudaError_t {
    const int n = (int)bs.size();
    if (n == 0) return cudaSuccess;
    const size_t at = ptrs.size();
    for (int q = 0; q < n; ++q) ptrs.push_back(bs[q]);
    for (int q = 0; q < n; ++q) ptrs.push_back(xs[q]);
    for (int q = 0; q < n; ++q) ptrs.push_back(outs[q]);
    const double** d = dptr + dpos;
    dpos += 3 * (size_t)n;
    cudaError_t e = cudaMemcpyAsync(d, ptrs.data() + at, 3 * n * sizeof(double*),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    // the third segment holds the (mutable) output pointers
    double* const* outs_dev = reinterpret_cast<double* const*>(const_cast<double**>(d + 2 * n));
    return gbatch_solve(c, d, d + n, outs_dev, n);
  };

  // ------------------------------------------------ forward replay
  // Slice by slice (a version depends only on versions of the previous slice):
  // the fine propagations of a slice's updates in batches of B, its coarse
  // solves in one batch started from the slice's predictor value, then the
  // corrections in version order.
  PR_CUDA(c, cudaMemcpyAsync(V(ver, 0, 0), p.u0_dev, M * sizeof(double), cudaMemcpyDeviceToDevice,
                             c->stream));
  for (int i = 1; i <= N; ++i) PR_CUDA(c, solve(V(ver, i - 1, 0), V(ver, i - 1, 0), V(ver, i, 0)));
  unsigned long long* dscratch = c->delta_dev;
  for (int i = 1; i <= N; ++i) {
    const int K = (int)ev[i].size();
    {
      std::vector<const double*> bs, xs;
      std::vector<double*> outs;
      for (int k = 1; k <= K; ++k) {
        const AEvent& a = ev[i][k - 1];
        if (a.vG == a.vF) continue;
        bs.push_back(V(ver, i - 1, a.vG));
        xs.push_back(V(ver, i, 0));
        outs.push_back(W + (wbase[i] + k - 1) * M);
      }
      PR_CUDA(c, batch(bs, xs, outs));
    }
    for (int k0 = 1; k0 <= K; k0 += B) {
      const int cnt = std::min(B, K - k0 + 1);
      for (int q = 0; q < cnt; ++q)
        PR_CUDA(c, cudaMemcpyAsync(xbuf + (size_t)q * M, V(ver, i - 1, ev[i][k0 + q - 1].vF),
                                   M * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      PR_CUDA(c, fine_apply(c, xbuf, abuf0, cnt));
      for (int q = 0; q < cnt; ++q) {
        const int k = k0 + q;
        PR_CUDA(c, cudaMemcpyAsync(V(ver, i, k), V(ver, i, k - 1), M * sizeof(double),
                                   cudaMemcpyDeviceToDevice, c->stream));
        PR_CUDA(c, correct(c, w_after(i, k), abuf0 + (size_t)q * M, w_before(i, k), V(ver, i, k),
                           dscratch));
      }
    }
  }
  if (gbatch_take_error(c)) return fail(c, PR_ECUDA, "batched coarse solve: a bounded wait expired");
  const int lastN = (int)ev[N].size();
  if (lamN)
    PR_CUDA(c, cudaMemcpyAsync(lamN, V(ver, N, lastN), M * sizeof(double), cudaMemcpyDeviceToDevice,
                               c->stream));

  // ------------------------------------------------------------- reverse
  PR_CUDA(c, cudaMemsetAsync(lb, 0, nver * M * sizeof(double), c->stream));
  if (var) PR_CUDA(c, cudaMemsetAsync(kbar, 0, Mr * sizeof(double), c->stream));
  PR_CUDA(c, axpy(V(lb, N, lastN), gN, 1.0, M));
  for (int i = N; i >= 1; --i) {
    const int K = (int)ev[i].size();
    // coarse terms: the solves z = G g of the updates whose coarse input changed,
    // in batches of B (their seeds g = lbar(i, k) are final), then the adjoint
    // accumulations and kappa terms in version order
    {
      std::vector<int> ks;
      for (int k = K; k >= 1; --k)
        if (ev[i][k - 1].vG != ev[i][k - 1].vF) ks.push_back(k);
      for (size_t q0 = 0; q0 < ks.size(); q0 += B) {
        const int cnt = (int)std::min<size_t>(B, ks.size() - q0);
        std::vector<const double*> bs, xs;
        std::vector<double*> outs;
        for (int q = 0; q < cnt; ++q) {
          bs.push_back(V(lb, i, ks[q0 + q]));
          xs.push_back(V(lb, i, ks[q0 + q]));
          outs.push_back(states + (size_t)q * M);
        }
        PR_CUDA(c, batch(bs, xs, outs));
        for (int q = 0; q < cnt; ++q) {
          const int k = ks[q0 + q];
          const AEvent& a = ev[i][k - 1];
          const double* z = states + (size_t)q * M;
          PR_CUDA(c, axpy(V(lb, i - 1, a.vG), z, 1.0, M));
          PR_CUDA(c, axpy(V(lb, i - 1, a.vF), z, -1.0, M));
          if (var) {
            facegrad_kernel<<<blocks, 256, 0, c->stream>>>(g, kbar, z, w_after(i, k), 1, -c->dT);
            facegrad_kernel<<<blocks, 256, 0, c->stream>>>(g, kbar, z, w_before(i, k), 1, c->dT);
            PR_CUDA(c, cudaGetLastError());
          }
        }
      }
    }
    // fine terms, batched over up to B events: gather inputs and adjoint seeds
    for (int k0 = 1; k0 <= K; k0 += B) {
      const int cnt = std::min(B, K - k0 + 1);
      for (int q = 0; q < cnt; ++q) {
        const AEvent& a = ev[i][k0 + q - 1];
        PR_CUDA(c, cudaMemcpyAsync(xbuf + (size_t)q * M, V(ver, i - 1, a.vF), M * sizeof(double),
                                   cudaMemcpyDeviceToDevice, c->stream));
        PR_CUDA(c, cudaMemcpyAsync(abuf0 + (size_t)q * M, V(lb, i, k0 + q), M * sizeof(double),
                                   cudaMemcpyDeviceToDevice, c->stream));
      }
      for (int j = 1; j < nf; ++j) {
        const double* src = j == 1 ? xbuf : states + (size_t)(j - 2) * B * M;
        PR_CUDA(c, explicit_step64(c, src, states + (size_t)(j - 1) * B * M, cnt));
      }
      double* a = abuf0;
      double* b = abuf1;
      for (int j = nf - 1; j >= 0; --j) {
        const double* uj = j == 0 ? xbuf : states + (size_t)(j - 1) * B * M;
        if (var) {
          facegrad_kernel<<<blocks, 256, 0, c->stream>>>(g, kbar, a, uj, cnt, -c->dt);
          PR_CUDA(c, cudaGetLastError());
        }
        PR_CUDA(c, explicit_step64(c, a, b, cnt));
        std::swap(a, b);
      }
      for (int q = 0; q < cnt; ++q) {
        scatter_add_kernel<<<blocks, 256, 0, c->stream>>>(V(lb, i - 1, ev[i][k0 + q - 1].vF),
                                                          a + (size_t)q * M, 1.0, M);
        PR_CUDA(c, cudaGetLastError());
      }
    }
    // predictor: lambda_i^0 = G lambda_{i-1}^0
    PR_CUDA(c, solve(V(lb, i, 0), V(lb, i, 0), zbuf));
    PR_CUDA(c, axpy(V(lb, i - 1, 0), zbuf, 1.0, M));
    if (var) {
      facegrad_kernel<<<blocks, 256, 0, c->stream>>>(g, kbar, zbuf, V(ver, i, 0), 1, -c->dT);
      PR_CUDA(c, cudaGetLastError());
    }
  }
  PR_CUDA(c, cudaMemcpyAsync(grad_u0, V(lb, 0, 0), M * sizeof(double), cudaMemcpyDeviceToDevice,
                             c->stream));
  if (grad_kappa)
    PR_CUDA(c, cudaMemcpyAsync(grad_kappa, kbar, Mr * sizeof(double), cudaMemcpyDeviceToDevice,
                               c->stream));
  PR_CUDA(c, cudaStreamSynchronize(c->stream));
  return PR_OK;
}

}  // namespace pr
