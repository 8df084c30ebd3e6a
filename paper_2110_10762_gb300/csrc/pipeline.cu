// Pipelined synchronous Parareal: the same arithmetic as Algorithm 1 (§4.1,
// Eq. (11)), scheduled so that the fine propagation of iteration k+1 overlaps
// the sequential coarse sweep of iteration k.
//
// F for slice i at iteration k+1 needs only lam_{i-1}^{k+1}, which the sweep of
// iteration k produces at its slice i-1 (Algorithm 1's processor i-1 likewise
// starts its F before processor i).  The sweep runs on a high-priority stream;
// as soon as it has produced the inputs of a chunk of slices, that chunk's
// fine steps are launched on a low-priority stream, so they fill the GPU
// while the latency-bound coarse solves run.  The fine outputs are
// double-buffered by iteration parity; the sweep of iteration k+1 waits, slice
// chunk by slice chunk, for the fine results it consumes.  The predictor chain
// overlaps F of iteration 0 the same way.  If iteration k meets the tolerance,
// the speculative fine work of iteration k+1 is drained and discarded.
// Results are bitwise identical to the non-pipelined driver.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace pr {

void pipeline_free(pr_ctx* c) {
  if (c->s_sweep) cudaStreamDestroy(c->s_sweep);
  if (c->s_fine) cudaStreamDestroy(c->s_fine);
  for (cudaEvent_t e : c->pev) cudaEventDestroy(e);
  c->pev.clear();
  c->s_sweep = c->s_fine = nullptr;
  if (c->v2) cudaFree(c->v2);
  c->v2 = nullptr;
}

namespace {

cudaError_t fine_rows(pr_ctx* c, const double* lam, double* vbuf, int r0, int r1) {
  const long long M = c->g.M;
  if (r1 <= r0) return cudaSuccess;
  return fine_apply(c, lam + (size_t)r0 * M, vbuf + (size_t)r0 * M, r1 - r0);
}

}  // namespace

int run_sync_pipelined(pr_ctx* c, double* lam, pr_stats* st) {
  const pr_problem& p = c->prob;
  const long long M = c->g.M;
  const int N = p.N;
  const bool thomas = p.g_solver == PR_SOLVER_THOMAS;
  const int nch = std::max(1, std::min(c->opt_chunks, N));
  const int B = (N + nch - 1) / nch;  // rows per chunk
  cudaStream_t user = c->stream;
  if (!c->s_sweep) {
    int least = 0, greatest = 0;
    PR_CUDA(c, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    PR_CUDA(c, cudaStreamCreateWithPriority(&c->s_sweep, cudaStreamNonBlocking, greatest));
    PR_CUDA(c, cudaStreamCreateWithPriority(&c->s_fine, cudaStreamNonBlocking, least));
  }
  if (!c->v2) PR_CUDA(c, cudaMalloc(&c->v2, (size_t)N * M * sizeof(double)));
  // events: [0,2) run begin/end, then per parity: nch "fine chunk done", nch "inputs ready",
  // nch chunk-start and nch chunk-end timers
  const size_t need = 2 + 2 * 4 * (size_t)nch;
  while (c->pev.size() < need) {
    cudaEvent_t e;
    PR_CUDA(c, cudaEventCreate(&e));
    c->pev.push_back(e);
  }
  auto evF = [&](int par, int ch) { return c->pev[2 + (size_t)par * 4 * nch + ch]; };
  auto evL = [&](int par, int ch) { return c->pev[2 + (size_t)par * 4 * nch + nch + ch]; };
  auto evT0 = [&](int par, int ch) { return c->pev[2 + (size_t)par * 4 * nch + 2 * nch + ch]; };
  auto evT1 = [&](int par, int ch) { return c->pev[2 + (size_t)par * 4 * nch + 3 * nch + ch]; };
  double* vbuf[2] = {c->v, c->v2};

  pr_stats S{};
  float t_f = 0.f;
  std::vector<unsigned long long> dbits(N);
  std::vector<int> iters(N + 1);
  cudaEvent_t ev_begin = c->pev[0], ev_end = c->pev[1];

  // chunk bookkeeping of the fine batch of iteration kk: rows [kk, N) in chunks of B
  struct Batch {
    int kk = -1, next = 0, nchunks = 0;
    long long lups = 0;  // counted into the stats only if an iteration consumes the batch
  };
  auto chunk_lo = [&](int kk, int ch) { return kk + ch * B; };
  auto chunk_hi = [&](int kk, int ch) { return std::min(N, kk + (ch + 1) * B); };
  auto chunks_of = [&](int kk) { return kk >= N ? 0 : (N - kk + B - 1) / B; };
  // launch every chunk of batch b whose input rows are all ready (rows <= ready)
  auto launch_ready = [&](Batch& b, int ready) -> int {
    while (b.next < b.nchunks && chunk_hi(b.kk, b.next) - 1 <= ready) {
      const int par = b.kk & 1, ch = b.next;
      cudaError_t e = cudaEventRecord(evL(par, ch), c->s_sweep);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_fine, evL(par, ch), 0);
      if (e == cudaSuccess) e = cudaEventRecord(evT0(par, ch), c->s_fine);
      if (e == cudaSuccess) {
        c->stream = c->s_fine;
        e = fine_rows(c, lam, vbuf[par], chunk_lo(b.kk, ch), chunk_hi(b.kk, ch));
        c->stream = c->s_sweep;
      }
      if (e == cudaSuccess) e = cudaEventRecord(evT1(par, ch), c->s_fine);
      if (e == cudaSuccess) e = cudaEventRecord(evF(par, ch), c->s_fine);
      if (e != cudaSuccess) return cuda_fail(c, e, "pipelined fine chunk");
      S.launches += fine_launch_count(c);
      b.lups += (long long)(chunk_hi(b.kk, ch) - chunk_lo(b.kk, ch)) * M * p.f_steps;
      ++b.next;
    }
    return PR_OK;
  };
  auto fail_restore = [&](int code) {
    cudaStreamSynchronize(c->s_sweep);
    cudaStreamSynchronize(c->s_fine);
    c->stream = user;
    return code;
  };
  // fine time of a finished batch: sum of its chunk spans
  auto batch_time = [&](const Batch& b) {
    float tot = 0.f;
    for (int ch = 0; ch < b.next; ++ch) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, evT0(b.kk & 1, ch), evT1(b.kk & 1, ch));
      tot += ms;
    }
    return tot;
  };

  PR_CUDA(c, cudaEventRecord(ev_begin, user));
  PR_CUDA(c, cudaStreamWaitEvent(c->s_sweep, ev_begin, 0));
  PR_CUDA(c, cudaStreamWaitEvent(c->s_fine, ev_begin, 0));
  c->stream = c->s_sweep;
  int rc = PR_OK;
  Batch cur;
  cur.kk = 0;
  cur.nchunks = chunks_of(0);
  cudaError_t e = cudaMemcpyAsync(lam, p.u0_dev, M * sizeof(double), cudaMemcpyDeviceToDevice,
                                  c->s_sweep);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->cg_iters_dev, 0, (N + 1) * sizeof(int), c->s_sweep);
  if (e != cudaSuccess) return fail_restore(cuda_fail(c, e, "pipelined setup"));
  if ((rc = launch_ready(cur, 0)) != PR_OK) return fail_restore(rc);
  // predictor chain, overlapped with F of iteration 0
  for (int i = 1; i <= N; ++i) {
    double* wi = c->w + (size_t)(i - 1) * M;
    double* li = lam + (size_t)i * M;
    const double* lp = lam + (size_t)(i - 1) * M;
    if (thomas) {
      e = tri_solve_steps(c, &c->tri_g, lp, wi, 1, p.g_steps);
      if (e == cudaSuccess) e = vec_copy(c, li, wi, M);
      S.launches += 2;
    } else {
      CgArgs a{};
      a.b = lp;
      a.x0 = lp;
      a.out = wi;
      a.lam = li;
      a.iters = c->cg_iters_dev + i;
      a.mode = CG_PREDICTOR;
      e = cg_solve(c, a);
      S.launches += 1;
    }
    if (e != cudaSuccess) return fail_restore(cuda_fail(c, e, "pipelined predictor"));
    if ((rc = launch_ready(cur, i)) != PR_OK) return fail_restore(rc);
  }
  e = cudaMemcpyAsync(iters.data(), c->cg_iters_dev, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost,
                      c->s_sweep);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_sweep);
  if (e != cudaSuccess) return fail_restore(cuda_fail(c, e, "pipelined predictor"));
  for (int i = 1; i <= N; ++i) {
    if (iters[i] < 0)
      return fail_restore(fail(c, PR_ECUDA, "coarse solve: a bounded wait of the TMA-fed "
                                            "Chebyshev steps expired"));
    S.cg_iterations += iters[i];
    S.coarse_solves += 1;
  }
  S.predictor_cg_iterations = S.cg_iterations;

  int k = 0;
  double maxd = 0.0;
  bool conv = false;
  while (k < p.max_iter) {
    Batch nxt;
    nxt.kk = k + 1;
    nxt.nchunks = (k + 1 < p.max_iter) ? chunks_of(k + 1) : 0;
    const int par = k & 1;
    double* v = vbuf[par];
    e = cudaMemsetAsync(c->delta_dev, 0, N * sizeof(unsigned long long), c->s_sweep);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->cg_iters_dev, 0, (N + 1) * sizeof(int), c->s_sweep);
    if (e != cudaSuccess) return fail_restore(cuda_fail(c, e, "pipelined sweep"));
    int waited = -1;  // last chunk of batch k the sweep has waited for
    for (int i = k + 1; i <= N; ++i) {
      const int row = i - 1;  // fine input row of slice i
      const int ch = (row - k) / B;
      if (ch > waited) {
        if ((e = cudaStreamWaitEvent(c->s_sweep, evF(par, ch), 0)) != cudaSuccess)
          return fail_restore(cuda_fail(c, e, "pipelined wait"));
        waited = ch;
      }
      double* wi = c->w + (size_t)(i - 1) * M;
      double* vi = v + (size_t)(i - 1) * M;
      double* li = lam + (size_t)i * M;
      unsigned long long* di = c->delta_dev + (i - 1);
      if (i - 1 > k) {
        const double* lp = lam + (size_t)(i - 1) * M;
        if (thomas) {
          e = tri_solve_steps(c, &c->tri_g, lp, c->cg_x, 1, p.g_steps);
          if (e == cudaSuccess) e = correct(c, c->cg_x, vi, wi, li, di);
          if (e == cudaSuccess) e = vec_copy(c, wi, c->cg_x, M);
          S.launches += 3;
        } else {
          CgArgs a{};
          a.b = lp;
          a.x0 = wi;
          a.out = wi;
          a.lam = li;
          a.v = vi;
          a.delta = di;
          a.iters = c->cg_iters_dev + i;
          a.mode = CG_CORRECT;
          e = cg_solve(c, a);
          S.launches += cg_solve_launches(CG_CORRECT);
        }
      } else {
        e = correct(c, wi, vi, wi, li, di);
        S.launches += 1;
      }
      if (e != cudaSuccess) return fail_restore(cuda_fail(c, e, "pipelined sweep"));
      // lam_i^{k+1} is final: start the fine chunks of iteration k+1 whose inputs are ready
      if ((rc = launch_ready(nxt, i)) != PR_OK) return fail_restore(rc);
    }
    e = cudaMemcpyAsync(dbits.data(), c->delta_dev, N * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, c->s_sweep);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(iters.data(), c->cg_iters_dev, (N + 1) * sizeof(int),
                          cudaMemcpyDeviceToHost, c->s_sweep);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_sweep);
    if (e != cudaSuccess) return fail_restore(cuda_fail(c, e, "pipelined sweep"));
    t_f += batch_time(cur);
    S.fine_lups += cur.lups;  // speculative work of a batch no iteration uses is not counted
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
      if (iters[i] < 0)
        return fail_restore(fail(c, PR_ECUDA, "coarse solve: a bounded wait of the TMA-fed "
                                              "Chebyshev steps expired"));
      S.cg_iterations += iters[i];
      S.coarse_solves += 1;
    }
    ++k;
    cur = nxt;
    if (nan) maxd = NAN;
    if (maxd < p.tol || k == N) {
      conv = true;
      break;
    }
  }
  // drain speculative fine work of an iteration that will not run
  e = cudaEventRecord(ev_end, c->s_fine);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_sweep, ev_end, 0);
  if (e == cudaSuccess) e = cudaEventRecord(ev_end, c->s_sweep);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, ev_end, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_sweep);
  c->stream = user;
  if (e != cudaSuccess) return cuda_fail(c, e, "pipelined drain");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev_begin, ev_end);
  for (int i = 0; i < N; ++i) c->last_k[i] = k;
  S.iterations = k;
  S.converged = conv ? 1 : 0;
  S.max_delta = maxd;
  S.t_total_ms = ms;
  S.t_fine_ms = t_f;       // sum of the fine chunks' spans (they overlap the sweep)
  S.t_coarse_ms = 0.0;     // the sweep is not separable from the overlapped fine work
  if (st) *st = S;
  if (!conv && p.tol > 0.0) return fail(c, PR_ENOTCONV, "max_iter reached before tol");
  return PR_OK;
}

}  // namespace pr
