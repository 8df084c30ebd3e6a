// Asynchronous Parareal (Eq. (12), Algorithm 2 of §4.1) as one persistent
// cooperative kernel.
//
// Work decomposition.  The grid is T teams of C co-resident CTAs.  Team t
// owns slices t+1, t+1+T, ... and updates them one at a time; a team barrier
// (bounded wait) separates the phases of an update.  There is no global
// barrier: teams communicate only through the published versions of lam_i.
//
// One update of slice i (Algorithm 2's loop body), done by its team:
//   vF := the version of lam_{i-1} held in the slice's snapshot xs_i
//         (it is the coarse input of the previous update, so
//          w_i = G(lam_{i-1}^{vF}) is already known)
//   v   = F(xs_i)                                   fine propagation
//   vG  = freshest visible version of lam_{i-1}     (>= vF)
//   if vG > vF: xs_i := lam_{i-1}^{vG} (seqlock-checked copy),
//               w_new = G(xs_i) by CG started from w_i
//   else:       w_new = w_i  (unchanged input, no solve)
//   lam_i^{k+1} = (w_new + v) - w_i;  delta_i = max |lam_i^{k+1} - lam_i^k|
//   publish lam_i^{k+1} into ring slot (k+1) % R, then w_i := w_new.
// A version becomes visible to the successor at publish time + an optional
// injected delay (communication delay).  Each update is logged as
// (i, k+1, vF, vG, ...), which is all the oracle needs to replay the run.
//
// A slice is re-updated only when a newer predecessor version is visible
// (or always, in paper-literal mode).  The run stops when every slice has
// updated at least once and its last increment is below tol, or when no
// slice can change any more (quiescence: lam_i = F(lam_{i-1}) for all i),
// or at the wall-clock limit (status PR_ETIMEOUT).  Every spin is bounded.
// Optionally (verify mode) the host confirms a stop by the increment rule with
// the fixed-point residual max_i |lam_i - F(lam_{i-1})| (one batched F) and
// relaunches the kernel on its persistent state when the residual is too large.
#include <string.h>

#include <algorithm>
#include <vector>

#include <cmath>

#include "device.cuh"

namespace pr {
namespace {

constexpr int ATHREADS = RED_THREADS;
constexpr int RING = 3;

enum { DEC_IDLE = 0, DEC_UPDATE = 1, DEC_STOP = 2 };
enum { AST_OK = 0, AST_TIMEOUT = 1, AST_LOGFULL = 2, AST_BARRIER = 3 };

struct AsyncDev {
  Geom g;
  int N, T, C;
  int f_steps, f_prec;
  bool var;
  StencilConst fst, gst;
  StencilVar<double> fv, gv;
  StencilVar<float> fv32;
  double rtol, tol;
  int maxit;
  int paper_literal, quiescence, lazy;
  // trapezoidal F (2D/3D): right-hand side fst/fv, system fsys/fsv, CG f_rtol/f_maxit
  int cn;
  StencilConst fsys;
  StencilVar<double> fsv;
  double f_rtol;
  int f_maxit;
  int tcg_stride;                 // vectors per team in tcg (4, or 5 with the trapezoidal rhs)
  // scaled FP64 explicit steps (constant kappa): coefficients {c0/rx, -, ry/rx, rz/rx},
  // return period R (0: plain form) and the factors rx^R and rx^(steps since the
  // last return, at the final step)
  StencilConst fsc;
  int f_period;
  double f_sigma_R, f_sigma_last;
  unsigned long long* fine_cg;    // CG iterations of the trapezoidal fine steps
  const double* u0;
  // per slice (index i-1)
  double* ring;                   // N * RING * M
  int* ring_ver;                  // N * RING   (-1: empty or being written)
  unsigned long long* ring_vis;   // N * RING   visible-at time (globaltimer ns)
  int* latest;                    // N + 1      latest published version (slot 0: u0)
  double* xs;                     // N * M      predecessor snapshot (next F input)
  double* w;                      // N * M      coarse value G(xs)
  int* xver;                      // N          version held in xs
  int* kcount;                    // N          updates published
  double* delta;                  // N          last increment
  int* lastfg;                    // N          last update had vF == vG
  // per team
  double* tv;                     // T * M      fine result v
  double* tcg;                    // T * tcg_stride * M  CG x, r, p, q (FP64 fine ping-pong aliases
                                  // r, p), then the trapezoidal right-hand side b
  double* tpart;                  // T * 6 * C
  unsigned long long* bar;        // T      team barrier arrival counters
  int* ctrl;                      // T * 8  (two decision slots, seqlock words)
  unsigned long long* tdelta;     // T
  // global
  int* stop;
  int* status;
  int* barrier_err;
  unsigned long long* log_count;
  pr_event* log;
  long long log_cap;
  const int* delays;
  int delay_cols;
  double delay_unit_ns;
  unsigned long long timeout_ns;  // wall-clock limit, counted from each block's start
};

__device__ __forceinline__ long long slice_off(const AsyncDev& a, int i) {
  return (long long)(i - 1) * a.g.M;
}
__device__ __forceinline__ double* ring_slot(const AsyncDev& a, int i, int slot) {
  return a.ring + ((long long)(i - 1) * RING + slot) * a.g.M;
}

// Freshest version of lam_{j} visible at `now` (j >= 1); -1 if none; slot in *slot.
__device__ int freshest_visible(const AsyncDev& a, int j, unsigned long long now, int* slot) {
  int best = -1;
  for (int s = 0; s < RING; ++s) {
    const int v = ld_acquire(a.ring_ver + (j - 1) * RING + s);
    if (v < 0 || v <= best) continue;
    const unsigned long long vis = ld_acquire_u64(a.ring_vis + (j - 1) * RING + s);
    if (vis <= now) {
      best = v;
      *slot = s;
    }
  }
  return best;
}

// Slice i has work unless its last update is idempotent: it used the same
// predecessor version for F and G (vF == vG) and no newer version is
// visible.  In paper-literal mode it always has work.
__device__ bool has_work(const AsyncDev& a, int i, unsigned long long now) {
  if (ld_acquire(a.kcount + i - 1) == 0 || a.paper_literal) return true;
  int slot = -1;
  const bool newer = i > 1 && freshest_visible(a, i - 1, now, &slot) > ld_acquire(a.xver + i - 1);
  if (newer) return true;
  if (ld_acquire(a.lastfg + i - 1)) return false;  // idempotent: nothing to do
  if (!a.lazy || i == 1) return true;
  // lazy: the pending vF == vG update waits until the predecessor has settled
  // (its own last update idempotent with the latest of its predecessor)
  const int j = i - 1;
  const int pred_latest = j == 1 ? 0 : ld_acquire(a.latest + j - 1);
  return ld_acquire(a.kcount + j - 1) > 0 && ld_acquire(a.lastfg + j - 1) &&
         ld_acquire(a.xver + j - 1) == pred_latest;
}

// Stop test of the monitor (any team leader may evaluate it), scanning the
// slices in order.  Slice i is "settled" when its last update was idempotent
// (vF == vG == the predecessor's latest version): it cannot change again
// unless its predecessor does, and by induction along the scan a settled
// prefix stays settled.  Quiescence = every slice settled (then
// lam_i = F(lam_{i-1}) for all i).  Tolerance rule (Eq. (22) read per
// slice): every slice has updated and is settled or had a last increment
// below tol.
__device__ bool stop_condition(const AsyncDev& a) {
  bool quiet = true;
  bool below = !a.quiescence;
  for (int i = 1; i <= a.N; ++i) {
    const int k = ld_acquire(a.kcount + i - 1);
    if (k < 1) return false;
    const int pred_latest = i == 1 ? 0 : ld_acquire(a.latest + i - 1);
    const bool settled = !a.paper_literal && ld_acquire(a.lastfg + i - 1) &&
                         ld_acquire(a.xver + i - 1) == pred_latest;
    if (!settled) quiet = false;
    if (below && !settled) {
      const double d = __ldcg(a.delta + i - 1);
      if (!(d < a.tol)) below = false;
    }
    if (!quiet && !below) return false;
  }
  return quiet || below;
}

__device__ void set_status(const AsyncDev& a, int st) {
  atomicCAS(a.status, AST_OK, st);
  atomicExch(a.stop, 1);
}

// Trapezoidal fine propagation v = F(xs_i) by the team (Table 1's F): per
// step the right-hand side b = (I - dt/2 A) u, then (I + dt/2 A) x = b by the
// team CG from x0 = u; the iterates alternate between ws.x and v so that the
// last step ends in v.
__device__ bool team_fine_cn(const AsyncDev& a, const TeamBarrier& bar, const double* xs, double* v,
                             const CgWork& ws, double* b, int tb) {
  const Geom& g = a.g;
  const int S = a.f_steps;
  const double* src = xs;
  unsigned long long total = 0;
  for (int s = 0; s < S; ++s) {
    double* dst = ((S - 1 - s) % 2 == 0) ? v : ws.x;
    for_each_point(g, tb, a.C, [&](int x, int y, int z, long long i) {
      b[i] = fstep_xyz<double, double>(g, a.fst.c0, a.fst.rx, a.fst.ry, a.fst.rz, a.var, a.fv, src,
                                       x, y, z, i);
    });
    if (!bar.sync()) return false;
    CgWork w2 = ws;
    w2.x = dst;
    const int it = cg_core(g, a.fsys, a.var, a.fsv, b, src, a.f_rtol, a.f_maxit, w2, bar, a.C, tb);
    if (it < 0) return false;
    total += (unsigned long long)it;
    src = dst;
  }
  if (tb == 0 && threadIdx.x == 0 && total) atomicAdd(a.fine_cg, total);
  return true;
}

#ifndef PR_ASYNC_TILE2D
#define PR_ASYNC_TILE2D 1
#endif
constexpr int TEAM_RY = 4;  // rows per 2D tile of the team's fine steps

// FP64 constant-kappa fine propagation in the scaled form (as the batched
// kernel): the team carries v = u / sigma with sigma multiplied by rx every
// step, v' = (c0/rx) v + (w + e) + (ry/rx)(s + n) + (rz/rx)(b + f), and returns
// to u (times sigma = rx^j) every R steps and on the last step.
__device__ bool team_fine_scaled(const AsyncDev& a, const TeamBarrier& bar, const double* xs,
                                 double* v, double* pp0, double* pp1, int tb) {
  const Geom& g = a.g;
  const double ca = a.fsc.c0, cb = a.fsc.ry, cc = a.fsc.rz;
  const int S = a.f_steps, R = a.f_period;
  const double* src = xs;
  int since = 0;
  for (int s = 0; s < S; ++s) {
    double* dst = (s == S - 1) ? v : ((s & 1) ? pp1 : pp0);
    ++since;
    const bool back = s == S - 1 || since == R;
    const double sig = s == S - 1 ? a.f_sigma_last : a.f_sigma_R;
    const long long plane = (long long)g.nx * g.ny;
#if PR_ASYNC_TILE2D
    if (g.dim == 2) {
      // 2D: each warp walks tiles of 32 columns x TEAM_RY rows, carrying the
      // vertical neighbours in registers (three loads per update instead of five)
      const int nx = g.nx, ny = g.ny;
      const int tiles_x = (nx + 31) / 32;
      const int ntiles = tiles_x * ((ny + TEAM_RY - 1) / TEAM_RY);
      const int wpb = blockDim.x / 32, lane = threadIdx.x % 32;
      for (int t = tb * wpb + threadIdx.x / 32; t < ntiles; t += a.C * wpb) {
        const int ty = t / tiles_x;
        const int x = (t - ty * tiles_x) * 32 + lane;
        const int y0 = ty * TEAM_RY;
        if (x >= nx) continue;
        double sv = y0 > 0 ? src[(long long)(y0 - 1) * nx + x] : 0.0;
        double cur = src[(long long)y0 * nx + x];
#pragma unroll
        for (int j = 0; j < TEAM_RY; ++j) {
          const int y = y0 + j;
          if (y >= ny) break;
          const long long i = (long long)y * nx + x;
          const double nv = y + 1 < ny ? src[i + nx] : 0.0;
          const double w = x > 0 ? src[i - 1] : 0.0;
          const double e = x + 1 < nx ? src[i + 1] : 0.0;
          double res = fma(ca, cur, w + e);
          res = fma(cb, sv + nv, res);
          dst[i] = back ? res * sig : res;
          sv = cur;
          cur = nv;
        }
      }
    } else
#endif
    for_each_point(g, tb, a.C, [&](int x, int y, int z, long long i) {
      const double w = x > 0 ? src[i - 1] : 0.0;
      const double e = x + 1 < g.nx ? src[i + 1] : 0.0;
      double res = fma(ca, src[i], w + e);
      if (g.dim > 1) {
        const double sv = y > 0 ? src[i - g.nx] : 0.0;
        const double nv = y + 1 < g.ny ? src[i + g.nx] : 0.0;
        res = fma(cb, sv + nv, res);
      }
      if (g.dim > 2) {
        const double bv = z > 0 ? src[i - plane] : 0.0;
        const double fv = z + 1 < g.nz ? src[i + plane] : 0.0;
        res = fma(cc, bv + fv, res);
      }
      dst[i] = back ? res * sig : res;
    });
    if (back) since = 0;
    if (!bar.sync()) return false;
    src = dst;
  }
  return true;
}

// Fine propagation v = F(xs_i) by the team: f_steps explicit steps, one team
// barrier after each.  FP64 steps ping-pong through the CG r/p vectors; FP32
// steps through the same memory viewed as floats.
template <typename T>
__device__ bool team_fine(const AsyncDev& a, const TeamBarrier& bar, const double* xs, double* v,
                          double* pp0, double* pp1, int tb) {
  const Geom& g = a.g;
  const T c0 = T(a.fst.c0), rx = T(a.fst.rx), ry = T(a.fst.ry), rz = T(a.fst.rz);
  StencilVar<T> cv;
  if constexpr (sizeof(T) == 8) {
    cv = a.fv;
  } else {
    cv = a.fv32;
  }
  T* buf0 = reinterpret_cast<T*>(pp0);
  T* buf1 = reinterpret_cast<T*>(pp1);
  const int S = a.f_steps;
  if (S == 1) {
    for_each_point(g, tb, a.C, [&](int x, int y, int z, long long i) {
      v[i] = double(fstep_xyz<T, double>(g, c0, rx, ry, rz, a.var, cv, xs, x, y, z, i));
    });
    return bar.sync();
  }
  for_each_point(g, tb, a.C, [&](int x, int y, int z, long long i) {
    buf0[i] = fstep_xyz<T, double>(g, c0, rx, ry, rz, a.var, cv, xs, x, y, z, i);
  });
  if (!bar.sync()) return false;
  const T* src = buf0;
  for (int s = 1; s < S - 1; ++s) {
    T* dst = (src == buf0) ? buf1 : buf0;
    for_each_point(g, tb, a.C, [&](int x, int y, int z, long long i) {
      dst[i] = fstep_xyz<T, T>(g, c0, rx, ry, rz, a.var, cv, src, x, y, z, i);
    });
    if (!bar.sync()) return false;
    src = dst;
  }
  for_each_point(g, tb, a.C, [&](int x, int y, int z, long long i) {
    v[i] = double(fstep_xyz<T, T>(g, c0, rx, ry, rz, a.var, cv, src, x, y, z, i));
  });
  return bar.sync();
}

__global__ void __launch_bounds__(ATHREADS, 2) async_kernel(AsyncDev a) {
  const int team = blockIdx.x / a.C;
  const int tb = blockIdx.x % a.C;
  const bool leader = tb == 0 && threadIdx.x == 0;
  const long long M = a.g.M;
  const long long t0 = tb * (long long)blockDim.x + threadIdx.x;
  const long long nt = (long long)a.C * blockDim.x;
  const unsigned long long deadline = globaltimer() + a.timeout_ns;
  // barrier waits get a grace period beyond the run limit so that a normal
  // stop at the limit is not reported as a barrier failure
  TeamBarrier bar{a.bar + team, a.C, deadline + 2000000000ull, a.barrier_err};
  int* ctrl = a.ctrl + 8 * team;
  double* tv = a.tv + (long long)team * M;
  double* cgx = a.tcg + (long long)team * a.tcg_stride * M;
  CgWork ws{cgx, cgx + M, cgx + 2 * M, cgx + 3 * M, a.tpart + (long long)team * 6 * a.C};
  int cursor = 0;                        // round-robin over owned slices (leader only)
  const int n_own = team < a.N ? (a.N - 1 - team) / a.T + 1 : 0;
  // Decision words alternate between two slots: after an IDLE decision the
  // leader writes the next decision while a slower block of the team may still
  // be reading the previous one, so consecutive decisions must not share words.
  unsigned dnum = 0;

  while (true) {
    int* dslot = ctrl + 2 * (dnum++ & 1u);
    // ---------------- decision (leader) ----------------
    if (leader) {
      int dec = DEC_IDLE, slice = 0;
      const unsigned long long now = globaltimer();
      if (now > deadline) set_status(a, AST_TIMEOUT);
      if (ld_acquire(a.stop) || ld_acquire(a.barrier_err)) {
        dec = DEC_STOP;
      } else {
        for (int c = 0; c < n_own; ++c) {
          const int i = team + 1 + ((cursor + c) % n_own) * a.T;
          if (has_work(a, i, now)) {
            dec = DEC_UPDATE;
            slice = i;
            cursor = (cursor + c + 1) % n_own;
            break;
          }
        }
        if (dec == DEC_IDLE) {
          if (stop_condition(a)) {
            atomicExch(a.stop, 1);
            dec = DEC_STOP;
          } else {
            __nanosleep(2000);
          }
        }
      }
      dslot[0] = dec;
      dslot[1] = slice;
    }
    if (!bar.sync()) break;
    const int dec = __ldcg(dslot);
    if (dec == DEC_STOP) break;
    if (dec == DEC_IDLE) continue;
    const int i = __ldcg(dslot + 1);
    double* xs = a.xs + slice_off(a, i);
    double* w = a.w + slice_off(a, i);
    const int vF = ld_acquire(a.xver + i - 1);
    const int k = ld_acquire(a.kcount + i - 1);
    unsigned long long t_start = 0;
    if (leader) t_start = globaltimer();

    // ---------------- fine propagation v = F(xs_i) ----------------
    const bool ok = a.cn ? team_fine_cn(a, bar, xs, tv, ws, cgx + 4 * M, tb)
                    : a.f_prec == 32 ? team_fine<float>(a, bar, xs, tv, ws.r, ws.p, tb)
                    : a.f_period > 0 ? team_fine_scaled(a, bar, xs, tv, ws.r, ws.p, tb)
                                     : team_fine<double>(a, bar, xs, tv, ws.r, ws.p, tb);
    if (!ok) break;

    // ---------------- freshest visible predecessor version ----------------
    int vG = vF;
    for (int attempt = 0;; ++attempt) {
      if (leader) {
        int slot = -1, cand = -1;
        if (i > 1) cand = freshest_visible(a, i - 1, globaltimer(), &slot);
        ctrl[4] = cand > vF ? cand : vF;
        ctrl[5] = cand > vF ? slot : -1;
      }
      if (!bar.sync()) return;
      vG = __ldcg(ctrl + 4);
      const int slot = __ldcg(ctrl + 5);
      if (vG == vF) break;
      const double* src = ring_slot(a, i - 1, slot);
      for (long long p = t0; p < M; p += nt) xs[p] = __ldcg(src + p);
      __threadfence();
      if (!bar.sync()) return;
      if (leader) ctrl[6] = ld_acquire(a.ring_ver + (i - 2) * RING + slot) == vG ? 1 : 0;
      if (!bar.sync()) return;
      if (__ldcg(ctrl + 6)) break;   // copy consistent (seqlock check passed)
      if (attempt > 1000) {
        if (leader) set_status(a, AST_BARRIER);
        return;
      }
    }

    // ---------------- coarse solve w_new = G(xs_i) ----------------
    const double* wn = w;
    int cg_it = 0;
    if (vG > vF) {
      cg_it = cg_core(a.g, a.gst, a.var, a.gv, xs, w, a.rtol, a.maxit, ws, bar, a.C, tb);
      if (cg_it < 0) break;
      wn = ws.x;
    }

    // ---------------- correction, increment, publish ----------------
    const int s_new = (k + 1) % RING, s_cur = k % RING;
    if (leader) {
      atomicExch(a.ring_ver + (i - 1) * RING + s_new, -1);  // seqlock: slot being written
      a.tdelta[team] = 0ull;
      __threadfence();
    }
    if (!bar.sync()) break;
    {
      double* dst = ring_slot(a, i, s_new);
      const double* cur = ring_slot(a, i, s_cur);
      unsigned long long dmax = 0ull;
      for (long long p = t0; p < M; p += nt) {
        const double wo = w[p];
        const double x = wn[p];
        const double ln = __dsub_rn(__dadd_rn(x, tv[p]), wo);
        const unsigned long long d = abs_bits(__dsub_rn(ln, cur[p]));
        dmax = d > dmax ? d : dmax;
        dst[p] = ln;
        if (wn != w) w[p] = x;
      }
      dmax = warp_max_u64(dmax);
      if ((threadIdx.x & 31) == 0 && dmax) atomicMax(a.tdelta + team, dmax);
      __threadfence();
    }
    if (!bar.sync()) break;
    if (leader) {
      const unsigned long long now = globaltimer();
      unsigned long long vis = now;
      if (a.delays && a.delay_cols > 0)
        vis += (unsigned long long)(a.delays[(long long)(i - 1) * a.delay_cols + (k % a.delay_cols)] *
                                    a.delay_unit_ns);
      const unsigned long long dbits = atomicAdd(a.tdelta + team, 0ull);
      double dl;
      memcpy(&dl, &dbits, sizeof dl);
      st_release_u64(a.ring_vis + (i - 1) * RING + s_new, vis);
      st_release(a.ring_ver + (i - 1) * RING + s_new, k + 1);
      st_release(a.latest + i, k + 1);
      __stcg(a.delta + i - 1, dl);
      st_release(a.xver + i - 1, vG);
      st_release(a.lastfg + i - 1, vG == vF ? 1 : 0);
      __threadfence();
      st_release(a.kcount + i - 1, k + 1);
      const unsigned long long idx = atomicAdd(a.log_count, 1ull);
      if ((long long)idx < a.log_cap) {
        pr_event e;
        e.slice = i;
        e.version = k + 1;
        e.vF = vF;
        e.vG = vG;
        e.cg_iters = cg_it;
        e.team = team;
        e.delta = dl;
        e.t_start = t_start;
        e.t_end = vis;
        a.log[idx] = e;
      } else {
        set_status(a, AST_LOGFULL);
      }
      if (stop_condition(a)) atomicExch(a.stop, 1);
    }
  }
}

__global__ void async_init(AsyncDev a) {
  const long long M = a.g.M;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)a.N * RING;
       t += (long long)gridDim.x * blockDim.x) {
    a.ring_ver[t] = (t % RING) == 0 ? 0 : -1;
    a.ring_vis[t] = 0ull;
  }
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t <= a.N;
       t += (long long)gridDim.x * blockDim.x) {
    a.latest[t] = 0;
    if (t < a.N) {
      a.xver[t] = 0;
      a.kcount[t] = 0;
      a.delta[t] = __longlong_as_double(0x7ff0000000000000LL);  // +inf
      a.lastfg[t] = 0;
    }
  }
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < a.T;
       t += (long long)gridDim.x * blockDim.x)
    a.bar[t] = 0ull;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 8LL * a.T;
       t += (long long)gridDim.x * blockDim.x)
    a.ctrl[t] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.stop = 0;
    *a.status = 0;
    *a.barrier_err = 0;
    *a.log_count = 0ull;
    *a.fine_cg = 0ull;
  }
  (void)M;
}

constexpr int ASYNC_MAX_VERIFY = 100;  // residual checks of one run (verify mode)

// out <- bits of max_p |a_p - b_p| over n values (non-negative doubles order
// like their bit patterns); out must be zero beforehand.
__global__ void resid_kernel(const double* __restrict__ a, const double* __restrict__ b,
                             long long n, unsigned long long* out) {
  unsigned long long m = 0ull;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long d = abs_bits(a[i] - b[i]);
    m = d > m ? d : m;
  }
  m = warp_max_u64(m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// lam_out row i <- slice i's latest version (row 0 = u0 already there).
__global__ void async_gather(AsyncDev a, double* lam) {
  const long long M = a.g.M;
  for (int i = 1 + blockIdx.y; i <= a.N; i += gridDim.y) {
    const int k = a.kcount[i - 1];
    const double* src = ring_slot(a, i, k % RING);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < M;
         p += (long long)gridDim.x * blockDim.x)
      lam[(long long)i * M + p] = src[p];
  }
}

int async_max_blocks_per_sm() {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, async_kernel, ATHREADS, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm;
}

}  // namespace

int run_async(pr_ctx* c, const pr_async_opts* o, double* lam, pr_stats* st, pr_event* log_host,
              size_t log_cap, size_t* log_len) {
  const pr_problem& p = c->prob;
  const bool cn = p.f_scheme == PR_CRANK_NICOLSON;
  if ((p.f_scheme != PR_EXPLICIT_EULER && !(cn && c->g.dim > 1)) || p.g_solver != PR_SOLVER_CG)
    return fail(c, PR_EINVAL,
                "asynchronous path needs the explicit (or, in 2D/3D, trapezoidal) fine scheme and "
                "the CG coarse solver");
  if (o->timeout_s <= 0.0) return fail(c, PR_EINVAL, "timeout_s must be > 0");
  if (o->delays_dev && o->delay_cols <= 0) return fail(c, PR_EINVAL, "delay_cols must be > 0");
  const long long M = c->g.M;
  const int N = p.N;
  const int capacity = c->num_sms * async_max_blocks_per_sm();
  int C = o->ctas_per_slice;
  if (C <= 0) {
    // automatic: about as many teams as their CG working sets (six or seven
    // M-vectors each) fit in L2.  A team's update then runs from L2 instead of
    // streaming its vectors from HBM, and fewer, larger teams also pass the
    // fresh coarse values on sooner (measured at 1024^2: 3 teams of 101 CTAs
    // 6.7 s against 19.9 s for 64 teams of 4; at 192^3 one team 23.8 s against
    // a time-out for 128 teams of 2).  Grids so small that every slice's team
    // fits keep small teams (at most 8 CTAs).
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device) != cudaSuccess) l2 = 0;
    const double per_team = (cn ? 7.0 : 6.0) * (double)M * sizeof(double);
    long long t_l2 = l2 > 0 ? std::llround(l2 / per_team) : N;
    if (t_l2 < 1) t_l2 = 1;
    if (t_l2 >= N)
      C = std::max(1, std::min(8, capacity / N));
    else
      C = std::max(1, capacity / (int)t_l2);
  }
  if (C > capacity) C = capacity;
  int T = std::min(N, capacity / C);
  if (T < 1) return fail(c, PR_EINVAL, "ctas_per_slice exceeds the co-resident capacity");

  // workspace layout (doubles first, then 8-byte scalars, then ints)
  const size_t d_ring = (size_t)N * RING * M, d_xs = (size_t)N * M, d_tv = (size_t)T * M,
               d_tcg = (size_t)T * (cn ? 5 : 4) * M, d_tpart = (size_t)T * 6 * C, d_delta = N;
  const size_t n_dbl = d_ring + d_xs + d_tv + d_tcg + d_tpart + d_delta;
  const size_t n_u64 = (size_t)N * RING + T + 1 + T + 1;  // ring_vis, tdelta, log_count, bar, fine_cg
  const size_t n_int = (size_t)N * RING + (N + 1) + 4 * (size_t)N + 2 * (size_t)T + 8 * (size_t)T + 3;
  const size_t bytes = n_dbl * 8 + n_u64 * 8 + n_int * 4 + 256;
  if (c->async_ws_bytes < bytes) {
    if (c->async_ws) cudaFree(c->async_ws);
    c->async_ws = nullptr;
    c->async_ws_bytes = 0;
    PR_CUDA(c, cudaMalloc(&c->async_ws, bytes));
    c->async_ws_bytes = bytes;
  }
  pr_event* dlog = nullptr;
  if (log_cap) PR_CUDA(c, cudaMalloc(&dlog, log_cap * sizeof(pr_event)));

  AsyncDev a{};
  a.g = c->g;
  a.N = N;
  a.T = T;
  a.C = C;
  a.f_steps = p.f_steps;
  a.f_prec = p.f_prec;
  a.var = c->var_kappa;
  a.fst = c->fst;
  a.gst = c->gst;
  a.fv = c->fvar;
  a.gv = c->gvar;
  a.fv32 = c->fvar32;
  a.rtol = p.g_rtol;
  a.tol = p.tol;
  a.maxit = p.g_maxit;
  a.paper_literal = o->paper_literal;
  a.quiescence = o->quiescence;
  a.lazy = o->lazy;
  a.cn = cn ? 1 : 0;
  a.fsys = c->fsys;
  a.fsv = c->fsysvar;
  a.f_rtol = p.f_rtol;
  a.f_maxit = p.f_maxit;
  a.tcg_stride = cn ? 5 : 4;
  a.f_period = 0;
  if (!cn && !c->var_kappa && p.f_prec == 64 && p.f_steps > 1) {
    const int R = scaled_period(c->fst.rx);
    if (R > 0) {
      const double rx = c->fst.rx;
      a.f_period = R;
      a.fsc = {c->fst.c0 / rx, 1.0, c->fst.ry / rx, c->fst.rz / rx};
      a.f_sigma_R = std::pow(rx, R);
      const int rem = p.f_steps % R;
      a.f_sigma_last = std::pow(rx, rem == 0 ? R : rem);
    }
  }
  a.u0 = p.u0_dev;
  double* dp = static_cast<double*>(c->async_ws);
  a.ring = dp;
  dp += d_ring;
  a.xs = dp;
  dp += d_xs;
  a.tv = dp;
  dp += d_tv;
  a.tcg = dp;
  dp += d_tcg;
  a.tpart = dp;
  dp += d_tpart;
  a.delta = dp;
  dp += d_delta;
  unsigned long long* up = reinterpret_cast<unsigned long long*>(dp);
  a.ring_vis = up;
  up += (size_t)N * RING;
  a.tdelta = up;
  up += T;
  a.log_count = up;
  up += 1;
  a.bar = up;
  up += T;
  a.fine_cg = up;
  up += 1;
  int* ip = reinterpret_cast<int*>(up);
  a.ring_ver = ip;
  ip += (size_t)N * RING;
  a.latest = ip;
  ip += N + 1;
  a.xver = ip;
  ip += N;
  a.kcount = ip;
  ip += N;
  a.lastfg = ip;
  ip += N;
  ip += N;  // reserved
  ip += 2 * T;  // reserved
  a.ctrl = ip;
  ip += 8 * T;
  a.stop = ip++;
  a.status = ip++;
  a.barrier_err = ip++;
  a.w = c->w;
  a.log = dlog;
  a.log_cap = (long long)log_cap;
  a.delays = o->delays_dev;
  a.delay_cols = o->delay_cols;
  a.delay_unit_ns = o->delay_unit_ns;

  PR_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
  // predictor (Algorithm 2, first lines): lam_i^0 = w_i^0 = G(lam_{i-1}^0)
  PR_CUDA(c, cudaMemcpyAsync(lam, p.u0_dev, M * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  long long launches = 0, cg_total = 0;
  for (int i = 1; i <= N; ++i) {
    CgArgs g{};
    g.b = lam + (size_t)(i - 1) * M;
    g.x0 = g.b;
    g.out = c->w + (size_t)(i - 1) * M;
    g.lam = lam + (size_t)i * M;
    g.iters = c->cg_iters_dev + i;
    g.mode = CG_PREDICTOR;
    PR_CUDA(c, cg_solve(c, g));
    ++launches;
  }
  // version 0 of every slice, snapshots xs_i = lam_{i-1}^0
  async_init<<<64, 256, 0, c->stream>>>(a);
  ++launches;
  PR_CUDA(c, cudaMemcpy2DAsync(a.ring, RING * M * sizeof(double), lam + M, M * sizeof(double),
                               M * sizeof(double), N, cudaMemcpyDeviceToDevice, c->stream));
  PR_CUDA(c, cudaMemcpyAsync(a.xs, lam, (size_t)N * M * sizeof(double), cudaMemcpyDeviceToDevice,
                             c->stream));
  std::vector<int> pit(N + 1);
  PR_CUDA(c, cudaMemcpyAsync(pit.data(), c->cg_iters_dev, (N + 1) * sizeof(int),
                             cudaMemcpyDeviceToHost, c->stream));
  PR_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int i = 1; i <= N; ++i) cg_total += pit[i];

  a.timeout_ns = (unsigned long long)(o->timeout_s * 1e9);

  // the persistent kernel: all T*C blocks co-resident (cooperative launch).  In
  // verify mode a stop by the increment rule is followed by a check of the
  // fixed-point residual max_i |lam_i - F(lam_{i-1})| on the latest versions
  // (one batched F into the sync workspace v); unless it is below tol the
  // kernel resumes from its persistent state with every slice's increment
  // forgotten (NaN: "not below"), so each unsettled slice publishes again.
  PR_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
  void* args[] = {&a};
  int flags[3] = {0, 0, 0};
  int rounds = 0;
  double resid = 0.0;
  for (;;) {
    cudaError_t e = cudaLaunchCooperativeKernel((void*)async_kernel, dim3(T * C), dim3(ATHREADS),
                                                args, 0, c->stream);
    if (e != cudaSuccess) {
      if (dlog) cudaFree(dlog);
      return cuda_fail(c, e, "async kernel launch");
    }
    ++launches;
    async_gather<<<dim3(64, std::min(N, 64)), 256, 0, c->stream>>>(a, lam);
    ++launches;
    PR_CUDA(c, cudaMemcpyAsync(flags, a.stop, 3 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PR_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!o->verify || o->quiescence || flags[1] != AST_OK || flags[2]) break;
    PR_CUDA(c, fine_apply(c, lam, c->v, N));
    launches += (p.f_scheme == PR_EXPLICIT_EULER) ? p.f_steps : 1;
    PR_CUDA(c, cudaMemsetAsync(c->delta_dev, 0, sizeof(unsigned long long), c->stream));
    resid_kernel<<<c->num_sms * 4, 256, 0, c->stream>>>(lam + M, c->v, (long long)N * M,
                                                         c->delta_dev);
    ++launches;
    unsigned long long rbits = 0;
    PR_CUDA(c, cudaMemcpyAsync(&rbits, c->delta_dev, sizeof rbits, cudaMemcpyDeviceToHost,
                               c->stream));
    PR_CUDA(c, cudaStreamSynchronize(c->stream));
    memcpy(&resid, &rbits, sizeof resid);
    ++rounds;
    if (resid < p.tol || rounds >= ASYNC_MAX_VERIFY) break;
    PR_CUDA(c, cudaMemsetAsync(a.delta, 0xFF, (size_t)N * sizeof(double), c->stream));
    PR_CUDA(c, cudaMemsetAsync(a.stop, 0, sizeof(int), c->stream));
  }
  PR_CUDA(c, cudaEventRecord(c->ev[2], c->stream));
  PR_CUDA(c, cudaEventRecord(c->ev[3], c->stream));
  unsigned long long nlog = 0, fine_cg = 0;
  PR_CUDA(c, cudaMemcpyAsync(&fine_cg, a.fine_cg, sizeof fine_cg, cudaMemcpyDeviceToHost, c->stream));
  std::vector<int> kc(N);
  std::vector<double> dl(N);
  PR_CUDA(c, cudaMemcpyAsync(&nlog, a.log_count, sizeof nlog, cudaMemcpyDeviceToHost, c->stream));
  PR_CUDA(c, cudaMemcpyAsync(kc.data(), a.kcount, N * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PR_CUDA(c, cudaMemcpyAsync(dl.data(), a.delta, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PR_CUDA(c, cudaStreamSynchronize(c->stream));
  const size_t nkeep = std::min<size_t>((size_t)nlog, log_cap);
  std::vector<pr_event> ev(nkeep);
  if (nkeep) {
    PR_CUDA(c, cudaMemcpy(ev.data(), dlog, nkeep * sizeof(pr_event), cudaMemcpyDeviceToHost));
    if (log_host) memcpy(log_host, ev.data(), nkeep * sizeof(pr_event));
  }
  if (dlog) cudaFree(dlog);
  if (log_len) *log_len = nkeep;
  for (const pr_event& x : ev) cg_total += x.cg_iters;
  float t_all = 0, t_kernel = 0;
  cudaEventElapsedTime(&t_all, c->ev[0], c->ev[3]);
  cudaEventElapsedTime(&t_kernel, c->ev[1], c->ev[2]);
  int kmax = 0;
  double dmax = 0.0;
  for (int i = 0; i < N; ++i) {
    // a slice that published nothing after the last residual check (verify
    // mode) was settled: another update would not move it
    if (std::isnan(dl[i])) dl[i] = 0.0;
    c->last_k[i] = kc[i];
    c->last_delta[i] = dl[i];
    kmax = std::max(kmax, kc[i]);
    dmax = std::max(dmax, dl[i]);
  }
  pr_stats S{};
  S.iterations = kmax;
  S.max_delta = dmax;
  S.events = (long long)nlog;
  long long ups = 0;
  for (int i = 0; i < N; ++i) ups += kc[i];
  S.fine_lups = ups * M * p.f_steps;
  S.cg_iterations = cg_total;
  S.t_total_ms = t_all;
  S.t_fine_ms = 0;
  S.t_coarse_ms = 0;
  S.launches = launches;
  S.fine_cg_iterations = (long long)fine_cg;
  const int status = flags[1], berr = flags[2];
  S.converged = (status == AST_OK && !berr && (rounds == 0 || resid < p.tol)) ? 1 : 0;
  S.verify_rounds = rounds;
  S.residual = rounds ? resid : 0.0;
  if (st) *st = S;
  if (berr || status == AST_BARRIER) return fail(c, PR_ETIMEOUT, "async: a bounded barrier wait expired");
  if (status == AST_TIMEOUT) return fail(c, PR_ETIMEOUT, "async: wall-clock limit reached");
  if (status == AST_LOGFULL) return fail(c, PR_ELOGFULL, "async: event log capacity exceeded");
  (void)t_kernel;
  return PR_OK;
}

}  // namespace pr
