// Device building blocks shared by the cooperative CG kernel, the
// asynchronous persistent kernel and the adjoint kernels: pointwise stencils,
// fixed-order reductions, a bounded team barrier, and the CG iteration
// written once for any group of co-resident blocks.
#pragma once

#include "common.cuh"
#include "convert.cuh"

namespace pr {

// ----------------------------------------------------------------- stencils
// Warp-row iterator of a group of `nblk` blocks (this one is `blk`): warp w of
// the group visits items w, w + nw, w + 2 nw, ... of the (z, y, x-segment)
// enumeration, each item 32 consecutive x of one row.  The start and the
// stride are split into (segment, y, z) once; each step then advances with
// carries instead of 64-bit divisions (an emulated multi-instruction sequence
// per division, which dominates the integer work of a light pass).
struct RowIter {
  int seg, y, z;     // current item
  int dseg, dy, dz;  // the stride nw split the same way
  int xseg, ny;
  RowIter() = default;
  __device__ __forceinline__ RowIter(const Geom& g, int blk, int nblk) {
    const int wpb = blockDim.x >> 5;
    const long long gw = (long long)blk * wpb + (threadIdx.x >> 5);
    const long long nw = (long long)nblk * wpb;
    xseg = (g.nx + 31) >> 5;
    ny = g.ny;
    const long long row = gw / xseg, drow = nw / xseg;
    seg = (int)(gw - row * xseg);
    y = (int)(row % g.ny);
    z = (int)(row / g.ny);
    dseg = (int)(nw - drow * xseg);
    dy = (int)(drow % g.ny);
    dz = (int)(drow / g.ny);
  }
  __device__ __forceinline__ void advance() {
    seg += dseg;
    y += dy;
    z += dz;
    if (seg >= xseg) {
      seg -= xseg;
      ++y;
    }
    if (y >= ny) {
      y -= ny;
      ++z;
    }
  }
};

// Visit every grid point with a group of `nblk` blocks (this one is `blk`):
// each warp takes 32 consecutive x of one (y, z) row, so the row's coordinates
// are derived once per 32 points (RowIter).
// f(x, y, z, idx) is called for every interior point exactly once.
template <class Fn>
__device__ __forceinline__ void for_each_point(const Geom& g, int blk, int nblk, Fn&& f) {
  const int lane = threadIdx.x & 31;
  for (RowIter r(g, blk, nblk); r.z < g.nz; r.advance()) {
    const int x = r.seg * 32 + lane;
    if (x >= g.nx) continue;
    f(x, r.y, r.z, ((long long)r.z * g.ny + r.y) * g.nx + x);
  }
}

// Pointwise explicit-Euler step u' = c0 u + sum_faces c_f u_q at point (x, y, z) = idx.
template <typename T, typename Tin>
__device__ __forceinline__ T fstep_xyz(const Geom& g, T c0, T rx, T ry, T rz, bool var,
                                       const StencilVar<T>& cv, const Tin* __restrict__ u, int x,
                                       int y, int z, long long idx) {
  const long long plane = (long long)g.nx * g.ny;
  const T w = x > 0 ? T(u[idx - 1]) : T(0);
  const T e = x + 1 < g.nx ? T(u[idx + 1]) : T(0);
  const T s = y > 0 ? T(u[idx - g.nx]) : T(0);
  const T n = y + 1 < g.ny ? T(u[idx + g.nx]) : T(0);
  const T b = z > 0 ? T(u[idx - plane]) : T(0);
  const T f = z + 1 < g.nz ? T(u[idx + plane]) : T(0);
  const T uc = T(u[idx]);
  if (!var) {
    T res = c0 * uc + rx * (w + e);
    if (g.dim > 1) res += ry * (s + n);
    if (g.dim > 2) res += rz * (b + f);
    return res;
  }
  const long long fx = ((long long)z * g.ny + y) * (g.nx + 1) + x;
  T res = cv.c0[idx] * uc + cv.cx[fx] * w + cv.cx[fx + 1] * e;
  if (g.dim > 1) {
    const long long fy = ((long long)z * (g.ny + 1) + y) * g.nx + x;
    res += cv.cy[fy] * s + cv.cy[fy + g.nx] * n;
  }
  if (g.dim > 2) res += cv.cz[idx] * b + cv.cz[idx + plane] * f;
  return res;
}

// (I + dT A) u at point (x, y, z) = idx; constant coefficients c0 = 1 + 2 sum R_a and
// off-diagonals -R_a, or the variable-kappa arrays (diagonal c0, faces positive).
__device__ __forceinline__ double gop_xyz(const Geom& g, const StencilConst& k, bool var,
                                          const StencilVar<double>& gv,
                                          const double* __restrict__ u, int x, int y, int z,
                                          long long idx) {
  const long long plane = (long long)g.nx * g.ny;
  const double w = x > 0 ? u[idx - 1] : 0.0;
  const double e = x + 1 < g.nx ? u[idx + 1] : 0.0;
  const double s = y > 0 ? u[idx - g.nx] : 0.0;
  const double n = y + 1 < g.ny ? u[idx + g.nx] : 0.0;
  const double bz = z > 0 ? u[idx - plane] : 0.0;
  const double fz = z + 1 < g.nz ? u[idx + plane] : 0.0;
  const double uc = u[idx];
  if (!var) {
    double res = k.c0 * uc - k.rx * (w + e);
    if (g.dim > 1) res -= k.ry * (s + n);
    if (g.dim > 2) res -= k.rz * (bz + fz);
    return res;
  }
  const long long fx = ((long long)z * g.ny + y) * (g.nx + 1) + x;
  double res = gv.c0[idx] * uc - gv.cx[fx] * w - gv.cx[fx + 1] * e;
  if (g.dim > 1) {
    const long long fy = ((long long)z * (g.ny + 1) + y) * g.nx + x;
    res -= gv.cy[fy] * s + gv.cy[fy + g.nx] * n;
  }
  if (g.dim > 2) res -= gv.cz[idx] * bz + gv.cz[idx + plane] * fz;
  return res;
}

// --------------------------------------------------------------- reductions
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of NV (<= 3) values into part[3*blk + j] (fixed order).  Each value
// costs 5 FP64 adds per thread in the warp tree, so callers reduce only what
// they need (FP64 is the scarce pipe on this GPU).
template <int NV>
__device__ __forceinline__ void block_sum(const double (&v)[NV], double* part, int blk) {
  __shared__ double sh[3][32];  // up to 32 warps per block
  const int wid = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const double s = warp_sum(v[j]);
    if (lane == 0) sh[j][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = 0.0;
      for (int i = 0; i < (int)(blockDim.x / 32); ++i) s += sh[j][i];
      part[3 * blk + j] = s;
    }
  }
  __syncthreads();
}

// Sum of nblk block partials in a fixed order; identical result in every block.
// `derive` runs in thread 0 on the sums (slots 0..NV-1) and may fill slots
// NV..7 with scalars computed from them: a division or square root then costs
// one thread per block instead of every thread (FP64 division and square root
// are multi-instruction sequences on the FP64 pipe, the scarce one here).
template <int NV, int NO, class Fn>
__device__ __forceinline__ void group_sum(const double* part, int nblk, double (&o)[NO], Fn&& derive) {
  __shared__ double res[8];
  if (threadIdx.x < 32) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = 0.0;
      for (int i = threadIdx.x; i < nblk; i += 32) s += __ldcg(part + 3 * i + j);
      s = warp_sum(s);
      if (threadIdx.x == 0) res[j] = s;
    }
    if (threadIdx.x == 0) derive(res);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NO; ++j) o[j] = res[j];
  __syncthreads();
}

template <int NV>
__device__ __forceinline__ void group_sum(const double* part, int nblk, double (&o)[NV]) {
  group_sum<NV, NV>(part, nblk, o, [](double*) {});
}

__device__ __forceinline__ unsigned long long abs_bits(double d) {
  return (unsigned long long)__double_as_longlong(fabs(d));
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, v, o);
    v = other > v ? other : v;
  }
  return v;
}

// ------------------------------------------------------------ timing, flags
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Barrier over `nblk` co-resident blocks (a cooperative launch guarantees
// co-residency).  Arrival counter that only grows: the n-th barrier completes
// when the 64-bit counter reaches n * nblk, so there is no reset and no
// separate generation word (about 1.2 us per barrier on GB300, against 2-5 us
// for a reset-and-release scheme).  The wait is bounded by `deadline`
// (globaltimer ns): on expiry *err is set to 1 and the function returns false
// in every thread of the block.  Never traps.
struct TeamBarrier {
  unsigned long long* counter;  // zero before the first barrier of the group
  int nblk;
  unsigned long long deadline;
  int* err;

  __device__ bool sync() const {
    __shared__ int timed_out;
    __syncthreads();
    if (threadIdx.x == 0) {
      timed_out = 0;
      if (nblk > 1) {
        __threadfence();
        const unsigned long long old = atomicAdd(counter, 1ull);
        const unsigned long long target = (old / nblk + 1) * nblk;
        unsigned spins = 0;
        while (ld_acquire_u64(counter) < target) {
          if ((++spins & 255u) == 0 && globaltimer() > deadline) {
            atomicExch(err, 1);
            timed_out = 1;
            break;
          }
        }
      } else {
        __threadfence();
      }
    }
    __syncthreads();
    return !timed_out;
  }
};

// --------------------------------------------------------- conjugate gradients
// Textbook CG for (I + dT A) x = b over a group of `nblk` blocks (this block
// is number `blk`), stopping when ||r||_2 <= rtol ||b||_2, r == 0 or after
// maxit iterations.  x0 may alias nothing it writes (x, r, p, q are the
// group's workspace).  Every block computes bit-identical scalars (fixed-order
// reductions), so all blocks take the same branches.  Returns the iteration
// count, or -1 when a barrier timed out.
struct CgWork {
  double* x;
  double* r;
  double* p;
  double* q;     // textbook: q = B p; single-reduction: s = B p (by recurrence)
  double* part;  // 2 parity buffers x 3 values x nblk
  double* w;     // single-reduction CG only: w = B r
};

#ifndef PR_CG_FAST
#define PR_CG_FAST 1
#endif

// Operator of the CG passes at one point.  SCALED (constant kappa): k holds
// {c0/R_x, -, R_y/R_x, R_z/R_x} and the result is (I + dT A) u / R_x, whose x
// pair needs no multiplier (4 FP64 instructions in 2D, 6 in 3D, against 5 and 7).
__device__ __forceinline__ double op_point(const Geom& g, const StencilConst& k, bool var,
                                           bool scaled, const StencilVar<double>& gv,
                                           const double* __restrict__ u, int x, int y, int z,
                                           long long idx) {
  if (var || !scaled) return gop_xyz(g, k, var, gv, u, x, y, z, idx);
  const long long plane = (long long)g.nx * g.ny;
  const double w = x > 0 ? u[idx - 1] : 0.0;
  const double e = x + 1 < g.nx ? u[idx + 1] : 0.0;
  const double uc = u[idx];
  double res = fma(k.c0, uc, -(w + e));
  if (g.dim > 1) {
    const double s = y > 0 ? u[idx - g.nx] : 0.0;
    const double n = y + 1 < g.ny ? u[idx + g.nx] : 0.0;
    res = fma(-k.ry, s + n, res);
  }
  if (g.dim > 2) {
    const double bz = z > 0 ? u[idx - plane] : 0.0;
    const double fz = z + 1 < g.nz ? u[idx + plane] : 0.0;
    res = fma(-k.rz, bz + fz, res);
  }
  return res;
}

// q = B p on this block's rows and the partial dot product p.q.  Two warp-rows
// per trip with p read-only and q write-only (restrict), so the loads of both
// rows are in flight together instead of one row's latency per trip.
__device__ __forceinline__ double cg_matvec_dot(const Geom& g, const StencilConst& k, bool var,
                                                bool scaled, const StencilVar<double>& gv,
                                                const double* __restrict__ p,
                                                double* __restrict__ q, int blk, int nblk) {
  const int lane = threadIdx.x & 31;
  double sa = 0.0, sb = 0.0;
  // items j and j + 1 of this warp's sequence on each trip
  RowIter ra(g, blk, nblk), rb(g, blk, nblk);
  rb.advance();
  while (ra.z < g.nz) {
    const int xa = ra.seg * 32 + lane;
    const int xb = rb.seg * 32 + lane;
    const bool oka = xa < g.nx;
    const bool okb = rb.z < g.nz && xb < g.nx;
    const long long ia = ((long long)ra.z * g.ny + ra.y) * g.nx + xa;
    const long long ib = ((long long)rb.z * g.ny + rb.y) * g.nx + xb;
    double qa = 0.0, qb = 0.0;
    if (oka) qa = op_point(g, k, var, scaled, gv, p, xa, ra.y, ra.z, ia);
    if (okb) qb = op_point(g, k, var, scaled, gv, p, xb, rb.y, rb.z, ib);
    if (oka) {
      q[ia] = qa;
      sa = fma(p[ia], qa, sa);
    }
    if (okb) {
      q[ib] = qb;
      sb = fma(p[ib], qb, sb);
    }
    ra.advance();
    ra.advance();
    rb.advance();
    rb.advance();
  }
  return sa + sb;
}

// x += ax p, r -= ar q over this block's share; returns the partial r.r.
__device__ __forceinline__ double cg_update_xr(double* __restrict__ x, double* __restrict__ r,
                                               const double* __restrict__ p,
                                               const double* __restrict__ q, double ax, double ar,
                                               long long t0, long long nt, long long M) {
  double s0 = 0.0, s1 = 0.0;
  long long i = t0;
  for (; i + nt < M; i += 2 * nt) {
    const long long j = i + nt;
    const double pi = p[i], pj = p[j], qi = q[i], qj = q[j];
    const double ri = fma(-ar, qi, r[i]);
    const double rj = fma(-ar, qj, r[j]);
    x[i] = fma(ax, pi, x[i]);
    x[j] = fma(ax, pj, x[j]);
    r[i] = ri;
    r[j] = rj;
    s0 = fma(ri, ri, s0);
    s1 = fma(rj, rj, s1);
  }
  if (i < M) {
    const double ri = fma(-ar, q[i], r[i]);
    x[i] = fma(ax, p[i], x[i]);
    r[i] = ri;
    s0 = fma(ri, ri, s0);
  }
  return s0 + s1;
}

// p = r + beta p over this block's share.
__device__ __forceinline__ void cg_update_p(double* __restrict__ p, const double* __restrict__ r,
                                            double beta, long long t0, long long nt, long long M) {
  long long i = t0;
  for (; i + nt < M; i += 2 * nt) {
    const long long j = i + nt;
    const double pi = fma(beta, p[i], r[i]);
    const double pj = fma(beta, p[j], r[j]);
    p[i] = pi;
    p[j] = pj;
  }
  if (i < M) p[i] = fma(beta, p[i], r[i]);
}

// w = B r on this block's rows with the partial products r.r and w.r (the two
// inner products of the single-reduction CG), two warp-rows per trip.
__device__ __forceinline__ void cg1_matvec_dots(const Geom& g, const StencilConst& k, bool var,
                                                bool scaled, const StencilVar<double>& gv,
                                                const double* __restrict__ r,
                                                double* __restrict__ w, int blk, int nblk,
                                                double& rr, double& wr) {
  const int lane = threadIdx.x & 31;
  double ga = 0.0, gb = 0.0, da = 0.0, db = 0.0;
  RowIter ra(g, blk, nblk), rb(g, blk, nblk);
  rb.advance();
  while (ra.z < g.nz) {
    const int xa = ra.seg * 32 + lane;
    const int xb = rb.seg * 32 + lane;
    const bool oka = xa < g.nx;
    const bool okb = rb.z < g.nz && xb < g.nx;
    const long long ia = ((long long)ra.z * g.ny + ra.y) * g.nx + xa;
    const long long ib = ((long long)rb.z * g.ny + rb.y) * g.nx + xb;
    double wa = 0.0, wb = 0.0;
    if (oka) wa = op_point(g, k, var, scaled, gv, r, xa, ra.y, ra.z, ia);
    if (okb) wb = op_point(g, k, var, scaled, gv, r, xb, rb.y, rb.z, ib);
    if (oka) {
      const double rv = r[ia];
      w[ia] = wa;
      ga = fma(rv, rv, ga);
      da = fma(wa, rv, da);
    }
    if (okb) {
      const double rv = r[ib];
      w[ib] = wb;
      gb = fma(rv, rv, gb);
      db = fma(wb, rv, db);
    }
    ra.advance();
    ra.advance();
    rb.advance();
    rb.advance();
  }
  rr = ga + gb;
  wr = da + db;
}

// Direction and solution updates of the single-reduction CG over this block's
// share: p = r + beta p, s = w + beta s (s = B p), x += ax p, r -= ar s.  On the
// first iteration (first = true) p = r and s = w without reading p and s.
__device__ __forceinline__ void cg1_update(const CgWork& ws, double beta, double ax, double ar,
                                           bool first, long long t0, long long nt, long long M) {
  double* __restrict__ x = ws.x;
  double* __restrict__ r = ws.r;
  double* __restrict__ p = ws.p;
  double* __restrict__ s = ws.q;
  const double* __restrict__ w = ws.w;
  if (first) {
    for (long long i = t0; i < M; i += nt) {
      const double ri = r[i], wi = w[i];
      p[i] = ri;
      s[i] = wi;
      x[i] = fma(ax, ri, x[i]);
      r[i] = fma(-ar, wi, ri);
    }
    return;
  }
  long long i = t0;
  for (; i + nt < M; i += 2 * nt) {
    const long long j = i + nt;
    const double ri = r[i], rj = r[j];
    const double pi = fma(beta, p[i], ri);
    const double pj = fma(beta, p[j], rj);
    const double si = fma(beta, s[i], w[i]);
    const double sj = fma(beta, s[j], w[j]);
    p[i] = pi;
    p[j] = pj;
    s[i] = si;
    s[j] = sj;
    x[i] = fma(ax, pi, x[i]);
    x[j] = fma(ax, pj, x[j]);
    r[i] = fma(-ar, si, ri);
    r[j] = fma(-ar, sj, rj);
  }
  if (i < M) {
    const double ri = r[i];
    const double pi = fma(beta, p[i], ri);
    const double si = fma(beta, s[i], w[i]);
    p[i] = pi;
    s[i] = si;
    x[i] = fma(ax, pi, x[i]);
    r[i] = fma(-ar, si, ri);
  }
}

// Single-reduction CG (Chronopoulos and Gear) for (I + dT A) x = b over a group
// of `nblk` blocks: the Krylov iterates of textbook CG with both inner products
// of an iteration, r.r and (B r).r, reduced together, so an iteration takes two
// group barriers (after the update of r, whose neighbours the operator reads;
// after the partial sums) instead of three, and one reduction instead of two:
//   p = r + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s;
//   w = B r,  gamma' = r.r,  delta = w.r;
//   beta = gamma' / gamma,  alpha = gamma' / (delta - beta gamma' / alpha).
// Start, stopping rule (||r||_2 <= rtol ||b||_2 on the recursively updated
// residual, r == 0, or maxit) and return value as cg_core.  Needs ws.w.
template <class Barrier>
__device__ int cg1_core(const Geom& g, const StencilConst& k, bool var,
                        const StencilVar<double>& gv, const double* __restrict__ b,
                        const double* __restrict__ x0, double rtol, int maxit, const CgWork& ws,
                        const Barrier& bar, int nblk, int blk) {
  const long long M = g.M;
  const long long t0 = blk * (long long)blockDim.x + threadIdx.x;
  const long long nt = (long long)nblk * blockDim.x;
  int parity = 0;
  auto part = [&]() { return ws.part + (size_t)parity * 3 * nblk; };
  double s_rr = 0.0, s_bb = 0.0;
  for_each_point(g, blk, nblk, [&](int x, int y, int z, long long i) {
    const double bi = b[i];
    const double ri = bi - gop_xyz(g, k, var, gv, x0, x, y, z, i);
    ws.x[i] = x0[i];
    ws.r[i] = ri;
    s_rr += ri * ri;
    s_bb += bi * bi;
  });
  {
    const double v[2] = {s_rr, s_bb};
    block_sum<2>(v, part(), blk);
  }
  if (!bar.sync()) return -1;
  // threshold, stop flag and the operator scaled by 1/R_x (constant kappa):
  // w' = w / R_x, s' = s / R_x, delta' = delta / R_x, alpha' = R_x alpha;
  // r -= alpha' s', x += (alpha' / R_x) p
  double o8[8];
  group_sum<2, 8>(part(), nblk, o8, [&](double* r) {
    r[2] = rtol * sqrt(r[1]);
    r[3] = (sqrt(r[0]) <= r[2] || r[0] == 0.0 || maxit <= 0) ? 1.0 : 0.0;
    r[4] = k.c0 / k.rx;
    r[5] = k.ry / k.rx;
    r[6] = k.rz / k.rx;
    r[7] = 1.0 / k.rx;
  });
  parity ^= 1;
  if (o8[3] != 0.0) return 0;
  double gamma = o8[0];
  const double thresh = o8[2];
  const bool scaled = !var;
  const StencilConst ks = scaled ? StencilConst{o8[4], 1.0, o8[5], o8[6]} : k;
  const double sc = scaled ? o8[7] : 1.0;
  {
    double rr, wr;
    cg1_matvec_dots(g, ks, var, scaled, gv, ws.r, ws.w, blk, nblk, rr, wr);
    const double v[1] = {wr};
    block_sum<1>(v, part(), blk);
  }
  if (!bar.sync()) return -1;
  double o2[2];
  group_sum<1, 2>(part(), nblk, o2, [&](double* r) { r[1] = gamma / r[0]; });
  parity ^= 1;
  double alpha = o2[1], beta = 0.0;
  int it = 0;
  while (true) {
    cg1_update(ws, beta, alpha * sc, alpha, it == 0, t0, nt, M);
    if (!bar.sync()) return -1;
    {
      double rr, wr;
      cg1_matvec_dots(g, ks, var, scaled, gv, ws.r, ws.w, blk, nblk, rr, wr);
      const double v[2] = {rr, wr};
      block_sum<2>(v, part(), blk);
    }
    if (!bar.sync()) return -1;
    ++it;
    double o5[5];
    group_sum<2, 5>(part(), nblk, o5, [&](double* r) {
      const double gn = r[0];
      r[2] = (sqrt(gn) <= thresh || gn == 0.0 || it >= maxit) ? 1.0 : 0.0;
      const double bt = gn / gamma;
      r[3] = bt;
      r[4] = gn / (r[1] - bt * gn / alpha);
    });
    parity ^= 1;
    if (o5[2] != 0.0) return it;
    gamma = o5[0];
    beta = o5[3];
    alpha = o5[4];
  }
}

template <class Barrier>
__device__ int cg_core(const Geom& g, const StencilConst& k, bool var, const StencilVar<double>& gv,
                       const double* __restrict__ b, const double* __restrict__ x0, double rtol,
                       int maxit, const CgWork& ws, const Barrier& bar, int nblk, int blk) {
  const long long M = g.M;
  const long long t0 = blk * (long long)blockDim.x + threadIdx.x;
  const long long nt = (long long)nblk * blockDim.x;
  int parity = 0;
  auto part = [&]() { return ws.part + (size_t)parity * 3 * nblk; };
  double s_rr = 0.0, s_bb = 0.0;
  for_each_point(g, blk, nblk, [&](int x, int y, int z, long long i) {
    const double bi = b[i];
    const double ri = bi - gop_xyz(g, k, var, gv, x0, x, y, z, i);
    ws.x[i] = x0[i];
    ws.r[i] = ri;
    ws.p[i] = ri;
    s_rr += ri * ri;
    s_bb += bi * bi;
  });
  {
    const double v[2] = {s_rr, s_bb};
    block_sum<2>(v, part(), blk);
  }
  if (!bar.sync()) return -1;
  // scalars derived once per block by thread 0: threshold, stop flag and the
  // coefficients of the operator scaled by 1/R_x (constant kappa): q' = q / R_x,
  // alpha' = rr / p.q' = R_x alpha; r -= alpha' q', x += (alpha' / R_x) p
  double o8[8];
  group_sum<2, 8>(part(), nblk, o8, [&](double* r) {
    r[2] = rtol * sqrt(r[1]);
    r[3] = (sqrt(r[0]) <= r[2] || r[0] == 0.0 || maxit <= 0) ? 1.0 : 0.0;
    r[4] = k.c0 / k.rx;
    r[5] = k.ry / k.rx;
    r[6] = k.rz / k.rx;
    r[7] = 1.0 / k.rx;
  });
  parity ^= 1;
  double rr = o8[0];
  const double thresh = o8[2];
  int it = 0;
  bool done = o8[3] != 0.0;
#if PR_CG_FAST
  const bool scaled = !var;
  const StencilConst ks = scaled ? StencilConst{o8[4], 1.0, o8[5], o8[6]} : k;
  const double sc = scaled ? o8[7] : 1.0;
#endif
  while (!done) {
#if PR_CG_FAST
    {
      const double v[1] = {cg_matvec_dot(g, ks, var, scaled, gv, ws.p, ws.q, blk, nblk)};
      block_sum<1>(v, part(), blk);
    }
#else
    // two accumulators per thread break the dependent FMA chain of the dot product
    double s_a = 0.0, s_b = 0.0;
    for_each_point(g, blk, nblk, [&](int x, int y, int z, long long i) {
      const double qi = gop_xyz(g, k, var, gv, ws.p, x, y, z, i);
      ws.q[i] = qi;
      const double t = s_a + ws.p[i] * qi;  // alternate the two accumulators
      s_a = s_b;
      s_b = t;
    });
    {
      const double v[1] = {s_a + s_b};
      block_sum<1>(v, part(), blk);
    }
#endif
    if (!bar.sync()) return -1;
    double o2[2];
    group_sum<1, 2>(part(), nblk, o2, [&](double* r) { r[1] = rr / r[0]; });
    parity ^= 1;
    const double alpha = o2[1];
#if PR_CG_FAST
    {
      const double v[1] = {cg_update_xr(ws.x, ws.r, ws.p, ws.q, alpha * sc, alpha, t0, nt, M)};
      block_sum<1>(v, part(), blk);
    }
#else
    double s_rn[2] = {0.0, 0.0};
    long long i = t0;
    for (; i + nt < M; i += 2 * nt) {
      const long long j = i + nt;
      ws.x[i] += alpha * ws.p[i];
      ws.x[j] += alpha * ws.p[j];
      const double ri = ws.r[i] - alpha * ws.q[i];
      const double rj = ws.r[j] - alpha * ws.q[j];
      ws.r[i] = ri;
      ws.r[j] = rj;
      s_rn[0] += ri * ri;
      s_rn[1] += rj * rj;
    }
    if (i < M) {
      ws.x[i] += alpha * ws.p[i];
      const double ri = ws.r[i] - alpha * ws.q[i];
      ws.r[i] = ri;
      s_rn[0] += ri * ri;
    }
    {
      const double v[1] = {s_rn[0] + s_rn[1]};
      block_sum<1>(v, part(), blk);
    }
#endif
    if (!bar.sync()) return -1;
    ++it;
    double o3[3];
    group_sum<1, 3>(part(), nblk, o3, [&](double* r) {
      r[1] = (sqrt(r[0]) <= thresh || r[0] == 0.0 || it >= maxit) ? 1.0 : 0.0;
      r[2] = r[0] / rr;
    });
    parity ^= 1;
    const double rr_new = o3[0];
    done = o3[1] != 0.0;
    if (!done) {
      const double beta = o3[2];
#if PR_CG_FAST
      cg_update_p(ws.p, ws.r, beta, t0, nt, M);
#else
      for (long long i = t0; i < M; i += nt) ws.p[i] = ws.r[i] + beta * ws.p[i];
#endif
      rr = rr_new;
      if (!bar.sync()) return -1;
    }
  }
  return it;
}

}  // namespace pr
