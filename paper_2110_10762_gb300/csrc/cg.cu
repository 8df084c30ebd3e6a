// Coarse propagator G: one backward-Euler step (I + dT A) x = b (§5.1),
// solved by conjugate gradients in FP64 -- textbook (Hestenes-Stiefel) or the
// single-reduction recurrence of Chronopoulos and Gear, which has the same
// iterates -- as one
// cooperative persistent kernel: every block owns a grid-stride share of the
// points, dot products are warp-shuffle + block reductions followed by one
// grid barrier and a fixed-order sum of the block partials (deterministic:
// every block computes bit-identical scalars, so all take the same branch).
//
// The correction of Algorithm 1 (§4.1) follows each sweep solve in one pass
// (cg_correct_kernel, launched right after the solve on its stream): from the
// solution x still in the workspace it forms
//     lam_i^{k+1} = (x + v_i) - w_i^k        (this operation order, no FMA)
// its max-norm increment against lam_i^k (Eq. (22)), and stores w_i = x.  The
// plain and predictor stores run as the solve kernel's epilogue.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cooperative_groups.h>

#include "device.cuh"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace pr {

namespace {

constexpr int CG_THREADS = RED_THREADS;

// Chebyshev-preconditioned CG (option PR_OPT_G_CHEBYSHEV): the preconditioner
// z = p_m(B) r is m steps of Chebyshev iteration on the spectrum bounds [lo, hi]
// of B = I + dT A, run in FP32 (the FP64 pipe is the scarce one on this GPU);
// the CG recurrences, the residual and the stopping test stay FP64.
constexpr int CHEB_MAX = 64;

struct ChebDev {
  int m;                      // 0: plain CG
  int vec;                    // 1: vectorised three-term steps (dim >= 2, kappa = 1, nx % 4 == 0)
  const unsigned char* tmaps; // 3D: tensor maps of y, d0, d1 (128 B each, device), or NULL
  int* err;                   // set to 1 when a bounded wait of the TMA-fed steps expired
  double lo, hi;              // spectrum bounds of B
  float inv_c;                // 1 / centre of [lo, hi]
  float c1[CHEB_MAX], c2[CHEB_MAX];  // step k: d_k = c1[k] d_{k-1} + c2[k] res_k
  float c0, rx, ry, rz;       // constant-kappa B in FP32 (off-diagonals -r)
  StencilVar<float> gv32;     // variable-kappa B in FP32
  double* z;                  // FP64 preconditioned residual
  float *res, *y, *d0, *d1;   // FP32 Chebyshev vectors
};

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
  ChebDev ch;
};

struct GridBarrier {
  __device__ bool sync() const {
    cg::this_grid().sync();
    return true;
  }
};

// B d in FP32 at one point (coarse-operator form: diagonal c0, faces -c_f).
__device__ __forceinline__ float op32(const Geom& g, const ChebDev& ch, bool var,
                                      const float* __restrict__ u, int x, int y, int z,
                                      long long idx) {
  const long long plane = (long long)g.nx * g.ny;
  const float w = x > 0 ? u[idx - 1] : 0.f;
  const float e = x + 1 < g.nx ? u[idx + 1] : 0.f;
  const float s = y > 0 ? u[idx - g.nx] : 0.f;
  const float n = y + 1 < g.ny ? u[idx + g.nx] : 0.f;
  const float bz = z > 0 ? u[idx - plane] : 0.f;
  const float fz = z + 1 < g.nz ? u[idx + plane] : 0.f;
  const float uc = u[idx];
  if (!var) {
    float res = ch.c0 * uc - ch.rx * (w + e);
    if (g.dim > 1) res -= ch.ry * (s + n);
    if (g.dim > 2) res -= ch.rz * (bz + fz);
    return res;
  }
  const long long fx = ((long long)z * g.ny + y) * (g.nx + 1) + x;
  float res = ch.gv32.c0[idx] * uc - ch.gv32.cx[fx] * w - ch.gv32.cx[fx + 1] * e;
  if (g.dim > 1) {
    const long long fy = ((long long)z * (g.ny + 1) + y) * g.nx + x;
    res -= ch.gv32.cy[fy] * s + ch.gv32.cy[fy + g.nx] * n;
  }
  if (g.dim > 2) res -= ch.gv32.cz[idx] * bz + ch.gv32.cz[idx + plane] * fz;
  return res;
}

#ifndef PR_CHEB_ROWS
#define PR_CHEB_ROWS 2
#endif
constexpr int CHEB_U = PR_CHEB_ROWS;  // warp-rows in flight per trip of a Chebyshev step

// One Chebyshev step on this block's rows: res -= B dp, dn = c1 dp + c2 res,
// y += dn; with LAST also z = y (FP64) and the partial r.z.  CHEB_U warp-rows
// per trip: the step is light FP32 work, so it is bound by load latency
// unless several rows are in flight.
template <bool LAST>
__device__ __forceinline__ double cheb_step(const Geom& g, const ChebDev& ch, bool var,
                                            const float* __restrict__ dp, float* __restrict__ dn,
                                            float* __restrict__ res, float* __restrict__ y,
                                            double* __restrict__ z, const double* __restrict__ r,
                                            float c1, float c2, int blk, int nblk) {
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  RowIter it[CHEB_U];
#pragma unroll
  for (int u = 0; u < CHEB_U; ++u) {
    it[u] = RowIter(g, blk, nblk);
    for (int v = 0; v < u; ++v) it[u].advance();
  }
  while (it[0].z < g.nz) {
    long long idx[CHEB_U];
    bool ok[CHEB_U];
    float rs[CHEB_U], dv[CHEB_U], yv[CHEB_U];
#pragma unroll
    for (int u = 0; u < CHEB_U; ++u) {
      const int x = it[u].seg * 32 + lane;
      ok[u] = it[u].z < g.nz && x < g.nx;
      idx[u] = ((long long)it[u].z * g.ny + it[u].y) * g.nx + x;
      rs[u] = 0.f;
      dv[u] = 0.f;
      yv[u] = 0.f;
      if (ok[u]) {
        rs[u] = res[idx[u]] - op32(g, ch, var, dp, x, it[u].y, it[u].z, idx[u]);
        dv[u] = c1 * dp[idx[u]] + c2 * rs[u];
        yv[u] = y[idx[u]] + dv[u];
      }
    }
#pragma unroll
    for (int u = 0; u < CHEB_U; ++u) {
      if (ok[u]) {
        res[idx[u]] = rs[u];
        dn[idx[u]] = dv[u];
        y[idx[u]] = yv[u];
        if (LAST) {
          const double zi = static_cast<double>(yv[u]);
          z[idx[u]] = zi;
          acc = fma(r[idx[u]], zi, acc);
        }
      }
#pragma unroll
      for (int v = 0; v < CHEB_U; ++v) it[u].advance();
    }
  }
  return acc;
}

// Vectorised Chebyshev step in three-term form (constant kappa, dim >= 2,
// nx % 4 == 0).  The d-form above, d_k = c1 d_{k-1} + c2 (f - B y_k),
// y_{k+1} = y_k + d_k with d_{k-1} = y_k - y_{k-1}, is the same recurrence as
//     y_{k+1} = y_k + c1 (y_k - y_{k-1}) + c2 (f - B y_k),      y_0 = 0,
// which reads y_k (with its stencil), y_{k-1} and f and writes y_{k+1}: 16
// bytes per point instead of 24.  y_1 = f / c is never stored: the first step
// (KIND 1) reads f with its stencil and scales every value by 1/c (8 bytes per
// point), the second (KIND 2) forms y_1 from the f it reads anyway (12 bytes),
// the later ones (KIND 0) read the stored y_{k-1};
// the scaling is an uncontracted FP32 product, so the values are those a
// stored y_1 would hold.  A warp owns 128 consecutive x (one float4 per lane)
// of one row of the middle axis (y in 3D) and streams CV_ZC planes of the
// slowest axis (z in 3D, y in 2D), carrying the previous, current and next
// plane of y_k in registers; x-neighbours come from the adjacent lanes by
// shuffles (the warp's two edge values by one scalar load each), middle-axis
// neighbours by float4 loads.  The last step's y_m is z, kept in FP32 (it is
// an FP32 value; the CG passes read it exactly widened to FP64), and the step
// returns this thread's part of r.z.
constexpr int CV_ZC = 8;

__device__ __forceinline__ float4 ldf4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// FP32 <-> FP64 in the vectorised passes: integer-pipe conversions (a conversion
// instruction would issue on the FP64 pipe, at the DFMA rate)
__device__ __forceinline__ double f2d(float v) { return widen_f32(v); }
__device__ __forceinline__ float d2f(double v) { return narrow_f64_rn(v); }

__device__ __forceinline__ float4 mulf4(float4 v, float s) {
  return make_float4(__fmul_rn(v.x, s), __fmul_rn(v.y, s), __fmul_rn(v.z, s), __fmul_rn(v.w, s));
}

template <int DIM, int KIND, bool LAST>
__device__ __forceinline__ double cheb3_step(const Geom& g, const ChebDev& ch,
                                             const float* __restrict__ yk,
                                             const float* __restrict__ ykm,
                                             const float* __restrict__ f, float* __restrict__ yn,
                                             const double* __restrict__ r, float c1, float c2,
                                             int blk, int nblk) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const long long gw = (long long)blk * wpb + (threadIdx.x >> 5);
  const long long nw = (long long)nblk * wpb;
  const int nx = g.nx;
  const int ns = DIM == 3 ? g.nz : g.ny;             // streamed axis
  const int nm = DIM == 3 ? g.ny : 1;                // middle axis
  const long long sst = DIM == 3 ? (long long)g.nx * g.ny : (long long)g.nx;
  const int XC = (nx + 127) >> 7;
  const int SC = (ns + CV_ZC - 1) / CV_ZC;
  const long long items = (long long)XC * nm * SC;
  const float c0 = ch.c0, rx = ch.rx;
  const float rm = DIM == 3 ? ch.ry : 0.f;           // middle-axis coupling
  const float rs = DIM == 3 ? ch.rz : ch.ry;         // streamed-axis coupling
  const float ic = ch.inv_c;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  // KIND 1 streams f itself, scaled to y_1 as it is loaded (its centre f is
  // loaded again, from cache)
  auto sc4 = [&](float4 v) { return KIND == 1 ? mulf4(v, ic) : v; };
  auto sc1 = [&](float v) { return KIND == 1 ? __fmul_rn(v, ic) : v; };
  const float* src = KIND == 1 ? f : yk;
  double acc = 0.0;
  for (long long j = gw; j < items; j += nw) {
    const int xc = (int)(j % XC);
    const long long t = j / XC;
    const int ym = (int)(t % nm);
    const int s0 = (int)(t / nm) * CV_ZC;
    const int s1 = min(s0 + CV_ZC, ns);
    const int x = xc * 128 + 4 * lane;
    const bool act = x < nx;
    const long long row = (DIM == 3 ? (long long)ym * nx : 0) + x;
    float4 prv = zero, cur = zero;
    if (act) {
      if (s0 > 0) prv = sc4(ldf4(src + (s0 - 1) * sst + row));
      cur = sc4(ldf4(src + s0 * sst + row));
    }
    for (int sl = s0; sl < s1; ++sl) {
      const long long o = sl * sst + row;
      float4 nxt = zero, mid = zero, fv = zero, pv = zero;
      float wv = 0.f, ev = 0.f;
      if (act) {
        if (sl + 1 < ns) nxt = sc4(ldf4(src + o + sst));
        if (DIM == 3) {
          if (ym > 0) mid = sc4(ldf4(src + o - nx));
          if (ym + 1 < nm) {
            const float4 q = sc4(ldf4(src + o + nx));
            mid.x += q.x;
            mid.y += q.y;
            mid.z += q.z;
            mid.w += q.w;
          }
        }
        fv = ldf4(f + o);
        if (KIND == 2) pv = mulf4(fv, ic);
        if (KIND == 0) pv = ldf4(ykm + o);
        if (lane == 0 && x > 0) wv = sc1(src[o - 1]);
        if (lane == 31 && x + 4 < nx) ev = sc1(src[o + 4]);
      }
      const float wsh = __shfl_up_sync(FULL, cur.w, 1);
      const float esh = __shfl_down_sync(FULL, cur.x, 1);
      if (lane > 0) wv = wsh;
      if (lane < 31) ev = esh;
      // B y at the four points, then y_{k+1}
      float4 out;
      {
        const float b0 = c0 * cur.x - rx * (wv + cur.y) - rm * mid.x - rs * (prv.x + nxt.x);
        const float b1 = c0 * cur.y - rx * (cur.x + cur.z) - rm * mid.y - rs * (prv.y + nxt.y);
        const float b2 = c0 * cur.z - rx * (cur.y + cur.w) - rm * mid.z - rs * (prv.z + nxt.z);
        const float b3 = c0 * cur.w - rx * (cur.z + ev) - rm * mid.w - rs * (prv.w + nxt.w);
        out.x = cur.x + c1 * (cur.x - pv.x) + c2 * (fv.x - b0);
        out.y = cur.y + c1 * (cur.y - pv.y) + c2 * (fv.y - b1);
        out.z = cur.z + c1 * (cur.z - pv.z) + c2 * (fv.z - b2);
        out.w = cur.w + c1 * (cur.w - pv.w) + c2 * (fv.w - b3);
      }
      if (act) {
        *reinterpret_cast<float4*>(yn + o) = out;
        if (LAST) {
          const double2* rp = reinterpret_cast<const double2*>(r + o);
          const double2 r01 = rp[0], r23 = rp[1];
          acc = fma(r01.x, f2d(out.x), acc);
          acc = fma(r01.y, f2d(out.y), acc);
          acc = fma(r23.x, f2d(out.z), acc);
          acc = fma(r23.y, f2d(out.w), acc);
        }
      }
      prv = cur;
      cur = nxt;
    }
  }
  return acc;
}

// TMA-fed three-term Chebyshev step (3D, constant kappa, nx % 4 == 0): the same
// arithmetic and step kinds as cheb3_step, with y_k (f for the first step)
// staged through shared memory.  The group's
// blocks take 64 x 16 x (13-16) bricks round-robin; for each brick one elected
// thread issues cp.async.bulk.tensor loads of the 72 x 18 planes of y_k (x halo
// 4 wide so that every load starts on a 16-byte boundary; the copy engine fills
// zeros outside the grid, the Dirichlet values) into a CT_ST-stage ring, each
// stage completed on its own mbarrier, two planes ahead of the computed one.
// f and y_{k-1} (no stencil) come by float4 loads issued before the wait.  A
// thread computes 4 consecutive x points.  `gl` counts the loads this block has
// issued in this launch (stage = gl % CT_ST, phase parity = gl / CT_ST); every
// load is waited before the brick ends.  A wait that expires marks the block
// dead (it drains its loads, sets ch.err and skips all later TMA work; the
// solve is reported as failed).
constexpr int CT_TX = 64, CT_TY = 16, CT_ST = 4;
constexpr int CT_PX = CT_TX + 8, CT_PY = CT_TY + 2;
constexpr unsigned CT_BYTES = CT_PX * CT_PY * sizeof(float);
constexpr int CT_STRIDE = (int)(((CT_BYTES + 127) / 128) * 128 / sizeof(float));
constexpr int CT_SMEM = CT_ST * CT_STRIDE * (int)sizeof(float) + CT_ST * 8;

struct ChebTma {
  float* stage;              // CT_ST stages of CT_STRIDE floats (dynamic shared memory)
  unsigned long long* bar;   // CT_ST mbarriers
  unsigned gl;               // loads issued by this block so far (block-uniform)
  bool dead;                 // a bounded wait expired (block-uniform)
};

template <int KIND, bool LAST>
__device__ __forceinline__ double cheb_tma_step(const Geom& g, const ChebDev& ch, const void* map,
                                                const float* __restrict__ ykm,
                                                const float* __restrict__ f,
                                                float* __restrict__ yn,
                                                const double* __restrict__ r, float c1, float c2,
                                                int blk, int nblk, ChebTma& tm) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int TXn = (g.nx + CT_TX - 1) / CT_TX, TYn = (g.ny + CT_TY - 1) / CT_TY;
  const long long plane = (long long)g.nx * g.ny;
  const float c0 = ch.c0, rx = ch.rx, ry = ch.ry, rz = ch.rz;
  const int c = (ty + 1) * CT_PX + 4 + 4 * tx;  // this thread's first point in a stage
  double acc = 0.0;
  // Bricks of TXn x TYn column tiles and TZn z ranges, dealt round-robin in
  // x-fastest order (the blocks of a round stream whole planes together and share
  // their halos in L2).  TZn is chosen so that the bricks fill whole rounds of the
  // group: 16-plane bricks left a partial last round (1024 bricks at 256^3 over 608
  // blocks kept 84% of them busy); 19 z ranges of 13-14 planes make two full rounds.
  const long long cols = (long long)TXn * TYn;
  const long long base = cols * ((g.nz + 15) / 16);
  const long long rounds = (base + nblk - 1) / nblk;
  const int TZn = (int)max(1LL, min((long long)g.nz, rounds * nblk / cols));
  const long long nbricks = cols * TZn;
  for (long long t = blk; t < nbricks && !tm.dead; t += nblk) {
    const long long tile = t % cols;
    const int zt = (int)(t / cols);
    const int x0 = (int)(tile % TXn) * CT_TX, y0 = (int)(tile / TXn) * CT_TY;
    const int z0 = (int)((long long)zt * g.nz / TZn), z1 = (int)((long long)(zt + 1) * g.nz / TZn);
    const int nload = z1 - z0 + 2;   // planes z0-1 .. z1; load index L = plane - (z0 - 1)
    const unsigned gl = tm.gl;
    auto issue = [&](int L) {
      const unsigned q = gl + L;
      float* dst = tm.stage + (q % CT_ST) * CT_STRIDE;
      mbar_arrive_expect_tx(&tm.bar[q % CT_ST], CT_BYTES);
      tma_load_3d(dst, map, x0 - 4, y0 - 1, z0 - 1 + L, &tm.bar[q % CT_ST]);
    };
    if (tid == 0) {
      // the stages were last read through the generic proxy (previous brick or step)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int L = 0; L < CT_ST && L < nload; ++L) issue(L);
    }
    int issued = CT_ST < nload ? CT_ST : nload;
    int waited = 0;
    bool ok = true;
    const int gx = x0 + 4 * tx, gy = y0 + ty;
    const bool inside = gx < g.nx && gy < g.ny;
    for (int zi = z0; zi < z1; ++zi) {
      const int L = zi - z0 + 1;
      const long long o = zi * plane + (long long)gy * g.nx + gx;
      float4 fv = make_float4(0.f, 0.f, 0.f, 0.f), pv = fv;
      if (inside && KIND != 1) {
        fv = ldf4(f + o);
        if (KIND == 2) pv = mulf4(fv, ch.inv_c);
        else if (KIND == 0) pv = ldf4(ykm + o);
      }
      while (ok && waited <= L + 1) {
        const unsigned q = gl + waited;
        ok = mbar_wait(&tm.bar[q % CT_ST], (q / CT_ST) & 1u);
        if (ok) ++waited;
      }
      if (__syncthreads_or(!ok)) {
        tm.dead = true;
        break;
      }
      if (inside) {
        const float* Pm = tm.stage + ((gl + L - 1) % CT_ST) * CT_STRIDE;
        const float* Pc = tm.stage + ((gl + L) % CT_ST) * CT_STRIDE;
        const float* Pp = tm.stage + ((gl + L + 1) % CT_ST) * CT_STRIDE;
        float4 cur = *reinterpret_cast<const float4*>(Pc + c);
        float4 s4 = *reinterpret_cast<const float4*>(Pc + c - CT_PX);
        float4 n4 = *reinterpret_cast<const float4*>(Pc + c + CT_PX);
        float4 b4 = *reinterpret_cast<const float4*>(Pm + c);
        float4 f4 = *reinterpret_cast<const float4*>(Pp + c);
        float w = Pc[c - 1], e = Pc[c + 4];
        if (KIND == 1) {
          // staged f: the centre is f itself, every stencil value is y_1 = f / c
          const float ic = ch.inv_c;
          fv = cur;
          cur = mulf4(cur, ic);
          s4 = mulf4(s4, ic);
          n4 = mulf4(n4, ic);
          b4 = mulf4(b4, ic);
          f4 = mulf4(f4, ic);
          w = __fmul_rn(w, ic);
          e = __fmul_rn(e, ic);
        }
        const float b0 = c0 * cur.x - rx * (w + cur.y) - ry * (s4.x + n4.x) - rz * (b4.x + f4.x);
        const float b1 = c0 * cur.y - rx * (cur.x + cur.z) - ry * (s4.y + n4.y) - rz * (b4.y + f4.y);
        const float b2 = c0 * cur.z - rx * (cur.y + cur.w) - ry * (s4.z + n4.z) - rz * (b4.z + f4.z);
        const float b3 = c0 * cur.w - rx * (cur.z + e) - ry * (s4.w + n4.w) - rz * (b4.w + f4.w);
        float4 out;
        out.x = cur.x + c1 * (cur.x - pv.x) + c2 * (fv.x - b0);
        out.y = cur.y + c1 * (cur.y - pv.y) + c2 * (fv.y - b1);
        out.z = cur.z + c1 * (cur.z - pv.z) + c2 * (fv.z - b2);
        out.w = cur.w + c1 * (cur.w - pv.w) + c2 * (fv.w - b3);
        *reinterpret_cast<float4*>(yn + o) = out;
        if (LAST) {
          const double2* rp = reinterpret_cast<const double2*>(r + o);
          const double2 r01 = rp[0], r23 = rp[1];
          acc = fma(r01.x, f2d(out.x), acc);
          acc = fma(r01.y, f2d(out.y), acc);
          acc = fma(r23.x, f2d(out.z), acc);
          acc = fma(r23.y, f2d(out.w), acc);
        }
      }
      // every thread is done with the stage of load L-1: refill it two planes ahead
      __syncthreads();
      if (L - 1 + CT_ST < nload) {
        if (tid == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue(L - 1 + CT_ST);
        }
        ++issued;
      }
    }
    if (tm.dead) {
      if (tid == 0) {
        atomicExch(ch.err, 1);
        for (int L = waited; L < issued; ++L) {
          const unsigned q = gl + L;
          mbar_wait(&tm.bar[q % CT_ST], (q / CT_ST) & 1u);
        }
      }
      __syncthreads();
    }
    tm.gl = gl + nload;
  }
  return acc;
}

// Steps k = 1..m-1 of the vectorised preconditioner: y_1 = f / c is formed from
// f (never stored), y_k for k >= 2 is in ring slot k % 3, and z = y_m ends in
// slot m % 3.  Tensor maps (3D): slot q at tmaps + 128 q, f at tmaps + 384.
__device__ __forceinline__ float* cheb_slot(const ChebDev& ch, int s) {
  return s == 0 ? ch.y : s == 1 ? ch.d0 : ch.d1;
}

template <int DIM>
__device__ __forceinline__ double cheb3_dispatch(const Geom& g, const ChebDev& ch,
                                                 const double* __restrict__ r, int kk, int blk,
                                                 int nblk, ChebTma& tm) {
  const int sk = kk % 3;
  const float c1 = ch.c1[kk], c2 = ch.c2[kk];
  const float* yk = cheb_slot(ch, sk);
  const float* ykm = cheb_slot(ch, (kk + 2) % 3);
  float* yn = cheb_slot(ch, (kk + 1) % 3);
  const bool last = kk == ch.m - 1;
  const float* f = ch.res;
  if (DIM == 3 && ch.tmaps) {
    if (tm.dead) return 0.0;
    if (kk == 1) {
      const void* map = ch.tmaps + 128 * 3;
      if (last) return cheb_tma_step<1, true>(g, ch, map, ykm, f, yn, r, c1, c2, blk, nblk, tm);
      return cheb_tma_step<1, false>(g, ch, map, ykm, f, yn, r, c1, c2, blk, nblk, tm);
    }
    const void* map = ch.tmaps + 128 * sk;
    if (kk == 2) {
      if (last) return cheb_tma_step<2, true>(g, ch, map, ykm, f, yn, r, c1, c2, blk, nblk, tm);
      return cheb_tma_step<2, false>(g, ch, map, ykm, f, yn, r, c1, c2, blk, nblk, tm);
    }
    if (last) return cheb_tma_step<0, true>(g, ch, map, ykm, f, yn, r, c1, c2, blk, nblk, tm);
    return cheb_tma_step<0, false>(g, ch, map, ykm, f, yn, r, c1, c2, blk, nblk, tm);
  }
  if (kk == 1) {
    if (last) return cheb3_step<DIM, 1, true>(g, ch, yk, ykm, f, yn, r, c1, c2, blk, nblk);
    return cheb3_step<DIM, 1, false>(g, ch, yk, ykm, f, yn, r, c1, c2, blk, nblk);
  }
  if (kk == 2) {
    if (last) return cheb3_step<DIM, 2, true>(g, ch, yk, ykm, f, yn, r, c1, c2, blk, nblk);
    return cheb3_step<DIM, 2, false>(g, ch, yk, ykm, f, yn, r, c1, c2, blk, nblk);
  }
  if (last) return cheb3_step<DIM, 0, true>(g, ch, yk, ykm, f, yn, r, c1, c2, blk, nblk);
  return cheb3_step<DIM, 0, false>(g, ch, yk, ykm, f, yn, r, c1, c2, blk, nblk);
}

// ---- vectorised FP64 passes of the preconditioned CG (constant kappa, dim >= 2,
// nx % 4 == 0).  A warp owns 64 consecutive x (two values per lane) of one row
// of the middle axis (y in 3D) and streams CV_ZC planes of the slowest axis,
// carrying the previous, current and next plane of the stencil operand u
// (FP64, or FP32 widened exactly) in registers; x-neighbours come by shuffles
// (the warp's edge values by one load each), middle-axis neighbours by pair
// loads.  fn(o, cur, w, e, mid, bf) is called for every lane that owns points:
// o = offset of its first point, cur = its two values, w / e = the west
// neighbour of the first and the east neighbour of the second, mid = the sum of
// the middle-axis neighbours (3D), bf = the sum of the streamed-axis neighbours.
__device__ __forceinline__ double2 ld2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ double2 ld2(const float* p) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  return make_double2(f2d(v.x), f2d(v.y));
}
__device__ __forceinline__ double ld1(const double* p) { return *p; }
__device__ __forceinline__ double ld1(const float* p) { return f2d(*p); }

template <int DIM, class T, class Fn>
__device__ __forceinline__ void stream64(const Geom& g, const T* __restrict__ u, int blk,
                                         int nblk, Fn&& fn) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const long long gw = (long long)blk * wpb + (threadIdx.x >> 5);
  const long long nw = (long long)nblk * wpb;
  const int nx = g.nx;
  const int ns = DIM == 3 ? g.nz : g.ny;
  const int nm = DIM == 3 ? g.ny : 1;
  const long long sst = DIM == 3 ? (long long)g.nx * g.ny : (long long)g.nx;
  const int XC = (nx + 63) >> 6;
  const int SC = (ns + CV_ZC - 1) / CV_ZC;
  const long long items = (long long)XC * nm * SC;
  const double2 zero = make_double2(0.0, 0.0);
  for (long long j = gw; j < items; j += nw) {
    const int xc = (int)(j % XC);
    const long long t = j / XC;
    const int ym = (int)(t % nm);
    const int s0 = (int)(t / nm) * CV_ZC;
    const int s1 = min(s0 + CV_ZC, ns);
    const int x = xc * 64 + 2 * lane;
    const bool act = x < nx;
    const long long row = (DIM == 3 ? (long long)ym * nx : 0) + x;
    double2 prv = zero, cur = zero;
    if (act) {
      if (s0 > 0) prv = ld2(u + (s0 - 1) * sst + row);
      cur = ld2(u + s0 * sst + row);
    }
    for (int sl = s0; sl < s1; ++sl) {
      const long long o = sl * sst + row;
      double2 nxt = zero, mid = zero;
      double wv = 0.0, ev = 0.0;
      if (act) {
        if (sl + 1 < ns) nxt = ld2(u + o + sst);
        if (DIM == 3) {
          if (ym > 0) mid = ld2(u + o - nx);
          if (ym + 1 < nm) {
            const double2 q = ld2(u + o + nx);
            mid.x += q.x;
            mid.y += q.y;
          }
        }
        if (lane == 0 && x > 0) wv = ld1(u + o - 1);
        if (lane == 31 && x + 2 < nx) ev = ld1(u + o + 2);
      }
      const double wsh = __shfl_up_sync(FULL, cur.y, 1);
      const double esh = __shfl_down_sync(FULL, cur.x, 1);
      if (lane > 0) wv = wsh;
      if (lane < 31) ev = esh;
      if (act) fn(o, cur, wv, ev, mid, make_double2(prv.x + nxt.x, prv.y + nxt.y));
      prv = cur;
      cur = nxt;
    }
  }
}

// Scaled coarse operator B' u = (I + dT A) u / R_x at one point (constant kappa):
// c0' u - (w + e) - R_y' (s + n) - R_z' (b + f), with the same operation order as
// op_point.  In 2D the middle-axis sum is absent and the streamed axis is y.
template <int DIM>
__device__ __forceinline__ double bop(const StencilConst& ks, double u, double w, double e,
                                      double mid, double bf) {
  double r = fma(ks.c0, u, -(w + e));
  if (DIM == 3) {
    r = fma(-ks.ry, mid, r);
    r = fma(-ks.rz, bf, r);
  } else {
    r = fma(-ks.ry, bf, r);
  }
  return r;
}

// Unscaled (I + dT A) u at one point, the operation order of gop_xyz.
template <int DIM>
__device__ __forceinline__ double gop_pt(const StencilConst& k, double u, double w, double e,
                                         double mid, double bf) {
  double r = k.c0 * u - k.rx * (w + e);
  if (DIM == 3) {
    r -= k.ry * mid;
    r -= k.rz * bf;
  } else {
    r -= k.ry * bf;
  }
  return r;
}

// Start of the preconditioned CG on the vectorised path: r = b - B x0 and
// f = FP32(r); returns the partial r.r and b.b.  x is read from x0 by the first
// solution update (pcg_xr_vec), and y_1 = f / c is formed by the first step.
template <int DIM>
__device__ __forceinline__ void pcg_setup_vec(const CgDev& a, double& rr, double& bb, int blk,
                                              int nblk) {
  const CgWork& ws = a.ws;
  const ChebDev& ch = a.ch;
  const StencilConst k = a.k;
  double srr = 0.0, sbb = 0.0;
  stream64<DIM>(a.g, a.x0, blk, nblk,
                [&](long long o, double2 c, double w, double e, double2 mid, double2 bf) {
                  const double2 b = *reinterpret_cast<const double2*>(a.b + o);
                  const double r0 = b.x - gop_pt<DIM>(k, c.x, w, c.y, mid.x, bf.x);
                  const double r1 = b.y - gop_pt<DIM>(k, c.y, c.x, e, mid.y, bf.y);
                  *reinterpret_cast<double2*>(ws.r + o) = make_double2(r0, r1);
                  const float f0 = d2f(r0), f1 = d2f(r1);
                  *reinterpret_cast<float2*>(ch.res + o) = make_float2(f0, f1);
                  srr = fma(r0, r0, fma(r1, r1, srr));
                  sbb = fma(b.x, b.x, fma(b.y, b.y, sbb));
                });
  rr = srr;
  bb = sbb;
}

// Direction update fused with the operator on the vectorised path:
//   p = z + beta p,   q = B' z + beta q   (= B' p, the operator being linear),
// one pass over z (FP32, with its stencil), p and q; returns the partial p.q.
// On the first iteration p = z and q = B' z.
template <int DIM>
__device__ __forceinline__ double pcg_pq_vec(const CgDev& a, const float* __restrict__ z,
                                             const StencilConst& ks, double beta, bool first,
                                             int blk, int nblk) {
  const CgWork& ws = a.ws;
  double acc = 0.0;
  stream64<DIM>(a.g, z, blk, nblk,
                [&](long long o, double2 c, double w, double e, double2 mid, double2 bf) {
                  const double q0 = bop<DIM>(ks, c.x, w, c.y, mid.x, bf.x);
                  const double q1 = bop<DIM>(ks, c.y, c.x, e, mid.y, bf.y);
                  double2 pn = c, qn = make_double2(q0, q1);
                  if (!first) {
                    const double2 po = *reinterpret_cast<const double2*>(ws.p + o);
                    const double2 qo = *reinterpret_cast<const double2*>(ws.q + o);
                    pn = make_double2(fma(beta, po.x, c.x), fma(beta, po.y, c.y));
                    qn = make_double2(fma(beta, qo.x, q0), fma(beta, qo.y, q1));
                  }
                  *reinterpret_cast<double2*>(ws.p + o) = pn;
                  *reinterpret_cast<double2*>(ws.q + o) = qn;
                  acc = fma(pn.x, qn.x, fma(pn.y, qn.y, acc));
                });
  return acc;
}

// x = xs + (alpha sc) p, r -= alpha q, f = FP32(r) on the vectorised path (xs is x0
// on the first iteration, the workspace x after it), two points per thread and two
// pairs in flight per trip; returns the partial r.r.
__device__ __forceinline__ double pcg_xr_vec(const CgDev& a, double alpha, double ax,
                                             const double* __restrict__ xs, int blk, int nblk) {
  const CgWork& ws = a.ws;
  const ChebDev& ch = a.ch;
  const long long P = a.g.M / 2;  // pairs (M is even on this path)
  const long long t0 = blk * (long long)blockDim.x + threadIdx.x;
  const long long nt = (long long)nblk * blockDim.x;
  double s0 = 0.0, s1 = 0.0;
  auto one = [&](long long i, double& acc) {
    const double2 x = reinterpret_cast<const double2*>(xs)[i];
    const double2 p = reinterpret_cast<const double2*>(ws.p)[i];
    const double2 r = reinterpret_cast<const double2*>(ws.r)[i];
    const double2 q = reinterpret_cast<const double2*>(ws.q)[i];
    const double r0 = fma(-alpha, q.x, r.x), r1 = fma(-alpha, q.y, r.y);
    reinterpret_cast<double2*>(ws.x)[i] = make_double2(fma(ax, p.x, x.x), fma(ax, p.y, x.y));
    reinterpret_cast<double2*>(ws.r)[i] = make_double2(r0, r1);
    const float f0 = d2f(r0), f1 = d2f(r1);
    reinterpret_cast<float2*>(ch.res)[i] = make_float2(f0, f1);
    acc = fma(r0, r0, fma(r1, r1, acc));
  };
  long long i = t0;
  for (; i + nt < P; i += 2 * nt) {
    one(i, s0);
    one(i + nt, s1);
  }
  if (i < P) one(i, s0);
  return s0 + s1;
}

// Preconditioned CG (Hestenes-Stiefel with z = p_m(B) r), same start, stopping
// rule and return value as cg_core.  Per iteration: q = B p and p.q (reduction);
// x, r and r.r, which also starts the preconditioner res = r, d_0 = res / c,
// y = d_0 (reduction); m - 1 Chebyshev steps
//   res -= B d_{k-1},  d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / e) res,  y += d_k
// (one grid barrier each; the last one writes z = y and reduces r.z); then
// p = z + beta p.  The vectorised path uses the three-term steps above and fuses
// q = B' z + beta q into the direction update; its x lives in x0 until the
// first solution update.
__device__ int pcg_core(const CgDev& a, int nblk, int blk) {
  const Geom& g = a.g;
  const ChebDev& ch = a.ch;
  const CgWork& ws = a.ws;
  const bool var = a.var != 0;
  const long long M = g.M;
  const long long t0 = blk * (long long)blockDim.x + threadIdx.x;
  const long long nt = (long long)nblk * blockDim.x;
  // TMA-fed 3D steps read, through the async proxy, vectors that this kernel
  // wrote through the generic proxy before a grid barrier: every thread fences
  // its global writes toward the async proxy before each barrier
  struct PcgBarrier {
    bool tma;
    __device__ void sync() const {
      if (tma) asm volatile("fence.proxy.async.global;" ::: "memory");
      cg::this_grid().sync();
    }
  };
  const PcgBarrier bar{ch.tmaps != nullptr};
  // TMA-fed 3D steps: stage ring and mbarriers in dynamic shared memory
  extern __shared__ __align__(128) unsigned char cheb_smem[];
  ChebTma tm{nullptr, nullptr, 0u, false};
  if (ch.tmaps) {
    tm.stage = reinterpret_cast<float*>(cheb_smem);
    tm.bar = reinterpret_cast<unsigned long long*>(cheb_smem + CT_ST * CT_STRIDE * sizeof(float));
    if (threadIdx.x == 0) {
      for (int q = 0; q < CT_ST; ++q) mbar_init(&tm.bar[q], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      // the tensor maps were written to global memory before the launch
      for (int q = 0; q < 4; ++q)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(ch.tmaps + 128 * q)
                     : "memory");
    }
    __syncthreads();
  }
  int parity = 0;
  auto part = [&]() { return ws.part + (size_t)parity * 3 * nblk; };
  double s_rr = 0.0, s_bb = 0.0;
  if (ch.vec) {
    if (g.dim == 3)
      pcg_setup_vec<3>(a, s_rr, s_bb, blk, nblk);
    else
      pcg_setup_vec<2>(a, s_rr, s_bb, blk, nblk);
  } else {
    for_each_point(g, blk, nblk, [&](int x, int y, int z, long long i) {
      const double bi = a.b[i];
      const double ri = bi - gop_xyz(g, a.k, var, a.gv, a.x0, x, y, z, i);
      ws.x[i] = a.x0[i];
      ws.r[i] = ri;
      const float rf = static_cast<float>(ri);
      const float d = rf * ch.inv_c;
      ch.res[i] = rf;
      ch.d0[i] = d;
      ch.y[i] = d;
      s_rr += ri * ri;
      s_bb += bi * bi;
    });
  }
  {
    const double v[2] = {s_rr, s_bb};
    block_sum<2>(v, part(), blk);
  }
  bar.sync();
  const int maxit = a.maxit;
  const double rtol = a.rtol;
  const StencilConst& k = a.k;
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
  const double thresh = o8[2];
  if (o8[3] != 0.0) return 0;
  const bool scaled = !var;
  const StencilConst ks = scaled ? StencilConst{o8[4], 1.0, o8[5], o8[6]} : k;
  const double sc = scaled ? o8[7] : 1.0;
  int it = 0;
  double rz = 0.0, beta = 0.0;
  while (true) {
    // ---- z = p_m(B) r: steps k = 1..m-1 (res, d_0, y set by the previous pass)
    for (int kk = 1; kk < ch.m; ++kk) {
      const float c1 = ch.c1[kk], c2 = ch.c2[kk];
      const float* dp = (kk & 1) ? ch.d0 : ch.d1;
      float* dn = (kk & 1) ? ch.d1 : ch.d0;
      const bool last = kk == ch.m - 1;
      double s_rz = 0.0;
      if (ch.vec)
        s_rz = g.dim == 3 ? cheb3_dispatch<3>(g, ch, ws.r, kk, blk, nblk, tm)
                          : cheb3_dispatch<2>(g, ch, ws.r, kk, blk, nblk, tm);
      else if (last)
        s_rz = cheb_step<true>(g, ch, var, dp, dn, ch.res, ch.y, ch.z, ws.r, c1, c2, blk, nblk);
      else
        cheb_step<false>(g, ch, var, dp, dn, ch.res, ch.y, ch.z, ws.r, c1, c2, blk, nblk);
      if (last) {
        const double v[1] = {s_rz};
        block_sum<1>(v, part(), blk);
      }
      bar.sync();
      if (last) {
        double o2[2];
        group_sum<1, 2>(part(), nblk, o2, [&](double* r) { r[1] = it == 0 ? 0.0 : r[0] / rz; });
        parity ^= 1;
        beta = o2[1];
        rz = o2[0];
      }
    }
    if (ch.vec) {
      // ---- p = z + beta p and q = B' z + beta q in one pass, p.q (z = y_m is the
      // FP32 ring slot m % 3)
      const float* zf = cheb_slot(ch, ch.m % 3);
      const double v[1] = {g.dim == 3 ? pcg_pq_vec<3>(a, zf, ks, beta, it == 0, blk, nblk)
                                      : pcg_pq_vec<2>(a, zf, ks, beta, it == 0, blk, nblk)};
      block_sum<1>(v, part(), blk);
    } else {
      // ---- p = z + beta p (p = z on the first iteration)
      for (long long i = t0; i < M; i += nt) ws.p[i] = it == 0 ? ch.z[i] : fma(beta, ws.p[i], ch.z[i]);
      bar.sync();
      // ---- q = B p, p.q
      const double v[1] = {cg_matvec_dot(g, ks, var, scaled, a.gv, ws.p, ws.q, blk, nblk)};
      block_sum<1>(v, part(), blk);
    }
    bar.sync();
    double o2[2];
    group_sum<1, 2>(part(), nblk, o2, [&](double* r) { r[1] = rz / r[0]; });
    parity ^= 1;
    const double alpha = o2[1];
    // ---- x, r, r.r; start the next preconditioner application
    double s0 = 0.0;
    if (ch.vec) {
      s0 = pcg_xr_vec(a, alpha, alpha * sc, it == 0 ? a.x0 : ws.x, blk, nblk);
    } else {
      for (long long i = t0; i < M; i += nt) {
        const double ri = fma(-alpha, ws.q[i], ws.r[i]);
        ws.x[i] = fma(alpha * sc, ws.p[i], ws.x[i]);
        ws.r[i] = ri;
        s0 = fma(ri, ri, s0);
        const float rf = static_cast<float>(ri);
        const float d = rf * ch.inv_c;
        ch.res[i] = rf;
        ch.d0[i] = d;
        ch.y[i] = d;
      }
    }
    {
      const double v[1] = {s0};
      block_sum<1>(v, part(), blk);
    }
    bar.sync();
    ++it;
    group_sum<1, 2>(part(), nblk, o2, [&](double* r) {
      r[1] = (sqrt(r[0]) <= thresh || r[0] == 0.0 || it >= maxit) ? 1.0 : 0.0;
    });
    parity ^= 1;
    if (o2[1] != 0.0) {
      // a block whose TMA wait expired set the error word before the last barrier
      if (ch.tmaps && *reinterpret_cast<volatile int*>(ch.err) != 0) return -1;
      return it;
    }
  }
}

// MINB = blocks per SM the register budget must allow.  The CG vectors of a
// grid up to about 2 M points stay in L2 and 2 blocks/SM are best (fewer
// partials and barrier arrivals); beyond that the phases stream from HBM and
// are latency-bound, so a 4-blocks/SM instance (<= 64 registers) keeps twice
// as many loads in flight (measured 707 -> ~550 us per iteration at 256^3).
// ALG: CG_TEXTBOOK, CG_SINGLE (single-reduction recurrence) or CG_CHEB
// (Chebyshev-preconditioned).
enum { CG_TEXTBOOK = 0, CG_SINGLE = 1, CG_CHEB = 2 };

// Epilogue of a coarse solve, the solution x in hand: the plain or predictor
// stores, or the fused correction of Algorithm 1 with its increment.
__device__ __forceinline__ void cg_epilogue(const CgDev& a, const double* __restrict__ x) {
  const long long M = a.g.M;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
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
    if ((M & 1) == 0) {
      // two points per thread (every array is 16-byte aligned when M is even)
      for (long long i = t0; i < M / 2; i += nt) {
        const double2 xi = reinterpret_cast<const double2*>(x)[i];
        const double2 wo = reinterpret_cast<const double2*>(a.out)[i];
        const double2 vi = reinterpret_cast<const double2*>(a.v)[i];
        const double2 lo = reinterpret_cast<const double2*>(a.lam)[i];
        const double l0 = __dsub_rn(__dadd_rn(xi.x, vi.x), wo.x);
        const double l1 = __dsub_rn(__dadd_rn(xi.y, vi.y), wo.y);
        const unsigned long long d0 = abs_bits(__dsub_rn(l0, lo.x));
        const unsigned long long d1 = abs_bits(__dsub_rn(l1, lo.y));
        dmax = d0 > dmax ? d0 : dmax;
        dmax = d1 > dmax ? d1 : dmax;
        reinterpret_cast<double2*>(a.lam)[i] = make_double2(l0, l1);
        reinterpret_cast<double2*>(a.out)[i] = xi;
      }
    } else {
      for (long long i = t0; i < M; i += nt) {
        const double xi = x[i];
        const double wo = a.out[i];
        const double ln = __dsub_rn(__dadd_rn(xi, a.v[i]), wo);
        const unsigned long long d = abs_bits(__dsub_rn(ln, a.lam[i]));
        dmax = d > dmax ? d : dmax;
        a.lam[i] = ln;
        a.out[i] = xi;
      }
    }
    dmax = warp_max_u64(dmax);
    if ((threadIdx.x & 31) == 0 && dmax) atomicMax(a.delta, dmax);
  }
}

template <int MINB, int ALG>
__global__ void __launch_bounds__(CG_THREADS, MINB) cg_kernel(CgDev a) {
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (a.mode == CG_CORRECT && t0 == 0) *a.delta = 0ull;   // the correction kernel follows
  int it;
  if constexpr (ALG == CG_CHEB) {
    it = pcg_core(a, gridDim.x, blockIdx.x);
    // vectorised path: x is x0 until the first solution update
    if (a.mode != CG_CORRECT) cg_epilogue(a, a.ch.vec && it <= 0 ? a.x0 : a.ws.x);
  } else {
    if constexpr (ALG == CG_SINGLE)
      it = cg1_core(a.g, a.k, a.var != 0, a.gv, a.b, a.x0, a.rtol, a.maxit, a.ws, GridBarrier{},
                    gridDim.x, blockIdx.x);
    else
      it = cg_core(a.g, a.k, a.var != 0, a.gv, a.b, a.x0, a.rtol, a.maxit, a.ws, GridBarrier{},
                   gridDim.x, blockIdx.x);
    if (a.mode != CG_CORRECT) cg_epilogue(a, a.ws.x);
  }
  if (t0 == 0) *a.iters = it;
}

// The fused correction of Algorithm 1 after a coarse solve, as a kernel of its own
// on the solve's stream: inside the cooperative solve kernel, whose registers the
// iteration's passes size, the pass ran measurably slower (spilled state).  The
// solve's iteration count tells where its solution is (x0 when the vectorised
// preconditioned CG stopped before its first update).
__global__ void __launch_bounds__(256) cg_correct_kernel(CgDev a) {
  const int it = *a.iters;
  cg_epilogue(a, a.ch.vec && it <= 0 ? a.x0 : a.ws.x);
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
#ifndef PR_CG_BIG_MINB
#define PR_CG_BIG_MINB 4
#endif
constexpr int CG_BIG = PR_CG_BIG_MINB;  // blocks per SM of the instance for grids beyond L2

template <int MINB, int ALG = CG_TEXTBOOK>
int cg_blocks_of(int num_sms, size_t dsmem = 0) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_kernel<MINB, ALG>, CG_THREADS,
                                                    dsmem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (per_sm > MINB) per_sm = MINB;
  return per_sm * num_sms;
}

template <int ALG>
int cg_blocks_any(int num_sms) {
  return std::max(cg_blocks_of<2, ALG>(num_sms), cg_blocks_of<CG_BIG, ALG>(num_sms));
}

}  // namespace

int cg_max_blocks(int num_sms) {
  return std::max(cg_blocks_any<CG_TEXTBOOK>(num_sms),
                  std::max(cg_blocks_any<CG_SINGLE>(num_sms), cg_blocks_any<CG_CHEB>(num_sms)));
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
  a.ws = {c->cg_x, c->cg_r, c->cg_p, c->cg_q, c->cg_part, c->cg_w};
  a.rtol = c->prob.g_rtol;
  a.maxit = c->prob.g_maxit;
  if (c->opt_g_cheb >= 2 && c->cheb_z) {
    ChebDev& ch = a.ch;
    ch.m = c->opt_g_cheb;
    ch.vec = (c->g.dim >= 2 && !c->var_kappa && c->g.nx % 4 == 0) ? 1 : 0;
    ch.tmaps = (ch.vec && c->g.dim == 3) ? static_cast<const unsigned char*>(c->cheb_tmaps) : nullptr;
    ch.err = c->cheb_err;
    ch.lo = c->g_lo;
    ch.hi = c->g_hi;
    // Chebyshev recurrence coefficients on [lo, hi] (centre cc, half width ee)
    const double cc = 0.5 * (c->g_hi + c->g_lo), ee = 0.5 * (c->g_hi - c->g_lo);
    const double sigma = cc / ee;
    double rho = 1.0 / sigma;
    ch.inv_c = static_cast<float>(1.0 / cc);
    for (int k = 1; k < ch.m; ++k) {
      const double rho_n = 1.0 / (2.0 * sigma - rho);
      ch.c1[k] = static_cast<float>(rho_n * rho);
      ch.c2[k] = static_cast<float>(2.0 * rho_n / ee);
      rho = rho_n;
    }
    ch.c0 = static_cast<float>(c->gst.c0);
    ch.rx = static_cast<float>(c->gst.rx);
    ch.ry = static_cast<float>(c->gst.ry);
    ch.rz = static_cast<float>(c->gst.rz);
    ch.gv32 = c->gvar32;
    ch.z = c->cheb_z;
    ch.res = c->cheb_f32;
    ch.y = ch.res + c->g.M;
    ch.d0 = ch.y + c->g.M;
    ch.d1 = ch.d0 + c->g.M;
  }
  const bool big = c->g.M > CG_L2_POINTS;
  // recurrence: preconditioned, or single-reduction when asked for (PR_OPT_G_CG =
  // 2), textbook otherwise: measured per iteration at 128^2 .. 1448^2, the
  // single-reduction recurrence (one barrier and one reduction fewer, one vector
  // update more) was faster only at 256^2 (12.0 against 13.0 us) and slower from
  // 512^2 up (15.9 / 15.4, 30.2 / 29.8, 56.9 / 47.9 us): the FP64 pipe and the
  // extra vector traffic outweigh the barrier it saves
  const int alg = a.ch.m >= 2 ? CG_CHEB : c->opt_g_cg == 2 ? CG_SINGLE : CG_TEXTBOOK;
  int cap = 0;
  void* fn = nullptr;
  const size_t dsmem = (alg == CG_CHEB && a.ch.tmaps) ? (size_t)CT_SMEM : 0;
  if (alg == CG_CHEB) {
    cap = big ? cg_blocks_of<CG_BIG, CG_CHEB>(c->num_sms, dsmem)
              : cg_blocks_of<2, CG_CHEB>(c->num_sms, dsmem);
    fn = big ? (void*)cg_kernel<CG_BIG, CG_CHEB> : (void*)cg_kernel<2, CG_CHEB>;
  } else if (alg == CG_SINGLE) {
    cap = big ? cg_blocks_of<CG_BIG, CG_SINGLE>(c->num_sms) : cg_blocks_of<2, CG_SINGLE>(c->num_sms);
    fn = big ? (void*)cg_kernel<CG_BIG, CG_SINGLE> : (void*)cg_kernel<2, CG_SINGLE>;
  } else {
    cap = big ? cg_blocks_of<CG_BIG>(c->num_sms) : cg_blocks_of<2>(c->num_sms);
    fn = big ? (void*)cg_kernel<CG_BIG, CG_TEXTBOOK> : (void*)cg_kernel<2, CG_TEXTBOOK>;
  }
  // a caller-chosen blocks-per-SM cap leaves room for concurrent kernels
  if (c->opt_cg_bps > 0 && c->opt_cg_bps * c->num_sms < cap) cap = c->opt_cg_bps * c->num_sms;
  long long want = (c->g.M + CG_THREADS * 4 - 1) / (CG_THREADS * 4);
  int blocks = (int)(want < cap ? want : cap);
  if (blocks > c->cg_blocks) blocks = c->cg_blocks;  // partials are sized for cg_blocks
  if (blocks < 1) blocks = 1;
  void* args[] = {&a};
  if (a.mode == CG_CORRECT) {
    const cudaError_t e =
        cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(CG_THREADS), args, dsmem, c->stream);
    if (e != cudaSuccess) return e;
    cg_correct_kernel<<<c->num_sms * 8, 256, 0, c->stream>>>(a);
    return cudaGetLastError();
  }
  return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(CG_THREADS), args, dsmem, c->stream);
}

int cg_solve_launches(int mode) { return mode == CG_CORRECT ? 2 : 1; }

namespace {

__device__ __forceinline__ void atomic_max_pos(unsigned long long* a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_pos(unsigned long long* a, double v) {
  atomicMin(a, (unsigned long long)__double_as_longlong(v));
}

// out[0] = min face kappa, out[1] = max face kappa, out[2] = max diagonal of
// I + dT A (bits of positive doubles, which order like the values); the face
// arrays hold dT kappa_f / h^2.
__global__ void bounds_kernel(Geom g, StencilVar<double> gv, double dT,
                              unsigned long long* out) {
  const long long nfx = (long long)(g.nx + 1) * g.ny * g.nz;
  const long long nfy = g.dim > 1 ? (long long)g.nx * (g.ny + 1) * g.nz : 0;
  const long long nfz = g.dim > 2 ? (long long)g.nx * g.ny * (g.nz + 1) : 0;
  double kmin = 1e300, kmax = 0.0, dmax = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nfx + nfy + nfz + g.M;
       t += (long long)gridDim.x * blockDim.x) {
    double kf = -1.0;
    if (t < nfx) kf = gv.cx[t] * g.hx * g.hx / dT;
    else if (t < nfx + nfy) kf = gv.cy[t - nfx] * g.hy * g.hy / dT;
    else if (t < nfx + nfy + nfz) kf = gv.cz[t - nfx - nfy] * g.hz * g.hz / dT;
    else dmax = fmax(dmax, gv.c0[t - nfx - nfy - nfz]);
    if (kf >= 0.0) {
      kmin = fmin(kmin, kf);
      kmax = fmax(kmax, kf);
    }
  }
  atomic_min_pos(out, kmin);
  atomic_max_pos(out + 1, kmax);
  atomic_max_pos(out + 2, dmax);
}

__global__ void to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = static_cast<float>(a[i]);
}

}  // namespace

// Spectrum bounds [lo, hi] of I + dT A (the Chebyshev preconditioner's
// interval): exact for constant kappa (extreme discrete sine modes); for
// variable kappa lo = 1 + dT kmin lambda_min(A_1) and hi = min(Gershgorin,
// 1 + dT kmax lambda_max(A_1)) with kmin/kmax over the faces.
cudaError_t coarse_bounds(pr_ctx* c) {
  const Geom& g = c->g;
  const int n[3] = {g.nx, g.ny, g.nz};
  const double h[3] = {g.hx, g.hy, g.hz};
  double lo1 = 0.0, hi1 = 0.0;
  for (int ax = 0; ax < g.dim; ++ax) {
    const double s1 = sin(M_PI * h[ax] / 2.0), sn = sin(n[ax] * M_PI * h[ax] / 2.0);
    lo1 += 4.0 / (h[ax] * h[ax]) * s1 * s1;
    hi1 += 4.0 / (h[ax] * h[ax]) * sn * sn;
  }
  const double dT = c->dT;
  if (!c->var_kappa) {
    c->g_lo = 1.0 + dT * lo1;
    c->g_hi = 1.0 + dT * hi1;
    return cudaSuccess;
  }
  const double big = 1e300;
  unsigned long long init[3] = {0ull, 0ull, 0ull};
  memcpy(&init[0], &big, sizeof big);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(c->cg_part);  // scratch
  cudaError_t e = cudaMemcpyAsync(d, init, sizeof init, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return e;
  bounds_kernel<<<c->num_sms * 4, 256, 0, c->stream>>>(g, c->gvar, dT, d);
  unsigned long long res[3];
  e = cudaMemcpyAsync(res, d, sizeof res, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  double v[3];
  memcpy(v, res, sizeof v);
  const double gersh = 2.0 * v[2] - 1.0;  // 1 + 2 * (diag - 1)
  c->g_lo = 1.0 + dT * v[0] * lo1;
  c->g_hi = std::min(gersh, 1.0 + dT * v[1] * hi1);
  return cudaSuccess;
}

// Workspaces of the Chebyshev-preconditioned coarse CG (z, four FP32 vectors,
// FP32 copies of the variable-kappa arrays); allocated when the option is on.
cudaError_t cheb_alloc(pr_ctx* c) {
  if (c->cheb_z) return cudaSuccess;
  const Geom& g = c->g;
  cudaError_t e = cudaMalloc(&c->cheb_z, g.M * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->cheb_f32, 4 * g.M * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&c->cheb_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->cheb_err, 0, sizeof(int), c->stream);
  // 3D constant kappa with nx % 4 == 0: tensor maps of the three ring vectors
  // (y, d0, d1, stored after the FP32 right-hand side f) and of f itself for the
  // TMA-fed steps; the steps fall back to plain vector loads when encoding is
  // not possible
  if (e == cudaSuccess && g.dim == 3 && !c->var_kappa && g.nx % 4 == 0) {
    unsigned char maps[4 * 128];
    bool ok = true;
    for (int q = 0; q < 4 && ok; ++q)
      ok = encode_f32_3d_map(maps + 128 * q, c->cheb_f32 + (size_t)((q + 1) % 4) * g.M, g.nx, g.ny,
                             g.nz, CT_PX, CT_PY);
    if (ok && cudaMalloc(&c->cheb_tmaps, sizeof maps) == cudaSuccess) {
      e = cudaMemcpyAsync(c->cheb_tmaps, maps, sizeof maps, cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    } else {
      cudaGetLastError();  // optional path: no error left behind
    }
  }
  if (e == cudaSuccess && c->var_kappa) {
    const long long nfx = (long long)(g.nx + 1) * g.ny * g.nz;
    const long long nfy = g.dim > 1 ? (long long)g.nx * (g.ny + 1) * g.nz : 0;
    const long long nfz = g.dim > 2 ? (long long)g.nx * g.ny * (g.nz + 1) : 0;
    const long long total = g.M + nfx + nfy + nfz;
    e = cudaMalloc(&c->gcoef32, total * sizeof(float));
    if (e == cudaSuccess) {
      to_f32_kernel<<<c->num_sms * 8, 256, 0, c->stream>>>(c->gcoef, c->gcoef32, total);
      e = cudaGetLastError();
      float* q0 = c->gcoef32;
      float* qx = q0 + g.M;
      float* qy = qx + nfx;
      float* qz = qy + nfy;
      c->gvar32 = {q0, qx, nfy ? qy : nullptr, nfz ? qz : nullptr};
    }
  }
  if (e != cudaSuccess) cheb_free(c);  // the solver uses the option only when cheb_z is set
  return e;
}

void cheb_free(pr_ctx* c) {
  if (c->cheb_z) cudaFree(c->cheb_z);
  if (c->cheb_f32) cudaFree(c->cheb_f32);
  if (c->cheb_tmaps) cudaFree(c->cheb_tmaps);
  if (c->cheb_err) cudaFree(c->cheb_err);
  c->cheb_tmaps = nullptr;
  c->cheb_err = nullptr;
  if (c->gcoef32) cudaFree(c->gcoef32);
  c->cheb_z = nullptr;
  c->cheb_f32 = nullptr;
  c->gcoef32 = nullptr;
  c->gvar32 = {};
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
