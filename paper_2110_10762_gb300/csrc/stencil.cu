// Explicit-Euler fine propagator F (§3.1 F, §5.1 time stepping), batched over
// time slices: one launch advances every state of the batch by one step
//   u' = u - dt A_kappa u
// written as u' = c0 u + sum_faces c_f u_q (zero Dirichlet: u_q = 0 outside).
//
// Layout: state c of the batch starts at c*M; x fastest.  A warp covers 32
// consecutive x (coalesced rows); each thread walks a short column in y (2D)
// or z (3D, 2.5D streaming) keeping the centre line in registers, so every
// value is loaded from L2/HBM once per step and x/y neighbours come from L1.
//
// Precision: T is the arithmetic type.  Tin/Tout let the first and last step
// of an FP32 fine solve read and write the FP64 states directly (the casts
// of the mixed form are fused into those steps).
#include <cmath>

#include "common.cuh"
#include "convert.cuh"

namespace pr {

namespace {

#ifndef PR_STENCIL_BY
#define PR_STENCIL_BY 8
#endif
#ifndef PR_STENCIL_RY
#define PR_STENCIL_RY 4
#endif
constexpr int BX = 32;
constexpr int BY = PR_STENCIL_BY;
constexpr int RY = PR_STENCIL_RY;  // rows per thread (2D)
constexpr int ZC = 16;             // z planes per thread (3D)

template <typename T, typename S>
__device__ __forceinline__ T ld(const S* p) {
  return static_cast<T>(__ldg(p));
}

// Coefficients of one constant-kappa step.
//   MODE 0 (plain):   u' = c0 u + rx (w + e) + ry (s + n) + rz (b + f)
//   MODE 1 (scaled):  the batch carries v = u / sigma, sigma multiplied by rx
//                     every step, which takes the x multiplier out of the
//                     update:  v' = c0 v + (w + e) + ry (s + n) + rz (b + f)
//                     with c0, ry, rz divided by rx on the host
//                     (one FP64 instruction less per point: 4 in 2D, 6 in 3D)
//   MODE 2 (scaled, back to u): as MODE 1, then times sc = sigma.
// The same products are formed in another order, so the two forms differ by
// rounding only.
template <typename T>
struct StepK {
  T c0, rx, ry, rz, sc;
};

// 1D and 2D.  DIM = 1 ignores y coupling (ny = 1).
template <typename Tin, typename Tout, typename T, bool VAR, int DIM, int MODE>
__global__ void __launch_bounds__(BX* BY) step2d(const Tin* __restrict__ in, Tout* __restrict__ out,
                                                 int nx, int ny, long long M, StepK<T> k,
                                                 StencilVar<T> cv) {
  const int x = blockIdx.x * BX + threadIdx.x;
  const int y0 = (blockIdx.y * BY + threadIdx.y) * RY;
  if (x >= nx || y0 >= ny) return;
  const long long base = (long long)blockIdx.z * M;
  const Tin* u = in + base;
  Tout* o = out + base;
  T s = (DIM > 1 && y0 > 0) ? ld<T>(u + (long long)(y0 - 1) * nx + x) : T(0);
  T cur = ld<T>(u + (long long)y0 * nx + x);
#pragma unroll
  for (int j = 0; j < RY; ++j) {
    const int y = y0 + j;
    if (y >= ny) break;
    const long long p = (long long)y * nx + x;
    const T n = (DIM > 1 && y + 1 < ny) ? ld<T>(u + p + nx) : T(0);
    const T w = x > 0 ? ld<T>(u + p - 1) : T(0);
    const T e = x + 1 < nx ? ld<T>(u + p + 1) : T(0);
    T res;
    if (!VAR && MODE == 0) {
      res = k.c0 * cur + k.rx * (w + e);
      if (DIM > 1) res += k.ry * (s + n);
    } else if (!VAR) {
      res = fma(k.c0, cur, w + e);
      if (DIM > 1) res = fma(k.ry, s + n, res);
      if (MODE == 2) res *= k.sc;
    } else {
      const long long fx = (long long)y * (nx + 1) + x;
      res = ld<T>(cv.c0 + p) * cur;
      res += ld<T>(cv.cx + fx) * w;
      res += ld<T>(cv.cx + fx + 1) * e;
      if (DIM > 1) {
        res += ld<T>(cv.cy + p) * s;
        res += ld<T>(cv.cy + p + nx) * n;
      }
    }
    o[p] = static_cast<Tout>(res);
    s = cur;
    cur = n;
  }
}

template <typename Tin, typename Tout, typename T, bool VAR, int MODE>
__global__ void __launch_bounds__(BX* BY) step3d(const Tin* __restrict__ in, Tout* __restrict__ out,
                                                 int nx, int ny, int nz, int zchunks, long long M,
                                                 StepK<T> k, StencilVar<T> cv) {
  const int x = blockIdx.x * BX + threadIdx.x;
  const int y = blockIdx.y * BY + threadIdx.y;
  const int slice = blockIdx.z / zchunks;
  const int z0 = (blockIdx.z - slice * zchunks) * ZC;
  if (x >= nx || y >= ny || z0 >= nz) return;
  const long long plane = (long long)nx * ny;
  const long long base = (long long)slice * M;
  const Tin* u = in + base;
  Tout* o = out + base;
  const long long yx = (long long)y * nx + x;
  T b = z0 > 0 ? ld<T>(u + (z0 - 1) * plane + yx) : T(0);
  T cur = ld<T>(u + z0 * plane + yx);
#pragma unroll 4
  for (int j = 0; j < ZC; ++j) {
    const int z = z0 + j;
    if (z >= nz) break;
    const long long p = z * plane + yx;
    const T f = z + 1 < nz ? ld<T>(u + p + plane) : T(0);
    const T w = x > 0 ? ld<T>(u + p - 1) : T(0);
    const T e = x + 1 < nx ? ld<T>(u + p + 1) : T(0);
    const T s = y > 0 ? ld<T>(u + p - nx) : T(0);
    const T n = y + 1 < ny ? ld<T>(u + p + nx) : T(0);
    T res;
    if (!VAR && MODE == 0) {
      res = k.c0 * cur + k.rx * (w + e) + k.ry * (s + n) + k.rz * (b + f);
    } else if (!VAR) {
      res = fma(k.rz, b + f, fma(k.ry, s + n, fma(k.c0, cur, w + e)));
      if (MODE == 2) res *= k.sc;
    } else {
      const long long fx = ((long long)z * ny + y) * (nx + 1) + x;
      const long long fy = ((long long)z * (ny + 1) + y) * nx + x;
      res = ld<T>(cv.c0 + p) * cur;
      res += ld<T>(cv.cx + fx) * w;
      res += ld<T>(cv.cx + fx + 1) * e;
      res += ld<T>(cv.cy + fy) * s;
      res += ld<T>(cv.cy + fy + nx) * n;
      res += ld<T>(cv.cz + p) * b;
      res += ld<T>(cv.cz + p + plane) * f;
    }
    o[p] = static_cast<Tout>(res);
    b = cur;
    cur = f;
  }
}

// ---- FP32 3D step with 4 consecutive x points per thread (HBM-bound path of
// the mixed form).  16-byte vector loads/stores (or 2 x 16 B for the FP64 input
// of the first step and output of the last) keep 4x more bytes in flight per
// instruction than the scalar kernel; the x-neighbours of a thread's 4 points
// come from the adjacent lanes of its 16-lane row segment by warp shuffles.
// Needs nx % 4 == 0 (and, for variable kappa, 16-byte aligned face arrays).
constexpr int V4X = 16;  // threads along x (64 points)
constexpr int V4Y = 8;   // rows
constexpr int V4Z = 16;  // z planes per thread

__device__ __forceinline__ float4 load4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
// FP64 <-> FP32 at the ends of the FP32 steps by the integer-pipe conversions
// (a conversion instruction issues on the FP64 pipe at the DFMA rate)
__device__ __forceinline__ float4 load4(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return make_float4(narrow_f64_rn(a.x), narrow_f64_rn(a.y), narrow_f64_rn(b.x), narrow_f64_rn(b.y));
}
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return narrow_f64_rn(v); }
__device__ __forceinline__ void store4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void store4(double* p, float4 v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(widen_f32(v.x), widen_f32(v.y));
  reinterpret_cast<double2*>(p)[1] = make_double2(widen_f32(v.z), widen_f32(v.w));
}
__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }

template <typename Tin, typename Tout, bool VAR>
__global__ void __launch_bounds__(V4X* V4Y) step3d_v4(const Tin* __restrict__ in,
                                                      Tout* __restrict__ out, int nx, int ny,
                                                      int nz, int zchunks, long long M, float c0,
                                                      float rx, float ry, float rz,
                                                      StencilVar<float> cv) {
  const int tx = threadIdx.x;
  const int x4 = (blockIdx.x * V4X + tx) * 4;
  const int y = blockIdx.y * V4Y + threadIdx.y;
  const int slice = blockIdx.z / zchunks;
  const int z0 = (blockIdx.z - slice * zchunks) * V4Z;
  // no early return: every lane takes part in the shuffles
  const bool valid = x4 < nx && y < ny;
  const long long plane = (long long)nx * ny;
  const Tin* u = in + (long long)slice * M;
  Tout* o = out + (long long)slice * M;
  const long long yx = (long long)y * nx + x4;
  float4 b = zero4(), cur = zero4();
  if (valid) {
    if (z0 > 0) b = load4(u + (long long)(z0 - 1) * plane + yx);
    cur = load4(u + (long long)z0 * plane + yx);
  }
  for (int j = 0; j < V4Z; ++j) {
    const int z = z0 + j;
    if (z >= nz) break;  // uniform over the block
    const long long p = (long long)z * plane + yx;
    float4 f = zero4(), s = zero4(), n = zero4();
    if (valid) {
      if (z + 1 < nz) f = load4(u + p + plane);
      if (y > 0) s = load4(u + p - nx);
      if (y + 1 < ny) n = load4(u + p + nx);
    }
    float w = __shfl_up_sync(0xffffffffu, cur.w, 1, V4X);
    float e = __shfl_down_sync(0xffffffffu, cur.x, 1, V4X);
    if (tx == 0) w = (valid && x4 > 0) ? to_f32(__ldg(u + p - 1)) : 0.f;
    if (tx == V4X - 1 || x4 + 4 >= nx) e = (valid && x4 + 4 < nx) ? to_f32(__ldg(u + p + 4)) : 0.f;
    float4 r;
    if (!VAR) {
      r.x = c0 * cur.x + rx * (w + cur.y) + ry * (s.x + n.x) + rz * (b.x + f.x);
      r.y = c0 * cur.y + rx * (cur.x + cur.z) + ry * (s.y + n.y) + rz * (b.y + f.y);
      r.z = c0 * cur.z + rx * (cur.y + cur.w) + ry * (s.z + n.z) + rz * (b.z + f.z);
      r.w = c0 * cur.w + rx * (cur.z + e) + ry * (s.w + n.w) + rz * (b.w + f.w);
    } else {
      r = zero4();
      if (valid) {
        const float4 d = load4(cv.c0 + p);
        const long long fx = ((long long)z * ny + y) * (nx + 1) + x4;
        const float x0 = __ldg(cv.cx + fx), x1 = __ldg(cv.cx + fx + 1), x2 = __ldg(cv.cx + fx + 2),
                    x3 = __ldg(cv.cx + fx + 3), x4f = __ldg(cv.cx + fx + 4);
        const long long fy = ((long long)z * (ny + 1) + y) * nx + x4;
        const float4 ys = load4(cv.cy + fy), yn = load4(cv.cy + fy + nx);
        const float4 zb = load4(cv.cz + p), zf = load4(cv.cz + p + plane);
        r.x = d.x * cur.x + x0 * w + x1 * cur.y + ys.x * s.x + yn.x * n.x + zb.x * b.x + zf.x * f.x;
        r.y = d.y * cur.y + x1 * cur.x + x2 * cur.z + ys.y * s.y + yn.y * n.y + zb.y * b.y + zf.y * f.y;
        r.z = d.z * cur.z + x2 * cur.y + x3 * cur.w + ys.z * s.z + yn.z * n.z + zb.z * b.z + zf.z * f.z;
        r.w = d.w * cur.w + x3 * cur.z + x4f * e + ys.w * s.w + yn.w * n.w + zb.w * b.w + zf.w * f.w;
      }
    }
    if (valid) store4(o + p, r);
    b = cur;
    cur = f;
  }
}

bool v4_path_ok(const pr_ctx* c) {
  const Geom& g = c->g;
  if (g.dim != 3 || g.nx % 4 != 0) return false;
  if (!c->var_kappa) return true;
  // face arrays must start on 16-byte boundaries: (nx+1)*ny*nz and M multiples of 4
  return ((long long)g.ny * g.nz) % 4 == 0;
}

template <typename Tin, typename Tout>
cudaError_t launch_step_v4(const pr_ctx* c, const Tin* in, Tout* out, int count,
                           const StencilVar<float>& cv) {
  const Geom& g = c->g;
  const int zchunks = (g.nz + V4Z - 1) / V4Z;
  dim3 blk(V4X, V4Y);
  dim3 grd((g.nx / 4 + V4X - 1) / V4X, (g.ny + V4Y - 1) / V4Y, count * zchunks);
  const float c0 = static_cast<float>(c->fst.c0), rx = static_cast<float>(c->fst.rx),
              ry = static_cast<float>(c->fst.ry), rz = static_cast<float>(c->fst.rz);
  if (c->var_kappa)
    step3d_v4<Tin, Tout, true><<<grd, blk, 0, c->stream>>>(in, out, g.nx, g.ny, g.nz, zchunks, g.M,
                                                            c0, rx, ry, rz, cv);
  else
    step3d_v4<Tin, Tout, false><<<grd, blk, 0, c->stream>>>(in, out, g.nx, g.ny, g.nz, zchunks, g.M,
                                                             c0, rx, ry, rz, cv);
  return cudaGetLastError();
}

template <typename Tin, typename Tout, typename T, bool VAR, int MODE>
cudaError_t launch_step_mode(const pr_ctx* c, const Tin* in, Tout* out, int count,
                             const StepK<T>& k, const StencilVar<T>& cv) {
  const Geom& g = c->g;
  dim3 blk(BX, BY);
  if (g.dim <= 2) {
    dim3 grd((g.nx + BX - 1) / BX, (g.ny + BY * RY - 1) / (BY * RY), count);
    if (g.dim == 1)
      step2d<Tin, Tout, T, VAR, 1, MODE><<<grd, blk, 0, c->stream>>>(in, out, g.nx, 1, g.M, k, cv);
    else
      step2d<Tin, Tout, T, VAR, 2, MODE><<<grd, blk, 0, c->stream>>>(in, out, g.nx, g.ny, g.M, k, cv);
  } else {
    const int zchunks = (g.nz + ZC - 1) / ZC;
    dim3 grd((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, count * zchunks);
    step3d<Tin, Tout, T, VAR, MODE><<<grd, blk, 0, c->stream>>>(in, out, g.nx, g.ny, g.nz, zchunks,
                                                                g.M, k, cv);
  }
  return cudaGetLastError();
}

// One plain step (either precision, constant or variable kappa).
template <typename Tin, typename Tout, typename T>
cudaError_t launch_step(const pr_ctx* c, const Tin* in, Tout* out, int count,
                        const StencilVar<T>& cv) {
  if constexpr (sizeof(T) == 4) {
    if (v4_path_ok(c)) return launch_step_v4<Tin, Tout>(c, in, out, count, cv);
  }
  const StepK<T> k{static_cast<T>(c->fst.c0), static_cast<T>(c->fst.rx),
                   static_cast<T>(c->fst.ry), static_cast<T>(c->fst.rz), T(1)};
  if (c->var_kappa) return launch_step_mode<Tin, Tout, T, true, 0>(c, in, out, count, k, cv);
  return launch_step_mode<Tin, Tout, T, false, 0>(c, in, out, count, k, cv);
}

// `steps` FP64 constant-kappa steps in the scaled form, ping-ponging between
// `out` and c->tmp so that the last step writes `out`.
cudaError_t scaled_fine64(pr_ctx* c, const double* in, double* out, int count, int steps) {
  const int R = scaled_period(c->fst.rx);
  const double rx = c->fst.rx;
  StepK<double> k{c->fst.c0 / rx, 1.0, c->fst.ry / rx, c->fst.rz / rx, 1.0};
  const double* src = in;
  int since = 0;
  for (int s = 0; s < steps; ++s) {
    double* dst = ((steps - 1 - s) % 2 == 0) ? out : c->tmp;
    ++since;
    cudaError_t e;
    if (s == steps - 1 || since == R) {
      k.sc = std::pow(rx, since);
      e = launch_step_mode<double, double, double, false, 2>(c, src, dst, count, k, c->fvar);
      since = 0;
    } else {
      e = launch_step_mode<double, double, double, false, 1>(c, src, dst, count, k, c->fvar);
    }
    if (e != cudaSuccess) return e;
    src = dst;
  }
  return cudaSuccess;
}

// ---- variable-kappa coefficient construction (one thread per face / node)
__device__ __forceinline__ long long ring_index(const Geom& g, int xr, int yr, int zr) {
  if (g.dim == 1) return xr;
  if (g.dim == 2) return (long long)yr * (g.nx + 2) + xr;
  return ((long long)zr * (g.ny + 2) + yr) * (g.nx + 2) + xr;
}

// Face diffusivity kappa_f = (kappa_p + kappa_q)/2 scaled by s/h^2 for F (s = dt)
// and G (s = dT).  Interior node (x,y,z) has ring coordinates (x+1, y+1, z+1)
// along the axes that exist.
__global__ void faces_kernel(Geom g, const double* __restrict__ kap, double sF, double sG,
                             double* fcx, double* fcy, double* fcz, double* gcx, double* gcy,
                             double* gcz) {
  const long long nfx = (long long)(g.nx + 1) * g.ny * g.nz;
  const long long nfy = g.dim > 1 ? (long long)g.nx * (g.ny + 1) * g.nz : 0;
  const long long nfz = g.dim > 2 ? (long long)g.nx * g.ny * (g.nz + 1) : 0;
  const int oy = g.dim > 1 ? 1 : 0, oz = g.dim > 2 ? 1 : 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nfx + nfy + nfz;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < nfx) {
      const int xf = t % (g.nx + 1);
      const long long line = t / (g.nx + 1);
      const int y = line % g.ny, z = line / g.ny;
      const double kf = 0.5 * (kap[ring_index(g, xf, y + oy, z + oz)] +
                               kap[ring_index(g, xf + 1, y + oy, z + oz)]);
      fcx[t] = sF * kf / (g.hx * g.hx);
      gcx[t] = sG * kf / (g.hx * g.hx);
    } else if (t < nfx + nfy) {
      const long long q = t - nfx;
      const int x = q % g.nx;
      const long long r = q / g.nx;
      const int yf = r % (g.ny + 1), z = r / (g.ny + 1);
      const double kf = 0.5 * (kap[ring_index(g, x + 1, yf, z + oz)] +
                               kap[ring_index(g, x + 1, yf + 1, z + oz)]);
      fcy[q] = sF * kf / (g.hy * g.hy);
      gcy[q] = sG * kf / (g.hy * g.hy);
    } else {
      const long long q = t - nfx - nfy;
      const int x = q % g.nx;
      const long long r = q / g.nx;
      const int y = r % g.ny, zf = r / g.ny;
      const double kf = 0.5 * (kap[ring_index(g, x + 1, y + 1, zf)] +
                               kap[ring_index(g, x + 1, y + 1, zf + 1)]);
      fcz[q] = sF * kf / (g.hz * g.hz);
      gcz[q] = sG * kf / (g.hz * g.hz);
    }
  }
}

__global__ void diag_kernel(Geom g, const double* fcx, const double* fcy, const double* fcz,
                            const double* gcx, const double* gcy, const double* gcz, double* f0,
                            double* g0, double* fs0) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.M;
       p += (long long)gridDim.x * blockDim.x) {
    const int x = p % g.nx;
    const long long r = p / g.nx;
    const int y = r % g.ny, z = r / g.ny;
    const long long fx = ((long long)z * g.ny + y) * (g.nx + 1) + x;
    double sf = fcx[fx] + fcx[fx + 1];
    double sg = gcx[fx] + gcx[fx + 1];
    if (g.dim > 1) {
      const long long fy = ((long long)z * (g.ny + 1) + y) * g.nx + x;
      sf += fcy[fy] + fcy[fy + g.nx];
      sg += gcy[fy] + gcy[fy + g.nx];
    }
    if (g.dim > 2) {
      const long long plane = (long long)g.nx * g.ny;
      sf += fcz[p] + fcz[p + plane];
      sg += gcz[p] + gcz[p + plane];
    }
    f0[p] = 1.0 - sf;
    g0[p] = 1.0 + sg;
    if (fs0) fs0[p] = 1.0 + sf;
  }
}

__global__ void to_float_kernel(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = static_cast<float>(a[i]);
}

// FP64 -> FP32 copy of n4 groups of four values (32 bytes in, 16 out per thread and
// trip, two groups in flight; integer-pipe rounding): the entry of the TMA-fed
// FP32 steps.
__global__ void to_float4_kernel(const double* __restrict__ a, float* __restrict__ b, long long n4) {
  const long long nt = (long long)gridDim.x * blockDim.x;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i + nt < n4; i += 2 * nt) {
    const double2* p = reinterpret_cast<const double2*>(a) + 2 * i;
    const double2* q = reinterpret_cast<const double2*>(a) + 2 * (i + nt);
    const double2 p0 = p[0], p1 = p[1], q0 = q[0], q1 = q[1];
    reinterpret_cast<float4*>(b)[i] = make_float4(narrow_f64_rn(p0.x), narrow_f64_rn(p0.y),
                                                  narrow_f64_rn(p1.x), narrow_f64_rn(p1.y));
    reinterpret_cast<float4*>(b)[i + nt] =
        make_float4(narrow_f64_rn(q0.x), narrow_f64_rn(q0.y), narrow_f64_rn(q1.x),
                    narrow_f64_rn(q1.y));
  }
  if (i < n4) {
    const double2* p = reinterpret_cast<const double2*>(a) + 2 * i;
    const double2 p0 = p[0], p1 = p[1];
    reinterpret_cast<float4*>(b)[i] = make_float4(narrow_f64_rn(p0.x), narrow_f64_rn(p0.y),
                                                  narrow_f64_rn(p1.x), narrow_f64_rn(p1.y));
  }
}

}  // namespace

// Steps between two returns to u in the scaled form: sigma^-1 = rx^-R stays
// below 1e100, so intermediate values stay within 1e100 of the input's
// magnitude (FP64 range: inputs up to 1e200 in magnitude are safe).
int scaled_period(double rx) {
  if (!(rx > 0.0 && rx < 1.0)) return 0;
  const double r = std::floor(100.0 / std::log10(1.0 / rx));
  return r < 1.0 ? 1 : (r > 1e6 ? 1000000 : static_cast<int>(r));
}

cudaError_t build_var_coefficients(pr_ctx* c) {
  const Geom& g = c->g;
  const long long nfx = (long long)(g.nx + 1) * g.ny * g.nz;
  const long long nfy = g.dim > 1 ? (long long)g.nx * (g.ny + 1) * g.nz : 0;
  const long long nfz = g.dim > 2 ? (long long)g.nx * g.ny * (g.nz + 1) : 0;
  const long long total = g.M + nfx + nfy + nfz;
  cudaError_t e;
  if ((e = cudaMalloc(&c->fcoef, total * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->gcoef, total * sizeof(double))) != cudaSuccess) return e;
  double* f0 = c->fcoef;
  double* fx = f0 + g.M;
  double* fy = fx + nfx;
  double* fz = fy + nfy;
  double* g0 = c->gcoef;
  double* gx = g0 + g.M;
  double* gy = gx + nfx;
  double* gz = gy + nfy;
  const int blocks = c->num_sms * 8;
  // trapezoidal F: the F arrays describe the half step (I - dt/2 A), and the
  // system I + dt/2 A shares their faces with its own diagonal fsys0
  const bool cn = c->prob.f_scheme == PR_CRANK_NICOLSON;
  if (cn && (e = cudaMalloc(&c->fsys0, g.M * sizeof(double))) != cudaSuccess) return e;
  faces_kernel<<<blocks, 256, 0, c->stream>>>(g, c->prob.kappa_dev, cn ? 0.5 * c->dt : c->dt, c->dT,
                                              fx, fy, fz, gx, gy, gz);
  diag_kernel<<<blocks, 256, 0, c->stream>>>(g, fx, fy, fz, gx, gy, gz, f0, g0, c->fsys0);
  if (cn) c->fsysvar = {c->fsys0, fx, nfy ? fy : nullptr, nfz ? fz : nullptr};
  c->fvar = {f0, fx, nfy ? fy : nullptr, nfz ? fz : nullptr};
  c->gvar = {g0, gx, nfy ? gy : nullptr, nfz ? gz : nullptr};
  if (c->prob.f_prec == 32) {
    if ((e = cudaMalloc(&c->fcoef32, total * sizeof(float))) != cudaSuccess) return e;
    to_float_kernel<<<blocks, 256, 0, c->stream>>>(c->fcoef, c->fcoef32, total);
    float* q0 = c->fcoef32;
    float* qx = q0 + g.M;
    float* qy = qx + nfx;
    float* qz = qy + nfy;
    c->fvar32 = {q0, qx, nfy ? qy : nullptr, nfz ? qz : nullptr};
  }
  return cudaGetLastError();
}

cudaError_t explicit_step64(pr_ctx* c, const double* in, double* out, int count) {
  if (count <= 0) return cudaSuccess;
  return launch_step<double, double, double>(c, in, out, count, c->fvar);
}

// Kernel launches of one batched F (the dispatch below): one per fine step,
// except the TMA-fed FP32 middle steps, which run two per launch when enabled.
int fine_launch_count(const pr_ctx* c) {
  const pr_problem& p = c->prob;
  if (p.f_scheme != PR_EXPLICIT_EULER) return 1;
  const int steps = p.f_steps;
  if (p.f_prec == 32 && c->tma_ok && steps > 1) {
    // conversion, steps - 1 TMA-fed steps (one or two per launch), the last step
    const int mid = steps - 1;
    return 2 + (c->opt_f_blocking == 2 ? mid / 2 + mid % 2 : mid);
  }
  return steps;
}

cudaError_t explicit_fine(pr_ctx* c, const double* in, double* out, int count, int steps,
                          int prec) {
  if (count <= 0 || steps <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (prec == 64) {
    if (!c->var_kappa && steps > 1 && scaled_period(c->fst.rx) > 0)
      return scaled_fine64(c, in, out, count, steps);
    const double* src = in;
    for (int s = 0; s < steps; ++s) {
      double* dst = ((steps - 1 - s) % 2 == 0) ? out : c->tmp;
      e = launch_step<double, double, double>(c, src, dst, count, c->fvar);
      if (e != cudaSuccess) return e;
      src = dst;
    }
    return e;
  }
  // FP32 steps, FP64 input and output
  if (steps == 1) return launch_step<double, double, float>(c, in, out, count, c->fvar32);
  int s = 1;
  if (c->tma_ok) {
    // TMA path: the input converted to FP32 by a streaming copy (a stencil step that
    // reads FP64 runs into the texture pipe's throughput, 12 against 4.5 ms at 256^3 x
    // 124 slices), then every step but the last TMA-fed
    const long long n4 = (long long)count * c->g.M / 4;   // M % 4 == 0 on this path
    long long blocks = (n4 + 255) / 256;
    if (blocks > c->num_sms * 8) blocks = c->num_sms * 8;
    if (blocks < 1) blocks = 1;
    to_float4_kernel<<<(int)blocks, 256, 0, c->stream>>>(in, c->f32a, n4);
    e = cudaGetLastError();
    s = 0;
  } else {
    e = launch_step<double, float, float>(c, in, c->f32a, count, c->fvar32);
  }
  if (e != cudaSuccess) return e;
  const float* src = c->f32a;
  for (; s < steps - 1;) {
    float* dst = (src == c->f32a) ? c->f32b : c->f32a;
    // TMA path: two middle steps per pass where two remain (temporal blocking)
    const bool two = c->tma_ok && c->opt_f_blocking == 2 && s + 1 < steps - 1;
    e = two ? tma_step2(c, src, dst, count)
        : c->tma_ok ? tma_step(c, src, dst, count)
                    : launch_step<float, float, float>(c, src, dst, count, c->fvar32);
    if (e != cudaSuccess) return e;
    s += two ? 2 : 1;
    src = dst;
  }
  e = launch_step<float, double, float>(c, src, out, count, c->fvar32);
  if (e == cudaSuccess && c->tma_ok && tma_take_error(c)) e = cudaErrorTimeout;
  return e;
}

}  // namespace pr
