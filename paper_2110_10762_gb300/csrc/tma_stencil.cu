// FP32 3D constant-kappa explicit step fed by the Tensor Memory Accelerator
// (the HBM-bound middle steps of the mixed form, §3.1 F run in FP32).
//
// A block owns a 64 x 16 column of the grid for 32 z planes and streams z
// (2.5D): one elected thread issues cp.async.bulk.tensor loads of whole planes
// of the tile plus halo (72 x 18 floats: the x halo is 4 wide so that every
// load starts on a 16-byte boundary) into a four-stage shared-memory ring,
// each stage completed by its own mbarrier (transaction bytes).  Loads run two
// planes ahead of the plane being computed.  Outside the grid the copy engine
// fills zeros, which are exactly the Dirichlet boundary values, so the compute
// loop has no boundary branches.  Each thread computes 4 consecutive x points
// (one float4 from shared memory, x neighbours at the ends) and stores them
// with one 16-byte store.
//
// Every mbarrier wait is bounded; on expiry the block records an error word,
// waits (again bounded) for its own loads still in flight, and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tma.cuh"

namespace pr {

namespace {

constexpr int TTX = 64, TTY = 16;          // output tile
constexpr int TZC = 32;                   // z planes per block
constexpr int TST = 4;                    // ring stages
constexpr int TPX = TTX + 8, TPY = TTY + 2;  // staged plane
constexpr int TPLANE = TPX * TPY;            // floats per staged plane
constexpr unsigned TBYTES = TPLANE * sizeof(float);
// stage pitch rounded up to 128 bytes, so that every stage starts 128-byte aligned
constexpr int TSTRIDE = (int)(((TBYTES + 127) / 128) * 128 / sizeof(float));
constexpr int TMA_THREADS = (TTX / 4) * TTY;  // 256

struct TmaArgs {
  int nx, ny, nz, zchunks;
  long long M;
  float c0, rx, ry, rz;
  float* out;
  int* err;
};

// One explicit step at four consecutive x points, written with explicit FMAs in
// a fixed order so that the one-step and two-step kernels round identically:
// u' = c0 u + rx (w + e) + ry (s + n) + rz (b + f).
__device__ __forceinline__ float step1(float c0, float rx, float ry, float rz, float u, float w,
                                       float e, float sn, float bf) {
  return fmaf(rz, bf, fmaf(ry, sn, fmaf(rx, w + e, c0 * u)));
}

__device__ __forceinline__ float4 step4(float c0, float rx, float ry, float rz, float4 cur, float w,
                                        float e, float4 s4, float4 n4, float4 b4, float4 f4) {
  float4 r;
  r.x = step1(c0, rx, ry, rz, cur.x, w, cur.y, s4.x + n4.x, b4.x + f4.x);
  r.y = step1(c0, rx, ry, rz, cur.y, cur.x, cur.z, s4.y + n4.y, b4.y + f4.y);
  r.z = step1(c0, rx, ry, rz, cur.z, cur.y, cur.w, s4.z + n4.z, b4.z + f4.z);
  r.w = step1(c0, rx, ry, rz, cur.w, cur.z, e, s4.w + n4.w, b4.w + f4.w);
  return r;
}

__global__ void __launch_bounds__(TMA_THREADS, 4) step3d_tma(const __grid_constant__ CUtensorMap src,
                                                          TmaArgs a) {
  __shared__ __align__(128) float stage[TST][TSTRIDE];
  __shared__ __align__(8) unsigned long long bar[TST];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int slice = blockIdx.z / a.zchunks;
  const int z0 = (blockIdx.z - slice * a.zchunks) * TZC;
  const int zend = min(z0 + TZC, a.nz);
  const int nload = zend - z0 + 2;  // planes z0-1 .. zend, load index L = plane - (z0-1)
  const int x0 = blockIdx.x * TTX, y0 = blockIdx.y * TTY;
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < TST; ++s) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int L) {
    const int s = L % TST;
    mbar_arrive_expect_tx(&bar[s], TBYTES);
    tma_load_4d(stage[s], &src, x0 - 4, y0 - 1, z0 - 1 + L, slice, &bar[s]);
  };
  if (tid == 0)
    for (int L = 0; L < TST && L < nload; ++L) issue(L);
  int issued = TST < nload ? TST : nload;  // loads issued so far (uniform: only thread 0 issues)
  int waited = 0;                          // loads 0..waited-1 completed
  bool ok = true, aborted = false;
  const float c0 = a.c0, rx = a.rx, ry = a.ry, rz = a.rz;
  const long long plane = (long long)a.nx * a.ny;
  float* out = a.out + (long long)slice * a.M;
  const int gx = x0 + 4 * tx, gy = y0 + ty;
  const bool inside = gx < a.nx && gy < a.ny;
  const int c = (ty + 1) * TPX + 4 + 4 * tx;  // this thread's first point in a stage
  for (int zi = z0; zi < zend; ++zi) {
    const int L = zi - z0 + 1;  // load index of the output plane
    while (ok && waited <= L + 1) {
      ok = mbar_wait(&bar[waited % TST], (waited / TST) & 1);
      if (ok) ++waited;
    }
    if (__syncthreads_or(!ok)) {  // block-uniform decision
      aborted = true;
      break;
    }
    if (inside) {
      const float* Pm = stage[(L - 1) % TST];
      const float* Pc = stage[L % TST];
      const float* Pp = stage[(L + 1) % TST];
      const float4 cur = *reinterpret_cast<const float4*>(Pc + c);
      const float4 s4 = *reinterpret_cast<const float4*>(Pc + c - TPX);
      const float4 n4 = *reinterpret_cast<const float4*>(Pc + c + TPX);
      const float4 b4 = *reinterpret_cast<const float4*>(Pm + c);
      const float4 f4 = *reinterpret_cast<const float4*>(Pp + c);
      const float w = Pc[c - 1], e = Pc[c + 4];
      const float4 r = step4(c0, rx, ry, rz, cur, w, e, s4, n4, b4, f4);
      *reinterpret_cast<float4*>(out + zi * plane + (long long)gy * a.nx + gx) = r;
    }
    // every thread is done with the stage of load L-1: refill it two planes ahead
    __syncthreads();
    if (L - 1 + TST < nload) {
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(L - 1 + TST);
      }
      ++issued;
    }
  }
  if (aborted && tid == 0) {
    atomicExch(a.err, 1);
    // wait (bounded) for this block's own loads still in flight before exiting,
    // so that no copy lands in shared memory after the block has left
    for (int L = waited; L < issued; ++L) mbar_wait(&bar[L % TST], (L / TST) & 1);
  }
}

// ---- two fine steps per pass (temporal blocking).  The block owns the same
// 64 x 16 output column and streams z; input planes come in with a 2-point halo
// (72 x 20 floats, the x halo 4 wide for alignment) through the same kind of
// mbarrier ring.  Per plane j: the first step is computed on the 72 x 18 region
// the second step needs (324 float4 items over 256 threads) into a three-plane
// shared ring S1, with every value outside the grid set to the Dirichlet zero;
// then the second step of plane j - 1 is computed from S1 and stored.  Each
// thread carries the z-neighbours of its own items in registers (the previous
// and current plane of its input column, and of its first-step column), so a
// plane costs one block barrier, and shared memory is read only for in-plane
// neighbours.  Ring reuse: S1 slot (j + 1) % 3 is written while slots j % 3 and
// (j - 1) % 3 are read, and the input stage of plane j is refilled after the
// barrier that ends its last use.  HBM traffic: one read and one write of the
// state per two steps.
constexpr int T2Y = TTY + 4;                    // staged input rows (halo 2)
constexpr unsigned T2BYTES = TPX * T2Y * sizeof(float);
constexpr int T2STRIDE = (int)(((T2BYTES + 127) / 128) * 128 / sizeof(float));
constexpr int S1Y = TTY + 2;                    // first-step rows
constexpr int S1PLANE = TPX * S1Y;              // 72 x 18
constexpr int T2ITEMS = (TPX / 4) * S1Y;        // 324 float4 items of the first step

__global__ void __launch_bounds__(TMA_THREADS, 4) step3d_tma2(const __grid_constant__ CUtensorMap src,
                                                           TmaArgs a) {
  __shared__ __align__(128) float stage[TST][T2STRIDE];
  __shared__ __align__(16) float s1[3][S1PLANE];
  __shared__ __align__(8) unsigned long long bar[TST];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int slice = blockIdx.z / a.zchunks;
  const int z0 = (blockIdx.z - slice * a.zchunks) * TZC;
  const int zend = min(z0 + TZC, a.nz);
  const int nload = zend - z0 + 4;  // input planes z0-2 .. zend+1; load L = plane - (z0-2)
  const int x0 = blockIdx.x * TTX, y0 = blockIdx.y * TTY;
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < TST; ++q) mbar_init(&bar[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int L) {
    const int q = L % TST;
    mbar_arrive_expect_tx(&bar[q], T2BYTES);
    tma_load_4d(stage[q], &src, x0 - 4, y0 - 2, z0 - 2 + L, slice, &bar[q]);
  };
  if (tid == 0)
    for (int L = 0; L < TST && L < nload; ++L) issue(L);
  int issued = TST < nload ? TST : nload;
  int waited = 0;
  bool ok = true, aborted = false;
  auto wait_upto = [&](int L) {  // loads 0..L complete
    while (ok && waited <= L) {
      ok = mbar_wait(&bar[waited % TST], (waited / TST) & 1);
      if (ok) ++waited;
    }
  };
  const float c0 = a.c0, rx = a.rx, ry = a.ry, rz = a.rz;
  const long long plane = (long long)a.nx * a.ny;
  float* out = a.out + (long long)slice * a.M;
  // first-step items of this thread: item i -> row r = i / 18, float4 column q = i % 18
  // (grid x = x0 - 4 + 4 q, y = y0 - 1 + r; stage row r + 1, column 4 q)
  const int nitem = tid + TMA_THREADS < T2ITEMS ? 2 : 1;
  int ir[2], iq[2];
  bool ixy[2];
  float4 in_prev[2], in_cur[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int i = tid + k * TMA_THREADS;
    ir[k] = i / (TPX / 4);
    iq[k] = i % (TPX / 4);
    const int gx1 = x0 - 4 + 4 * iq[k], gy1 = y0 - 1 + ir[k];
    ixy[k] = k < nitem && gx1 >= 0 && gx1 < a.nx && gy1 >= 0 && gy1 < a.ny;
    in_prev[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    in_cur[k] = in_prev[k];
  }
  // second-step point of this thread
  const int gx = x0 + 4 * tx, gy = y0 + ty;
  const bool inside = gx < a.nx && gy < a.ny;
  const int c2 = (ty + 1) * TPX + 4 + 4 * tx;  // its first point in an S1 plane
  float4 s1_prev = make_float4(0.f, 0.f, 0.f, 0.f), s1_cur = s1_prev;
  // prologue: own input columns of planes z0-2 and z0-1
  wait_upto(1);
  if (!__syncthreads_or(!ok)) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (k < nitem) {
        const int o = (ir[k] + 1) * TPX + 4 * iq[k];
        in_prev[k] = *reinterpret_cast<const float4*>(stage[0] + o);
        in_cur[k] = *reinterpret_cast<const float4*>(stage[1] + o);
      }
  } else {
    aborted = true;
  }
  __syncthreads();
  if (!aborted && TST < nload) {   // the stage of load 0 is free: refill it
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(TST);
    }
    ++issued;
  }
  for (int j = z0 - 1; j <= zend && !aborted; ++j) {
    const int Lj = j - z0 + 2;  // load index of input plane j
    wait_upto(Lj + 1);
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    // (b) first step at plane j into S1[(j + 3) % 3]
    {
      const float* Pc = stage[Lj % TST];
      const float* Pn = stage[(Lj + 1) % TST];
      float* S = s1[(j + 3) % 3];
      const bool zin = j >= 0 && j < a.nz;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        // x-neighbours from the adjacent lanes, which hold the adjacent items of the
        // same row (a scalar shared load only at row and warp edges: the stride-4
        // scalar loads conflict in the shared-memory banks)
        const float4 cur = in_cur[k];
        const float wsh = __shfl_up_sync(0xffffffffu, cur.w, 1);
        const float esh = __shfl_down_sync(0xffffffffu, cur.x, 1);
        if (k >= nitem) continue;
        const int o = (ir[k] + 1) * TPX + 4 * iq[k];
        const float4 nx4 = *reinterpret_cast<const float4*>(Pn + o);
        const float4 s4 = *reinterpret_cast<const float4*>(Pc + o - TPX);
        const float4 n4 = *reinterpret_cast<const float4*>(Pc + o + TPX);
        const int lane = tid & 31;
        const float w = iq[k] == 0 ? 0.f : lane > 0 ? wsh : Pc[o - 1];
        const float e = iq[k] == TPX / 4 - 1 ? 0.f : lane < 31 ? esh : Pc[o + 4];
        const float4 b4 = in_prev[k];
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        if (zin && ixy[k]) r = step4(c0, rx, ry, rz, cur, w, e, s4, n4, b4, nx4);
        *reinterpret_cast<float4*>(S + ir[k] * TPX + 4 * iq[k]) = r;
        in_prev[k] = cur;
        in_cur[k] = nx4;
      }
    }
    // (c) S1 plane j complete; the input stage of plane j has had its last use
    __syncthreads();
    if (Lj + TST < nload) {
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(Lj + TST);
      }
      ++issued;
    }
    // (d) second step at plane j - 1 from S1 planes j - 2, j - 1 (registers) and j
    const float4 s1_next = *reinterpret_cast<const float4*>(s1[(j + 3) % 3] + c2);
    const int zo = j - 1;
    const float4 cur = s1_cur;
    const float wsh = __shfl_up_sync(0xffffffffu, cur.w, 1);   // lanes 0-15 and 16-31: two rows
    const float esh = __shfl_down_sync(0xffffffffu, cur.x, 1);
    if (zo >= z0 && zo < zend && inside) {
      const float* Q = s1[(j + 2) % 3];   // plane j - 1
      const float4 s4 = *reinterpret_cast<const float4*>(Q + c2 - TPX);
      const float4 n4 = *reinterpret_cast<const float4*>(Q + c2 + TPX);
      const float w = tx > 0 ? wsh : Q[c2 - 1];
      const float e = tx < 15 ? esh : Q[c2 + 4];
      const float4 r = step4(c0, rx, ry, rz, cur, w, e, s4, n4, s1_prev, s1_next);
      *reinterpret_cast<float4*>(out + zo * plane + (long long)gy * a.nx + gx) = r;
    }
    s1_prev = s1_cur;
    s1_cur = s1_next;
  }
  if (aborted && tid == 0) {
    atomicExch(a.err, 1);
    for (int L = waited; L < issued; ++L) mbar_wait(&bar[L % TST], (L / TST) & 1);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

// Tiled tensor map of a 3D FP32 array (x fastest, then y, then z) with a box of
// box_x x box_y x 1 elements and zero fill outside the array; false when the
// driver entry point is missing or the encoding is rejected (base not 16-byte
// aligned, strides not multiples of 16 bytes, ...).  out receives 128 bytes.
bool encode_f32_3d_map(void* out, float* base, int nx, int ny, int nz, int box_x, int box_y) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUtensorMap m;
  if (fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  memcpy(out, &m, sizeof m);
  return true;
}

#ifndef PR_TMA
#define PR_TMA 1
#endif

// Tensor maps of the two FP32 ping-pong buffers (4D: x, y, z, slice; box of
// one staged plane); false when the path does not apply or encoding fails.
bool tma_prepare(pr_ctx* c) {
  c->tma_ok = false;
  const Geom& g = c->g;
  if (!PR_TMA || g.dim != 3 || g.nx % 4 != 0 || c->var_kappa || c->prob.f_prec != 32 ||
      c->prob.f_scheme != PR_EXPLICIT_EULER || !c->f32a || !c->f32b)
    return false;
  if (g.nx > (1 << 30) || g.ny > (1 << 30) || g.nz > (1 << 30)) return false;
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  static_assert(sizeof(CUtensorMap) == sizeof(c->tma_map[0]), "tensor map size");
  const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz,
                              (cuuint64_t)c->prob.N};
  const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nx * g.ny * 4,
                                 (cuuint64_t)g.M * 4};
  const cuuint32_t box[4] = {TPX, TPY, 1, 1};
  const cuuint32_t box2[4] = {TPX, T2Y, 1, 1};   // two steps per pass: 2-point halo
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  float* bufs[2] = {c->f32a, c->f32b};
  for (int i = 0; i < 2; ++i) {
    CUtensorMap m, m2;
    if (fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, bufs[i], dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
    if (fn(&m2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, bufs[i], dims, strides, box2, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
    memcpy(c->tma_map[i], &m, sizeof m);
    memcpy(c->tma_map2[i], &m2, sizeof m2);
  }
  if (cudaMalloc(&c->tma_err, sizeof(int)) != cudaSuccess ||
      cudaMemsetAsync(c->tma_err, 0, sizeof(int), c->stream) != cudaSuccess) {
    // optional path: fall back to the vector kernel, leaving no error behind
    if (c->tma_err) cudaFree(c->tma_err);
    c->tma_err = nullptr;
    cudaGetLastError();
    return false;
  }
  c->tma_ok = true;
  return true;
}

// One FP32 step from one ping-pong buffer to the other (src must be f32a or f32b).
cudaError_t tma_step(pr_ctx* c, const float* src, float* dst, int count) {
  const Geom& g = c->g;
  const int which = src == c->f32a ? 0 : 1;
  CUtensorMap m;
  memcpy(&m, c->tma_map[which], sizeof m);
  TmaArgs a{};
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.zchunks = (g.nz + TZC - 1) / TZC;
  a.M = g.M;
  a.c0 = static_cast<float>(c->fst.c0);
  a.rx = static_cast<float>(c->fst.rx);
  a.ry = static_cast<float>(c->fst.ry);
  a.rz = static_cast<float>(c->fst.rz);
  a.out = dst;
  a.err = c->tma_err;
  dim3 grd((g.nx + TTX - 1) / TTX, (g.ny + TTY - 1) / TTY, count * a.zchunks);
  step3d_tma<<<grd, TMA_THREADS, 0, c->stream>>>(m, a);
  return cudaGetLastError();
}

// Two FP32 steps from one ping-pong buffer to the other in one pass (temporal
// blocking; src must be f32a or f32b).
cudaError_t tma_step2(pr_ctx* c, const float* src, float* dst, int count) {
  const Geom& g = c->g;
  const int which = src == c->f32a ? 0 : 1;
  CUtensorMap m;
  memcpy(&m, c->tma_map2[which], sizeof m);
  TmaArgs a{};
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.zchunks = (g.nz + TZC - 1) / TZC;
  a.M = g.M;
  a.c0 = static_cast<float>(c->fst.c0);
  a.rx = static_cast<float>(c->fst.rx);
  a.ry = static_cast<float>(c->fst.ry);
  a.rz = static_cast<float>(c->fst.rz);
  a.out = dst;
  a.err = c->tma_err;
  dim3 grd((g.nx + TTX - 1) / TTX, (g.ny + TTY - 1) / TTY, count * a.zchunks);
  step3d_tma2<<<grd, TMA_THREADS, 0, c->stream>>>(m, a);
  return cudaGetLastError();
}

// Error word of the TMA path (1 after a bounded wait expired); resets it.
int tma_take_error(pr_ctx* c) {
  if (!c->tma_err) return 0;
  int v = 0;
  if (cudaMemcpyAsync(&v, c->tma_err, sizeof v, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->tma_err, 0, sizeof v, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return 1;
  return v;
}

}  // namespace pr
