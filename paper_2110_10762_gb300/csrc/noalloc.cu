// Allocation-free coarse solve: one backward-Euler step (I + dT A) x = b with
// kappa = 1, by the same conjugate-gradient iteration as the coarse
// propagator, whose vectors live in a file-scope device array instead of
// memory obtained from cudaMalloc.
//
// Why: some callers must not allocate device memory once they are running --
// code inside a framework's allocator hook or a host callback (where a
// cudaMalloc would re-enter the allocator or is not permitted), code with a
// fixed memory budget checked at start-up, and latency-critical loops that
// cannot afford the implicit device synchronisation of cudaMalloc/cudaFree.
// This entry point needs no context and allocates nothing.
//
// The scratch array is NOT thread- or stream-safe: every call on a device
// uses the same array, so calls whose kernels overlap on the GPU (different
// streams, or host threads sharing a device) race and corrupt each other.
// Serialise them.
#include <cooperative_groups.h>

#include <mutex>

#include "device.cuh"

namespace cg = cooperative_groups;

namespace pr {
namespace {

constexpr long long NOALLOC_MAX_POINTS = 131072;           // M limit (4 vectors: 4 MiB)
constexpr int NOALLOC_THREADS = RED_THREADS;
constexpr int NOALLOC_MAX_BLOCKS = (int)(NOALLOC_MAX_POINTS / (NOALLOC_THREADS * 4));  // 128
constexpr long long NOALLOC_WORDS =
    4 * NOALLOC_MAX_POINTS + 6LL * NOALLOC_MAX_BLOCKS + 32;  // x, r, p, q, partials, count

// Every GPU that loads the library holds this array (about 4.01 MiB) until exit.
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_WORDS];

struct NoallocArgs {
  Geom g;
  StencilConst k;
  const double* b;
  const double* x0;
  double* x;
  double rtol;
  int maxit;
  double* scratch;  // device address of g_noalloc_scratch
};

struct GridBarrierNA {
  __device__ bool sync() const {
    cg::this_grid().sync();
    return true;
  }
};

__global__ void __launch_bounds__(NOALLOC_THREADS) noalloc_cg_kernel(NoallocArgs a) {
  const long long M = a.g.M;
  CgWork ws;
  ws.x = a.scratch;
  ws.r = ws.x + M;
  ws.p = ws.r + M;
  ws.q = ws.p + M;
  ws.part = a.scratch + 4 * NOALLOC_MAX_POINTS;
  double* count = ws.part + 6 * NOALLOC_MAX_BLOCKS;
  // cg_core writes every vector entry and every partial before reading it,
  // so nothing left in the array by an earlier call is ever read.
  const int it = cg_core(a.g, a.k, false, StencilVar<double>{}, a.b, a.x0, a.rtol, a.maxit, ws,
                         GridBarrierNA{}, gridDim.x, blockIdx.x);
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  for (long long i = t0; i < M; i += nt) a.x[i] = ws.x[i];
  if (t0 == 0) *count = (double)it;
}

struct DeviceSetup {
  double* scratch = nullptr;
  int max_blocks = 0;
  unsigned long long ctx_id = 0;  // context the address was resolved in (0: unknown)
  bool ready = false;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[128];

typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

// Identity of the calling thread's current context, or 0 when the driver does
// not report one.  A device's primary context gets a new identity when it is
// recreated (after cudaDeviceReset), and the module holding the array is then
// loaded again, possibly at another address: the set-up below is redone.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    looked_up = true;
  }
  if (!get_current || !get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Once per device (and again if the device's context was recreated), with
// that device current: resolve the array's device address (the host-side
// symbol is only a stand-in and must never be passed to a kernel) and the
// co-resident block limit of the cooperative kernel.
cudaError_t setup_current_device(int dev, DeviceSetup** out) {
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  const unsigned long long ctx_id = current_context_id();
  if (!s.ready || s.ctx_id != ctx_id) {
    s.ready = false;
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, noalloc_cg_kernel, NOALLOC_THREADS, 0);
    if (e != cudaSuccess) return e;
    s.scratch = static_cast<double*>(ptr);
    s.max_blocks = sms * (per_sm > 0 ? per_sm : 1);
    s.ctx_id = ctx_id;
    s.ready = true;
  }
  *out = &s;
  return cudaSuccess;
}

}  // namespace
}  // namespace pr

extern "C" int parareal_coarse_noalloc(int dim, const int* n, double dT, const double* b_dev,
                                       const double* x0_dev, double* x_dev, double rtol,
                                       int maxit, int* iters_host, void* cuda_stream) {
  using namespace pr;
  if (dim < 1 || dim > 3 || !n || !b_dev || !x_dev || !(dT > 0.0) || !(rtol >= 0.0))
    return PR_EINVAL;
  long long M = 1;
  int nn[3] = {1, 1, 1};
  // each axis and the running product are checked before the next multiplication,
  // so no product of large axes can overflow past the limit
  for (int a = 0; a < dim; ++a) {
    if (n[a] < 1 || n[a] > NOALLOC_MAX_POINTS) return PR_EINVAL;
    nn[a] = n[a];
    M *= n[a];
    if (M > NOALLOC_MAX_POINTS) return PR_EINVAL;  // beyond the static scratch: rejected
  }
  if ((((uintptr_t)b_dev | (uintptr_t)x_dev | (uintptr_t)x0_dev) & 15u) != 0) return PR_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PR_ECUDA;
  DeviceSetup* s = nullptr;
  if (setup_current_device(dev, &s) != cudaSuccess) return PR_ECUDA;

  NoallocArgs a{};
  a.g.dim = dim;
  a.g.nx = nn[0];
  a.g.ny = nn[1];
  a.g.nz = nn[2];
  a.g.M = M;
  a.g.hx = 1.0 / (nn[0] + 1);
  a.g.hy = 1.0 / (nn[1] + 1);
  a.g.hz = 1.0 / (nn[2] + 1);
  const double Rx = dT / (a.g.hx * a.g.hx), Ry = dim > 1 ? dT / (a.g.hy * a.g.hy) : 0.0,
               Rz = dim > 2 ? dT / (a.g.hz * a.g.hz) : 0.0;
  a.k = {1.0 + 2.0 * (Rx + Ry + Rz), Rx, Ry, Rz};
  a.b = b_dev;
  a.x0 = x0_dev ? x0_dev : b_dev;
  a.x = x_dev;
  a.rtol = rtol;
  a.maxit = maxit > 0 ? maxit : 20000;
  a.scratch = s->scratch;
  long long want = (M + NOALLOC_THREADS * 4 - 1) / (NOALLOC_THREADS * 4);
  int blocks = (int)(want < s->max_blocks ? want : s->max_blocks);
  if (blocks > NOALLOC_MAX_BLOCKS) blocks = NOALLOC_MAX_BLOCKS;
  if (blocks < 1) blocks = 1;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel((void*)noalloc_cg_kernel, dim3(blocks), dim3(NOALLOC_THREADS),
                                  args, 0, st) != cudaSuccess)
    return PR_ECUDA;
  if (iters_host) {
    double cnt = 0.0;
    const double* count = s->scratch + 4 * NOALLOC_MAX_POINTS + 6 * NOALLOC_MAX_BLOCKS;
    if (cudaMemcpyAsync(&cnt, count, sizeof cnt, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return PR_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PR_ECUDA;
    *iters_host = (int)cnt;
  }
  return PR_OK;
}
