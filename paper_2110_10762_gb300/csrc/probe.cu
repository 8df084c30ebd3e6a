// FP64-pipe throughput probe: a measurement aid for the roofline of the FP64
// kernels (the explicit FP64 fine steps and the coarse CG are bound by the
// FP64 pipe on this GPU, whose FP64 rate no vendor table lists for it).
// Every thread runs eight independent dependency chains of DFMA (x = x a + b)
// or DADD (x = x + b); the grid holds 4 blocks of 256 threads per SM, enough
// warps to cover the pipe latency.  The chains' results are folded into one
// word that is written only when it is not finite, so nothing is optimised
// away and the output costs nothing.
#include <math.h>

#include "common.cuh"
#include "device.cuh"

namespace pr {
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS) fp64_probe_kernel(double* out, long long iters,
                                                                   double a, double b) {
  double x[PROBE_CHAINS];
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) x[j] = 1e-3 * (threadIdx.x + j);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) {
      if (KIND == 0)
        x[j] = fma(x[j], a, b);
      else
        x[j] = x[j] + b;
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) s += x[j];
  if (!isfinite(s)) out[0] = s;
}

// The integer-pipe conversions of the coarse solver applied elementwise, so that
// a test can compare them with the hardware conversions.
__global__ void convert_check_kernel(const float* __restrict__ f_in, double* __restrict__ d_out,
                                     const double* __restrict__ d_in, float* __restrict__ f_out,
                                     long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    d_out[i] = widen_f32(f_in[i]);
    f_out[i] = narrow_f64_rn(d_in[i]);
  }
}

}  // namespace
}  // namespace pr

extern "C" int parareal_probe_convert(const float* f_in_dev, double* d_out_dev,
                                      const double* d_in_dev, float* f_out_dev, long long n,
                                      void* cuda_stream) {
  using namespace pr;
  if (n < 0 || (n > 0 && (!f_in_dev || !d_out_dev || !d_in_dev || !f_out_dev))) return PR_EINVAL;
  if (n == 0) return PR_OK;
  const long long want = (n + 255) / 256;
  const int blocks = (int)(want < 4096 ? want : 4096);
  convert_check_kernel<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>(f_in_dev, d_out_dev, d_in_dev,
                                                                        f_out_dev, n);
  return cudaGetLastError() == cudaSuccess ? PR_OK : PR_ECUDA;
}

extern "C" int parareal_probe_fp64(int kind, long long iters, double* scratch_dev,
                                   double* ops_per_s_host, long long* ops_host,
                                   void* cuda_stream) {
  using namespace pr;
  if ((kind != 0 && kind != 1) || iters < 1 || iters > (1LL << 32) || !scratch_dev ||
      !ops_per_s_host)
    return PR_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PR_ECUDA;
  const int blocks = 4 * sms;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return PR_ECUDA;
  }
  // one untimed launch (clocks ramp, module load), then the timed one
  int status = PR_OK;
  for (int rep = 0; rep < 2 && status == PR_OK; ++rep) {
    if (rep == 1 && cudaEventRecord(e0, st) != cudaSuccess) status = PR_ECUDA;
    if (kind == 0)
      fp64_probe_kernel<0><<<blocks, PROBE_THREADS, 0, st>>>(scratch_dev, iters, 0.9999999, 1e-7);
    else
      fp64_probe_kernel<1><<<blocks, PROBE_THREADS, 0, st>>>(scratch_dev, iters, 0.9999999, 1e-7);
    if (cudaGetLastError() != cudaSuccess) status = PR_ECUDA;
  }
  float ms = 0.f;
  if (status == PR_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                          cudaEventSynchronize(e1) != cudaSuccess ||
                          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    status = PR_ECUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != PR_OK) return status;
  const long long ops = (long long)blocks * PROBE_THREADS * PROBE_CHAINS * iters;
  *ops_per_s_host = ms > 0.f ? ops / (ms * 1e-3) : 0.0;
  if (ops_host) *ops_host = ops;
  return PR_OK;
}
