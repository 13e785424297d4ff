// Throughput probe of the FP64 fused multiply-add pipe (declared in include/lbm_gb300.h as
// lbm_probe_fp64_fma).  Measurement support with no counterpart in the paper: the FP64 step of
// the method is bound by this pipe on GB300, so its roofline needs the pipe's measured rate.
// Every thread runs kChains independent dependent chains x <- x a + b, enough to keep the pipe
// busy; the result feeds a store that never happens at run time (the sum cannot equal the
// sentinel) but that the compiler cannot remove.
#include "lbm_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__device__ double g_probe_sink;

__global__ void __launch_bounds__(kThreads) dfma_probe_kernel(int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3 * threadIdx.x + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = __fma_rn(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == -1234.5) g_probe_sink = s;  // x stays near b / (1 - a) > 0
}

}  // namespace

lbm_status lbm_probe_fp64_fma(int32_t iters, void* stream, double* gflops, double* ms) {
  if (!gflops || !ms || iters < 1 || iters > (1 << 24)) return LBM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, dfma_probe_kernel, kThreads, 0) !=
          cudaSuccess || per < 1) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  const long long blocks = (long long)sms * per;  // one full wave of resident CTAs
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // one untimed launch (clocks up, code loaded), then the timed one
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
    if (rep == 1) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      dfma_probe_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(iters, 0.9999999, 1e-7);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess || !(t > 0.f)) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  const double fma_count = (double)blocks * kThreads * kChains * (double)iters;
  *ms = t;
  *gflops = 2.0 * fma_count / (t * 1e-3) / 1e9;
  return LBM_OK;
}
