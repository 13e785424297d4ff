// Allocation-free variant of the mass ledger (declared in include/lbm_gb300.h as
// lbm_mass_noalloc).  The per-block partial sums live in a fixed-size file-scope device array
// instead of memory obtained from an allocator, so a caller that owns the population and flag
// arrays can get the total mass without the library allocating anything.
#include <mutex>

#include "lbm_internal.h"

namespace {

constexpr int kNodesPerBlock = 8192;  // each block reduces one fixed range of nodes
constexpr int kMaxBlocks = 8192;      // at most 8192 * 8192 = 67,108,864 nodes
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: [0, kMaxBlocks) block sums, [kMaxBlocks, 2 kMaxBlocks)
// per-block "bad density seen" flags.  Every slot a call reads was written earlier in the same
// call, so the contents left by a previous call never matter.
static __device__ __align__(256) double g_mass_scratch[2 * kMaxBlocks];

double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

struct Neumaier {
  double s = 0.0, c = 0.0;
  __device__ void add(double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x))
      c += (s - t) + x;
    else
      c += (x - t) + s;
    s = t;
  }
};

__device__ double block_sum(double v) {
  __shared__ double sh[kThreads / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < kThreads / 32 ? sh[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  }
  __syncthreads();
  return v;
}

// Block b sums sum_a f_a over the fluid nodes of [b * kNodesPerBlock, (b + 1) * kNodesPerBlock).
template <typename S>
__global__ void __launch_bounds__(kThreads) noalloc_partial_kernel(int N, double rho_ref,
                                                                   const S* __restrict__ f,
                                                                   const uint8_t* __restrict__ flags,
                                                                   double* __restrict__ scratch) {
  const int b = blockIdx.x;
  const int end = min(N, (b + 1) * kNodesPerBlock);
  const size_t NN = (size_t)N;
  Neumaier acc;
  double bad = 0.0;
  for (int n = b * kNodesPerBlock + threadIdx.x; n < end; n += kThreads) {
    if (flags && (flags[n] & 1)) continue;
    double r = 0.0;
#pragma unroll
    for (int a = 0; a < 9; ++a) r += double(f[a * NN + n]);
    if (sizeof(S) == 4) r += rho_ref;
    if (!(r > 0.0) || !isfinite(r)) bad = 1.0;
    acc.add(r);
  }
  const double t = block_sum(acc.s + acc.c);
  const double anybad = block_sum(bad);
  if (threadIdx.x == 0) {
    scratch[b] = t;
    scratch[kMaxBlocks + b] = anybad > 0.0 ? 1.0 : 0.0;
  }
}

__global__ void __launch_bounds__(kThreads) noalloc_final_kernel(const double* __restrict__ scratch,
                                                                 int nblocks,
                                                                 double* __restrict__ mass_out,
                                                                 int* __restrict__ status_out) {
  Neumaier acc;
  double bad = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += kThreads) {
    acc.add(scratch[k]);
    bad += scratch[kMaxBlocks + k];
  }
  const double t = block_sum(acc.s + acc.c);
  const double anybad = block_sum(bad);
  if (threadIdx.x == 0) {
    *mass_out = t;
    *status_out = anybad > 0.0 ? LBM_EUNSTABLE : LBM_OK;
  }
}

// Device address of the scratch array for the current device, looked up once per device.
lbm_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_mass_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LBM_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_mass_noalloc(const void* f, const uint8_t* flags, int32_t nx, int32_t ny,
                                       int32_t precision, double rho_ref, double* mass_out,
                                       int32_t* status_out, void* stream) {
  if (!f || !mass_out || !status_out) return LBM_EINVAL;
  if (nx < 1 || ny < 1 || precision < LBM_FP64 || precision > LBM_FP32_DEV) return LBM_EINVAL;
  const long long N = (long long)nx * ny;
  if (N > (long long)kNodesPerBlock * kMaxBlocks) return LBM_EINVAL;  // beyond the scratch
  double* scratch = nullptr;
  const lbm_status st = scratch_for_current_device(&scratch);
  if (st != LBM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int nblocks = (int)((N + kNodesPerBlock - 1) / kNodesPerBlock);
  if (precision == LBM_FP32_DEV)
    noalloc_partial_kernel<float><<<nblocks, kThreads, 0, s>>>((int)N, rho_ref, (const float*)f,
                                                               flags, scratch);
  else
    noalloc_partial_kernel<double><<<nblocks, kThreads, 0, s>>>((int)N, 0.0, (const double*)f,
                                                                flags, scratch);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  noalloc_final_kernel<<<1, kThreads, 0, s>>>(scratch, nblocks, mass_out, (int*)status_out);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  return LBM_OK;
}
