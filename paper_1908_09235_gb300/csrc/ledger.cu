// Mass ledger (total mass m = sum over fluid nodes and directions of f, the quantity whose ratio
// m/m0 the paper plots in Figs. 4, 8 and 11) and the equilibrium initialisation f = f_eq(rho, u).
//
// The ledger reduces in FP64 with a fixed grid and a fixed reduction tree, so the same state
// always gives the same bits: each thread keeps a compensated (Neumaier) sum over a grid-stride
// range of nodes, warps combine by shuffles, blocks write partials, one block adds the partials.
#include "d2q9.cuh"

namespace lbm {

namespace {

constexpr int kLedgerThreads = 256;
constexpr int kLedgerMaxBlocks = 152 * 8;

struct Comp {
  double s, c;
  __device__ void add(double x) {
    double t = s + x;
    if (fabs(s) >= fabs(x))
      c += (s - t) + x;
    else
      c += (x - t) + s;
    s = t;
  }
};

__device__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// Block-wide sum in a fixed order; result valid in thread 0.
__device__ double block_sum(double v) {
  __shared__ double sh[kLedgerThreads / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < kLedgerThreads / 32 ? sh[lane] : 0.0;
    v = warp_sum(v);
  }
  return v;
}

template <typename S>
__global__ void __launch_bounds__(kLedgerThreads) mass_partial_kernel(
    int N, double rho_ref, const void* __restrict__ f, const uint8_t* __restrict__ flags,
    double* __restrict__ partials, int* __restrict__ err) {
  Comp acc{0.0, 0.0};
  bool bad = false;
  for (int n = blockIdx.x * kLedgerThreads + threadIdx.x; n < N; n += gridDim.x * kLedgerThreads) {
    if (flags[n] & FLAG_SOLID) continue;
    double r = 0.0;
#pragma unroll
    for (int a = 0; a < 9; ++a) r += double(Pop<S>::load(f, a, N, n));
    if (Pop<S>::dev) r += rho_ref;
    if (!(r > 0.0) || !isfinite(r)) bad = true;
    acc.add(r);
  }
  if (bad) atomicOr(err, 1);
  const double t = block_sum(acc.s + acc.c);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kLedgerThreads) mass_final_kernel(const double* __restrict__ partials,
                                                                    int nblocks,
                                                                    double* __restrict__ result) {
  Comp acc{0.0, 0.0};
  for (int k = threadIdx.x; k < nblocks; k += kLedgerThreads) acc.add(partials[k]);
  const double t = block_sum(acc.s + acc.c);
  if (threadIdx.x == 0) *result = t;
}

template <typename S>
__global__ void init_eq_kernel(DevParams p, const uint8_t* __restrict__ flags,
                               const double* __restrict__ rho, const double* __restrict__ ux,
                               const double* __restrict__ uy, void* __restrict__ f) {
  using C = typename Pop<S>::C;
  const int N = p.N;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < p.N; n += gridDim.x * blockDim.x) {
    if (flags[n] & FLAG_SOLID) {
#pragma unroll
      for (int a = 0; a < 9; ++a) Pop<S>::store(f, a, N, n, C(0));
      continue;
    }
    // Eq. (4), f_eq = w rho (A + 3 e.u + 4.5 (e.u)^2) with A = 1 - 1.5 u.u, in FP64 (the FP64
    // pipe bounds this kernel): opposite directions share w rho (A + 4.5 (e.u)^2) and differ in
    // the sign of 3 w rho e.u; the deviation formats take w rho_ref off the shared part
    const double r = rho[n], u = ux[n], v = uy[n];
    const double A = 1.0 - 1.5 * (u * u + v * v);
    const double ref = Pop<S>::dev ? p.rho_ref : 0.0;
    Pop<S>::store(f, 0, N, n, C(wgt<double>(0) * (r * A - ref)));
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int a = i == 0 ? 1 : (i == 1 ? 2 : (i == 2 ? 5 : 6));  // e_a = (1,0) (0,1) (1,1) (-1,1)
      const double eu = i == 0 ? u : (i == 1 ? v : (i == 2 ? u + v : v - u));
      const double w = wgt<double>(a);
      const double P = w * (r * (A + 4.5 * eu * eu) - ref), Q = 3.0 * w * r * eu;
      Pop<S>::store(f, a, N, n, C(P + Q));
      Pop<S>::store(f, opposite(a), N, n, C(P - Q));
    }
  }
}

__global__ void droplet_kernel(DevParams p, double cx, double cy, double R, double W, double rin,
                               double rout, double* __restrict__ rho, double* __restrict__ ux,
                               double* __restrict__ uy) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < p.N; n += gridDim.x * blockDim.x) {
    const double dx = double(n % p.nx) - cx, dy = double(n / p.nx) - cy;
    const double r = sqrt(dx * dx + dy * dy);
    rho[n] = 0.5 * (rin + rout) - 0.5 * (rin - rout) * tanh(2.0 * (r - R) / W);
    ux[n] = 0.0;
    uy[n] = 0.0;
  }
}

int grid_for(int N) {
  int b = (N + 255) / 256;
  return b > 152 * 32 ? 152 * 32 : b;
}

}  // namespace

int ledger_num_blocks(int N) {
  int b = (N + kLedgerThreads - 1) / kLedgerThreads;
  return b > kLedgerMaxBlocks ? kLedgerMaxBlocks : b;
}

cudaError_t launch_mass(int precision, const DevParams& p, const void* f, const uint8_t* flags,
                        double* partials, int nblocks, double* result, int* err_flag,
                        cudaStream_t s) {
  if (precision == LBM_FP32_DEV)
    mass_partial_kernel<float><<<nblocks, kLedgerThreads, 0, s>>>(p.N, p.rho_ref, f, flags,
                                                                   partials, err_flag);
  else if (precision == LBM_FP16_DEV)
    mass_partial_kernel<__half><<<nblocks, kLedgerThreads, 0, s>>>(p.N, p.rho_ref, f, flags,
                                                                    partials, err_flag);
  else
    mass_partial_kernel<double><<<nblocks, kLedgerThreads, 0, s>>>(p.N, 0.0, f, flags, partials,
                                                                    err_flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  mass_final_kernel<<<1, kLedgerThreads, 0, s>>>(partials, nblocks, result);
  return cudaGetLastError();
}

cudaError_t launch_init_eq(int precision, const DevParams& p, const uint8_t* flags,
                           const double* rho, const double* ux, const double* uy, void* f,
                           cudaStream_t s) {
  if (precision == LBM_FP32_DEV)
    init_eq_kernel<float><<<grid_for(p.N), 256, 0, s>>>(p, flags, rho, ux, uy, f);
  else if (precision == LBM_FP16_DEV)
    init_eq_kernel<__half><<<grid_for(p.N), 256, 0, s>>>(p, flags, rho, ux, uy, f);
  else
    init_eq_kernel<double><<<grid_for(p.N), 256, 0, s>>>(p, flags, rho, ux, uy, f);
  return cudaGetLastError();
}

cudaError_t launch_droplet_rho(const DevParams& p, double cx, double cy, double R, double W,
                               double rho_in, double rho_out, double* rho, double* ux, double* uy,
                               cudaStream_t s) {
  droplet_kernel<<<grid_for(p.N), 256, 0, s>>>(p, cx, cy, R, W, rho_in, rho_out, rho, ux, uy);
  return cudaGetLastError();
}

// Smallest positive finite value of v[0..n): the automatic reference density of the deviation
// formats.  Positive finite doubles order like their bit patterns as unsigned integers, so the
// minimum is an exact atomicMin on the bits (order-independent, the same value as any serial
// scan).  *out = +inf when there is no such value.
__global__ void min_init_kernel(unsigned long long* out) { *out = 0x7ff0000000000000ULL; }

__global__ void min_positive_kernel(const double* __restrict__ v, long long n,
                                    unsigned long long* __restrict__ out) {
  unsigned long long m = 0x7ff0000000000000ULL;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const double x = v[k];
    if (x > 0.0 && x < __longlong_as_double(0x7ff0000000000000LL)) {
      const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
      m = b < m ? b : m;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t < m ? t : m;
  }
  if ((threadIdx.x & 31) == 0 && m != 0x7ff0000000000000ULL) atomicMin(out, m);
}

cudaError_t launch_min_positive(const double* v, long long n, double* out, cudaStream_t s) {
  unsigned long long* o = reinterpret_cast<unsigned long long*>(out);
  min_init_kernel<<<1, 1, 0, s>>>(o);
  long long blocks = (n + 255) / 256;
  if (blocks > 1216) blocks = 1216;
  if (blocks < 1) blocks = 1;
  min_positive_kernel<<<(unsigned)blocks, 256, 0, s>>>(v, n, o);
  return cudaGetLastError();
}

}  // namespace lbm
