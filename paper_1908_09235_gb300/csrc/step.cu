// The fused per-node pass of one time step (Sec. 2.1, Sec. 3.2):
//   density and velocity (Eq. 5), pseudopotential force (Eq. 16) from psi of the 8 neighbours,
//   BGK collision with Guo forcing (Eqs. 2, 4), streaming (Eq. 3).
//
// Layout: two lattices of 9 planes [a][j][i] (structure of arrays).  The source lattice holds
// f(x, t) at x; each fluid node writes f*_a(x, t) to x + e_a of the destination lattice (push),
// including into solid nodes, whose slots then hold the outgoing populations the boundary pass
// reads.  Every population is read once and written once per step.
//
// A CTA covers a 32 x (8 RY) tile; each thread keeps the 9 populations of its RY nodes in
// registers.  psi of the tile and of a one-node ring around it goes to shared memory (ring nodes
// recompute their density from their own 9 populations), so the force needs no second pass over
// memory.  RY = 4 rows per thread for FP32 arithmetic, 2 for FP64 (register budget).
#include "step_core.cuh"

namespace lbm {

namespace {

using namespace step_core;

// CTAs per SM the tile kernels are compiled for (register budget 65536 / (256 x this)), as
// measured on the batched workload: FP32 storage, 3 for 32-row tiles (at 4 they spill; 5% slower)
// and 4 for shorter ones; FP16 storage, 4 (at 3 its 32-row tiles ran 11% slower); FP64, 2.
template <typename S, int RY>
constexpr int tile_ctas() {
  return sizeof(S) == 8 ? 2 : (sizeof(S) == 4 && RY == 4 ? 3 : 4);
}

template <typename S, int EOS, bool FIELDS>
__global__ void __launch_bounds__(TX* TYT, tile_ctas<S, StoreTraits<S>::RY>())
    step_kernel(DevParams p, const void* __restrict__ fa, void* __restrict__ fb,
                const uint8_t* __restrict__ flags, double* __restrict__ rho_m,
                double* __restrict__ ux_m, double* __restrict__ uy_m) {
  using C = typename StoreTraits<S>::C;
  constexpr int RY = StoreTraits<S>::RY;
  __shared__ C psi_s[TYT * RY + 2][TX + 2];
  step_tile<S, EOS, FIELDS, RY>(p, fa, fb, flags, rho_m, ux_m, uy_m, blockIdx.x * TX,
                                blockIdx.y * TYT * RY, psi_s);
}

// Many lattices in one launch: a persistent grid works through a queue of tiles (domain, x0,
// y0).  With claim == nullptr each CTA takes every gridDim.x-th tile; otherwise CTAs claim the
// next tile from the device counter *claim (reset to 0 by the advance kernel after every step),
// one atomic per tile, taken while the previous tile is still being worked on.  Tiles of domains
// whose step budget is spent are skipped.  RY (rows per thread, so the tile height 8 RY) and the
// queue are chosen by the batch's tuner.
template <typename S, int EOS, int RY>
__global__ void __launch_bounds__(TX* TYT, tile_ctas<S, RY>())
    batch_step_kernel(const BatchDomain* __restrict__ doms, const int4* __restrict__ tiles,
                      const int* __restrict__ n_tiles, int* __restrict__ claim) {
  using C = typename StoreTraits<S>::C;
  __shared__ C psi_s[TYT * RY + 2][TX + 2];
  __shared__ int next_s[2];  // claimed tiles, double-buffered across the end-of-tile barrier
  const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
  const int nt = *n_tiles;
  int t = blockIdx.x;
  if (claim) {
    if (lead) next_s[0] = atomicAdd(claim, 1);
    __syncthreads();
    t = next_s[0];
  }
  for (int k = 1; t < nt; ++k) {
    if (claim && lead) next_s[k & 1] = atomicAdd(claim, 1);
    const int4 tile = tiles[t];  // (domain, x0, y0, -)
    const BatchDomain& D = doms[tile.x];
    if (D.steps_left > 0) {
      const int cur = D.cur;
      step_tile<S, EOS, false, RY>(D.p, D.f[cur], D.f[cur ^ 1], D.flags, D.rho_m, D.ux_m,
                                   D.uy_m, tile.y, tile.z, psi_s);
    }
    __syncthreads();  // psi_s is reused by the next tile; next_s[k & 1] is visible
    t = claim ? next_s[k & 1] : t + gridDim.x;
  }
}


template <typename S, int EOS>
cudaError_t launch_t(const DevParams& p, const void* fa, void* fb, const uint8_t* flags,
                     double* rho_m, double* ux_m, double* uy_m, bool fields_only,
                     cudaStream_t s) {
  constexpr int TH = TYT * StoreTraits<S>::RY;
  dim3 block(TX, TYT);
  dim3 grid((p.nx + TX - 1) / TX, (p.ny + TH - 1) / TH);
  if (fields_only)
    step_kernel<S, EOS, true><<<grid, block, 0, s>>>(p, fa, fb, flags, rho_m, ux_m, uy_m);
  else
    step_kernel<S, EOS, false><<<grid, block, 0, s>>>(p, fa, fb, flags, rho_m, ux_m, uy_m);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_s(const DevParams& p, const void* fa, void* fb, const uint8_t* flags,
                     double* rho_m, double* ux_m, double* uy_m, bool fields_only,
                     cudaStream_t s) {
  switch (p.eos) {
    case LBM_EOS_EXP:
      return launch_t<S, LBM_EOS_EXP>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s);
    case LBM_EOS_CS:
      return launch_t<S, LBM_EOS_CS>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s);
    default:
      return launch_t<S, LBM_EOS_NONE>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s);
  }
}

template <typename S, int EOS, int RY>
cudaError_t launch_batch_t(const BatchDomain* doms, const int4* tiles, const int* n_tiles,
                           int* claim, int grid, cudaStream_t s) {
  batch_step_kernel<S, EOS, RY><<<grid, dim3(TX, TYT), 0, s>>>(doms, tiles, n_tiles, claim);
  return cudaGetLastError();
}

template <typename S, int RY>
cudaError_t launch_batch_e(int eos, const BatchDomain* doms, const int4* tiles, const int* n_tiles,
                           int* claim, int grid, cudaStream_t s) {
  switch (eos) {
    case LBM_EOS_EXP:
      return launch_batch_t<S, LBM_EOS_EXP, RY>(doms, tiles, n_tiles, claim, grid, s);
    case LBM_EOS_CS: return launch_batch_t<S, LBM_EOS_CS, RY>(doms, tiles, n_tiles, claim, grid, s);
    default: return launch_batch_t<S, LBM_EOS_NONE, RY>(doms, tiles, n_tiles, claim, grid, s);
  }
}

template <typename S>
cudaError_t launch_batch_s(int eos, int ry, const BatchDomain* doms, const int4* tiles,
                           const int* n_tiles, int* claim, int grid, cudaStream_t s) {
  if (ry == 1) return launch_batch_e<S, 1>(eos, doms, tiles, n_tiles, claim, grid, s);
  if (ry == 2) return launch_batch_e<S, 2>(eos, doms, tiles, n_tiles, claim, grid, s);
  if constexpr (sizeof(typename Pop<S>::C) == 4) {
    if (ry == 4) return launch_batch_e<S, 4>(eos, doms, tiles, n_tiles, claim, grid, s);
  }
  return cudaErrorInvalidValue;
}

template <typename S>
int batch_grid_s(int eos, int ry) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fn = nullptr;
  auto pick = [&](auto k) { fn = reinterpret_cast<const void*>(k); };
  if (ry == 1) pick(batch_step_kernel<S, LBM_EOS_CS, 1>);
  else if (ry == 2) pick(batch_step_kernel<S, LBM_EOS_CS, 2>);
  else if constexpr (sizeof(typename Pop<S>::C) == 4) pick(batch_step_kernel<S, LBM_EOS_CS, 4>);
  if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, TX * TYT, 0) != cudaSuccess) {
    cudaGetLastError();
    per = 2;
  }
  (void)eos;
  return sms * (per > 0 ? per : 1);
}

}  // namespace

int batch_tile_rows(int ry) { return TYT * ry; }
int batch_tile_cols() { return TX; }

int batch_step_grid(int precision, int eos, int ry) {
  if (precision == LBM_FP32_DEV) return batch_grid_s<float>(eos, ry);
  if (precision == LBM_FP16_DEV) return batch_grid_s<__half>(eos, ry);
  return batch_grid_s<double>(eos, ry);
}

cudaError_t launch_batch_step(int precision, int eos, int ry, const BatchDomain* doms,
                              const int4* tiles, const int* n_tiles, int* claim, int grid,
                              cudaStream_t s) {
  if (precision == LBM_FP32_DEV)
    return launch_batch_s<float>(eos, ry, doms, tiles, n_tiles, claim, grid, s);
  if (precision == LBM_FP16_DEV)
    return launch_batch_s<__half>(eos, ry, doms, tiles, n_tiles, claim, grid, s);
  return launch_batch_s<double>(eos, ry, doms, tiles, n_tiles, claim, grid, s);
}

cudaError_t launch_step(int precision, const DevParams& p, const void* fa, void* fb,
                        const uint8_t* flags, double* rho_m, double* ux_m, double* uy_m,
                        bool fields_only, cudaStream_t s, int path, int* err) {
  // FP64 is bound by the FP64 pipe, where the scalar tiling (fewer ring psi per node) is faster
  const bool vec = path == 3 || ((path == 0 || path == 4) && precision != LBM_FP64);
  if (vec && step_vec_supported(precision, p.nx, p.ny))
    return launch_step_vec(precision, p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s,
                           (path == 0 || path == 4) && err != nullptr, err);
  if (precision == LBM_FP32_DEV)
    return launch_s<float>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s);
  if (precision == LBM_FP16_DEV)
    return launch_s<__half>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s);
  return launch_s<double>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s);
}

}  // namespace lbm
