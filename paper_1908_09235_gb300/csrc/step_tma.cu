// Fused step with TMA halo staging (FP32 deviation storage): the same per-node arithmetic as
// step_kernel (csrc/step_core.cuh), but a persistent CTA of 512 threads (two CTAs per SM) stages
// each 32 x 32 tile together with
// its one-node ring, in all nine planes, into shared memory with a single tensor copy
// (cp.async.bulk.tensor.3d, box 40 x 34 x 9 starting at (x0 - 4, y0 - 1): the x start stays
// 16-byte aligned), double-buffered on mbarriers so the copy of the CTA's next tile runs while
// the current one is computed.  Tiles that touch the periodic seam (whose ring wraps) are staged
// with plain loads instead.  Every mbarrier wait is bounded (about 2 s): on expiry the CTA
// records an error (kErrTimeout in the context's error word, reported as LBM_ETIMEOUT by
// lbm_mass), waits boundedly for its own copies in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "step_core.cuh"
#include "tma.cuh"

namespace lbm {

namespace {

using namespace step_core;
using namespace tma;

constexpr int TYM = 16;                   // threads of a CTA in y (512 threads)
constexpr int RYT = 2;                    // rows per thread: tile 32 x 32
constexpr int TH = TYM * RYT;             // 32
constexpr int NT = TX * TYM;              // threads per CTA
constexpr int SW = TX + 8;                // staged width: x0 - 4 .. x0 + 35
constexpr int SH = TH + 2;                // staged height: y0 - 1 .. y0 + 32
constexpr int PLANE = SH * SW;            // floats per plane of a stage
constexpr int STAGE_FLOATS = 9 * PLANE;   // 12240 floats
constexpr uint32_t POP_BYTES = STAGE_FLOATS * 4;   // 48960 bytes of populations per tile
constexpr int FW = 64;                             // staged flag width: x0 - 16 .. x0 + 47
constexpr uint32_t FLAG_BYTES = FW * SH;           // 2176 bytes of node flags per tile
constexpr uint32_t FLAG_OFF = (POP_BYTES + 127) / 128 * 128;
constexpr uint32_t STAGE_BYTES = POP_BYTES + FLAG_BYTES;  // bytes the copies bring per tile
constexpr uint32_t STAGE_STRIDE = (FLAG_OFF + FLAG_BYTES + 127) / 128 * 128;
constexpr int NSTAGE = 2;
constexpr size_t SMEM_BYTES = NSTAGE * STAGE_STRIDE + (TH + 2) * (TX + 2) * 4;

// A tile whose staged boxes lie inside the lattice (no periodic wrap): copied by TMA.
__device__ __forceinline__ bool tma_tile(int x0, int y0, int nx, int ny) {
  return x0 >= 32 && x0 + 48 <= nx && y0 >= 1 && y0 + 33 <= ny;
}

// Self-test of the bounded wait: one CTA waits on phase 0 of a barrier that expects one arrival.
// With arrive, thread 0 arrives and the phase completes; without, nothing completes it and the
// wait must give up after limit_ns.  out[0]: 1 if the wait saw the phase complete, else 0.
__global__ void wait_selftest_kernel(unsigned long long limit_ns, int arrive, int* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&bar)) : "memory");
  const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
  if (threadIdx.x == 0) out[0] = ok ? 1 : 0;
}

template <int EOS>
__global__ void __launch_bounds__(TX* TYM, 2)
    step_tma_kernel(const __grid_constant__ CUtensorMap tmap,
                    const __grid_constant__ CUtensorMap fmap, DevParams p,
                    const float* __restrict__ fa, void* __restrict__ fb,
                    const uint8_t* __restrict__ flags, double* __restrict__ rho_m,
                    double* __restrict__ ux_m, double* __restrict__ uy_m, int tiles_x,
                    int n_tiles, int* __restrict__ err) {
  using C = float;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* stage[NSTAGE] = {reinterpret_cast<float*>(smem_raw),
                          reinterpret_cast<float*>(smem_raw + STAGE_STRIDE)};
  C(*psi_s)[TX + 2] = reinterpret_cast<C(*)[TX + 2]>(smem_raw + NSTAGE * STAGE_STRIDE);
  __shared__ __align__(8) uint64_t bars[NSTAGE];

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int nx = p.nx, ny = p.ny, N = p.N;
  const Consts<C>& k = p.k<C>();
  const C rho_ref = k.rho_ref, psi_w = k.psi_wall;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto tile_xy = [&](int t, int& x0, int& y0) {
    x0 = (t % tiles_x) * TX;
    y0 = (t / tiles_x) * TH;
  };
  auto issue = [&](int t, int s) {  // by thread 0
    int x0, y0;
    tile_xy(t, x0, y0);
    fence_proxy_async();  // generic reads of this stage precede the async-proxy writes
    mbar_expect_tx(&bars[s], STAGE_BYTES);
    tma_load_3d(stage[s], &tmap, &bars[s], x0 - 4, y0 - 1, 0);
    tma_load_2d(reinterpret_cast<unsigned char*>(stage[s]) + FLAG_OFF, &fmap, &bars[s], x0 - 16,
                y0 - 1);
  };

  uint32_t phase = 0;     // bit s: parity of the next completion of stage s
  uint32_t inflight = 0;  // bit s: a copy into stage s has been issued and not waited for
  int t = blockIdx.x;
  if (t < n_tiles) {
    int x0, y0;
    tile_xy(t, x0, y0);
    if (tma_tile(x0, y0, nx, ny)) {
      if (tid == 0) issue(t, 0);
      inflight |= 1u;
    }
  }
  for (int it = 0; t < n_tiles; ++it, t += gridDim.x) {
    const int s = it & 1;
    int x0, y0;
    tile_xy(t, x0, y0);
    // prefetch the next tile of this CTA into the other stage (freed at the end of the last
    // iteration)
    const int tn = t + gridDim.x;
    if (tn < n_tiles) {
      int xn, yn;
      tile_xy(tn, xn, yn);
      if (tma_tile(xn, yn, nx, ny)) {
        if (tid == 0) issue(tn, s ^ 1);
        inflight |= 1u << (s ^ 1);
      }
    }
    float* st = stage[s];
    uint8_t* sfl = reinterpret_cast<uint8_t*>(st) + FLAG_OFF;  // [SH][FW], column 16 is x0
    if (inflight & (1u << s)) {
      const bool ok = mbar_wait_bounded(&bars[s], (phase >> s) & 1u);
      phase ^= 1u << s;
      inflight &= ~(1u << s);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(err, kErrTimeout);
        for (int q = 0; q < NSTAGE; ++q)  // bounded drain of this CTA's copies in flight
          if (inflight & (1u << q)) mbar_wait_bounded(&bars[q], (phase >> q) & 1u);
        return;
      }
    } else {
      // staged by plain loads with periodic wrap
      for (int e = tid; e < STAGE_FLOATS; e += NT) {
        const int a = e / PLANE, rem = e - a * PLANE;
        const int row = rem / SW, col = rem - row * SW;
        const int gx = wrap_any(x0 - 4 + col, nx), gy = wrap_any(y0 - 1 + row, ny);
        st[e] = fa[a * N + gy * nx + gx];
      }
      for (int e = tid; e < (int)FLAG_BYTES; e += NT) {
        const int row = e / FW, col = e - row * FW;
        const int gx = wrap_any(x0 - 16 + col, nx), gy = wrap_any(y0 - 1 + row, ny);
        sfl[e] = flags[gy * nx + gx];
      }
      __syncthreads();
    }

    // phase 1 from the stage: own nodes and the ring (lattices of at least 64 x 64: one wrap)
    C f[RYT][9];
    C rho[RYT];
    uint8_t fl[RYT];
#pragma unroll
    for (int r = 0; r < RYT; ++r) {
      const int row = ty + r * TYM + 1;
      fl[r] = sfl[row * FW + tx + 16];
#pragma unroll
      for (int a = 0; a < 9; ++a) f[r][a] = st[a * PLANE + row * SW + tx + 4];
      rho[r] = (fl[r] & FLAG_SOLID) ? C(1) : r_add(rho_ref, pop_sum<C>(f[r]));
      if constexpr (EOS != LBM_EOS_NONE)
        psi_s[row][tx + 1] = (fl[r] & FLAG_SOLID) ? psi_w : psi_of<C, EOS>(k, rho[r]);
    }
    if constexpr (EOS != LBM_EOS_NONE) {
      constexpr int kRing = 2 * (TX + 2) + 2 * TH;
      if (tid < kRing) {
        const int c = tid;
        int hx, hy;
        if (c < 2 * (TX + 2)) {
          hx = c < TX + 2 ? c : c - (TX + 2);
          hy = c < TX + 2 ? 0 : TH + 1;
        } else {
          const int kk = c - 2 * (TX + 2);
          hx = kk < TH ? 0 : TX + 1;
          hy = (kk < TH ? kk : kk - TH) + 1;
        }
        C ps = psi_w;
        if (!(sfl[hy * FW + hx + 15] & FLAG_SOLID)) {
          C v[9];
#pragma unroll
          for (int a = 0; a < 9; ++a) v[a] = st[a * PLANE + hy * SW + hx + 3];
          ps = psi_of<C, EOS>(k, r_add(rho_ref, pop_sum<C>(v)));
        }
        psi_s[hy][hx] = ps;
      }
    }
    __syncthreads();
    tile_phase2<float, EOS, false, RYT, TYM>(p, fb, rho_m, ux_m, uy_m, x0, y0, psi_s, f, rho,
                                             fl);
    __syncthreads();  // the stage and psi_s are free for the next tile
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    else
      cudaGetLastError();
  }
  return fn;
}

template <int EOS>
cudaError_t launch_tma_t(const CUtensorMap& map, const CUtensorMap& fmap, const DevParams& p,
                         const void* fa, void* fb,
                         const uint8_t* flags, double* rho_m, double* ux_m, double* uy_m,
                         int* err, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(step_tma_kernel<EOS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles_x = (p.nx + TX - 1) / TX, tiles_y = (p.ny + TH - 1) / TH;
  const int n_tiles = tiles_x * tiles_y;
  int grid = 2 * sms;
  if (grid > n_tiles) grid = n_tiles;
  step_tma_kernel<EOS><<<grid, dim3(TX, TYM), SMEM_BYTES, s>>>(
      map, fmap, p, static_cast<const float*>(fa), fb, flags, rho_m, ux_m, uy_m, tiles_x, n_tiles, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned long long limit_ns, int arrive, int* out,
                                 cudaStream_t s) {
  wait_selftest_kernel<<<1, 128, 0, s>>>(limit_ns, arrive, out);
  return cudaGetLastError();
}

bool tma_step_supported(int precision, int nx, int ny) {
  return precision == LBM_FP32_DEV && nx % 16 == 0 && nx >= 64 && ny >= 64 &&
         encoder() != nullptr;
}

// Tensor map of the node flags: dims (nx, ny) bytes, box 64 x 34.
bool make_flags_tensor_map(void* map, const void* base, int nx, int ny) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
  const cuuint64_t strides[1] = {(cuuint64_t)nx};
  const cuuint32_t box[2] = {FW, SH};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                  const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Tensor map of one FP32 lattice for the vector step kernel's psi ring: dims (nx, ny, 9), box
// box_w x 1 x 9 (one staged row of all nine planes).
bool make_ring_tensor_map(void* map, const void* base, int nx, int ny, int box_w) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 9};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)box_w, 1, 9};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                  const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Tensor maps of one FP16-deviation lattice for the vector step kernel's psi ring: map0 the FP32
// rest plane (dims (nx, ny), box w0 x 1), map1 the eight FP16 planes after it (dims (nx, ny, 8),
// box w1 x 1 x 8).  The FP16 row pitch must be a multiple of 16 bytes (nx % 8 == 0).
bool make_ring_tensor_maps_fp16(void* map0, void* map1, const void* base, int nx, int ny, int w0,
                                int w1) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
  if (!fn || nx % 8 != 0) return false;
  const cuuint64_t d0[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
  const cuuint64_t s0[1] = {(cuuint64_t)nx * 4};
  const cuuint32_t b0[2] = {(cuuint32_t)w0, 1};
  const cuuint32_t e0[2] = {1, 1};
  CUresult r = fn(static_cast<CUtensorMap*>(map0), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void*>(base), d0, s0, b0, e0, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  const size_t N = (size_t)nx * ny;
  void* moving = static_cast<char*>(const_cast<void*>(base)) + N * 4;
  const cuuint64_t d1[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 8};
  const cuuint64_t s1[2] = {(cuuint64_t)nx * 2, (cuuint64_t)N * 2};
  const cuuint32_t b1[3] = {(cuuint32_t)w1, 1, 8};
  const cuuint32_t e1[3] = {1, 1, 1};
  r = fn(static_cast<CUtensorMap*>(map1), CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, moving, d1, s1, b1,
         e1, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// A tiled tensor map over a dense array of dims[0] x dims[1] (x dims[2]) elements of esize
// bytes, row-major with dims[0] innermost, box box[0] x box[1] (x box[2]).
bool encode_box(void* map, CUtensorMapDataType type, int esize, int rank, const void* base,
                const cuuint64_t* dims, const cuuint32_t* box) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
  if (!fn) return false;
  const cuuint64_t strides[2] = {dims[0] * (cuuint64_t)esize,
                                 dims[0] * dims[1] * (cuuint64_t)esize};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(static_cast<CUtensorMap*>(map), type, rank, const_cast<void*>(base), dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Tensor maps of one lattice whose box is a whole tile of the vector step kernel (tw x vh nodes,
// every plane), for L2 prefetches: FP32 deviations map0 dims (nx, ny, 9); FP16 deviations map0
// the FP32 rest plane (nx, ny) and map1 the eight FP16 planes (nx, ny, 8; nx % 8 == 0).
bool make_tile_prefetch_maps(void* map0, void* map1, const void* base, int nx, int ny, int tw,
                             int vh, bool fp16) {
  const cuuint64_t d3[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 9};
  if (!fp16) {
    const cuuint32_t b[3] = {(cuuint32_t)tw, (cuuint32_t)vh, 9};
    return encode_box(map0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 3, base, d3, b);
  }
  if (nx % 8 != 0) return false;
  const cuuint32_t b0[2] = {(cuuint32_t)tw, (cuuint32_t)vh};
  if (!encode_box(map0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 2, base, d3, b0)) return false;
  const cuuint64_t d1[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 8};
  const cuuint32_t b1[3] = {(cuuint32_t)tw, (cuuint32_t)vh, 8};
  const void* moving = static_cast<const char*>(base) + (size_t)nx * ny * 4;
  return encode_box(map1, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, 3, moving, d1, b1);
}

// Tensor map of a lattice's node flags (dims (nx, ny) bytes) whose box is a whole tile of the
// vector step kernel (tw x vh), for L2 prefetches; the row pitch must be a multiple of 16 bytes.
bool make_flags_prefetch_map(void* map, const uint8_t* flags, int nx, int ny, int tw, int vh) {
  if (nx % 16 != 0) return false;
  const cuuint64_t d[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
  const cuuint32_t b[2] = {(cuuint32_t)tw, (cuuint32_t)vh};
  return encode_box(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, 2, flags, d, b);
}

// Tensor map of one FP32 lattice: dims (nx, ny, 9), box 40 x 34 x 9.
bool make_lattice_tensor_map(void* map, const void* base, int nx, int ny) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 9};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  const cuuint32_t box[3] = {SW, SH, 9};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                  const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

cudaError_t launch_step_tma(const void* map, const void* flag_map, const DevParams& p,
                            const void* fa, void* fb, const uint8_t* flags, double* rho_m,
                            double* ux_m, double* uy_m, int* err, cudaStream_t s) {
  const CUtensorMap& m = *static_cast<const CUtensorMap*>(map);
  const CUtensorMap& fm = *static_cast<const CUtensorMap*>(flag_map);
  switch (p.eos) {
    case LBM_EOS_EXP:
      return launch_tma_t<LBM_EOS_EXP>(m, fm, p, fa, fb, flags, rho_m, ux_m, uy_m, err, s);
    case LBM_EOS_CS:
      return launch_tma_t<LBM_EOS_CS>(m, fm, p, fa, fb, flags, rho_m, ux_m, uy_m, err, s);
    default:
      return launch_tma_t<LBM_EOS_NONE>(m, fm, p, fa, fb, flags, rho_m, ux_m, uy_m, err, s);
  }
}

}  // namespace lbm
