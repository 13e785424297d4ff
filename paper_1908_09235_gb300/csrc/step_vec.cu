// The vectorised fused per-node pass of one time step (Sec. 2.1, Sec. 3.2): density and velocity
// (Eq. 5), pseudopotential force (Eq. 16), BGK collision with Guo forcing (Eqs. 2, 4), streaming
// (Eq. 3), for lattices whose width is a multiple of the vector width V.
//
// Each lane owns V consecutive nodes of one row and moves every population plane as one vector
// (FP32: 4 x 4 B, FP64: 2 x 8 B = 128-bit accesses; FP16 deviations: the FP32 rest plane as
// 4 x 4 B and each FP16 plane as 4 x 2 B), so a warp reads or writes 32 V nodes of a plane with
// one request.  A CTA of VH warps covers a (32 V) x VH tile, one row per warp (VH = 8; 12 for
// the FP16 format).
//
// psi stencil: psi of the tile's own nodes comes from the lanes' registers; psi of the one-node
// ring around the tile (the rows above and below, one column on each side) comes from
// populations staged in shared memory, which needs no registers and fetches the side columns as
// aligned vectors instead of single-element loads: the two rows by tensor copies where the tile
// allows (TR), otherwise, and the side columns always, by cp.async.  With TR the FP32 kernel
// also prefetches into L2, by tensor-copy prefetches, the populations and flags of the tile that
// the CTA launched 152 CTAs later (one per SM of GB300) will load.
//
// Streaming is push (f*_a of node x goes to x + e_a of the destination lattice, into solid nodes
// too, whose slots then hold the outgoing populations the wall pass reads).  A population moving
// in +x enters a lane's destination vector from the lane on its left (warp shuffle), so lanes
// write whole aligned vectors; at the tile's left edge lane 0 writes the V - 1 elements it owns
// and the last lane of the tile on the left writes the first element (likewise in -x).  Every
// destination element is written exactly once.  Elements whose source node is solid carry the
// collision of that node's slot contents: the wall pass overwrites those slots of fluid nodes,
// and those of solid nodes are never read.
//
// The per-node arithmetic is collide_node() and psi_of(), explicitly rounded, so a node gets the
// same bits here, in the scalar tile kernel and in the batched kernel.
#include <type_traits>

#include "step_core.cuh"
#include "tma.cuh"

namespace lbm {

namespace {

using namespace step_core;

constexpr int VW = 32;  // lanes

// async global -> shared copy of 8 or 16 bytes (both addresses aligned to the size), L2 only
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// Vector access to the storage formats of Pop<S>.  Element e of plane a at node n; n % V == 0.
template <typename S>
struct Vec;
template <>
struct Vec<float> {
  static constexpr int V = 4;
  static constexpr int ES = 4;  // largest element size in bytes
  static constexpr int VH = 8;  // warps per CTA = rows per tile
  static constexpr int kBlocks = 3;
  static constexpr bool kOwnFirst = true;  // issue order of the loads (step_vec_kernel)
  // L2 prefetch of the populations and the flags of the tile this many CTAs later in launch
  // order (one CTA per SM ahead): 200 us against 209 us at 4096^2 (populations alone: 206 us; 48
  // ahead: 207, 228: 207, 456: 215, 912: 251; flags 76 or 304 ahead: no better)
  static constexpr int kPrefetchAhead = 152;
  static constexpr bool kPrefetchPops = true, kPrefetchFlags = true;
  // a staged ring row: 9 planes of SWE elements (x0 - V .. x0 + 32 V + V - 1), plane a at
  // ring_off(a); a tensor copy brings kTmaWidth columns from x0 - kTmaLeft
  static constexpr int SWE = VW * V + 2 * V;
  static constexpr int kTmaLeft = V, kTmaWidth = SWE;
  template <bool TMA>
  __host__ __device__ static constexpr int ring_row_bytes() { return 9 * SWE * ES; }
  template <bool TMA>
  static __device__ __forceinline__ int ring_off(int a) { return a * SWE * ES; }
  static __device__ __forceinline__ const float* at(const void* b, int a, int N, int n) {
    return static_cast<const float*>(b) + a * N + LBM_CHK(n, N - 3);
  }
  static __device__ __forceinline__ void load(const void* b, int a, int N, int n, float (&o)[4]) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(at(b, a, N, n)));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  static __device__ __forceinline__ void store(void* b, int a, int N, int n, const float (&v)[4]) {
    *reinterpret_cast<float4*>(static_cast<float*>(b) + a * N + LBM_CHK(n, N - 3)) =
        make_float4(v[0], v[1], v[2], v[3]);
  }
  static __device__ __forceinline__ void store1(void* b, int a, int N, int n, float v) {
    static_cast<float*>(b)[a * N + LBM_CHK(n, N)] = v;
  }
  static __device__ __forceinline__ void store2(void* b, int a, int N, int n, float v0, float v1) {
    *reinterpret_cast<float2*>(static_cast<float*>(b) + a * N + LBM_CHK(n, N - 1)) =
        make_float2(v0, v1);
  }
  static __device__ __forceinline__ int bytes(int a) { return 16; }
  static __device__ __forceinline__ const void* src(const void* b, int a, int N, int n) {
    return at(b, a, N, n);
  }
  // element j of a staged plane
  static __device__ __forceinline__ float staged(const unsigned char* plane, int a, int j) {
    return reinterpret_cast<const float*>(plane)[j];
  }
};
template <>
struct Vec<double> {
  static constexpr int V = 2;
  static constexpr int ES = 8;
  static constexpr int VH = 8;
  static constexpr int kBlocks = 2;
  static constexpr bool kOwnFirst = false;
  static constexpr int kPrefetchAhead = 0;
  static constexpr bool kPrefetchPops = false, kPrefetchFlags = false;
  static constexpr int SWE = VW * V + 2 * V;
  static constexpr int kTmaLeft = V, kTmaWidth = SWE;
  template <bool TMA>
  __host__ __device__ static constexpr int ring_row_bytes() { return 9 * SWE * ES; }
  template <bool TMA>
  static __device__ __forceinline__ int ring_off(int a) { return a * SWE * ES; }
  static __device__ __forceinline__ const double* at(const void* b, int a, int N, int n) {
    return static_cast<const double*>(b) + a * N + LBM_CHK(n, N - 1);
  }
  static __device__ __forceinline__ void load(const void* b, int a, int N, int n,
                                              double (&o)[2]) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(at(b, a, N, n)));
    o[0] = v.x; o[1] = v.y;
  }
  static __device__ __forceinline__ void store(void* b, int a, int N, int n,
                                               const double (&v)[2]) {
    *reinterpret_cast<double2*>(static_cast<double*>(b) + a * N + LBM_CHK(n, N - 1)) =
        make_double2(v[0], v[1]);
  }
  static __device__ __forceinline__ void store1(void* b, int a, int N, int n, double v) {
    static_cast<double*>(b)[a * N + LBM_CHK(n, N)] = v;
  }
  static __device__ __forceinline__ void store2(void* b, int a, int N, int n, double v0,
                                                double v1) {
    *reinterpret_cast<double2*>(static_cast<double*>(b) + a * N + LBM_CHK(n, N - 1)) =
        make_double2(v0, v1);
  }
  static __device__ __forceinline__ int bytes(int a) { return 16; }
  static __device__ __forceinline__ const void* src(const void* b, int a, int N, int n) {
    return at(b, a, N, n);
  }
  static __device__ __forceinline__ double staged(const unsigned char* plane, int a, int j) {
    return reinterpret_cast<const double*>(plane)[j];
  }
};
template <>
struct Vec<__half> {
  // plane 0 FP32 at the base, planes 1..8 FP16 after N floats
  static constexpr int V = 4;
  static constexpr int ES = 4;
  // 12 rows: the ring (two staged rows and their psi) is shared by more nodes; the FP16 step
  // ran 3% faster than with 8 rows, the FP32 step 7% slower
  static constexpr int VH = 12;
  static constexpr int kBlocks = 2;
  static constexpr bool kOwnFirst = false;
  // slower with prefetches (populations 152 or 304 ahead: 195 against 187 us; flags alone 152 or
  // 304 ahead: 194 us)
  static constexpr int kPrefetchAhead = 0;
  static constexpr bool kPrefetchPops = false, kPrefetchFlags = false;
  // a staged ring row (ring_off(a): element x0 - V of plane a).  Staged by cp.async: 9 plane
  // regions of SWE 4-byte slots.  Staged by tensor copies (TMA): the FP32 rest plane (SWE
  // floats from x0 - V) at 0, then the eight FP16 planes densely, kTmaWidth halves each from
  // x0 - 8 (16-byte aligned), from the next 128-byte boundary on.
  static constexpr int SWE = VW * V + 2 * V;
  static constexpr int kTmaLeft = 8, kTmaWidth = SWE + 8;
  static constexpr int kMovOff = (SWE * 4 + 127) / 128 * 128;
  template <bool TMA>
  __host__ __device__ static constexpr int ring_row_bytes() { return TMA ? kMovOff + 8 * kTmaWidth * 2 : 9 * SWE * ES; }
  template <bool TMA>
  static __device__ __forceinline__ int ring_off(int a) {
    if constexpr (TMA)
      return a == 0 ? 0 : kMovOff + (a - 1) * kTmaWidth * 2 + (kTmaLeft - V) * 2;
    else
      return a * SWE * ES;
  }
  static __device__ __forceinline__ const __half* moving(const void* b, int a, int N, int n) {
    return reinterpret_cast<const __half*>(static_cast<const float*>(b) + N) + (a - 1) * N +
           LBM_CHK(n, N);
  }
  static __device__ __forceinline__ void load(const void* b, int a, int N, int n, float (&o)[4]) {
    n = LBM_CHK(n, N - 3);
    if (a == 0) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(static_cast<const float*>(b) + n));
      o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else {
      const uint2 u = __ldcg(reinterpret_cast<const uint2*>(moving(b, a, N, n)));
      const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
      const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
      o[0] = lo.x; o[1] = lo.y; o[2] = hi.x; o[3] = hi.y;
    }
  }
  // v already rounded to the storage format (Pop<__half>::rounded), so the conversion is exact
  static __device__ __forceinline__ void store(void* b, int a, int N, int n, const float (&v)[4]) {
    n = LBM_CHK(n, N - 3);
    if (a == 0) {
      *reinterpret_cast<float4*>(static_cast<float*>(b) + n) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
      const __half2 lo = __floats2half2_rn(v[0], v[1]), hi = __floats2half2_rn(v[2], v[3]);
      uint2 u;
      u.x = *reinterpret_cast<const uint32_t*>(&lo);
      u.y = *reinterpret_cast<const uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(const_cast<__half*>(moving(b, a, N, n))) = u;
    }
  }
  // moving planes only (the rest plane never streams in x)
  static __device__ __forceinline__ void store1(void* b, int a, int N, int n, float v) {
    *const_cast<__half*>(moving(b, a, N, n)) = __float2half_rn(v);
  }
  static __device__ __forceinline__ void store2(void* b, int a, int N, int n, float v0, float v1) {
    *reinterpret_cast<__half2*>(const_cast<__half*>(moving(b, a, N, LBM_CHK(n, N - 1)))) =
        __floats2half2_rn(v0, v1);
  }
  static __device__ __forceinline__ int bytes(int a) { return a == 0 ? 16 : 8; }
  static __device__ __forceinline__ const void* src(const void* b, int a, int N, int n) {
    n = LBM_CHK(n, N - 3);
    return a == 0 ? static_cast<const void*>(static_cast<const float*>(b) + n)
                  : static_cast<const void*>(moving(b, a, N, n));
  }
  static __device__ __forceinline__ float staged(const unsigned char* plane, int a, int j) {
    return a == 0 ? reinterpret_cast<const float*>(plane)[j]
                  : __half2float(reinterpret_cast<const __half*>(plane)[j]);
  }
};

// lane values: element e of a packed pair, and packing (a single node ignores the second)
template <typename L>
__device__ __forceinline__ typename Elem<L>::C el(const L& x, int e) {
  if constexpr (Elem<L>::W == 2) return e == 0 ? x.x : x.y; else return x;
}
template <typename L>
__device__ __forceinline__ L pack(typename Elem<L>::C a, typename Elem<L>::C b) {
  if constexpr (Elem<L>::W == 2) return make_float2(a, b); else return a;
}

template <int V>
__device__ __forceinline__ void load_flags(const uint8_t* flags, int n, uint8_t (&o)[V]) {
  if constexpr (V == 4) {
    const uchar4 u = *reinterpret_cast<const uchar4*>(flags + n);
    o[0] = u.x; o[1] = u.y; o[2] = u.z; o[3] = u.w;
  } else {
    const uchar2 u = *reinterpret_cast<const uchar2*>(flags + n);
    o[0] = u.x; o[1] = u.y;
  }
}

// TR: the two ring rows of tiles away from the x seam are staged by tensor copies
// (cp.async.bulk.tensor) issued by one thread, instead of cp.async by every lane: FP32 one copy
// per row (rmap, box SWE x 1 x 9); FP16 two (rmap: the FP32 rest plane, box SWE x 1; rmap2: the
// eight FP16 planes, box kTmaWidth x 1 x 8).  Their wait is bounded (an expired wait sets
// kErrTimeout in *err).
template <typename S, int EOS, bool FIELDS, bool TR>
__global__ void __launch_bounds__(VW* Vec<S>::VH, Vec<S>::kBlocks)
    step_vec_kernel(DevParams p, const void* __restrict__ fa, void* __restrict__ fb,
                    const uint8_t* __restrict__ flags, double* __restrict__ rho_m,
                    double* __restrict__ ux_m, double* __restrict__ uy_m,
                    const __grid_constant__ CUtensorMap rmap,
                    const __grid_constant__ CUtensorMap rmap2,
                    const __grid_constant__ CUtensorMap pmap,
                    const __grid_constant__ CUtensorMap pmap2,
                    const __grid_constant__ CUtensorMap fmap, int pf_flags,
                    int* __restrict__ err) {
  using C = typename Pop<S>::C;
  using VT = Vec<S>;
  constexpr int V = VT::V;
  constexpr int VH = VT::VH;  // warps per CTA = rows per tile
  constexpr int TW = VW * V;      // tile width
  constexpr int SW = TW + 2 * V;  // staged / psi row: x0 - V .. x0 + TW + V - 1
  constexpr int ES = VT::ES;
  constexpr bool DEV = Pop<S>::dev;
  constexpr bool PSI = EOS != LBM_EOS_NONE;
  // staged populations: the two ring rows (each 9 plane rows of SW elements, rows 128-byte
  // aligned for the tensor copies), and the side vectors (x0 - V, x0 + V nv) of the own rows;
  // plane regions sized for the largest element
  constexpr int RS = (VT::template ring_row_bytes<TR>() + 127) / 128 * 128;
  __shared__ __align__(128) unsigned char ring_st[PSI ? 2 * RS : 16];
  __shared__ __align__(16) unsigned char side_st[PSI ? VH * 2 * 9 * V * ES : 16];
  // psi of x0 - V + j, rows y0 - 1 .. y0 + VH, at column pj(j) = j + j / V: one pad element after
  // every V, so lane l's nodes and their x-neighbours sit at fixed offsets -2, 0 .. V - 1, V + 1
  // from (V + 1)(l + 1), and lanes (stride V + 1 elements) hit distinct banks
  constexpr int SWP = SW + SW / V;
  __shared__ C psi_s[VH + 2][SWP];
  auto pj = [](int j) { return j + j / V; };

  const int lane = threadIdx.x, w = threadIdx.y, tid = w * VW + lane;
  const int nx = p.nx, ny = p.ny, N = p.N;
  const int x0 = blockIdx.x * TW, y0 = blockIdx.y * VH;
  if constexpr (TR && PSI && (VT::kPrefetchPops || VT::kPrefetchFlags)) {
    // the populations and flags of the tile kPrefetchAhead CTAs later in launch order go to L2
    // now, by tensor-copy prefetches of one tile-sized box each, so that its loads find them there
    const int t = blockIdx.y * gridDim.x + blockIdx.x + VT::kPrefetchAhead;
    if (tid == 32 && t < gridDim.x * gridDim.y) {
      const int px = (t % gridDim.x) * TW, py = (t / gridDim.x) * VH;
      if constexpr (VT::kPrefetchPops) {
        if constexpr (sizeof(S) == 2) {
          tma::tma_prefetch_2d(&pmap, px, py);
          tma::tma_prefetch_3d(&pmap2, px, py, 0);
        } else {
          tma::tma_prefetch_3d(&pmap, px, py, 0);
        }
      }
      if constexpr (VT::kPrefetchFlags) {
        if (pf_flags) tma::tma_prefetch_2d(&fmap, px, py);
      }
    }
  }
  const int nv = min(VW, (nx - x0) / V);  // vectors of this tile inside the lattice
  const Consts<C>& k = p.k<C>();
  const C rho_ref = DEV ? k.rho_ref : C(0);
  const C psi_w = k.psi_wall;
  // one wrap suffices: nx >= V and ny >= VH (checked by the launcher)
  auto wrapx = [nx](int x) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); };
  auto wrapy = [ny](int y) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); };

  // tensor copies of the ring rows: a whole tile whose staged columns x0 - V .. x0 + TW + V - 1
  // lie inside the lattice (no wrap in x; rows are addressed wrapped)
  __shared__ __align__(8) uint64_t ring_bar;
  bool tma_rows = false;
  if constexpr (TR && PSI) {
    tma_rows = x0 >= VT::kTmaLeft && x0 - VT::kTmaLeft + VT::kTmaWidth <= nx;
  }

  // nodes whose psi comes from the staged populations: the ring rows' x0 - 1 .. x0 + V nv
  // (rj each, at most RJ), then x0 - 1 and x0 + V nv of each own row
  constexpr int RJ = TW + 2;
  constexpr int nnode = 2 * RJ + 2 * VH;
  // flags of the staged nodes: staged too where a 4-byte copy is aligned (V = 4), else loaded
  // by the thread that computes the node's psi
  constexpr bool SFL = V == 4;
  __shared__ __align__(16) uint8_t ring_fl[SFL && PSI ? 2 * SW : 4];
  __shared__ __align__(16) uint8_t side_fl[SFL && PSI ? VH * 2 * 4 : 4];
  const int nslot = nv + 2, rj = V * nv + 2;
  uint8_t qfl[2] = {0, 0};
  // the tile's own row: V nodes per lane
  const int y = y0 + w, yo = wrapy(y);
  const bool lane_ok = lane < nv;
  const int n = yo * nx + x0 + V * (lane_ok ? lane : 0);
  // the lane's V nodes as NP lane values of W nodes (FP32 arithmetic: pairs in f32x2 registers)
  using L = std::conditional_t<sizeof(C) == 4, float2, C>;
  constexpr int W = Elem<L>::W, NP = V / W;
  L f[NP][9];
  uint8_t fl[V];

  // ---- staged copies: ring rows (slot s at x0 + V (s - 1), s = 0 .. nv + 1) and the side
  // vectors (x0 - V, x0 + V nv) of the own rows.  Warp w copies the ring's (row, plane) pairs
  // w, w + VH, w + 2 VH (those below 18), one slot per lane, and the side vectors of its own
  // row. ----
  auto stage_copies = [&] {
    if constexpr (PSI) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int c = w + VH * i;  // ring row r = c / 9, plane a = c % 9
        if (c < 18 && !tma_rows) {
          const int r = c >= 9 ? 1 : 0, a = c - 9 * r;
          const int grow = wrapy(r == 0 ? y0 - 1 : y0 + VH) * nx;
          unsigned char* plane = ring_st + r * RS + VT::template ring_off<TR>(a);
          const int vb = VT::bytes(a);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int sl = lane + VW * h;
            if (sl < nslot)
              cp_async(plane + sl * vb, VT::src(fa, a, N, grow + wrapx(x0 + V * (sl - 1))), vb);
          }
        }
      }
      const int grow_w = wrapy(y0 + w) * nx;
      if (lane < 18) {
        const int side = lane >= 9 ? 1 : 0, a = lane - 9 * side;
        cp_async(side_st + ((w * 2 + side) * 9 + a) * V * ES,
                 VT::src(fa, a, N, grow_w + wrapx(side == 0 ? x0 - V : x0 + V * nv)),
                 VT::bytes(a));
      }
      if constexpr (SFL) {
        if (w >= VH - 2) {  // the two warps with the fewest ring pairs: ring flags
          const int r = w - (VH - 2);
          const int grow = wrapy(r == 0 ? y0 - 1 : y0 + VH) * nx;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int sl = lane + VW * h;
            if (sl < nslot)
              cp_async4(ring_fl + r * SW + 4 * sl,
                        flags + LBM_CHK(grow + wrapx(x0 + 4 * (sl - 1)), N - 3));
          }
        }
        if (lane == 18 || lane == 19) {
          const int side = lane - 18;
          cp_async4(side_fl + (w * 2 + side) * 4,
                    flags + LBM_CHK(grow_w + wrapx(side == 0 ? x0 - 4 : x0 + 4 * nv), N - 3));
        }
      } else {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int q = tid + i * VW * VH;
          if (q < nnode) {
            int gx, gy;
            if (q < 2 * RJ) {
              const int r = q / RJ, c = q - r * RJ;
              if (c >= rj) continue;
              gy = wrapy(r == 0 ? y0 - 1 : y0 + VH);
              gx = wrapx(x0 - 1 + c);
            } else {
              const int qq = q - 2 * RJ;
              gy = wrapy(y0 + (qq >> 1));
              gx = wrapx((qq & 1) == 0 ? x0 - 1 : x0 + V * nv);
            }
            qfl[i] = flags[LBM_CHK(gy * nx + gx, N)];
          }
        }
      }
    }
  };

  // ---- own populations and flags ----
  auto load_own = [&] {
    load_flags<V>(flags, LBM_CHK(n, N - V + 1), fl);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      C t[V];
      VT::load(fa, a, N, n, t);
#pragma unroll
      for (int q = 0; q < NP; ++q) f[q][a] = pack<L>(t[W * q], t[W * q + W - 1]);
    }
  };

  // ---- ring rows by tensor copies (one thread).  Only thread 0 touches ring_bar before the
  // CTA barrier that follows the staging, so its initialisation needs no barrier of its own.
  auto issue_ring_copies = [&] {
    if constexpr (TR && PSI) {
      if (tma_rows) {  // uniform over the CTA
        if (tid == 0) {
          tma::mbar_init(&ring_bar, 1);
          tma::fence_mbar_init();
          if constexpr (sizeof(S) == 2) {
            tma::mbar_expect_tx(&ring_bar, 2u * (SW * 4u + 8u * VT::kTmaWidth * 2u));
            for (int r = 0; r < 2; ++r) {
              const int yr = wrapy(r == 0 ? y0 - 1 : y0 + VH);
              tma::tma_load_2d(ring_st + r * RS, &rmap, &ring_bar, x0 - V, yr);
              tma::tma_load_3d(ring_st + r * RS + VT::kMovOff, &rmap2, &ring_bar,
                               x0 - VT::kTmaLeft, yr, 0);
            }
          } else {
            tma::mbar_expect_tx(&ring_bar, 2u * 9u * SW * ES);
            tma::tma_load_3d(ring_st, &rmap, &ring_bar, x0 - V, wrapy(y0 - 1), 0);
            tma::tma_load_3d(ring_st + RS, &rmap, &ring_bar, x0 - V, wrapy(y0 + VH), 0);
          }
        }
      }
    }
  };

  // The order in which a CTA issues these loads changes the step time: FP32 runs fastest with
  // its own populations first, the FP16 format with the staged copies first (measured at
  // 4096^2: FP32 208 us own-first against 217-221 us staged-first; FP16 186-187 us against
  // 198-206 us).
  if constexpr (VT::kOwnFirst) {
    load_own();
    stage_copies();
    issue_ring_copies();
  } else {
    stage_copies();
    issue_ring_copies();
    load_own();
  }

  L rho[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const L r = density_of<DEV>(rho_ref, f[q]);
    C re[W];
#pragma unroll
    for (int e = 0; e < W; ++e) re[e] = (fl[W * q + e] & FLAG_SOLID) ? C(1) : el(r, e);
    rho[q] = pack<L>(re[0], re[W - 1]);
    if constexpr (PSI) {
      const L ps = psi_of<C, EOS>(k, rho[q]);
#pragma unroll
      for (int e = 0; e < W; ++e)
        if (lane_ok)
          psi_s[w + 1][LBM_CHK(pj(V * (lane + 1) + W * q + e), SWP)] =
              (fl[W * q + e] & FLAG_SOLID) ? psi_w : el(ps, e);
    }
  }
  if constexpr (PSI) {
    cp_async_wait_all();
    __syncthreads();  // staged populations visible
    if constexpr (TR) {
      // every thread observes the tensor copies' completion (which makes their data visible
      // to it); a wait that expires is reported, and waited out once more with a short bound
      if (tma_rows && !tma::mbar_wait_bounded(&ring_bar, 0)) {
        if (tid == 0) atomicOr(err, kErrTimeout);
        tma::mbar_wait_bounded(&ring_bar, 0, 100000000ull);
      }
    }
    // psi of the ring and side nodes from the staged populations
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int q = tid + i * VW * VH;
      if (q < nnode) {
        const unsigned char* base;
        int j, prow, pcol;
        if (q < 2 * RJ) {
          const int r = q / RJ, c = q - r * RJ;
          if (c >= rj) continue;
          j = V - 1 + c;  // x0 - V + j; staged ring slots hold the same columns
          base = ring_st + r * RS;
          prow = r == 0 ? 0 : VH + 1;
          pcol = j;
        } else {
          const int qq = q - 2 * RJ, row = qq >> 1, side = qq & 1;
          j = side == 0 ? V - 1 : 0;  // element of the side vector
          base = side_st + (row * 2 + side) * 9 * V * ES;
          prow = row + 1;
          pcol = side == 0 ? V - 1 : V * (nv + 1);
        }
        const bool ringq = q < 2 * RJ;
        C g[9];
#pragma unroll
        for (int a = 0; a < 9; ++a)
          g[a] = VT::staged(base + (ringq ? VT::template ring_off<TR>(a) : a * V * ES), a, j);
        uint8_t nf = qfl[i];
        if constexpr (SFL) {
          if (q < 2 * RJ)
            nf = ring_fl[(q >= RJ ? SW : 0) + j];
          else
            nf = side_fl[((q - 2 * RJ) >> 1) * 8 + (((q - 2 * RJ) & 1) ? 4 : 0) + j];
        }
        psi_s[LBM_CHK(prow, VH + 2)][LBM_CHK(pj(pcol), SWP)] = (nf & FLAG_SOLID)
                                ? psi_w
                                : psi_of<C, EOS>(k, density_of<DEV>(rho_ref, g));
      }
    }
    __syncthreads();  // psi_s complete
  }

  if (y >= ny) return;  // a wrapped row of a ragged tile: psi only

  // ---- collisions of the own nodes ----
  // psi row segment of this lane's node v and its x-neighbours: pj(V (lane + 1) + v + dx)
  const int pbase = (V + 1) * (lane + 1);
  auto pcol = [](int v, int dx) {  // offset from pbase (compile-time for unrolled v, dx)
    const int j = v + dx;          // -1 .. V
    return j < 0 ? -2 : (j < V ? j : V + 1);
  };
  // psi values of lane value q (nodes W q .. W q + W - 1) at x-offset dx in row rr
  auto psi_at = [&](const C* rr, int q, int dx) {
    return pack<L>(rr[pcol(W * q, dx)], rr[pcol(W * q + W - 1, dx)]);
  };
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    L d13, d24, d57, d86, psic;
    if constexpr (PSI) {
      const C* rm = &psi_s[w][pbase];
      const C* r0 = &psi_s[w + 1][pbase];
      const C* rp = &psi_s[w + 2][pbase];
      d13 = r_sub(psi_at(r0, q, 1), psi_at(r0, q, -1));
      d24 = r_sub(psi_at(rp, q, 0), psi_at(rm, q, 0));
      d57 = r_sub(psi_at(rp, q, 1), psi_at(rm, q, -1));
      d86 = r_sub(psi_at(rm, q, 1), psi_at(rp, q, -1));
      psic = psi_at(r0, q, 0);
    } else {
      d13 = d24 = d57 = d86 = psic = splat<L>(C(0));
    }
    const int x = x0 + V * lane + W * q;
    L st[9], ux, uy;
    collide_node<S, EOS, L>(p, k, f[q], rho[q], d13, d24, d57, d86, psic,
                            pack<L>(C(x), C(x + W - 1)), splat<L>(C(yo)), st, ux, uy);
#pragma unroll
    for (int e = 0; e < W; ++e) {
      const int nn = yo * nx + x + e;  // used by lanes inside the lattice only
      const uint8_t fe = fl[W * q + e];
      if constexpr (FIELDS) {
        if (lane_ok) {
          const double nan = __longlong_as_double(0x7ff8000000000000LL);
          const bool solid = fe & FLAG_SOLID;
          rho_m[LBM_CHK(nn, N)] = solid ? nan : double(el(rho[q], e));
          ux_m[LBM_CHK(nn, N)] = solid ? nan : double(el(ux, e));
          uy_m[LBM_CHK(nn, N)] = solid ? nan : double(el(uy, e));
        }
      } else if (lane_ok && (fe & FLAG_MACRO)) {  // for the wall pass (fluid nodes only)
        if constexpr (DEV) {
          reinterpret_cast<float*>(rho_m)[LBM_CHK(nn, N)] = el(rho[q], e);
          reinterpret_cast<float*>(ux_m)[LBM_CHK(nn, N)] = el(ux, e);
          reinterpret_cast<float*>(uy_m)[LBM_CHK(nn, N)] = el(uy, e);
        } else {
          rho_m[LBM_CHK(nn, N)] = el(rho[q], e);
          ux_m[LBM_CHK(nn, N)] = el(ux, e);
          uy_m[LBM_CHK(nn, N)] = el(uy, e);
        }
      }
    }
    // (a solid node's values go to slots nothing reads or the wall pass overwrites)
    if constexpr (!FIELDS) {
#pragma unroll
      for (int a = 0; a < 9; ++a) f[q][a] = st[a];
    }
  }
  if constexpr (FIELDS) return;

  // ---- push: lanes write the vectors of their own columns of row y + e_a,y; at the tile's
  // edges (x0, x0 + V nv - 1 receive from the neighbouring tiles) partial vectors, and the
  // populations that leave the tile in x as single elements into the neighbours' columns ----
  const int rowp = wrapy(yo + 1) * nx, rowm = wrapy(yo - 1) * nx, row0 = yo * nx;
  const int col = x0 + V * (lane_ok ? lane : 0);
  const int col_l = wrapx(x0 - 1), col_r = wrapx(x0 + V * nv);
  const bool first = lane == 0, last = lane == nv - 1;
  auto fv = [&](int v, int a) { return el(f[v / W][a], v % W); };  // node v's value, plane a
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const int d = (ey(a) > 0 ? rowp : (ey(a) < 0 ? rowm : row0));
    C out[V];
    if (ex(a) == 0) {
#pragma unroll
      for (int v = 0; v < V; ++v) out[v] = fv(v, a);
      if (lane_ok) VT::store(fb, a, N, d + col, out);
    } else if (ex(a) > 0) {
      out[0] = __shfl_up_sync(0xffffffffu, fv(V - 1, a), 1);
#pragma unroll
      for (int v = 1; v < V; ++v) out[v] = fv(v - 1, a);
      if (lane_ok && !first) VT::store(fb, a, N, d + col, out);
      if (first) {  // elements 1 .. V - 1
        if constexpr (V == 4) {
          VT::store1(fb, a, N, d + col + 1, out[1]);
          VT::store2(fb, a, N, d + col + 2, out[2], out[3]);
        } else {
          VT::store1(fb, a, N, d + col + 1, out[1]);
        }
      }
      if (last) VT::store1(fb, a, N, d + col_r, fv(V - 1, a));
    } else {
      out[V - 1] = __shfl_down_sync(0xffffffffu, fv(0, a), 1);
#pragma unroll
      for (int v = 0; v < V - 1; ++v) out[v] = fv(v + 1, a);
      if (lane_ok && !last) VT::store(fb, a, N, d + col, out);
      if (last) {  // elements 0 .. V - 2
        if constexpr (V == 4) {
          VT::store2(fb, a, N, d + col, out[0], out[1]);
          VT::store1(fb, a, N, d + col + 2, out[2]);
        } else {
          VT::store1(fb, a, N, d + col, out[0]);
        }
      }
      if (first) VT::store1(fb, a, N, d + col_l, fv(0, a));
    }
  }
}

template <typename S, int EOS>
cudaError_t launch_vec_t(const DevParams& p, const void* fa, void* fb, const uint8_t* flags,
                         double* rho_m, double* ux_m, double* uy_m, bool fields_only,
                         cudaStream_t s, bool tma_ring, int* err) {
  constexpr int TW = VW * Vec<S>::V, VH = Vec<S>::VH;
  dim3 block(VW, VH);
  dim3 grid((p.nx + TW - 1) / TW, (p.ny + VH - 1) / VH);
  // ring-row and tile-prefetch maps; unused by the kernels without tensor copies
  CUtensorMap map{}, map2{}, pmap{}, pmap2{}, fmap{};
  int pf_flags = 0;  // fmap valid (row pitch of the flags a multiple of 16 bytes)
  if constexpr (!std::is_same<S, double>::value && EOS != LBM_EOS_NONE) {
    constexpr bool fp16 = std::is_same<S, __half>::value;
    bool maps = tma_ring && !fields_only && err;
    if (maps) {
      if constexpr (fp16)
        maps = make_ring_tensor_maps_fp16(&map, &map2, fa, p.nx, p.ny, Vec<S>::SWE,
                                          Vec<S>::kTmaWidth);
      else
        maps = make_ring_tensor_map(&map, fa, p.nx, p.ny, Vec<S>::kTmaWidth);
      if (Vec<S>::kPrefetchPops)
        maps = maps && make_tile_prefetch_maps(&pmap, &pmap2, fa, p.nx, p.ny, TW, VH, fp16);
      if (maps && Vec<S>::kPrefetchFlags)
        pf_flags = make_flags_prefetch_map(&fmap, flags, p.nx, p.ny, TW, VH) ? 1 : 0;
    }
    if (maps) {
      step_vec_kernel<S, EOS, false, true><<<grid, block, 0, s>>>(
          p, fa, fb, flags, rho_m, ux_m, uy_m, map, map2, pmap, pmap2, fmap, pf_flags, err);
      return cudaGetLastError();
    }
  }
  if (fields_only)
    step_vec_kernel<S, EOS, true, false><<<grid, block, 0, s>>>(
        p, fa, fb, flags, rho_m, ux_m, uy_m, map, map2, pmap, pmap2, fmap, 0, err);
  else
    step_vec_kernel<S, EOS, false, false><<<grid, block, 0, s>>>(
        p, fa, fb, flags, rho_m, ux_m, uy_m, map, map2, pmap, pmap2, fmap, 0, err);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_vec_s(const DevParams& p, const void* fa, void* fb, const uint8_t* flags,
                         double* rho_m, double* ux_m, double* uy_m, bool fields_only,
                         cudaStream_t s, bool tma_ring, int* err) {
  switch (p.eos) {
    case LBM_EOS_EXP:
      return launch_vec_t<S, LBM_EOS_EXP>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s,
                                          tma_ring, err);
    case LBM_EOS_CS:
      return launch_vec_t<S, LBM_EOS_CS>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s,
                                         tma_ring, err);
    default:
      return launch_vec_t<S, LBM_EOS_NONE>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s,
                                           tma_ring, err);
  }
}

}  // namespace

int step_vec_width(int precision) { return precision == LBM_FP64 ? 2 : 4; }

bool step_vec_supported(int precision, int nx, int ny) {
  const int vh = precision == LBM_FP16_DEV   ? Vec<__half>::VH
                 : precision == LBM_FP32_DEV ? Vec<float>::VH
                                             : Vec<double>::VH;
  return nx % step_vec_width(precision) == 0 && ny >= vh;
}

cudaError_t launch_step_vec(int precision, const DevParams& p, const void* fa, void* fb,
                            const uint8_t* flags, double* rho_m, double* ux_m, double* uy_m,
                            bool fields_only, cudaStream_t s, bool tma_ring, int* err) {
  if (precision == LBM_FP32_DEV)
    return launch_vec_s<float>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s, tma_ring,
                               err);
  if (precision == LBM_FP16_DEV)
    return launch_vec_s<__half>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s, tma_ring,
                                err);
  return launch_vec_s<double>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s, false, err);
}

}  // namespace lbm
