// Solid flags and the boundary-link list with the wall fraction q of Eq. (6), built on the GPU.
//
// The list is in canonical order (node index ascending, then direction ascending) and is built by
// a count / scan / emit pass over blocks of 4096 consecutive nodes.  q is evaluated in FP64 with
// explicit round-to-nearest operations (no contraction into fused multiply-adds), so it is the
// correctly rounded result of the stated sequence of operations on any IEEE machine.
#include "d2q9.cuh"

namespace lbm {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;  // consecutive nodes per thread
constexpr int kNodesPerBlock = kThreads * kItems;

__device__ bool circle_solid(const GeomCircle& c, int i, int j) {
  double dx = __dsub_rn((double)i, c.cx);
  double dy = __dsub_rn((double)j, c.cy);
  double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  double r2 = __dmul_rn(c.r, c.r);
  return c.outside ? (d2 >= r2) : (d2 <= r2);
}

__device__ bool node_solid(const GeomParams& g, int i, int j) {
  if (g.wall_q_lo > 0.0 && j == 0) return true;
  if (g.wall_q_hi > 0.0 && j == g.ny - 1) return true;
  for (int k = 0; k < g.n_circles; ++k)
    if (circle_solid(g.c[k], i, j)) return true;
  return false;
}

// Root t of |x_b + t e - c| = r: a t^2 + 2 bq t + cq = 0, a = e.e, bq = e.d, cq = d.d - r^2,
// d = x_b - c; the smaller root enters a solid disc, the larger leaves a fluid disc.
__device__ double circle_q(const GeomCircle& c, int i, int j, int a) {
  double dx = __dsub_rn((double)i, c.cx);
  double dy = __dsub_rn((double)j, c.cy);
  double exd = (double)ex(a), eyd = (double)ey(a);
  double aa = __dadd_rn(__dmul_rn(exd, exd), __dmul_rn(eyd, eyd));
  double bq = __dadd_rn(__dmul_rn(exd, dx), __dmul_rn(eyd, dy));
  double cq = __dsub_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(c.r, c.r));
  double disc = __dsub_rn(__dmul_rn(bq, bq), __dmul_rn(aa, cq));
  if (disc < 0.0) disc = 0.0;
  double sq = __dsqrt_rn(disc);
  double t = c.outside ? __ddiv_rn(__dadd_rn(-bq, sq), aa) : __ddiv_rn(__dsub_rn(-bq, sq), aa);
  if (t > 1.0) t = 1.0;
  return t;
}

__device__ double link_q(const GeomParams& g, int i, int j, int a) {
  int si = wrap_once(i + ex(a), g.nx), sj = wrap_once(j + ey(a), g.ny);
  double q = 2.0;
  if (g.wall_q_lo > 0.0 && sj == 0 && g.wall_q_lo < q) q = g.wall_q_lo;
  if (g.wall_q_hi > 0.0 && sj == g.ny - 1 && g.wall_q_hi < q) q = g.wall_q_hi;
  for (int k = 0; k < g.n_circles; ++k)
    if (circle_solid(g.c[k], si, sj)) {
      double t = circle_q(g.c[k], i, j, a);
      if (t < q) q = t;
    }
  return q;
}

// Bitmask of directions a = 1..8 whose neighbour is solid (bit a), for a fluid node.
__device__ unsigned cut_mask(const GeomParams& g, const uint8_t* flags, int n) {
  if (flags[n] & FLAG_SOLID) return 0u;
  int i = n % g.nx, j = n / g.nx;
  unsigned m = 0u;
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    int s = wrap_once(j + ey(a), g.ny) * g.nx + wrap_once(i + ex(a), g.nx);
    if (flags[s] & FLAG_SOLID) m |= 1u << a;
  }
  return m;
}

__global__ void geom_solid_kernel(GeomParams g, uint8_t* flags) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < g.N; n += gridDim.x * blockDim.x)
    flags[n] = node_solid(g, n % g.nx, n / g.nx) ? FLAG_SOLID : 0;
}

// Inclusive block scan of int2 over kThreads threads (Hillis-Steele in shared memory).
__device__ int2 block_inclusive_scan(int2 v, int2* sh) {
  int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int off = 1; off < kThreads; off <<= 1) {
    int2 add = make_int2(0, 0);
    if (t >= off) add = sh[t - off];
    __syncthreads();
    v.x += add.x;
    v.y += add.y;
    sh[t] = v;
    __syncthreads();
  }
  return v;
}

__device__ int2 thread_counts(const GeomParams& g, const uint8_t* flags, int first) {
  int2 c = make_int2(0, 0);
  for (int k = 0; k < kItems; ++k) {
    int n = first + k;
    if (n >= g.N) break;
    unsigned m = cut_mask(g, flags, n);
    if (m) {
      c.x += 1;
      c.y += __popc(m);
    }
  }
  return c;
}

__global__ void geom_count_kernel(GeomParams g, const uint8_t* flags, int2* block_tot) {
  __shared__ int2 sh[kThreads];
  int first = blockIdx.x * kNodesPerBlock + threadIdx.x * kItems;
  int2 inc = block_inclusive_scan(thread_counts(g, flags, first), sh);
  if (threadIdx.x == kThreads - 1) block_tot[blockIdx.x] = inc;
}

// Exclusive scan of the per-block totals in place (one block), grand totals to totals[0..1].
__global__ void geom_scan_kernel(int2* block_tot, int nblocks, long long* totals) {
  __shared__ int2 sh[kThreads];
  int2 carry = make_int2(0, 0);
  for (int base = 0; base < nblocks; base += kThreads) {
    int k = base + threadIdx.x;
    int2 v = k < nblocks ? block_tot[k] : make_int2(0, 0);
    int2 inc = block_inclusive_scan(v, sh);
    if (k < nblocks) block_tot[k] = make_int2(carry.x + inc.x - v.x, carry.y + inc.y - v.y);
    __syncthreads();
    int2 last = sh[kThreads - 1];
    carry.x += last.x;
    carry.y += last.y;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    totals[0] = carry.x;
    totals[1] = carry.y;
  }
}

__device__ void flag_or(uint8_t* flags, int n, uint8_t bits) {
  unsigned* word = reinterpret_cast<unsigned*>(flags) + (n >> 2);
  atomicOr(word, (unsigned)bits << (8 * (n & 3)));
}

__global__ void geom_emit_kernel(GeomParams g, uint8_t* flags, const int2* block_off,
                                 int32_t* bnode, int32_t* boff, uint8_t* ldir, double* lq) {
  __shared__ int2 sh[kThreads];
  int first = blockIdx.x * kNodesPerBlock + threadIdx.x * kItems;
  int2 own = thread_counts(g, flags, first);
  int2 inc = block_inclusive_scan(own, sh);
  int bi = block_off[blockIdx.x].x + inc.x - own.x;
  int li = block_off[blockIdx.x].y + inc.y - own.y;
  for (int k = 0; k < kItems; ++k) {
    int n = first + k;
    if (n >= g.N) break;
    unsigned m = cut_mask(g, flags, n);
    if (!m) continue;
    int i = n % g.nx, j = n / g.nx;
    bnode[bi] = n;
    boff[bi] = li;
    ++bi;
    flag_or(flags, n, FLAG_BOUNDARY | FLAG_MACRO);
    for (int a = 1; a < 9; ++a) {
      if (!(m & (1u << a))) continue;
      ldir[li] = (uint8_t)a;
      lq[li] = link_q(g, i, j, a);
      ++li;
      // x_f = x_b - e_a: its velocity enters the Mei-Luo-Shyy branch q < 1/2 (Eq. 11)
      int nf = wrap_once(j - ey(a), g.ny) * g.nx + wrap_once(i - ex(a), g.nx);
      flag_or(flags, nf, FLAG_MACRO);
    }
  }
}

}  // namespace

int geom_num_blocks(int N) { return (N + kNodesPerBlock - 1) / kNodesPerBlock; }

cudaError_t launch_geom_solid(const GeomParams& g, uint8_t* flags, cudaStream_t s) {
  int blocks = (g.N + 255) / 256;
  if (blocks > 65535 * 16) blocks = 65535 * 16;
  geom_solid_kernel<<<blocks, 256, 0, s>>>(g, flags);
  return cudaGetLastError();
}

cudaError_t launch_geom_count_scan(const GeomParams& g, const uint8_t* flags, int2* block_tot,
                                   int nblocks, long long* totals, cudaStream_t s) {
  geom_count_kernel<<<nblocks, kThreads, 0, s>>>(g, flags, block_tot);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  geom_scan_kernel<<<1, kThreads, 0, s>>>(block_tot, nblocks, totals);
  return cudaGetLastError();
}

cudaError_t launch_geom_emit(const GeomParams& g, uint8_t* flags, const int2* block_off,
                             int32_t* bnode, int32_t* boff, uint8_t* ldir, double* lq,
                             cudaStream_t s) {
  geom_emit_kernel<<<geom_num_blocks(g.N), kThreads, 0, s>>>(g, flags, block_off, bnode, boff,
                                                              ldir, lq);
  return cudaGetLastError();
}

}  // namespace lbm
