// Shared tile arithmetic of the step kernels (csrc/step.cu, csrc/step_tma.cu).
#pragma once
#include "d2q9.cuh"

namespace lbm {
namespace step_core {


constexpr int TX = 32;   // threads (and nodes) of a tile in x
constexpr int TYT = 8;   // threads of a tile in y; each handles RY rows, TYT apart

template <typename S>
struct StoreTraits {
  using C = typename Pop<S>::C;  // compute type
  static constexpr bool deviation = Pop<S>::dev;  // stores f_a - w_a rho_ref
  static constexpr int RY = sizeof(C) == 8 ? 2 : 4;  // rows per thread (register budget)
};

// Sum of the nine stored values in direction order (a node's density, less rho_ref for the
// deviation format).  Own nodes and ring nodes use the same arithmetic, so every CTA that needs
// psi of a node computes the same value.
template <typename C>
__device__ __forceinline__ C pop_sum(const C (&f)[9]) {
  C r = f[0];
#pragma unroll
  for (int a = 1; a < 9; ++a) r += f[a];
  return r;
}

// Phase 2 of a tile: force (Eq. 16 from psi_s), velocity (Eq. 5), collision (Eq. 2) and push
// (Eq. 3) of the RY nodes (x0 + tx, y0 + ty + TYN r) of this thread (TYN threads in y), given their populations f,
// densities rho and flags fl; psi of the tile and its ring is in psi_s (complete: the caller
// has synchronised the CTA).
template <typename S, int EOS, bool FIELDS, int RY, int TYN = TYT>
__device__ __forceinline__ void tile_phase2(const DevParams& p, void* __restrict__ fb,
                                            double* __restrict__ rho_m,
                                            double* __restrict__ ux_m,
                                            double* __restrict__ uy_m, int x0, int y0,
                                            const typename Pop<S>::C (*psi_s)[TX + 2],
                                            typename Pop<S>::C (&f)[RY][9],
                                            const typename Pop<S>::C (&rho)[RY],
                                            const uint8_t (&fl)[RY]) {
  using C = typename StoreTraits<S>::C;
  constexpr bool DEV = StoreTraits<S>::deviation;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int nx = p.nx, ny = p.ny;
  const int N = p.N;
  const Consts<C>& k = p.k<C>();
  const C rho_ref = DEV ? k.rho_ref : C(0);
  const int x = x0 + tx;
  const C omega = k.omega, one_m_omega = k.one_m_omega;
  const C K = k.K;  // 3 (1 - 1/(2 tau)): Guo prefactor times 1/c_s^2
  const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int y = y0 + ty + r * TYN;
    if (x >= nx || y >= ny) continue;
    const int n = y * nx + x;
    if (fl[r] & FLAG_SOLID) {
      if constexpr (FIELDS) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        rho_m[n] = nan;
        ux_m[n] = nan;
        uy_m[n] = nan;
      }
      continue;
    }
    const C rh = rho[r];
    // Total force: Eq. (16) plus body forces.
    C Fx = C(0), Fy = C(0);
    if constexpr (EOS != LBM_EOS_NONE) {
      const int cx = tx + 1, cy = ty + r * TYN + 1;
      // sum_a w_a psi(x + e_a) e_a as weighted differences of opposite neighbours: the
      // subtractions of nearly equal psi are exact, which keeps FP32 forces accurate in smooth
      // regions
      const C d13 = psi_s[cy][cx + 1] - psi_s[cy][cx - 1];
      const C d24 = psi_s[cy + 1][cx] - psi_s[cy - 1][cx];
      const C d57 = psi_s[cy + 1][cx + 1] - psi_s[cy - 1][cx - 1];
      const C d86 = psi_s[cy - 1][cx + 1] - psi_s[cy + 1][cx - 1];
      const C sx = wpsi<C>(1) * d13 + wpsi<C>(5) * (d57 + d86);
      const C sy = wpsi<C>(2) * d24 + wpsi<C>(5) * (d57 - d86);
      const C mg = -k.G * psi_s[cy][cx];
      Fx = mg * sx;
      Fy = mg * sy;
    }
    if (p.has_body) {
      Fx += rh * k.gx;
      Fy += rh * k.gy;
      if (k.azC != C(0)) {
        const C dx = C(x) - k.azcx, dy = C(y) - k.azcy;
        const C r2 = dx * dx + dy * dy;
        Fx += k.azC * (-dy) / r2;
        Fy += k.azC * dx / r2;
      }
    }
    const C(&g)[9] = f[r];
    // Velocity with the half-force term, Eq. (5).
    const C mx = ((g[1] - g[3]) + (g[5] - g[7])) + (g[8] - g[6]);
    const C my = ((g[2] - g[4]) + (g[5] - g[7])) + (g[6] - g[8]);
    const C inv_rho = q_rcp(rh);
    const C ux = (mx + C(0.5) * Fx) * inv_rho;
    const C uy = (my + C(0.5) * Fy) * inv_rho;
    if constexpr (FIELDS) {
      rho_m[n] = double(rh);
      ux_m[n] = double(ux);
      uy_m[n] = double(uy);
      continue;
    } else {
      if (fl[r] & FLAG_MACRO) {  // for the wall pass, in its arithmetic type
        if constexpr (DEV) {
          reinterpret_cast<float*>(rho_m)[n] = rh;
          reinterpret_cast<float*>(ux_m)[n] = ux;
          reinterpret_cast<float*>(uy_m)[n] = uy;
        } else {
          rho_m[n] = rh;
          ux_m[n] = ux;
          uy_m[n] = uy;
        }
      }
      // Collision, Eq. (2): f* = (1 - omega) f + omega f_eq + F_a, with f_eq of Eq. (4),
      //   f_eq = w [c0 + rho eu (3 + 4.5 eu)],  c0 = rho (1 - 1.5 u.u) (less rho_ref if stored
      //   as a deviation), and Guo's term F_a = w [K eF (1 + 3 eu) - K u.F], K = 3 (1 - 1/2tau),
      //   eu = e_a.u, eF = e_a.F.
      const C uu = ux * ux + uy * uy;
      const C c0 = (rh - rho_ref) - C(1.5) * rh * uu;
      const C uF = ux * Fx + uy * Fy;
      const C A0 = omega * c0 - K * uF;
      const C orho = omega * rh;
      // Opposite directions a, abar share |e.u| and |e.F|: h_a = P + Q, h_abar = P - Q with the
      // even part P = A0 + 4.5 rho omega eu^2 + 3 K eF eu and the odd part
      // Q = 3 rho omega eu + K eF.
      C out[9];
      out[0] = one_m_omega * g[0] + wgt<C>(0) * A0;
      const C o45 = C(4.5) * orho, o3 = C(3) * orho, K3 = C(3) * K;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int a = i == 0 ? 1 : (i == 1 ? 2 : (i == 2 ? 5 : 6)), ab = opposite(a);
        const C eu = (ex(a) ? C(ex(a)) * ux : C(0)) + (ey(a) ? C(ey(a)) * uy : C(0));
        const C eF = (ex(a) ? C(ex(a)) * Fx : C(0)) + (ey(a) ? C(ey(a)) * Fy : C(0));
        const C P = A0 + (o45 * eu + K3 * eF) * eu;
        const C Q = o3 * eu + K * eF;
        const C w = wgt<C>(a);
        out[a] = one_m_omega * g[a] + w * (P + Q);
        out[ab] = one_m_omega * g[ab] + w * (P - Q);
      }
      C st[9];  // the values as stored (rounded to the storage format)
#pragma unroll
      for (int a = 0; a < 9; ++a) st[a] = Pop<S>::rounded(a, out[a]);
      if constexpr (DEV) {
        // The collision conserves mass exactly (sum of f_eq is rho, sum of the Guo term is 0),
        // but rounding the nine FP32 results does not, and near a steady state the rounding
        // repeats every step, so mass would drift linearly.  The rest population therefore
        // takes the node's stored mass minus the eight rounded moving populations, written as
        // g_0 + sum_a (g_a - g*_a) so that only small differences are added.
        C d = C(0);
#pragma unroll
        for (int a = 1; a < 9; ++a) d += g[a] - st[a];
        st[0] = g[0] + d;
      }
      const int row = y * nx;
      const int rowp = (y + 1 == ny ? 0 : y + 1) * nx, rowm = (y == 0 ? ny - 1 : y - 1) * nx;
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        const int dxn = ex(a) > 0 ? xp : (ex(a) < 0 ? xm : x);
        const int drow = ey(a) > 0 ? rowp : (ey(a) < 0 ? rowm : row);
        Pop<S>::store(fb, a, N, drow + dxn, st[a]);
      }
    }
  }
}


// One tile (x0, y0) of one lattice: every thread of the CTA calls it with the same arguments.
// psi_s: shared memory of (TYT RY + 2) x (TX + 2) values.
template <typename S, int EOS, bool FIELDS, int RY>
__device__ __forceinline__ void step_tile(const DevParams& p, const void* __restrict__ fa,
                                          void* __restrict__ fb,
                                          const uint8_t* __restrict__ flags,
                                          double* __restrict__ rho_m, double* __restrict__ ux_m,
                                          double* __restrict__ uy_m, int x0, int y0,
                                          typename Pop<S>::C (*psi_s)[TX + 2]) {
  using C = typename StoreTraits<S>::C;
  constexpr bool DEV = StoreTraits<S>::deviation;
  constexpr int TH = TYT * RY;  // tile height in nodes

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int nx = p.nx, ny = p.ny;
  const int N = p.N;  // 9 N < 2^31 (checked at creation): 32-bit element offsets
  // ragged tiles of lattices narrower than a tile wrap more than once
  const bool small = nx <= TX + 1 || ny <= TH + 1;
  const Consts<C>& k = p.k<C>();
  const C rho_ref = DEV ? k.rho_ref : C(0);
  const C psi_w = k.psi_wall;

  // ---- phase 1: own nodes' populations, density and psi; psi of the ring ----
  const int x = x0 + tx;
  const int xo = x < nx ? x : (small ? wrap_any(x, nx) : x - nx);
  C f[RY][9];
  C rho[RY];
  uint8_t fl[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int y = y0 + ty + r * TYT;
    const int yo = y < ny ? y : (small ? wrap_any(y, ny) : y - ny);
    const int n = yo * nx + xo;
    fl[r] = flags[n];
    rho[r] = C(1);
    if (!(fl[r] & FLAG_SOLID)) {
#pragma unroll
      for (int a = 0; a < 9; ++a) f[r][a] = Pop<S>::load(fa, a, N, n);
    } else {
#pragma unroll
      for (int a = 0; a < 9; ++a) f[r][a] = C(0);
    }
  }
  if constexpr (EOS != LBM_EOS_NONE) {
    // One-node ring around the tile, 2 (TX + 2) + 2 TH cells, one per thread of the first
    // kRing threads.  Its loads are issued before any own node's psi is computed, so a CTA
    // waits for memory once.
    constexpr int kRing = 2 * (TX + 2) + 2 * TH;
    static_assert(kRing <= TX * TYT, "one ring cell per thread");
    const int c = ty * TX + tx;
    int hx = 0, hy = 0;
    bool ring_fluid = false;
    C v[9];
    if (c < kRing) {
      if (c < 2 * (TX + 2)) {
        hx = c < TX + 2 ? c : c - (TX + 2);
        hy = c < TX + 2 ? 0 : TH + 1;
      } else {
        const int kk = c - 2 * (TX + 2);
        hx = kk < TH ? 0 : TX + 1;
        hy = (kk < TH ? kk : kk - TH) + 1;
      }
      int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
      if (small) {
        gx = wrap_any(gx, nx);
        gy = wrap_any(gy, ny);
      } else {
        gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
        gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
      }
      const int m = gy * nx + gx;
      ring_fluid = !(flags[m] & FLAG_SOLID);
      if (ring_fluid) {
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = Pop<S>::load(fa, a, N, m);
      }
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      if (!(fl[r] & FLAG_SOLID)) rho[r] = rho_ref + pop_sum<C>(f[r]);
      psi_s[ty + r * TYT + 1][tx + 1] = (fl[r] & FLAG_SOLID) ? psi_w : psi_of<C, EOS>(k, rho[r]);
    }
    if (c < kRing) psi_s[hy][hx] = ring_fluid ? psi_of<C, EOS>(k, rho_ref + pop_sum<C>(v)) : psi_w;
    __syncthreads();
  } else {
#pragma unroll
    for (int r = 0; r < RY; ++r)
      if (!(fl[r] & FLAG_SOLID)) rho[r] = rho_ref + pop_sum<C>(f[r]);
  }

  tile_phase2<S, EOS, FIELDS, RY>(p, fb, rho_m, ux_m, uy_m, x0, y0, psi_s, f, rho, fl);
}

}  // namespace step_core
}  // namespace lbm
