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
  for (int a = 1; a < 9; ++a) r = r_add(r, f[a]);
  return r;
}

// A node's density from its nine stored values: their sum, plus rho_ref for the deviation
// formats (FP64 storage holds the populations themselves).
template <bool DEV, typename L>
__device__ __forceinline__ L density_of(typename Elem<L>::C rho_ref, const L (&f)[9]) {
  if constexpr (DEV)
    return r_add(splat<L>(rho_ref), pop_sum<L>(f));
  else
    return pop_sum<L>(f);
}

// A post-collision value rounded to the storage format of plane a (per element).  Node pairs of
// the FP16 format round both elements in one paired conversion each way (round to nearest even
// per element, the same values as one at a time).
template <typename S, typename L>
__device__ __forceinline__ L round_st(int a, L v) {
  if constexpr (Elem<L>::W == 2) {
    if constexpr (sizeof(S) == 2) {
      return a == 0 ? v : __half22float2(__float22half2_rn(v));
    } else {
      return make_float2(Pop<S>::rounded(a, v.x), Pop<S>::rounded(a, v.y));
    }
  } else {
    return Pop<S>::rounded(a, v);
  }
}

// The arithmetic of one fluid node (x, y), or of two nodes at once when L is float2 (the paired
// FP32 instructions; each element is rounded exactly as alone): total force (Eq. 16 plus body
// forces) from the psi differences of its opposite neighbours d13 = psi(x+1,y) - psi(x-1,y),
// d24 = psi(x,y+1) - psi(x,y-1), d57 = psi(x+1,y+1) - psi(x-1,y-1), d86 = psi(x+1,y-1) -
// psi(x-1,y+1) and its own psi; velocity with the half-force term (Eq. 5); BGK collision with
// Guo forcing (Eqs. 2, 4).  g: the node's nine stored values (deviations less w_a rho_ref for
// the deviation formats), rh: its density, xf, yf: its coordinates.  st: the nine post-collision
// values as they will be stored (rounded to the storage format).  Every operation is explicitly
// rounded, so all callers give the same bits.
template <typename S, int EOS, typename L>
__device__ __forceinline__ void collide_node(const DevParams& p,
                                             const Consts<typename Pop<S>::C>& k,
                                             const L (&g)[9], L rh, L d13, L d24, L d57, L d86,
                                             L psic, L xf, L yf, L (&st)[9], L& ux, L& uy) {
  using C = typename Pop<S>::C;
  constexpr bool DEV = Pop<S>::dev;
  auto c_ = [](C v) { return splat<L>(v); };
  L Fx = c_(C(0)), Fy = c_(C(0));
  if constexpr (EOS != LBM_EOS_NONE) {
    // -G psi(x) sum_a w_a psi(x + e_a) e_a, as weighted differences of opposite neighbours (the
    // subtractions of nearly equal psi are exact, which keeps FP32 forces accurate in smooth
    // regions).  FP64: -G folded into the weights (gw1 = -G/3, gw5 = -G/12), one operation less.
    if constexpr (sizeof(C) == 8) {
      const L sx = r_fma(c_(k.gw1), d13, r_mul(c_(k.gw5), r_add(d57, d86)));
      const L sy = r_fma(c_(k.gw1), d24, r_mul(c_(k.gw5), r_sub(d57, d86)));
      Fx = r_mul(psic, sx);
      Fy = r_mul(psic, sy);
    } else {
      const L sx = r_fma(c_(wpsi<C>(1)), d13, r_mul(c_(wpsi<C>(5)), r_add(d57, d86)));
      const L sy = r_fma(c_(wpsi<C>(2)), d24, r_mul(c_(wpsi<C>(5)), r_sub(d57, d86)));
      const L mg = r_mul(c_(-k.G), psic);
      Fx = r_mul(mg, sx);
      Fy = r_mul(mg, sy);
    }
  }
  if (p.has_body) {
    Fx = r_fma(rh, c_(k.gx), Fx);
    Fy = r_fma(rh, c_(k.gy), Fy);
    if (k.azC != C(0)) {
      const L dx = r_sub(xf, c_(k.azcx)), dy = r_sub(yf, c_(k.azcy));
      const L r2 = r_fma(dx, dx, r_mul(dy, dy));
      Fx = r_add(Fx, q_div(r_mul(c_(-k.azC), dy), r2));
      Fy = r_add(Fy, q_div(r_mul(c_(k.azC), dx), r2));
    }
  }
  // Velocity with the half-force term, Eq. (5).
  const L mx = r_add(r_add(r_sub(g[1], g[3]), r_sub(g[5], g[7])), r_sub(g[8], g[6]));
  const L my = r_add(r_add(r_sub(g[2], g[4]), r_sub(g[5], g[7])), r_sub(g[6], g[8]));
  const L inv_rho = q_rcp(rh);
  ux = r_mul(r_fma(c_(C(0.5)), Fx, mx), inv_rho);
  uy = r_mul(r_fma(c_(C(0.5)), Fy, my), inv_rho);
  // Collision, Eq. (2): f* = (1 - omega) f + omega f_eq + F_a, with f_eq of Eq. (4),
  //   f_eq = w [c0 + rho eu (3 + 4.5 eu)],  c0 = rho (1 - 1.5 u.u) (less rho_ref if stored
  //   as a deviation), and Guo's term F_a = w [K eF (1 + 3 eu) - K u.F], K = 3 (1 - 1/2tau),
  //   eu = e_a.u, eF = e_a.F.
  const L uu = r_fma(ux, ux, r_mul(uy, uy));
  L rd = rh;  // rho, less rho_ref for the deviation formats
  if constexpr (DEV) rd = r_sub(rh, c_(k.rho_ref));
  const L c0 = r_fma(r_mul(c_(C(-1.5)), rh), uu, rd);
  const L uF = r_fma(ux, Fx, r_mul(uy, Fy));
  const L A0 = r_fma(c_(k.omega), c0, r_mul(c_(-k.K), uF));
  const L one_m_omega = c_(k.one_m_omega);
  // Opposite directions a, abar share |e.u| and |e.F|: h_a = w (P + Q), h_abar = w (P - Q) with
  // the even part P = A0 + (4.5 rho omega eu + 3 K eF) eu and the odd part Q = 3 rho omega eu +
  // K eF.
  L out[9];
  out[0] = r_fma(one_m_omega, g[0], r_mul(c_(wgt<C>(0)), A0));
  if constexpr (sizeof(C) == 8) {
    // FP64 arithmetic is bound by the FP64 pipe: w is folded into coefficients per weight class
    // c (axis, diagonal), al = w 4.5 omega rho, be = w 3 omega rho, Aw = w A0 and the constants
    // w 3 K, w K, which saves two operations per direction pair.
    L al[2], be[2], Aw[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      al[c] = r_mul(c_(k.wo45[c]), rh);
      be[c] = r_mul(c_(k.wo3[c]), rh);
      Aw[c] = r_mul(c_(wgt<C>(c == 0 ? 1 : 5)), A0);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int a = i == 0 ? 1 : (i == 1 ? 2 : (i == 2 ? 5 : 6)), ab = opposite(a), c = i >> 1;
      // e_a = (1,0), (0,1), (1,1), (-1,1)
      const L eu = i == 0 ? ux : (i == 1 ? uy : (i == 2 ? r_add(ux, uy) : r_sub(uy, ux)));
      const L eF = i == 0 ? Fx : (i == 1 ? Fy : (i == 2 ? r_add(Fx, Fy) : r_sub(Fy, Fx)));
      const L wP = r_fma(r_fma(al[c], eu, r_mul(c_(k.wK3[c]), eF)), eu, Aw[c]);
      const L wQ = r_fma(be[c], eu, r_mul(c_(k.wK[c]), eF));
      out[a] = r_fma(one_m_omega, g[a], r_add(wP, wQ));
      out[ab] = r_fma(one_m_omega, g[ab], r_sub(wP, wQ));
    }
  } else {
    // FP32 arithmetic (issue- and register-bound kernels): fewer live values per node
    const L orho = r_mul(c_(k.omega), rh);
    const L o45 = r_mul(c_(C(4.5)), orho), o3 = r_mul(c_(C(3)), orho);
    const L K = c_(k.K), K3 = r_mul(c_(C(3)), K);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int a = i == 0 ? 1 : (i == 1 ? 2 : (i == 2 ? 5 : 6)), ab = opposite(a);
      const L eu = i == 0 ? ux : (i == 1 ? uy : (i == 2 ? r_add(ux, uy) : r_sub(uy, ux)));
      const L eF = i == 0 ? Fx : (i == 1 ? Fy : (i == 2 ? r_add(Fx, Fy) : r_sub(Fy, Fx)));
      const L P = r_fma(r_fma(o45, eu, r_mul(K3, eF)), eu, A0);
      const L Q = r_fma(o3, eu, r_mul(K, eF));
      const L w = c_(wgt<C>(a));
      out[a] = r_fma(one_m_omega, g[a], r_mul(w, r_add(P, Q)));
      out[ab] = r_fma(one_m_omega, g[ab], r_mul(w, r_sub(P, Q)));
    }
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) st[a] = round_st<S>(a, out[a]);
  if constexpr (DEV) {
    // The collision conserves mass exactly (sum of f_eq is rho, sum of the Guo term is 0), but
    // rounding the nine results does not, and near a steady state the rounding repeats every
    // step, so mass would drift linearly.  The rest population therefore takes the node's
    // stored mass minus the eight rounded moving populations, written as
    // g_0 + sum_a (g_a - g*_a) so that only small differences are added.
    L d = c_(C(0));
#pragma unroll
    for (int a = 1; a < 9; ++a) d = r_add(d, r_sub(g[a], st[a]));
    st[0] = r_add(g[0], d);
  }
}

// Phase 2 of a tile: the nodes (x0 + tx, y0 + ty + TYN r) of this thread (TYN threads in y),
// given their populations f, densities rho and flags fl; psi of the tile and its ring is in
// psi_s (complete: the caller has synchronised the CTA).  Writes the moments of FLAG_MACRO nodes
// for the wall pass (FIELDS: the moments of every node instead) and pushes (Eq. 3) the
// post-collision populations to x + e_a of fb.
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
  const int x = x0 + tx;
  const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int y = y0 + ty + r * TYN;
    if (x >= nx || y >= ny) continue;
    const int n = LBM_CHK(y * nx + x, N);
    if (fl[r] & FLAG_SOLID) {
      if constexpr (FIELDS) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        rho_m[n] = nan;
        ux_m[n] = nan;
        uy_m[n] = nan;
      }
      continue;
    }
    const int cx = tx + 1, cy = ty + r * TYN + 1;
    C d13 = C(0), d24 = C(0), d57 = C(0), d86 = C(0), psic = C(0);
    if constexpr (EOS != LBM_EOS_NONE) {
      d13 = r_sub(psi_s[cy][cx + 1], psi_s[cy][cx - 1]);
      d24 = r_sub(psi_s[cy + 1][cx], psi_s[cy - 1][cx]);
      d57 = r_sub(psi_s[cy + 1][cx + 1], psi_s[cy - 1][cx - 1]);
      d86 = r_sub(psi_s[cy - 1][cx + 1], psi_s[cy + 1][cx - 1]);
      psic = psi_s[cy][cx];
    }
    C st[9], ux, uy;
    collide_node<S, EOS>(p, k, f[r], rho[r], d13, d24, d57, d86, psic, C(x), C(y), st, ux, uy);
    if constexpr (FIELDS) {
      rho_m[n] = double(rho[r]);
      ux_m[n] = double(ux);
      uy_m[n] = double(uy);
    } else {
      if (fl[r] & FLAG_MACRO) {  // for the wall pass, in its arithmetic type
        if constexpr (DEV) {
          reinterpret_cast<float*>(rho_m)[n] = rho[r];
          reinterpret_cast<float*>(ux_m)[n] = ux;
          reinterpret_cast<float*>(uy_m)[n] = uy;
        } else {
          rho_m[n] = rho[r];
          ux_m[n] = ux;
          uy_m[n] = uy;
        }
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
  // In a ragged tile only the first column (row) past the lattice's edge is needed: it holds
  // column 0 (row 0), the periodic neighbour of the last one.  Slots beyond it load nothing.
  const int x = x0 + tx;
  const int xo = x < nx ? x : 0;
  C f[RY][9];
  C rho[RY];
  uint8_t fl[RY];
  auto load_own = [&] {
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const int y = y0 + ty + r * TYT;
      const int yo = y < ny ? y : 0;
      const int n = yo * nx + xo;
      fl[r] = (x <= nx && y <= ny) ? flags[LBM_CHK(n, N)] : uint8_t(FLAG_SOLID);
      rho[r] = C(1);
      if (!(fl[r] & FLAG_SOLID)) {
#pragma unroll
        for (int a = 0; a < 9; ++a) f[r][a] = Pop<S>::load(fa, a, N, n);
      } else {
#pragma unroll
        for (int a = 0; a < 9; ++a) f[r][a] = C(0);
      }
    }
  };
  if constexpr (EOS != LBM_EOS_NONE) {
    // One-node ring around the tile, 2 (TX + 2) + 2 TH cells, one per thread of the first
    // kRing threads.  Its loads are issued first, then the own nodes' (the batched FP16 step ran
    // 4.5% faster than with the own loads first), and no psi is computed before both are in
    // flight, so a CTA waits for memory once.
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
      const bool ring_need = gx <= nx && gy <= ny;  // past the first wrapped column: unused
      if (small) {
        gx = wrap_any(gx, nx);
        gy = wrap_any(gy, ny);
      } else {
        gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
        gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
      }
      const int m = gy * nx + gx;
      ring_fluid = ring_need && !(flags[LBM_CHK(m, N)] & FLAG_SOLID);
      if (ring_fluid) {
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = Pop<S>::load(fa, a, N, m);
      }
    }
    load_own();
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      if (!(fl[r] & FLAG_SOLID)) rho[r] = density_of<DEV>(rho_ref, f[r]);
      psi_s[ty + r * TYT + 1][tx + 1] = (fl[r] & FLAG_SOLID) ? psi_w : psi_of<C, EOS>(k, rho[r]);
    }
    if (c < kRing)
      psi_s[hy][hx] = ring_fluid ? psi_of<C, EOS>(k, density_of<DEV>(rho_ref, v)) : psi_w;
    __syncthreads();
  } else {
    load_own();
#pragma unroll
    for (int r = 0; r < RY; ++r)
      if (!(fl[r] & FLAG_SOLID)) rho[r] = density_of<DEV>(rho_ref, f[r]);
  }

  tile_phase2<S, EOS, FIELDS, RY>(p, fb, rho_m, ux_m, uy_m, x0, y0, psi_s, f, rho, fl);
}

}  // namespace step_core
}  // namespace lbm
