// The fused per-node pass of one time step (Sec. 2.1, Sec. 3.2):
//   density and velocity (Eq. 5), pseudopotential force (Eq. 16) from psi of the 8 neighbours,
//   BGK collision with Guo forcing (Eqs. 2, 4), streaming (Eq. 3).
//
// Layout: two lattices of 9 planes [a][j][i] (structure of arrays).  The source lattice holds
// f(x, t) at x; each fluid node writes f*_a(x, t) to x + e_a of the destination lattice (push),
// including into solid nodes, whose slots then hold the outgoing populations the boundary pass
// reads.  Every population is read once and written once per step.
//
// A CTA covers a TX x TY tile.  Each thread keeps its node's 9 populations in registers; psi of
// the tile and of a one-node ring around it goes to shared memory (ring nodes recompute their
// density from their own 9 populations), so the force needs no second pass over memory.
#include "d2q9.cuh"

namespace lbm {

namespace {

constexpr int TX = 32;
constexpr int TY = 8;

template <typename S>
struct StoreTraits;
template <>
struct StoreTraits<double> {
  using C = double;  // compute type
  static constexpr bool deviation = false;
};
template <>
struct StoreTraits<float> {
  using C = float;
  static constexpr bool deviation = true;  // stores f_a - w_a rho_ref
};

// Density of the node at linear index m from its nine stored values (deviation-aware).
template <typename S>
__device__ __forceinline__ typename StoreTraits<S>::C node_rho(const S* __restrict__ f, size_t N,
                                                              int m, typename StoreTraits<S>::C rho_ref) {
  using C = typename StoreTraits<S>::C;
  C r = C(f[m]);
#pragma unroll
  for (int a = 1; a < 9; ++a) r += C(f[a * N + m]);
  if constexpr (StoreTraits<S>::deviation) r += rho_ref;
  return r;
}

template <typename S, int EOS, bool FIELDS>
__global__ void __launch_bounds__(TX* TY) step_kernel(DevParams p, const S* __restrict__ fa,
                                                      S* __restrict__ fb,
                                                      const uint8_t* __restrict__ flags,
                                                      double* __restrict__ rho_m,
                                                      double* __restrict__ ux_m,
                                                      double* __restrict__ uy_m) {
  using C = typename StoreTraits<S>::C;
  constexpr bool DEV = StoreTraits<S>::deviation;
  __shared__ C psi_s[TY + 2][TX + 2];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int x = x0 + tx, y = y0 + ty;
  const int nx = p.nx, ny = p.ny;
  const size_t N = (size_t)p.N;
  const bool inside = (x < nx) && (y < ny);
  const C rho_ref = DEV ? C(p.rho_ref) : C(0);
  const C psi_w = C(p.psi_wall);

  // Own node (out-of-range threads of a ragged tile stand in for the wrapped node).
  const int xo = inside ? x : wrap_any(x, nx);
  const int yo = inside ? y : wrap_any(y, ny);
  const int n = yo * nx + xo;
  const uint8_t fl = flags[n];
  const bool solid = fl & FLAG_SOLID;
  C f[9];
  C rho = C(1);
  if (!solid) {
#pragma unroll
    for (int a = 0; a < 9; ++a) f[a] = C(fa[a * N + n]);
    rho = f[0];
#pragma unroll
    for (int a = 1; a < 9; ++a) rho += f[a];
    if constexpr (DEV) rho += rho_ref;
  }
  if constexpr (EOS != LBM_EOS_NONE) {
    psi_s[ty + 1][tx + 1] = solid ? psi_w : psi_of<C, EOS>(p, rho);
    // one-node ring around the tile: 2 (TX + 2) + 2 TY cells
    const int tid = ty * TX + tx;
    constexpr int kRing = 2 * (TX + 2) + 2 * TY;
    for (int k = tid; k < kRing; k += TX * TY) {
      int hx, hy;
      if (k < TX + 2) {
        hx = k;
        hy = 0;
      } else if (k < 2 * (TX + 2)) {
        hx = k - (TX + 2);
        hy = TY + 1;
      } else if (k < 2 * (TX + 2) + TY) {
        hx = 0;
        hy = k - 2 * (TX + 2) + 1;
      } else {
        hx = TX + 1;
        hy = k - 2 * (TX + 2) - TY + 1;
      }
      const int gxh = wrap_any(x0 - 1 + hx, nx), gyh = wrap_any(y0 - 1 + hy, ny);
      const int m = gyh * nx + gxh;
      C ps;
      if (flags[m] & FLAG_SOLID)
        ps = psi_w;
      else
        ps = psi_of<C, EOS>(p, node_rho<S>(fa, N, m, rho_ref));
      psi_s[hy][hx] = ps;
    }
    __syncthreads();
  }
  if (!inside) return;
  if (solid) {
    if constexpr (FIELDS) {
      const double nan = __longlong_as_double(0x7ff8000000000000LL);
      rho_m[n] = nan;
      ux_m[n] = nan;
      uy_m[n] = nan;
    }
    return;
  }

  // Total force: Eq. (16) plus body forces.
  C Fx = C(0), Fy = C(0);
  if constexpr (EOS != LBM_EOS_NONE) {
    const int cx = tx + 1, cy = ty + 1;
    // sum_a w_a psi(x + e_a) e_a, accumulated in direction order 1..8
    C sx = wpsi<C>(1) * psi_s[cy][cx + 1];
    sx -= wpsi<C>(3) * psi_s[cy][cx - 1];
    sx += wpsi<C>(5) * psi_s[cy + 1][cx + 1];
    sx -= wpsi<C>(6) * psi_s[cy + 1][cx - 1];
    sx -= wpsi<C>(7) * psi_s[cy - 1][cx - 1];
    sx += wpsi<C>(8) * psi_s[cy - 1][cx + 1];
    C sy = wpsi<C>(2) * psi_s[cy + 1][cx];
    sy -= wpsi<C>(4) * psi_s[cy - 1][cx];
    sy += wpsi<C>(5) * psi_s[cy + 1][cx + 1];
    sy += wpsi<C>(6) * psi_s[cy + 1][cx - 1];
    sy -= wpsi<C>(7) * psi_s[cy - 1][cx - 1];
    sy -= wpsi<C>(8) * psi_s[cy - 1][cx + 1];
    const C mg = -C(p.G) * psi_s[cy][cx];
    Fx = mg * sx;
    Fy = mg * sy;
  }
  if (p.has_body) {
    Fx += rho * C(p.gx);
    Fy += rho * C(p.gy);
    if (p.azC != 0.0) {
      C dx = C(x) - C(p.azcx), dy = C(y) - C(p.azcy);
      C r2 = dx * dx + dy * dy;
      Fx += C(p.azC) * (-dy) / r2;
      Fy += C(p.azC) * dx / r2;
    }
  }

  // Velocity with the half-force term, Eq. (5).
  C mx = f[1];
  mx -= f[3];
  mx += f[5];
  mx -= f[6];
  mx -= f[7];
  mx += f[8];
  C my = f[2];
  my -= f[4];
  my += f[5];
  my += f[6];
  my -= f[7];
  my -= f[8];
  const C ux = (mx + C(0.5) * Fx) / rho;
  const C uy = (my + C(0.5) * Fy) / rho;

  if constexpr (FIELDS) {
    rho_m[n] = double(rho);
    ux_m[n] = double(ux);
    uy_m[n] = double(uy);
    return;
  } else {
    if (fl & FLAG_MACRO) {
      rho_m[n] = double(rho);
      ux_m[n] = double(ux);
      uy_m[n] = double(uy);
    }
    // Collision, Eq. (2), with f_eq of Eq. (4) and the Guo forcing term, then push (Eq. 3).
    const C omega = C(p.omega), pref = C(p.guo_pref);
    const C uu = ux * ux + uy * uy;
    const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
    const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const C eu = C(ex(a)) * ux + C(ey(a)) * uy;
      const C w = wgt<C>(a);
      C feq;
      if constexpr (DEV)
        feq = w * (rho - rho_ref) + w * rho * (C(3) * eu + C(4.5) * eu * eu - C(1.5) * uu);
      else
        feq = w * rho * (C(1) + C(3) * eu + C(4.5) * eu * eu - C(1.5) * uu);
      const C gxa = C(3) * (C(ex(a)) - ux) + C(9) * eu * C(ex(a));
      const C gya = C(3) * (C(ey(a)) - uy) + C(9) * eu * C(ey(a));
      const C Fa = pref * w * (gxa * Fx + gya * Fy);
      const C fs = f[a] - omega * (f[a] - feq) + Fa;
      const int dxn = ex(a) > 0 ? xp : (ex(a) < 0 ? xm : x);
      const int dyn = ey(a) > 0 ? yp : (ey(a) < 0 ? ym : y);
      fb[a * N + (size_t)dyn * nx + dxn] = S(fs);
    }
  }
}

template <typename S, int EOS>
cudaError_t launch_t(const DevParams& p, const void* fa, void* fb, const uint8_t* flags,
                     double* rho_m, double* ux_m, double* uy_m, bool fields_only,
                     cudaStream_t s) {
  dim3 block(TX, TY);
  dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY);
  if (fields_only)
    step_kernel<S, EOS, true><<<grid, block, 0, s>>>(p, (const S*)fa, (S*)fb, flags, rho_m, ux_m,
                                                      uy_m);
  else
    step_kernel<S, EOS, false><<<grid, block, 0, s>>>(p, (const S*)fa, (S*)fb, flags, rho_m,
                                                       ux_m, uy_m);
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

}  // namespace

cudaError_t launch_step(int precision, const DevParams& p, const void* fa, void* fb,
                        const uint8_t* flags, double* rho_m, double* ux_m, double* uy_m,
                        bool fields_only, cudaStream_t s) {
  if (precision == LBM_FP32_DEV)
    return launch_s<float>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s);
  return launch_s<double>(p, fa, fb, flags, rho_m, ux_m, uy_m, fields_only, s);
}

}  // namespace lbm
