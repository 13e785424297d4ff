// Curved-wall pass of one time step (Sec. 2.2, Sec. 3.1, Sec. 4.1): for every boundary node x_b
// and every cut link a (x_s = x_b + e_a solid, fraction q), the unknown incoming population
// f_abar(x_b, t+1) from the time-t values, then the per-node leakage of Eq. (15) and the
// correction of scheme A (Eq. 18) or the fictitious density of scheme B (Eq. 22) / Bao (Eq. 23).
//
// An 8-lane group per boundary node, one lane per link (the links of a node are consecutive in
// the CSR arrays).  Arithmetic is FP64 for every storage format.  With the push layout of the step kernel (destination lattice B,
// source lattice A) the time-t values of a link are found at:
//   f*_a(x_b)    = B_a(x_s)        (pushed into the solid slot)
//   f*_abar(x_b) = B_abar(x_f)     f*_a(x_f) = B_a(x_b)      f*_a(x_ff) = B_a(x_f)
//   f*_abar(x_f) = B_abar(x_ff)    f_a(x_b) (pre-collision) = A_a(x_b)
// with x_f = x_b - e_a and x_ff = x_b - 2 e_a; rho and u at x_b and x_f come from the step
// kernel's macro arrays.  The pass writes B_abar(x_b) and, for scheme A, B_0(x_b); none of the
// slots it reads is written by another boundary thread, so the pass is race-free.
#include "d2q9.cuh"

namespace lbm {

namespace {

template <typename S>
struct Lat {
  const S* __restrict__ src;  // lattice A: f(t)
  S* __restrict__ dst;        // lattice B: streamed values of step t
  size_t N;
  double rho_ref;
  static constexpr bool dev = sizeof(S) == 4;
  __device__ double load(const S* base, int a, int m) const {
    double v = double(base[a * N + m]);
    if (dev) v += wgt<double>(a) * rho_ref;
    return v;
  }
  __device__ double B(int a, int m) const { return load(dst, a, m); }
  __device__ double A(int a, int m) const { return load(src, a, m); }
  // store f_a at m, returns the rounding residue (intended - stored) in FP64
  __device__ double storeB(int a, int m, double v) const {
    if (dev) {
      double d = v - wgt<double>(a) * rho_ref;
      S s = S(d);
      dst[a * N + m] = s;
      return d - double(s);
    } else {
      dst[a * N + m] = S(v);
      return 0.0;
    }
  }
};

// The bracket of Eqs. (8), (20), (22): w_a [1 + 3 e_a.u_s + 4.5 (e_a.u_b)^2 - 1.5 u_b.u_b].
__device__ __forceinline__ double bracket(int a, double usx, double usy, double ubx, double uby) {
  double eus = ex(a) * usx + ey(a) * usy;
  double eub = ex(a) * ubx + ey(a) * uby;
  return wgt<double>(a) * (1.0 + 3.0 * eus + 4.5 * eub * eub - 1.5 * (ubx * ubx + uby * uby));
}

// chi and u_s of the ghost-node family: FH q < 1/2 Eq. (9); MLS q < 1/2 Eq. (11);
// both q >= 1/2 Eq. (10) with u_w = 0.  False when MLS needs u_f and x_f is solid.
__device__ __forceinline__ bool ghost(const DevParams& p, bool fh, int n, int nf, bool f_solid,
                                      double q, const double* ux_m, const double* uy_m,
                                      double* chi, double* usx, double* usy) {
  if (q < 0.5) {
    if (fh) {
      *chi = (2.0 * q - 1.0) / (p.tau - 1.0);
      *usx = ux_m[n];
      *usy = uy_m[n];
    } else {
      if (f_solid) return false;
      *chi = (2.0 * q - 1.0) / (p.tau - 2.0);
      *usx = ux_m[nf];
      *usy = uy_m[nf];
    }
  } else {
    *chi = (2.0 * q - 1.0) / p.tau;
    *usx = (q - 1.0) / q * ux_m[n];
    *usy = (q - 1.0) / q * uy_m[n];
  }
  return true;
}

// Sum over the 8 lanes of a node's group in a fixed tree order (bitwise reproducible).
__device__ __forceinline__ double group8_sum(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// One 8-lane group per boundary node, one lane per cut link (a fluid node has at most 8), so the
// loads of all links of a node are in flight together; per-node sums use group8_sum.
template <typename S>
__global__ void __launch_bounds__(128) boundary_kernel(DevParams p, int nb,
                                                       const int32_t* __restrict__ bnode,
                                                       const int32_t* __restrict__ boff,
                                                       const uint8_t* __restrict__ ldir,
                                                       const double* __restrict__ lq,
                                                       const uint8_t* __restrict__ flags, Lat<S> L,
                                                       const double* __restrict__ rho_m,
                                                       const double* __restrict__ ux_m,
                                                       const double* __restrict__ uy_m,
                                                       double* __restrict__ carry) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = gt >> 3, k = gt & 7;
  const bool node_ok = b < nb;
  const int nx = p.nx, ny = p.ny, scheme = p.scheme;
  int n = 0, l0 = 0, nl = 0;
  if (node_ok) {
    n = bnode[b];
    l0 = boff[b];
    nl = boff[b + 1] - l0;
  }
  const bool act = node_ok && k < nl;
  const bool ghost_family = scheme == LBM_FH || scheme == LBM_MLS || scheme == LBM_MOD_A ||
                            scheme == LBM_MOD_B || scheme == LBM_BAO;
  const bool fh = scheme == LBM_FH;

  int a = 1, ab = 3, nf = 0, ns = 0, nff = 0;
  double q = 0.5, fo = 0.0, rho_b = 1.0, ubx = 0.0, uby = 0.0;
  bool f_solid = false, ff_solid = false;
  if (act) {
    const int i = n % nx, j = n / nx;
    a = ldir[l0 + k];
    ab = opposite(a);
    q = lq[l0 + k];
    ns = wrap_once(j + ey(a), ny) * nx + wrap_once(i + ex(a), nx);
    nf = wrap_once(j - ey(a), ny) * nx + wrap_once(i - ex(a), nx);
    nff = wrap_once(j - 2 * ey(a), ny) * nx + wrap_once(i - 2 * ex(a), nx);
    f_solid = flags[nf] & FLAG_SOLID;
    ff_solid = flags[nff] & FLAG_SOLID;
    fo = L.B(a, ns);  // outgoing f*_a(x_b, t)
    rho_b = rho_m[n];
    ubx = ux_m[n];
    uby = uy_m[n];
  }
  double chi = 0.0, usx = 0.0, usy = 0.0;
  bool gh = false;
  if (act && ghost_family)
    gh = ghost(p, fh, n, nf, f_solid, q, ux_m, uy_m, &chi, &usx, &usy);

  double rho_s = rho_b;
  if (scheme == LBM_MOD_B || scheme == LBM_BAO) {
    double num = 0.0, den = 0.0;
    if (gh) {  // links without a ghost value (MLS fallback) are halfway bounce-back: chi = 0
      const double br = bracket(a, usx, usy, ubx, uby);
      num = scheme == LBM_MOD_B ? chi * fo : fo;  // Eq. (22) / Eq. (23)
      den = scheme == LBM_MOD_B ? chi * br : br;
    }
    num = group8_sum(num);
    den = group8_sum(den);
    if (den != 0.0) rho_s = num / den;
  }

  double val = fo;
  if (act) {
    if (ghost_family) {
      if (gh) {
        const double rr = (scheme == LBM_MOD_B || scheme == LBM_BAO) ? rho_s : rho_b;
        const double feq_s = rr * bracket(a, usx, usy, ubx, uby);  // Eq. (8) / Eq. (20)
        val = (1.0 - chi) * fo + chi * feq_s;                      // Eq. (7) / Eq. (17)
      }
    } else if (scheme == LBM_BOUZIDI_L || scheme == LBM_BOUZIDI_L_A) {  // Eq. (12)
      if (q < 0.5) {
        if (!f_solid) val = 2.0 * q * fo + (1.0 - 2.0 * q) * L.B(a, n);
      } else {
        val = 1.0 / (2.0 * q) * fo + (2.0 * q - 1.0) / (2.0 * q) * L.B(ab, nf);
      }
    } else if (scheme == LBM_BOUZIDI_Q) {  // Eq. (13)
      if (q < 0.5) {
        if (!f_solid) {
          if (ff_solid)
            val = 2.0 * q * fo + (1.0 - 2.0 * q) * L.B(a, n);
          else
            val = q * (1.0 + 2.0 * q) * fo + (1.0 - 4.0 * q * q) * L.B(a, n) -
                  q * (1.0 - 2.0 * q) * L.B(a, nf);
        }
      } else {
        if (f_solid)
          val = 1.0 / (2.0 * q) * fo + (2.0 * q - 1.0) / (2.0 * q) * L.B(ab, nf);
        else
          val = 1.0 / (q * (2.0 * q + 1.0)) * fo + (2.0 * q - 1.0) / q * L.B(ab, nf) -
                (2.0 * q - 1.0) / (2.0 * q + 1.0) * L.B(ab, nff);
      }
    } else if (scheme == LBM_ZHAO_YONG) {  // Eq. (14)
      val = 2.0 * q / (1.0 + 2.0 * q) * L.B(ab, nf) + 1.0 / (1.0 + 2.0 * q) * L.A(a, n);
    }
  }
  double resid = 0.0;
  if (act) resid = L.storeB(ab, n, val);

  const bool fix_f0 = scheme == LBM_MOD_A || scheme == LBM_BOUZIDI_L_A;
  const bool conserving = fix_f0 || scheme == LBM_MOD_B || scheme == LBM_HBB;
  double dm = 0.0;
  if (fix_f0) dm = group8_sum(act ? fo - val : 0.0);  // Eq. (15)
  if (L.dev && conserving) resid = group8_sum(resid);
  if (node_ok && k == 0) {
    if (fix_f0) {
      double f0 = L.B(0, n) + dm;  // Eq. (18)
      if (L.dev) f0 += carry[b];
      resid += L.storeB(0, n, f0);
    } else if (L.dev && conserving && carry[b] != 0.0) {
      resid += L.storeB(0, n, L.B(0, n) + carry[b]);
    }
    if (L.dev && conserving) carry[b] = resid;
  }
}

template <typename S>
cudaError_t launch_b(const DevParams& p, int nb, const int32_t* bnode, const int32_t* boff,
                     const uint8_t* ldir, const double* lq, const uint8_t* flags, const void* fa,
                     void* fb, const double* rho_m, const double* ux_m, const double* uy_m,
                     double* carry, cudaStream_t s) {
  Lat<S> L{(const S*)fa, (S*)fb, (size_t)p.N, p.rho_ref};
  const long long threads = 8LL * nb;
  boundary_kernel<S><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(
      p, nb, bnode, boff, ldir, lq, flags, L, rho_m, ux_m, uy_m, carry);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_boundary(int precision, const DevParams& p, int nb, const int32_t* bnode,
                            const int32_t* boff, const uint8_t* ldir, const double* lq,
                            const uint8_t* flags, const void* fa, void* fb, const double* rho_m,
                            const double* ux_m, const double* uy_m, double* carry,
                            cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  if (precision == LBM_FP32_DEV)
    return launch_b<float>(p, nb, bnode, boff, ldir, lq, flags, fa, fb, rho_m, ux_m, uy_m, carry,
                           s);
  return launch_b<double>(p, nb, bnode, boff, ldir, lq, flags, fa, fb, rho_m, ux_m, uy_m, carry,
                          s);
}

}  // namespace lbm
