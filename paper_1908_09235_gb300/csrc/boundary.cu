// Curved-wall pass of one time step (Sec. 2.2, Sec. 3.1, Sec. 4.1): for every boundary node x_b
// and every cut link a (x_s = x_b + e_a solid, fraction q), the unknown incoming population
// f_abar(x_b, t+1) from the time-t values, then the per-node leakage of Eq. (15) and the
// correction of scheme A (Eq. 18) or the fictitious density of scheme B (Eq. 22) / Bao (Eq. 23).
//
// With the push layout of the step kernel (destination lattice B, source lattice A) the time-t
// values of a link are found at:
//   f*_a(x_b)    = B_a(x_s)        (pushed into the solid slot)
//   f*_abar(x_b) = B_abar(x_f)     f*_a(x_f) = B_a(x_b)      f*_a(x_ff) = B_a(x_f)
//   f*_abar(x_f) = B_abar(x_ff)    f_a(x_b) (pre-collision) = A_a(x_b)
// with x_f = x_b - e_a and x_ff = x_b - 2 e_a; rho and u at x_b and x_f come from the step
// kernel's macro arrays.  The pass writes B_abar(x_b) and, for scheme A, B_0(x_b); none of the
// slots it reads is written by another link, so the pass is race-free.
//
// Everything that depends only on q, tau and the scheme (chi of Eqs. 9-11, u_s of Eq. 10, the
// weights of Eqs. 12-14, which operands a link reads) is evaluated once at creation by
// link_setup_kernel into a per-link recipe, with the same operations the equations state; a step
// then costs each link a few loads and FMAs.  An 8-lane group handles a boundary node, one lane
// per link; per-node sums use fixed-order shuffles (bitwise reproducible).  Arithmetic is FP64
// for every storage format.
#include "d2q9.cuh"

namespace lbm {

namespace {

constexpr uint8_t kFromA = 1;   // X2 is read from lattice A (pre-collision)
constexpr uint8_t kGhost = 2;   // the link has the ghost-node term chi f_eq(x_s)

// The bracket of Eqs. (8), (20), (22): w_a [1 + 3 e_a.u_s + 4.5 (e_a.u_b)^2 - 1.5 u_b.u_b].
__device__ __forceinline__ double bracket(int a, double usx, double usy, double ubx, double uby) {
  double eus = ex(a) * usx + ey(a) * usy;
  double eub = ex(a) * ubx + ey(a) * uby;
  return wgt<double>(a) * (1.0 + 3.0 * eus + 4.5 * eub * eub - 1.5 * (ubx * ubx + uby * uby));
}

// One thread per boundary node: the recipe of each of its links.
__global__ void link_setup_kernel(DevParams p, int nb, const int32_t* __restrict__ bnode,
                                  const int32_t* __restrict__ boff,
                                  const uint8_t* __restrict__ ldir, const double* __restrict__ lq,
                                  const uint8_t* __restrict__ flags, LinkRecipe r) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int nx = p.nx, ny = p.ny, N = p.N, scheme = p.scheme;
  const double tau = p.tau;
  const int n = bnode[b];
  const int i = n % nx, j = n / nx;
  for (int l = boff[b]; l < boff[b + 1]; ++l) {
    const int a = ldir[l], ab = opposite(a);
    const double q = lq[l];
    const int ns = wrap_once(j + ey(a), ny) * nx + wrap_once(i + ex(a), nx);
    const int nf = wrap_once(j - ey(a), ny) * nx + wrap_once(i - ex(a), nx);
    const int nff = wrap_once(j - 2 * ey(a), ny) * nx + wrap_once(i - 2 * ex(a), nx);
    const bool f_solid = flags[nf] & FLAG_SOLID, ff_solid = flags[nff] & FLAG_SOLID;
    double c0 = 1.0, c1 = 0.0, c2 = 0.0, chi = 0.0, cus = 0.0;  // default: halfway bounce-back
    int x1 = -1, x2 = -1, uf = -1;
    uint8_t kind = 0;
    switch (scheme) {
      case LBM_FH:
      case LBM_MLS:
      case LBM_MOD_A:
      case LBM_MOD_B:
      case LBM_BAO:
        if (q < 0.5) {
          if (scheme == LBM_FH) {  // Eq. (9): u_s = u_b
            chi = (2.0 * q - 1.0) / (tau - 1.0);
            cus = 1.0;
            kind = kGhost;
          } else if (!f_solid) {   // Eq. (11): u_s = u(x_f)
            chi = (2.0 * q - 1.0) / (tau - 2.0);
            uf = nf;
            kind = kGhost;
          }                        // x_f solid: halfway bounce-back for this link
        } else {                   // Eq. (10) with u_w = 0
          chi = (2.0 * q - 1.0) / tau;
          cus = (q - 1.0) / q;
          kind = kGhost;
        }
        if (kind & kGhost) c0 = 1.0 - chi;  // Eq. (7) / Eq. (17)
        break;
      case LBM_BOUZIDI_L:
      case LBM_BOUZIDI_L_A:  // Eq. (12)
        if (q < 0.5) {
          if (!f_solid) {
            c0 = 2.0 * q;
            c1 = 1.0 - 2.0 * q;
            x1 = a * N + n;
          }
        } else {
          c0 = 1.0 / (2.0 * q);
          c1 = (2.0 * q - 1.0) / (2.0 * q);
          x1 = ab * N + nf;
        }
        break;
      case LBM_BOUZIDI_Q:  // Eq. (13)
        if (q < 0.5) {
          if (!f_solid) {
            if (ff_solid) {  // x_ff solid: linear Bouzidi
              c0 = 2.0 * q;
              c1 = 1.0 - 2.0 * q;
              x1 = a * N + n;
            } else {
              c0 = q * (1.0 + 2.0 * q);
              c1 = 1.0 - 4.0 * q * q;
              x1 = a * N + n;
              c2 = -(q * (1.0 - 2.0 * q));
              x2 = a * N + nf;
            }
          }
        } else if (f_solid) {  // x_f solid: linear Bouzidi
          c0 = 1.0 / (2.0 * q);
          c1 = (2.0 * q - 1.0) / (2.0 * q);
          x1 = ab * N + nf;
        } else {
          c0 = 1.0 / (q * (2.0 * q + 1.0));
          c1 = (2.0 * q - 1.0) / q;
          x1 = ab * N + nf;
          c2 = -((2.0 * q - 1.0) / (2.0 * q + 1.0));
          x2 = ab * N + nff;
        }
        break;
      case LBM_ZHAO_YONG:  // Eq. (14): post-collision f*_abar(x_b), pre-collision f_a(x_b)
        c0 = 0.0;
        c1 = 2.0 * q / (1.0 + 2.0 * q);
        x1 = ab * N + nf;
        c2 = 1.0 / (1.0 + 2.0 * q);
        x2 = a * N + n;
        kind = kFromA;
        break;
      default:
        break;
    }
    r.src[l] = a * N + ns;
    r.dst[l] = ab * N + n;
    r.x1[l] = x1;
    r.x2[l] = x2;
    r.uf[l] = uf;
    r.kind[l] = kind;
    r.c0[l] = c0;
    r.c1[l] = c1;
    r.c2[l] = c2;
    r.chi[l] = chi;
    r.cus[l] = cus;
  }
}

template <typename S>
struct Lat {
  const void* __restrict__ src;  // lattice A: f(t)
  void* __restrict__ dst;        // lattice B: streamed values of step t
  int N;
  double rho_ref;
  static constexpr bool dev = Pop<S>::dev;
  // value of element e of a plane with weight w (deviation formats store f - w rho_ref)
  __device__ double load(const void* base, int e, double w) const {
    double v = Pop<S>::load_e(base, e, N);
    if (dev) v += w * rho_ref;
    return v;
  }
  // store f at element e, returns the rounding residue (intended - stored) in FP64
  __device__ double store(int e, double w, double v) const {
    if (dev) {
      const double d = v - w * rho_ref;
      return d - Pop<S>::store_e(dst, e, N, d);
    }
    Pop<S>::store_e(dst, e, N, v);
    return 0.0;
  }
};

// Sum over the 8 lanes of a node's group in a fixed tree order (bitwise reproducible).
__device__ __forceinline__ double group8_sum(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

template <typename S>
__global__ void __launch_bounds__(128) boundary_kernel(DevParams p, int nb,
                                                       const int32_t* __restrict__ bnode,
                                                       const int32_t* __restrict__ boff,
                                                       const uint8_t* __restrict__ ldir,
                                                       LinkRecipe r, Lat<S> L,
                                                       const double* __restrict__ rho_m,
                                                       const double* __restrict__ ux_m,
                                                       const double* __restrict__ uy_m,
                                                       double* __restrict__ carry) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = gt >> 3, k = gt & 7;
  const bool node_ok = b < nb;
  const int scheme = p.scheme;
  const bool fix_f0 = scheme == LBM_MOD_A || scheme == LBM_BOUZIDI_L_A;
  const bool conserving = fix_f0 || scheme == LBM_MOD_B || scheme == LBM_HBB;
  const bool fict = scheme == LBM_MOD_B || scheme == LBM_BAO;

  // round 1: node and link records
  int n = 0, l0 = 0, nl = 0;
  if (node_ok) {
    n = bnode[b];
    l0 = boff[b];
    nl = boff[b + 1] - l0;
  }
  const bool act = node_ok && k < nl;
  int a = 1, src = 0, dst = 0, x1 = -1, x2 = -1, uf = -1;
  uint8_t kind = 0;
  double c0 = 1.0, c1 = 0.0, c2 = 0.0, chi = 0.0, cus = 0.0;
  double rho_b = 1.0, ubx = 0.0, uby = 0.0;
  if (act) {
    const int l = l0 + k;
    a = ldir[l];
    src = r.src[l];
    dst = r.dst[l];
    x1 = r.x1[l];
    x2 = r.x2[l];
    uf = r.uf[l];
    kind = r.kind[l];
    c0 = r.c0[l];
    c1 = r.c1[l];
    c2 = r.c2[l];
    chi = r.chi[l];
    cus = r.cus[l];
    rho_b = rho_m[n];
    ubx = ux_m[n];
    uby = uy_m[n];
  }
  // round 2: lattice values
  const double w = wgt<double>(a);
  double fo = 0.0, X1 = 0.0, X2 = 0.0, usx = 0.0, usy = 0.0;
  if (act) {
    fo = L.load(L.dst, src, w);  // outgoing f*_a(x_b, t)
    if (x1 >= 0) X1 = L.load(L.dst, x1, w);
    if (x2 >= 0) X2 = L.load((kind & kFromA) ? L.src : L.dst, x2, w);
    if (kind & kGhost) {
      if (uf >= 0) {
        usx = ux_m[uf];
        usy = uy_m[uf];
      } else {
        usx = cus * ubx;
        usy = cus * uby;
      }
    }
  }
  double f0_old = 0.0;
  if (node_ok && k == 0 && (fix_f0 || (L.dev && conserving))) f0_old = L.load(L.dst, n, wgt<double>(0));

  const bool gh = act && (kind & kGhost);
  const double br = gh ? bracket(a, usx, usy, ubx, uby) : 0.0;
  double rho_s = rho_b;
  if (fict) {
    double num = 0.0, den = 0.0;
    if (gh) {  // links without a ghost term are halfway bounce-back: chi = 0
      num = scheme == LBM_MOD_B ? chi * fo : fo;  // Eq. (22) / Eq. (23)
      den = scheme == LBM_MOD_B ? chi * br : br;
    }
    num = group8_sum(num);
    den = group8_sum(den);
    if (den != 0.0) rho_s = num / den;
  }
  double val = c0 * fo + c1 * X1 + c2 * X2;
  if (gh) val += chi * ((fict ? rho_s : rho_b) * br);  // Eq. (8) / Eq. (20) in Eq. (7) / (17)
  double resid = 0.0;
  if (act) resid = L.store(dst, w, val);

  double dm = 0.0;
  if (fix_f0) dm = group8_sum(act ? fo - val : 0.0);  // Eq. (15)
  if (L.dev && conserving) resid = group8_sum(resid);
  if (node_ok && k == 0) {
    if (fix_f0) {
      double f0 = f0_old + dm;  // Eq. (18)
      if (L.dev) f0 += carry[b];
      resid += L.store(n, wgt<double>(0), f0);
    } else if (L.dev && conserving && carry[b] != 0.0) {
      resid += L.store(n, wgt<double>(0), f0_old + carry[b]);
    }
    if (L.dev && conserving) carry[b] = resid;
  }
}

template <typename S>
cudaError_t launch_b(const DevParams& p, int nb, const int32_t* bnode, const int32_t* boff,
                     const uint8_t* ldir, LinkRecipe r, const void* fa, void* fb,
                     const double* rho_m, const double* ux_m, const double* uy_m, double* carry,
                     cudaStream_t s) {
  Lat<S> L{fa, fb, p.N, p.rho_ref};
  const long long threads = 8LL * nb;
  boundary_kernel<S><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(
      p, nb, bnode, boff, ldir, r, L, rho_m, ux_m, uy_m, carry);
  return cudaGetLastError();
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

size_t link_recipe_bytes(long long nl) {
  return 5 * align256(nl * 4) + align256(nl) + 5 * align256(nl * 8);
}

void link_recipe_carve(char* base, long long nl, LinkRecipe* r) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = base + off;
    off += align256(bytes);
    return q;
  };
  r->src = (int32_t*)take(nl * 4);
  r->dst = (int32_t*)take(nl * 4);
  r->x1 = (int32_t*)take(nl * 4);
  r->x2 = (int32_t*)take(nl * 4);
  r->uf = (int32_t*)take(nl * 4);
  r->kind = (uint8_t*)take(nl);
  r->c0 = (double*)take(nl * 8);
  r->c1 = (double*)take(nl * 8);
  r->c2 = (double*)take(nl * 8);
  r->chi = (double*)take(nl * 8);
  r->cus = (double*)take(nl * 8);
}

cudaError_t launch_link_setup(const DevParams& p, int nb, const int32_t* bnode,
                              const int32_t* boff, const uint8_t* ldir, const double* lq,
                              const uint8_t* flags, LinkRecipe r, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  link_setup_kernel<<<(nb + 127) / 128, 128, 0, s>>>(p, nb, bnode, boff, ldir, lq, flags, r);
  return cudaGetLastError();
}

cudaError_t launch_boundary(int precision, const DevParams& p, int nb, const int32_t* bnode,
                            const int32_t* boff, const uint8_t* ldir, LinkRecipe r,
                            const void* fa, void* fb, const double* rho_m, const double* ux_m,
                            const double* uy_m, double* carry, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  if (precision == LBM_FP32_DEV)
    return launch_b<float>(p, nb, bnode, boff, ldir, r, fa, fb, rho_m, ux_m, uy_m, carry, s);
  if (precision == LBM_FP16_DEV)
    return launch_b<__half>(p, nb, bnode, boff, ldir, r, fa, fb, rho_m, ux_m, uy_m, carry, s);
  return launch_b<double>(p, nb, bnode, boff, ldir, r, fa, fb, rho_m, ux_m, uy_m, carry, s);
}

}  // namespace lbm
