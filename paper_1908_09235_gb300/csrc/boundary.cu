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
// per link; per-node sums use fixed-order shuffles (bitwise reproducible).  Link values are
// computed in the step's arithmetic type (FP64 for FP64 storage, FP32 for the deviation
// formats); each boundary node's mass bookkeeping is FP64 for every format.  (FP64 link
// arithmetic for the deviation formats was measured: 4.3 us more per step at 4096^2 and 0.25 ms
// more per batched step of 512 lattices, on GB300's narrow FP64 pipe.)
#include "d2q9.cuh"

namespace lbm {

namespace {

constexpr uint8_t kFromA = 1;   // X2 is read from lattice A (pre-collision)
constexpr uint8_t kGhost = 2;   // the link has the ghost-node term chi f_eq(x_s)

// The bracket of Eqs. (8), (20), (22): w_a [1 + 3 e_a.u_s + 4.5 (e_a.u_b)^2 - 1.5 u_b.u_b].
template <typename T>
__device__ __forceinline__ T bracket(int a, T usx, T usy, T ubx, T uby) {
  const T eus = T(ex(a)) * usx + T(ey(a)) * usy;
  const T eub = T(ex(a)) * ubx + T(ey(a)) * uby;
  return wgt<T>(a) * (T(1) + T(3) * eus + T(4.5) * eub * eub - T(1.5) * (ubx * ubx + uby * uby));
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
    const bool f_solid = flags[LBM_CHK(nf, N)] & FLAG_SOLID;
    const bool ff_solid = flags[LBM_CHK(nff, N)] & FLAG_SOLID;
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
    r.c0f[l] = float(c0);
    r.c1f[l] = float(c1);
    r.c2f[l] = float(c2);
    r.chif[l] = float(chi);
    r.cusf[l] = float(cus);
  }
}

template <typename S>
struct Lat {
  const void* __restrict__ src;  // lattice A: f(t)
  void* __restrict__ dst;        // lattice B: streamed values of step t
  int N;
  double rho_ref;
};

// Sum over the 8 lanes of a node's group in a fixed tree order (bitwise reproducible); `mask`
// holds the 8 lanes of the group.
template <typename T>
__device__ __forceinline__ T group8_sum(T v, unsigned mask) {
  v += __shfl_xor_sync(mask, v, 4);
  v += __shfl_xor_sync(mask, v, 2);
  v += __shfl_xor_sync(mask, v, 1);
  return v;
}

template <typename T>
__device__ __forceinline__ T pick(const double* d, const float* f, int l) {
  if constexpr (sizeof(T) == 8) return d[l]; else return f[l];
}

// Boundary node b of a lattice handled by lane k (0..7) of an 8-lane group (node_ok false: a
// padding group, which still takes part in the shuffles).  Arithmetic type T: FP64 for FP64
// storage; FP32 for the deviation formats, whose mass bookkeeping is exact instead: each node's
// imbalance between the stored outgoing and incoming values is summed in FP64 and goes, with the
// previous step's FP64 rounding residue, into its rest population.  For schemes A and
// L-Bouzidi + A that is Eq. (18); for B (balanced by construction, Eq. 19) and halfway
// bounce-back it only returns the FP32 rounding.
template <typename S>
__device__ __forceinline__ void boundary_group(const DevParams& p, int b, int k, bool node_ok,
                                               const int32_t* __restrict__ bnode,
                                               const int32_t* __restrict__ boff,
                                               const uint8_t* __restrict__ ldir,
                                               const LinkRecipe& r, const Lat<S>& L,
                                               const double* __restrict__ rho_m,
                                               const double* __restrict__ ux_m,
                                               const double* __restrict__ uy_m,
                                               double* __restrict__ carry,
                                               double* __restrict__ force, unsigned mask) {
  using T = typename Pop<S>::C;
  constexpr bool DEV = Pop<S>::dev;
  const int scheme = p.scheme;
  const int N = L.N;
  const bool fix_f0 = scheme == LBM_MOD_A || scheme == LBM_BOUZIDI_L_A;
  const bool conserving = fix_f0 || scheme == LBM_MOD_B || scheme == LBM_HBB;
  const bool fict = scheme == LBM_MOD_B || scheme == LBM_BAO;
  const T rref = DEV ? p.k<T>().rho_ref : T(0);
  // macro arrays: FP64 for FP64 storage, FP32 (in the same memory) for the deviation formats
  const T* rhoT = reinterpret_cast<const T*>(rho_m);
  const T* uxT = reinterpret_cast<const T*>(ux_m);
  const T* uyT = reinterpret_cast<const T*>(uy_m);

  // first loads: node and link records
  int n = 0, l0 = 0, nl = 0;
  if (node_ok) {
    n = bnode[b];
    l0 = boff[b];
    nl = boff[b + 1] - l0;
  }
  const bool act = node_ok && k < nl;
  int a = 1, src = 0, dst = 0, x1 = -1, x2 = -1, uf = -1;
  uint8_t kind = 0;
  T c0 = T(1), c1 = T(0), c2 = T(0), chi = T(0), cus = T(0);
  T rho_b = T(1), ubx = T(0), uby = T(0);
  if (act) {
    const int l = l0 + k;
    a = ldir[l];
    src = r.src[l];
    dst = r.dst[l];
    x1 = r.x1[l];
    x2 = r.x2[l];
    uf = r.uf[l];
    kind = r.kind[l];
    c0 = pick<T>(r.c0, r.c0f, l);
    c1 = pick<T>(r.c1, r.c1f, l);
    c2 = pick<T>(r.c2, r.c2f, l);
    chi = pick<T>(r.chi, r.chif, l);
    cus = pick<T>(r.cus, r.cusf, l);
  }
  // Everything above is fixed for the lattice's lifetime; everything below (the moments in the
  // macro arrays, the lattice values, the FP64 carry) was written by the kernels before this
  // one.  Launched as a programmatic dependent of the step kernel, the pass waits here for that
  // grid to complete and its writes to be visible; otherwise the wait returns at once.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (act) {
    rho_b = rhoT[LBM_CHK(n, N)];
    ubx = uxT[n];
    uby = uyT[n];
  }
  // second loads: lattice values (deviations d_ for the FP32 formats; f = d_ + w rho_ref)
  const T w = wgt<T>(a);
  const T wr = w * rref;
  T fo_d = T(0), X1 = T(0), X2 = T(0), usx = T(0), usy = T(0);
  if (act) {
    fo_d = Pop<S>::load_t(L.dst, src, N);  // outgoing f*_a(x_b, t)
    if (x1 >= 0) X1 = Pop<S>::load_t(L.dst, x1, N) + wr;
    if (x2 >= 0) X2 = Pop<S>::load_t((kind & kFromA) ? L.src : L.dst, x2, N) + wr;
    if (kind & kGhost) {
      if (uf >= 0) {
        usx = uxT[LBM_CHK(uf, N)];
        usy = uyT[uf];
      } else {
        usx = cus * ubx;
        usy = cus * uby;
      }
    }
  }
  const T fo = fo_d + wr;
  const bool lane0 = node_ok && k == 0;
  T f0_d = T(0);
  if (lane0 && (fix_f0 || (DEV && conserving))) f0_d = Pop<S>::load_t(L.dst, n, N);

  const bool gh = act && (kind & kGhost);
  const T br = gh ? bracket<T>(a, usx, usy, ubx, uby) : T(0);
  T rho_s = rho_b;
  if (fict) {
    T num = T(0), den = T(0);
    if (gh) {  // links without a ghost term are halfway bounce-back: chi = 0
      num = scheme == LBM_MOD_B ? chi * fo : fo;  // Eq. (22) / Eq. (23)
      den = scheme == LBM_MOD_B ? chi * br : br;
    }
    num = group8_sum(num, mask);
    den = group8_sum(den, mask);
    if (den != T(0)) rho_s = num / den;
  }
  T val = c0 * fo + c1 * X1 + c2 * X2;
  if (gh) val += chi * ((fict ? rho_s : rho_b) * br);  // Eq. (8) / Eq. (20) in Eq. (7) / (17)
  T in_d = T(0);
  if (act) {
    // a pure bounce-back link (halfway bounce-back or a fallback) copies the stored value
    const bool copy = DEV && !gh && x1 < 0 && x2 < 0 && c0 == T(1);
    in_d = Pop<S>::store_t(L.dst, dst, N, copy ? fo_d : val - wr);
  }
  if (force) {
    // Momentum exchange (Sec. 4.2, after Mei et al. 2002): through link a the wall receives
    // e_a (f*_a(x_b, t) + f_abar(x_b, t+1)), with the incoming value as stored; FP64 sums over
    // the node's links in the fixed group order, one (fx, fy) per boundary node.
    const double m = act ? double(fo_d) + double(in_d) + 2.0 * wgt<double>(a) * L.rho_ref : 0.0;
    const double fx = group8_sum(double(ex(a)) * m, mask);
    const double fy = group8_sum(double(ey(a)) * m, mask);
    if (lane0) {
      force[2 * b] = fx;
      force[2 * b + 1] = fy;
    }
  }

  if constexpr (DEV) {
    if (conserving) {
      // exact FP64 imbalance of the stored deviations (the w rho_ref parts cancel)
      const double dm = group8_sum(act ? double(fo_d) - double(in_d) : 0.0, mask);
      if (lane0) {
        const double want = double(f0_d) + dm + carry[b];
        if (want != double(f0_d)) {
          const T st = Pop<S>::store_t(L.dst, n, N, T(want));
          carry[b] = want - double(st);
        } else {
          carry[b] = 0.0;
        }
      }
    }
  } else {
    if (fix_f0) {
      const double dm = group8_sum(act ? fo - val : 0.0, mask);  // Eq. (15)
      if (lane0) Pop<S>::store_t(L.dst, n, N, f0_d + dm);     // Eq. (18)
    }
  }
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
                                                       double* __restrict__ carry,
                                                       double* __restrict__ force) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = gt >> 3;
  boundary_group<S>(p, b, gt & 7, b < nb, bnode, boff, ldir, r, L, rho_m, ux_m, uy_m, carry,
                    force, 0xffffffffu);
}

// Channel ends (Sec. 4.2), after streaming and the wall pass; one thread per row j.  Inlet
// i = 0: the populations entering from the left (1, 5, 8) follow from the prescribed velocity
// (u_in, 0) and the known ones by Zou and He's rule:
//   rho = (f0 + f2 + f4 + 2 (f3 + f6 + f7)) / (1 - u_in),  f1 = f3 + 2/3 rho u_in,
//   f5 = f7 - (f2 - f4)/2 + rho u_in / 6,  f8 = f6 + (f2 - f4)/2 + rho u_in / 6.
// Outlet i = nx - 1 (fully developed flow): the populations entering from the right (3, 6, 7)
// equal those of column nx - 2.  FP64 arithmetic on the full populations (deviation + w rho_ref).
template <typename S>
__global__ void open_x_kernel(DevParams p, void* __restrict__ fb,
                              const uint8_t* __restrict__ flags, double u_in) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p.ny) return;
  const int nx = p.nx, N = p.N;
  const double rr = p.rho_ref;
  auto get = [&](int a, int n) { return Pop<S>::load_e(fb, a * N + n, N) + wgt<double>(a) * rr; };
  auto put = [&](int a, int n, double v) { Pop<S>::store_e(fb, a * N + n, N, v - wgt<double>(a) * rr); };
  const int n0 = j * nx;
  if (!(flags[n0] & FLAG_SOLID)) {
    const double f0 = get(0, n0), f2 = get(2, n0), f3 = get(3, n0), f4 = get(4, n0);
    const double f6 = get(6, n0), f7 = get(7, n0);
    const double rho = (f0 + f2 + f4 + 2.0 * (f3 + f6 + f7)) / (1.0 - u_in);
    put(1, n0, f3 + 2.0 / 3.0 * rho * u_in);
    put(5, n0, f7 - 0.5 * (f2 - f4) + rho * u_in / 6.0);
    put(8, n0, f6 + 0.5 * (f2 - f4) + rho * u_in / 6.0);
  }
  const int n1 = j * nx + nx - 1;
  if (!(flags[n1] & FLAG_SOLID)) {
    // copies of stored values: no rounding for any format
    Pop<S>::store_e(fb, 3 * N + n1, N, Pop<S>::load_e(fb, 3 * N + n1 - 1, N));
    Pop<S>::store_e(fb, 6 * N + n1, N, Pop<S>::load_e(fb, 6 * N + n1 - 1, N));
    Pop<S>::store_e(fb, 7 * N + n1, N, Pop<S>::load_e(fb, 7 * N + n1 - 1, N));
  }
}

// Boundary nodes of many lattices: items are (domain, boundary node); a persistent grid of
// 8-lane groups walks them.  Lattices whose step budget is spent are skipped.
template <typename S>
// 12 CTAs per SM (40 registers, a few spilled): more resident 8-lane groups for the chains of
// dependent loads each item is (80 against 83 us per batched step FP32, 78 against 84 FP16)
__global__ void __launch_bounds__(128, 12) batch_boundary_kernel(const BatchDomain* __restrict__ doms,
                                                             const int2* __restrict__ items,
                                                             const int* __restrict__ n_items) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = gt & 7;
  const unsigned mask = 0xffu << (threadIdx.x & 24);
  const int ni = *n_items;
  for (int i = gt >> 3; i < ni; i += (gridDim.x * blockDim.x) >> 3) {
    const int2 it = items[i];
    const BatchDomain& D = doms[it.x];
    if (D.steps_left <= 0) continue;  // uniform over the group
    const int cur = D.cur;
    const Lat<S> L{D.f[cur], D.f[cur ^ 1], D.p.N, D.p.rho_ref};
    boundary_group<S>(D.p, it.y, k, true, D.bnode, D.boff, D.ldir, D.recipe, L, D.rho_m, D.ux_m,
                      D.uy_m, D.carry, nullptr, mask);
  }
}

__global__ void batch_advance_kernel(BatchDomain* __restrict__ doms, int n, int* claim) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d == 0) *claim = 0;  // the step kernel of the next step claims tiles from 0
  if (d < n && doms[d].steps_left > 0) {
    doms[d].cur ^= 1;
    --doms[d].steps_left;
    ++doms[d].steps_done;
  }
}

template <typename S>
cudaError_t launch_b(const DevParams& p, int nb, const int32_t* bnode, const int32_t* boff,
                     const uint8_t* ldir, LinkRecipe r, const void* fa, void* fb,
                     const double* rho_m, const double* ux_m, const double* uy_m, double* carry,
                     double* force, cudaStream_t s) {
  Lat<S> L{fa, fb, p.N, p.rho_ref};  // rho_ref also in p.k<T>() for the FP32 formats
  const long long threads = 8LL * nb;
  // a programmatic dependent of the kernel before it in the stream (the step kernel): its CTAs
  // may start, and load their link records, while that grid drains; they wait for it before
  // reading anything it wrote (griddepcontrol.wait in boundary_group)
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)((threads + 127) / 128));
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, boundary_kernel<S>, p, nb, bnode, boff, ldir, r, L, rho_m, ux_m,
                            uy_m, carry, force);
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

size_t link_recipe_bytes(long long nl) {
  return 5 * align256(nl * 4) + align256(nl) + 5 * align256(nl * 8) + 5 * align256(nl * 4);
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
  r->c0f = (float*)take(nl * 4);
  r->c1f = (float*)take(nl * 4);
  r->c2f = (float*)take(nl * 4);
  r->chif = (float*)take(nl * 4);
  r->cusf = (float*)take(nl * 4);
}

cudaError_t launch_link_setup(const DevParams& p, int nb, const int32_t* bnode,
                              const int32_t* boff, const uint8_t* ldir, const double* lq,
                              const uint8_t* flags, LinkRecipe r, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  link_setup_kernel<<<(nb + 127) / 128, 128, 0, s>>>(p, nb, bnode, boff, ldir, lq, flags, r);
  return cudaGetLastError();
}

cudaError_t launch_batch_boundary(int precision, const BatchDomain* doms, const int2* items,
                                  const int* n_items, int grid, cudaStream_t s) {
  if (precision == LBM_FP32_DEV)
    batch_boundary_kernel<float><<<grid, 128, 0, s>>>(doms, items, n_items);
  else if (precision == LBM_FP16_DEV)
    batch_boundary_kernel<__half><<<grid, 128, 0, s>>>(doms, items, n_items);
  else
    batch_boundary_kernel<double><<<grid, 128, 0, s>>>(doms, items, n_items);
  return cudaGetLastError();
}

int batch_boundary_grid(int precision) {
  // every 8-lane group walks items one after the other, each a chain of dependent loads: fill
  // the GPU with as many resident groups as it takes
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fn = precision == LBM_FP32_DEV ? (const void*)batch_boundary_kernel<float>
                   : precision == LBM_FP16_DEV ? (const void*)batch_boundary_kernel<__half>
                                               : (const void*)batch_boundary_kernel<double>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 128, 0) != cudaSuccess || per < 1) {
    cudaGetLastError();
    per = 8;
  }
  return sms * per;
}

cudaError_t launch_batch_advance(BatchDomain* doms, int n_doms, int* claim, cudaStream_t s) {
  if (n_doms <= 0) return cudaSuccess;
  batch_advance_kernel<<<(n_doms + 127) / 128, 128, 0, s>>>(doms, n_doms, claim);
  return cudaGetLastError();
}

cudaError_t launch_boundary(int precision, const DevParams& p, int nb, const int32_t* bnode,
                            const int32_t* boff, const uint8_t* ldir, LinkRecipe r,
                            const void* fa, void* fb, const double* rho_m, const double* ux_m,
                            const double* uy_m, double* carry, double* force, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  if (precision == LBM_FP32_DEV)
    return launch_b<float>(p, nb, bnode, boff, ldir, r, fa, fb, rho_m, ux_m, uy_m, carry, force, s);
  if (precision == LBM_FP16_DEV)
    return launch_b<__half>(p, nb, bnode, boff, ldir, r, fa, fb, rho_m, ux_m, uy_m, carry, force,
                            s);
  return launch_b<double>(p, nb, bnode, boff, ldir, r, fa, fb, rho_m, ux_m, uy_m, carry, force, s);
}

cudaError_t launch_open_x(int precision, const DevParams& p, void* fb, const uint8_t* flags,
                          double u_in, cudaStream_t s) {
  const unsigned grid = (unsigned)((p.ny + 127) / 128);
  if (precision == LBM_FP32_DEV)
    open_x_kernel<float><<<grid, 128, 0, s>>>(p, fb, flags, u_in);
  else if (precision == LBM_FP16_DEV)
    open_x_kernel<__half><<<grid, 128, 0, s>>>(p, fb, flags, u_in);
  else
    open_x_kernel<double><<<grid, 128, 0, s>>>(p, fb, flags, u_in);
  return cudaGetLastError();
}

}  // namespace lbm
