/*
 * lbm_oracle.c -- TEST INFRASTRUCTURE ONLY (see lbm_oracle.h).
 *
 * A deliberately plain FP64 implementation of one time step of the two-phase lattice Boltzmann
 * method of Yu, Li & Wen (arXiv:1908.09235), written stage by stage with a separate array per
 * stage:  f (pre-collision) -> rho, psi, F, u -> f* (post-collision) -> f_new (streamed) ->
 * curved-wall schemes at the boundary nodes -> f_new becomes f.
 * No blocking, fusion or reordering beyond what the equations state.  Compile with
 * -O2 -ffp-contract=off (no fused multiply-add, no fast-math).  The per-node loops carry OpenMP
 * pragmas (ignored without -fopenmp): each node's arithmetic is the same in either build, every
 * value is written by one iteration, and the ledger, the wall pass and the set-up stay serial,
 * so the multi-threaded build gives the same bits.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* D2Q9 lattice, Sec. 2.1 below Eq. (4). */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* Interaction weights of Eq. (16): 1/3 for |e|^2 = 1, 1/12 for |e|^2 = 2. */
static const double WPSI[9] = {0.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0,
                               1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0};

struct or_sim {
  or_params p;
  or_circle* circles;
  int nx, ny, N;
  uint8_t* solid;
  double* f;   /* pre-collision f(x,t), 9*N        */
  double* fs;  /* post-collision f*(x,t), Eq. (2)  */
  double* fn;  /* streamed f(x,t+1), Eq. (3)       */
  double *rho, *psi, *Fx, *Fy, *ux, *uy;
  /* boundary nodes in ascending node index, each with its links in ascending direction */
  int nb, nl;
  int* bnode;
  int* boff; /* nb+1 */
  int* ldir;
  double* lq;
  long fallbacks;
  double last_leak, last_max_node_leak;
  /* channel mode (flow past a cylinder, Sec. 4.2): velocity inlet at i = 0, outlet at nx - 1 */
  int open_x;
  double u_in;
  /* momentum-exchange force on the solid nodes during the last step */
  double force_x, force_y;
};

/* ------------------------------------------------------------------------------------------ */
/* Building blocks                                                                             */
/* ------------------------------------------------------------------------------------------ */

/* Eq. (4) with c_s^2 = 1/3: f_eq = w rho [1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u]. */
void or_feq(double rho, double ux, double uy, double out[9]) {
  double uu = ux * ux + uy * uy;
  for (int a = 0; a < 9; ++a) {
    double eu = EX[a] * ux + EY[a] * uy;
    out[a] = W[a] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
  }
}

/* Forcing term of Guo, Zheng & Shi (2002), the scheme the paper adopts in Sec. 3.2:
 * F_a = (1 - 1/(2 tau)) w_a [ (e_a - u)/c_s^2 + (e_a.u) e_a / c_s^4 ] . F,  with delta_t = 1. */
void or_guo(double tau, double ux, double uy, double Fx, double Fy, double out[9]) {
  double pref = 1.0 - 1.0 / (2.0 * tau);
  for (int a = 0; a < 9; ++a) {
    double eu = EX[a] * ux + EY[a] * uy;
    double cx = 3.0 * (EX[a] - ux) + 9.0 * eu * EX[a];
    double cy = 3.0 * (EY[a] - uy) + 9.0 * eu * EY[a];
    out[a] = pref * W[a] * (cx * Fx + cy * Fy);
  }
}

/* Moments of Eq. (5) then the collision of Eq. (2) at one node, given its total force F. */
void or_collide_node(const double f[9], double tau, double Fx, double Fy, double out[9]) {
  double rho = 0.0, mx = 0.0, my = 0.0;
  for (int a = 0; a < 9; ++a) {
    rho += f[a];
    mx += f[a] * EX[a];
    my += f[a] * EY[a];
  }
  double ux = (mx + 0.5 * Fx) / rho;
  double uy = (my + 0.5 * Fy) / rho;
  double feq[9], fa[9];
  or_feq(rho, ux, uy, feq);
  or_guo(tau, ux, uy, Fx, Fy, fa);
  for (int a = 0; a < 9; ++a) out[a] = f[a] - (f[a] - feq[a]) / tau + fa[a];
}

/* Carnahan-Starling equation of state, eta = b rho / 4:
 * p = rho R T (1 + eta + eta^2 - eta^3) / (1 - eta)^3 - a rho^2. */
double or_cs_pressure(double a, double b, double R, double T, double rho) {
  double eta = b * rho / 4.0;
  double om = 1.0 - eta;
  return rho * R * T * (1.0 + eta + eta * eta - eta * eta * eta) / (om * om * om) - a * rho * rho;
}

/* Pseudopotential psi(rho).  Exponential form of Sec. 3.2: psi0 exp(-rho0/rho).  For an EOS p(rho)
 * the pressure of the Eq. (16) force is p = rho c_s^2 + G psi^2 / 2 (the Eq. (16) weights give
 * sum_a w_a e_a e_a = I), hence psi = sqrt(2 (p - rho/3) / G). */
double or_psi(const or_params* p, double rho) {
  if (p->eos == OR_EOS_EXP) return p->psi0 * exp(-p->rho0 / rho);
  if (p->eos == OR_EOS_CS) {
    double pr = or_cs_pressure(p->a, p->b, p->R, p->T, rho);
    return sqrt(2.0 * (pr - rho / 3.0) / p->G);
  }
  return 0.0;
}

static int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

/* Eq. (16) on a periodic nx*ny field of psi values (no solids): F = -G psi(x) sum w psi(x+e) e. */
void or_force_from_psi(int nx, int ny, double G, const double* psi, double* Fx, double* Fy) {
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double sx = 0.0, sy = 0.0;
      for (int a = 1; a < 9; ++a) {
        double pn = psi[wrapi(j + EY[a], ny) * nx + wrapi(i + EX[a], nx)];
        sx += WPSI[a] * pn * EX[a];
        sy += WPSI[a] * pn * EY[a];
      }
      Fx[j * nx + i] = -G * psi[j * nx + i] * sx;
      Fy[j * nx + i] = -G * psi[j * nx + i] * sy;
    }
}

/* ---- Carnahan-Starling critical point and Maxwell coexistence (set-up, not the step) ---- */
/* With h(eta) = eta Z(eta), Z = (1+eta+eta^2-eta^3)/(1-eta)^3, p = (4RT/b) h(eta) - 16 a eta^2/b^2.
 * The critical point solves dp/deta = d2p/deta2 = 0, i.e. h'(eta) = eta h''(eta), and then
 * T_c = 8 a / (b R h''(eta_c)). */
static double cs_h1(double e) { /* h'(eta) */
  double N = e + e * e + e * e * e - e * e * e * e;
  double N1 = 1.0 + 2.0 * e + 3.0 * e * e - 4.0 * e * e * e;
  double s = 1.0 - e;
  return N1 / (s * s * s) + 3.0 * N / (s * s * s * s);
}
static double cs_h2(double e) { /* h''(eta) */
  double N = e + e * e + e * e * e - e * e * e * e;
  double N1 = 1.0 + 2.0 * e + 3.0 * e * e - 4.0 * e * e * e;
  double N2 = 2.0 + 6.0 * e - 12.0 * e * e;
  double s = 1.0 - e;
  return N2 / (s * s * s) + 6.0 * N1 / (s * s * s * s) + 12.0 * N / (s * s * s * s * s);
}

int or_cs_critical(double a, double b, double R, double* Tc, double* rhoc) {
  double lo = 0.01, hi = 0.5; /* h' - eta h'' is positive at lo, negative at hi */
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double g = cs_h1(mid) - mid * cs_h2(mid);
    if (g > 0.0) lo = mid; else hi = mid;
  }
  double ec = 0.5 * (lo + hi);
  *rhoc = 4.0 * ec / b;
  *Tc = 8.0 * a / (b * R * cs_h2(ec));
  return 0;
}

/* Integral of p / rho^2 d rho for Carnahan-Starling, up to a constant:
 * R T [ln eta + 1/(1-eta)^2 + 2/(1-eta)] - a rho  (uses Z - 1 = (4 eta - 2 eta^2)/(1-eta)^3). */
static double cs_phi(double a, double b, double R, double T, double rho) {
  double eta = b * rho / 4.0;
  double s = 1.0 - eta;
  return R * T * (log(eta) + 1.0 / (s * s) + 2.0 / s) - a * rho;
}

/* Root of p(rho) = p0 by bisection on [lo, hi] where p - p0 changes sign. */
static double cs_root(double a, double b, double R, double T, double p0, double lo, double hi) {
  double flo = or_cs_pressure(a, b, R, T, lo) - p0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double fm = or_cs_pressure(a, b, R, T, mid) - p0;
    if ((fm > 0.0) == (flo > 0.0)) { lo = mid; flo = fm; } else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* Maxwell equal-area construction: p(rhoV) = p(rhoL) = p0 and
 * integral_{rhoV}^{rhoL} (p - p0) / rho^2 d rho = 0.  Bisection on p0 between the spinodal
 * pressures; for each p0 the outer roots come from bisection too. */
int or_cs_coexistence(double a, double b, double R, double T, double* rhoL, double* rhoV) {
  double Tc, rhoc;
  or_cs_critical(a, b, R, &Tc, &rhoc);
  if (!(T < Tc)) return -1;
  double rmax = 4.0 / b * 0.999;
  /* spinodals: dp/drho = 0 on either side of rhoc, by bisection on the sign of a difference */
  double lo = 1e-9, hi = rhoc, h = 1e-7;
  for (int it = 0; it < 200; ++it) { /* vapour spinodal: dp/drho goes from + to - */
    double mid = 0.5 * (lo + hi);
    double d = or_cs_pressure(a, b, R, T, mid + h) - or_cs_pressure(a, b, R, T, mid - h);
    if (d > 0.0) lo = mid; else hi = mid;
  }
  double rs_v = 0.5 * (lo + hi);
  lo = rhoc; hi = rmax;
  for (int it = 0; it < 200; ++it) { /* liquid spinodal: dp/drho goes from - to + */
    double mid = 0.5 * (lo + hi);
    double d = or_cs_pressure(a, b, R, T, mid + h) - or_cs_pressure(a, b, R, T, mid - h);
    if (d < 0.0) lo = mid; else hi = mid;
  }
  double rs_l = 0.5 * (lo + hi);
  double pmax = or_cs_pressure(a, b, R, T, rs_v);
  double pmin = or_cs_pressure(a, b, R, T, rs_l);
  double plo = pmin > 0.0 ? pmin : 1e-300, phi_ = pmax;
  double rv = 0.0, rl = 0.0;
  for (int it = 0; it < 200; ++it) {
    double p0 = 0.5 * (plo + phi_);
    rv = cs_root(a, b, R, T, p0, 1e-12, rs_v);
    rl = cs_root(a, b, R, T, p0, rs_l, rmax);
    /* area A(p0) = integral (p - p0)/rho^2 = [phi] - p0 (1/rv - 1/rl); decreasing in p0 */
    double area = cs_phi(a, b, R, T, rl) - cs_phi(a, b, R, T, rv) - p0 * (1.0 / rv - 1.0 / rl);
    if (area > 0.0) plo = p0; else phi_ = p0;
  }
  *rhoL = rl;
  *rhoV = rv;
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Geometry: solid nodes and the wall fraction q of Eq. (6)                                    */
/* ------------------------------------------------------------------------------------------ */

static int circle_solid(const or_circle* c, int i, int j) {
  double dx = (double)i - c->cx;
  double dy = (double)j - c->cy;
  double d2 = dx * dx + dy * dy;
  double r2 = c->r * c->r;
  return c->solid_outside ? (d2 >= r2) : (d2 <= r2);
}

static int node_solid(const or_sim* s, int i, int j) {
  if (s->p.wall_q_lo > 0.0 && j == 0) return 1;
  if (s->p.wall_q_hi > 0.0 && j == s->ny - 1) return 1;
  for (int c = 0; c < s->p.n_circles; ++c)
    if (circle_solid(&s->circles[c], i, j)) return 1;
  return 0;
}

/* Eq. (6): q = |x_b - x_w| / |x_b - x_s| is the parameter t in (0, 1] at which the segment
 * x_b + t e crosses the circle |x - c| = r: a t^2 + 2 bq t + cq = 0 with a = e.e, bq = e.d,
 * cq = d.d - r^2, d = x_b - c.  Entering a solid disc takes the smaller root, leaving the fluid
 * disc of an outside-solid circle the larger one. */
static double circle_q(const or_circle* c, int i, int j, int a) {
  double dx = (double)i - c->cx;
  double dy = (double)j - c->cy;
  double ex = (double)EX[a], ey = (double)EY[a];
  double aa = ex * ex + ey * ey;
  double bq = ex * dx + ey * dy;
  double cq = (dx * dx + dy * dy) - c->r * c->r;
  double disc = bq * bq - aa * cq;
  if (disc < 0.0) disc = 0.0;
  double sq = sqrt(disc);
  double t = c->solid_outside ? (-bq + sq) / aa : (-bq - sq) / aa;
  if (t > 1.0) t = 1.0;
  return t;
}

static double link_q(const or_sim* s, int i, int j, int a) {
  int si = wrapi(i + EX[a], s->nx), sj = wrapi(j + EY[a], s->ny);
  double q = 2.0;
  if (s->p.wall_q_lo > 0.0 && sj == 0 && s->p.wall_q_lo < q) q = s->p.wall_q_lo;
  if (s->p.wall_q_hi > 0.0 && sj == s->ny - 1 && s->p.wall_q_hi < q) q = s->p.wall_q_hi;
  for (int c = 0; c < s->p.n_circles; ++c)
    if (circle_solid(&s->circles[c], si, sj)) {
      double t = circle_q(&s->circles[c], i, j, a);
      if (t < q) q = t;
    }
  return q;
}

static void build_geometry(or_sim* s) {
  int nx = s->nx, ny = s->ny, N = s->N;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) s->solid[j * nx + i] = (uint8_t)node_solid(s, i, j);
  /* count links */
  int nb = 0, nl = 0;
  for (int n = 0; n < N; ++n) {
    if (s->solid[n]) continue;
    int i = n % nx, j = n / nx, k = 0;
    for (int a = 1; a < 9; ++a)
      if (s->solid[wrapi(j + EY[a], ny) * nx + wrapi(i + EX[a], nx)]) ++k;
    if (k) { ++nb; nl += k; }
  }
  s->nb = nb;
  s->nl = nl;
  s->bnode = (int*)malloc(sizeof(int) * (nb > 0 ? nb : 1));
  s->boff = (int*)malloc(sizeof(int) * (nb + 1));
  s->ldir = (int*)malloc(sizeof(int) * (nl > 0 ? nl : 1));
  s->lq = (double*)malloc(sizeof(double) * (nl > 0 ? nl : 1));
  int b = 0, l = 0;
  for (int n = 0; n < N; ++n) {
    if (s->solid[n]) continue;
    int i = n % nx, j = n / nx, k = 0;
    for (int a = 1; a < 9; ++a)
      if (s->solid[wrapi(j + EY[a], ny) * nx + wrapi(i + EX[a], nx)]) {
        if (!k) { s->bnode[b] = n; s->boff[b] = l; }
        s->ldir[l] = a;
        s->lq[l] = link_q(s, i, j, a);
        ++l;
        ++k;
      }
    if (k) ++b;
  }
  s->boff[nb] = nl;
}

/* ------------------------------------------------------------------------------------------ */
/* Simulation                                                                                  */
/* ------------------------------------------------------------------------------------------ */

or_sim* or_create(const or_params* p) {
  or_sim* s = (or_sim*)calloc(1, sizeof(or_sim));
  s->p = *p;
  s->nx = p->nx;
  s->ny = p->ny;
  s->N = p->nx * p->ny;
  s->circles = (or_circle*)malloc(sizeof(or_circle) * (p->n_circles > 0 ? p->n_circles : 1));
  if (p->n_circles > 0) memcpy(s->circles, p->circles, sizeof(or_circle) * p->n_circles);
  s->p.circles = s->circles;
  size_t N = (size_t)s->N;
  s->solid = (uint8_t*)calloc(N, 1);
  s->f = (double*)calloc(9 * N, sizeof(double));
  s->fs = (double*)calloc(9 * N, sizeof(double));
  s->fn = (double*)calloc(9 * N, sizeof(double));
  s->rho = (double*)calloc(N, sizeof(double));
  s->psi = (double*)calloc(N, sizeof(double));
  s->Fx = (double*)calloc(N, sizeof(double));
  s->Fy = (double*)calloc(N, sizeof(double));
  s->ux = (double*)calloc(N, sizeof(double));
  s->uy = (double*)calloc(N, sizeof(double));
  build_geometry(s);
  return s;
}

void or_destroy(or_sim* s) {
  if (!s) return;
  free(s->circles); free(s->solid); free(s->f); free(s->fs); free(s->fn);
  free(s->rho); free(s->psi); free(s->Fx); free(s->Fy); free(s->ux); free(s->uy);
  free(s->bnode); free(s->boff); free(s->ldir); free(s->lq);
  free(s);
}

int or_num_links(const or_sim* s) { return s->nl; }
int or_num_boundary_nodes(const or_sim* s) { return s->nb; }

void or_flags(const or_sim* s, uint8_t* flags) {
  for (int n = 0; n < s->N; ++n) flags[n] = s->solid[n] ? 1 : 0;
  for (int b = 0; b < s->nb; ++b) flags[s->bnode[b]] |= 2;
}

void or_links(const or_sim* s, int32_t* node, uint8_t* dir, double* q) {
  for (int b = 0; b < s->nb; ++b)
    for (int l = s->boff[b]; l < s->boff[b + 1]; ++l) {
      node[l] = s->bnode[b];
      dir[l] = (uint8_t)s->ldir[l];
      q[l] = s->lq[l];
    }
}

void or_init_fields(or_sim* s, const double* rho, const double* ux, const double* uy) {
  size_t N = (size_t)s->N;
  memset(s->f, 0, sizeof(double) * 9 * N);
  for (int n = 0; n < s->N; ++n) {
    if (s->solid[n]) continue;
    double feq[9];
    or_feq(rho[n], ux ? ux[n] : 0.0, uy ? uy[n] : 0.0, feq);
    for (int a = 0; a < 9; ++a) s->f[a * N + n] = feq[a];
  }
}

/* Droplet of radius R and interface width W centred at (cx, cy):
 * rho(r) = (rho_in + rho_out)/2 - (rho_in - rho_out)/2 tanh(2 (r - R) / W), u = 0. */
void or_init_droplet(or_sim* s, double cx, double cy, double R, double W, double rho_in,
                     double rho_out) {
  double* rho = (double*)malloc(sizeof(double) * s->N);
  for (int j = 0; j < s->ny; ++j)
    for (int i = 0; i < s->nx; ++i) {
      double dx = (double)i - cx, dy = (double)j - cy;
      double r = sqrt(dx * dx + dy * dy);
      rho[j * s->nx + i] =
          0.5 * (rho_in + rho_out) - 0.5 * (rho_in - rho_out) * tanh(2.0 * (r - R) / W);
    }
  or_init_fields(s, rho, NULL, NULL);
  free(rho);
}

/* Density, pseudopotential, total force and velocity of every fluid node from f:
 * rho by Eq. (5); psi of fluid nodes from rho and of solid nodes from the virtual wall density
 * (Sec. 3.2); F by Eq. (16) plus the body forces; u by Eq. (5) with the half-force term. */
static void compute_macros(or_sim* s) {
  int nx = s->nx, ny = s->ny, N = s->N;
  const double* f = s->f;
#pragma omp parallel for
  for (int n = 0; n < N; ++n) {
    if (s->solid[n]) { s->rho[n] = 0.0; continue; }
    double r = 0.0;
    for (int a = 0; a < 9; ++a) r += f[(size_t)a * N + n];
    s->rho[n] = r;
  }
  int multiphase = s->p.eos != OR_EOS_NONE;
  double psi_w = multiphase ? or_psi(&s->p, s->p.rho_wall) : 0.0;
#pragma omp parallel for
  for (int n = 0; n < N; ++n) s->psi[n] = s->solid[n] ? psi_w : (multiphase ? or_psi(&s->p, s->rho[n]) : 0.0);
#pragma omp parallel for
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      int n = j * nx + i;
      if (s->solid[n]) { s->Fx[n] = s->Fy[n] = 0.0; continue; }
      double Fx = 0.0, Fy = 0.0;
      if (multiphase) {
        double sx = 0.0, sy = 0.0;
        for (int a = 1; a < 9; ++a) {
          double pn = s->psi[wrapi(j + EY[a], ny) * nx + wrapi(i + EX[a], nx)];
          sx += WPSI[a] * pn * EX[a];
          sy += WPSI[a] * pn * EY[a];
        }
        Fx = -s->p.G * s->psi[n] * sx;
        Fy = -s->p.G * s->psi[n] * sy;
      }
      Fx += s->rho[n] * s->p.gx;
      Fy += s->rho[n] * s->p.gy;
      if (s->p.azim_C != 0.0) {
        double dx = (double)i - s->p.azim_cx, dy = (double)j - s->p.azim_cy;
        double r2 = dx * dx + dy * dy;
        Fx += s->p.azim_C * (-dy) / r2;
        Fy += s->p.azim_C * dx / r2;
      }
      s->Fx[n] = Fx;
      s->Fy[n] = Fy;
    }
#pragma omp parallel for
  for (int n = 0; n < N; ++n) {
    if (s->solid[n]) { s->ux[n] = s->uy[n] = 0.0; continue; }
    double mx = 0.0, my = 0.0;
    for (int a = 0; a < 9; ++a) {
      mx += f[(size_t)a * N + n] * EX[a];
      my += f[(size_t)a * N + n] * EY[a];
    }
    s->ux[n] = (mx + 0.5 * s->Fx[n]) / s->rho[n];
    s->uy[n] = (my + 0.5 * s->Fy[n]) / s->rho[n];
  }
}

/* Ghost-node parameters of one link for the FH / MLS family: chi and the fictitious velocity u_s.
 * FH, q < 1/2: Eq. (9).  MLS, q < 1/2: Eq. (11) with u_f = u(x_b - e_a).  Both, q >= 1/2:
 * Eq. (10) with u_w = 0.  Returns 0 when the MLS branch needs u_f but x_f is solid. */
static int ghost_params(const or_sim* s, int fh, int n, int a, double q, double* chi, double* usx,
                        double* usy) {
  double tau = s->p.tau;
  if (q < 0.5) {
    if (fh) {
      *chi = (2.0 * q - 1.0) / (tau - 1.0);
      *usx = s->ux[n];
      *usy = s->uy[n];
    } else {
      int i = n % s->nx, j = n / s->nx;
      int nf = wrapi(j - EY[a], s->ny) * s->nx + wrapi(i - EX[a], s->nx);
      if (s->solid[nf]) return 0;
      *chi = (2.0 * q - 1.0) / (tau - 2.0);
      *usx = s->ux[nf];
      *usy = s->uy[nf];
    }
  } else {
    *chi = (2.0 * q - 1.0) / tau;
    *usx = (q - 1.0) / q * s->ux[n];
    *usy = (q - 1.0) / q * s->uy[n];
  }
  return 1;
}

/* The bracket of Eqs. (8), (20), (22): w_a [1 + 3 e_a.u_s + 4.5 (e_a.u_b)^2 - 1.5 u_b.u_b]. */
static double ghost_bracket(int a, double usx, double usy, double ubx, double uby) {
  double eus = EX[a] * usx + EY[a] * usy;
  double eub = EX[a] * ubx + EY[a] * uby;
  return W[a] * (1.0 + 3.0 * eus + 4.5 * eub * eub - 1.5 * (ubx * ubx + uby * uby));
}

/* The unknown incoming populations of every boundary node (Sec. 2.2, Sec. 4.1). */
static void apply_boundary(or_sim* s) {
  size_t N = (size_t)s->N;
  int nx = s->nx, ny = s->ny, scheme = s->p.scheme;
  double leak = 0.0, maxleak = 0.0, force_x = 0.0, force_y = 0.0;
  for (int b = 0; b < s->nb; ++b) {
    int n = s->bnode[b];
    int i = n % nx, j = n / nx;
    int l0 = s->boff[b], l1 = s->boff[b + 1];
    double rho_b = s->rho[n], ubx = s->ux[n], uby = s->uy[n];
    /* Scheme B / Bao: fictitious density rho_s of the ghost equilibria, Eq. (22) / Eq. (23). */
    double rho_s = rho_b;
    if (scheme == OR_MOD_B || scheme == OR_BAO) {
      double num = 0.0, den = 0.0;
      for (int l = l0; l < l1; ++l) {
        int a = s->ldir[l];
        double chi, usx, usy;
        if (!ghost_params(s, 0, n, a, s->lq[l], &chi, &usx, &usy)) continue; /* HBB fallback */
        double br = ghost_bracket(a, usx, usy, ubx, uby);
        if (scheme == OR_MOD_B) {
          num += chi * s->fs[a * N + n];
          den += chi * br;
        } else {
          num += s->fs[a * N + n];
          den += br;
        }
      }
      if (den != 0.0) rho_s = num / den; /* den = 0 only when every chi = 0: rho_s then unused */
    }
    double sum_out = 0.0, sum_in = 0.0;
    double node_fx = 0.0, node_fy = 0.0;
    for (int l = l0; l < l1; ++l) {
      int a = s->ldir[l], ab = OPP[a];
      double q = s->lq[l];
      double fo = s->fs[a * N + n]; /* outgoing f*_a(x_b, t) */
      int nf = wrapi(j - EY[a], ny) * nx + wrapi(i - EX[a], nx);          /* x_f  */
      int nff = wrapi(j - 2 * EY[a], ny) * nx + wrapi(i - 2 * EX[a], nx); /* x_ff */
      double val;
      switch (scheme) {
        case OR_HBB:
          val = fo;
          break;
        case OR_FH:
        case OR_MLS:
        case OR_MOD_A:
        case OR_MOD_B:
        case OR_BAO: {
          double chi, usx, usy;
          if (!ghost_params(s, scheme == OR_FH, n, a, q, &chi, &usx, &usy)) {
            ++s->fallbacks;
            val = fo;
            break;
          }
          double rr = (scheme == OR_MOD_B || scheme == OR_BAO) ? rho_s : rho_b;
          double feq_s = rr * ghost_bracket(a, usx, usy, ubx, uby); /* Eq. (8) / Eq. (20) */
          val = (1.0 - chi) * fo + chi * feq_s;                       /* Eq. (7) / Eq. (17) */
          break;
        }
        case OR_BOUZIDI_L:
        case OR_BOUZIDI_L_A:
          if (q < 0.5) {
            if (s->solid[nf]) { ++s->fallbacks; val = fo; break; }
            val = 2.0 * q * fo + (1.0 - 2.0 * q) * s->fs[a * N + nf];
          } else {
            val = 1.0 / (2.0 * q) * fo + (2.0 * q - 1.0) / (2.0 * q) * s->fs[ab * N + n];
          }
          break;
        case OR_BOUZIDI_Q:
          if (q < 0.5) {
            if (s->solid[nf]) { ++s->fallbacks; val = fo; break; }
            if (s->solid[nff]) { /* linear Bouzidi for this link */
              ++s->fallbacks;
              val = 2.0 * q * fo + (1.0 - 2.0 * q) * s->fs[a * N + nf];
              break;
            }
            val = q * (1.0 + 2.0 * q) * fo + (1.0 - 4.0 * q * q) * s->fs[a * N + nf] -
                  q * (1.0 - 2.0 * q) * s->fs[a * N + nff];
          } else {
            if (s->solid[nf]) {
              ++s->fallbacks;
              val = 1.0 / (2.0 * q) * fo + (2.0 * q - 1.0) / (2.0 * q) * s->fs[ab * N + n];
              break;
            }
            val = 1.0 / (q * (2.0 * q + 1.0)) * fo + (2.0 * q - 1.0) / q * s->fs[ab * N + n] -
                  (2.0 * q - 1.0) / (2.0 * q + 1.0) * s->fs[ab * N + nf];
          }
          break;
        case OR_ZHAO_YONG: /* Eq. (14): post-collision f*_abar and pre-collision f_a at x_b */
          val = 2.0 * q / (1.0 + 2.0 * q) * s->fs[ab * N + n] + 1.0 / (1.0 + 2.0 * q) * s->f[a * N + n];
          break;
        default:
          val = fo;
      }
      s->fn[ab * N + n] = val;
      sum_out += fo;
      sum_in += val;
      /* Momentum exchange (Sec. 4.2, after Mei et al. 2002): f*_a(x_b) goes into the wall
       * along e_a and f_abar(x_b, t+1) comes back along -e_a, so the wall receives
       * e_a (f*_a + f_abar) through this link. */
      node_fx += EX[a] * (fo + val);
      node_fy += EY[a] * (fo + val);
    }
    force_x += node_fx;
    force_y += node_fy;
    double dm = sum_out - sum_in; /* Eq. (15) */
    leak += dm;
    if (scheme == OR_MOD_A || scheme == OR_BOUZIDI_L_A) {
      s->fn[n] = s->fs[n] + dm; /* Eq. (18): rest population at x_b takes the leakage */
      dm = sum_out - sum_in - (s->fn[n] - s->fs[n]);
    }
    if (fabs(dm) > maxleak) maxleak = fabs(dm);
  }
  s->last_leak = leak;
  s->last_max_node_leak = maxleak;
  s->force_x = force_x;
  s->force_y = force_y;
}

/* Channel ends (Sec. 4.2), after streaming and the wall schemes.  Inlet i = 0: the populations
 * entering from the left (1, 5, 8) follow from the prescribed velocity (u_in, 0) and the known
 * ones by Zou and He's rule (bounce-back of the non-equilibrium part normal to the inlet):
 *   rho = (f0 + f2 + f4 + 2 (f3 + f6 + f7)) / (1 - u_in)
 *   f1 = f3 + 2/3 rho u_in,  f5 = f7 - (f2 - f4)/2 + rho u_in/6,  f8 = f6 + (f2 - f4)/2 + rho u_in/6.
 * Outlet i = nx - 1, fully developed flow: the populations entering from the right (3, 6, 7)
 * equal those of column nx - 2. */
static void apply_open_x(or_sim* s) {
  size_t N = (size_t)s->N;
  int nx = s->nx, ny = s->ny;
  double u = s->u_in;
  for (int j = 0; j < ny; ++j) {
    int n = j * nx;
    if (!s->solid[n]) {
      double* f = s->fn;
      double f0 = f[0 * N + n], f2 = f[2 * N + n], f3 = f[3 * N + n], f4 = f[4 * N + n];
      double f6 = f[6 * N + n], f7 = f[7 * N + n];
      double rho = (f0 + f2 + f4 + 2.0 * (f3 + f6 + f7)) / (1.0 - u);
      f[1 * N + n] = f3 + 2.0 / 3.0 * rho * u;
      f[5 * N + n] = f7 - 0.5 * (f2 - f4) + rho * u / 6.0;
      f[8 * N + n] = f6 + 0.5 * (f2 - f4) + rho * u / 6.0;
    }
    int m = j * nx + nx - 1;
    if (!s->solid[m]) {
      const int in_dirs[3] = {3, 6, 7};
      for (int k = 0; k < 3; ++k) s->fn[in_dirs[k] * N + m] = s->fn[in_dirs[k] * N + m - 1];
    }
  }
}

void or_step(or_sim* s, int nsteps) {
  int nx = s->nx, ny = s->ny, N = s->N;
  size_t NN = (size_t)N;
  double tau = s->p.tau;
  for (int step = 0; step < nsteps; ++step) {
    compute_macros(s);
    /* collision, Eq. (2) */
#pragma omp parallel for
    for (int n = 0; n < N; ++n) {
      if (s->solid[n]) continue;
      double feq[9], fa[9];
      or_feq(s->rho[n], s->ux[n], s->uy[n], feq);
      or_guo(tau, s->ux[n], s->uy[n], s->Fx[n], s->Fy[n], fa);
      for (int a = 0; a < 9; ++a) {
        double fv = s->f[a * NN + n];
        s->fs[a * NN + n] = fv - (fv - feq[a]) / tau + fa[a];
      }
    }
    /* streaming, Eq. (3); populations that would enter a solid node leave the fluid */
    memset(s->fn, 0, sizeof(double) * 9 * NN);
#pragma omp parallel for
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int n = j * nx + i;
        if (s->solid[n]) continue;
        for (int a = 0; a < 9; ++a) {
          int m = wrapi(j + EY[a], ny) * nx + wrapi(i + EX[a], nx);
          if (!s->solid[m]) s->fn[a * NN + m] = s->fs[a * NN + n];
        }
      }
    apply_boundary(s);
    if (s->open_x) apply_open_x(s);
    double* t = s->f;
    s->f = s->fn;
    s->fn = t;
  }
}

/* Total mass: sum over fluid nodes and directions, Neumaier-compensated. */
double or_mass(const or_sim* s) {
  double sum = 0.0, c = 0.0;
  size_t N = (size_t)s->N;
  for (int n = 0; n < s->N; ++n) {
    if (s->solid[n]) continue;
    for (int a = 0; a < 9; ++a) {
      double x = s->f[a * N + n];
      double t = sum + x;
      if (fabs(sum) >= fabs(x)) c += (sum - t) + x; else c += (x - t) + sum;
      sum = t;
    }
  }
  return sum + c;
}

void or_fields(or_sim* s, double* rho, double* ux, double* uy) {
  compute_macros(s);
  for (int n = 0; n < s->N; ++n) {
    if (s->solid[n]) { rho[n] = ux[n] = uy[n] = NAN; continue; }
    rho[n] = s->rho[n];
    ux[n] = s->ux[n];
    uy[n] = s->uy[n];
  }
}

void or_get_f(const or_sim* s, double* f) { memcpy(f, s->f, sizeof(double) * 9 * (size_t)s->N); }
void or_set_f(or_sim* s, const double* f) { memcpy(s->f, f, sizeof(double) * 9 * (size_t)s->N); }
double or_last_leak(const or_sim* s) { return s->last_leak; }
void or_set_inflow(or_sim* s, double u_in) {
  s->open_x = 1;
  s->u_in = u_in;
}
void or_force(const or_sim* s, double* fx, double* fy) {
  *fx = s->force_x;
  *fy = s->force_y;
}
double or_last_max_node_leak(const or_sim* s) { return s->last_max_node_leak; }
long or_fallbacks(const or_sim* s) { return s->fallbacks; }
int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
