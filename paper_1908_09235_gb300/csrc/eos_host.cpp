// Host-side set-up of the Carnahan-Starling equation of state: critical point and Maxwell
// coexistence densities (used to place the initial droplet), and psi of the virtual wall density.
//
// p(rho) = rho R T Z(eta) - a rho^2, eta = b rho / 4, Z = 1 + (4 eta - 2 eta^2)/(1 - eta)^3.
// The critical point is the double root of dp/drho; coexistence solves equal pressure and equal
// chemical potential mu = f + p/rho with f(rho) = integral p/rho^2 d rho
//   = R T [ln eta + (1 - eta)^-2 + 2 (1 - eta)^-1] - a rho + const,
// by Newton's method on (rho_v, rho_l) started from the spinodals.
#include <cmath>

#include "lbm_internal.h"

namespace lbm {

namespace {

struct CS {
  double a, b, R, T;
  // d^k/d eta^k of g(eta) = eta Z(eta) = eta + (4 eta^2 - 2 eta^3)(1 - eta)^-3
  static double g1(double e) {
    double s = 1.0 - e;
    double u = 4.0 * e * e - 2.0 * e * e * e, du = 8.0 * e - 6.0 * e * e;
    return 1.0 + du / (s * s * s) + 3.0 * u / (s * s * s * s);
  }
  static double g2(double e) {
    double s = 1.0 - e;
    double u = 4.0 * e * e - 2.0 * e * e * e, du = 8.0 * e - 6.0 * e * e, d2u = 8.0 - 12.0 * e;
    return d2u / (s * s * s) + 6.0 * du / (s * s * s * s) + 12.0 * u / (s * s * s * s * s);
  }
  double p(double rho) const {
    double e = 0.25 * b * rho, s = 1.0 - e;
    return rho * R * T * (1.0 + (4.0 * e - 2.0 * e * e) / (s * s * s)) - a * rho * rho;
  }
  double dp(double rho) const { return R * T * g1(0.25 * b * rho) - 2.0 * a * rho; }
  double mu(double rho) const {
    double e = 0.25 * b * rho, s = 1.0 - e;
    double f = R * T * (std::log(e) + 1.0 / (s * s) + 2.0 / s) - a * rho;
    return f + p(rho) / rho;
  }
};

}  // namespace

bool cs_critical_point(double a, double b, double R, double* Tc, double* rhoc) {
  if (!(a > 0 && b > 0 && R > 0)) return false;
  // eta_c solves g'(eta) = eta g''(eta); Newton with a numerically differentiated residual,
  // safeguarded to stay in (0.05, 0.3).
  auto res = [](double e) { return CS::g1(e) - e * CS::g2(e); };
  double e = 0.13;
  for (int it = 0; it < 100; ++it) {
    double h = 1e-7;
    double r = res(e), d = (res(e + h) - res(e - h)) / (2 * h);
    double step = r / d;
    double en = e - step;
    if (en < 0.05) en = 0.5 * (e + 0.05);
    if (en > 0.3) en = 0.5 * (e + 0.3);
    if (std::fabs(en - e) < 1e-16) {
      e = en;
      break;
    }
    e = en;
  }
  *rhoc = 4.0 * e / b;
  // dp/drho = R T g'(eta) - 2 a rho = 0 and d2p/drho2 = R T g''(eta) b/4 - 2 a = 0
  *Tc = 8.0 * a / (b * R * CS::g2(e));
  return std::isfinite(*Tc) && *Tc > 0;
}

bool cs_maxwell(double a, double b, double R, double T, double* rho_l, double* rho_v) {
  double Tc, rhoc;
  if (!cs_critical_point(a, b, R, &Tc, &rhoc) || !(T > 0 && T < Tc)) return false;
  CS eos{a, b, R, T};
  const double rmax = 4.0 / b;
  // spinodals: zeros of dp/drho on either side of rhoc (dp decreases then increases)
  double lo = 1e-12, hi = rhoc;
  for (int it = 0; it < 300; ++it) {
    double m = 0.5 * (lo + hi);
    (eos.dp(m) > 0 ? lo : hi) = m;
  }
  const double sv = lo;
  lo = rhoc;
  hi = rmax * (1 - 1e-12);
  for (int it = 0; it < 300; ++it) {
    double m = 0.5 * (lo + hi);
    (eos.dp(m) < 0 ? lo : hi) = m;
  }
  const double sl = hi;
  // starting point: the outer roots of p = p0 at the pressure midway between the spinodals
  const double p_hi = eos.p(sv), p_lo = eos.p(sl) > 0 ? eos.p(sl) : 0.0;
  const double p0 = 0.5 * (p_hi + p_lo);
  auto root = [&](double lo_, double hi_) {  // p - p0 changes sign on [lo_, hi_]
    const bool up = eos.p(hi_) > eos.p(lo_);
    for (int it = 0; it < 300; ++it) {
      double m = 0.5 * (lo_ + hi_);
      ((eos.p(m) < p0) == up ? lo_ : hi_) = m;
    }
    return 0.5 * (lo_ + hi_);
  };
  double rv = root(1e-14, sv), rl = root(sl, rmax * (1 - 1e-9));
  for (int it = 0; it < 200; ++it) {
    const double F1 = eos.p(rv) - eos.p(rl);
    const double F2 = eos.mu(rv) - eos.mu(rl);
    const double pv = eos.dp(rv), pl = eos.dp(rl);
    // Jacobian [[pv, -pl], [pv/rv, -pl/rl]] (d mu = dp / rho at fixed T)
    const double j11 = pv, j12 = -pl, j21 = pv / rv, j22 = -pl / rl;
    const double det = j11 * j22 - j12 * j21;
    if (det == 0.0 || !std::isfinite(det)) return false;
    double dv = (F1 * j22 - F2 * j12) / det;
    double dl = (j11 * F2 - j21 * F1) / det;
    double lam = 1.0;
    while (lam > 1e-6) {  // damped step that keeps both roots on their branches
      double nv = rv - lam * dv, nl = rl - lam * dl;
      if (nv > 0 && nv < sv && nl > sl && nl < rmax) {
        rv = nv;
        rl = nl;
        break;
      }
      lam *= 0.5;
    }
    if (std::fabs(dv) < 1e-17 * rv && std::fabs(dl) < 1e-17 * rl) break;
  }
  const double scale = std::fabs(eos.p(rl)) + 1e-300;
  if (std::fabs(eos.p(rv) - eos.p(rl)) > 1e-10 * scale) return false;
  *rho_l = rl;
  *rho_v = rv;
  return std::isfinite(rl) && std::isfinite(rv) && rv < rl;
}

template <typename C>
static void fill(Consts<C>& k, const DevParams& p) {
  k.omega = C(p.omega);
  k.one_m_omega = C(1.0 - p.omega);
  k.K = C(3.0 * p.guo_pref);
  const double w[2] = {1.0 / 9.0, 1.0 / 36.0};
  for (int c = 0; c < 2; ++c) {
    k.wo45[c] = C(w[c] * 4.5 * p.omega);
    k.wo3[c] = C(w[c] * 3.0 * p.omega);
    k.wK3[c] = C(w[c] * 9.0 * p.guo_pref);
    k.wK[c] = C(w[c] * 3.0 * p.guo_pref);
  }
  k.gw1 = C(-p.G / 3.0);
  k.gw5 = C(-p.G / 12.0);
  k.G = C(p.G);
  k.psi0 = C(p.psi0);
  k.rho0 = C(p.rho0);
  k.a = C(p.a);
  k.b4 = C(p.b4);
  k.RT = C(p.RT);
  k.two_over_G = C(p.two_over_G);
  k.psi_wall = C(p.psi_wall);
  k.gx = C(p.gx);
  k.gy = C(p.gy);
  k.azC = C(p.azC);
  k.azcx = C(p.azcx);
  k.azcy = C(p.azcy);
  k.rho_ref = C(p.rho_ref);
}

void finalize_consts(DevParams& p) {
  // The deviation formats store f_a - w_a rho_ref; the FP32 step kernels hold rho_ref as a
  // float, the wall pass and the ledger as a double: one value, representable in both.
  p.rho_ref = (double)(float)p.rho_ref;
  fill(p.cd, p);
  fill(p.cf, p);
}

double host_psi(const DevParams& p, double rho) {
  if (p.eos == LBM_EOS_EXP) return p.psi0 * std::exp(-p.rho0 / rho);
  if (p.eos == LBM_EOS_CS) {
    double eta = p.b4 * rho, om = 1.0 - eta;
    double pr = rho * p.RT * (1.0 + eta + eta * eta - eta * eta * eta) / (om * om * om) -
                p.a * rho * rho;
    return std::sqrt(2.0 * (pr - rho / 3.0) / p.G);
  }
  return 0.0;
}

}  // namespace lbm
