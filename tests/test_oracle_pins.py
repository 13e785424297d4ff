"""Pins of the oracle's building blocks against mathematics and the paper, not against itself.

Each test states what fixes the expected value: a moment identity of the D2Q9 lattice, a closed
form, a published constant, or a brute-force computation written independently here.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
RNG = np.random.default_rng(20190825)


def _moments(f):
    return f.sum(), (f * EX).sum(), (f * EY).sum(), (f * EX * EX).sum(), (f * EX * EY).sum(), \
        (f * EY * EY).sum()


# --- Eq. (4): the D2Q9 equilibrium reproduces the Maxwellian moments up to second order -------
@pytest.mark.parametrize("k", range(6))
def test_feq_moments(k):
    rho = RNG.uniform(0.05, 3.0)
    ux, uy = RNG.uniform(-0.1, 0.1, 2)
    m0, mx, my, mxx, mxy, myy = _moments(O.feq(rho, ux, uy))
    assert m0 == pytest.approx(rho, rel=1e-14)
    assert mx == pytest.approx(rho * ux, abs=1e-15)
    assert my == pytest.approx(rho * uy, abs=1e-15)
    assert mxx == pytest.approx(rho / 3 + rho * ux * ux, rel=1e-14)
    assert myy == pytest.approx(rho / 3 + rho * uy * uy, rel=1e-14)
    assert mxy == pytest.approx(rho * ux * uy, abs=1e-15)


def test_feq_rest_weights():
    # u = 0: f_eq = w rho with w0 = 4/9, w1-4 = 1/9, w5-8 = 1/36 (Sec. 2.1)
    f = O.feq(2.0, 0.0, 0.0)
    assert np.allclose(f, 2.0 * np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4), rtol=0, atol=1e-16)


# --- Guo forcing: zeroth moment 0, first (1 - 1/2tau) F, second (1 - 1/2tau)(uF + Fu) ---------
@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_guo_moments(tau):
    ux, uy, Fx, Fy = RNG.uniform(-0.1, 0.1, 4)
    m0, mx, my, mxx, mxy, myy = _moments(O.guo(tau, ux, uy, Fx, Fy))
    c = 1 - 1 / (2 * tau)
    assert abs(m0) < 1e-16
    assert mx == pytest.approx(c * Fx, rel=1e-13)
    assert my == pytest.approx(c * Fy, rel=1e-13)
    assert mxx == pytest.approx(c * 2 * ux * Fx, rel=1e-12, abs=1e-17)
    assert myy == pytest.approx(c * 2 * uy * Fy, rel=1e-12, abs=1e-17)
    assert mxy == pytest.approx(c * (ux * Fy + uy * Fx), rel=1e-12, abs=1e-17)


# --- Eq. (2) with Eq. (5): collision keeps mass and adds exactly F to the momentum -----------
@pytest.mark.parametrize("tau", [0.55, 1.0, 1.9])
def test_collision_invariants(tau):
    f = O.feq(1.3, 0.05, -0.02) + RNG.uniform(-0.01, 0.01, 9)
    Fx, Fy = RNG.uniform(-1e-3, 1e-3, 2)
    fs = O.collide_node(f, tau, Fx, Fy)
    assert fs.sum() == pytest.approx(f.sum(), rel=1e-15)
    assert (fs * EX).sum() == pytest.approx((f * EX).sum() + Fx, abs=1e-15)
    assert (fs * EY).sum() == pytest.approx((f * EY).sum() + Fy, abs=1e-15)


def test_collision_tau_one_is_equilibrium():
    # tau = 1, F = 0: f* = f_eq(rho, u) exactly as Eq. (2) states
    f = O.feq(0.9, 0.03, 0.01) + RNG.uniform(-0.01, 0.01, 9)
    rho, mx, my = f.sum(), (f * EX).sum(), (f * EY).sum()
    assert np.allclose(O.collide_node(f, 1.0, 0.0, 0.0), O.feq(rho, mx / rho, my / rho),
                       rtol=0, atol=1e-16)


# --- Eq. (16): closed form on a sinusoidal psi field ------------------------------------------
def test_force_sinusoid_closed_form():
    # psi = c + A sin(k x): sum_a w_a psi(x + e_a) e_ax = A sin(k) cos(k x) for the weights
    # 1/3 (axis) and 1/12 (diagonal); the y component vanishes.
    nx, ny, G = 32, 6, -10.0 / 3.0
    k = 2 * math.pi / nx
    x = np.arange(nx)
    psi = np.tile(0.7 + 0.2 * np.sin(k * x), (ny, 1))
    Fx, Fy = O.force_from_psi(psi, G)
    expect = -G * psi * 0.2 * math.sin(k) * np.cos(k * x)[None, :]
    assert np.max(np.abs(Fx - expect)) < 1e-15
    assert np.max(np.abs(Fy)) < 1e-15
    Fx2, Fy2 = O.force_from_psi(psi.T.copy(), G)  # same field along y
    assert np.max(np.abs(Fy2 - expect.T)) < 1e-15
    assert np.max(np.abs(Fx2)) < 1e-15


def test_force_pairwise_total_zero():
    # Pairs (x, x + e) and (x + e, x) cancel on a periodic lattice: sum_x F(x) = 0.
    psi = RNG.uniform(0.2, 1.0, (17, 23))
    Fx, Fy = O.force_from_psi(psi, -1.0)
    assert abs(Fx.sum()) < 1e-13 and abs(Fy.sum()) < 1e-13
    assert np.abs(Fx).max() > 1e-3


# --- Carnahan-Starling: critical point and Maxwell construction -------------------------------
def test_cs_critical_published_constants():
    # Published CS critical point: eta_c = b rho_c / 4 = 0.13044, T_c = 0.3773 a / (b R).
    for a, b, R in [(0.25, 4.0, 1.0), (1.0, 4.0, 1.0), (0.5, 2.0, 0.7)]:
        Tc, rhoc = O.cs_critical(a, b, R)
        assert b * rhoc / 4 == pytest.approx(0.13044, abs=5e-5)
        assert Tc * b * R / a == pytest.approx(0.3773, abs=5e-5)
        # independent check of the critical conditions by finite differences
        h = 1e-4 * rhoc
        p = lambda r: O.cs_pressure(a, b, R, Tc, r)
        d1 = (p(rhoc + h) - p(rhoc - h)) / (2 * h)
        d2 = (p(rhoc + h) - 2 * p(rhoc) + p(rhoc - h)) / h**2
        scale = p(rhoc) / rhoc
        assert abs(d1) < 1e-7 * scale and abs(d2) < 1e-4 * scale / rhoc


@pytest.mark.parametrize("t", [0.7, 0.8, 0.86, 0.95])
def test_cs_maxwell_equal_area(t):
    a, b, R = 0.25, 4.0, 1.0
    Tc, rhoc = O.cs_critical(a, b, R)
    T = t * Tc
    rl, rv = O.cs_coexistence(a, b, R, T)
    assert rv < rhoc < rl
    p = lambda r: O.cs_pressure(a, b, R, T, r)
    p0 = p(rl)
    assert p(rv) == pytest.approx(p0, rel=1e-9, abs=1e-15)
    area, _ = integrate.quad(lambda r: (p(r) - p0) / r**2, rv, rl, epsabs=1e-14, epsrel=1e-12,
                             limit=200)
    scale = integrate.quad(lambda r: abs(p(r) - p0) / r**2, rv, rl, limit=200)[0]
    assert abs(area) < 1e-9 * scale


def test_cs_psi_pressure_identity():
    # The EOS is recovered from psi through p = rho/3 + G psi^2 / 2 (Eq. (16) weights).  This
    # pins the sign of G and the factor 2 inside psi.
    Tc, _ = O.cs_critical(0.25, 4.0, 1.0)
    for rho in [0.02, 0.1, 0.3]:
        ps = O.psi(rho, eos=O.EOS_CS, G=-1.0, a=0.25, b=4.0, R=1.0, T=0.86 * Tc)
        assert rho / 3 + (-1.0) * ps * ps / 2 == pytest.approx(
            O.cs_pressure(0.25, 4.0, 1.0, 0.86 * Tc, rho), rel=1e-13)


def test_psi_exponential():
    for rho in [0.3, 1.0, 2.8]:
        assert O.psi(rho, eos=O.EOS_EXP, psi0=1.0, rho0=1.0) == pytest.approx(math.exp(-1 / rho),
                                                                               rel=1e-15)


# --- Geometry: flags, links and q of Eq. (6) against a brute-force enumeration ----------------
def _brute_geometry(nx, ny, circles, wall_lo=0.0, wall_hi=0.0):
    def solid(i, j):
        if wall_lo > 0 and j == 0:
            return True
        if wall_hi > 0 and j == ny - 1:
            return True
        for c in circles:
            d2 = (i - c[0]) ** 2 + (j - c[1]) ** 2
            inside = d2 <= c[2] ** 2
            if (len(c) > 3 and c[3]) and d2 >= c[2] ** 2:
                return True
            if not (len(c) > 3 and c[3]) and inside:
                return True
        return False

    def crossing(i, j, a, c):
        # bisection on g(t) = |x_b + t e - c|^2 - r^2 over (0, 1]
        out = len(c) > 3 and c[3]
        g = lambda t: (i + t * EX[a] - c[0]) ** 2 + (j + t * EY[a] - c[1]) ** 2 - c[2] ** 2
        lo, hi = 0.0, 1.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            inside_solid = g(mid) >= 0 if out else g(mid) <= 0
            if inside_solid:
                hi = mid
            else:
                lo = mid
        return hi

    sol = np.zeros((ny, nx), bool)
    links = []
    for j in range(ny):
        for i in range(nx):
            sol[j, i] = solid(i, j)
    flags = sol.astype(np.uint8)
    for j in range(ny):
        for i in range(nx):
            if sol[j, i]:
                continue
            for a in range(1, 9):
                si, sj = (i + EX[a]) % nx, (j + EY[a]) % ny
                if not sol[sj, si]:
                    continue
                flags[j, i] |= 2
                q = 2.0
                if wall_lo > 0 and sj == 0:
                    q = min(q, wall_lo)
                if wall_hi > 0 and sj == ny - 1:
                    q = min(q, wall_hi)
                for c in circles:
                    d2 = (si - c[0]) ** 2 + (sj - c[1]) ** 2
                    out = len(c) > 3 and c[3]
                    if (out and d2 >= c[2] ** 2) or (not out and d2 <= c[2] ** 2):
                        q = min(q, crossing(i, j, a, c))
                links.append((j * nx + i, a, q))
    return flags, links


@pytest.mark.parametrize("case", [
    dict(nx=40, ny=36, circles=[(20, 15, 7.0)]),
    dict(nx=41, ny=37, circles=[(19.3, 17.8, 6.55), (33.1, 9.4, 3.2)]),
    dict(nx=48, ny=48, circles=[(23.7, 24.2, 9.3), (23.7, 24.2, 21.1, 1)]),
    dict(nx=12, ny=20, circles=[], wall_q_lo=0.3, wall_q_hi=0.8),
])
def test_geometry_brute_force(case):
    s = O.OracleSim(case["nx"], case["ny"], 1.0, circles=case["circles"],
                    wall_q_lo=case.get("wall_q_lo", 0.0), wall_q_hi=case.get("wall_q_hi", 0.0))
    flags, links = _brute_geometry(case["nx"], case["ny"], case["circles"],
                                   case.get("wall_q_lo", 0.0), case.get("wall_q_hi", 0.0))
    assert np.array_equal(s.flags(), flags)
    node, d, q = s.links()
    assert len(node) == len(links) > 0
    assert [(int(n), int(a)) for n, a in zip(node, d)] == [(n, a) for n, a, _ in links]
    qb = np.array([x[2] for x in links])
    assert np.all((q > 0) & (q <= 1))
    # Near-tangent crossings are ill-conditioned (q moves by ~sqrt(eps)); there the residual of
    # the circle equation is checked instead of the bisection value.
    nx = case["nx"]
    for k in range(len(q)):
        i, j, a = int(node[k]) % nx, int(node[k]) // nx, int(d[k])
        slope = 1.0
        resid = 0.0
        for c in case["circles"]:
            px, py = i + q[k] * EX[a] - c[0], j + q[k] * EY[a] - c[1]
            gk = px * px + py * py - c[2] ** 2
            if abs(gk) <= abs(resid) or resid == 0.0:
                resid, slope = gk, abs(2 * (EX[a] * px + EY[a] * py))
        if slope > 1e-3 or not case["circles"]:
            assert abs(q[k] - qb[k]) < 1e-12
        else:
            assert abs(resid) < 1e-12 * max(1.0, max(c[2] for c in case["circles"]) ** 2)


# --- Eq. (3): with tau -> infinity and no force, each plane translates by e_a per step ------
def test_streaming_translates_planes():
    nx, ny = 11, 7
    s = O.OracleSim(nx, ny, 1e15)
    f = RNG.uniform(0.01, 0.2, (9, ny, nx))
    s.set_f(f)
    s.step(3)
    g = s.get_f()
    for a in range(9):
        expect = np.roll(f[a], shift=(3 * EY[a], 3 * EX[a]), axis=(0, 1))
        assert np.max(np.abs(g[a] - expect)) < 1e-12


# --- Eqs. (7), (8), (10) and (12) at q = 1, tau = 1 -----------------------------------------
@pytest.mark.parametrize("scheme", [O.FH, O.MLS, O.MOD_A, O.BOUZIDI_L])
def test_wall_on_solid_node_gives_symmetric_equilibrium(scheme):
    # Uniform state f = f_eq(rho, u) next to flat walls through the solid nodes (q = 1), tau = 1,
    # no force: the collision returns f_eq.  Eq. (10) then has chi = 1 and u_s = 0, so Eq. (7)
    # returns the ghost equilibrium of Eq. (8) with e.u_s = 0, i.e. the part of f_eq_a that is
    # even in e_a: (f_eq_a + f_eq_abar) / 2.  Linear Bouzidi at q = 1 (Eq. (12)) averages
    # f*_a and f*_abar, which is the same mean.  Scheme A keeps MLS's incoming values.
    rho, ux, uy = 1.1, 0.08, 0.03
    nx, ny = 4, 6
    s = O.OracleSim(nx, ny, 1.0, scheme=scheme, wall_q_lo=1.0, wall_q_hi=1.0)
    s.init_fields(np.full((ny, nx), rho), np.full((ny, nx), ux), np.full((ny, nx), uy))
    s.step(1)
    f = s.get_f()
    feq = O.feq(rho, ux, uy)
    opp = [0, 3, 4, 1, 2, 7, 8, 5, 6]
    for j, into_wall in ((1, (4, 7, 8)), (ny - 2, (2, 5, 6))):
        for a in into_wall:
            expect = 0.5 * (feq[a] + feq[opp[a]])
            assert np.max(np.abs(f[opp[a], j, :] - expect)) < 1e-16, (a, j)
    # not vacuous: the incoming values differ from halfway bounce-back's f*_a = f_eq_a
    assert abs(0.5 * (feq[7] + feq[5]) - feq[7]) > 1e-3
