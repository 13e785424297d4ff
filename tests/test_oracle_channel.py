"""Oracle pins for the flow-past-a-cylinder set-up of Sec. 4.2: the momentum-exchange force on
solid bodies and the channel ends (Zou-He velocity inlet, fully developed outlet).

Each pin is a fact fixed by the mathematics, not a restatement of the oracle's code:
- at rest (uniform density, no force) the momentum exchange on any closed body is zero: every
  lattice line enters and leaves the body equally often, so the cut links come in opposite pairs
  with equal weights;
- per step, the fluid's momentum changes by exactly the body force it received minus the
  momentum the walls took (collision with Guo forcing adds exactly F, streaming moves momentum);
- at steady state the walls take exactly the body force (the drag balances the driving force);
- the Zou-He rule imposes the inlet velocity exactly, and the outlet copies the populations
  entering from the right.
"""
import numpy as np
import pytest

import oracle as O

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
ALL = (O.HBB, O.FH, O.MLS, O.BOUZIDI_L, O.BOUZIDI_Q, O.ZHAO_YONG, O.MOD_A, O.MOD_B, O.BAO,
       O.BOUZIDI_L_A)
CONSERVING = (O.HBB, O.MOD_A, O.MOD_B)
BODIES = [(15.3, 16.6, 6.2), (31.7, 9.4, 3.3)]


def _sim(scheme, nx=48, ny=32, tau=0.9, gx=0.0, circles=BODIES):
    s = O.OracleSim(nx, ny, tau, scheme=scheme, circles=circles, eos=O.EOS_NONE, gx=gx)
    s.init_fields(np.ones(nx * ny))
    return s


def _momentum(s, fluid):
    f = s.get_f()
    return ((f * EX[:, None, None]).sum(0)[fluid].sum(),
            (f * EY[:, None, None]).sum(0)[fluid].sum())


@pytest.mark.parametrize("scheme", ALL)
def test_force_on_bodies_at_rest_is_zero(scheme):
    s = _sim(scheme)
    s.step(5)
    fx, fy = s.force()
    # each cut link carries 2 w_a rho e_a at rest; pairs cancel to round-off
    assert abs(fx) < 1e-14 and abs(fy) < 1e-14


@pytest.mark.parametrize("scheme", ALL)
def test_momentum_exchange_closes_the_momentum_budget(scheme):
    g = 2e-5
    s = _sim(scheme, gx=g)
    fluid = (s.flags() & 1) == 0
    s.step(150)  # a developing flow: every term of the budget is non-zero
    for _ in range(3):
        px0, py0 = _momentum(s, fluid)
        rho, _, _ = s.fields()
        body = g * rho[fluid].sum()
        s.step(1)
        px1, py1 = _momentum(s, fluid)
        fx, fy = s.force()
        assert abs(fx) > 1e-4  # the wall takes momentum
        assert abs((px1 - px0) - (body - fx)) < 1e-12
        assert abs((py1 - py0) - (0.0 - fy)) < 1e-12


@pytest.mark.parametrize("scheme", CONSERVING)
def test_drag_balances_the_body_force_at_steady_state(scheme):
    # periodic box driven by a body force: at steady state the momentum exchange with the
    # cylinder equals the total body force on the fluid.  Halfway bounce-back keeps a
    # period-2 oscillation at tau = 1, so the force is averaged over four steps.
    g = 1e-5
    s = _sim(scheme, nx=32, ny=32, tau=1.0, gx=g, circles=[(15.3, 16.6, 6.2)])
    fluid = (s.flags() & 1) == 0
    s.step(8000)
    wall, body = 0.0, 0.0
    for _ in range(4):
        rho, _, _ = s.fields()
        body += g * rho[fluid].sum()
        s.step(1)
        wall += s.force()[0]
    assert abs(wall / body - 1.0) < 1e-9


def test_zou_he_inlet_and_fully_developed_outlet():
    u_in = 0.06
    s = _sim(O.MOD_B, nx=60, ny=24, circles=[(20.2, 12.3, 4.1)])
    s.set_inflow(u_in)
    s.step(40)
    f = s.get_f()
    rho = f.sum(0)[:, :3]  # the inlet columns (no solid there)
    ux = (f * EX[:, None, None]).sum(0)[:, :3] / rho
    uy = (f * EY[:, None, None]).sum(0)[:, :3] / rho
    # the inlet column carries exactly the prescribed velocity (no body force here)
    assert np.max(np.abs(ux[:, 0] - u_in)) < 1e-15
    assert np.max(np.abs(uy[:, 0])) < 1e-15
    # the populations entering the outlet column are those of the column before it
    for a in (3, 6, 7):
        assert np.array_equal(f[a, :, -1], f[a, :, -2])
    # the flow has reached the cylinder and pushes it downstream
    s.step(200)
    assert s.force()[0] > 0.0
