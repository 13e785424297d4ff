"""The paper's own experiments on the GPU path, shortened: what the paper states about mass.

- Sec. 3.2 (Fig. 8): on its 300 x 350 droplet-on-cylinder run (exponential psi, |G| = 10/3,
  nu = 0.15) the Zhao-Yong scheme loses mass fastest, the original ghost-node scheme (MLS) also
  leaks, and (Sec. 4.2, Fig. 11) the modified schemes A and B keep it.
- Sec. 3.1 (Fig. 5): static flow under gravity between flat walls at fraction q; MLS conserves
  mass at q = 1/2 only and Zhao-Yong leaks more than MLS.
"""
import numpy as np
import pytest

from paper_1908_09235_gb300 import lbm

pytestmark = pytest.mark.gpu


def _droplet_mass_change(scheme, steps):
    eos = lbm.make_eos(lbm.EOS_EXP, G=-10.0 / 3.0, psi0=1.0, rho0=1.0, rho_wall=1.5)
    lat = lbm.Lattice(300, 350, 0.95, scheme, circles=[(150.0, 130.0, 70.0)], eos=eos)
    lat.init_droplet(150.0, 200.0, 50.0, 5.0, 2.783, 0.3675)
    m0 = lat.mass()
    lat.step(steps)
    m = lat.mass()
    lat.close()
    return m / m0 - 1.0


def test_paper_droplet_on_cylinder_mass(gpu_lib):
    d = {s: _droplet_mass_change(s, 1000)
         for s in (lbm.ZHAO_YONG, lbm.MLS, lbm.MOD_A, lbm.MOD_B, lbm.HBB)}
    print({k: "%.3e" % v for k, v in d.items()})
    # the original schemes lose mass, Zhao-Yong the most (a quarter or more by step 1000)
    assert d[lbm.ZHAO_YONG] < -0.2
    assert d[lbm.ZHAO_YONG] < d[lbm.MLS] < -1e-3
    # the modified schemes and halfway bounce-back keep it to round-off
    for s in (lbm.MOD_A, lbm.MOD_B, lbm.HBB):
        assert abs(d[s]) < 1e-10, (s, d[s])


def _gravity_mass_change(scheme, q, steps):
    nx, ny = 100, 50
    lat = lbm.Lattice(nx, ny, 1.0, scheme, wall_q_lo=q, wall_q_hi=q,
                      eos=lbm.make_eos(lbm.EOS_NONE, gy=-0.001))
    lat.init_fields(np.ones(nx * ny))
    m0 = lat.mass()
    lat.step(steps)
    m = lat.mass()
    lat.close()
    return abs(m / m0 - 1.0)


def test_paper_gravity_leakage(gpu_lib):
    assert _gravity_mass_change(lbm.MLS, 0.5, 5000) < 1e-11
    mls = _gravity_mass_change(lbm.MLS, 0.3, 5000)
    zy = _gravity_mass_change(lbm.ZHAO_YONG, 0.3, 5000)
    assert 1e-4 < mls < zy, (mls, zy)
    for s in (lbm.MOD_A, lbm.MOD_B):
        assert _gravity_mass_change(s, 0.3, 5000) < 1e-11
