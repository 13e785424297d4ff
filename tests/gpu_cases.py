"""Shared set-up of the GPU-vs-oracle cases: one description drives both sides.

Both sides receive the same problem definition (sizes, geometry, model constants, initial
condition recipe); each resolves method quantities (coexistence densities, psi) itself.
"""
import numpy as np

import oracle as O
from paper_1908_09235_gb300 import lbm, workloads

SCHEME_ORACLE = {lbm.HBB: O.HBB, lbm.FH: O.FH, lbm.MLS: O.MLS, lbm.BOUZIDI_L: O.BOUZIDI_L,
                 lbm.BOUZIDI_Q: O.BOUZIDI_Q, lbm.ZHAO_YONG: O.ZHAO_YONG, lbm.MOD_A: O.MOD_A,
                 lbm.MOD_B: O.MOD_B, lbm.BAO: O.BAO, lbm.BOUZIDI_L_A: O.BOUZIDI_L_A}


class Case:
    """kind: 'cs' (Carnahan-Starling droplet), 'exp' (exponential psi droplet), 'none' (single
    phase with body force).  init: ('droplet', cx, cy, R, W) or ('fields', rho, ux, uy)."""

    def __init__(self, nx, ny, tau, kind, circles=(), wall_q_lo=0.0, wall_q_hi=0.0, init=None,
                 rho_wall=None, gx=0.0, gy=0.0, azim=None, drop_rho=None, G=None):
        self.nx, self.ny, self.tau, self.kind = nx, ny, tau, kind
        self.circles = list(circles)
        self.wall_q_lo, self.wall_q_hi = wall_q_lo, wall_q_hi
        self.init = init
        self.gx, self.gy = gx, gy
        self.azim = azim
        self.rho_wall = rho_wall
        self.drop_rho = drop_rho
        self.G = G

    # ---- GPU side ----
    def gpu(self, scheme, precision=lbm.FP64, graph_steps=0):
        kw = dict(gx=self.gx, gy=self.gy)
        if self.azim:
            kw.update(azim_C=self.azim[0], azim_cx=self.azim[1], azim_cy=self.azim[2])
        if self.kind == "cs":
            eos = lbm.make_eos(lbm.EOS_CS, **workloads.CS, **kw)
            rl, rv = lbm.lbm_coexistence(eos)
            eos.rho_wall = rv if self.rho_wall is None else self.rho_wall
            drop = (rl, rv)
        elif self.kind == "exp":
            eos = lbm.make_eos(lbm.EOS_EXP, G=self.G if self.G else -10.0 / 3.0, psi0=1.0,
                               rho0=1.0, rho_wall=self.rho_wall or 1.5, **kw)
            drop = self.drop_rho or (2.783, 0.3675)
        else:
            eos = lbm.make_eos(lbm.EOS_NONE, **kw)
            drop = None
        lat = lbm.Lattice(self.nx, self.ny, self.tau, scheme, circles=self.circles,
                          wall_q_lo=self.wall_q_lo, wall_q_hi=self.wall_q_hi, eos=eos,
                          precision=precision, graph_steps=graph_steps)
        self._init(lat, drop)
        return lat

    # ---- oracle side ----
    def oracle(self, scheme):
        kw = dict(gx=self.gx, gy=self.gy)
        if self.azim:
            kw.update(azim_C=self.azim[0], azim_cx=self.azim[1], azim_cy=self.azim[2])
        if self.kind == "cs":
            c = workloads.CS
            Tc, _ = O.cs_critical(c["a"], c["b"], c["R"])
            rl, rv = O.cs_coexistence(c["a"], c["b"], c["R"], c["T_over_Tc"] * Tc)
            s = O.OracleSim(self.nx, self.ny, self.tau, scheme=SCHEME_ORACLE[scheme],
                            circles=self.circles, wall_q_lo=self.wall_q_lo,
                            wall_q_hi=self.wall_q_hi, eos=O.EOS_CS, G=c["G"], a=c["a"],
                            b=c["b"], R=c["R"], T_over_Tc=c["T_over_Tc"],
                            rho_wall=rv if self.rho_wall is None else self.rho_wall, **kw)
            drop = (rl, rv)
        elif self.kind == "exp":
            s = O.OracleSim(self.nx, self.ny, self.tau, scheme=SCHEME_ORACLE[scheme],
                            circles=self.circles, wall_q_lo=self.wall_q_lo,
                            wall_q_hi=self.wall_q_hi, eos=O.EOS_EXP,
                            G=self.G if self.G else -10.0 / 3.0, psi0=1.0, rho0=1.0,
                            rho_wall=self.rho_wall or 1.5, **kw)
            drop = self.drop_rho or (2.783, 0.3675)
        else:
            s = O.OracleSim(self.nx, self.ny, self.tau, scheme=SCHEME_ORACLE[scheme],
                            circles=self.circles, wall_q_lo=self.wall_q_lo,
                            wall_q_hi=self.wall_q_hi, **kw)
            drop = None
        self._init(s, drop)
        return s

    def _init(self, sim, drop):
        if self.init[0] == "droplet":
            sim.init_droplet(*self.init[1:], *drop)
        else:
            sim.init_fields(*self.init[1:])


def c0_case():
    w = workloads.SMALL
    return Case(w.nx, w.ny, w.tau, "cs", circles=w.circles, init=("droplet",) + tuple(w.drop))


def compare_fields(a, b):
    """max-abs difference of (rho, ux, uy) over nodes where the oracle is finite; the solid
    pattern (NaN) must agree exactly."""
    out = []
    for x, y in zip(a, b):
        assert np.array_equal(np.isnan(x), np.isnan(y))
        m = np.isfinite(y)
        out.append(float(np.max(np.abs(x[m] - y[m]))) if m.any() else 0.0)
    return out
