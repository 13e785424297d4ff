"""Synthetic workloads: lattice sizes, geometry, model constants and seeds.

This module holds only problem definitions (numbers), none of the method's arithmetic, so both
the CUDA path and the CPU oracle can be driven from it.  Quantities that need the method (the
Maxwell coexistence densities, the pseudopotential) are resolved by each side itself.

Droplet on a cylinder (Sec. 3.2 geometry): a solid cylinder of radius r_cyl centred at
(L/2, round(0.35 L)) and a droplet of radius R_drop centred on the cylinder's top point,
tanh profile of width W.  The Carnahan-Starling fluid (a = 0.25, b = 4, R = 1) runs at
T = 0.86 T_c with tau = 1.  The virtual wall density is the vapour density ("rho_wall":
"vapour"); the paper leaves it free.
"""
from dataclasses import dataclass, field

SEED = 20190825

CS = dict(a=0.25, b=4.0, R=1.0, T_over_Tc=0.86, G=-1.0)
SCHEMES_C1 = ("mls", "bouzidi_l", "zhao_yong", "mod_a", "mod_b")


@dataclass
class DropletOnCylinder:
    name: str
    nx: int
    ny: int
    cyl: tuple          # (cx, cy, r)
    drop: tuple         # (cx, cy, R, W)
    tau: float = 1.0
    eos: dict = field(default_factory=lambda: dict(CS))
    rho_wall: str = "vapour"

    @property
    def circles(self):
        return [self.cyl]


def droplet_on_cylinder(L, r_cyl, r_drop, width=5.0, name=None):
    cy = round(0.35 * L)
    return DropletOnCylinder(name or "droplet_on_cylinder_%d" % L, L, L, (L / 2, cy, r_cyl),
                             (L / 2, cy + r_cyl, r_drop, width))


# 100 x 100, cylinder radius 15 at (50, 35), droplet radius 20 on top, 1000 steps.
SMALL = droplet_on_cylinder(100, 15.0, 20.0, name="droplet_on_cylinder_100x100")
# 4096 x 4096, cylinder radius 600, droplet radius 800.
LARGE = droplet_on_cylinder(4096, 600.0, 800.0, name="droplet_on_cylinder_4096x4096")
# the paper's own droplet test (Sec. 3.2): 300 x 350, cylinder R = 70 at (150, 130),
# exponential psi with G = -10/3, nu = 0.15 (tau = 0.95), periodic box.
PAPER_E2 = dict(nx=300, ny=350, cyl=(150.0, 130.0, 70.0), tau=0.95,
                eos=dict(G=-10.0 / 3.0, psi0=1.0, rho0=1.0), rho_l=2.783, rho_v=0.3675)


def batched_domains(n=512, seed=SEED, side_lo=64, side_hi=512):
    """The batched workload: n independent droplet-on-cylinder lattices with side uniform in
    {side_lo..side_hi}, cylinder radius 0.15-0.3 x side, droplet radius 0.2-0.35 x side,
    T/T_c uniform in [0.80, 0.90], tau uniform in [0.6, 1.2] (seeded)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        L = int(rng.integers(side_lo, side_hi + 1))
        r = float(rng.uniform(0.15, 0.3)) * L
        R = float(rng.uniform(0.2, 0.35)) * L
        t = float(rng.uniform(0.80, 0.90))
        tau = float(rng.uniform(0.6, 1.2))
        cy = round(0.35 * L)
        out.append(dict(name="batch_%d" % k, nx=L, ny=L, cyl=(L / 2, cy, r),
                        drop=(L / 2, cy + r, R, 5.0), tau=tau,
                        eos=dict(CS, T_over_Tc=t)))
    return out


SERVED_SCHEMES = ("mls", "bouzidi_l", "zhao_yong", "mod_a", "mod_b")


def served_requests(n=2000, rate=200.0, seed=SEED, side_lo=128, side_hi=1024, steps_lo=2000,
                    steps_hi=20000, schemes=SERVED_SCHEMES):
    """The served stream: n droplet-on-cylinder requests with Poisson arrivals (mean `rate` per
    second), lattice side log-uniform in [side_lo, side_hi], steps uniform in [steps_lo,
    steps_hi], boundary scheme drawn from `schemes`; geometry and fluid as the 4096^2 lattice,
    scaled (cylinder 0.15 L, droplet 0.2 L)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    out = []
    for k in range(n):
        L = int(round(np.exp(rng.uniform(np.log(side_lo), np.log(side_hi)))))
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        scheme = schemes[int(rng.integers(len(schemes)))]
        cy = round(0.35 * L)
        r = 0.15 * L
        out.append(dict(rid=k, arrival=float(t[k]), nx=L, ny=L, steps=steps, scheme=scheme,
                        cyl=(L / 2, cy, r), drop=(L / 2, cy + r, 0.2 * L, 5.0), tau=1.0,
                        eos=dict(CS)))
    return out
