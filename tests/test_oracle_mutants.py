"""Planted mistakes in a copy of the oracle must each fail one of the oracle's pins.

The oracle is only as trustworthy as the pins that hold it to the paper and to mathematics.
Each case below copies ``oracle/`` to a temporary directory, makes one plausible slip in
``lbm_oracle.c`` (a dropped term, a wrong sign, index or denominator, a transposed operand),
builds that copy and runs, in a fresh interpreter that imports the mutated copy, the pin that
is meant to catch it.  The case passes when that pin fails with an AssertionError.  Nothing here
touches the GPU or the oracle in the repository.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")

# (name, text in oracle/lbm_oracle.c, replacement, pin run against the mutated copy).
# In a pin, P is tests/test_oracle_physics.py, PIN tests/test_oracle_pins.py, CH
# tests/test_oracle_channel.py and O the mutated oracle.
MUTANTS = [
    # Eq. (9): Filippova-Haenel, q < 1/2
    ("fh_chi_denominator", "*chi = (2.0 * q - 1.0) / (tau - 1.0);",
     "*chi = (2.0 * q - 1.0) / (tau - 2.0);", "P.test_poiseuille_second_order(O.FH, 0.8)"),
    ("fh_us_dropped", "      *usx = s->ux[n];\n      *usy = s->uy[n];",
     "      *usx = 0.0;\n      *usy = 0.0;", "P.test_poiseuille_second_order(O.FH, 0.8)"),
    # Eq. (11): MLS, q < 1/2
    ("mls_chi_denominator", "*chi = (2.0 * q - 1.0) / (tau - 2.0);",
     "*chi = (2.0 * q - 1.0) / (tau - 1.0);", "P.test_poiseuille_second_order(O.MLS, 0.8)"),
    ("mls_uf_wrong_side", "int nf = wrapi(j - EY[a], s->ny) * s->nx + wrapi(i - EX[a], s->nx);\n"
     "      if (s->solid[nf]) return 0;",
     "int nf = wrapi(j + EY[a], s->ny) * s->nx + wrapi(i + EX[a], s->nx);\n"
     "      if (s->solid[nf]) return 0;", "P.test_poiseuille_second_order(O.MLS, 0.8)"),
    # Eq. (10): q >= 1/2
    ("ghost_chi_q_ge_half", "*chi = (2.0 * q - 1.0) / tau;", "*chi = (2.0 * q - 1.0) / (tau - 1.0);",
     "P.test_poiseuille_second_order(O.MLS, 0.8)"),
    ("ghost_us_sign", "*usx = (q - 1.0) / q * s->ux[n];", "*usx = (1.0 - q) / q * s->ux[n];",
     "P.test_poiseuille_second_order(O.MLS, 0.8)"),
    # Eq. (8): the quadratic term uses u_b, not u_s
    ("ghost_bracket_quadratic_us", "4.5 * eub * eub", "4.5 * eus * eus",
     "PIN.test_wall_on_solid_node_gives_symmetric_equilibrium(O.MLS)"),
    ("ghost_bracket_square_us", "1.5 * (ubx * ubx + uby * uby)", "1.5 * (usx * usx + usy * usy)",
     "PIN.test_wall_on_solid_node_gives_symmetric_equilibrium(O.MLS)"),
    ("ghost_bracket_linear_term", "1.0 + 3.0 * eus", "1.0 + 3.0 * eub",
     "P.test_poiseuille_second_order(O.MLS, 0.8)"),
    # Eq. (12): linear Bouzidi
    ("bouzidi_l_lt_half_opposite", "val = 2.0 * q * fo + (1.0 - 2.0 * q) * s->fs[a * N + nf];\n"
     "          } else {\n            val = 1.0 / (2.0 * q)",
     "val = 2.0 * q * fo + (1.0 - 2.0 * q) * s->fs[ab * N + nf];\n"
     "          } else {\n            val = 1.0 / (2.0 * q)",
     "P.test_poiseuille_second_order(O.BOUZIDI_L, 0.8)"),
    ("bouzidi_l_ge_half_same_direction",
     "          } else {\n            val = 1.0 / (2.0 * q) * fo + (2.0 * q - 1.0) / (2.0 * q) * "
     "s->fs[ab * N + n];\n          }\n          break;\n        case OR_BOUZIDI_Q:",
     "          } else {\n            val = 1.0 / (2.0 * q) * fo + (2.0 * q - 1.0) / (2.0 * q) * "
     "s->fs[a * N + n];\n          }\n          break;\n        case OR_BOUZIDI_Q:",
     "P.test_poiseuille_second_order(O.BOUZIDI_L, 0.8)"),
    # Eq. (13): quadratic Bouzidi
    ("bouzidi_q_lt_half_weight", "(1.0 - 4.0 * q * q)", "(1.0 - 2.0 * q * q)",
     "P.test_poiseuille_second_order(O.BOUZIDI_Q, 0.8)"),
    ("bouzidi_q_lt_half_xff_weight", "q * (1.0 - 2.0 * q) * s->fs[a * N + nff];",
     "q * (1.0 + 2.0 * q) * s->fs[a * N + nff];", "P.test_poiseuille_second_order(O.BOUZIDI_Q, 0.8)"),
    ("bouzidi_q_ge_half_xf_direction", "(2.0 * q - 1.0) / (2.0 * q + 1.0) * s->fs[ab * N + nf];",
     "(2.0 * q - 1.0) / (2.0 * q + 1.0) * s->fs[a * N + nf];",
     "P.test_poiseuille_second_order(O.BOUZIDI_Q, 0.8)"),
    # Eq. (14): Zhao-Yong, post-collision f*_abar and pre-collision f_a
    ("zhao_yong_pre_post_swapped",
     "2.0 * q / (1.0 + 2.0 * q) * s->fs[ab * N + n] + 1.0 / (1.0 + 2.0 * q) * s->f[a * N + n];",
     "2.0 * q / (1.0 + 2.0 * q) * s->f[ab * N + n] + 1.0 / (1.0 + 2.0 * q) * s->fs[a * N + n];",
     "P.test_poiseuille_second_order(O.ZHAO_YONG, 0.8)"),
    ("zhao_yong_weight", "2.0 * q / (1.0 + 2.0 * q) * s->fs[ab * N + n]",
     "q / (1.0 + 2.0 * q) * s->fs[ab * N + n]", "P.test_poiseuille_second_order(O.ZHAO_YONG, 0.8)"),
    # Eq. (15) and Eq. (18): scheme A
    ("leak_sign", "double dm = sum_out - sum_in; /* Eq. (15) */",
     "double dm = sum_in - sum_out; /* Eq. (15) */", "P.test_closed_box_mass_conserved(O.MOD_A)"),
    ("scheme_a_from_streamed_rest", "s->fn[n] = s->fs[n] + dm;", "s->fn[n] = s->f[n] + dm;",
     "P.test_closed_box_mass_conserved(O.MOD_A)"),
    ("scheme_a_on_fh", "if (!ghost_params(s, scheme == OR_FH, n, a, q, &chi, &usx, &usy)) {",
     "if (!ghost_params(s, scheme == OR_FH || scheme == OR_MOD_A, n, a, q, &chi, &usx, &usy)) {",
     "P.test_flat_walls_modified_schemes_reduce_to_mls(O.MOD_A)"),
    ("scheme_b_on_fh", "if (!ghost_params(s, 0, n, a, s->lq[l], &chi, &usx, &usy)) continue;",
     "if (!ghost_params(s, 1, n, a, s->lq[l], &chi, &usx, &usy)) continue;",
     "P.test_closed_box_mass_conserved(O.MOD_B)"),
    # Eq. (22): scheme B's fictitious density
    ("scheme_b_numerator_direction", "num += chi * s->fs[a * N + n];",
     "num += chi * s->fs[OPP[a] * N + n];", "P.test_closed_box_mass_conserved(O.MOD_B)"),
    ("scheme_b_chi_dropped_from_denominator", "den += chi * br;", "den += br;",
     "P.test_closed_box_mass_conserved(O.MOD_B)"),
    ("scheme_b_uses_rho_b", "double rr = (scheme == OR_MOD_B || scheme == OR_BAO) ? rho_s : rho_b;",
     "double rr = (scheme == OR_BAO) ? rho_s : rho_b;", "P.test_closed_box_mass_conserved(O.MOD_B)"),
    # Eq. (23): Bao keeps chi out of the sums
    ("bao_becomes_b", "num += s->fs[a * N + n];\n          den += br;",
     "num += chi * s->fs[a * N + n];\n          den += chi * br;", "P.test_bao_differs_from_scheme_b()"),
    # Eq. (4), Guo forcing, Eq. (5), Eq. (2)
    ("feq_quadratic_coefficient", "out[a] = W[a] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);",
     "out[a] = W[a] * rho * (1.0 + 3.0 * eu + 4.0 * eu * eu - 1.5 * uu);",
     "[PIN.test_feq_moments(k) for k in range(6)]"),
    ("guo_velocity_sign", "double cx = 3.0 * (EX[a] - ux) + 9.0 * eu * EX[a];",
     "double cx = 3.0 * (EX[a] + ux) + 9.0 * eu * EX[a];", "PIN.test_guo_moments(1.0)"),
    ("guo_prefactor", "double pref = 1.0 - 1.0 / (2.0 * tau);", "double pref = 1.0 - 1.0 / tau;",
     "PIN.test_guo_moments(0.6)"),
    ("half_force_dropped", "s->ux[n] = (mx + 0.5 * s->Fx[n]) / s->rho[n];",
     "s->ux[n] = (mx + s->Fx[n]) / s->rho[n];", "CH.test_drag_balances_the_body_force_at_steady_state(O.HBB)"),
    ("half_force_dropped_y", "s->uy[n] = (my + 0.5 * s->Fy[n]) / s->rho[n];",
     "s->uy[n] = (my + s->Fy[n]) / s->rho[n];", "P.test_hydrostatic_profile()"),
    ("collision_relaxation", "s->fs[a * NN + n] = fv - (fv - feq[a]) / tau + fa[a];",
     "s->fs[a * NN + n] = fv - (fv - feq[a]) * tau + fa[a];", "P.test_poiseuille_second_order(O.MLS, 0.8)"),
    # Eq. (16) and the pseudopotentials
    ("force_sign", "Fx = -s->p.G * s->psi[n] * sx;", "Fx = s->p.G * s->psi[n] * sx;",
     "P.test_momentum_conserved_two_phase_periodic()"),
    ("force_diagonal_weight", "1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0};",
     "1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0, 1.0 / 6.0};", "PIN.test_force_sinusoid_closed_form()"),
    ("psi_exponential_sign", "return p->psi0 * exp(-p->rho0 / rho);",
     "return p->psi0 * exp(p->rho0 / rho);", "PIN.test_psi_exponential()"),
    ("psi_cs_missing_ideal_part", "return sqrt(2.0 * (pr - rho / 3.0) / p->G);",
     "return sqrt(2.0 * (pr - rho / 2.0) / p->G);", "PIN.test_cs_psi_pressure_identity()"),
    ("cs_repulsion_power", "(1.0 + eta + eta * eta - eta * eta * eta) / (om * om * om) - a * rho * rho;",
     "(1.0 + eta + eta * eta - eta * eta * eta) / (om * om) - a * rho * rho;",
     "PIN.test_cs_critical_published_constants()"),
    # Eq. (3) and Eq. (6)
    ("stream_wrong_way", "int m = wrapi(j + EY[a], ny) * nx + wrapi(i + EX[a], nx);",
     "int m = wrapi(j - EY[a], ny) * nx + wrapi(i - EX[a], nx);", "PIN.test_streaming_translates_planes()"),
    ("q_far_root", "double t = c->solid_outside ? (-bq + sq) / aa : (-bq - sq) / aa;",
     "double t = c->solid_outside ? (-bq + sq) / aa : (-bq + sq) / aa;",
     "PIN.test_geometry_brute_force(dict(nx=40, ny=36, circles=[(20, 15, 7.0)]))"),
    # Sec. 4.2 channel: Zou-He inlet and the momentum exchange
    ("zou_he_normal_population", "f[1 * N + n] = f3 + 2.0 / 3.0 * rho * u;",
     "f[1 * N + n] = f3 + 1.0 / 3.0 * rho * u;", "CH.test_zou_he_inlet_and_fully_developed_outlet()"),
    ("zou_he_density", "double rho = (f0 + f2 + f4 + 2.0 * (f3 + f6 + f7)) / (1.0 - u);",
     "double rho = (f0 + f2 + f4 + 2.0 * (f3 + f6 + f7)) / (1.0 + u);",
     "CH.test_zou_he_inlet_and_fully_developed_outlet()"),
    ("momentum_exchange_sign", "node_fx += EX[a] * (fo + val);", "node_fx += EX[a] * (fo - val);",
     "CH.test_momentum_exchange_closes_the_momentum_budget(O.MLS)"),
    ("mass_ledger_skips_rest", "for (int a = 0; a < 9; ++a) {\n      double x = s->f[a * N + n];",
     "for (int a = 1; a < 9; ++a) {\n      double x = s->f[a * N + n];",
     "P.test_closed_box_mass_conserved(O.HBB)"),
]

_RUNNER = """
import sys
sys.path[:0] = [{tmp!r}, {tests!r}]
import oracle as O
assert O.__file__.startswith({tmp!r}), O.__file__
import test_oracle_physics as P, test_oracle_pins as PIN, test_oracle_channel as CH
try:
    {pin}
except AssertionError:
    sys.exit(17)
sys.exit(0)
"""


def _run_mutant(case, workdir):
    name, old, new, pin = case
    src = os.path.join(ROOT, "oracle")
    tmp = os.path.join(workdir, name)
    shutil.copytree(src, os.path.join(tmp, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    path = os.path.join(tmp, "oracle", "lbm_oracle.c")
    text = open(path).read()
    count = text.count(old)
    if count != 1:
        return name, "the planted text occurs %d times" % count, ""
    open(path, "w").write(text.replace(old, new))
    env = dict(os.environ, OMP_NUM_THREADS="1", PYTHONDONTWRITEBYTECODE="1")
    p = subprocess.run([sys.executable, "-c", _RUNNER.format(tmp=tmp, tests=TESTS, pin=pin)],
                       capture_output=True, text=True, env=env, timeout=600)
    return name, p.returncode, p.stderr[-2000:]


def test_mutants_are_distinct_and_apply():
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    text = open(os.path.join(ROOT, "oracle", "lbm_oracle.c")).read()
    for name, old, new, _ in MUTANTS:
        assert text.count(old) == 1, name
        assert old != new, name


def test_every_planted_mistake_fails_a_pin():
    workdir = tempfile.mkdtemp(prefix="oracle_mutants_")
    try:
        with cf.ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
            results = list(ex.map(lambda c: _run_mutant(c, workdir), MUTANTS))
    finally:
        shutil.rmtree(workdir, ignore_errors=True)
    # exit 17: the pin raised AssertionError on the mutated oracle, as it must
    survived = [(n, rc, err) for n, rc, err in results if rc != 17]
    assert not survived, "\n".join("%s: %s\n%s" % s for s in survived)
