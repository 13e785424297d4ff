"""The -fopenmp build of the oracle (its per-node loops on all host cores, used only to time the
oracle on the GPU machine's host) gives the same bits as the serial build: same arithmetic per node,
every value written by one iteration, serial ledger and wall pass."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1908_09235_gb300 import workloads


def _run(openmp, scheme, steps, inflow=False, **kw):
    w = workloads.SMALL
    c = workloads.CS
    if inflow:
        s = O.OracleSim(80, 40, 0.8, scheme=scheme, circles=[(25.3, 19.6, 6.1)],
                        eos=O.EOS_NONE, openmp=openmp)
        s.init_fields(np.ones(80 * 40))
        s.set_inflow(0.05)
    else:
        Tc, _ = O.cs_critical(c["a"], c["b"], c["R"])
        rl, rv = O.cs_coexistence(c["a"], c["b"], c["R"], c["T_over_Tc"] * Tc)
        s = O.OracleSim(w.nx, w.ny, w.tau, scheme=scheme, circles=w.circles, eos=O.EOS_CS,
                        G=c["G"], a=c["a"], b=c["b"], R=c["R"], T_over_Tc=c["T_over_Tc"],
                        rho_wall=rv, openmp=openmp, **kw)
        s.init_droplet(*w.drop, rl, rv)
    s.step(steps)
    return s.get_f(), s.mass(), s.force()


@pytest.fixture(scope="module", autouse=True)
def _threads():
    # libgomp reads the thread count when the library is loaded
    old = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "4"
    yield
    if old is None:
        os.environ.pop("OMP_NUM_THREADS", None)
    else:
        os.environ["OMP_NUM_THREADS"] = old


def _same(x, y):
    return np.array_equal(np.asarray(x), np.asarray(y), equal_nan=True)


@pytest.mark.parametrize("scheme", [O.MOD_B, O.ZHAO_YONG])  # ZY diverges here: NaNs must match
def test_openmp_build_gives_the_same_bits(scheme):
    a = _run(False, scheme, 60)
    b = _run(True, scheme, 60)
    assert _same(a[0], b[0])
    assert _same(a[1], b[1])


def test_openmp_build_same_bits_with_body_force_and_channel():
    a = _run(False, O.MOD_A, 40, gy=-2e-6)
    b = _run(True, O.MOD_A, 40, gy=-2e-6)
    assert np.array_equal(a[0], b[0])
    a = _run(False, O.MOD_B, 80, inflow=True)
    b = _run(True, O.MOD_B, 80, inflow=True)
    assert np.array_equal(a[0], b[0]) and a[2] == b[2]
