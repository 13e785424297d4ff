"""GPU channel flow past a cylinder (Sec. 4.2 set-up) through the C ABI, against the oracle:
Zou-He velocity inlet, fully developed outlet, curved walls, momentum-exchange force."""
import numpy as np
import pytest

import oracle as O
from gpu_cases import SCHEME_ORACLE
from paper_1908_09235_gb300 import lbm

pytestmark = pytest.mark.gpu

NX, NY = 120, 64
CYL = (40.3, 31.7, 7.8)
TAU, U_IN = 0.8, 0.05


def _gpu(scheme, precision, path=0, steps=400, inflow=True):
    lat = lbm.Lattice(NX, NY, TAU, scheme, circles=[CYL], eos=lbm.make_eos(lbm.EOS_NONE),
                      precision=precision, kernel_path=path, track_force=not inflow)
    lat.init_fields(np.ones(NX * NY))
    if inflow:
        lat.set_inflow(U_IN)
    lat.step(steps)
    out = lat.fields(), lat.force(), lat.mass()
    lat.close()
    return out


def _oracle(scheme, steps=400):
    s = O.OracleSim(NX, NY, TAU, scheme=SCHEME_ORACLE[scheme], circles=[CYL], eos=O.EOS_NONE)
    s.init_fields(np.ones(NX * NY))
    s.set_inflow(U_IN)
    s.step(steps)
    return s.fields(), s.force()


SCHEMES = [lbm.HBB, lbm.MLS, lbm.BOUZIDI_Q, lbm.ZHAO_YONG, lbm.MOD_A, lbm.MOD_B]


@pytest.mark.parametrize("scheme", SCHEMES)
def test_channel_matches_oracle_fp64(gpu_lib, scheme):
    (g, fg, _), (o, fo) = _gpu(scheme, lbm.FP64), _oracle(scheme)
    for x, y in zip(g, o):
        m = np.isfinite(y)
        assert np.array_equal(m, np.isfinite(x))
        assert np.max(np.abs(x[m] - y[m])) <= 1e-11
    assert fo[0] > 1e-3  # the flow pushes the cylinder downstream
    assert abs(fg[0] - fo[0]) <= 1e-9 * abs(fo[0])
    assert abs(fg[1] - fo[1]) <= 1e-9 * abs(fo[0])


@pytest.mark.parametrize("scheme", [lbm.MOD_A, lbm.MOD_B])
def test_channel_fp32_dev_against_oracle(gpu_lib, scheme):
    # FP32 storage of deviations from w_a rho_ref, FP32 arithmetic: rho ~ 1, u ~ 0.05 here
    (g, fg, _), (o, fo) = _gpu(scheme, lbm.FP32_DEV), _oracle(scheme)
    for x, y in zip(g, o):
        m = np.isfinite(y)
        assert np.max(np.abs(x[m] - y[m])) <= 1e-5
    assert abs(fg[0] - fo[0]) <= 1e-4 * abs(fo[0])


@pytest.mark.parametrize("precision", [lbm.FP32_DEV, lbm.FP16_DEV])
def test_channel_vector_kernel_equals_scalar_tiles(gpu_lib, precision):
    a = _gpu(lbm.MOD_B, precision, path=0, steps=300)
    b = _gpu(lbm.MOD_B, precision, path=1, steps=300)
    for x, y in zip(a[0], b[0]):
        assert np.array_equal(np.nan_to_num(x, nan=-7.0), np.nan_to_num(y, nan=-7.0))
    assert a[1] == b[1] and a[2] == b[2]


def test_force_at_rest_is_zero(gpu_lib):
    _, (fx, fy), _ = _gpu(lbm.MOD_B, lbm.FP64, steps=20, inflow=False)
    assert abs(fx) < 1e-13 and abs(fy) < 1e-13


def test_force_needs_recording(gpu_lib):
    lat = lbm.Lattice(64, 32, 1.0, lbm.MOD_B, circles=[(20.0, 16.0, 5.0)],
                      eos=lbm.make_eos(lbm.EOS_NONE))
    lat.init_fields(np.ones(64 * 32))
    lat.step(2)
    with pytest.raises(lbm.LBMError) as e:
        lat.force()
    assert e.value.status == 6  # LBM_ESTATE
    lat.close()


def test_inflow_rejects_two_phase_and_bad_velocity(gpu_lib):
    eos = lbm.make_eos(lbm.EOS_EXP, G=-10.0 / 3.0)
    lat = lbm.Lattice(64, 32, 1.0, lbm.MOD_B, circles=[(20.0, 16.0, 5.0)], eos=eos)
    with pytest.raises(lbm.LBMError) as e:
        lat.set_inflow(0.05)
    assert e.value.status == 1
    lat.close()
    lat = lbm.Lattice(64, 32, 1.0, lbm.MOD_B, circles=[(20.0, 16.0, 5.0)],
                      eos=lbm.make_eos(lbm.EOS_NONE))
    with pytest.raises(lbm.LBMError):
        lat.set_inflow(0.7)
    lat.close()
