"""Checkpoint and resume through the C ABI (lbm_state_bytes / lbm_save_state / lbm_load_state):
a lattice saved after k steps and restored into a fresh context continues bit for bit like the
uninterrupted run, in every storage format (the FP64 rounding carry of the deviation formats is
part of the state) and in channel mode; blobs of another lattice are refused."""
import numpy as np
import pytest

from gpu_cases import c0_case
from paper_1908_09235_gb300 import lbm

pytestmark = pytest.mark.gpu


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(np.nan_to_num(x, nan=-7.0), np.nan_to_num(y, nan=-7.0))


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32_DEV, lbm.FP16_DEV])
@pytest.mark.parametrize("scheme", [lbm.MOD_B, lbm.MOD_A, lbm.BOUZIDI_Q])
def test_resume_is_bit_exact(gpu_lib, precision, scheme):
    case = c0_case()
    ref = case.gpu(scheme, precision=precision)
    ref.step(70)
    want_fields, want_mass = ref.fields(), ref.mass()
    ref.close()

    a = case.gpu(scheme, precision=precision)
    a.step(30)
    blob = a.save_state()
    a.step(5)  # the saved state must not change with the source context
    a.close()
    b = case.gpu(scheme, precision=precision)
    b.step(3)  # some other state, replaced by the blob
    b.load_state(blob)
    assert b.info()["steps"] == 30
    b.step(40)
    _same(b.fields(), want_fields)
    assert b.mass() == want_mass
    b.close()


def test_resume_in_channel_mode(gpu_lib):
    def lattice():
        lat = lbm.Lattice(96, 48, 0.8, lbm.MOD_B, circles=[(30.3, 23.7, 6.2)],
                          eos=lbm.make_eos(lbm.EOS_NONE), precision=lbm.FP32_DEV)
        lat.init_fields(np.ones(96 * 48))
        return lat

    ref = lattice()
    ref.set_inflow(0.04)
    ref.step(200)
    want = ref.fields(), ref.force()
    ref.close()
    a = lattice()
    a.set_inflow(0.04)
    a.step(120)
    blob = a.save_state()
    a.close()
    b = lattice()  # periodic until the blob restores the channel settings
    b.load_state(blob)
    b.step(80)
    _same(b.fields(), want[0])
    assert b.force() == want[1]
    b.close()


def test_foreign_and_short_blobs_are_refused(gpu_lib):
    case = c0_case()
    a = case.gpu(lbm.MOD_B, precision=lbm.FP32_DEV)
    a.step(2)
    blob = a.save_state()
    a.close()
    for other in (dict(precision=lbm.FP64), dict(precision=lbm.FP16_DEV)):
        b = case.gpu(lbm.MOD_B, **other)
        with pytest.raises(lbm.LBMError) as e:
            b.load_state(blob)
        assert e.value.status == 1
        b.close()
    b = case.gpu(lbm.MOD_A, precision=lbm.FP32_DEV)  # another scheme
    with pytest.raises(lbm.LBMError):
        b.load_state(blob)
    b.close()
    b = case.gpu(lbm.MOD_B, precision=lbm.FP32_DEV)
    with pytest.raises(lbm.LBMError):
        b.load_state(blob[:-8])
    b.close()
    b = case.gpu(lbm.MOD_B, precision=lbm.FP32_DEV)
    bad = blob.copy()
    bad[0] ^= 0xFF  # not a state blob
    with pytest.raises(lbm.LBMError):
        b.load_state(bad)
    b.close()


def test_save_before_initialisation_and_batch_members(gpu_lib):
    lat = lbm.Lattice(32, 24, 1.0, lbm.MOD_B, circles=[(15.0, 11.0, 4.0)],
                      eos=lbm.make_eos(lbm.EOS_NONE))
    with pytest.raises(lbm.LBMError) as e:
        lat.save_state()
    assert e.value.status == 6  # LBM_ESTATE
    lat.close()
    b = lbm.Batch(lbm.FP32_DEV, lbm.EOS_NONE, max_domains=2)
    s = b.add(lbm.make_domain(32, 24, 1.0, lbm.MOD_B, circles=[(15.0, 11.0, 4.0)],
                              eos=lbm.make_eos(lbm.EOS_NONE)), 10)
    b.step(4)
    ctx = b.ctx(s)
    blob = lbm.lbm_save_state(ctx)  # the batch's current state can be saved
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_load_state(ctx, blob)  # but not restored under the batch
    assert e.value.status == 6
    b.close()
