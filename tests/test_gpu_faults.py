"""Failure detection without a GPU fault.  Host-side injection: device allocations that fail at
every point of lbm_create, of a lattice's first initialisation and of lbm_batch_add; each
failure comes back as LBM_ENOMEM, every block allocated before it is returned, and the same calls
succeed afterwards.  On the GPU: a bounded wait on a barrier phase that nothing completes gives
up after its limit and reports LBM_ETIMEOUT, and the device stays usable."""
import ctypes as C

import numpy as np
import pytest

from paper_1908_09235_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu


class FailingMemory(lbm.TorchDeviceMemory):
    """The torch allocation hook, failing its k-th allocation (k = 1, 2, ...; 0: never)."""

    def __init__(self, fail_at):
        super().__init__()
        self.fail_at = fail_at
        self.calls = 0

    def _alloc(self, nbytes, user):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        return super()._alloc(nbytes, user)


def _options(mem, precision=lbm.FP32_DEV):
    import torch
    opt = lbm.Options()
    opt.precision = precision
    opt.stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    opt.alloc = mem.alloc_fn
    opt.free = mem.free_fn
    return opt


def _geometry_and_eos():
    eos = lbm.make_eos(lbm.EOS_CS, **workloads.CS)
    rl, rv = lbm.lbm_coexistence(eos)
    eos.rho_wall = rv
    return lbm.make_geometry(96, 64, [(48.3, 22.6, 9.1)]), eos, (rl, rv)


def test_allocation_failures_in_create_and_initialisation(gpu_lib):
    geo, eos, (rl, rv) = _geometry_and_eos()
    # how many allocations a full create + initialisation makes
    mem = FailingMemory(0)
    ctx = lbm.lbm_create(geo, eos, 1.0, lbm.MOD_B, _options(mem))
    lbm.lbm_init_droplet(ctx, 48.0, 32.0, 12.0, 4.0, rl, rv)
    lbm.lbm_step(ctx, 3)
    want = lbm.lbm_mass(ctx)
    lbm.lbm_destroy(ctx)
    total = mem.calls
    assert total >= 2 and not mem.live
    for k in range(1, total + 1):
        mem = FailingMemory(k)
        try:
            ctx = lbm.lbm_create(geo, eos, 1.0, lbm.MOD_B, _options(mem))
        except lbm.LBMError as e:
            assert e.status == 2  # LBM_ENOMEM
            assert not mem.live  # everything allocated before the failure was returned
            continue
        try:
            lbm.lbm_init_droplet(ctx, 48.0, 32.0, 12.0, 4.0, rl, rv)
            lbm.lbm_step(ctx, 3)
            assert lbm.lbm_mass(ctx) == want
        except lbm.LBMError as e:
            assert e.status == 2
        lbm.lbm_destroy(ctx)
        assert not mem.live
    # afterwards the same calls succeed
    mem = FailingMemory(0)
    ctx = lbm.lbm_create(geo, eos, 1.0, lbm.MOD_B, _options(mem))
    lbm.lbm_init_droplet(ctx, 48.0, 32.0, 12.0, 4.0, rl, rv)
    lbm.lbm_step(ctx, 3)
    assert lbm.lbm_mass(ctx) == want
    lbm.lbm_destroy(ctx)


def test_allocation_failure_in_batch_add_leaves_the_batch_usable(gpu_lib):
    ws = workloads.batched_domains(n=3, seed=workloads.SEED, side_lo=40, side_hi=80)

    def domain(w):
        eos = lbm.make_eos(lbm.EOS_CS, **w["eos"])
        rl, rv = lbm.lbm_coexistence(eos)
        eos.rho_wall = rv
        return lbm.make_domain(w["nx"], w["ny"], w["tau"], lbm.MOD_B, circles=[w["cyl"]],
                               eos=eos, droplet=tuple(w["drop"]) + (rl, rv))

    mem = FailingMemory(0)
    b = lbm.Batch(lbm.FP32_DEV, lbm.EOS_CS, max_domains=3, memory=mem)
    s0 = b.add(domain(ws[0]), 20)
    live = len(mem.live)
    mem.fail_at = mem.calls + 1  # the new lattice's first block
    with pytest.raises(lbm.LBMError) as e:
        b.add(domain(ws[1]), 20)
    assert e.value.status == 2
    assert len(mem.live) == live
    s1 = b.add(domain(ws[2]), 20)  # the batch still takes lattices and steps them
    b.step(20)
    assert b.progress(s0) == (20, 0) and b.progress(s1) == (20, 0)
    b.close()
    assert not mem.live


def test_bounded_wait_gives_up_and_the_device_stays_usable(gpu_lib):
    # the bounded mbarrier wait of the TMA-staged kernel, on a phase nothing completes
    import time
    t0 = time.perf_counter()
    st, done = lbm.lbm_selftest_bounded_wait(200_000_000, 0)  # 0.2 s
    dt = time.perf_counter() - t0
    assert (st, done) == (5, 0)  # LBM_ETIMEOUT: the wait gave up
    assert 0.19 < dt < 10.0
    assert lbm.lbm_selftest_bounded_wait(200_000_000, 1) == (0, 1)  # completed phase
    # the device and the library keep working
    lat = lbm.Lattice(64, 32, 1.0, lbm.MOD_B, circles=[(20.0, 16.0, 5.0)],
                      eos=lbm.make_eos(lbm.EOS_NONE), precision=lbm.FP32_DEV, kernel_path=2)
    lat.init_fields(np.ones(64 * 32))
    lat.step(5)
    assert abs(lat.mass() / lat.info()["n_fluid"] - 1) < 1e-6
    lat.close()
