"""Batches: many uneven lattices advanced by one set of launches per step.

Each lattice must give the same bits inside a batch as alone (same per-node arithmetic), whatever
the batch's other members, join/leave times, step budgets or tile shape; and a batched lattice
matches the FP64 oracle like a single one does.
"""
import numpy as np
import pytest

from gpu_cases import SCHEME_ORACLE
from paper_1908_09235_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu


def _member(w, scheme, precision):
    eos = lbm.make_eos(lbm.EOS_CS, **w["eos"])
    rl, rv = lbm.lbm_coexistence(eos)
    eos.rho_wall = rv
    return lbm.make_domain(w["nx"], w["ny"], w["tau"], scheme, circles=[w["cyl"]], eos=eos,
                           droplet=tuple(w["drop"]) + (rl, rv))


def _alone(w, scheme, precision, steps):
    eos = lbm.make_eos(lbm.EOS_CS, **w["eos"])
    rl, rv = lbm.lbm_coexistence(eos)
    eos.rho_wall = rv
    lat = lbm.Lattice(w["nx"], w["ny"], w["tau"], scheme, circles=[w["cyl"]], eos=eos,
                      precision=precision)
    lat.init_droplet(*w["drop"], rl, rv)
    lat.step(steps)
    out = lat.fields(), lat.mass()
    lat.close()
    return out


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(np.nan_to_num(x, nan=-7.0), np.nan_to_num(y, nan=-7.0))


def _stable_members(n, seed):
    # uneven sides 40..140, parameters from the stable part of the batched workload
    ws = workloads.batched_domains(n=n, seed=seed, side_lo=40, side_hi=140)
    for w in ws:
        w["tau"] = 0.8 + 0.4 * (w["tau"] - 0.6) / 0.6
        w["eos"]["T_over_Tc"] = 0.85 + 0.05 * (w["eos"]["T_over_Tc"] - 0.8) / 0.1
    return ws


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32_DEV, lbm.FP16_DEV])
def test_batch_members_match_standalone_runs(gpu_lib, precision):
    ws = _stable_members(6, workloads.SEED)
    schemes = [lbm.MOD_B, lbm.MOD_A, lbm.MLS, lbm.BOUZIDI_L, lbm.BOUZIDI_Q, lbm.HBB]
    budgets = [60, 45, 60, 17, 33, 60]
    b = lbm.Batch(precision, lbm.EOS_CS, max_domains=8)
    slots = [b.add(_member(w, s, precision), n) for w, s, n in zip(ws, schemes, budgets)]
    b.step(20)          # graph of 16 steps + 4 single steps
    b.remove(slots[1])  # leaves after 20 of its 45 steps
    late = b.add(_member(ws[1], lbm.MOD_A, precision), 40)  # joins now with a budget of 40
    b.step(50)
    for k in (0, 2, 3, 4, 5):
        done, left = b.progress(slots[k])
        assert done == budgets[k] and left == 0
        fields, mass = _alone(ws[k], schemes[k], precision, budgets[k])
        _same(b.fields(slots[k]), fields)
        assert b.mass(slots[k]) == mass
    done, left = b.progress(late)
    assert (done, left) == (40, 0)
    _same(b.fields(late), _alone(ws[1], lbm.MOD_A, precision, 40)[0])
    b.close()


def _run_with(ws, precision, rows_sched, steps=40):
    b = lbm.Batch(precision, lbm.EOS_CS, max_domains=len(ws))
    slots = [b.add(_member(w, lbm.MOD_B, precision), steps) for w in ws]
    if rows_sched == "tuned":
        assert b.tune(3) in (8, 16, 32)
    elif rows_sched is not None:
        b.set_schedule(*rows_sched)
    b.step(steps)
    info = b.info()
    out = [b.fields(s) for s in slots]
    b.close()
    return out, info


SCHEDS = (lbm.SCHED_STRIDED, lbm.SCHED_CLAIM, lbm.SCHED_CLAIM_LARGEST_FIRST)


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32_DEV])
def test_tile_shape_and_schedule_do_not_change_results(gpu_lib, precision):
    # uneven sides, so the largest-first order differs from the slot order
    ws = _stable_members(5, workloads.SEED + 1)
    ref, _ = _run_with(ws, precision, None)
    rows = (8, 16) if precision == lbm.FP64 else (8, 16, 32)
    for r in rows:
        for sc in SCHEDS:
            out, info = _run_with(ws, precision, (r, sc))
            assert (info["tile_rows"], info["schedule"]) == (r, sc)
            for a, c in zip(ref, out):
                _same(a, c)
    out, info = _run_with(ws, precision, "tuned")
    assert info["schedule"] in SCHEDS
    for a, c in zip(ref, out):
        _same(a, c)


def test_tuner_times_every_tile_height_and_schedule(gpu_lib):
    ws = _stable_members(4, workloads.SEED + 2)
    b = lbm.Batch(lbm.FP32_DEV, lbm.EOS_CS, max_domains=4)
    for w in ws:
        b.add(_member(w, lbm.MOD_B, lbm.FP32_DEV), 100)
    assert b.tune_trials() == []
    rows = b.tune(2)
    trials = b.tune_trials()
    assert [(r, s) for r, s, _ in trials] == [(r, s) for r in (8, 16, 32) for s in SCHEDS]
    best = min(trials, key=lambda t: t[2])
    info = b.info()
    assert (rows, info["schedule"]) == best[:2] == (info["tile_rows"], info["schedule"])
    assert all(t[2] > 0 for t in trials)
    # tuning changed no state: every lattice still has its full budget
    assert all(b.progress(s) == (0, 100) for s in range(4))
    with pytest.raises(lbm.LBMError):
        b.set_schedule(12, lbm.SCHED_CLAIM)
    with pytest.raises(lbm.LBMError):
        b.set_schedule(16, 7)
    b.close()
    b = lbm.Batch(lbm.FP64, lbm.EOS_CS, max_domains=2)
    with pytest.raises(lbm.LBMError):
        b.set_schedule(32, lbm.SCHED_STRIDED)  # FP64 register budget: 8 or 16 rows
    b.close()


def test_batched_lattice_matches_oracle(gpu_lib):
    import oracle as O
    w = workloads.SMALL
    member = dict(nx=w.nx, ny=w.ny, cyl=w.cyl, drop=w.drop, tau=w.tau, eos=dict(w.eos))
    others = _stable_members(3, workloads.SEED + 2)
    b = lbm.Batch(lbm.FP64, lbm.EOS_CS, max_domains=4)
    for o in others:
        b.add(_member(o, lbm.MOD_A, lbm.FP64), 300)
    slot = b.add(_member(member, lbm.MOD_B, lbm.FP64), 300)
    b.step(300)
    c = w.eos
    Tc, _ = O.cs_critical(c["a"], c["b"], c["R"])
    rl, rv = O.cs_coexistence(c["a"], c["b"], c["R"], c["T_over_Tc"] * Tc)
    s = O.OracleSim(w.nx, w.ny, w.tau, scheme=SCHEME_ORACLE[lbm.MOD_B], circles=w.circles,
                    eos=O.EOS_CS, G=c["G"], a=c["a"], b=c["b"], R=c["R"],
                    T_over_Tc=c["T_over_Tc"], rho_wall=rv)
    s.init_droplet(*w.drop, rl, rv)
    s.step(300)
    g, o = b.fields(slot), s.fields()
    for x, y in zip(g, o):
        m = np.isfinite(y)
        assert np.max(np.abs(x[m] - y[m])) <= 1e-11
    b.close()


def test_batch_rejects_other_eos_and_full_batches(gpu_lib):
    b = lbm.Batch(lbm.FP32_DEV, lbm.EOS_CS, max_domains=1)
    d_none = lbm.make_domain(64, 64, 1.0, lbm.HBB, rho=1.0)
    with pytest.raises(lbm.LBMError) as e:
        b.add(d_none, 10)
    assert e.value.status == 1
    ws = _stable_members(2, workloads.SEED + 3)
    b.add(_member(ws[0], lbm.MOD_B, lbm.FP32_DEV), 10)
    with pytest.raises(lbm.LBMError) as e:
        b.add(_member(ws[1], lbm.MOD_B, lbm.FP32_DEV), 10)
    assert e.value.status == 2
    b.close()


def test_full_batched_workload_sampled_members(gpu_lib):
    # the 512-lattice workload of the benchmark, in its launch configuration (FP32 deviations,
    # tuned tile height, graphs): sampled members give the same bits as the same lattice alone
    # (diverging members included: their NaN pattern must match too)
    ws = workloads.batched_domains()
    b = lbm.Batch(lbm.FP32_DEV, lbm.EOS_CS, max_domains=len(ws))
    slots = [b.add(_member(w, lbm.MOD_B, lbm.FP32_DEV), 10**9) for w in ws]
    assert b.tune(3) in (8, 16, 32)
    b.step(40)
    for k in (0, 137, 311, 511):
        fields, _ = _alone(ws[k], lbm.MOD_B, lbm.FP32_DEV, 40)
        _same(b.fields(slots[k]), fields)
    b.close()


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32_DEV])
def test_batch_flags_the_lattices_the_oracle_flags(gpu_lib, precision):
    # the smallest members of the 512-lattice workload: the batch reports LBM_EUNSTABLE for
    # exactly the lattices whose FP64 oracle run diverges within the same steps
    from test_workloads_cpu import oracle_diverges
    ws = [w for w in workloads.batched_domains() if w["nx"] <= 70]
    b = lbm.Batch(precision, lbm.EOS_CS, max_domains=len(ws))
    slots = [b.add(_member(w, lbm.MOD_B, precision), 300) for w in ws]
    b.step(300)
    for w, s in zip(ws, slots):
        try:
            b.mass(s)
            gpu_unstable = False
        except lbm.LBMError as e:
            assert e.status == 4  # LBM_EUNSTABLE
            gpu_unstable = True
        assert gpu_unstable == oracle_diverges(w, 300), w["name"]
    b.close()
