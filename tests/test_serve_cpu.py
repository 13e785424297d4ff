"""Host logic of the continuous-batching server (serve.py) without a GPU: the batch is replaced by
a fake that counts each lattice's step budget down, so admission by the memory budget, slot
reuse, arrival-order admission and completion can be checked exactly.  The library's host-only
calls (coexistence densities, lbm_domain_bytes) are the real ones."""
import numpy as np
import pytest

from paper_1908_09235_gb300 import lbm, serve, workloads


class FakeBatch:
    """Slots with step budgets; step(n) advances every active slot by up to n steps."""

    def __init__(self, precision, eos_kind, max_domains):
        self.left = {}
        self.max_domains = max_domains
        self.added = []

    def add(self, domain, steps):
        slot = min(k for k in range(self.max_domains) if k not in self.left)
        self.left[slot] = int(steps)
        self.added.append((slot, domain.geometry.nx))
        return slot

    def step(self, n):
        for s in self.left:
            self.left[s] = max(0, self.left[s] - n)

    def poll(self, n):
        return [self.left.get(s, -1) for s in range(n)]

    def remove(self, slot):
        del self.left[slot]

    def ctx(self, slot):
        return slot

    def close(self):
        pass


@pytest.fixture
def fake_gpu(monkeypatch):
    monkeypatch.setattr(serve.lbm, "Batch", FakeBatch)
    monkeypatch.setattr(serve.lbm, "lbm_info", lambda ctx: {"n_fluid": 100})


def _requests(n, side=128, steps=400):
    rs = workloads.served_requests(n=n, side_lo=side, side_hi=side, steps_lo=steps,
                                   steps_hi=steps)
    for k, r in enumerate(rs):
        r["arrival"] = float(k)  # in order
    return rs


def test_admission_by_memory_budget_and_slot_reuse(fake_gpu):
    rs = _requests(7)
    need = lbm.lbm_domain_bytes(serve.request_domain(rs[0]), lbm.FP32_DEV)
    srv = serve.Server(precision=lbm.FP32_DEV, max_slots=16, hbm_bytes=3 * need + need // 2,
                       chunk=100)
    done = srv.run(rs, collect=None, realtime=False)
    assert sorted(r.rid for r in done) == list(range(7))
    assert srv.max_concurrent == 3  # three lattices fit the budget, a fourth does not
    assert srv.peak_bytes == 3 * need
    # admitted in arrival order, each after its predecessor
    by_rid = sorted(done, key=lambda r: r.rid)
    assert all(a.admitted <= b.admitted for a, b in zip(by_rid, by_rid[1:]))
    # slots are reused: never more than three distinct slots
    assert max(slot for slot, _ in srv.batch.added) <= 2
    srv.close()


def test_slot_limit_and_oversized_request(fake_gpu):
    rs = _requests(5)
    srv = serve.Server(precision=lbm.FP32_DEV, max_slots=2, hbm_bytes=1 << 40, chunk=400)
    done = srv.run(rs, collect=None, realtime=False)
    assert len(done) == 5 and srv.max_concurrent == 2
    srv.close()
    srv = serve.Server(precision=lbm.FP32_DEV, max_slots=2, hbm_bytes=1000, chunk=400)
    with pytest.raises(RuntimeError):
        srv.run(_requests(1), collect=None, realtime=False)
    srv.close()


def test_fifo_model_and_latency_statistics():
    # one server, one request at a time: the plain loop the benchmark compares with
    lat = serve.fifo_latencies([0.0, 1.0, 2.0, 10.0], [2.0, 2.0, 2.0, 1.0])
    assert np.allclose(lat, [2.0, 3.0, 4.0, 1.0])

    class R:
        def __init__(self, x):
            self.latency = x
    st = serve.latency_stats([R(float(x)) for x in range(1, 101)])
    assert st["p50_s"] == pytest.approx(50.5) and st["max_s"] == 100.0
    assert st["p99_s"] == pytest.approx(99.01)


def test_one_at_a_time_loop_follows_arrivals_and_matches_the_fifo_model():
    # The plain FP64 loop, run with a fake lattice whose step costs steps / 100 seconds of a
    # fake clock: requests run in arrival order, each waits for its arrival and for the one
    # before it, and the latencies equal the FIFO model's for the same service times.
    clock = {"t": 0.0}

    class FakeLattice:
        def __init__(self, req, precision):
            self.req = req
            assert precision == lbm.FP64

        def step(self, n):
            clock["t"] += n / 100.0

        def info(self):
            return {"n_fluid": 7}

        def close(self):
            pass

    rs = _requests(4, steps=200)
    for r, a in zip(rs, (0.0, 0.5, 1.0, 9.0)):
        r["arrival"] = a
    done = serve.run_one_at_a_time(rs, make=FakeLattice, collect=None,
                                   clock=lambda: clock["t"],
                                   sleep=lambda s: clock.__setitem__("t", clock["t"] + s))
    assert [r.rid for r in done] == [r["rid"] for r in rs]
    expect = serve.fifo_latencies([r["arrival"] for r in rs], [2.0] * 4)
    assert np.allclose([r.latency for r in done], expect)
    assert np.allclose([r.latency for r in done], [2.0, 3.5, 5.0, 2.0])
    assert all(r.fluid_nodes == 7 for r in done)
