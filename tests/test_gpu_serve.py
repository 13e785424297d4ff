"""Continuous batching: requests that arrive while others run are admitted as slots and memory
free up, share the launches, and give the same bits as the same request run alone."""
import numpy as np
import pytest

from paper_1908_09235_gb300 import lbm, serve, workloads

pytestmark = pytest.mark.gpu


def _alone(req, precision):
    dom = serve.request_domain(req)
    eos = lbm.make_eos(lbm.EOS_CS, **req["eos"])
    rl, rv = lbm.lbm_coexistence(eos)
    eos.rho_wall = rv
    lat = lbm.Lattice(req["nx"], req["ny"], req["tau"], req["scheme"], circles=[req["cyl"]],
                      eos=eos, precision=precision)
    lat.init_droplet(*req["drop"], rl, rv)
    lat.step(req["steps"])
    out = lat.fields()
    lat.close()
    del dom
    return out


def test_served_results_equal_standalone_runs(gpu_lib):
    reqs = workloads.served_requests(n=10, rate=400.0, side_lo=40, side_hi=96, steps_lo=30,
                                     steps_hi=160, schemes=("mls", "bouzidi_l", "mod_a",
                                                            "mod_b"))
    prec = lbm.FP32_DEV
    need = max(lbm.lbm_domain_bytes(serve.request_domain(r), prec) for r in reqs)
    srv = serve.Server(precision=prec, max_slots=8, hbm_bytes=3 * need, chunk=20)
    done = srv.run(reqs, collect=lambda b, s: {"fields": b.fields(s)})
    srv.close()
    assert len(done) == len(reqs)
    assert 2 <= srv.max_concurrent <= 3          # overlap, bounded by the memory budget
    assert srv.peak_bytes <= 3 * need
    by_id = {r["rid"]: r for r in reqs}
    for rec in done:
        req = by_id[rec.rid]
        assert rec.steps == req["steps"] and rec.finished > rec.arrival
        for x, y in zip(rec.result["fields"], _alone(req, prec)):
            assert np.array_equal(np.nan_to_num(x, nan=-7.0), np.nan_to_num(y, nan=-7.0))
    stats = serve.latency_stats(done)
    assert 0 < stats["p50_s"] <= stats["p99_s"]


def test_fifo_latencies_of_the_plain_loop():
    # one request at a time: the second waits for the first
    lat = serve.fifo_latencies([0.0, 0.5, 10.0], [2.0, 1.0, 1.0])
    assert np.allclose(lat, [2.0, 2.5, 1.0])
