"""Continuous-batching server for lattice Boltzmann requests.

Requests (a droplet-on-cylinder lattice, a boundary scheme and a number of time steps) arrive
over time.  The server keeps one batch (lbm_batch_* of the C ABI) resident on the GPU: a request
is admitted into a free slot as soon as it has arrived and the batch's memory budget has room for
it (admission by free HBM, in arrival order), its populations stay on the device until it is done,
and every lattice in the batch advances in the same launches (one set of kernels per time step
for all of them) in chunks of `chunk` steps.  The device stops each lattice exactly at its own
step budget; after each chunk the server polls the budgets in one call, reads finished results,
frees their slots and memory, and admits waiting requests.  Latency is measured from arrival to
the moment the result is on the host.
"""
import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import lbm


@dataclass
class Served:
    rid: int
    arrival: float
    nodes: int
    fluid_nodes: int = 0
    steps: int = 0
    admitted: float = float("nan")
    finished: float = float("nan")
    slot: int = -1
    bytes: int = 0
    result: dict = field(default_factory=dict)

    @property
    def latency(self):
        return self.finished - self.arrival


def request_domain(req):
    """The lbm_domain of a request dict (workloads.served_requests / batched_domains format)."""
    eos = lbm.make_eos(lbm.EOS_CS, **req["eos"])
    rl, rv = lbm.lbm_coexistence(eos)
    eos.rho_wall = rv
    return lbm.make_domain(req["nx"], req["ny"], req["tau"], req["scheme"], circles=[req["cyl"]],
                           eos=eos, droplet=tuple(req["drop"]) + (rl, rv))


def summary_result(batch, slot):
    """Default result of a finished request: total mass and density extremes (NaN if the run
    became unstable)."""
    try:
        m = batch.mass(slot)
    except lbm.LBMError:
        return {"mass": float("nan"), "unstable": True}
    rho, _, _ = batch.fields(slot)
    return {"mass": m, "rho_min": float(np.nanmin(rho)), "rho_max": float(np.nanmax(rho)),
            "unstable": False}


class Server:
    def __init__(self, precision=lbm.FP32_DEV, max_slots=256, hbm_bytes=None, chunk=200,
                 clock=time.perf_counter):
        import torch
        self.precision = precision
        self.max_slots = max_slots
        if hbm_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_bytes = int(0.8 * free)
        self.hbm_bytes = int(hbm_bytes)
        self.chunk = int(chunk)
        self.clock = clock
        self.batch = lbm.Batch(precision, lbm.EOS_CS, max_domains=max_slots)
        self.max_concurrent = 0
        self.peak_bytes = 0
        self.slot_rid = {}  # slot -> rid of the request it holds (for collect functions)

    def close(self):
        self.batch.close()

    def run(self, requests, collect=summary_result, realtime=True):
        """Serve `requests` (dicts with at least rid, arrival, nx, ny, steps, ...).  With realtime
        the arrivals follow the wall clock from the start of the call; otherwise every request
        is available at once.  collect(batch, slot) makes a finished request's result while it
        is still in the batch (self.slot_rid[slot] names the request).  Returns the list of
        Served records in completion order."""
        b = self.batch
        pending = collections.deque(sorted(requests, key=lambda r: r["arrival"]))
        active = {}
        used = 0
        done = []
        t0 = self.clock()
        while pending or active:
            now = self.clock() - t0
            # admission: arrived requests in order, while a slot and memory are free
            while pending and (not realtime or pending[0]["arrival"] <= now):
                req = pending[0]
                dom = request_domain(req)
                need = lbm.lbm_domain_bytes(dom, self.precision)
                if len(active) >= self.max_slots or used + need > self.hbm_bytes:
                    if not active:
                        raise RuntimeError("request %d needs %d bytes, over the budget of %d"
                                           % (req["rid"], need, self.hbm_bytes))
                    break
                slot = b.add(dom, req["steps"])
                self.slot_rid[slot] = req["rid"]
                rec = Served(rid=req["rid"], arrival=req["arrival"] if realtime else 0.0,
                             nodes=req["nx"] * req["ny"], steps=req["steps"], slot=slot,
                             bytes=need, admitted=self.clock() - t0)
                active[slot] = rec
                used += need
                pending.popleft()
            self.max_concurrent = max(self.max_concurrent, len(active))
            self.peak_bytes = max(self.peak_bytes, used)
            if not active:
                if pending and realtime:
                    time.sleep(max(0.0, min(0.01, pending[0]["arrival"] - (self.clock() - t0))))
                continue
            b.step(self.chunk)
            left = b.poll(self.max_slots)
            for slot, rec in list(active.items()):
                if left[slot] == 0:
                    rec.result = collect(b, slot) if collect else {}
                    rec.fluid_nodes = lbm.lbm_info(b.ctx(slot))["n_fluid"]
                    rec.finished = self.clock() - t0
                    b.remove(slot)
                    used -= rec.bytes
                    del active[slot]
                    done.append(rec)
        return done


def request_lattice(req, precision=lbm.FP64):
    """A standalone lattice (lbm_create) of a request dict, initialised with its droplet."""
    eos = lbm.make_eos(lbm.EOS_CS, **req["eos"])
    rl, rv = lbm.lbm_coexistence(eos)
    eos.rho_wall = rv
    lat = lbm.Lattice(req["nx"], req["ny"], req["tau"], lbm.SCHEMES[req["scheme"]]
                      if isinstance(req["scheme"], str) else req["scheme"], circles=[req["cyl"]],
                      eos=eos, precision=precision)
    lat.init_droplet(*req["drop"], rl, rv)
    return lat


def lattice_result(lat):
    """Result of a finished standalone run, as summary_result makes it for a batch member."""
    try:
        m = lat.mass()
    except lbm.LBMError:
        return {"mass": float("nan"), "unstable": True}
    rho, _, _ = lat.fields()
    return {"mass": m, "rho_min": float(np.nanmin(rho)), "rho_max": float(np.nanmax(rho)),
            "unstable": False}


def run_one_at_a_time(requests, precision=lbm.FP64, make=request_lattice,
                      collect=lattice_result, clock=time.perf_counter, sleep=time.sleep):
    """The plain serving loop the continuous-batching server is compared with: requests in
    arrival order, one lattice at a time (created, stepped to its budget, its result read back,
    destroyed), the next one started when the previous is done and it has arrived.  Arrivals
    follow the clock from the start of the call; latency is arrival to result on the host.
    Returns Served records in completion order."""
    done = []
    t0 = clock()
    for req in sorted(requests, key=lambda r: r["arrival"]):
        wait = req["arrival"] - (clock() - t0)
        if wait > 0:
            sleep(wait)
        rec = Served(rid=req["rid"], arrival=req["arrival"], nodes=req["nx"] * req["ny"],
                     steps=req["steps"], admitted=clock() - t0)
        lat = make(req, precision)
        lat.step(req["steps"])
        rec.result = collect(lat) if collect else {}
        rec.fluid_nodes = lat.info()["n_fluid"]
        rec.finished = clock() - t0
        lat.close()
        done.append(rec)
    return done


def latency_stats(done):
    lat = np.array([r.latency for r in done])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}


def fifo_latencies(arrivals, service_times):
    """Latencies of a single FIFO server (one request at a time) for given arrival and service
    times: the plain one-lattice-at-a-time loop."""
    t = 0.0
    out = []
    for a, s in zip(arrivals, service_times):
        start = max(t, a)
        t = start + s
        out.append(t - a)
    return np.array(out)
