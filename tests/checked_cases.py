"""Small lattices over every kernel path, storage format and link stencil, for the
index-checking debug build (LBM_GB300_CHECKED=1 loads liblbm_gb300_checked.so).

Run as a script it prints one JSON object: case name -> sha256 of the case's fields and mass
(or its status).  tests/test_gpu_checked.py runs it with the checked and with the normal
library and compares; the checked library prints "LBM_OOB ..." for any index outside its buffer.
"""
import hashlib
import json

import numpy as np

from paper_1908_09235_gb300 import lbm, workloads

# 1040 x 256: vector-kernel tiles whose psi ring rows come by tensor copies (FP32 and FP16) and,
# for FP32, more than 152 CTAs, so the L2 prefetches of later tiles (with the flags map) run too
SHAPES = [(256, 192), (100, 100), (132, 68), (16, 12), (4, 130), (130, 4), (5, 6), (1040, 256)]
SCHEMES = [lbm.MOD_B, lbm.BOUZIDI_Q, lbm.ZHAO_YONG, lbm.HBB]
STEPS = 20


def _digest(lat):
    h = hashlib.sha256()
    for a in lat.fields():
        h.update(np.nan_to_num(a, nan=-7.0).tobytes())
    try:
        h.update(np.float64(lat.mass()).tobytes())
    except lbm.LBMError as e:
        h.update(b"status %d" % e.status)
    return h.hexdigest()


def _droplet(nx, ny, precision, path, scheme):
    eos = lbm.make_eos(lbm.EOS_CS, **workloads.CS)
    rl, rv = lbm.lbm_coexistence(eos)
    eos.rho_wall = rv
    r = max(1.0, 0.15 * min(nx, ny))
    cx, cy = nx / 2 + 0.3, 0.35 * ny + 0.2
    # a cylinder where it clears the periodic seam (lbm_create's rule), else none
    fits = cx - r - 2 >= 0 and cx + r + 2 <= nx - 1 and cy - r - 2 >= 0 and cy + r + 2 <= ny - 1
    lat = lbm.Lattice(nx, ny, 1.0, scheme, circles=[(cx, cy, r)] if fits else [], eos=eos,
                      precision=precision, kernel_path=path)
    lat.init_droplet(nx / 2, 0.35 * ny + r, max(1.0, 0.2 * min(nx, ny)), 4.0, rl, rv)
    return lat


def run_cases():
    out = {}
    for nx, ny in SHAPES:
        for precision in (lbm.FP64, lbm.FP32_DEV, lbm.FP16_DEV):
            paths = (0, 1, 3, 2) if precision == lbm.FP32_DEV else (0, 1, 3)
            for path in paths:
                for scheme in SCHEMES:
                    lat = _droplet(nx, ny, precision, path, scheme)
                    lat.step(STEPS)
                    out["%dx%d/p%d/k%d/s%d" % (nx, ny, precision, path, scheme)] = _digest(lat)
                    lat.close()
    # channel ends (Sec. 4.2) with the momentum exchange recorded
    for precision in (lbm.FP64, lbm.FP32_DEV, lbm.FP16_DEV):
        lat = lbm.Lattice(64, 20, 0.8, lbm.MOD_B, circles=[(20.3, 9.7, 4.1)],
                          eos=lbm.make_eos(lbm.EOS_NONE), precision=precision)
        lat.init_fields(np.ones(64 * 20))
        lat.set_inflow(0.05)
        lat.step(STEPS)
        out["channel/p%d" % precision] = _digest(lat) + " %r" % (lat.force(),)
        lat.close()
    # a batch of uneven lattices under every tile height and schedule
    ws = workloads.batched_domains(n=3, seed=workloads.SEED, side_lo=20, side_hi=70)
    for rows in (8, 16, 32):
        for sched in (lbm.SCHED_STRIDED, lbm.SCHED_CLAIM, lbm.SCHED_CLAIM_LARGEST_FIRST):
            b = lbm.Batch(lbm.FP32_DEV, lbm.EOS_CS, max_domains=3)
            slots = []
            for w in ws:
                eos = lbm.make_eos(lbm.EOS_CS, **w["eos"])
                rl, rv = lbm.lbm_coexistence(eos)
                eos.rho_wall = rv
                slots.append(b.add(lbm.make_domain(w["nx"], w["ny"], w["tau"], lbm.MOD_B,
                                                   circles=[w["cyl"]], eos=eos,
                                                   droplet=tuple(w["drop"]) + (rl, rv)), STEPS))
            b.set_schedule(rows, sched)
            b.step(STEPS)
            h = hashlib.sha256()
            for s in slots:
                for a in b.fields(s):
                    h.update(np.nan_to_num(a, nan=-7.0).tobytes())
            out["batch/r%d/s%d" % (rows, sched)] = h.hexdigest()
            b.close()
    return out


if __name__ == "__main__":
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(run_cases()), flush=True)
