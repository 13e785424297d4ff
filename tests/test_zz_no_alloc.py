"""lbm_mass_noalloc: the total mass of caller-owned device arrays without any allocation.

Callers that cannot allocate device memory (a host framework that holds the device memory in its
own pool, or a latency-critical loop that must not call cudaMalloc, which may synchronise the
device) pass their population and flag arrays and get the FP64 mass and a status back on the
device.  Checked against lbm_mass, the ledger of a context, on the same state, with the FP64
ledger tolerance of the parity tests (1e-12 relative).  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1908_09235_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _populations(torch, rho, precision, rho_ref):
    """The populations lbm_init_fields(rho, u = 0) stores: f_a = w_a rho (FP64), or the FP32
    deviation w_a rho - w_a rho_ref."""
    r = torch.from_numpy(rho).cuda()
    w = torch.tensor(W, dtype=torch.float64, device="cuda")[:, None, None]
    if precision == lbm.FP64:
        return (w * r).contiguous()
    return (w * r - w * rho_ref).to(torch.float32).contiguous()


def _call(lib, torch, f, flags, nx, ny, precision, rho_ref, out, status):
    st = lib.lbm_mass_noalloc(f.data_ptr(), flags.data_ptr() if flags is not None else None, nx,
                              ny, precision, rho_ref, out.data_ptr(), status.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, float(out.item()), int(status.item())


CASES = [
    dict(nx=100, ny=100, circles=[(50.0, 35.0, 15.0)], precision=lbm.FP64, rho_ref=0.0),
    dict(nx=257, ny=190, circles=[(60.5, 80.25, 20.0), (180.0, 100.0, 33.3)],
         precision=lbm.FP32_DEV, rho_ref=0.5),
]


def test_mass_noalloc_matches_lbm_mass(gpu_lib):
    import torch
    lib = lbm.load_library()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(workloads.SEED)
    for case in CASES:
        nx, ny = case["nx"], case["ny"]
        lat = lbm.Lattice(nx, ny, 1.0, lbm.HBB, circles=case["circles"],
                          precision=case["precision"], rho_ref=case["rho_ref"] or 0.0)
        rho = rng.uniform(0.2, 2.0, (ny, nx))
        lat.init_fields(rho)
        m_ref = lat.mass()
        flags = torch.from_numpy(np.ascontiguousarray(lat.flags())).cuda()
        lat.close()
        f = _populations(torch, rho, case["precision"], case["rho_ref"])
        results = []
        for _ in range(2):  # two calls in a row on the shared scratch
            st, m, s = _call(lib, torch, f, flags, nx, ny, case["precision"], case["rho_ref"],
                             out, status)
            assert st == 0 and s == 0
            assert abs(m - m_ref) <= 1e-12 * m_ref, (m, m_ref)
            results.append(m)
        assert results[0] == results[1]  # fixed reduction order


def test_mass_noalloc_status_does_not_stick(gpu_lib):
    import torch
    lib = lbm.load_library()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    nx, ny = 64, 48
    rho = np.full((ny, nx), 1.0)
    f = _populations(torch, rho, lbm.FP64, 0.0)
    f_bad = f.clone()
    f_bad[0, 10, 10] = float("nan")
    st, _, s = _call(lib, torch, f_bad, None, nx, ny, lbm.FP64, 0.0, out, status)
    assert st == 0 and s == 4  # LBM_EUNSTABLE
    st, m, s = _call(lib, torch, f, None, nx, ny, lbm.FP64, 0.0, out, status)
    assert st == 0 and s == 0
    assert abs(m - nx * ny) <= 1e-12 * nx * ny


def test_mass_noalloc_rejects_lattices_beyond_its_scratch(gpu_lib):
    import torch
    lib = lbm.load_library()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # 8193 x 8193 nodes exceed the 8192 x 8192 the fixed scratch covers: rejected before launch
    st = lib.lbm_mass_noalloc(out.data_ptr(), None, 8193, 8193, lbm.FP64, 0.0, out.data_ptr(),
                              status.data_ptr(), None)
    assert st == 1
    assert C.c_int(st).value == 1
