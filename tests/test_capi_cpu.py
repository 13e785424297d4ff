"""The C-ABI library builds, loads and exports every declared entry point; host-side logic that
needs no GPU (argument validation, the Carnahan-Starling set-up) behaves as documented."""
import ctypes as C
import math
import re

import pytest

import oracle as O
from paper_1908_09235_gb300 import _build, lbm

HEADER = "include/lbm_gb300.h"
O_CS = dict(a=0.25, b=4.0, R=1.0, T_over_Tc=0.86, G=-1.0)


def _declared():
    import os
    src = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), HEADER)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = _build.build()
    lib = C.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(lbm.EXPORTS)


def test_coexistence_matches_oracle():
    for t in (0.7, 0.8, 0.86, 0.9, 0.95):
        eos = lbm.make_eos(lbm.EOS_CS, G=-1.0, a=0.25, b=4.0, R=1.0, T_over_Tc=t)
        rl, rv = lbm.lbm_coexistence(eos)
        Tc, _ = O.cs_critical(0.25, 4.0, 1.0)
        ol, ov = O.cs_coexistence(0.25, 4.0, 1.0, t * Tc)
        assert rl == pytest.approx(ol, rel=1e-12)
        assert rv == pytest.approx(ov, rel=1e-12)


def test_coexistence_rejects_supercritical():
    eos = lbm.make_eos(lbm.EOS_CS, G=-1.0, T_over_Tc=1.05)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_coexistence(eos)
    assert e.value.status == 1


@pytest.mark.parametrize("kw", [
    dict(tau=0.5),                                        # tau must exceed 1/2
    dict(tau=float("nan")),
    dict(scheme=lbm.FH, tau=1.0),                         # chi of Eq. (9) is singular
    dict(scheme=42),
    dict(nx=3),
    dict(nx=16384, ny=16384),                             # 9 nx ny must stay below 2^31
    dict(circles=[(3.0, 50.0, 10.0)]),                    # crosses the periodic seam
    dict(circles=[(50.0, 50.0, -1.0)]),
    dict(eos=lbm.make_eos(lbm.EOS_CS, G=1.0, T_over_Tc=0.86)),  # CS needs G < 0
    dict(eos=lbm.make_eos(lbm.EOS_EXP, G=0.0)),
    dict(precision=7),
])
def test_create_rejects_invalid_arguments_before_touching_the_gpu(kw):
    # Validation happens before any CUDA call, so this runs without a GPU.
    args = dict(nx=100, ny=100, tau=1.0, scheme=lbm.HBB, circles=[(50.0, 35.0, 15.0)],
                eos=lbm.make_eos(), precision=lbm.FP64)
    args.update(kw)
    geo = lbm.make_geometry(args["nx"], args.get("ny", 100), args["circles"])
    opt = lbm.Options()
    opt.precision = args["precision"]
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_create(geo, args["eos"], args["tau"], args["scheme"], opt)
    assert e.value.status == 1


def test_status_strings():
    lib = lbm.load_library()
    for s in range(7):
        assert lib.lbm_status_string(s).decode()
    assert not math.isnan(1.0)


# C structs of the header and their ctypes mirrors in the binding: same size and field offsets
_STRUCTS = {"lbm_circle": "Circle", "lbm_geometry": "Geometry", "lbm_eos": "Eos",
            "lbm_options": "Options", "lbm_info_t": "Info", "lbm_domain": "Domain",
            "lbm_batch_info_t": "BatchInfo", "lbm_tune_trial": "TuneTrial"}


def test_header_is_plain_c_and_matches_the_binding_layouts():
    import os
    import pathlib
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    tmp_path = pathlib.Path(_build.LIBDIR) / "layout_check"  # in-tree build directory
    tmp_path.mkdir(parents=True, exist_ok=True)
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "lbm_gb300.h"',
             "int main(void) {"]
    for cname, pyname in _STRUCTS.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in getattr(lbm, pyname)._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));'
                         % (cname, field, cname, field))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    # plain C99 with warnings as errors: no C++ or CUDA types in the interface
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                           str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        key, value = line.rsplit(" ", 1)
        got[key] = int(value)
    for cname, pyname in _STRUCTS.items():
        py = getattr(lbm, pyname)
        assert got["%s size" % cname] == C.sizeof(py), cname
        for field, _ in py._fields_:
            assert got["%s %s" % (cname, field)] == getattr(py, field).offset, (cname, field)


def test_domain_bytes_estimate_is_host_only_and_ordered():
    # the server's admission estimate (no GPU needed): grows with the lattice, FP64 > FP32 > FP16
    def dom(L):
        eos = lbm.make_eos(lbm.EOS_CS, **O_CS)
        return lbm.make_domain(L, L, 1.0, lbm.MOD_B, circles=[(L / 2, 0.35 * L, 0.15 * L)],
                               eos=eos, droplet=(L / 2, 0.5 * L, 0.2 * L, 5.0, 0.27, 0.034))
    sizes = {}
    for L in (128, 512):
        for prec in (lbm.FP64, lbm.FP32_DEV, lbm.FP16_DEV):
            sizes[L, prec] = lbm.lbm_domain_bytes(dom(L), prec)
    for L in (128, 512):
        assert sizes[L, lbm.FP64] > sizes[L, lbm.FP32_DEV] > sizes[L, lbm.FP16_DEV]
        # at least the two lattices of populations
        assert sizes[L, lbm.FP32_DEV] >= 2 * 36 * L * L
    assert all(sizes[512, p] > 10 * sizes[128, p] for p in (lbm.FP64, lbm.FP32_DEV))


def test_new_entry_points_reject_invalid_arguments_without_a_gpu():
    # argument checks come before any CUDA call (documented error behaviour of the header)
    lib = lbm.load_library()
    n = C.c_int64()
    done = C.c_int32()
    assert lib.lbm_state_bytes(None, C.byref(n)) == 1
    assert lib.lbm_save_state(None, None, 0) == 1
    assert lib.lbm_load_state(None, None, 0) == 1
    for limit in (0, -5, 10**11):  # outside 1 .. 1e10 ns
        assert lib.lbm_selftest_bounded_wait(limit, 1, None, C.byref(done)) == 1
    assert lib.lbm_selftest_bounded_wait(1000, 1, None, None) == 1
    gf, ms = C.c_double(), C.c_double()
    for iters in (0, -1, 2**24 + 1):
        assert lib.lbm_probe_fp64_fma(iters, None, C.byref(gf), C.byref(ms)) == 1
    assert lib.lbm_probe_fp64_fma(1000, None, None, C.byref(ms)) == 1
    assert lib.lbm_batch_set_schedule(None, 16, lbm.SCHED_CLAIM) == 1
    assert lib.lbm_batch_tune(None, 3, None) == 1
    cnt = C.c_int32()
    assert lib.lbm_batch_tune_trials(None, 0, None, C.byref(cnt)) == 1
    assert lib.lbm_set_inflow(None, 0.05) == 1
    fx, fy = C.c_double(), C.c_double()
    assert lib.lbm_force(None, C.byref(fx), C.byref(fy)) == 1
