"""The index-checking debug build: every computed global index of the step kernels (vectorised,
scalar, TMA-staged, batched), the wall pass and the channel ends stays inside its buffer on small,
ragged and self-wrapping lattices, and the checks change no result.

The cases of tests/checked_cases.py run twice in child processes: with the normal library and
with liblbm_gb300_checked.so (LBM_GB300_CHECKED=1), which reports an out-of-range index by device
printf ("LBM_OOB ...") and clamps the access instead of making it."""
import json
import os
import subprocess
import sys

import pytest

from paper_1908_09235_gb300 import _build

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _run(checked):
    env = dict(os.environ)
    env.pop("LBM_GB300_CHECKED", None)
    if checked:
        env["LBM_GB300_CHECKED"] = "1"
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    p = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py")], env=env,
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-2000:]
    lines = p.stdout.splitlines()
    js = [k for k, ln in enumerate(lines) if ln.startswith("{")]
    assert js, p.stdout[-2000:]
    return json.loads(lines[js[-1]]), lines[:js[-1]] + lines[js[-1] + 1:]


def test_checked_build_finds_no_out_of_range_index_and_changes_nothing(gpu_lib):
    _build.build(checked=True)
    checked, log = _run(True)
    oob = [ln for ln in log if "LBM_OOB" in ln]
    assert not oob, "\n".join(oob[:20])
    plain, _ = _run(False)
    assert set(checked) == set(plain) and len(plain) > 250
    differ = [k for k in plain if plain[k] != checked[k]]
    assert not differ, differ[:10]
