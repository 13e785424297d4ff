"""In-tree build of the CUDA library ``_lib/liblbm_gb300.so`` for sm_103a (GB300).

Each translation unit is compiled in parallel with nvcc (one ``-gencode``), then linked into a
shared library with a plain C ABI (include/lbm_gb300.h).  Nothing is installed.  The debug
variant ``_lib/liblbm_gb300_checked.so`` (``checked=True``, macro LBM_CHECKED) checks the
kernels' computed indices (device printf "LBM_OOB ..." and a clamped access instead of an
out-of-range one); it is loaded when LBM_GB300_CHECKED=1.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liblbm_gb300.so")
CHECKED_LIB = os.path.join(LIBDIR, "liblbm_gb300_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_SOURCES = ["step.cu", "step_vec.cu", "step_tma.cu", "boundary.cu", "geometry.cu", "ledger.cu", "capi.cu",
                "batch.cu", "mass_noalloc.cu", "probe.cu"]
CXX_SOURCES = ["eos_host.cpp"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _sources():
    names = CUDA_SOURCES + CXX_SOURCES + ["d2q9.cuh", "step_core.cuh", "tma.cuh", "lbm_internal.h"]
    paths = [os.path.join(CSRC, n) for n in names]
    paths.append(os.path.join(os.path.dirname(HERE), "include", "lbm_gb300.h"))
    paths.append(os.path.abspath(__file__))
    return paths


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _sources())


def build(force=False, verbose=False, checked=False):
    """Compile the library (checked: the index-checking debug variant) if any source is newer
    than it.  Returns the library path."""
    lib = CHECKED_LIB if checked else LIB
    if not force and up_to_date(lib):
        return lib
    nvcc = _nvcc()
    objdir = os.path.join(LIBDIR, "obj_checked" if checked else "obj")
    defs = ["-DLBM_CHECKED"] if checked else []
    os.makedirs(objdir, exist_ok=True)
    procs = []
    for src in CUDA_SOURCES:
        obj = os.path.join(objdir, src + ".o")
        # The wall pass is compiled without multiply-add contraction: its per-link arithmetic is
        # inlined into the single-lattice and the batched kernels, and must round identically in
        # both so a lattice gives the same bits alone and in a batch.
        fmad = ["--fmad=false"] if src == "boundary.cu" else []
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", *fmad, *defs, "-Xcompiler", "-fPIC",
               "-Xcompiler", "-ffp-contract=off", "-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
    for src in CXX_SOURCES:
        obj = os.path.join(objdir, src + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I" + cuda_inc, "-c",
               os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("building the CUDA library failed:\n" + msg)
    objs = [os.path.join(objdir, s + ".o") for s in CUDA_SOURCES + CXX_SOURCES]
    tmp = lib + ".%d.tmp" % os.getpid()
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
