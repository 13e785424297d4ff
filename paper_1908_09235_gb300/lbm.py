"""Python binding of the C ABI in include/lbm_gb300.h (ctypes; argument marshalling only).

Functions named ``lbm_*`` mirror the C entry points one to one.  ``Lattice`` bundles them for
convenience.  Device memory comes from PyTorch's caching allocator through the library's
allocation hook, and work runs on the caller's current torch CUDA stream.  There is no CPU
fallback: if the shared library cannot be loaded every call raises.
"""
import ctypes as C
import os
import threading

import numpy as np

from . import _build

HBB, FH, MLS, BOUZIDI_L, BOUZIDI_Q, ZHAO_YONG, MOD_A, MOD_B, BAO, BOUZIDI_L_A = range(10)
SCHEMES = {
    "hbb": HBB, "fh": FH, "mls": MLS, "bouzidi_l": BOUZIDI_L, "bouzidi_q": BOUZIDI_Q,
    "zhao_yong": ZHAO_YONG, "mod_a": MOD_A, "mod_b": MOD_B, "bao": BAO,
    "bouzidi_l_a": BOUZIDI_L_A,
}
FP64, FP32_DEV, FP16_DEV = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32_dev": FP32_DEV, "fp16_dev": FP16_DEV}
EOS_NONE, EOS_EXP, EOS_CS = 0, 1, 2
STATUS = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_EUNSTABLE",
          5: "LBM_ETIMEOUT", 6: "LBM_ESTATE"}

# Every entry point declared in include/lbm_gb300.h.
EXPORTS = ("lbm_create", "lbm_coexistence", "lbm_init_fields", "lbm_init_droplet", "lbm_step",
           "lbm_step_timed", "lbm_mass", "lbm_fields", "lbm_fields_device", "lbm_flags",
           "lbm_links", "lbm_info", "lbm_last_error", "lbm_status_string", "lbm_destroy",
           "lbm_mass_noalloc", "lbm_batch_create", "lbm_batch_add", "lbm_batch_remove",
           "lbm_batch_set_steps", "lbm_batch_step", "lbm_batch_step_timed", "lbm_batch_progress",
           "lbm_batch_domain", "lbm_batch_tune", "lbm_batch_info", "lbm_domain_bytes",
           "lbm_batch_last_error", "lbm_batch_destroy", "lbm_batch_poll", "lbm_set_inflow",
           "lbm_force", "lbm_batch_tune_trials", "lbm_batch_set_schedule", "lbm_state_bytes",
           "lbm_save_state", "lbm_load_state", "lbm_selftest_bounded_wait",
           "lbm_probe_fp64_fma")

# lbm_schedule: how the CTAs of a batch's step kernel take tiles from its queue
SCHED_STRIDED, SCHED_CLAIM, SCHED_CLAIM_LARGEST_FIRST = 0, 1, 2


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Circle(C.Structure):
    _fields_ = [("cx", C.c_double), ("cy", C.c_double), ("r", C.c_double),
                ("solid_outside", C.c_int32), ("pad", C.c_int32)]


class Geometry(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("n_circles", C.c_int32),
                ("pad", C.c_int32), ("circles", C.POINTER(Circle)),
                ("wall_q_lo", C.c_double), ("wall_q_hi", C.c_double)]


class Eos(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("G", C.c_double),
                ("psi0", C.c_double), ("rho0", C.c_double), ("a", C.c_double),
                ("b", C.c_double), ("R", C.c_double), ("T_over_Tc", C.c_double),
                ("rho_wall", C.c_double), ("gx", C.c_double), ("gy", C.c_double),
                ("azim_C", C.c_double), ("azim_cx", C.c_double), ("azim_cy", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("graph_steps", C.c_int32), ("stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
                ("rho_ref", C.c_double), ("kernel_path", C.c_int32), ("track_force", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("n_fluid", C.c_int64),
                ("n_boundary_nodes", C.c_int64), ("n_links", C.c_int64), ("steps", C.c_int64),
                ("device_bytes", C.c_int64), ("fallbacks", C.c_int64), ("T", C.c_double),
                ("psi_wall", C.c_double)]


class Domain(C.Structure):
    _fields_ = [("geometry", Geometry), ("eos", Eos), ("tau", C.c_double), ("scheme", C.c_int32),
                ("init", C.c_int32), ("cx", C.c_double), ("cy", C.c_double), ("R", C.c_double),
                ("W", C.c_double), ("rho_in", C.c_double), ("rho_out", C.c_double)]


class BatchInfo(C.Structure):
    _fields_ = [("active", C.c_int32), ("tiles", C.c_int32), ("tile_rows", C.c_int32),
                ("tile_cols", C.c_int32), ("nodes", C.c_int64), ("fluid_nodes", C.c_int64),
                ("boundary_links", C.c_int64), ("device_bytes", C.c_int64),
                ("schedule", C.c_int32), ("pad", C.c_int32)]


class TuneTrial(C.Structure):
    _fields_ = [("tile_rows", C.c_int32), ("schedule", C.c_int32), ("ms", C.c_double)]


_lib = None
_lock = threading.Lock()


def library_path():
    return _build.CHECKED_LIB if os.environ.get("LBM_GB300_CHECKED") == "1" else _build.LIB


def load_library(build_if_missing=True):
    """Load the CUDA library (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        checked = os.environ.get("LBM_GB300_CHECKED") == "1"  # index-checking debug build
        if build_if_missing:
            path = _build.build(checked=checked)
        else:
            path = _build.CHECKED_LIB if checked else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is missing; run __graft_entry__.build()" % path)
        lib = C.CDLL(path)
        P, D, V = C.c_void_p, C.POINTER(C.c_double), C.c_void_p
        sig = {
            "lbm_create": (C.c_int, [C.POINTER(Geometry), C.POINTER(Eos), C.c_double, C.c_int32,
                                     C.POINTER(Options), C.POINTER(C.c_void_p)]),
            "lbm_coexistence": (C.c_int, [C.POINTER(Eos), D, D]),
            "lbm_init_fields": (C.c_int, [P, V, V, V]),
            "lbm_init_droplet": (C.c_int, [P] + [C.c_double] * 6),
            "lbm_step": (C.c_int, [P, C.c_int32]),
            "lbm_step_timed": (C.c_int, [P, C.c_int32, D, D, D]),
            "lbm_mass": (C.c_int, [P, D]),
            "lbm_fields": (C.c_int, [P, V, V, V]),
            "lbm_fields_device": (C.c_int, [P, V, V, V]),
            "lbm_flags": (C.c_int, [P, V]),
            "lbm_links": (C.c_int, [P, V, V, V, C.POINTER(C.c_int64)]),
            "lbm_info": (C.c_int, [P, C.POINTER(Info)]),
            "lbm_last_error": (C.c_char_p, [P]),
            "lbm_status_string": (C.c_char_p, [C.c_int]),
            "lbm_destroy": (None, [P]),
            "lbm_mass_noalloc": (C.c_int, [V, V, C.c_int32, C.c_int32, C.c_int32, C.c_double, V,
                                           V, V]),
            "lbm_batch_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.POINTER(Options),
                                           C.POINTER(C.c_void_p)]),
            "lbm_batch_add": (C.c_int, [P, C.POINTER(Domain), C.c_int64, C.POINTER(C.c_int32)]),
            "lbm_batch_remove": (C.c_int, [P, C.c_int32]),
            "lbm_batch_set_steps": (C.c_int, [P, C.c_int32, C.c_int64]),
            "lbm_batch_step": (C.c_int, [P, C.c_int32]),
            "lbm_batch_step_timed": (C.c_int, [P, C.c_int32, D, D, D]),
            "lbm_batch_progress": (C.c_int, [P, C.c_int32, C.POINTER(C.c_int64),
                                             C.POINTER(C.c_int64)]),
            "lbm_batch_domain": (C.c_int, [P, C.c_int32, C.POINTER(C.c_void_p)]),
            "lbm_batch_tune": (C.c_int, [P, C.c_int32, C.POINTER(C.c_int32)]),
            "lbm_batch_info": (C.c_int, [P, C.POINTER(BatchInfo)]),
            "lbm_domain_bytes": (C.c_int, [C.POINTER(Domain), C.c_int32, C.POINTER(C.c_int64)]),
            "lbm_batch_last_error": (C.c_char_p, [P]),
            "lbm_batch_destroy": (None, [P]),
            "lbm_batch_poll": (C.c_int, [P, C.c_int32, C.POINTER(C.c_int64)]),
            "lbm_set_inflow": (C.c_int, [P, C.c_double]),
            "lbm_force": (C.c_int, [P, D, D]),
            "lbm_batch_tune_trials": (C.c_int, [P, C.c_int32, C.POINTER(TuneTrial),
                                                C.POINTER(C.c_int32)]),
            "lbm_batch_set_schedule": (C.c_int, [P, C.c_int32, C.c_int32]),
            "lbm_state_bytes": (C.c_int, [P, C.POINTER(C.c_int64)]),
            "lbm_save_state": (C.c_int, [P, C.c_void_p, C.c_int64]),
            "lbm_load_state": (C.c_int, [P, C.c_void_p, C.c_int64]),
            "lbm_selftest_bounded_wait": (C.c_int, [C.c_int64, C.c_int32, C.c_void_p,
                                                    C.POINTER(C.c_int32)]),
            "lbm_probe_fp64_fma": (C.c_int, [C.c_int32, C.c_void_p, D, D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(ctx, status):
    if status != 0:
        lib = load_library()
        msg = lib.lbm_last_error(ctx).decode() if ctx else lib.lbm_status_string(status).decode()
        raise LBMError(status, msg or lib.lbm_status_string(status).decode())


def make_geometry(nx, ny, circles=(), wall_q_lo=0.0, wall_q_hi=0.0):
    arr = (Circle * max(1, len(circles)))()
    for k, c in enumerate(circles):
        arr[k] = Circle(float(c[0]), float(c[1]), float(c[2]), int(c[3]) if len(c) > 3 else 0, 0)
    g = Geometry(int(nx), int(ny), len(circles), 0, C.cast(arr, C.POINTER(Circle)),
                 float(wall_q_lo), float(wall_q_hi))
    g._keep = arr
    return g


def make_eos(kind=EOS_NONE, G=0.0, psi0=1.0, rho0=1.0, a=0.25, b=4.0, R=1.0, T_over_Tc=0.0,
             rho_wall=1.0, gx=0.0, gy=0.0, azim_C=0.0, azim_cx=0.0, azim_cy=0.0):
    return Eos(kind, 0, G, psi0, rho0, a, b, R, T_over_Tc, rho_wall, gx, gy, azim_C, azim_cx,
               azim_cy)


# ---- thin wrappers with the C names ------------------------------------------------------------
def lbm_create(geometry, eos, tau, scheme, options=None):
    lib = load_library()
    out = C.c_void_p()
    st = lib.lbm_create(C.byref(geometry), C.byref(eos), float(tau), int(scheme),
                        C.byref(options) if options is not None else None, C.byref(out))
    _check(None, st)
    return out.value


def lbm_coexistence(eos):
    lib = load_library()
    rl, rv = C.c_double(), C.c_double()
    _check(None, lib.lbm_coexistence(C.byref(eos), C.byref(rl), C.byref(rv)))
    return rl.value, rv.value


def _host(a, n):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def lbm_init_fields(ctx, rho, ux=None, uy=None, n=None):
    lib = load_library()
    rho = _host(rho, n or np.size(rho))
    ux = _host(ux, rho.size)
    uy = _host(uy, rho.size)
    _check(ctx, lib.lbm_init_fields(ctx, rho.ctypes.data, ux.ctypes.data if ux is not None else None,
                                    uy.ctypes.data if uy is not None else None))


def lbm_init_droplet(ctx, cx, cy, R, W, rho_in, rho_out):
    _check(ctx, load_library().lbm_init_droplet(ctx, cx, cy, R, W, rho_in, rho_out))


def lbm_step(ctx, n):
    _check(ctx, load_library().lbm_step(ctx, int(n)))


def lbm_step_timed(ctx, n):
    a, b, t = C.c_double(), C.c_double(), C.c_double()
    _check(ctx, load_library().lbm_step_timed(ctx, int(n), C.byref(a), C.byref(b), C.byref(t)))
    return a.value, b.value, t.value


def lbm_mass(ctx):
    m = C.c_double()
    _check(ctx, load_library().lbm_mass(ctx, C.byref(m)))
    return m.value


def lbm_set_inflow(ctx, u_in):
    _check(ctx, load_library().lbm_set_inflow(ctx, float(u_in)))


def lbm_force(ctx):
    fx, fy = C.c_double(), C.c_double()
    _check(ctx, load_library().lbm_force(ctx, C.byref(fx), C.byref(fy)))
    return fx.value, fy.value


def lbm_save_state(ctx):
    """The context's state blob (checkpoint) as a numpy uint8 array."""
    import numpy as np
    n = C.c_int64()
    _check(ctx, load_library().lbm_state_bytes(ctx, C.byref(n)))
    buf = np.empty(n.value, dtype=np.uint8)
    _check(ctx, load_library().lbm_save_state(ctx, buf.ctypes.data, n.value))
    return buf


def lbm_load_state(ctx, blob):
    import numpy as np
    buf = np.ascontiguousarray(blob, dtype=np.uint8)
    _check(ctx, load_library().lbm_load_state(ctx, buf.ctypes.data, buf.size))


def lbm_selftest_bounded_wait(limit_ns, complete, stream=None):
    """(status, completed) of the bounded-wait self-test (status 5, LBM_ETIMEOUT, when the wait
    gave up); see include/lbm_gb300.h."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    done = C.c_int32(-1)
    st = load_library().lbm_selftest_bounded_wait(int(limit_ns), int(complete),
                                                  C.c_void_p(int(stream)), C.byref(done))
    return st, done.value


def lbm_probe_fp64_fma(iters=100000, stream=None):
    """(GFLOP/s, ms) of the FP64 FMA pipe, measured on the current device; see
    include/lbm_gb300.h."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    gf, ms = C.c_double(), C.c_double()
    st = load_library().lbm_probe_fp64_fma(int(iters), C.c_void_p(int(stream)), C.byref(gf),
                                           C.byref(ms))
    if st != 0:
        raise LBMError(st, "lbm_probe_fp64_fma")
    return gf.value, ms.value


def lbm_info(ctx):
    info = Info()
    _check(ctx, load_library().lbm_info(ctx, C.byref(info)))
    return {k: getattr(info, k) for k, _ in Info._fields_}


def lbm_fields(ctx, nx, ny):
    rho, ux, uy = (np.empty((ny, nx)) for _ in range(3))
    _check(ctx, load_library().lbm_fields(ctx, rho.ctypes.data, ux.ctypes.data, uy.ctypes.data))
    return rho, ux, uy


def lbm_fields_device(ctx, rho, ux, uy):
    """rho, ux, uy: device tensors (float64, nx*ny elements each)."""
    _check(ctx, load_library().lbm_fields_device(ctx, rho.data_ptr(), ux.data_ptr(),
                                                 uy.data_ptr()))


def lbm_flags(ctx, nx, ny):
    out = np.empty((ny, nx), dtype=np.uint8)
    _check(ctx, load_library().lbm_flags(ctx, out.ctypes.data))
    return out


def lbm_links(ctx):
    lib = load_library()
    n = C.c_int64(0)
    _check(ctx, lib.lbm_links(ctx, None, None, None, C.byref(n)))
    node = np.empty(n.value, dtype=np.int32)
    d = np.empty(n.value, dtype=np.uint8)
    q = np.empty(n.value, dtype=np.float64)
    _check(ctx, lib.lbm_links(ctx, node.ctypes.data, d.ctypes.data, q.ctypes.data, C.byref(n)))
    return node, d, q


def lbm_destroy(ctx):
    if ctx:
        load_library().lbm_destroy(ctx)


# ---- torch-backed device memory ------------------------------------------------------------------
class TorchDeviceMemory:
    """Allocation hook that hands out torch CUDA tensors (kept alive until freed)."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = device if device is not None else torch.device("cuda",
                                                                     torch.cuda.current_device())
        self.live = {}
        self.alloc_fn = ALLOC_FN(self._alloc)
        self.free_fn = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            t = self.torch.empty(int(nbytes) + 256, dtype=self.torch.uint8, device=self.device)
        except Exception:
            return None
        ptr = (t.data_ptr() + 255) // 256 * 256
        self.live[ptr] = t
        return ptr

    def _free(self, ptr, user):
        self.live.pop(ptr, None)


class Lattice:
    """One simulation on the current CUDA device (see include/lbm_gb300.h for the semantics)."""

    def __init__(self, nx, ny, tau, scheme=HBB, circles=(), wall_q_lo=0.0, wall_q_hi=0.0,
                 eos=None, precision=FP64, stream=None, torch_memory=True, graph_steps=0,
                 rho_ref=0.0, kernel_path=0, track_force=False, memory=None):
        self.nx, self.ny = int(nx), int(ny)
        if isinstance(scheme, str):
            scheme = SCHEMES[scheme]
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self.precision = precision
        self.geometry = make_geometry(nx, ny, circles, wall_q_lo, wall_q_hi)
        self.eos = eos if eos is not None else make_eos()
        self.mem = None
        opt = Options()
        opt.precision = precision
        opt.graph_steps = int(graph_steps)
        opt.rho_ref = float(rho_ref)
        opt.kernel_path = int(kernel_path)
        opt.track_force = int(bool(track_force))
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        opt.stream = C.c_void_p(int(stream))
        if memory is not None or torch_memory:  # memory: an allocation hook like TorchDeviceMemory
            self.mem = memory if memory is not None else TorchDeviceMemory()
            opt.alloc = self.mem.alloc_fn
            opt.free = self.mem.free_fn
        self.options = opt
        self.ctx = None
        self.ctx = lbm_create(self.geometry, self.eos, tau, scheme, opt)

    def close(self):
        if self.ctx:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_droplet(self, cx, cy, R, W, rho_in, rho_out):
        lbm_init_droplet(self.ctx, cx, cy, R, W, rho_in, rho_out)

    def init_fields(self, rho, ux=None, uy=None):
        lbm_init_fields(self.ctx, rho, ux, uy, self.nx * self.ny)

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def step_timed(self, n):
        return lbm_step_timed(self.ctx, n)

    def mass(self):
        return lbm_mass(self.ctx)

    def fields(self):
        return lbm_fields(self.ctx, self.nx, self.ny)

    def flags(self):
        return lbm_flags(self.ctx, self.nx, self.ny)

    def links(self):
        return lbm_links(self.ctx)

    def info(self):
        return lbm_info(self.ctx)

    def set_inflow(self, u_in):
        """Channel mode (Sec. 4.2): velocity inlet (u_in, 0) at x = 0, fully developed outlet."""
        lbm_set_inflow(self.ctx, u_in)

    def force(self):
        """Momentum-exchange force (fx, fy) on the solid nodes during the last step."""
        return lbm_force(self.ctx)

    def save_state(self):
        """Checkpoint: the state blob (numpy uint8) that load_state restores bit for bit."""
        return lbm_save_state(self.ctx)

    def load_state(self, blob):
        lbm_load_state(self.ctx, blob)


# ---- batches -------------------------------------------------------------------------------------
def make_domain(nx, ny, tau, scheme, circles=(), eos=None, droplet=None, rho=1.0, wall_q_lo=0.0,
                wall_q_hi=0.0):
    """A lattice description for Batch.add: droplet = (cx, cy, R, W, rho_in, rho_out), else a
    uniform density rho at rest."""
    if isinstance(scheme, str):
        scheme = SCHEMES[scheme]
    g = make_geometry(nx, ny, circles, wall_q_lo, wall_q_hi)
    d = Domain()
    d.geometry = g
    d.eos = eos if eos is not None else make_eos()
    d.tau = float(tau)
    d.scheme = int(scheme)
    if droplet is not None:
        d.init = 1
        d.cx, d.cy, d.R, d.W, d.rho_in, d.rho_out = (float(v) for v in droplet)
    else:
        d.init = 0
        d.rho_in = float(rho)
    d._keep = g._keep
    return d


def lbm_domain_bytes(domain, precision):
    n = C.c_int64()
    _check(None, load_library().lbm_domain_bytes(C.byref(domain), int(precision), C.byref(n)))
    return n.value


class Batch:
    """Many lattices of one precision and EOS kind advanced together (lbm_batch_* of the C ABI).
    Device memory comes from PyTorch's allocator unless torch_memory is False."""

    def __init__(self, precision=FP64, eos_kind=EOS_CS, max_domains=64, stream=None,
                 torch_memory=True, memory=None):
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        lib = load_library()
        opt = Options()
        opt.precision = precision
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        opt.stream = C.c_void_p(int(stream))
        self.mem = None
        if memory is not None or torch_memory:  # memory: an allocation hook like TorchDeviceMemory
            self.mem = memory if memory is not None else TorchDeviceMemory()
            opt.alloc = self.mem.alloc_fn
            opt.free = self.mem.free_fn
        self.options = opt
        self.precision = precision
        out = C.c_void_p()
        _check(None, lib.lbm_batch_create(precision, eos_kind, max_domains, C.byref(opt),
                                          C.byref(out)))
        self.b = out.value
        self.shapes = {}

    def _chk(self, st):
        if st != 0:
            raise LBMError(st, load_library().lbm_batch_last_error(self.b).decode()
                           or load_library().lbm_status_string(st).decode())

    def add(self, domain, steps):
        slot = C.c_int32()
        self._chk(load_library().lbm_batch_add(self.b, C.byref(domain), int(steps),
                                               C.byref(slot)))
        self.shapes[slot.value] = (domain.geometry.nx, domain.geometry.ny)
        return slot.value

    def remove(self, slot):
        self._chk(load_library().lbm_batch_remove(self.b, int(slot)))
        self.shapes.pop(slot, None)

    def set_steps(self, slot, steps):
        self._chk(load_library().lbm_batch_set_steps(self.b, int(slot), int(steps)))

    def step(self, n):
        self._chk(load_library().lbm_batch_step(self.b, int(n)))

    def step_timed(self, n):
        t, a, b = C.c_double(), C.c_double(), C.c_double()
        self._chk(load_library().lbm_batch_step_timed(self.b, int(n), C.byref(t), C.byref(a),
                                                      C.byref(b)))
        return t.value, a.value, b.value

    def progress(self, slot):
        done, left = C.c_int64(), C.c_int64()
        self._chk(load_library().lbm_batch_progress(self.b, int(slot), C.byref(done),
                                                    C.byref(left)))
        return done.value, left.value

    def poll(self, n):
        """steps left of slots 0..n-1 (-1: empty), one synchronisation"""
        arr = (C.c_int64 * max(1, n))()
        self._chk(load_library().lbm_batch_poll(self.b, int(n), arr))
        return list(arr)[:n]

    def ctx(self, slot):
        c = C.c_void_p()
        self._chk(load_library().lbm_batch_domain(self.b, int(slot), C.byref(c)))
        return c.value

    def mass(self, slot):
        return lbm_mass(self.ctx(slot))

    def fields(self, slot):
        nx, ny = self.shapes[slot]
        return lbm_fields(self.ctx(slot), nx, ny)

    def tune(self, trial_steps=5):
        """time every tile height and schedule, keep the fastest; returns the tile height"""
        rows = C.c_int32()
        self._chk(load_library().lbm_batch_tune(self.b, int(trial_steps), C.byref(rows)))
        return rows.value

    def tune_trials(self):
        """[(tile_rows, schedule, ms per step-kernel launch)] of the last tune, in timed order"""
        n = C.c_int32()
        self._chk(load_library().lbm_batch_tune_trials(self.b, 0, None, C.byref(n)))
        arr = (TuneTrial * max(1, n.value))()
        self._chk(load_library().lbm_batch_tune_trials(self.b, n.value, arr, C.byref(n)))
        return [(t.tile_rows, t.schedule, t.ms) for t in arr[:n.value]]

    def set_schedule(self, tile_rows, schedule):
        self._chk(load_library().lbm_batch_set_schedule(self.b, int(tile_rows), int(schedule)))

    def info(self):
        i = BatchInfo()
        self._chk(load_library().lbm_batch_info(self.b, C.byref(i)))
        return {k: getattr(i, k) for k, _ in BatchInfo._fields_}

    def close(self):
        if getattr(self, "b", None):
            load_library().lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
