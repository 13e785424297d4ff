"""ctypes binding of the C oracle (TEST INFRASTRUCTURE ONLY).

Builds ``oracle/_build/liblbm_oracle.so`` from ``lbm_oracle.c`` with gcc on first use
(``-O2 -ffp-contract=off``: no fused multiply-add, no fast-math) and wraps it.
"""
import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
HDR = os.path.join(HERE, "lbm_oracle.h")
BUILD_DIR = os.path.join(HERE, "_build")

HBB, FH, MLS, BOUZIDI_L, BOUZIDI_Q, ZHAO_YONG, MOD_A, MOD_B, BAO, BOUZIDI_L_A = range(10)
SCHEME_NAMES = {
    HBB: "hbb", FH: "fh", MLS: "mls", BOUZIDI_L: "bouzidi_l", BOUZIDI_Q: "bouzidi_q",
    ZHAO_YONG: "zhao_yong", MOD_A: "mod_a", MOD_B: "mod_b", BAO: "bao",
    BOUZIDI_L_A: "bouzidi_l_a",
}
EOS_NONE, EOS_EXP, EOS_CS = 0, 1, 2

_lock = threading.Lock()
_libs = {}  # openmp flag -> loaded library


def library_path(openmp=False):
    return os.path.join(BUILD_DIR, "liblbm_oracle_omp.so" if openmp else "liblbm_oracle.so")


def build_oracle(force=False, openmp=False):
    """Compile the oracle with gcc (openmp: the same source with -fopenmp, its node loops on all
    host cores).  Returns the path of the shared library."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    out = library_path(openmp)
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        tmp = out + ".%d.tmp" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
             *(["-fopenmp"] if openmp else []), SRC, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


class _Circle(C.Structure):
    _fields_ = [("cx", C.c_double), ("cy", C.c_double), ("r", C.c_double),
                ("solid_outside", C.c_int32), ("pad", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("n_circles", C.c_int32),
                ("pad0", C.c_int32), ("circles", C.POINTER(_Circle)),
                ("wall_q_lo", C.c_double), ("wall_q_hi", C.c_double),
                ("eos", C.c_int32), ("scheme", C.c_int32),
                ("G", C.c_double), ("psi0", C.c_double), ("rho0", C.c_double),
                ("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("T", C.c_double),
                ("rho_wall", C.c_double), ("gx", C.c_double), ("gy", C.c_double),
                ("azim_C", C.c_double), ("azim_cx", C.c_double), ("azim_cy", C.c_double),
                ("tau", C.c_double)]


_D = C.POINTER(C.c_double)
_P = C.c_void_p


def _load(openmp=False):
    with _lock:
        if openmp in _libs:
            return _libs[openmp]
        lib = C.CDLL(build_oracle(openmp=openmp))
        sig = {
            "or_feq": (None, [C.c_double, C.c_double, C.c_double, _D]),
            "or_guo": (None, [C.c_double] * 5 + [_D]),
            "or_collide_node": (None, [_D, C.c_double, C.c_double, C.c_double, _D]),
            "or_psi": (C.c_double, [C.POINTER(_Params), C.c_double]),
            "or_cs_pressure": (C.c_double, [C.c_double] * 5),
            "or_force_from_psi": (None, [C.c_int, C.c_int, C.c_double, _D, _D, _D]),
            "or_cs_critical": (C.c_int, [C.c_double] * 3 + [_D, _D]),
            "or_cs_coexistence": (C.c_int, [C.c_double] * 4 + [_D, _D]),
            "or_create": (_P, [C.POINTER(_Params)]),
            "or_destroy": (None, [_P]),
            "or_num_links": (C.c_int, [_P]),
            "or_num_boundary_nodes": (C.c_int, [_P]),
            "or_flags": (None, [_P, C.c_void_p]),
            "or_links": (None, [_P, C.c_void_p, C.c_void_p, C.c_void_p]),
            "or_init_fields": (None, [_P, C.c_void_p, C.c_void_p, C.c_void_p]),
            "or_init_droplet": (None, [_P] + [C.c_double] * 6),
            "or_step": (None, [_P, C.c_int]),
            "or_mass": (C.c_double, [_P]),
            "or_fields": (None, [_P, C.c_void_p, C.c_void_p, C.c_void_p]),
            "or_get_f": (None, [_P, C.c_void_p]),
            "or_set_f": (None, [_P, C.c_void_p]),
            "or_last_leak": (C.c_double, [_P]),
            "or_last_max_node_leak": (C.c_double, [_P]),
            "or_fallbacks": (C.c_long, [_P]),
            "or_set_inflow": (None, [_P, C.c_double]),
            "or_force": (None, [_P, _D, _D]),
            "or_num_threads": (C.c_int, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _libs[openmp] = lib
        return lib


def num_threads(openmp=False):
    """Threads the oracle's per-node loops use in the serial (1) or the -fopenmp build."""
    return _load(openmp).or_num_threads()


def _dptr(a):
    return a.ctypes.data_as(_D)


def _vec(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def feq(rho, ux, uy):
    out = np.zeros(9)
    _load().or_feq(rho, ux, uy, _dptr(out))
    return out


def guo(tau, ux, uy, Fx, Fy):
    out = np.zeros(9)
    _load().or_guo(tau, ux, uy, Fx, Fy, _dptr(out))
    return out


def collide_node(f, tau, Fx, Fy):
    f = _vec(f)
    out = np.zeros(9)
    _load().or_collide_node(_dptr(f), tau, Fx, Fy, _dptr(out))
    return out


def _params(nx=8, ny=8, circles=(), wall_q_lo=0.0, wall_q_hi=0.0, eos=EOS_NONE, scheme=HBB,
            G=0.0, psi0=1.0, rho0=1.0, a=0.25, b=4.0, R=1.0, T=0.0, rho_wall=1.0, gx=0.0,
            gy=0.0, azim_C=0.0, azim_cx=0.0, azim_cy=0.0, tau=1.0):
    carr = (_Circle * max(1, len(circles)))()
    for k, c in enumerate(circles):
        cx, cy, r = c[0], c[1], c[2]
        outside = int(c[3]) if len(c) > 3 else 0
        carr[k] = _Circle(cx, cy, r, outside, 0)
    p = _Params(nx, ny, len(circles), 0, C.cast(carr, C.POINTER(_Circle)), wall_q_lo,
                wall_q_hi, eos, scheme, G, psi0, rho0, a, b, R, T, rho_wall, gx, gy, azim_C,
                azim_cx, azim_cy, tau)
    return p, carr


def psi(rho, **kw):
    p, _keep = _params(**kw)
    return _load().or_psi(C.byref(p), rho)


def cs_pressure(a, b, R, T, rho):
    return _load().or_cs_pressure(a, b, R, T, rho)


def force_from_psi(psi_field, G):
    psi_field = _vec(psi_field)
    ny, nx = psi_field.shape
    Fx = np.zeros_like(psi_field)
    Fy = np.zeros_like(psi_field)
    _load().or_force_from_psi(nx, ny, G, _dptr(psi_field), _dptr(Fx), _dptr(Fy))
    return Fx, Fy


def cs_critical(a, b, R):
    Tc, rhoc = C.c_double(), C.c_double()
    _load().or_cs_critical(a, b, R, C.byref(Tc), C.byref(rhoc))
    return Tc.value, rhoc.value


def cs_coexistence(a, b, R, T):
    rl, rv = C.c_double(), C.c_double()
    rc = _load().or_cs_coexistence(a, b, R, T, C.byref(rl), C.byref(rv))
    if rc != 0:
        raise ValueError("no coexistence above the critical temperature")
    return rl.value, rv.value


class OracleSim:
    """One FP64 oracle simulation.  Keyword arguments mirror ``or_params`` in lbm_oracle.h;
    for the Carnahan-Starling EOS pass either ``T`` or ``T_over_Tc``.  openmp: run it in the
    -fopenmp build (same bits; threads from OMP_NUM_THREADS, else all host cores)."""

    def __init__(self, nx, ny, tau, scheme=HBB, circles=(), T_over_Tc=None, openmp=False, **kw):
        lib = _load(openmp)
        if T_over_Tc is not None:
            Tc, _ = cs_critical(kw.get("a", 0.25), kw.get("b", 4.0), kw.get("R", 1.0))
            kw["T"] = T_over_Tc * Tc
        self.params, self._carr = _params(nx=nx, ny=ny, circles=circles, scheme=scheme,
                                          tau=tau, **kw)
        self.nx, self.ny = nx, ny
        self._lib = lib
        self._s = lib.or_create(C.byref(self.params))

    def __del__(self):
        s = getattr(self, "_s", None)
        if s:
            self._lib.or_destroy(s)
            self._s = None

    @property
    def n_links(self):
        return self._lib.or_num_links(self._s)

    @property
    def n_boundary_nodes(self):
        return self._lib.or_num_boundary_nodes(self._s)

    def flags(self):
        out = np.zeros((self.ny, self.nx), dtype=np.uint8)
        self._lib.or_flags(self._s, out.ctypes.data)
        return out

    def links(self):
        nl = self.n_links
        node = np.zeros(nl, dtype=np.int32)
        d = np.zeros(nl, dtype=np.uint8)
        q = np.zeros(nl, dtype=np.float64)
        self._lib.or_links(self._s, node.ctypes.data, d.ctypes.data, q.ctypes.data)
        return node, d, q

    def init_fields(self, rho, ux=None, uy=None):
        rho = _vec(rho)
        ux = _vec(ux) if ux is not None else np.zeros_like(rho)
        uy = _vec(uy) if uy is not None else np.zeros_like(rho)
        self._lib.or_init_fields(self._s, rho.ctypes.data, ux.ctypes.data, uy.ctypes.data)

    def init_droplet(self, cx, cy, R, W, rho_in, rho_out):
        self._lib.or_init_droplet(self._s, cx, cy, R, W, rho_in, rho_out)

    def step(self, n=1):
        self._lib.or_step(self._s, int(n))

    def mass(self):
        return self._lib.or_mass(self._s)

    def fields(self):
        shp = (self.ny, self.nx)
        rho, ux, uy = np.zeros(shp), np.zeros(shp), np.zeros(shp)
        self._lib.or_fields(self._s, rho.ctypes.data, ux.ctypes.data, uy.ctypes.data)
        return rho, ux, uy

    def get_f(self):
        f = np.zeros((9, self.ny, self.nx))
        self._lib.or_get_f(self._s, f.ctypes.data)
        return f

    def set_f(self, f):
        f = _vec(f).reshape(9, self.ny, self.nx)
        self._lib.or_set_f(self._s, f.ctypes.data)

    @property
    def last_leak(self):
        return self._lib.or_last_leak(self._s)

    @property
    def last_max_node_leak(self):
        return self._lib.or_last_max_node_leak(self._s)

    @property
    def fallbacks(self):
        return self._lib.or_fallbacks(self._s)

    def set_inflow(self, u_in):
        """Channel mode (Sec. 4.2): Zou-He velocity inlet at i = 0, fully developed outlet at
        i = nx - 1; single-phase flows."""
        self._lib.or_set_inflow(self._s, float(u_in))

    def force(self):
        """Momentum-exchange force (fx, fy) on the solid nodes during the last step."""
        fx, fy = C.c_double(), C.c_double()
        self._lib.or_force(self._s, C.byref(fx), C.byref(fy))
        return fx.value, fy.value
