"""ctypes wrapper of the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the
CPU-baseline leg of the benchmark.  The product path never loads it.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", f"liblbm_oracle_{platform.machine()}.so")
_lib = None
_lock = threading.Lock()

_BC_IN = {"inlet": 0, "periodic": 1}
_BC_OUT = {"outflow": 0, "wall": 1, "periodic": 2}
_BC_TOP = {"wall": 0, "open": 1}
_BC_BOTTOM = {"axis": 0, "wall": 1}


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("nr", C.c_int),
        ("bc_in", C.c_int), ("bc_out", C.c_int), ("bc_top", C.c_int), ("bc_bottom", C.c_int),
        ("axisym", C.c_int), ("nthreads", C.c_int),
        ("r0", C.c_double), ("rho0", C.c_double), ("T0", C.c_double),
        ("Cs", C.c_double), ("Pr_t", C.c_double),
        ("T_top", C.c_double), ("T_bottom", C.c_double), ("T_out", C.c_double),
        ("noise_amp", C.c_double), ("seed", C.c_uint64),
    ]


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source file with gcc (C99, OpenMP, no FMA contraction)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-fvisibility=hidden", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (once; again when the source is newer than the library)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


def lib():
    """The oracle library; ORACLE_LIB names a prebuilt one (the mutation tests use it)."""
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(os.environ.get("ORACLE_LIB") or build())
            dp = C.POINTER(C.c_double)
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.POINTER(_Params)]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_set_inlet.argtypes = [C.c_void_p, dp, dp]
            L.orc_set_properties.restype = C.c_int
            L.orc_set_properties.argtypes = [C.c_void_p, dp, dp, C.c_int, C.c_double, C.c_double]
            L.orc_set_state.argtypes = [C.c_void_p, dp, dp, C.c_longlong]
            L.orc_get_state.argtypes = [C.c_void_p, dp, dp]
            L.orc_get_step.restype = C.c_longlong
            L.orc_get_step.argtypes = [C.c_void_p]
            L.orc_step.argtypes = [C.c_void_p, C.c_int]
            L.orc_get_fields.argtypes = [C.c_void_p, dp]
            L.orc_get_streamed.argtypes = [C.c_void_p, dp, dp]
            L.orc_splitmix64.restype = C.c_uint64
            L.orc_splitmix64.argtypes = [C.c_uint64]
            L.orc_inlet_noise.restype = C.c_double
            L.orc_inlet_noise.argtypes = [C.c_uint64, C.c_longlong, C.c_int, C.c_double]
            L.orc_feq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
            L.orc_geq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
            L.orc_moments.argtypes = [dp, dp, dp]
            L.orc_tau_total.restype = C.c_double
            L.orc_tau_total.argtypes = [C.c_double, C.c_double, dp]
            L.orc_property.restype = C.c_double
            L.orc_property.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double]
            L.orc_collide_node.argtypes = [dp, dp, C.c_double, dp, C.c_double, C.c_double,
                                           C.c_double, C.c_double, C.c_int, dp, dp, dp]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- node-level functions -------------------------------------------------

def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def inlet_noise(seed: int, step: int, j: int, amp: float) -> float:
    return float(lib().orc_inlet_noise(C.c_uint64(seed), step, j, amp))


def feq(rho: float, ux: float, ur: float) -> np.ndarray:
    out = np.empty(9)
    lib().orc_feq(rho, ux, ur, _p(out))
    return out


def geq(T: float, ux: float, ur: float) -> np.ndarray:
    out = np.empty(4)
    lib().orc_geq(T, ux, ur, _p(out))
    return out


def moments(f, g) -> np.ndarray:
    f = _f64(f)
    g = _f64(g)
    out = np.empty(4)
    lib().orc_moments(_p(f), _p(g), _p(out))
    return out


def tau_total(tau_nu: float, Cs: float, f) -> float:
    f = _f64(f)
    return float(lib().orc_tau_total(tau_nu, Cs, _p(f)))


def prop(tab, T_lo: float, T_hi: float, T: float) -> float:
    tab = _f64(tab)
    return float(lib().orc_property(_p(tab), len(tab), T_lo, T_hi, T))


def collide_node(fs, gs, r, d, nu, alpha, Cs, Pr_t, axisym=True):
    """Post-collision populations of one node and {tau, tau_alpha, F1, F2x, F2r, S}."""
    fs = _f64(fs)
    gs = _f64(gs)
    d = _f64(d)
    fo = np.empty(9)
    go = np.empty(4)
    diag = np.empty(6)
    lib().orc_collide_node(_p(fs), _p(gs), r, _p(d), nu, alpha, Cs, Pr_t, int(axisym),
                           _p(fo), _p(go), _p(diag))
    return fo, go, diag


# ---- whole lattice --------------------------------------------------------

class Oracle:
    """One lattice advanced by the FP64 oracle."""

    def __init__(self, cfg, nthreads: int = 1):
        cfg.validate()
        self.cfg = cfg
        self.nx, self.nr = cfg.nx, cfg.nr
        p = _Params(nx=cfg.nx, nr=cfg.nr, bc_in=_BC_IN[cfg.bc_in], bc_out=_BC_OUT[cfg.bc_out],
                    bc_top=_BC_TOP[cfg.bc_top], bc_bottom=_BC_BOTTOM[cfg.bc_bottom],
                    axisym=int(cfg.axisym), nthreads=int(nthreads), r0=cfg.r0, rho0=cfg.rho0,
                    T0=cfg.T0, Cs=cfg.Cs, Pr_t=cfg.Pr_t, T_top=cfg.T_top,
                    T_bottom=cfg.T_bottom, T_out=cfg.T_out, noise_amp=cfg.noise_amp,
                    seed=cfg.seed & 0xFFFFFFFFFFFFFFFF)
        self._L = lib()
        self._h = self._L.orc_create(C.byref(p))
        if not self._h:
            raise ValueError("oracle rejected the lattice description")

    @classmethod
    def from_workload(cls, w, nthreads: int = 1) -> "Oracle":
        o = cls(w.cfg, nthreads)
        o.set_inlet(w.u_in, w.T_in)
        o.set_properties(w.nu_tab, w.alpha_tab, w.T_lo, w.T_hi)
        return o

    def close(self):
        if getattr(self, "_h", None):
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def set_inlet(self, u_in, T_in):
        u = _f64(u_in)
        T = _f64(T_in)
        assert u.shape == (self.nr,) and T.shape == (self.nr,)
        self._L.orc_set_inlet(self._h, _p(u), _p(T))

    def set_properties(self, nu_tab, alpha_tab, T_lo, T_hi):
        a = _f64(nu_tab)
        b = _f64(alpha_tab)
        if self._L.orc_set_properties(self._h, _p(a), _p(b), len(a), T_lo, T_hi) != 0:
            raise ValueError("bad property table")

    def set_state(self, f, g, step: int = 0):
        f = _f64(f)
        g = _f64(g)
        assert f.shape == (9, self.nr, self.nx) and g.shape == (4, self.nr, self.nx)
        self._L.orc_set_state(self._h, _p(f), _p(g), step)

    def get_state(self):
        f = np.empty((9, self.nr, self.nx))
        g = np.empty((4, self.nr, self.nx))
        self._L.orc_get_state(self._h, _p(f), _p(g))
        return f, g

    @property
    def step_count(self) -> int:
        return int(self._L.orc_get_step(self._h))

    def step(self, n: int = 1):
        self._L.orc_step(self._h, int(n))

    def fields(self) -> np.ndarray:
        """(4, nr, nx): rho, u_x, u_r, T at the current time."""
        out = np.empty((4, self.nr, self.nx))
        self._L.orc_get_fields(self._h, _p(out))
        return out

    def streamed(self):
        f = np.empty((9, self.nr, self.nx))
        g = np.empty((4, self.nr, self.nx))
        self._L.orc_get_streamed(self._h, _p(f), _p(g))
        return f, g
