"""Thin ctypes binding of liblbm (include/lbm.h).

Argument marshalling only: every step of the method runs in the CUDA
kernels of the library.  PyTorch supplies the device memory (a caching
allocator block handed to ``lbm_create``) and the CUDA stream.  There is no
CPU fallback: if the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

from . import build as _build
from .inputs import LatticeConfig, Workload

LBM_OK = 0
ERRORS = {-1: "LBM_ERR_INVALID_ARG", -2: "LBM_ERR_OOM", -3: "LBM_ERR_CUDA", -4: "LBM_ERR_DIVERGED"}
STORAGE = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3, "f16s": 4, "bf16s": 5}
# moment-split storage: FP32 moments beside 2-byte deviations from the linear equilibrium
SPLIT = ("f16s", "bf16s")
_BC_IN = {"inlet": 0, "periodic": 1}
_BC_OUT = {"outflow": 0, "wall": 1, "periodic": 2}
_BC_TOP = {"wall": 0, "open": 1}
_BC_BOTTOM = {"axis": 0, "wall": 1}
PATTERN = {"ab": 0, "aa": 1}

HEADER = os.path.join(_build.ROOT, "include", "lbm.h")


class LbmError(RuntimeError):
    def __init__(self, code: int, what: str, msg: str):
        super().__init__(f"{what} failed with {ERRORS.get(code, code)}: {msg}")
        self.code = code


class Desc(C.Structure):
    """Mirror of ``lbm_desc``."""

    _fields_ = [
        ("nx", C.c_int32), ("nr", C.c_int32), ("storage", C.c_int32),
        ("bc_in", C.c_int32), ("bc_out", C.c_int32), ("bc_top", C.c_int32), ("bc_bottom", C.c_int32),
        ("axisym", C.c_int32),
        ("r0", C.c_double), ("rho0", C.c_double), ("T0", C.c_double), ("Cs", C.c_double),
        ("Pr_t", C.c_double), ("T_top", C.c_double), ("T_bottom", C.c_double), ("T_out", C.c_double),
        ("noise_amp", C.c_double), ("seed", C.c_uint64), ("pattern", C.c_int32),
    ]


class Diag(C.Structure):
    """Mirror of ``lbm_diag``."""

    _fields_ = [("mass", C.c_double), ("mass_axi", C.c_double), ("heat", C.c_double), ("heat_axi", C.c_double),
                ("max_speed", C.c_double), ("residual_max", C.c_double), ("residual_l2", C.c_double),
                ("nonfinite", C.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def make_desc(cfg: LatticeConfig, storage: str, pattern: str = "ab") -> Desc:
    return Desc(pattern=PATTERN[pattern], nx=cfg.nx, nr=cfg.nr, storage=STORAGE[storage], bc_in=_BC_IN[cfg.bc_in],
                bc_out=_BC_OUT[cfg.bc_out], bc_top=_BC_TOP[cfg.bc_top],
                bc_bottom=_BC_BOTTOM[cfg.bc_bottom], axisym=int(cfg.axisym), r0=cfg.r0,
                rho0=cfg.rho0, T0=cfg.T0, Cs=cfg.Cs, Pr_t=cfg.Pr_t, T_top=cfg.T_top,
                T_bottom=cfg.T_bottom, T_out=cfg.T_out, noise_amp=cfg.noise_amp,
                seed=cfg.seed & 0xFFFFFFFFFFFFFFFF)


_lib = None
_lock = threading.Lock()


def declared_symbols():
    """Names of the functions include/lbm.h declares."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"LBM_API\s+[\w\s\*]*?\b(lbm_\w+)\s*\(", text)))


def lib(build: bool = True):
    """Load liblbm (building it first if it is stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"liblbm is not built ({path}); the CUDA path has no fallback")
            L = C.CDLL(path)
            vp, dp, i32, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_int64
            L.lbm_last_error.restype = C.c_char_p
            L.lbm_last_error.argtypes = []
            L.lbm_required_bytes.argtypes = [C.POINTER(Desc), C.POINTER(C.c_size_t)]
            L.lbm_create.argtypes = [C.POINTER(Desc), vp, C.c_size_t, C.POINTER(vp)]
            L.lbm_destroy.restype = None
            L.lbm_destroy.argtypes = [vp]
            L.lbm_set_inlet.argtypes = [vp, dp, dp, i32, vp]
            L.lbm_set_properties.argtypes = [vp, dp, dp, i32, C.c_double, C.c_double, vp]
            L.lbm_step.argtypes = [vp, i32, vp]
            L.lbm_get_step.restype = i64
            L.lbm_get_step.argtypes = [vp]
            L.lbm_get_fields.argtypes = [vp, vp, i32, vp]
            L.lbm_get_state.argtypes = [vp, vp, vp, vp]
            L.lbm_set_state.argtypes = [vp, vp, vp, i64, vp]
            L.lbm_checkpoint_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
            L.lbm_save.argtypes = [vp, vp, vp]
            L.lbm_restore.argtypes = [vp, vp, i64, vp]
            L.lbm_set_launch.argtypes = [vp, i32, i32]
            L.lbm_get_launch.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
            L.lbm_set_item_group.argtypes = [vp, i32]
            L.lbm_selftest_wait_timeout.argtypes = [vp, C.POINTER(i32)]
            L.lbm_get_item_group.restype = i32
            L.lbm_get_item_group.argtypes = [vp]
            L.lbm_check.argtypes = [vp, C.POINTER(i32)]
            L.lbm_diagnostics.argtypes = [vp, C.POINTER(Diag), vp]
            L.lbm_diagnostics_noalloc.argtypes = [vp, C.POINTER(Diag), vp]
            L.lbm_batch_create.argtypes = [i32, C.POINTER(vp)]
            L.lbm_batch_destroy.restype = None
            L.lbm_batch_destroy.argtypes = [vp]
            L.lbm_batch_add.argtypes = [vp, vp]
            L.lbm_batch_remove.argtypes = [vp, vp]
            L.lbm_batch_size.restype = i32
            L.lbm_batch_size.argtypes = [vp]
            L.lbm_batch_step.argtypes = [vp, i32, i32, vp]
            L.lbm_batch_set_launch.argtypes = [vp, i32, i32]
            L.lbm_batch_get_launch.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
            L.lbm_set_strip_width.argtypes = [vp, i32]
            L.lbm_get_strip_width.restype = i32
            L.lbm_get_strip_width.argtypes = [vp]
            L.lbm_batch_set_strip_width.argtypes = [vp, i32]
            L.lbm_batch_get_strip_width.restype = i32
            L.lbm_batch_get_strip_width.argtypes = [vp]
            for name in ("lbm_required_bytes", "lbm_create", "lbm_set_inlet", "lbm_set_properties",
                         "lbm_step", "lbm_get_fields", "lbm_get_state", "lbm_set_state",
                         "lbm_set_launch", "lbm_get_launch", "lbm_check", "lbm_batch_create",
                         "lbm_batch_add", "lbm_batch_remove", "lbm_batch_step", "lbm_batch_set_launch",
                         "lbm_batch_get_launch", "lbm_diagnostics", "lbm_diagnostics_noalloc",
                         "lbm_set_strip_width", "lbm_batch_set_strip_width"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != LBM_OK:
        raise LbmError(rc, what, lib().lbm_last_error().decode())


def required_bytes(cfg: LatticeConfig, storage: str = "f32", pattern: str = "ab") -> int:
    d = make_desc(cfg, storage, pattern)
    n = C.c_size_t(0)
    _check(lib().lbm_required_bytes(C.byref(d), C.byref(n)), "lbm_required_bytes")
    return int(n.value)


def _stream_ptr(stream, *users) -> C.c_void_p:
    """The stream's handle; the lattices in `users` note the stream for their ``close``."""
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    for u in users:
        u._used_on(s)
    return C.c_void_p(int(s.cuda_stream))


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Lattice:
    """One lattice resident on the GPU, advanced by the fused CUDA step.

    ``pattern`` is the memory layout: "ab" (two population buffers) or "aa"
    (one buffer updated in place, plus the tiles' edge moments; same results,
    no steady residual).
    """

    def __init__(self, cfg: LatticeConfig, storage: str = "f32", device=None, pattern: str = "ab"):
        import torch

        cfg.validate()
        if storage not in STORAGE:
            raise ValueError(f"storage must be one of {sorted(STORAGE)}")
        if pattern not in PATTERN:
            raise ValueError(f"pattern must be one of {sorted(PATTERN)}")
        self.cfg = cfg
        self.storage = storage
        self.pattern = pattern
        self.nx, self.nr = cfg.nx, cfg.nr
        self.device = torch.device(device if device is not None else "cuda")
        self._L = lib()
        self._desc = make_desc(cfg, storage, pattern)
        self.nbytes = required_bytes(cfg, storage, pattern)
        self._streams = {}
        with torch.cuda.device(self.device):
            # the caching allocator hands out 512-byte aligned blocks, in the order of the
            # current stream; the library's set-up runs on the default stream, so that
            # stream first waits for the work the block's previous owner queued
            self._mem = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
            self._alloc_stream = torch.cuda.current_stream(self.device)
            if self._alloc_stream != torch.cuda.default_stream(self.device):
                torch.cuda.default_stream(self.device).wait_stream(self._alloc_stream)
            h = C.c_void_p()
            _check(self._L.lbm_create(C.byref(self._desc), C.c_void_p(self._mem.data_ptr()),
                                      self.nbytes, C.byref(h)), "lbm_create")
        self._h = h

    @classmethod
    def from_workload(cls, w: Workload, storage: str = "f32", device=None, pattern: str = "ab") -> "Lattice":
        lat = cls(w.cfg, storage, device, pattern)
        lat.set_inlet(w.u_in, w.T_in)
        lat.set_properties(w.nu_tab, w.alpha_tab, w.T_lo, w.T_hi)
        return lat

    def close(self):
        if getattr(self, "_h", None):
            self._L.lbm_destroy(self._h)
            self._h = None
            # work queued on other streams may still use the block: the caching allocator
            # hands it out again only after that work
            for s in self._streams.values():
                self._mem.record_stream(s)
            self._streams = {}
            self._mem = None

    def _used_on(self, s):
        if s != self._alloc_stream:
            self._streams.setdefault(s.cuda_stream, s)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> C.c_void_p:
        return self._h

    def set_inlet(self, u_in, T_in, stream=None):
        u = np.ascontiguousarray(u_in, dtype=np.float64)
        T = np.ascontiguousarray(T_in, dtype=np.float64)
        _check(self._L.lbm_set_inlet(self._h, _dptr(u), _dptr(T), len(u), _stream_ptr(stream, self)),
               "lbm_set_inlet")

    def set_properties(self, nu, alpha, T_lo, T_hi, stream=None):
        a = np.ascontiguousarray(nu, dtype=np.float64)
        b = np.ascontiguousarray(alpha, dtype=np.float64)
        _check(self._L.lbm_set_properties(self._h, _dptr(a), _dptr(b), len(a), float(T_lo),
                                          float(T_hi), _stream_ptr(stream, self)), "lbm_set_properties")

    def set_launch(self, band_rows: int = 0, warps_per_cta: int = 0):
        """band_rows 0 = automatic (a few rounds of resident warps between dependent tiles); warps 0 = unchanged."""
        _check(self._L.lbm_set_launch(self._h, band_rows, warps_per_cta), "lbm_set_launch")

    def set_strip_width(self, columns: int = 0):
        """Tile width of the step kernel in lattice columns: 32 or 64 (0 = the default)."""
        _check(self._L.lbm_set_strip_width(self._h, int(columns)), "lbm_set_strip_width")

    @property
    def strip_width(self) -> int:
        return int(self._L.lbm_get_strip_width(self._h))

    def selftest_wait_timeout(self) -> int:
        """Run a launch whose waits can never be met; returns the device status it raised."""
        v = C.c_int32()
        _check(self._L.lbm_selftest_wait_timeout(self._h, C.byref(v)), "lbm_selftest_wait_timeout")
        return v.value

    def set_item_group(self, group: int = 0):
        """Warp tiles per work item of the persistent step launch (0 = automatic)."""
        _check(self._L.lbm_set_item_group(self._h, int(group)), "lbm_set_item_group")

    @property
    def item_group(self) -> int:
        return int(self._L.lbm_get_item_group(self._h))

    def launch(self):
        """(band rows, warps per CTA, CTAs) used by lbm_step."""
        b, w, c = C.c_int32(), C.c_int32(), C.c_int32()
        _check(self._L.lbm_get_launch(self._h, C.byref(b), C.byref(w), C.byref(c)), "lbm_get_launch")
        return b.value, w.value, c.value

    def step(self, n: int = 1, stream=None):
        _check(self._L.lbm_step(self._h, int(n), _stream_ptr(stream, self)), "lbm_step")

    def diagnostics(self, stream=None) -> dict:
        """FP64 mass, heat, max speed, steady residual and non-finite count (synchronises).

        ``diverged`` is True when some node has a non-finite or non-positive
        density or a non-finite velocity or temperature.
        """
        d = Diag()
        rc = self._L.lbm_diagnostics(self._h, C.byref(d), _stream_ptr(stream, self))
        if rc not in (LBM_OK, -4):
            _check(rc, "lbm_diagnostics")
        out = d.as_dict()
        out["diverged"] = rc == -4
        return out

    def check(self) -> int:
        """Device error flags since the last check (0 = none); synchronises."""
        v = C.c_int32()
        _check(self._L.lbm_check(self._h, C.byref(v)), "lbm_check")
        return v.value

    @property
    def step_count(self) -> int:
        return int(self._L.lbm_get_step(self._h))

    def fields(self, dtype=None, stream=None, out=None):
        """(4, nr, nx) device tensor of rho, u_x, u_r, T at the current time."""
        import torch

        dtype = dtype or torch.float64
        if out is None:
            out = torch.empty((4, self.nr, self.nx), dtype=dtype, device=self.device)
        code = 0 if out.dtype == torch.float64 else 1
        if out.dtype not in (torch.float64, torch.float32) or not out.is_contiguous():
            raise ValueError("fields output must be a contiguous float64/float32 tensor")
        _check(self._L.lbm_get_fields(self._h, C.c_void_p(out.data_ptr()), code, _stream_ptr(stream, self)),
               "lbm_get_fields")
        return out

    def get_state(self, stream=None):
        """Post-collision populations as device FP64 tensors f (9, nr, nx), g (4, nr, nx)."""
        import torch

        f = torch.empty((9, self.nr, self.nx), dtype=torch.float64, device=self.device)
        g = torch.empty((4, self.nr, self.nx), dtype=torch.float64, device=self.device)
        _check(self._L.lbm_get_state(self._h, C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()),
                                     _stream_ptr(stream, self)), "lbm_get_state")
        return f, g

    def set_state(self, f, g, step: int = 0, stream=None):
        import torch

        f = torch.as_tensor(f, dtype=torch.float64, device=self.device).contiguous()
        g = torch.as_tensor(g, dtype=torch.float64, device=self.device).contiguous()
        if tuple(f.shape) != (9, self.nr, self.nx) or tuple(g.shape) != (4, self.nr, self.nx):
            raise ValueError("state shapes must be (9, nr, nx) and (4, nr, nx)")
        _check(self._L.lbm_set_state(self._h, C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()),
                                     int(step), _stream_ptr(stream, self)), "lbm_set_state")
        # keep the inputs alive until the conversion kernel has run
        torch.cuda.current_stream(self.device).synchronize() if stream is None else stream.synchronize()

    def _checkpoint_shape(self):
        import torch

        if self.storage in SPLIT:  # 13 planes of 2-byte deviations, then 3 FP32 moment planes, as bytes
            return (13 * 2 + 3 * 4) * self.nr * self.nx, torch.uint8
        dt = {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[self.storage]
        return (13, self.nr, self.nx), dt

    def save(self, stream=None):
        """Checkpoint: (stored state in the storage type, step count); exact.  The state is the
        deviations (13, nr, nx); for moment-split storage the raw bytes of lbm_save's layout."""
        import torch

        n = C.c_size_t()
        _check(self._L.lbm_checkpoint_bytes(self._h, C.byref(n)), "lbm_checkpoint_bytes")
        shape, dt = self._checkpoint_shape()
        out = torch.empty(shape, dtype=dt, device=self.device)
        assert out.numel() * out.element_size() == n.value
        _check(self._L.lbm_save(self._h, C.c_void_p(out.data_ptr()), _stream_ptr(stream, self)), "lbm_save")
        return out, self.step_count

    def restore(self, planes, step: int, stream=None):
        """Resume from a checkpoint taken by ``save`` on a lattice of the same size and storage."""
        import torch

        n = C.c_size_t()
        _check(self._L.lbm_checkpoint_bytes(self._h, C.byref(n)), "lbm_checkpoint_bytes")
        shape, _ = self._checkpoint_shape()
        if tuple(planes.shape) != tuple(shape if isinstance(shape, tuple) else (shape,)) or \
                planes.numel() * planes.element_size() != n.value:
            raise ValueError("checkpoint does not match this lattice")
        planes = planes.to(self.device).contiguous()
        _check(self._L.lbm_restore(self._h, C.c_void_p(planes.data_ptr()), int(step), _stream_ptr(stream, self)),
               "lbm_restore")
        # keep the input alive until the copies have run
        torch.cuda.current_stream(self.device).synchronize() if stream is None else stream.synchronize()

    def restore_async(self, planes, step: int, stream=None):
        """``restore`` from a device tensor without synchronising: the caller keeps ``planes``
        alive until the stream has run the copies."""
        n = C.c_size_t()
        _check(self._L.lbm_checkpoint_bytes(self._h, C.byref(n)), "lbm_checkpoint_bytes")
        if (planes.numel() * planes.element_size() != n.value
                or planes.device != self.device or not planes.is_contiguous()):
            raise ValueError("checkpoint does not match this lattice (a contiguous device tensor)")
        _check(self._L.lbm_restore(self._h, C.c_void_p(planes.data_ptr()), int(step), _stream_ptr(stream, self)),
               "lbm_restore")


class Batch:
    """Independent lattices of one storage type stepped together in persistent multi-step launches."""

    def __init__(self, storage: str = "f16"):
        if storage not in STORAGE:
            raise ValueError(f"storage must be one of {sorted(STORAGE)}")
        self.storage = storage
        self._L = lib()
        h = C.c_void_p()
        _check(self._L.lbm_batch_create(STORAGE[storage], C.byref(h)), "lbm_batch_create")
        self._h = h
        self.members = []

    def close(self):
        if getattr(self, "_h", None):
            self._L.lbm_batch_destroy(self._h)
            self._h = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return int(self._L.lbm_batch_size(self._h))

    def add(self, lat: "Lattice"):
        _check(self._L.lbm_batch_add(self._h, lat.handle), "lbm_batch_add")
        self.members.append(lat)

    def remove(self, lat: "Lattice"):
        _check(self._L.lbm_batch_remove(self._h, lat.handle), "lbm_batch_remove")
        self.members = [m for m in self.members if m is not lat]

    def step(self, n: int = 1, graph: bool = True, stream=None):
        _check(self._L.lbm_batch_step(self._h, int(n), int(bool(graph)), _stream_ptr(stream, *self.members)),
               "lbm_batch_step")

    def set_launch(self, band_rows: int = 0, warps_per_cta: int = 0):
        _check(self._L.lbm_batch_set_launch(self._h, band_rows, warps_per_cta), "lbm_batch_set_launch")

    def set_strip_width(self, columns: int = 0):
        _check(self._L.lbm_batch_set_strip_width(self._h, int(columns)), "lbm_batch_set_strip_width")

    @property
    def strip_width(self) -> int:
        return int(self._L.lbm_batch_get_strip_width(self._h))

    def launch(self):
        """(band rows, warps per CTA, warp tiles per step) of the last rebuilt tables."""
        b, w, t = C.c_int32(), C.c_int32(), C.c_int32()
        _check(self._L.lbm_batch_get_launch(self._h, C.byref(b), C.byref(w), C.byref(t)), "lbm_batch_get_launch")
        return b.value, w.value, t.value
