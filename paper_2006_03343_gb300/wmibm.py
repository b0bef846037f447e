"""ctypes binding of libwmibm.so (C ABI in include/wmibm.h).

Argument marshalling only: every step of the stress stage runs in the CUDA
library.  torch supplies device memory and the current stream; fields are
passed as raw device pointers.  If the library has not been built, loading it
raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

F32, F64, BF16 = 0, 1, 2
OK, EINVAL, ENOMEM, ECUDA, ESTATE, ETIMEOUT = 0, 1, 2, 3, 4, 5
LIST_BAND_W, LIST_BAND_UV, LIST_SOLID_W, LIST_SOLID_UV, LIST_BODY_W, LIST_BODY_UV = range(6)
LIST_NAMES = ("band_w", "band_uv", "solid_w", "solid_uv", "body_w", "body_uv")
TAU_ORDER = ("txx", "txy", "tyy", "tzz", "txz", "tyz")
DTYPE_CODES = {"f32": F32, "f64": F64, "bf16": BF16}

# symbols the header declares (checked by the CPU test suite)
EXPORTED = ("wmibm_init", "wmibm_wall_stress", "wmibm_force", "wmibm_mask", "wmibm_step", "wmibm_list_size",
            "wmibm_export_list", "wmibm_traffic_bytes", "wmibm_destroy", "wmibm_status_string",
            "wmibm_last_error", "wmibm_wall_stress_force", "wmibm_set_tuning", "wmibm_get_tuning",
            "wmibm_device_status", "wmibm_force_mask", "wmibm_wall_stress_noalloc", "wmibm_batch_create",
            "wmibm_batch_set_fields", "wmibm_batch_set_tuning", "wmibm_batch_step", "wmibm_batch_traffic_bytes",
            "wmibm_batch_points", "wmibm_batch_last_error", "wmibm_batch_destroy", "wmibm_set_log_z0",
            "wmibm_backward", "wmibm_batch_wall_stress_force", "wmibm_force_spectral", "wmibm_spectral_shape", "wmibm_sgs_wall_terms", "wmibm_sgs_stress", "wmibm_sgs_force",
            "wmibm_heightfield_sdf", "wmibm_batch_device_status")


class WmibmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"wmibm status {status}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("phi_b", ctypes.c_double), ("kappa", ctypes.c_double),
                ("dtype", ctypes.c_int32), ("vel_dtype", ctypes.c_int32), ("zclamp", ctypes.c_int32),
                ("own_x0", ctypes.c_int32), ("own_x1", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("force_path", ctypes.c_int32), ("rows", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("consumer_warps", ctypes.c_int32), ("wall_warps", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("direct_bx", ctypes.c_int32), ("direct_by", ctypes.c_int32),
                ("direct_kc", ctypes.c_int32), ("wall_chunk", ctypes.c_int32), ("dyn_chunk", ctypes.c_int32),
                ("wall_grid", ctypes.c_int32)]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class MemberFields(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("tau", ctypes.c_void_p * 6), ("f", ctypes.c_void_p * 3)]


STATS_DTYPE = np.dtype([("count", "<i8"), ("sum_tw", "<f8"), ("sum_tw2", "<f8"), ("min_tw", "<f8"),
                        ("max_ur", "<f8"), ("n_zclamped", "<i8")])
STATS_WORDS = STATS_DTYPE.itemsize // 8          # 8-byte words of one wmibm_band_stats
ZCLAMP_CLAMP, ZCLAMP_REJECT = 0, 1

_lib = None
_VP = ctypes.c_void_p
_PVP = ctypes.POINTER(ctypes.c_void_p)


def lib_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load libwmibm.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: the CUDA library must be built "
                           "(paper_2006_03343_gb300.build.build()); there is no CPU fallback")
    L = ctypes.CDLL(path)
    L.wmibm_init.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(Grid), _VP, _VP, _VP, ctypes.c_int32,
                             ctypes.c_double, ctypes.POINTER(Opts), _VP]
    L.wmibm_init.restype = ctypes.c_int
    L.wmibm_wall_stress.argtypes = [_VP, _VP, _VP, _VP, _PVP, _VP, _VP]
    L.wmibm_wall_stress.restype = ctypes.c_int
    L.wmibm_force.argtypes = [_VP, _PVP, _VP, _VP, _VP, _VP]
    L.wmibm_force.restype = ctypes.c_int
    L.wmibm_force_spectral.argtypes = [_VP, _PVP, _VP, _VP, _VP, _VP]
    L.wmibm_force_spectral.restype = ctypes.c_int
    L.wmibm_spectral_shape.argtypes = [_VP, ctypes.POINTER(ctypes.c_int64)]
    L.wmibm_spectral_shape.restype = ctypes.c_int
    L.wmibm_sgs_wall_terms.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_int32, _VP, _VP, _VP]
    L.wmibm_sgs_wall_terms.restype = ctypes.c_int
    L.wmibm_sgs_stress.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _PVP, ctypes.c_double, _VP]
    L.wmibm_sgs_stress.restype = ctypes.c_int
    L.wmibm_sgs_force.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _PVP, _VP, _VP, _VP, ctypes.c_double, _VP]
    L.wmibm_sgs_force.restype = ctypes.c_int
    L.wmibm_heightfield_sdf.argtypes = [ctypes.POINTER(Grid), _VP, ctypes.c_double, _VP, _VP, _VP]
    L.wmibm_heightfield_sdf.restype = ctypes.c_int
    L.wmibm_mask.argtypes = [_VP, _VP, _VP, _VP, _PVP, ctypes.c_double, _VP]
    L.wmibm_mask.restype = ctypes.c_int
    L.wmibm_step.argtypes = [_VP, _VP, _VP, _VP, _PVP, _VP, _VP, _VP, _PVP, ctypes.c_double, _VP, _VP]
    L.wmibm_step.restype = ctypes.c_int
    L.wmibm_wall_stress_force.argtypes = [_VP, _VP, _VP, _VP, _PVP, _VP, _VP, _VP, _VP, _VP]
    L.wmibm_wall_stress_force.restype = ctypes.c_int
    L.wmibm_wall_stress_noalloc.argtypes = [_VP, _VP, _VP, _VP, _PVP, _VP, _VP]
    L.wmibm_wall_stress_noalloc.restype = ctypes.c_int
    L.wmibm_force_mask.argtypes = [_VP, _PVP, _VP, _VP, _VP, _VP, _VP, _VP, _PVP, ctypes.c_double, _VP]
    L.wmibm_force_mask.restype = ctypes.c_int
    L.wmibm_set_tuning.argtypes = [_VP, ctypes.POINTER(Tuning)]
    L.wmibm_set_tuning.restype = ctypes.c_int
    L.wmibm_get_tuning.argtypes = [_VP, ctypes.POINTER(Tuning)]
    L.wmibm_get_tuning.restype = ctypes.c_int
    L.wmibm_device_status.argtypes = [_VP, ctypes.POINTER(ctypes.c_int32), _VP]
    L.wmibm_device_status.restype = ctypes.c_int
    L.wmibm_batch_create.argtypes = [ctypes.POINTER(_VP), _PVP, ctypes.c_int32, _VP]
    L.wmibm_batch_create.restype = ctypes.c_int
    L.wmibm_batch_set_fields.argtypes = [_VP, ctypes.POINTER(MemberFields), _VP]
    L.wmibm_batch_set_fields.restype = ctypes.c_int
    L.wmibm_batch_set_tuning.argtypes = [_VP, ctypes.POINTER(Tuning)]
    L.wmibm_batch_set_tuning.restype = ctypes.c_int
    L.wmibm_batch_step.argtypes = [_VP, _VP, _VP]
    L.wmibm_batch_step.restype = ctypes.c_int
    L.wmibm_batch_wall_stress_force.argtypes = [_VP, _VP, _VP]
    L.wmibm_batch_wall_stress_force.restype = ctypes.c_int
    L.wmibm_batch_device_status.argtypes = [_VP, ctypes.POINTER(ctypes.c_int32), _VP]
    L.wmibm_batch_device_status.restype = ctypes.c_int
    L.wmibm_batch_traffic_bytes.argtypes = [_VP, ctypes.c_int32]
    L.wmibm_batch_traffic_bytes.restype = ctypes.c_int64
    L.wmibm_batch_points.argtypes = [_VP]
    L.wmibm_batch_points.restype = ctypes.c_int64
    L.wmibm_batch_last_error.argtypes = [_VP]
    L.wmibm_batch_last_error.restype = ctypes.c_char_p
    L.wmibm_batch_destroy.argtypes = [_VP]
    L.wmibm_batch_destroy.restype = None
    L.wmibm_set_log_z0.argtypes = [_VP, _VP, _VP]
    L.wmibm_set_log_z0.restype = ctypes.c_int
    L.wmibm_backward.argtypes = [_VP, _PVP, _PVP, _VP, _VP, _VP, _VP, _VP]
    L.wmibm_backward.restype = ctypes.c_int
    L.wmibm_list_size.argtypes = [_VP, ctypes.c_int32]
    L.wmibm_list_size.restype = ctypes.c_int64
    L.wmibm_export_list.argtypes = [_VP, ctypes.c_int32, _VP, ctypes.c_int64, _VP]
    L.wmibm_export_list.restype = ctypes.c_int
    L.wmibm_traffic_bytes.argtypes = [_VP, ctypes.c_int32]
    L.wmibm_traffic_bytes.restype = ctypes.c_int64
    L.wmibm_destroy.argtypes = [_VP]
    L.wmibm_destroy.restype = None
    L.wmibm_status_string.argtypes = [ctypes.c_int]
    L.wmibm_status_string.restype = ctypes.c_char_p
    L.wmibm_last_error.argtypes = [_VP]
    L.wmibm_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _ptrs(seq) -> ctypes.Array:
    arr = (ctypes.c_void_p * len(seq))()
    for i, t in enumerate(seq):
        arr[i] = None if t is None else ctypes.c_void_p(_dptr(t))
    return arr


def _dptr(t) -> int:
    if isinstance(t, int):
        return t
    return int(t.data_ptr())


def _stream_ptr(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) or None


def heightfield_sdf(grid, height, reach, phi_uv=None, phi_w=None, stream=None):
    """wmibm_heightfield_sdf: the exact signed distance (Sec. 3.1) to the piecewise-
    linear surface through the heights `height` (a CUDA float64 tensor [ny, nx]),
    within `reach`; z - h beyond it.  Returns (phi_uv, phi_w), CUDA float64
    tensors [nz, ny, nx] (allocated unless given)."""
    import torch
    L = load()
    nx, ny, nz, lx, ly, lz = grid
    if not (isinstance(height, torch.Tensor) and height.is_cuda and height.dtype == torch.float64
            and height.is_contiguous() and tuple(height.shape) == (ny, nx)):
        raise ValueError("height must be a contiguous CUDA float64 tensor of shape (ny, nx)")
    out = []
    for t in (phi_uv, phi_w):
        if t is None:
            t = torch.empty((nz, ny, nx), dtype=torch.float64, device=height.device)
        elif not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == nx * ny * nz):
            raise ValueError("phi_uv, phi_w must be contiguous CUDA float64 tensors of nx*ny*nz elements")
        out.append(t)
    g = Grid(int(nx), int(ny), int(nz), float(lx), float(ly), float(lz))
    st = L.wmibm_heightfield_sdf(ctypes.byref(g), _dptr(height), float(reach), _dptr(out[0]), _dptr(out[1]),
                                 _stream_ptr(stream))
    if st != OK:
        raise WmibmError(st, L.wmibm_last_error(None).decode())
    return out[0], out[1]


class Handle:
    """One terrain on one GPU: wraps wmibm_init / wmibm_destroy and the per-step calls.

    dtype: "f32" or "f64" (stress, force and arithmetic); vel_dtype: None (same as
    dtype) or "bf16" (with f32); zclamp: ZCLAMP_CLAMP (clamp the level of sample
    points outside the grid and count them) or ZCLAMP_REJECT (fail instead);
    own_x: None, or (x0, x1): the handle owns the nodes with x0 <= i < x1 of a slab
    whose other x-planes are halo (see slab.py)."""

    def __init__(self, grid, phi_uv, phi_w, z0, phi_c, phi_b=0.0, dtype="f32", vel_dtype=None, kappa=0.4,
                 stream=None, zclamp=0, own_x=None):
        import torch
        L = load()
        nx, ny, nz, lx, ly, lz = grid
        self.grid = tuple(grid)
        self.shape = (int(nz), int(ny), int(nx))
        self.dtype = dtype
        self.vel_dtype = vel_dtype or dtype
        self.torch_dtype = torch.float64 if dtype == "f64" else torch.float32
        self.torch_vel_dtype = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}[self.vel_dtype]
        self.device = torch.device("cuda", torch.cuda.current_device())
        phi_uv = np.ascontiguousarray(phi_uv, np.float64)
        phi_w = np.ascontiguousarray(phi_w, np.float64)
        if np.isscalar(z0):
            z0a = np.array([float(z0)], np.float64)
            is_field = 0
        else:
            z0a = np.ascontiguousarray(z0, np.float64)
            is_field = 1
        g = Grid(int(nx), int(ny), int(nz), float(lx), float(ly), float(lz))
        x0, x1 = own_x if own_x is not None else (0, 0)
        o = Opts(float(phi_b), float(kappa), DTYPE_CODES[dtype], DTYPE_CODES[self.vel_dtype], int(zclamp), int(x0),
                 int(x1))
        h = ctypes.c_void_p()
        st = L.wmibm_init(ctypes.byref(h), ctypes.byref(g), phi_uv.ctypes.data, phi_w.ctypes.data,
                          z0a.ctypes.data, is_field, float(phi_c), ctypes.byref(o), _stream_ptr(stream))
        if st != OK:
            raise WmibmError(st, L.wmibm_last_error(None).decode())
        self._h = h
        self._L = L

    @classmethod
    def from_case(cls, case, dtype=None, vel_dtype=None, stream=None, zclamp=0):
        return cls(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_c, case.phi_b,
                   dtype=dtype or case.dtype, vel_dtype=vel_dtype, stream=stream, zclamp=zclamp)

    # ------------------------------------------------------------------ #
    def _check(self, st):
        if st != OK:
            raise WmibmError(st, self._L.wmibm_last_error(self._h).decode())

    def _field(self, t, vel=False):
        want = self.torch_vel_dtype if vel else self.torch_dtype
        if t.dtype != want or not t.is_contiguous() or tuple(t.shape) != self.shape or t.device != self.device:
            raise ValueError(f"field must be a contiguous {want} tensor of shape {self.shape} on {self.device}, "
                             f"got {t.dtype} {tuple(t.shape)} on {t.device}")
        return t

    def new_stats(self):
        import torch
        return torch.zeros(2 * STATS_WORDS, dtype=torch.float64, device=self.device)

    @staticmethod
    def parse_stats(stats_tensor):
        raw = stats_tensor.detach().cpu().numpy().tobytes()
        return np.frombuffer(raw, dtype=STATS_DTYPE)

    def wall_stress(self, u, v, w, tau: Sequence, stats=None, stream=None):
        for t in (u, v, w):
            self._field(t, vel=True)
        for t in tau:
            self._field(t)
        self._check(self._L.wmibm_wall_stress(self._h, _dptr(u), _dptr(v), _dptr(w), _ptrs(tau),
                                              None if stats is None else _dptr(stats), _stream_ptr(stream)))

    def set_log_z0(self, logz0=None, stream=None):
        """Use a per-cell ln z0 field (device tensor of the handle's dtype, kept alive by
        the caller) in every later forward call; None returns to the init z0.  The
        first call builds the adjoint's transpose map (synchronizing)."""
        if logz0 is not None:
            self._field(logz0)
        self._logz0 = logz0
        self._check(self._L.wmibm_set_log_z0(self._h, None if logz0 is None else _dptr(logz0),
                                             _stream_ptr(stream)))

    def backward(self, g: Sequence, uvw: Sequence, du, dv, dw, dlogz0=None, stream=None):
        """dL/du, dL/dv, dL/dw (and dL/d ln z0) of one stage for L = sum(g . f)."""
        for t in list(g) + [du, dv, dw] + ([dlogz0] if dlogz0 is not None else []):
            self._field(t)
        for t in uvw:
            self._field(t, vel=True)
        self._check(self._L.wmibm_backward(self._h, _ptrs(g), _ptrs(uvw), _dptr(du), _dptr(dv), _dptr(dw),
                                           None if dlogz0 is None else _dptr(dlogz0), _stream_ptr(stream)))

    def wall_stress_noalloc(self, u, v, w, tau: Sequence, stats=None, stream=None):
        """wall_stress with the kernel's reduction scratch in a static device array
        (no device allocation; for callers that cannot allocate at call time)."""
        for t in (u, v, w):
            self._field(t, vel=True)
        for t in tau:
            self._field(t)
        self._check(self._L.wmibm_wall_stress_noalloc(self._h, _dptr(u), _dptr(v), _dptr(w), _ptrs(tau),
                                                      None if stats is None else _dptr(stats), _stream_ptr(stream)))

    def force(self, tau: Sequence, f: Sequence, stream=None):
        for t in list(tau) + list(f):
            self._field(t)
        self._check(self._L.wmibm_force(self._h, _ptrs(tau), _dptr(f[0]), _dptr(f[1]), _dptr(f[2]),
                                        _stream_ptr(stream)))

    def force_spectral(self, tau: Sequence, f: Sequence, stream=None):
        """f = -div(tau) with pseudo-spectral x and y derivatives (Eqs. 13-14)."""
        for t in list(tau) + list(f):
            self._field(t)
        self._check(self._L.wmibm_force_spectral(self._h, _ptrs(tau), _dptr(f[0]), _dptr(f[1]), _dptr(f[2]),
                                                 _stream_ptr(stream)))

    def sgs_wall_terms(self, phi_uv, phi_w, z0, stream=None):
        """The per-node wall terms of Mason's damping for sgs_stress -> (wt_uv, wt_w) device tensors
        (phi_uv, phi_w: the host FP64 fields given at init; z0 scalar or per-cell)."""
        import torch
        phi_uv = np.ascontiguousarray(phi_uv, np.float64)
        phi_w = np.ascontiguousarray(phi_w, np.float64)
        if np.isscalar(z0):
            z0a, is_field = np.array([float(z0)], np.float64), 0
        else:
            z0a, is_field = np.ascontiguousarray(z0, np.float64), 1
        wt = [torch.empty(self.shape, dtype=self.torch_dtype, device=self.device) for _ in range(2)]
        self._check(self._L.wmibm_sgs_wall_terms(self._h, phi_uv.ctypes.data, phi_w.ctypes.data, z0a.ctypes.data,
                                                 is_field, _dptr(wt[0]), _dptr(wt[1]), _stream_ptr(stream)))
        return wt[0], wt[1]

    def sgs_stress(self, u, v, w, wall_terms, tau: Sequence, cs=0.16, stream=None):
        """Smagorinsky stress with Mason's damping (Eqs. 4-7) into tau at fluid nodes."""
        for t in (u, v, w):
            self._field(t, vel=True)
        for t in list(wall_terms) + list(tau):
            self._field(t)
        self._check(self._L.wmibm_sgs_stress(self._h, _dptr(u), _dptr(v), _dptr(w), _dptr(wall_terms[0]),
                                             _dptr(wall_terms[1]), _ptrs(tau), float(cs), _stream_ptr(stream)))

    def sgs_force(self, u, v, w, wall_terms, tau: Sequence, f: Sequence, cs=0.16, stream=None):
        """f = -div tau with the fluid stress formed from the velocity on the fly (Eqs. 4-7);
        tau is read at band nodes (run wall_stress first) and on the floor, never written."""
        for t in (u, v, w):
            self._field(t, vel=True)
        for t in list(wall_terms) + list(tau) + list(f):
            self._field(t)
        self._check(self._L.wmibm_sgs_force(self._h, _dptr(u), _dptr(v), _dptr(w), _dptr(wall_terms[0]),
                                            _dptr(wall_terms[1]), _ptrs(tau), _dptr(f[0]), _dptr(f[1]), _dptr(f[2]),
                                            float(cs), _stream_ptr(stream)))

    def spectral_shape(self):
        """(rows per row unit, columns per column unit, levels per chunk, shared bytes
        per block) of the spectral launch, or None without spectral support."""
        out = (ctypes.c_int64 * 4)()
        if self._L.wmibm_spectral_shape(self._h, out) != OK:
            return None
        return tuple(int(x) for x in out)

    def mask(self, u, v, w, gradp=None, dt=0.0, stream=None):
        for t in (u, v, w):
            self._field(t, vel=True)
        if gradp is not None:
            for t in gradp:
                self._field(t)
        self._check(self._L.wmibm_mask(self._h, _dptr(u), _dptr(v), _dptr(w),
                                       None if gradp is None else _ptrs(gradp), float(dt), _stream_ptr(stream)))

    def wall_stress_force(self, u, v, w, tau, f, stats=None, stream=None):
        for t in (u, v, w):
            self._field(t, vel=True)
        for t in list(tau) + list(f):
            self._field(t)
        self._check(self._L.wmibm_wall_stress_force(self._h, _dptr(u), _dptr(v), _dptr(w), _ptrs(tau),
                                                    _dptr(f[0]), _dptr(f[1]), _dptr(f[2]),
                                                    None if stats is None else _dptr(stats), _stream_ptr(stream)))

    def force_mask(self, tau, f, u, v, w, gradp=None, dt=0.0, stream=None):
        for t in list(tau) + list(f):
            self._field(t)
        for t in (u, v, w):
            self._field(t, vel=True)
        if gradp is not None:
            for t in gradp:
                self._field(t)
        self._check(self._L.wmibm_force_mask(self._h, _ptrs(tau), _dptr(f[0]), _dptr(f[1]), _dptr(f[2]), _dptr(u),
                                             _dptr(v), _dptr(w), None if gradp is None else _ptrs(gradp),
                                             float(dt), _stream_ptr(stream)))

    def prepare_step(self, u, v, w, tau, f, stats=None, gradp=None, dt=0.0):
        """Validates the fields once and returns a PreparedStep whose calls only
        launch (for loops and graph capture)."""
        for t in (u, v, w):
            self._field(t, vel=True)
        for t in list(tau) + list(f):
            self._field(t)
        if gradp is not None:
            for t in gradp:
                self._field(t)
        return PreparedStep(self, u, v, w, tau, f, stats, gradp, dt)

    def set_tuning(self, **fields):
        """Replaces the handle's tuning: the given fields, every other field 0 (automatic)."""
        t = Tuning()
        for k, v in fields.items():
            setattr(t, k, int(v))
        self._check(self._L.wmibm_set_tuning(self._h, ctypes.byref(t)))

    def get_tuning(self) -> Tuning:
        t = Tuning()
        self._check(self._L.wmibm_get_tuning(self._h, ctypes.byref(t)))
        return t

    def device_status(self, stream=None) -> int:
        out = ctypes.c_int32(-1)
        self._check(self._L.wmibm_device_status(self._h, ctypes.byref(out), _stream_ptr(stream)))
        return int(out.value)

    def step(self, u, v, w, tau, f, gradp=None, dt=0.0, stats=None, stream=None):
        for t in (u, v, w):
            self._field(t, vel=True)
        for t in list(tau) + list(f):
            self._field(t)
        self._check(self._L.wmibm_step(self._h, _dptr(u), _dptr(v), _dptr(w), _ptrs(tau), _dptr(f[0]),
                                       _dptr(f[1]), _dptr(f[2]), None if gradp is None else _ptrs(gradp),
                                       float(dt), None if stats is None else _dptr(stats), _stream_ptr(stream)))

    def list_size(self, which: int) -> int:
        return int(self._L.wmibm_list_size(self._h, int(which)))

    def export_list(self, which: int) -> np.ndarray:
        n = self.list_size(which)
        out = np.empty(max(n, 1), np.int32)
        self._check(self._L.wmibm_export_list(self._h, int(which), out.ctypes.data, out.size, _stream_ptr(None)))
        return out[:n]

    def traffic_bytes(self, which: int) -> int:
        return int(self._L.wmibm_traffic_bytes(self._h, int(which)))

    @property
    def raw(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._L.wmibm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PreparedStep:
    """Pre-marshalled arguments of the per-step calls of one handle and one set of
    fields (the tensors must stay alive and in place)."""

    def __init__(self, handle, u, v, w, tau, f, stats, gradp, dt):
        self._keep = (u, v, w, tuple(tau), tuple(f), stats, gradp)
        self.h = handle
        self._L = handle._L
        self._u, self._v, self._w = _dptr(u), _dptr(v), _dptr(w)
        self._tau = _ptrs(tau)
        self._f = (_dptr(f[0]), _dptr(f[1]), _dptr(f[2]))
        self._stats = None if stats is None else _dptr(stats)
        self._gradp = None if gradp is None else _ptrs(gradp)
        self._dt = float(dt)

    def wall_stress(self, stream=None):
        self.h._check(self._L.wmibm_wall_stress(self.h._h, self._u, self._v, self._w, self._tau, self._stats,
                                                _stream_ptr(stream)))

    def force_mask(self, stream=None):
        self.h._check(self._L.wmibm_force_mask(self.h._h, self._tau, *self._f, self._u, self._v, self._w,
                                               self._gradp, self._dt, _stream_ptr(stream)))

    def force(self, stream=None):
        self.h._check(self._L.wmibm_force(self.h._h, self._tau, *self._f, _stream_ptr(stream)))

    def force_spectral(self, stream=None):
        self.h._check(self._L.wmibm_force_spectral(self.h._h, self._tau, *self._f, _stream_ptr(stream)))

    def wall_stress_force(self, stream=None):
        self.h._check(self._L.wmibm_wall_stress_force(self.h._h, self._u, self._v, self._w, self._tau, *self._f,
                                                      self._stats, _stream_ptr(stream)))

    def step(self, stream=None):
        self.h._check(self._L.wmibm_step(self.h._h, self._u, self._v, self._w, self._tau, *self._f, self._gradp,
                                         self._dt, self._stats, _stream_ptr(stream)))


class Batch:
    """Batched ensemble of handles stepped by the same persistent launches."""

    def __init__(self, handles, stream=None):
        L = load()
        self._L = L
        self.handles = list(handles)
        arr = (ctypes.c_void_p * len(self.handles))(*[h.raw.value for h in self.handles])
        b = ctypes.c_void_p()
        st = L.wmibm_batch_create(ctypes.byref(b), arr, len(self.handles), _stream_ptr(stream))
        if st != OK:
            raise WmibmError(st, "wmibm_batch_create failed (mixed devices/dtypes, or a member the pipelined "
                                 "stencil cannot take)")
        self._b = b
        self._keep = None

    def _check(self, st):
        if st != OK:
            raise WmibmError(st, self._L.wmibm_batch_last_error(self._b).decode())

    def set_fields(self, fields, stream=None):
        """fields: per member (u, v, w, tau[6], f[3]) tensors on the handles' device."""
        arr = (MemberFields * len(self.handles))()
        for m, (h, (u, v, w, tau, f)) in enumerate(zip(self.handles, fields)):
            for t in (u, v, w):
                h._field(t, vel=True)
            for t in list(tau) + list(f):
                h._field(t)
            arr[m].u, arr[m].v, arr[m].w = _dptr(u), _dptr(v), _dptr(w)
            for a in range(6):
                arr[m].tau[a] = _dptr(tau[a])
            for a in range(3):
                arr[m].f[a] = _dptr(f[a])
        self._keep = fields
        self._check(self._L.wmibm_batch_set_fields(self._b, arr, _stream_ptr(stream)))

    def set_tuning(self, **fields):
        """Replaces the batch's tile shape and form (force_path 3: wall kernel then
        stencil; 0 or 5: one interleaved launch); the fields given before are set
        again, since the unit offsets depend on the rows per strip."""
        t = Tuning()
        for k, v in fields.items():
            setattr(t, k, int(v))
        self._check(self._L.wmibm_batch_set_tuning(self._b, ctypes.byref(t)))
        self._tuning = {k: int(v) for k, v in fields.items()}
        if self._keep is not None:
            self.set_fields(self._keep)

    def get_tuning(self) -> dict:
        return dict(getattr(self, "_tuning", {}))

    def new_stats(self):
        import torch
        return torch.zeros(2 * STATS_WORDS * len(self.handles), dtype=torch.float64, device=self.handles[0].device)

    def step(self, stats=None, stream=None):
        self._check(self._L.wmibm_batch_step(self._b, None if stats is None else _dptr(stats), _stream_ptr(stream)))

    def wall_stress_force(self, stats=None, stream=None):
        """Wall stress + force of every member (the step without the body mask)."""
        self._check(self._L.wmibm_batch_wall_stress_force(self._b, None if stats is None else _dptr(stats),
                                                          _stream_ptr(stream)))

    def points(self) -> int:
        return int(self._L.wmibm_batch_points(self._b))

    def device_status(self, stream=None) -> int:
        out = ctypes.c_int32(-1)
        self._check(self._L.wmibm_batch_device_status(self._b, ctypes.byref(out), _stream_ptr(stream)))
        return int(out.value)

    def traffic_bytes(self, which: int) -> int:
        return int(self._L.wmibm_batch_traffic_bytes(self._b, int(which)))

    def close(self):
        if getattr(self, "_b", None):
            self._L.wmibm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
