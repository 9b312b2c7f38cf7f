"""Thin Python binding of the C ABI in ``include/ftk.h`` (argument marshalling
only: every step of the tracking pipeline runs in the CUDA library).

Functions keep the C names.  Field arguments may be CUDA torch tensors,
CPU torch tensors or numpy arrays (float32, C-contiguous, (nt, ny, nx) or
(nt, nz, ny, nx)); results come back as numpy structured arrays with the
layout of ``ftk_cp``.  The library must have been built
(``paper_2011_08697_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CP_DTYPE = np.dtype([
    ("face_id", "<i8"), ("label", "<i8"), ("base", "<i4", (4,)), ("off", "<f4", (4,)),
    ("morse_index", "i1"), ("ordinal", "u1"), ("ndim", "u1"), ("reserved", "u1", (5,)),
])
assert CP_DTYPE.itemsize == 56

FTK_OK = 0
FTK_FLAG_STAGE_TIMES = 1
FTK_FLAG_AUTOTUNE = 2
STATUS_NAMES = {0: "FTK_OK", 1: "FTK_ERR_ARG", 2: "FTK_ERR_RANGE", 3: "FTK_ERR_NOMEM",
                4: "FTK_ERR_CUDA", 5: "FTK_ERR_TIMEOUT", 6: "FTK_ERR_BUSY",
                7: "FTK_ERR_INVARIANT", 8: "FTK_ERR_STATE"}


class FtkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ftk_params(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("spacing", ctypes.c_double * 3),
                ("t0", ctypes.c_double), ("dt", ctypes.c_double),
                ("quant_shift", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("max_punctures", ctypes.c_int64)]


class ftk_device_view(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("face_id", ctypes.c_void_p), ("label", ctypes.c_void_p),
                ("off", ctypes.c_void_p), ("morse", ctypes.c_void_p)]


class ftk_plan_desc(ctypes.Structure):
    _fields_ = [("detect_variant", ctypes.c_int32), ("kernels_per_execute", ctypes.c_int32),
                ("rows_per_unit", ctypes.c_int32), ("slices_per_unit", ctypes.c_int32),
                ("detect_units", ctypes.c_int64), ("capacity", ctypes.c_int64)]


_lib = None

# every symbol the header declares (checked by the CPU test-suite)
EXPORTS = [
    "ftk_params_default", "ftk_status_string", "ftk_last_error", "ftk_version",
    "ftk_track_cp2d", "ftk_track_cp3d", "ftk_result_count", "ftk_result_data",
    "ftk_result_free", "ftk_plan_create", "ftk_plan_execute", "ftk_plan_count",
    "ftk_plan_download", "ftk_plan_download_into", "ftk_plan_device_view", "ftk_plan_stage_times", "ftk_plan_destroy",
    "ftk_track_cp2d_noalloc",
    "ftk_batch_create", "ftk_batch_execute", "ftk_batch_counts", "ftk_batch_download",
    "ftk_batch_destroy", "ftk_track_cp2d_batch", "ftk_plan_describe", "ftk_batch_kernels",
    "ftk_stream_open", "ftk_stream_push", "ftk_stream_close", "ftk_server_create",
    "ftk_server_used", "ftk_server_destroy", "ftk_stream_open_in",
    "ftk_streams_push", "ftk_stream_open_wait", "ftk_stream_footprint",
    "ftk_plan_trajectories", "ftk_traj_count", "ftk_traj_offsets", "ftk_traj_points", "ftk_traj_closed",
    "ftk_traj_free", "ftk_plan_slice", "ftk_slice_count", "ftk_slice_data", "ftk_slice_free",
    "ftk_debug_set_wait_limits", "ftk_plan_trajectories_filtered",
    "ftk_track_vec2d", "ftk_plan_create_vec2d",
    "ftk_track_iso2d", "ftk_track_iso3d", "ftk_iso_result_count", "ftk_iso_result_data", "ftk_iso_result_free",
    "ftk_iso_plan_create", "ftk_iso_plan_execute", "ftk_iso_plan_count", "ftk_iso_plan_download",
    "ftk_iso_plan_download_into", "ftk_iso_plan_device_records", "ftk_iso_plan_destroy",
    "ftk_iso_plan_stage_times",
]

ISO_DTYPE = np.dtype([
    ("edge_id", "<i8"), ("label", "<i8"), ("base", "<i4", (4,)), ("off", "<f4", (4,)),
    ("ordinal", "u1"), ("ndim", "u1"), ("reserved", "u1", (6,)),
])
assert ISO_DTYPE.itemsize == 56


class ftk_traj_filter(ctypes.Structure):
    _fields_ = [("min_duration", ctypes.c_double), ("min_points", ctypes.c_int64),
                ("drop_loops", ctypes.c_int32), ("smooth_half_window", ctypes.c_int32)]

SLICE_DTYPE = np.dtype([("label", "<i8"), ("face_a", "<i8"), ("face_b", "<i8"), ("pos", "<f8", (3,))])
assert SLICE_DTYPE.itemsize == 48


def lib():
    """Load libftk_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2011_08697_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "ftk_params_default": (None, [ctypes.POINTER(ftk_params)]),
        "ftk_status_string": (ctypes.c_char_p, [i32]),
        "ftk_last_error": (ctypes.c_char_p, []),
        "ftk_version": (ctypes.c_char_p, []),
        "ftk_track_cp2d": (i32, [vp, i64, i64, i64, ctypes.POINTER(ftk_params), pp, vp]),
        "ftk_track_cp3d": (i32, [vp, i64, i64, i64, i64, ctypes.POINTER(ftk_params), pp, vp]),
        "ftk_result_count": (ctypes.c_size_t, [vp]),
        "ftk_result_data": (vp, [vp]),
        "ftk_result_free": (None, [vp]),
        "ftk_plan_create": (i32, [i32, i64, i64, i64, i64, ctypes.POINTER(ftk_params), pp]),
        "ftk_track_vec2d": (i32, [vp, i64, i64, i64, ctypes.POINTER(ftk_params), pp, vp]),
        "ftk_plan_create_vec2d": (i32, [i64, i64, i64, ctypes.POINTER(ftk_params), pp]),
        "ftk_plan_execute": (i32, [vp, vp, vp]),
        "ftk_plan_count": (i32, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "ftk_plan_download": (i32, [vp, pp]),
        "ftk_plan_download_into": (i32, [vp, vp, i64, ctypes.POINTER(ctypes.c_int64)]),
        "ftk_plan_device_view": (i32, [vp, ctypes.POINTER(ftk_device_view)]),
        "ftk_plan_stage_times": (i32, [vp, ctypes.POINTER(ctypes.c_float), i32, ctypes.POINTER(ctypes.c_int)]),
        "ftk_plan_destroy": (i32, [vp]),
        "ftk_plan_describe": (i32, [vp, ctypes.POINTER(ftk_plan_desc)]),
        "ftk_batch_kernels": (i32, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "ftk_track_cp2d_noalloc": (i32, [vp, i64, i64, i64, ctypes.POINTER(ftk_params), vp, i64,
                                         ctypes.POINTER(ctypes.c_int64), vp]),
        "ftk_batch_create": (i32, [i32, vp, ctypes.POINTER(ftk_params), pp]),
        "ftk_batch_execute": (i32, [vp, vp, vp]),
        "ftk_batch_counts": (i32, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "ftk_batch_download": (i32, [vp, vp]),
        "ftk_batch_destroy": (i32, [vp]),
        "ftk_track_cp2d_batch": (i32, [i32, vp, vp, ctypes.POINTER(ftk_params), vp, vp]),
        "ftk_stream_open": (i32, [i32, i64, i64, i64, ctypes.POINTER(ftk_params), pp]),
        "ftk_stream_push": (i32, [vp, vp, pp]),
        "ftk_stream_close": (i32, [vp, pp]),
        "ftk_server_create": (i32, [ctypes.c_uint64, pp]),
        "ftk_server_used": (i32, [vp, ctypes.POINTER(ctypes.c_uint64)]),
        "ftk_server_destroy": (i32, [vp]),
        "ftk_stream_open_in": (i32, [vp, i32, i64, i64, i64, ctypes.POINTER(ftk_params), pp]),
        "ftk_streams_push": (i32, [i32, vp, vp, vp]),
        "ftk_stream_open_wait": (i32, [vp, i32, i64, i64, i64, ctypes.POINTER(ftk_params), i64, pp]),
        "ftk_stream_footprint": (i32, [i32, i64, i64, i64, ctypes.POINTER(ftk_params),
                                       ctypes.POINTER(ctypes.c_uint64)]),
        "ftk_debug_set_wait_limits": (i32, [i64, i64]),
        "ftk_plan_trajectories": (i32, [vp, pp]),
        "ftk_plan_trajectories_filtered": (i32, [vp, ctypes.POINTER(ftk_traj_filter), pp]),
        "ftk_traj_count": (i64, [vp]),
        "ftk_traj_offsets": (vp, [vp]),
        "ftk_traj_points": (vp, [vp]),
        "ftk_traj_closed": (vp, [vp]),
        "ftk_traj_free": (None, [vp]),
        "ftk_plan_slice": (i32, [vp, ctypes.c_double, pp]),
        "ftk_slice_count": (i64, [vp]),
        "ftk_slice_data": (vp, [vp]),
        "ftk_slice_free": (None, [vp]),
        "ftk_track_iso2d": (i32, [vp, i64, i64, i64, ctypes.c_double, pp, vp]),
        "ftk_track_iso3d": (i32, [vp, i64, i64, i64, i64, ctypes.c_double, pp, vp]),
        "ftk_iso_result_count": (ctypes.c_size_t, [vp]),
        "ftk_iso_result_data": (vp, [vp]),
        "ftk_iso_result_free": (None, [vp]),
        "ftk_iso_plan_create": (i32, [i32, i64, i64, i64, i64, pp]),
        "ftk_iso_plan_execute": (i32, [vp, vp, ctypes.c_double, vp]),
        "ftk_iso_plan_count": (i32, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "ftk_iso_plan_download": (i32, [vp, pp]),
        "ftk_iso_plan_download_into": (i32, [vp, vp, i64, ctypes.POINTER(ctypes.c_int64)]),
        "ftk_iso_plan_device_records": (i32, [vp, pp, ctypes.POINTER(ctypes.c_int64)]),
        "ftk_iso_plan_destroy": (i32, [vp]),
        "ftk_iso_plan_stage_times": (i32, [vp, ctypes.POINTER(ctypes.c_float), i32, ctypes.POINTER(ctypes.c_int)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != FTK_OK:
        raise FtkError(status, lib().ftk_last_error().decode())


def make_params(quant_shift: int = 20, flags: int = 0, max_punctures: int = 0, **kw) -> ftk_params:
    p = ftk_params()
    lib().ftk_params_default(ctypes.byref(p))
    p.quant_shift = quant_shift
    p.flags = flags
    p.max_punctures = max_punctures
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _field_ptr(f):
    """(pointer, keep-alive, shape) for a torch tensor or numpy array."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(f, torch.Tensor):
        if f.dtype != torch.float32 or not f.is_contiguous():
            raise ValueError("field must be a contiguous float32 tensor")
        return ctypes.c_void_p(f.data_ptr()), f, tuple(f.shape)
    a = np.ascontiguousarray(f, dtype=np.float32)
    return ctypes.c_void_p(a.ctypes.data), a, a.shape


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class _ResultOwner:
    """Frees an ftk_result when the array viewing its records is released."""

    def __init__(self, rp):
        self.rp = rp

    def __del__(self):
        try:
            lib().ftk_result_free(self.rp)
        except Exception:
            pass


class _TrajOwner:
    """Frees an ftk_traj when the array viewing its points is released."""

    def __init__(self, h):
        self.h = h

    def __del__(self):
        try:
            lib().ftk_traj_free(self.h)
        except Exception:
            pass


def _take_result(rp) -> np.ndarray:
    """A structured array viewing the result's records in place (no copy);
    the result is freed with the last reference to the array."""
    L = lib()
    owner = _ResultOwner(rp)
    n = L.ftk_result_count(rp)
    if n == 0:
        return np.empty(0, dtype=CP_DTYPE)
    data = L.ftk_result_data(rp)
    raw = (ctypes.c_char * (n * CP_DTYPE.itemsize)).from_address(data)
    raw.owner = owner
    return np.frombuffer(raw, dtype=CP_DTYPE)


def ftk_track_cp2d(f, params: ftk_params | None = None, stream=None) -> np.ndarray:
    ptr, keep, shape = _field_ptr(f)
    if len(shape) != 3:
        raise ValueError("2D field must have shape (nt, ny, nx)")
    nt, ny, nx = shape
    out = ctypes.c_void_p()
    p = params if params is not None else make_params()
    _check(lib().ftk_track_cp2d(ptr, nx, ny, nt, ctypes.byref(p), ctypes.byref(out), _stream_ptr(stream)))
    del keep
    return _take_result(out)


def ftk_track_cp3d(f, params: ftk_params | None = None, stream=None) -> np.ndarray:
    ptr, keep, shape = _field_ptr(f)
    if len(shape) != 4:
        raise ValueError("3D field must have shape (nt, nz, ny, nx)")
    nt, nz, ny, nx = shape
    out = ctypes.c_void_p()
    p = params if params is not None else make_params()
    _check(lib().ftk_track_cp3d(ptr, nx, ny, nz, nt, ctypes.byref(p), ctypes.byref(out), _stream_ptr(stream)))
    del keep
    return _take_result(out)


def ftk_track_vec2d(v, params: ftk_params | None = None, stream=None) -> np.ndarray:
    """Zeros of a 2D vector field v of shape (nt, ny, nx, 2) (components
    interleaved per vertex); morse_index = eigenvalues of the Jacobian with
    negative real part (0 source, 1 saddle, 2 sink, -1 degenerate)."""
    ptr, keep, shape = _field_ptr(v)
    if len(shape) != 4 or shape[3] != 2:
        raise ValueError("2D vector field must have shape (nt, ny, nx, 2)")
    nt, ny, nx, _ = shape
    out = ctypes.c_void_p()
    p = params if params is not None else make_params()
    _check(lib().ftk_track_vec2d(ptr, nx, ny, nt, ctypes.byref(p), ctypes.byref(out), _stream_ptr(stream)))
    del keep
    return _take_result(out)


class Plan:
    """Device workspace for repeated tracking of fields of one shape
    (``ftk_plan_*``); with ``vec2d`` a plan for 2D vector fields of shape
    (nt, ny, nx, 2) (``ftk_plan_create_vec2d``)."""

    def __init__(self, shape, params: ftk_params | None = None, vec2d: bool = False):
        shape = tuple(int(s) for s in shape)
        if vec2d:
            if len(shape) != 4 or shape[3] != 2:
                raise ValueError("vector plan shape must be (nt, ny, nx, 2)")
            nt, ny, nx, _ = shape
            self.shape = shape
            self.ndim = 2
            self._p = params if params is not None else make_params()
            h = ctypes.c_void_p()
            _check(lib().ftk_plan_create_vec2d(nx, ny, nt, ctypes.byref(self._p), ctypes.byref(h)))
            self._h = h
            self._keep = None
            return
        if len(shape) == 3:
            nt, ny, nx = shape
            nz, ndim = 1, 2
        elif len(shape) == 4:
            nt, nz, ny, nx = shape
            ndim = 3
        else:
            raise ValueError("shape must be (nt, ny, nx) or (nt, nz, ny, nx)")
        self.shape = shape
        self.ndim = ndim
        self._p = params if params is not None else make_params()
        h = ctypes.c_void_p()
        _check(lib().ftk_plan_create(ndim, nx, ny, nz, nt, ctypes.byref(self._p), ctypes.byref(h)))
        self._h = h
        self._keep = None

    def execute(self, f, stream=None):
        ptr, keep, shape = _field_ptr(f)
        if tuple(shape) != self.shape:
            raise ValueError(f"field shape {shape} != plan shape {self.shape}")
        self._keep = keep
        _check(lib().ftk_plan_execute(self._h, ptr, _stream_ptr(stream)))

    def count(self) -> int:
        c = ctypes.c_int64()
        _check(lib().ftk_plan_count(self._h, ctypes.byref(c)))
        return c.value

    def download(self) -> np.ndarray:
        out = ctypes.c_void_p()
        _check(lib().ftk_plan_download(self._h, ctypes.byref(out)))
        return _take_result(out)

    def download_into(self, buf: np.ndarray) -> np.ndarray:
        """Records of the last execute copied into ``buf`` (a CP_DTYPE array,
        ideally in pinned memory); returns the filled prefix of buf."""
        if buf.dtype != CP_DTYPE or not buf.flags.c_contiguous:
            raise ValueError("buffer must be a contiguous CP_DTYPE array")
        c = ctypes.c_int64()
        _check(lib().ftk_plan_download_into(self._h, ctypes.c_void_p(buf.ctypes.data), len(buf), ctypes.byref(c)))
        return buf[: c.value]

    def trajectories(self, min_duration: float | None = None, min_points: int = 0, drop_loops: bool = False,
                     smooth_half_window: int = 0):
        """(offsets [n+1], points [P] CP_DTYPE in trajectory then path order,
        closed [n] bool) of the last execute; with any filter argument set,
        the filtered and type-smoothed trajectories."""
        L = lib()
        h = ctypes.c_void_p()
        if min_duration is None and not min_points and not drop_loops and not smooth_half_window:
            _check(L.ftk_plan_trajectories(self._h, ctypes.byref(h)))
        else:
            flt = ftk_traj_filter(float(min_duration or 0.0), int(min_points), int(bool(drop_loops)),
                                  int(smooth_half_window))
            _check(L.ftk_plan_trajectories_filtered(self._h, ctypes.byref(flt), ctypes.byref(h)))
        owner = _TrajOwner(h)
        n = L.ftk_traj_count(h)
        off = np.ctypeslib.as_array(ctypes.cast(L.ftk_traj_offsets(h), ctypes.POINTER(ctypes.c_int64)),
                                    (n + 1,)).copy()
        P = int(off[-1])
        if P:
            # the points are viewed in place (no copy); the trajectories are
            # freed with the last reference to the array
            raw = (ctypes.c_char * (P * CP_DTYPE.itemsize)).from_address(L.ftk_traj_points(h))
            raw.owner = owner
            pts = np.frombuffer(raw, dtype=CP_DTYPE)
        else:
            pts = np.empty(0, dtype=CP_DTYPE)
        closed = np.zeros(n, dtype=bool)
        if n:
            closed = np.ctypeslib.as_array(ctypes.cast(L.ftk_traj_closed(h), ctypes.POINTER(ctypes.c_uint8)),
                                           (n,)).astype(bool)
        return off, pts, closed

    def slice(self, t: float) -> np.ndarray:
        """Crossings of the last execute's trajectories with time t (SLICE_DTYPE)."""
        L = lib()
        h = ctypes.c_void_p()
        _check(L.ftk_plan_slice(self._h, float(t), ctypes.byref(h)))
        try:
            n = L.ftk_slice_count(h)
            out = np.empty(n, dtype=SLICE_DTYPE)
            if n:
                ctypes.memmove(out.ctypes.data, L.ftk_slice_data(h), n * SLICE_DTYPE.itemsize)
            return out
        finally:
            L.ftk_slice_free(h)

    def device_view(self) -> ftk_device_view:
        v = ftk_device_view()
        _check(lib().ftk_plan_device_view(self._h, ctypes.byref(v)))
        return v

    def stage_times(self):
        ms = (ctypes.c_float * 8)()
        n = ctypes.c_int()
        _check(lib().ftk_plan_stage_times(self._h, ms, 8, ctypes.byref(n)))
        return list(ms[: n.value])

    def describe(self) -> dict:
        d = ftk_plan_desc()
        _check(lib().ftk_plan_describe(self._h, ctypes.byref(d)))
        return {k: getattr(d, k) for k, _ in ftk_plan_desc._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().ftk_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# C-ABI names for the plan calls
def ftk_plan_create(shape, params=None) -> Plan:
    return Plan(shape, params)


def ftk_plan_create_vec2d(shape, params=None) -> Plan:
    return Plan(shape, params, vec2d=True)


def ftk_plan_execute(plan: Plan, f, stream=None):
    plan.execute(f, stream)


def ftk_plan_count(plan: Plan) -> int:
    return plan.count()


def ftk_plan_download(plan: Plan) -> np.ndarray:
    return plan.download()


def ftk_plan_destroy(plan: Plan):
    plan.close()


def ftk_version() -> str:
    return lib().ftk_version().decode()


def _dims_array(shapes):
    """int64 [n][3] = (nx, ny, nt) from (nt, ny, nx) shapes."""
    return np.ascontiguousarray([[s[2], s[1], s[0]] for s in shapes], dtype=np.int64)


class Batch:
    """Many independent 2D fields tracked together (``ftk_batch_*``): one
    CUDA graph launch per execute after the first."""

    def __init__(self, shapes, params: ftk_params | None = None):
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        for s in self.shapes:
            if len(s) != 3:
                raise ValueError("batched fields are 2D: (nt, ny, nx)")
        self.n = len(self.shapes)
        self._dims = _dims_array(self.shapes)
        self._p = params if params is not None else make_params()
        h = ctypes.c_void_p()
        _check(lib().ftk_batch_create(self.n, self._dims.ctypes.data, ctypes.byref(self._p), ctypes.byref(h)))
        self._h = h
        self._keep = None

    def execute(self, fields, stream=None):
        if len(fields) != self.n:
            raise ValueError("one field per batch entry")
        ptrs = (ctypes.c_void_p * self.n)()
        keep = []
        for i, f in enumerate(fields):
            p, k, shape = _field_ptr(f)
            if tuple(shape) != self.shapes[i]:
                raise ValueError(f"field {i}: shape {shape} != {self.shapes[i]}")
            ptrs[i] = p.value
            keep.append(k)
        self._keep = (keep, ptrs)
        _check(lib().ftk_batch_execute(self._h, ptrs, _stream_ptr(stream)))

    def counts(self):
        out = np.zeros(self.n, dtype=np.int64)
        _check(lib().ftk_batch_counts(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return out

    def kernels(self) -> int:
        k = ctypes.c_int64()
        _check(lib().ftk_batch_kernels(self._h, ctypes.byref(k)))
        return k.value

    def download(self):
        outs = (ctypes.c_void_p * self.n)()
        _check(lib().ftk_batch_download(self._h, outs))
        return [_take_result(ctypes.c_void_p(outs[i])) for i in range(self.n)]

    def close(self):
        if getattr(self, "_h", None):
            lib().ftk_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def ftk_track_cp2d_batch(fields, params: ftk_params | None = None, stream=None):
    """One-shot batch of 2D device fields; returns one result array per field."""
    n = len(fields)
    ptrs = (ctypes.c_void_p * n)()
    keep = []
    shapes = []
    for i, f in enumerate(fields):
        p, k, shape = _field_ptr(f)
        ptrs[i] = p.value
        keep.append(k)
        shapes.append(shape)
    dims = _dims_array(shapes)
    outs = (ctypes.c_void_p * n)()
    prm = params if params is not None else make_params()
    _check(lib().ftk_track_cp2d_batch(n, ptrs, dims.ctypes.data, ctypes.byref(prm), outs, _stream_ptr(stream)))
    return [_take_result(ctypes.c_void_p(outs[i])) for i in range(n)]


class Server:
    """Admission of streams by device-memory footprint (``ftk_server_*``)."""

    def __init__(self, budget_bytes: int):
        h = ctypes.c_void_p()
        _check(lib().ftk_server_create(int(budget_bytes), ctypes.byref(h)))
        self._h = h

    def used(self) -> int:
        u = ctypes.c_uint64()
        _check(lib().ftk_server_used(self._h, ctypes.byref(u)))
        return u.value

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().ftk_server_destroy(self._h))
            self._h = None


def _spatial(shape):
    shp = tuple(int(v) for v in shape)
    if len(shp) == 2:
        return shp, 2, shp[1], shp[0], 1
    if len(shp) == 3:
        return shp, 3, shp[2], shp[1], shp[0]
    raise ValueError("spatial shape must be (ny, nx) or (nz, ny, nx)")


def ftk_stream_footprint(spatial_shape, params: ftk_params | None = None) -> int:
    """Device bytes a server charges for a stream of this shape at open."""
    _, ndim, nx, ny, nz = _spatial(spatial_shape)
    p = params if params is not None else make_params()
    b = ctypes.c_uint64()
    _check(lib().ftk_stream_footprint(ndim, nx, ny, nz, ctypes.byref(p), ctypes.byref(b)))
    return b.value


def ftk_streams_push(streams, slices):
    """One slice into each of several distinct streams in one call; returns
    the deltas in order."""
    n = len(streams)
    if len(slices) != n:
        raise ValueError("one slice per stream")
    hs = (ctypes.c_void_p * n)()
    ps = (ctypes.c_void_p * n)()
    keep = []
    for i, (st, sl) in enumerate(zip(streams, slices)):
        ptr, k, shape = _field_ptr(sl)
        if tuple(shape) != st.shape:
            raise ValueError(f"slice {i}: shape {shape} != {st.shape}")
        hs[i] = st._h.value
        ps[i] = ptr.value
        keep.append(k)
    outs = (ctypes.c_void_p * n)()
    status = lib().ftk_streams_push(n, hs, ps, outs)
    res = [_take_result(ctypes.c_void_p(outs[i])) if outs[i] else None for i in range(n)]
    _check(status)
    return res


class Stream:
    """In-situ stream (``ftk_stream_*``): push one slice at a time.  With a
    server, ``wait_ms`` > 0 waits (first come, first served) for admission."""

    def __init__(self, spatial_shape, params: ftk_params | None = None, server: Server | None = None,
                 wait_ms: int = 0):
        shp = tuple(int(v) for v in spatial_shape)
        if len(shp) == 2:
            ny, nx = shp
            nz, ndim = 1, 2
        elif len(shp) == 3:
            nz, ny, nx = shp
            ndim = 3
        else:
            raise ValueError("spatial shape must be (ny, nx) or (nz, ny, nx)")
        self.shape = shp
        self._p = params if params is not None else make_params()
        h = ctypes.c_void_p()
        if server is None:
            _check(lib().ftk_stream_open(ndim, nx, ny, nz, ctypes.byref(self._p), ctypes.byref(h)))
        elif wait_ms > 0:
            _check(lib().ftk_stream_open_wait(server._h, ndim, nx, ny, nz, ctypes.byref(self._p), int(wait_ms),
                                              ctypes.byref(h)))
        else:
            _check(lib().ftk_stream_open_in(server._h, ndim, nx, ny, nz, ctypes.byref(self._p), ctypes.byref(h)))
        self._h = h

    def push(self, slice_) -> np.ndarray:
        ptr, keep, shape = _field_ptr(slice_)
        if tuple(shape) != self.shape:
            raise ValueError(f"slice shape {shape} != {self.shape}")
        out = ctypes.c_void_p()
        _check(lib().ftk_stream_push(self._h, ptr, ctypes.byref(out)))
        del keep
        return _take_result(out)

    def close(self, want_final: bool = True):
        if not getattr(self, "_h", None):
            return None
        out = ctypes.c_void_p()
        st = lib().ftk_stream_close(self._h, ctypes.byref(out) if want_final else None)
        self._h = None
        _check(st)
        return _take_result(out) if want_final else None

    def __del__(self):
        try:
            self.close(False)
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Isovolume tracking (ftk_track_iso2d / ftk_track_iso3d, ftk_iso_plan_*)
# ---------------------------------------------------------------------------
class _IsoResultOwner:
    """Frees an ftk_iso_result when the array viewing its records is released."""

    def __init__(self, rp):
        self.rp = rp

    def __del__(self):
        try:
            lib().ftk_iso_result_free(self.rp)
        except Exception:
            pass


def _take_iso_result(rp) -> np.ndarray:
    L = lib()
    owner = _IsoResultOwner(rp)
    n = L.ftk_iso_result_count(rp)
    if n == 0:
        return np.empty(0, dtype=ISO_DTYPE)
    raw = (ctypes.c_char * (n * ISO_DTYPE.itemsize)).from_address(L.ftk_iso_result_data(rp))
    raw.owner = owner
    return np.frombuffer(raw, dtype=ISO_DTYPE)


def ftk_track_iso2d(f, isovalue: float, stream=None) -> np.ndarray:
    """Intersected edges of the level set f = isovalue of a 2D field
    (nt, ny, nx), sorted by edge id, with crossing points and piece labels."""
    ptr, keep, shape = _field_ptr(f)
    if len(shape) != 3:
        raise ValueError("2D field must have shape (nt, ny, nx)")
    nt, ny, nx = shape
    out = ctypes.c_void_p()
    _check(lib().ftk_track_iso2d(ptr, nx, ny, nt, float(isovalue), ctypes.byref(out), _stream_ptr(stream)))
    del keep
    return _take_iso_result(out)


def ftk_track_iso3d(f, isovalue: float, stream=None) -> np.ndarray:
    """As ftk_track_iso2d for a 3D field (nt, nz, ny, nx)."""
    ptr, keep, shape = _field_ptr(f)
    if len(shape) != 4:
        raise ValueError("3D field must have shape (nt, nz, ny, nx)")
    nt, nz, ny, nx = shape
    out = ctypes.c_void_p()
    _check(lib().ftk_track_iso3d(ptr, nx, ny, nz, nt, float(isovalue), ctypes.byref(out), _stream_ptr(stream)))
    del keep
    return _take_iso_result(out)


class IsoPlan:
    """Device workspace for repeated isovolume tracking of fields of one
    shape (``ftk_iso_plan_*``)."""

    def __init__(self, shape):
        shape = tuple(int(s) for s in shape)
        if len(shape) == 3:
            nt, ny, nx = shape
            nz, ndim = 1, 2
        elif len(shape) == 4:
            nt, nz, ny, nx = shape
            ndim = 3
        else:
            raise ValueError("shape must be (nt, ny, nx) or (nt, nz, ny, nx)")
        self.shape = shape
        self.ndim = ndim
        h = ctypes.c_void_p()
        _check(lib().ftk_iso_plan_create(ndim, nx, ny, nz, nt, ctypes.byref(h)))
        self._h = h
        self._keep = None

    def execute(self, f, isovalue: float, stream=None):
        ptr, keep, shape = _field_ptr(f)
        if tuple(shape) != self.shape:
            raise ValueError(f"field shape {shape} != plan shape {self.shape}")
        self._keep = keep
        _check(lib().ftk_iso_plan_execute(self._h, ptr, float(isovalue), _stream_ptr(stream)))

    def count(self) -> int:
        c = ctypes.c_int64()
        _check(lib().ftk_iso_plan_count(self._h, ctypes.byref(c)))
        return c.value

    def download(self) -> np.ndarray:
        out = ctypes.c_void_p()
        _check(lib().ftk_iso_plan_download(self._h, ctypes.byref(out)))
        return _take_iso_result(out)

    def download_into(self, buf: np.ndarray) -> np.ndarray:
        if buf.dtype != ISO_DTYPE or not buf.flags.c_contiguous:
            raise ValueError("buffer must be a contiguous ISO_DTYPE array")
        c = ctypes.c_int64()
        _check(lib().ftk_iso_plan_download_into(self._h, ctypes.c_void_p(buf.ctypes.data), len(buf),
                                                ctypes.byref(c)))
        return buf[: c.value]

    def stage_times(self):
        """Device ms of the last run: [edge bits, emission, cell pass, labels]."""
        buf = (ctypes.c_float * 4)()
        n = ctypes.c_int()
        _check(lib().ftk_iso_plan_stage_times(self._h, buf, 4, ctypes.byref(n)))
        return list(buf[: n.value])

    def close(self):
        if self._h:
            _check(lib().ftk_iso_plan_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
