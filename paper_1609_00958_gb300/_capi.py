"""ctypes binding of ``libgjp.so`` (the C ABI in ``include/gjp.h``).

Argument marshalling only: every step of the projector runs in the CUDA
library.  The functions keep the C names; pointers are passed as integers
(``tensor.data_ptr()``) and ``stream`` as a ``cudaStream_t`` integer.
If the library is missing this module raises at import of the first call
-- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgjp.so")

GJP_OK = 0
GJP_ERR_INVALID_ARG = 1
GJP_ERR_UNSUPPORTED = 2
GJP_ERR_OOM = 3
GJP_ERR_CUDA = 4
GJP_ERR_INTERNAL = 5
GJP_ERR_TIMEOUT = 6

GJP_F32 = 0
GJP_BF16 = 1
GJP_F16 = 2

GJP_WEIGHT_LIN = 0
GJP_WEIGHT_SPL = 1

GJP_PATH_AUTO = 0
GJP_PATH_GATHER = 1
GJP_PATH_SLAB = 2
GJP_PATH_PREFETCH = 3
GJP_PATH_COMBINE = 4
GJP_PATH_TEXTURE = 5
GJP_PATH_HWLIN = 6
GJP_PATH_PAIRS = 7

#: every symbol include/gjp.h declares
EXPORTS = ("gjp_geometry_create", "gjp_geometry_destroy", "gjp_geometry_info", "gjp_geometry_set_weight",
           "gjp_geometry_set_launch", "gjp_geometry_get_launch", "gjp_geometry_set_fov", "gjp_forward",
           "gjp_forward_ex", "gjp_forward_noalloc", "gjp_stream_status", "gjp_selftest_wait_timeout",
           "gjp_selftest_tap_check", "gjp_debug_fail_allocations", "gjp_trim_workspace", "gjp_adjoint", "gjp_adjoint_ex",
           "gjp_footprint", "gjp_batch_create", "gjp_batch_destroy", "gjp_batch_forward",
           "gjp_batch_autotune", "gjp_batch_launch_count", "gjp_batch_get_tuning", "gjp_batch_set_tuning", "gjp_status_string")

#: view limit of gjp_forward_noalloc (GJP_NOALLOC_MAX_VIEWS in include/gjp.h)
GJP_NOALLOC_MAX_VIEWS = 1024

_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D3 = ctypes.POINTER(ctypes.c_double)


class GjpProblem(ctypes.Structure):
    """``gjp_problem`` of include/gjp.h (one forward projection of a batch)."""
    _fields_ = [("d_volume", ctypes.c_void_p), ("dtype", ctypes.c_int), ("nx", ctypes.c_int64),
                ("ny", ctypes.c_int64), ("nz", ctypes.c_int64), ("voxel_size", ctypes.c_double * 3),
                ("volume_origin", ctypes.c_double * 3), ("has_origin", ctypes.c_int),
                ("geometry", ctypes.c_void_p), ("d_proj", ctypes.c_void_p)]


class GjpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {gjp_status_string(status)}")


def load(path: str | None = None):
    """Open the CUDA library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(p)
    lib.gjp_geometry_create.argtypes = [_I, _I, _I, _P, _P, _P, _P, ctypes.POINTER(_P)]
    lib.gjp_geometry_create.restype = _I
    lib.gjp_geometry_destroy.argtypes = [_P]
    lib.gjp_geometry_destroy.restype = None
    lib.gjp_geometry_info.argtypes = [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]
    lib.gjp_geometry_info.restype = _I
    lib.gjp_geometry_set_weight.argtypes = [_P, _I]
    lib.gjp_geometry_set_weight.restype = _I
    lib.gjp_geometry_set_launch.argtypes = [_P, _I, _I]
    lib.gjp_geometry_set_launch.restype = _I
    lib.gjp_geometry_get_launch.argtypes = [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]
    lib.gjp_geometry_get_launch.restype = _I
    lib.gjp_geometry_set_fov.argtypes = [_P, ctypes.c_double]
    lib.gjp_geometry_set_fov.restype = _I
    lib.gjp_forward.argtypes = [_P, _I, _I64, _I64, _I64, _D3, _D3, _P, _P, _P]
    lib.gjp_forward.restype = _I
    lib.gjp_forward_ex.argtypes = [_P, _I, _I64, _I64, _I64, _D3, _D3, _P, _P, _I, _P]
    lib.gjp_forward_ex.restype = _I
    lib.gjp_forward_noalloc.argtypes = [_P, _I, _I64, _I64, _I64, _D3, _D3, _P, _P, _P]
    lib.gjp_forward_noalloc.restype = _I
    lib.gjp_stream_status.argtypes = [_P]
    lib.gjp_stream_status.restype = _I
    lib.gjp_selftest_wait_timeout.argtypes = [_P]
    lib.gjp_selftest_wait_timeout.restype = _I
    lib.gjp_selftest_tap_check.argtypes = [_P]
    lib.gjp_selftest_tap_check.restype = _I
    lib.gjp_debug_fail_allocations.argtypes = [_I]
    lib.gjp_debug_fail_allocations.restype = _I
    lib.gjp_trim_workspace.argtypes = []
    lib.gjp_trim_workspace.restype = _I
    lib.gjp_adjoint.argtypes = [_P, _P, _I64, _I64, _I64, _D3, _D3, _P, _I, _P]
    lib.gjp_adjoint.restype = _I
    lib.gjp_adjoint_ex.argtypes = [_P, _P, _I64, _I64, _I64, _D3, _D3, _P, _I, _I, _P]
    lib.gjp_adjoint_ex.restype = _I
    lib.gjp_footprint.argtypes = [_P, _I, _I64, _I64, _I64, _D3, _D3, _P, _P]
    lib.gjp_footprint.restype = _I
    lib.gjp_batch_create.argtypes = [ctypes.POINTER(GjpProblem), _I, ctypes.POINTER(_P)]
    lib.gjp_batch_create.restype = _I
    lib.gjp_batch_destroy.argtypes = [_P]
    lib.gjp_batch_destroy.restype = None
    lib.gjp_batch_forward.argtypes = [_P, _P]
    lib.gjp_batch_forward.restype = _I
    lib.gjp_batch_autotune.argtypes = [_P, _P, _I]
    lib.gjp_batch_autotune.restype = _I
    lib.gjp_batch_launch_count.argtypes = [_P, ctypes.POINTER(_I)]
    lib.gjp_batch_launch_count.restype = _I
    lib.gjp_batch_get_tuning.argtypes = [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]
    lib.gjp_batch_get_tuning.restype = _I
    lib.gjp_batch_set_tuning.argtypes = [_P, _I, _I, _I]
    lib.gjp_batch_set_tuning.restype = _I
    lib.gjp_status_string.argtypes = [_I]
    lib.gjp_status_string.restype = ctypes.c_char_p
    if path is None:
        _lib = lib
    return lib


def _d3(x):
    if x is None:
        return None
    arr = (ctypes.c_double * 3)(*[float(v) for v in x])
    return arr


def _dptr(a):
    """Address of a C-contiguous float64 numpy array (kept alive by caller)."""
    return ctypes.c_void_p(a.ctypes.data)


def gjp_status_string(status: int) -> str:
    return load().gjp_status_string(int(status)).decode()


def gjp_geometry_create(n_views, nu, nv, src, det_origin, det_u, det_v):
    """Returns (status, handle).  Array arguments: float64 (n_views, 3)."""
    import numpy as np
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (src, det_origin, det_u, det_v)]
    for a in arrs:
        if a.size != 3 * int(n_views):
            return GJP_ERR_INVALID_ARG, None
    h = _P()
    st = load().gjp_geometry_create(int(n_views), int(nu), int(nv), *[_dptr(a) for a in arrs],
                                    ctypes.byref(h))
    return st, (h.value if st == GJP_OK else None)


def gjp_geometry_destroy(handle) -> None:
    if handle:
        load().gjp_geometry_destroy(_P(handle))


def gjp_geometry_info(handle):
    a, b, c = _I(), _I(), _I()
    st = load().gjp_geometry_info(_P(handle) if handle else None, ctypes.byref(a), ctypes.byref(b),
                                  ctypes.byref(c))
    return st, a.value, b.value, c.value


def gjp_geometry_set_weight(handle, weight: int) -> int:
    return load().gjp_geometry_set_weight(_P(handle) if handle else None, int(weight))


def gjp_geometry_set_launch(handle, tile_u: int, view_group: int) -> int:
    return load().gjp_geometry_set_launch(_P(handle) if handle else None, int(tile_u), int(view_group))


def gjp_geometry_set_fov(handle, radius: float) -> int:
    return load().gjp_geometry_set_fov(_P(handle) if handle else None, float(radius))


def gjp_geometry_get_launch(handle):
    a, b = _I(), _I()
    st = load().gjp_geometry_get_launch(_P(handle) if handle else None, ctypes.byref(a), ctypes.byref(b))
    return st, a.value, b.value


def gjp_forward(d_volume: int, dtype: int, nx: int, ny: int, nz: int, voxel_size, volume_origin,
                geometry, d_proj: int, stream: int) -> int:
    return load().gjp_forward(_P(d_volume), int(dtype), int(nx), int(ny), int(nz), _d3(voxel_size),
                              _d3(volume_origin), _P(geometry) if geometry else None, _P(d_proj),
                              _P(stream))


def gjp_forward_ex(d_volume: int, dtype: int, nx: int, ny: int, nz: int, voxel_size, volume_origin,
                   geometry, d_proj: int, path: int, stream: int) -> int:
    return load().gjp_forward_ex(_P(d_volume), int(dtype), int(nx), int(ny), int(nz), _d3(voxel_size),
                                 _d3(volume_origin), _P(geometry) if geometry else None, _P(d_proj), int(path),
                                 _P(stream))


def gjp_forward_noalloc(d_volume: int, dtype: int, nx: int, ny: int, nz: int, voxel_size, volume_origin,
                        geometry, d_proj: int, stream: int) -> int:
    """gjp_forward without any memory allocation (fixed per-device table of
    GJP_NOALLOC_MAX_VIEWS views; see include/gjp.h for the rules)."""
    return load().gjp_forward_noalloc(_P(d_volume), int(dtype), int(nx), int(ny), int(nz), _d3(voxel_size),
                                      _d3(volume_origin), _P(geometry) if geometry else None, _P(d_proj),
                                      _P(stream))


def gjp_stream_status(stream: int) -> int:
    return load().gjp_stream_status(_P(stream))


def gjp_selftest_wait_timeout(stream: int) -> int:
    return load().gjp_selftest_wait_timeout(_P(stream))


def gjp_selftest_tap_check(stream: int) -> int:
    return load().gjp_selftest_tap_check(_P(stream))


def gjp_debug_fail_allocations(n: int) -> int:
    return load().gjp_debug_fail_allocations(int(n))


def gjp_trim_workspace() -> int:
    return load().gjp_trim_workspace()


def gjp_adjoint(d_proj: int, geometry, nx: int, ny: int, nz: int, voxel_size, volume_origin,
                d_volume: int, accumulate: int, stream: int) -> int:
    return load().gjp_adjoint(_P(d_proj), _P(geometry) if geometry else None, int(nx), int(ny), int(nz),
                              _d3(voxel_size), _d3(volume_origin), _P(d_volume), int(accumulate),
                              _P(stream))


def gjp_adjoint_ex(d_proj: int, geometry, nx: int, ny: int, nz: int, voxel_size, volume_origin,
                   d_volume: int, accumulate: int, path: int, stream: int) -> int:
    return load().gjp_adjoint_ex(_P(d_proj), _P(geometry) if geometry else None, int(nx), int(ny), int(nz),
                                 _d3(voxel_size), _d3(volume_origin), _P(d_volume), int(accumulate), int(path),
                                 _P(stream))


def gjp_footprint(geometry, view: int, nx: int, ny: int, nz: int, voxel_size, volume_origin,
                  d_marks: int, stream: int) -> int:
    return load().gjp_footprint(_P(geometry) if geometry else None, int(view), int(nx), int(ny), int(nz),
                                _d3(voxel_size), _d3(volume_origin), _P(d_marks), _P(stream))


def gjp_batch_create(problems):
    """``problems``: sequence of GjpProblem.  Returns (status, handle)."""
    arr = (GjpProblem * max(1, len(problems)))(*problems)
    h = _P()
    st = load().gjp_batch_create(arr if problems else None, len(problems), ctypes.byref(h))
    return st, (h.value if st == GJP_OK else None)


def gjp_batch_destroy(handle) -> None:
    if handle:
        load().gjp_batch_destroy(_P(handle))


def gjp_batch_forward(handle, stream: int) -> int:
    return load().gjp_batch_forward(_P(handle) if handle else None, _P(stream))


def gjp_batch_autotune(handle, stream: int, reps: int) -> int:
    return load().gjp_batch_autotune(_P(handle) if handle else None, _P(stream), int(reps))


def gjp_batch_launch_count(handle):
    n = _I()
    st = load().gjp_batch_launch_count(_P(handle) if handle else None, ctypes.byref(n))
    return st, n.value


def gjp_batch_get_tuning(handle, problem: int):
    a, b = _I(), _I()
    st = load().gjp_batch_get_tuning(_P(handle) if handle else None, int(problem), ctypes.byref(a), ctypes.byref(b))
    return st, a.value, b.value


def gjp_batch_set_tuning(handle, problem: int, tile_u: int, view_group: int) -> int:
    return load().gjp_batch_set_tuning(_P(handle) if handle else None, int(problem), int(tile_u), int(view_group))
