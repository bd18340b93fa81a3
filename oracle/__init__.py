"""FP64 CPU oracle for the branchless generalized Joseph projector.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The CUDA library never calls it and shares no code with it.

The arithmetic lives in ``gjp_oracle.c`` (plain C, double precision,
OpenMP over rays); this module only marshals numpy arrays through ctypes.
Every function follows Algorithm 1 of the paper (Eq. 1-14) with the
readings listed at the top of ``gjp_oracle.c``.  All functions are pinned
by the ``-m "not gpu"`` tests in ``tests/test_oracle_pins.py`` (closed
forms, brute force, invariants); none is "parity unpinned" except the
absolute level of the analytic-phantom discretisation error, which the
paper does not print.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gjp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_gjp_oracle.so")
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into ``oracle/_gjp_oracle.so``."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-std=c11", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _open(path: str):
    """Open a compiled oracle and declare its signatures."""
    lib = ctypes.CDLL(path)
    lib.gjp_oracle_forward.argtypes = [_P, _I, _I64, _I64, _I64, _P, _P, _I, _I, _I,
                                       _P, _P, _P, _P, _I, ctypes.c_double, _I, _P]
    lib.gjp_oracle_rays.argtypes = [_P, _I, _I64, _I64, _I64, _P, _P, _P, _P, _P, _P,
                                    _I64, _P, _P, _P, _P, _I, ctypes.c_double, _I, _P]
    lib.gjp_oracle_ray_info.argtypes = [_I64, _I64, _I64, _P, _P, _P, _P, _P, _P,
                                        _I64, _P, _P, _P, _P, _P, _P]
    lib.gjp_oracle_adjoint.argtypes = [_P, _I64, _I64, _I64, _P, _P, _I, _I, _I,
                                       _P, _P, _P, _P, _I, ctypes.c_double, _I, ctypes.c_double, _P]
    lib.gjp_oracle_ellipsoid_project.argtypes = [_I, _P, _I, _I, _I, _P, _P, _P, _P,
                                                 _I, _I, _P]
    for f in (lib.gjp_oracle_forward, lib.gjp_oracle_rays, lib.gjp_oracle_ray_info,
              lib.gjp_oracle_adjoint, lib.gjp_oracle_ellipsoid_project):
        f.restype = _I
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _open(_LIB_PATH)
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _vol(vol):
    vol = np.asarray(vol)
    if vol.dtype == np.float64:
        return np.ascontiguousarray(vol), 0
    if vol.dtype == np.float32:
        return np.ascontiguousarray(vol), 1
    # 16-bit storage is widened exactly to float32 by the caller
    raise TypeError(f"oracle volumes are float64 or float32, got {vol.dtype}")


def _geom_arrays(geom):
    return _f64(geom.src), _f64(geom.det_origin), _f64(geom.det_u), _f64(geom.det_v)


def forward(vol, vg, geom, wfun: int = 0, threads: int = 0, fov: float = 0.0) -> np.ndarray:
    """Projections ``(n_views, nv, nu)`` float64 of ``vol`` ``(nx, ny, nz)``;
    ``fov`` > 0 restricts sampling to the cylinder of that world radius
    around the axis through the volume centre parallel to z."""
    v, dt = _vol(vol)
    if tuple(v.shape) != tuple(vg.n):
        raise ValueError("volume shape does not match the volume geometry")
    h, o = _f64(vg.h), _f64(vg.origin)
    src, org, du, dv = _geom_arrays(geom)
    out = np.empty((geom.n_views, geom.nv, geom.nu), dtype=np.float64)
    rc = _load().gjp_oracle_forward(v.ctypes.data, dt, *vg.n, h.ctypes.data, o.ctypes.data,
                                    geom.n_views, geom.nu, geom.nv, src.ctypes.data,
                                    org.ctypes.data, du.ctypes.data, dv.ctypes.data,
                                    int(wfun), float(fov), int(threads), out.ctypes.data)
    if rc:
        raise ValueError("gjp_oracle_forward rejected its arguments")
    return out


def rays(vol, vg, geom, views, ius, ivs, axis=None, wfun: int = 0, threads: int = 0,
         fov: float = 0.0) -> np.ndarray:
    """Line integrals of selected rays; ``axis`` (per ray, -1 = Eq. 3)
    forces the driving axis."""
    v, dt = _vol(vol)
    h, o = _f64(vg.h), _f64(vg.origin)
    src, org, du, dv = _geom_arrays(geom)
    views = np.ascontiguousarray(views, dtype=np.int32)
    ius = np.ascontiguousarray(ius, dtype=np.int32)
    ivs = np.ascontiguousarray(ivs, dtype=np.int32)
    n = views.shape[0]
    ax = None if axis is None else np.ascontiguousarray(np.broadcast_to(axis, (n,)), dtype=np.int32)
    out = np.empty(n, dtype=np.float64)
    rc = _load().gjp_oracle_rays(v.ctypes.data, dt, *vg.n, h.ctypes.data, o.ctypes.data,
                                 src.ctypes.data, org.ctypes.data, du.ctypes.data, dv.ctypes.data,
                                 n, views.ctypes.data, ius.ctypes.data, ivs.ctypes.data,
                                 None if ax is None else ax.ctypes.data, int(wfun), float(fov), int(threads),
                                 out.ctypes.data)
    if rc:
        raise ValueError("gjp_oracle_rays rejected its arguments")
    return out


def ray_info(vg, geom, views, ius, ivs):
    """(m, rt, margin) per ray: Eq. 3 axis, Eq. 4 increment, argmax margin."""
    h, o = _f64(vg.h), _f64(vg.origin)
    src, org, du, dv = _geom_arrays(geom)
    views = np.ascontiguousarray(views, dtype=np.int32)
    ius = np.ascontiguousarray(ius, dtype=np.int32)
    ivs = np.ascontiguousarray(ivs, dtype=np.int32)
    n = views.shape[0]
    m = np.empty(n, dtype=np.int32)
    rt = np.empty((n, 3), dtype=np.float64)
    margin = np.empty(n, dtype=np.float64)
    _load().gjp_oracle_ray_info(*vg.n, h.ctypes.data, o.ctypes.data, src.ctypes.data,
                                org.ctypes.data, du.ctypes.data, dv.ctypes.data, n,
                                views.ctypes.data, ius.ctypes.data, ivs.ctypes.data,
                                m.ctypes.data, rt.ctypes.data, margin.ctypes.data)
    return m, rt, margin


def adjoint(proj, vg, geom, wfun: int = 0, threads: int = 0, max_bytes: float = 4e9,
            fov: float = 0.0) -> np.ndarray:
    """``A^T proj`` as a float64 ``(nx, ny, nz)`` volume."""
    p = _f64(proj)
    if p.shape != (geom.n_views, geom.nv, geom.nu):
        raise ValueError("projection shape does not match the geometry")
    h, o = _f64(vg.h), _f64(vg.origin)
    src, org, du, dv = _geom_arrays(geom)
    out = np.zeros(tuple(vg.n), dtype=np.float64)
    rc = _load().gjp_oracle_adjoint(p.ctypes.data, *vg.n, h.ctypes.data, o.ctypes.data,
                                    geom.n_views, geom.nu, geom.nv, src.ctypes.data,
                                    org.ctypes.data, du.ctypes.data, dv.ctypes.data, int(wfun),
                                    float(fov), int(threads), float(max_bytes), out.ctypes.data)
    if rc:
        raise ValueError("gjp_oracle_adjoint failed")
    return out


def ellipsoid_project(ell, geom, sub: int = 8, threads: int = 0) -> np.ndarray:
    """Analytic projections ``(n_views, nv, nu)``: mean over ``sub x sub``
    sub-pixel rays of the closed-form ellipsoid line integrals."""
    e = _f64(ell).reshape(-1, 16)
    src, org, du, dv = _geom_arrays(geom)
    out = np.empty((geom.n_views, geom.nv, geom.nu), dtype=np.float64)
    rc = _load().gjp_oracle_ellipsoid_project(e.shape[0], e.ctypes.data, geom.n_views, geom.nu,
                                              geom.nv, src.ctypes.data, org.ctypes.data,
                                              du.ctypes.data, dv.ctypes.data, int(sub),
                                              int(threads), out.ctypes.data)
    if rc:
        raise ValueError("gjp_oracle_ellipsoid_project rejected its arguments")
    return out
