"""Seeded synthetic volumes (input generation only).

* :data:`SHEPP_LOGAN_SHAPED` -- a project-owned set of 10 ellipsoids with
  the structure of the 3-D Shepp-Logan head phantom used in the paper's
  quality experiments (a dense outer shell, a lower-density interior, two
  tilted ventricle-like ellipsoids and small +/- features).  The paper cites
  the parameter table it used but does not print it, so these numbers are
  this project's own; they are NOT the published Shepp-Logan table.
* :func:`voxelize` -- supersampled rasterisation of any ellipsoid set.
* :func:`random_field` -- seeded uniform [0, 1) volumes.

Ellipsoids are given in normalised coordinates, the cube [-1, 1]^3 mapped
onto the volume's world extent; :func:`ellipsoids_world` returns the
16-double records (rho, centre[3], semi-axes[3], R[9]) that both the
voxeliser and the analytic line-integral code take.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

from .geometry import VolumeGeometry

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_phantom.so")
_lib = None

# density, centre (x, y, z), semi-axes (x, y, z), rotation about z (deg),
# tilt about the ellipsoid's x axis (deg) -- normalised coordinates
SHEPP_LOGAN_SHAPED = [
    (1.00, 0.000, 0.000, 0.000, 0.700, 0.930, 0.880, 0.0, 0.0),
    (-0.78, 0.000, -0.015, 0.000, 0.665, 0.890, 0.845, 0.0, 0.0),
    (-0.22, 0.210, 0.020, -0.120, 0.120, 0.320, 0.230, -17.0, 0.0),
    (-0.22, -0.230, 0.020, -0.120, 0.160, 0.400, 0.260, 19.0, 0.0),
    (0.11, 0.000, 0.360, 0.240, 0.200, 0.240, 0.330, 0.0, 10.0),
    (0.09, 0.000, 0.100, 0.020, 0.045, 0.045, 0.045, 0.0, 0.0),
    (0.09, 0.000, -0.100, 0.020, 0.045, 0.045, 0.045, 0.0, 0.0),
    (0.10, -0.070, -0.600, 0.120, 0.045, 0.025, 0.045, 0.0, 0.0),
    (0.10, 0.000, -0.610, 0.120, 0.022, 0.022, 0.022, 0.0, 0.0),
    (0.10, 0.060, -0.600, 0.120, 0.022, 0.045, 0.022, 0.0, 0.0),
]


def rotation(phi_deg: float, tilt_deg: float) -> np.ndarray:
    """R = Rz(phi) @ Rx(tilt); columns are the ellipsoid's principal axes."""
    p, t = math.radians(phi_deg), math.radians(tilt_deg)
    rz = np.array([[math.cos(p), -math.sin(p), 0.0], [math.sin(p), math.cos(p), 0.0], [0.0, 0.0, 1.0]])
    rx = np.array([[1.0, 0.0, 0.0], [0.0, math.cos(t), -math.sin(t)], [0.0, math.sin(t), math.cos(t)]])
    return rz @ rx


def ellipsoids_world(vg: VolumeGeometry, table=None) -> np.ndarray:
    """(n_ell, 16) float64 records in world units: the normalised cube
    [-1, 1]^3 is scaled (per axis) onto the volume's world extent."""
    table = SHEPP_LOGAN_SHAPED if table is None else table
    centre = np.array(vg.origin) + (np.array(vg.n) - 1) / 2.0 * np.array(vg.h)
    half = np.array(vg.extent) / 2.0
    out = np.zeros((len(table), 16))
    for e, (rho, cx, cy, cz, ax, ay, az, phi, tilt) in enumerate(table):
        out[e, 0] = rho
        out[e, 1:4] = centre + half * np.array((cx, cy, cz))
        out[e, 4:7] = half * np.array((ax, ay, az))
        out[e, 7:16] = rotation(phi, tilt).reshape(-1)
    return out


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "phantom_voxelize.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.phantom_voxelize.restype = ctypes.c_int
        lib.phantom_voxelize.argtypes = [
            ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
        _lib = lib
    return _lib


def voxelize(vg: VolumeGeometry, ellipsoids: np.ndarray | None = None, supersample: int = 2,
             threads: int = 0) -> np.ndarray:
    """(nx, ny, nz) float32 volume: mean of ``supersample^3`` cell-centred
    sub-samples of the ellipsoid sum per voxel."""
    ell = ellipsoids_world(vg) if ellipsoids is None else np.ascontiguousarray(ellipsoids, dtype=np.float64)
    nx, ny, nz = vg.n
    out = np.empty((nx, ny, nz), dtype=np.float32)
    h = np.ascontiguousarray(vg.h, dtype=np.float64)
    o = np.ascontiguousarray(vg.origin, dtype=np.float64)
    rc = _load().phantom_voxelize(int(ell.shape[0]), ell.ctypes.data, nx, ny, nz,
                                  h.ctypes.data, o.ctypes.data, int(supersample),
                                  out.ctypes.data, int(threads))
    if rc != 0:
        raise ValueError("phantom_voxelize rejected its arguments")
    return out


def random_field(shape, seed: int, dtype=np.float32) -> np.ndarray:
    """Uniform [0, 1) field from ``numpy.random.default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    return rng.random(size=tuple(shape), dtype=np.float32).astype(dtype, copy=False)


def gaussian_field(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=tuple(shape), dtype=np.float32)
