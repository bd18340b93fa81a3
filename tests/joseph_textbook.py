"""An independent, per-axis "textbook" Joseph projector for pinning the
oracle (tests only; tiny inputs).

Unlike Algorithm 1's branchless vector form, this version branches on the
driving axis, parametrises each plane crossing by the line parameter
t = (plane - s_m) / r_m, and interpolates with an explicit 2-D (generalised)
bilinear formula in the plane perpendicular to the driving axis -- the
equivalence the paper states after Eq. 12.  Out-of-range neighbours read 0.
"""
from __future__ import annotations

import math

import numpy as np


def _w(d, wfun):
    if wfun == 1:
        return 1.0 - 3.0 * d * d + 2.0 * d ** 3
    return 1.0 - d


def _bilinear(plane: np.ndarray, a: float, b: float, wfun: int) -> float:
    na, nb = plane.shape
    a0, b0 = math.floor(a), math.floor(b)
    wa, wb = _w(a - a0, wfun), _w(b - b0, wfun)

    def f(i, j):
        if 0 <= i < na and 0 <= j < nb:
            return float(plane[i, j])
        return 0.0

    return (wa * wb * f(a0, b0) + (1 - wa) * wb * f(a0 + 1, b0)
            + wa * (1 - wb) * f(a0, b0 + 1) + (1 - wa) * (1 - wb) * f(a0 + 1, b0 + 1))


def ray(vol: np.ndarray, h, origin, src, pix, wfun: int = 0, force_m: int | None = None) -> float:
    h = np.asarray(h, dtype=np.float64)
    origin = np.asarray(origin, dtype=np.float64)
    s = (np.asarray(src, dtype=np.float64) - origin) / h
    d = (np.asarray(pix, dtype=np.float64) - origin) / h
    r = d - s
    if force_m is None:
        m = 0
        if abs(r[1]) > abs(r[m]):
            m = 1
        if abs(r[2]) > abs(r[m]):
            m = 2
    else:
        m = force_m
    world_step = float(np.linalg.norm(h * r)) / abs(r[m])
    total = 0.0
    if m == 0:
        for x in range(vol.shape[0]):
            t = (x - s[0]) / r[0]
            total += _bilinear(vol[x, :, :], s[1] + t * r[1], s[2] + t * r[2], wfun)
    elif m == 1:
        for y in range(vol.shape[1]):
            t = (y - s[1]) / r[1]
            total += _bilinear(vol[:, y, :], s[0] + t * r[0], s[2] + t * r[2], wfun)
    else:
        for z in range(vol.shape[2]):
            t = (z - s[2]) / r[2]
            total += _bilinear(vol[:, :, z], s[0] + t * r[0], s[1] + t * r[1], wfun)
    return total * world_step


def project(vol, vg, geom, wfun: int = 0) -> np.ndarray:
    out = np.zeros((geom.n_views, geom.nv, geom.nu))
    for v in range(geom.n_views):
        for iv in range(geom.nv):
            for iu in range(geom.nu):
                pix = geom.det_origin[v] + iu * geom.det_u[v] + iv * geom.det_v[v]
                out[v, iv, iu] = ray(vol, vg.h, vg.origin, geom.src[v], pix, wfun)
    return out
