"""Parity helpers: compare CUDA projections with the FP64 oracle.

Tolerance (spec contract): max |gpu - oracle| <= tol * max |oracle|
with tol = 1e-5 for float32 storage and 5e-3 for 16-bit storage against
the unquantised volume.

Driving-axis ties (reading C2): when the two largest |r_k| of a ray are
within a relative margin of 1e-5, float32 and float64 may pick different
axes; both are valid Joseph integrals of the same line.  For those rays the
GPU value is accepted if it matches the oracle with either axis forced.
"""
from __future__ import annotations

import numpy as np

import oracle

TIE_MARGIN = 1e-5


def all_rays(geom):
    v, iv, iu = np.meshgrid(np.arange(geom.n_views), np.arange(geom.nv), np.arange(geom.nu), indexing="ij")
    return v.ravel(), iu.ravel(), iv.ravel()


def sampled_rays(geom, n, seed):
    rng = np.random.default_rng(seed)
    return (rng.integers(0, geom.n_views, n), rng.integers(0, geom.nu, n), rng.integers(0, geom.nv, n))


def check_rays(gpu_vals, vol, vg, geom, views, ius, ivs, ref_max, tol, threads=0, ref=None):
    """Element-wise check of ``gpu_vals`` for the given rays; returns a dict
    with the max/RMS error (relative to ``ref_max``) and the tie count."""
    gpu_vals = np.asarray(gpu_vals, dtype=np.float64)
    if ref is None:
        ref = oracle.rays(vol, vg, geom, views, ius, ivs, threads=threads)
    err = np.abs(gpu_vals - ref)
    m, rt, margin = oracle.ray_info(vg, geom, views, ius, ivs)
    ties = np.nonzero(margin < TIE_MARGIN)[0]
    if ties.size:
        # second-largest |r| axis of each tied ray
        absrt = np.abs(rt[ties]).copy()
        absrt[np.arange(ties.size), m[ties]] = -1.0
        alt_axis = np.argmax(absrt, axis=1).astype(np.int32)
        alt = oracle.rays(vol, vg, geom, views[ties], ius[ties], ivs[ties], axis=alt_axis, threads=threads)
        err[ties] = np.minimum(err[ties], np.abs(gpu_vals[ties] - alt))
    scale = max(float(ref_max), 1e-30)
    out = {"max_rel": float(err.max() / scale) if err.size else 0.0,
           "rms_rel": float(np.sqrt(np.mean(err ** 2)) / scale) if err.size else 0.0,
           "ties": int(ties.size), "n": int(err.size)}
    assert out["max_rel"] <= tol, f"parity failed: {out} (tol {tol})"
    return out
