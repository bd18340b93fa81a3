"""On-disk cache of batched-launch tunings.

``gjp_batch_autotune`` times every problem of a batch under each candidate
launch shape -- the per-configuration block-size search of the paper's
speed section -- which costs several launches per problem.  The best
shapes depend only on the GPU and on the batch's problems (storage type,
grid, voxel size, views and detector, weight, field of view, the scan
geometry itself), so a caller that builds the same batch again can reuse
them.  This module keys a batch by those properties and keeps the chosen
``(tile_u, view_group)`` per problem in a JSON file.

Host-side bookkeeping only: nothing here computes a projection.
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile

VERSION = 1


def geometry_digest(src, det_origin, det_u, det_v, nu: int, nv: int) -> str:
    """Digest of a scan geometry (its float64 arrays and detector size)."""
    import numpy as np
    h = hashlib.sha256()
    for a in (src, det_origin, det_u, det_v):
        h.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    h.update(f"{int(nu)}x{int(nv)}".encode())
    return h.hexdigest()


def problem_signature(dtype: str, shape, voxel_size, origin, geometry_sha: str, weight: str = "lin",
                      fov: float = 0.0) -> dict:
    """The properties of one problem that a launch shape's speed depends on."""
    return {"dtype": str(dtype), "shape": [int(v) for v in shape],
            "voxel_size": [float(v) for v in voxel_size],
            "origin": None if origin is None else [float(v) for v in origin],
            "geometry": str(geometry_sha), "weight": str(weight), "fov": float(fov)}


def batch_key(gpu_name: str, signatures) -> str:
    """Key of a batch: the GPU model and its problems' signatures in order."""
    text = json.dumps({"version": VERSION, "gpu": str(gpu_name), "problems": list(signatures)}, sort_keys=True)
    return hashlib.sha256(text.encode()).hexdigest()


def _read(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def lookup(path: str, key: str, n_problems: int):
    """The cached ``[(tile_u, view_group), ...]`` of a batch, or None when the
    file has no valid entry for ``key``."""
    e = _read(path).get(key)
    try:
        tunings = [(int(t), int(v)) for t, v in e["tunings"]]
    except (TypeError, KeyError, ValueError):
        return None
    if len(tunings) != n_problems or not all(t in (1, 2, 4) and 1 <= v <= 64 for t, v in tunings):
        return None
    return tunings


def store(path: str, key: str, gpu_name: str, tunings) -> None:
    """Adds or replaces the entry of ``key``; the file is rewritten
    atomically (a reader sees the old or the new file, never a torn one)."""
    data = _read(path)
    data[key] = {"gpu": str(gpu_name), "tunings": [[int(t), int(v)] for t, v in tunings]}
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".gjp_tuning_", dir=d)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise
