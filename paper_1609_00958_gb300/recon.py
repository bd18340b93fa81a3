"""Iterative reconstruction with the GJP forward model.

CGLS (conjugate gradients on the normal equations A^T A x = A^T b) built on
the library's forward projection A and matched adjoint A^T -- the kind of
iterative solver the paper's reconstruction experiment drives with its
forward model (the system-matrix view g = A f).  Each iteration costs one
forward and one adjoint projection; the vector updates are a handful of
norms and axpys on device tensors, with the scalars kept on the device.

The solver state (x, r, p, gamma, iteration) can be checkpointed every k
iterations with ``torch.save`` and resumed from such a file.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import torch

from . import adjoint, forward


@dataclass
class CGLSHistory:
    residual: list = field(default_factory=list)   # |b - A x_k|
    rmse: list = field(default_factory=list)       # |x_k - x_true| / sqrt(N), when x_true is given


def _sq(t):
    """|t|^2 accumulated in float64 (a device scalar)."""
    return torch.linalg.vector_norm(t, dtype=torch.float64) ** 2


def cgls(b, geometry, shape, n_iter: int, voxel_size=(1.0, 1.0, 1.0), origin=None, x0=None, x_true=None,
         checkpoint: str | None = None, checkpoint_every: int = 0, resume: bool = False):
    """Run ``n_iter`` CGLS iterations for ``A x = b``.

    Returns ``(x, history)``.  The residual norm |b - A x_k| is
    non-increasing in exact arithmetic (CGLS minimises it over a growing
    Krylov space).  With ``checkpoint`` and ``checkpoint_every > 0`` the
    state is saved to that path every ``checkpoint_every`` iterations;
    ``resume=True`` continues from the file if it exists.

    The solver's scalars (float64 norms, step lengths) stay on the device,
    so an iteration queues its kernels without waiting for the GPU; the
    history is read back at the end and at each checkpoint.  An iteration
    whose step is undefined -- the projected search direction or the
    gradient is exactly zero, i.e. the solution is reached -- leaves the
    state unchanged, so the history always has ``n_iter + 1`` entries.
    """
    dev = b.device
    n_vox = math.prod(int(v) for v in shape)
    zero = torch.zeros((), dtype=torch.float64, device=dev)
    done = CGLSHistory()                  # entries already on the host
    res_d, rmse_d = [], []                # entries still on the device

    def record(r, x):
        res_d.append(torch.linalg.vector_norm(r, dtype=torch.float64))
        if x_true is not None:
            rmse_d.append(torch.linalg.vector_norm(x - x_true, dtype=torch.float64) / math.sqrt(n_vox))

    def flush():
        if res_d:
            done.residual.extend(torch.stack(res_d).tolist())
            res_d.clear()
        if rmse_d:
            done.rmse.extend(torch.stack(rmse_d).tolist())
            rmse_d.clear()

    start = 0
    if resume and checkpoint and os.path.exists(checkpoint):
        st = torch.load(checkpoint, map_location=dev, weights_only=False)
        x, r, p, gamma, start = st["x"], st["r"], st["p"], st["gamma"], st["iteration"]
        done = CGLSHistory(list(st["residual"]), list(st["rmse"]))
    else:
        x = torch.zeros(shape, device=dev, dtype=torch.float32) if x0 is None else x0.clone().float()
        r = b.clone().float()
        if x0 is not None:
            r -= forward(x, geometry, voxel_size, origin)
        s = adjoint(r, geometry, shape, voxel_size, origin)
        p = s.clone()
        gamma = _sq(s)
        record(r, x)
    q = torch.empty_like(b, dtype=torch.float32)
    s = torch.empty(shape, device=dev, dtype=torch.float32)
    for k in range(start, n_iter):
        forward(p, geometry, voxel_size, origin, out=q)
        delta = _sq(q)
        alpha = torch.where(delta > 0, gamma / delta, zero).float()
        x.addcmul_(p, alpha)
        r.addcmul_(q, alpha, value=-1.0)
        adjoint(r, geometry, shape, voxel_size, origin, out=s)
        gamma_new = _sq(s)
        beta = torch.where(gamma > 0, gamma_new / gamma, zero).float()
        p.mul_(beta).add_(s)
        gamma = gamma_new
        record(r, x)
        if checkpoint and checkpoint_every > 0 and (k + 1) % checkpoint_every == 0:
            flush()
            tmp = checkpoint + ".tmp"
            torch.save({"x": x, "r": r, "p": p, "gamma": gamma, "iteration": k + 1,
                        "residual": done.residual, "rmse": done.rmse}, tmp)
            os.replace(tmp, checkpoint)
    flush()
    return x, done
