"""Iterative reconstruction with the GJP forward model.

CGLS (conjugate gradients on the normal equations A^T A x = A^T b) built on
the library's forward projection A and matched adjoint A^T -- the kind of
iterative solver the paper's reconstruction experiment drives with its
forward model (the system-matrix view g = A f).  Each iteration costs one
forward and one adjoint projection; the vector updates are a handful of
dot products and axpys on device tensors.

The solver state (x, r, p, gamma, iteration) can be checkpointed every k
iterations with ``torch.save`` and resumed from such a file.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import torch

from . import adjoint, forward


@dataclass
class CGLSHistory:
    residual: list = field(default_factory=list)   # |b - A x_k|
    rmse: list = field(default_factory=list)       # |x_k - x_true| / sqrt(N), when x_true is given


def _dot(a, b):
    return torch.dot(a.reshape(-1).double(), b.reshape(-1).double())


def cgls(b, geometry, shape, n_iter: int, voxel_size=(1.0, 1.0, 1.0), origin=None, x0=None, x_true=None,
         checkpoint: str | None = None, checkpoint_every: int = 0, resume: bool = False):
    """Run ``n_iter`` CGLS iterations for ``A x = b``.

    Returns ``(x, history)``.  The residual norm |b - A x_k| is
    non-increasing in exact arithmetic (CGLS minimises it over a growing
    Krylov space).  With ``checkpoint`` and ``checkpoint_every > 0`` the
    state is saved to that path every ``checkpoint_every`` iterations;
    ``resume=True`` continues from the file if it exists.
    """
    dev = b.device
    hist = CGLSHistory()
    start = 0
    if resume and checkpoint and os.path.exists(checkpoint):
        st = torch.load(checkpoint, map_location=dev, weights_only=False)
        x, r, p, gamma, start = st["x"], st["r"], st["p"], st["gamma"], st["iteration"]
        hist = CGLSHistory(list(st["residual"]), list(st["rmse"]))
    else:
        x = torch.zeros(shape, device=dev, dtype=torch.float32) if x0 is None else x0.clone().float()
        r = b.clone().float()
        if x0 is not None:
            r -= forward(x, geometry, voxel_size, origin)
        s = adjoint(r, geometry, shape, voxel_size, origin)
        p = s.clone()
        gamma = _dot(s, s)
        hist.residual.append(float(torch.linalg.vector_norm(r.double())))
        if x_true is not None:
            hist.rmse.append(float(torch.sqrt(torch.mean((x.double() - x_true.double()) ** 2))))
    q = torch.empty_like(b, dtype=torch.float32)
    s = torch.empty(shape, device=dev, dtype=torch.float32)
    for k in range(start, n_iter):
        if float(gamma) == 0.0:
            break
        forward(p, geometry, voxel_size, origin, out=q)
        delta = _dot(q, q)
        if float(delta) == 0.0:
            break
        alpha = gamma / delta
        x.add_(p, alpha=float(alpha))
        r.sub_(q, alpha=float(alpha))
        adjoint(r, geometry, shape, voxel_size, origin, out=s)
        gamma_new = _dot(s, s)
        beta = gamma_new / gamma
        p.mul_(float(beta)).add_(s)
        gamma = gamma_new
        hist.residual.append(float(torch.linalg.vector_norm(r.double())))
        if x_true is not None:
            hist.rmse.append(float(torch.sqrt(torch.mean((x.double() - x_true.double()) ** 2))))
        if checkpoint and checkpoint_every > 0 and (k + 1) % checkpoint_every == 0:
            tmp = checkpoint + ".tmp"
            torch.save({"x": x, "r": r, "p": p, "gamma": gamma, "iteration": k + 1,
                        "residual": hist.residual, "rmse": hist.rmse}, tmp)
            os.replace(tmp, checkpoint)
    return x, hist
