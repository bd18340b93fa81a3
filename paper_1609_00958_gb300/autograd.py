"""Differentiable GJP projection.

``project(volume, geometry)`` behaves like ``forward`` but records the
operation for autograd: the forward pass is the GJP kernel (Algorithm 1) and
the backward pass is the library's matched adjoint, so a loss on the
projections differentiates into the volume with d<A x, y>/dx = A^T y.  Both
passes run in the CUDA library; torch only holds the tensors.
"""
from __future__ import annotations

import torch

from . import adjoint, forward


class GJPProjection(torch.autograd.Function):
    """y = A x with A the GJP system matrix of ``geometry``; dL/dx = A^T dL/dy."""

    @staticmethod
    def forward(ctx, volume, geometry, voxel_size, origin):
        ctx.geometry = geometry
        ctx.voxel_size = voxel_size
        ctx.origin = origin
        ctx.shape = tuple(volume.shape)
        ctx.volume_dtype = volume.dtype
        return forward(volume.detach().contiguous(), geometry, voxel_size, origin)

    @staticmethod
    def backward(ctx, grad_proj):
        grad_vol = None
        if ctx.needs_input_grad[0]:
            grad_vol = adjoint(grad_proj.contiguous().float(), ctx.geometry, ctx.shape, ctx.voxel_size, ctx.origin)
            if ctx.volume_dtype != torch.float32:
                grad_vol = grad_vol.to(ctx.volume_dtype)
        return grad_vol, None, None, None


def project(volume, geometry, voxel_size=(1.0, 1.0, 1.0), origin=None):
    """Differentiable forward projection (see :class:`GJPProjection`)."""
    return GJPProjection.apply(volume, geometry, tuple(float(v) for v in voxel_size),
                               None if origin is None else tuple(float(v) for v in origin))
