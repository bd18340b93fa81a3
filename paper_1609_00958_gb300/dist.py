"""Multi-rank projection of one scan: views split across ranks.

Every ray of every view is an independent line integral (Algorithm 1), so
the forward projection of one scan shards by views with no exchange: each
rank projects its contiguous range of views from its own copy of the
volume.  The adjoint is a sum over rays (g = A f makes A^T y a sum of the
view blocks' transposes), so each rank backprojects its views into a full
volume and one all-reduce (sum) of that volume completes A^T y.  That
all-reduce is the only collective on the data path; projections are
gathered onto one rank only when a caller asks for them.

Works with any ``torch.distributed`` backend: NCCL with CUDA tensors, or
gloo (tensors are staged through host memory for gloo).  The per-rank
projector calls default to this package's CUDA entry points; tests may pass
other callables with the same signature.
"""
from __future__ import annotations


def view_shard(n_views: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous range ``[start, stop)`` of views owned by ``rank``: the
    first ``n_views % world`` ranks get one extra view."""
    if world < 1 or not (0 <= rank < world) or n_views < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_views, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _group_info(group=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def _is_gloo(group=None) -> bool:
    import torch.distributed as dist
    return dist.get_backend(group) == "gloo"


def all_reduce_sum_(t, group=None):
    """In-place sum of ``t`` over the ranks (a no-op without a process group)."""
    import torch.distributed as dist
    rank, world = _group_info(group)
    if world == 1:
        return t
    if t.is_cuda and _is_gloo(group):
        host = t.cpu()
        dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
        t.copy_(host)
    else:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def _default_forward(volume, geometry, voxel_size, origin, out, stream):
    from . import forward
    return forward(volume, geometry, voxel_size, origin, out=out, stream=stream)


def _default_adjoint(proj, geometry, shape, voxel_size, origin, out, stream):
    from . import adjoint
    return adjoint(proj, geometry, shape, voxel_size, origin, out=out, stream=stream)


def _default_geometry(cone):
    from . import Geometry
    return Geometry.from_cone(cone)


class ShardedScan:
    """One cone-beam scan whose views are split across the ranks of a
    process group.

    ``cone`` is any object with ``src, det_origin, det_u, det_v`` (float64
    ``(n_views, 3)``), ``nu``, ``nv`` and ``subset(views)``.  This rank owns
    views ``[start, stop)`` (``view_shard``).  ``forward`` returns the
    projections of this rank's views; ``gather`` assembles all ranks'
    projections on every rank; ``adjoint`` returns the full ``A^T y`` on
    every rank (local backprojection, then one all-reduce of the volume).
    """

    def __init__(self, cone, group=None, make_geometry=None, forward_fn=None, adjoint_fn=None):
        self.group = group
        self.rank, self.world = _group_info(group)
        self.n_views, self.nu, self.nv = int(len(cone.src)), int(cone.nu), int(cone.nv)
        self.start, self.stop = view_shard(self.n_views, self.rank, self.world)
        self.local_cone = cone.subset(range(self.start, self.stop))
        self.geometry = (make_geometry or _default_geometry)(self.local_cone) if self.stop > self.start else None
        self._forward = forward_fn or _default_forward
        self._adjoint = adjoint_fn or _default_adjoint

    @property
    def local_views(self) -> int:
        return self.stop - self.start

    def forward(self, volume, voxel_size=(1.0, 1.0, 1.0), origin=None, out=None, stream=None):
        """Projections ``(local_views, nv, nu)`` of this rank's views."""
        if self.geometry is None:
            import torch
            return torch.empty((0, self.nv, self.nu), dtype=torch.float32, device=volume.device)
        return self._forward(volume, self.geometry, voxel_size, origin, out, stream)

    def gather(self, local_proj):
        """All ranks' projections ``(n_views, nv, nu)``, in view order, on
        every rank (float32, on ``local_proj``'s device)."""
        import torch
        import torch.distributed as dist
        if self.world == 1:
            return local_proj
        counts = [view_shard(self.n_views, r, self.world) for r in range(self.world)]
        width = max(b - a for a, b in counts)
        dev = local_proj.device
        stage = "cpu" if (local_proj.is_cuda and _is_gloo(self.group)) else dev
        pad = torch.zeros((width, self.nv, self.nu), dtype=torch.float32, device=stage)
        pad[: self.local_views].copy_(local_proj)
        parts = [torch.empty_like(pad) for _ in range(self.world)]
        dist.all_gather(parts, pad, group=self.group)
        full = torch.cat([p[: b - a] for p, (a, b) in zip(parts, counts)])
        return full.to(dev)

    def adjoint(self, local_proj, shape, voxel_size=(1.0, 1.0, 1.0), origin=None, out=None, stream=None):
        """``A^T y`` of the whole scan on every rank: this rank's views are
        backprojected into a full volume, then summed over the ranks."""
        import torch
        if self.geometry is None:                     # a rank without views adds zeros
            vol = out if out is not None else torch.empty(tuple(shape), dtype=local_proj.dtype,
                                                          device=local_proj.device)
            vol.zero_()
        else:
            vol = self._adjoint(local_proj, self.geometry, shape, voxel_size, origin, out, stream)
        return all_reduce_sum_(vol, self.group)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of ``x`` over all ranks (``x`` itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    if device is None:
        device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    """Sum of ``x`` over all ranks (work counters for whole-job rates)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    if device is None:
        device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
