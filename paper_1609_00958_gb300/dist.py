"""Multi-rank host logic.

Views of a cone-beam scan are independent problems, so the projector
shards by views (or by whole problems) with no collective on the data
path; ranks meet only to time a step (a barrier and a max-reduction of the
elapsed time).  Works with any ``torch.distributed`` backend (NCCL on GPUs,
gloo on CPU for tests).
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
