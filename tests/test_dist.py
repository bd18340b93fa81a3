"""Multi-rank host logic on CPU (gloo, world size 2): view shards cover the
scan exactly once, and the step time a rank reports is the maximum over
ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1609_00958_gb300 import dist as gdist  # noqa: E402


def test_view_shard_partition():
    for n in (0, 1, 7, 360, 361):
        for world in (1, 2, 3, 8):
            ranges = [gdist.view_shard(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c and b >= a
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        gdist.view_shard(10, 2, 2)


def test_single_process_reductions_are_identity():
    assert gdist.max_over_ranks(3.5) == 3.5
    assert gdist.sum_over_ranks(2.0) == 2.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        start, stop = gdist.view_shard(360, rank, world)
        owned = torch.zeros(360, dtype=torch.int64)
        owned[start:stop] = 1
        dist.all_reduce(owned)
        gdist.barrier()
        elapsed = 10.0 + rank           # the slower rank defines the step time
        q.put((rank, int(owned.min()), int(owned.max()), gdist.max_over_ranks(elapsed),
               gdist.sum_over_ranks(stop - start)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, lo, hi, tmax, total in out:
        assert (lo, hi) == (1, 1)           # every view owned by exactly one rank
        assert tmax == 11.0
        assert total == 360.0


# --- one scan split by views (ShardedScan), gloo ranks on CPU -----------------
# The per-rank projector is the FP64 oracle here (CPU ranks have no GPU); the
# test checks the split itself: shards, the gather of the projections and the
# all-reduce of the adjoint volume against one unsplit oracle call.

def _small_case(n_views):
    import synth
    from synth.geometry import VolumeGeometry
    vg = VolumeGeometry.centred((14, 12, 10), h=(1.0, 0.9, 1.1))
    cone = synth.circular(n_views, 12, 10, 60.0, 120.0, 1.7)
    return vg, cone


def _oracle_callables(vg):
    import numpy as np
    import oracle

    def fwd(volume, cone, voxel_size, origin, out, stream):
        return torch.from_numpy(oracle.forward(volume.numpy(), vg, cone, threads=1))

    def adj(proj, cone, shape, voxel_size, origin, out, stream):
        return torch.from_numpy(oracle.adjoint(proj.numpy().astype(np.float64), vg, cone, threads=1))

    return (lambda cone: cone), fwd, adj


def _scan_worker(rank, world, port, n_views, q):
    import numpy as np
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        vg, cone = _small_case(n_views)
        vol = torch.from_numpy(np.random.default_rng(3).random(vg.n))
        mk, fwd, adj = _oracle_callables(vg)
        scan = gdist.ShardedScan(cone, make_geometry=mk, forward_fn=fwd, adjoint_fn=adj)
        local = scan.forward(vol, vg.h).to(torch.float64)
        full = scan.gather(local.float())
        back = scan.adjoint(local, vg.n, vg.h)
        q.put((rank, scan.start, scan.stop, full.numpy(), back.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n_views", [(2, 7), (3, 2)])
def test_sharded_scan_equals_one_unsplit_scan(world, n_views):
    import numpy as np
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_scan_worker, args=(r, world, port, n_views, q)) for r in range(world)]
    for p in procs:
        p.start()
    outs = sorted((q.get(timeout=120) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    vg, cone = _small_case(n_views)
    vol = np.random.default_rng(3).random(vg.n)
    ref = oracle.forward(vol, vg, cone, threads=1)
    ref_back = oracle.adjoint(ref, vg, cone, threads=1)
    covered = np.zeros(n_views, dtype=int)
    for rank, start, stop, full, back in outs:
        covered[start:stop] += 1
        # every rank holds the whole scan's projections, in view order
        np.testing.assert_array_equal(full, ref.astype(np.float32))
        # and the whole A^T y: the sum of the ranks' view blocks
        assert np.abs(back - ref_back).max() <= 1e-12 * np.abs(ref_back).max()
    assert (covered == 1).all()
