"""One scan split by views across two ranks on the GPU (ShardedScan).

Two processes (gloo process group) share the one GPU.  Each projects its
range of views with the CUDA kernels; the projections are gathered and the
adjoint volumes summed through gloo (host memory).  No kernel of one rank
waits for the other's: the ranks meet only in the host-side collectives.
The gathered projections must be bitwise equal to one unsplit gjp_forward
(every ray is computed by the same kernel either way), the all-reduced
adjoint must match the unsplit gjp_adjoint to 1e-5 (float32 atomics sum in
another order) and the FP64 oracle's transpose to 1e-5.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def _case():
    import synth
    from synth.geometry import VolumeGeometry
    vg = VolumeGeometry.centred((40, 36, 32), h=(1.0, 1.0, 1.2))
    cone = synth.circular(23, 48, 40, 110.0, 220.0, 1.9)
    vol = np.random.default_rng(7).random(vg.n, dtype=np.float32)
    return vg, cone, vol


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1609_00958_gb300 import dist as gdist
        torch.cuda.set_device(0)
        vg, cone, vol = _case()
        v = torch.from_numpy(vol).cuda()
        scan = gdist.ShardedScan(cone)
        local = scan.forward(v, vg.h)
        full = scan.gather(local)
        back = scan.adjoint(local, vg.n, vg.h)
        torch.cuda.synchronize()
        np.save(os.path.join(outdir, f"proj{rank}.npy"), full.cpu().numpy())
        np.save(os.path.join(outdir, f"back{rank}.npy"), back.cpu().numpy())
        np.save(os.path.join(outdir, f"range{rank}.npy"), np.array([scan.start, scan.stop]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_one_scan():
    import torch.multiprocessing as mp
    import oracle
    import paper_1609_00958_gb300 as gjp
    from paper_1609_00958_gb300 import build
    build.build()
    world = 2
    with tempfile.TemporaryDirectory() as outdir:
        ctx = mp.get_context("spawn")
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, outdir)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        projs = [np.load(os.path.join(outdir, f"proj{r}.npy")) for r in range(world)]
        backs = [np.load(os.path.join(outdir, f"back{r}.npy")) for r in range(world)]
        ranges = [tuple(np.load(os.path.join(outdir, f"range{r}.npy"))) for r in range(world)]
    vg, cone, vol = _case()
    assert ranges == [(0, 12), (12, 23)]
    g = gjp.Geometry.from_cone(cone)
    v = torch.from_numpy(vol).cuda()
    ref = gjp.forward(v, g, vg.h)
    ref_back = gjp.adjoint(ref, g, vg.n, vg.h)
    torch.cuda.synchronize()
    ref, ref_back = ref.cpu().numpy(), ref_back.cpu().numpy()
    orc_back = oracle.adjoint(ref.astype(np.float64), vg, cone)
    for r in range(world):
        np.testing.assert_array_equal(projs[r], ref)
        scale = np.abs(ref_back).max()
        assert np.abs(backs[r] - ref_back).max() <= TOL32 * scale
        assert np.abs(backs[r] - orc_back).max() <= TOL32 * np.abs(orc_back).max()
