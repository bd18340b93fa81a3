"""Batched forward projection (gjp_batch_*): many independent problems in
one persistent launch.

Every projection of a batch is computed by the per-ray code of gjp_forward
(same arithmetic, same warp layout), so it must equal gjp_forward of the
same problem bit for bit; gjp_forward itself is held to the FP64 oracle by
tests/test_gpu_parity.py, and a few rays of every batched problem are
checked against the oracle here as well.
"""
import numpy as np
import pytest

import oracle
import synth
from synth.geometry import VolumeGeometry
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def gjp():
    from paper_1609_00958_gb300 import build
    build.build()
    import paper_1609_00958_gb300 as m
    return m


def _small_problems(gjp):
    """Five unlike problems: storage types, weights, anisotropic voxels,
    z-driven rays, ragged detectors, an off-centre grid and a tiny grid."""
    rng = np.random.default_rng(90)
    out = []
    vg, cg = synth.c1_geometry()
    out.append((synth.voxelize(vg, supersample=2), torch.float32, vg, cg.subset(range(0, 32, 3)), "lin"))
    vg = VolumeGeometry.centred((37, 29, 23), h=(0.8, 1.1, 1.3))
    out.append((rng.random(vg.n, dtype=np.float32), torch.bfloat16, vg,
                synth.random_geometry(rng, vg, 5, 45, 37, steep=True), "lin"))
    vg = VolumeGeometry((40, 36, 33), (1.0, 1.0, 1.0), (-17.0, -20.5, -15.0))
    out.append((rng.random(vg.n, dtype=np.float32), torch.float16, vg,
                synth.circular(5, 37, 45, 120.0, 240.0, 1.6, angles=[0.2, 1.1, 2.5, 3.9, 5.6]), "lin"))
    vg = VolumeGeometry.centred((40, 36, 32), h=(1.0, 0.9, 1.1))
    out.append((rng.random(vg.n, dtype=np.float32), torch.float32, vg, synth.cone_angle_geometry(40, 36, 6, 10.0),
                "spl"))
    vg = VolumeGeometry.centred((3, 2, 5))
    out.append((rng.random(vg.n, dtype=np.float32), torch.float32, vg, synth.circular(3, 7, 5, 20.0, 40.0, 0.9),
                "lin"))
    return out


def _batch_inputs(gjp, probs):
    items = []
    for vol_np, dt, vg, cg, w in probs:
        vol = torch.from_numpy(vol_np).cuda().to(dt)
        g = gjp.Geometry.from_cone(cg, weight=w)
        out = torch.full(g.proj_shape, float("nan"), device="cuda")
        items.append((vol, g, vg.h, vg.origin, out))
    return items


def test_small_batch_equals_forward_and_oracle(gjp):
    probs = _small_problems(gjp)
    items = _batch_inputs(gjp, probs)
    batch = gjp.Batch(items)
    assert batch.launches == 1                # every problem in the shared queue
    outs = batch.forward()
    gjp.stream_status()
    for (vol_np, dt, vg, cg, w), (vol, g, h, origin, out) in zip(probs, items):
        ref = gjp.forward(vol, g, h, origin)
        gjp.stream_status()
        assert torch.equal(out, ref)
        # the stored (possibly 16-bit) values against the oracle, all rays
        stored = vol.float().cpu().numpy()
        gpu = out.cpu().numpy().astype(np.float64)
        oref = oracle.forward(stored, vg, cg, wfun=1 if w == "spl" else 0)
        views, ius, ivs = parity.all_rays(cg)
        parity.check_rays(gpu[views, ivs, ius], stored, vg, cg, views, ius, ivs, np.abs(oref).max(), TOL32,
                          ref=oref[views, ivs, ius])
    assert outs[0] is items[0][4]


def test_batch_in_a_cuda_graph_follows_volume_contents(gjp):
    """Captured once, replayed after the volumes change in place: the graph
    reads the new contents (it holds pointers, not data)."""
    probs = _small_problems(gjp)[:3]
    items = _batch_inputs(gjp, probs)
    batch = gjp.Batch(items)
    batch.forward()                         # warm-up outside capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.forward()
    for scale in (1.0, -0.5):
        for vol, *_ in items:
            vol.mul_(scale)
        graph.replay()
        torch.cuda.synchronize()
        for vol, g, h, origin, out in items:
            assert torch.equal(out, gjp.forward(vol, g, h, origin))


def test_batch_autotune_changes_no_result(gjp):
    probs = _small_problems(gjp)
    items = _batch_inputs(gjp, probs)
    batch = gjp.Batch(items)
    before = [o.clone() for o in batch.forward()]
    tunings = batch.autotune(reps=1)
    assert len(tunings) == len(items)
    for tu, vgp in tunings:
        assert tu in (1, 2, 4) and vgp in (1, 4, 8, 16)
    for o in batch.outputs:
        o.fill_(float("nan"))
    after = batch.forward()
    gjp.stream_status()
    for a, b in zip(before, after):
        assert torch.equal(a, b)
    batch.set_tuning(1, 2, 3)
    assert batch.tuning(1) == (2, 3)
    assert torch.equal(batch.forward()[1], before[1])
    for bad in ((8, 1), (4, 0), (4, 65)):
        with pytest.raises(gjp.GjpError):
            batch.set_tuning(0, *bad)
    with pytest.raises(gjp.GjpError):
        batch.tuning(len(items))


def test_batch_autotune_cache(gjp, tmp_path, monkeypatch):
    """Shapes found once are read back from the cache file for the same GPU
    and problems, without timing; another batch is a miss."""
    from paper_1609_00958_gb300 import _capi
    probs = _small_problems(gjp)[:3]
    items = _batch_inputs(gjp, probs)
    cache = str(tmp_path / "tunings.json")
    first = gjp.Batch(items).autotune(reps=1, cache=cache)

    def no_timing(*args, **kwargs):
        raise AssertionError("the search ran although the cache holds this batch")

    monkeypatch.setattr(_capi, "gjp_batch_autotune", no_timing)
    again = gjp.Batch(items)
    assert again.autotune(reps=1, cache=cache) == first
    assert [again.tuning(i) for i in range(len(items))] == first
    ref = [gjp.forward(vol, g, h, origin) for vol, g, h, origin, _ in items]
    for r, o in zip(ref, again.forward()):
        assert torch.equal(r, o)
    with pytest.raises(AssertionError):                 # two of the three problems: not cached
        gjp.Batch(items[:2]).autotune(reps=1, cache=cache)


def test_batch_rejects_invalid_problems(gjp):
    vg = VolumeGeometry.centred((16, 16, 16))
    vol = torch.zeros(vg.n, device="cuda")
    inside = synth.circular(2, 8, 8, 4.0, 40.0, 1.0)          # source inside the volume
    g = gjp.Geometry.from_cone(inside)
    out = torch.empty(g.proj_shape, device="cuda")
    with pytest.raises(gjp.GjpError) as e:
        gjp.Batch([(vol, g, vg.h, None, out)])
    assert e.value.status == 1
    ok = gjp.Geometry.from_cone(synth.circular(2, 8, 8, 100.0, 200.0, 1.0))
    with pytest.raises(gjp.GjpError):
        gjp.Batch([(vol, ok, (1.0, 0.0, 1.0), None, torch.empty(ok.proj_shape, device="cuda"))])


def make_c5(gjp):
    """The 16-problem batching workload (synth.c5_manifest) on the GPU."""
    items, specs = [], synth.c5_manifest()
    for sp in specs:
        vg, cg = sp.geometry()
        vol_np = (synth.voxelize(vg, supersample=2) if sp.content == "phantom"
                  else synth.random_field(vg.n, seed=sp.seed))
        vol = torch.from_numpy(vol_np).cuda().to(getattr(torch, sp.dtype))
        g = gjp.Geometry.from_cone(cg)
        items.append((vol, g, vg.h, None, torch.empty(g.proj_shape, device="cuda")))
    return specs, items


def test_c5_batching_workload(gjp):
    """All 16 problems of the batching workload in one launch equal their
    separate projections bit for bit, and sampled rays of each match the
    oracle on the stored values."""
    specs, items = make_c5(gjp)
    batch = gjp.Batch(items)
    batch.forward()
    gjp.stream_status()
    for k, (sp, (vol, g, h, origin, out)) in enumerate(zip(specs, items)):
        ref = gjp.forward(vol, g, h, origin)
        gjp.stream_status()
        assert torch.equal(out, ref), k
        vg, cg = sp.geometry()
        stored = vol.float().cpu().numpy()
        rays = parity.sampled_rays(cg, 64, seed=k)
        got = out[torch.from_numpy(rays[0]).cuda(), torch.from_numpy(rays[2]).cuda(),
                  torch.from_numpy(rays[1]).cuda()].double().cpu().numpy()
        oref = oracle.rays(stored, vg, cg, *rays)
        scale = max(np.abs(oref).max(), float(out.abs().max()))
        parity.check_rays(got, stored, vg, cg, *rays, scale, TOL32, ref=oref)
        del ref


def test_batch_respects_field_of_view(gjp):
    """A geometry clipped to a field-of-view cylinder projects the same way
    batched and alone."""
    probs = _small_problems(gjp)[:3]
    items = _batch_inputs(gjp, probs)
    items[2][1].set_fov(12.0)
    batch = gjp.Batch(items)
    batch.forward()
    gjp.stream_status()
    for vol, g, h, origin, out in items:
        assert torch.equal(out, gjp.forward(vol, g, h, origin))
    assert not torch.equal(items[2][4], gjp.forward(items[2][0], gjp.Geometry.from_cone(probs[2][3]),
                                                    items[2][2], items[2][3]))


def test_batch_mixes_solo_and_queued_problems_in_a_graph(gjp):
    """Problems that fill the GPU 16 times over run as their own launches
    (a bfloat16 one over 48 views through its z-paired copy, a float32 one
    from its volume), the small ones through the shared queue; captured in a
    CUDA graph and replayed after the volumes change, every projection
    equals gjp_forward bit for bit, and sampled rays of the solo problems
    match the oracle on the stored values."""
    probs = _small_problems(gjp)[:3]
    vg, cg = synth.scaled_c2_geometry(256, 256, 48, 10.0)          # 48 x 64 x 8 = 24576 tiles
    for k, dt in enumerate((torch.bfloat16, torch.float32)):
        probs.append((synth.random_field(vg.n, seed=20 + k), dt, vg, cg, "lin"))
    items = _batch_inputs(gjp, probs)
    batch = gjp.Batch(items)
    assert batch.launches == 4                # queue + bf16 copy and gather + f32 gather
    batch.forward()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.forward()
    for scale in (1.0, -0.5):
        for vol, *_ in items:
            vol.mul_(scale)
        graph.replay()
        torch.cuda.synchronize()
        for vol, g, h, origin, out in items:
            assert torch.equal(out, gjp.forward(vol, g, h, origin))
    for k in (3, 4):
        vol, g, h, origin, out = items[k]
        stored = vol.float().cpu().numpy()
        rays = parity.sampled_rays(cg, 64, seed=k)
        got = out[torch.from_numpy(rays[0]).cuda(), torch.from_numpy(rays[2]).cuda(),
                  torch.from_numpy(rays[1]).cuda()].double().cpu().numpy()
        oref = oracle.rays(stored, vg, cg, *rays)
        parity.check_rays(got, stored, vg, cg, *rays, max(np.abs(oref).max(), float(out.abs().max())), TOL32,
                          ref=oref)
