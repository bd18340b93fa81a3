"""The z-paired tap source (GJP_PATH_PAIRS): the row-table march reads both
z taps of a transverse row (Eq. 12's v(., ., k) and v(., ., k + 1)) from one
word of a z-paired copy of the volume, so its results must be bitwise those
of the plain gather (GJP_PATH_GATHER), which reads the volume itself; AUTO
takes the paired copy for 16-bit storage.  Covered: circular, random and
steep (z-driven) geometries, ragged and off-centre grids, tiny grids, w_lin
and w_spl, a field-of-view cylinder, all three storage types, the full
512^3 grid, graph capture (AUTO reads the volume directly there, PAIRS
refuses), and the workspace trim."""
import numpy as np
import pytest

import oracle
import synth
from synth.geometry import VolumeGeometry
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DTYPES = ("float32", "bfloat16", "float16")


@pytest.fixture(scope="module")
def gjp():
    from paper_1609_00958_gb300 import build
    build.build()
    import paper_1609_00958_gb300 as m
    return m


def _case(name):
    rng = np.random.default_rng(310 + len(name))
    if name == "c1_phantom":
        vg, cg = synth.c1_geometry()
        return synth.voxelize(vg, supersample=2), vg, cg
    if name == "random_flat":
        vg = VolumeGeometry.centred((33, 40, 27))
        return rng.random(vg.n, dtype=np.float32), vg, synth.random_geometry(rng, vg, 4, 50, 41)
    if name == "random_steep":
        vg = VolumeGeometry.centred((37, 29, 23), h=(0.8, 1.1, 1.3))
        return rng.random(vg.n, dtype=np.float32), vg, synth.random_geometry(rng, vg, 5, 45, 37, steep=True)
    if name == "off_centre_ragged":
        vg = VolumeGeometry((40, 36, 33), (1.0, 1.0, 1.0), (-17.0, -20.5, -15.0))
        cg = synth.circular(5, 37, 45, 120.0, 240.0, 1.6, angles=[0.2, 1.1, 2.5, 3.9, 5.6])
        return rng.random(vg.n, dtype=np.float32), vg, cg
    if name == "tiny_2":
        vg = VolumeGeometry.centred((3, 2, 2))
        cg = synth.circular(4, 7, 35, 12.0, 24.0, 0.3, angles=[0.1, 0.9, 2.0, 4.4])
        return rng.random(vg.n, dtype=np.float32), vg, cg
    if name == "aniso_circular":                      # anisotropic voxels, circular orbit (shared rows)
        vg = VolumeGeometry.centred((40, 36, 32), h=(1.0, 0.9, 1.1))
        return rng.random(vg.n, dtype=np.float32), vg, synth.cone_angle_geometry(40, 36, 6, 10.0)
    if name == "rows_along_minus_z":                  # a warp's z indices fall lane by lane
        vg = VolumeGeometry.centred((40, 36, 64))
        cg = synth.cone_angle_geometry(40, 70, 5, 12.0)
        cg.det_origin = cg.det_origin + (cg.nv - 1) * cg.det_v
        cg.det_v = -cg.det_v
        return rng.random(vg.n, dtype=np.float32), vg, cg
    if name == "c2_small":                            # 64 views of 128^3 = 2^27: AUTO takes the paired copy
        vg, cg = synth.scaled_c2_geometry(128, 128, 64, 10.0)
        return synth.random_field(vg.n, seed=1), vg, cg
    raise ValueError(name)


CASES = ["c1_phantom", "random_flat", "random_steep", "off_centre_ragged", "tiny_2", "aniso_circular",
         "rows_along_minus_z", "c2_small"]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("weight", ["lin", "spl"])
def test_pairs_bitwise_equal_to_gather(gjp, case, weight):
    vol, vg, cg = _case(case)
    g = gjp.Geometry.from_cone(cg, weight=weight)
    for dt in DTYPES:
        v = torch.from_numpy(vol).cuda().to(getattr(torch, dt))
        a = gjp.forward(v, g, vg.h, vg.origin, path="gather")
        b = gjp.forward(v, g, vg.h, vg.origin, path="pairs")
        c = gjp.forward(v, g, vg.h, vg.origin)
        gjp.stream_status()
        assert torch.equal(a, b), (case, weight, dt)
        assert torch.equal(a, c), (case, weight, dt)
    # the paired march against the oracle on the stored bfloat16 values
    v16 = torch.from_numpy(vol).cuda().to(torch.bfloat16)
    got = gjp.forward(v16, g, vg.h, vg.origin, path="pairs").cpu().numpy().astype(np.float64)
    stored = v16.float().cpu().numpy()
    ref = oracle.forward(stored, vg, cg, wfun=1 if weight == "spl" else 0)
    v, iu, iv = parity.all_rays(cg)
    parity.check_rays(got[v, iv, iu], stored, vg, cg, v, iu, iv, np.abs(ref).max(), 1e-5, ref=ref[v, iv, iu])


def test_pairs_with_field_of_view_and_oracle(gjp):
    vg = VolumeGeometry.centred((40, 36, 24), h=(1.0, 1.1, 0.9))
    radius = 16.0
    x = (np.arange(vg.n[0]) - 0.5 * (vg.n[0] - 1)) * vg.h[0]
    y = (np.arange(vg.n[1]) - 0.5 * (vg.n[1] - 1)) * vg.h[1]
    mask = (x[:, None] ** 2 + y[None, :] ** 2 <= (radius - 2.5) ** 2)[:, :, None]
    vol = (np.random.default_rng(8).random(vg.n) * mask).astype(np.float32)
    cg = synth.circular(6, 47, 30, 90.0, 180.0, 1.3, angles=[0.05, 0.8, 1.57, 2.4, 3.9, 5.5])
    g = gjp.Geometry.from_cone(cg)
    g.set_fov(radius)
    v16 = torch.from_numpy(vol).cuda().to(torch.bfloat16)
    a = gjp.forward(v16, g, vg.h, path="gather")
    b = gjp.forward(v16, g, vg.h, path="pairs")
    assert torch.equal(a, b)
    ref = oracle.forward(v16.float().cpu().numpy(), vg, cg, fov=radius)   # the stored values
    got = b.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("dt", DTYPES)
def test_pairs_full_grid(gjp, dt):
    """The 512^3 grid with a 512^2 detector (first 24 of the 360 views)."""
    vg, cg = synth.scaled_c2_geometry(512, 512, 360, 10.0)
    cg = cg.subset(np.arange(24))
    g = gjp.Geometry.from_cone(cg)
    v = torch.from_numpy(synth.random_field(vg.n, seed=0)).cuda().to(getattr(torch, dt))
    a = gjp.forward(v, g, vg.h, path="gather")
    b = gjp.forward(v, g, vg.h, path="pairs")
    gjp.stream_status()
    assert torch.equal(a, b)


def test_pairs_under_graph_capture(gjp):
    from paper_1609_00958_gb300 import _capi
    vol, vg, cg = _case("c2_small")
    g = gjp.Geometry.from_cone(cg)
    v = torch.from_numpy(vol).cuda().to(torch.bfloat16)
    ref = gjp.forward(v, g, vg.h, path="gather")
    out = torch.zeros_like(ref)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        gjp.forward(v, g, vg.h, out=out)              # warm-up: the view table exists before capture
    torch.cuda.synchronize()
    out.zero_()
    graph = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(graph):
        try:
            gjp.forward(v, g, vg.h, out=out, path="pairs")
        except gjp.GjpError as e:
            refused = e.status
        gjp.forward(v, g, vg.h, out=out)              # AUTO reads the volume directly
    assert refused == _capi.GJP_ERR_UNSUPPORTED
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_trim_workspace(gjp):
    vol, vg, cg = _case("c2_small")
    g = gjp.Geometry.from_cone(cg)
    v = torch.from_numpy(vol).cuda().to(torch.float16)
    a = gjp.forward(v, g, vg.h, path="pairs")
    gjp.trim_workspace()                              # the copy of the queued call stays valid
    b = gjp.forward(v, g, vg.h, path="pairs")
    gjp.trim_workspace()
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_pairs_unaligned_volume(gjp):
    """A 16-bit volume that starts 2 bytes past an 8-byte boundary takes the
    one-voxel copy; nz = 128 would otherwise take the four-voxel one."""
    vg, cg = synth.scaled_c2_geometry(64, 64, 6, 10.0)
    vol = synth.random_field((64, 64, 128), seed=3)
    vg = VolumeGeometry.centred((64, 64, 128))
    flat = torch.empty(vol.size + 1, dtype=torch.bfloat16, device="cuda")
    v = flat[1:].view(vol.shape)
    v.copy_(torch.from_numpy(vol).cuda())
    assert v.data_ptr() % 8 != 0
    g = gjp.Geometry.from_cone(cg)
    a = gjp.forward(v, g, vg.h, path="gather")
    b = gjp.forward(v, g, vg.h, path="pairs")
    gjp.stream_status()
    assert torch.equal(a, b)
    ref = gjp.forward(v.contiguous().clone(), g, vg.h, path="pairs")   # aligned copy: the four-voxel form
    assert torch.equal(a, ref)


def test_pairs_on_two_streams_at_once(gjp):
    """The copy's workspace is stream-ordered: forwards of different volumes
    on two streams, queued alternately without waiting, each read their own
    copy and equal the volume read."""
    vol, vg, cg = _case("c2_small")
    g = gjp.Geometry.from_cone(cg)
    vols = [torch.from_numpy(synth.random_field(vg.n, seed=40 + k)).cuda().to(torch.bfloat16) for k in range(4)]
    refs = [gjp.forward(v, g, vg.h, path="gather") for v in vols]
    outs = [torch.empty_like(r) for r in refs]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    for rep in range(3):
        for k, v in enumerate(vols):
            with torch.cuda.stream(streams[k % 2]):
                gjp.forward(v, g, vg.h, out=outs[k], path="pairs")
        torch.cuda.synchronize()
        for k in range(len(vols)):
            assert torch.equal(outs[k], refs[k]), (rep, k)
            outs[k].zero_()
