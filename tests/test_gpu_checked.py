"""The debug build (GJP_CHECK_TAPS=1): every tap that the interior plane
marches read or reduce without a per-tap test is range-checked first.  The
interior ranges come from a float estimate trimmed with exact integer
arithmetic; a wrong trim would read or reduce outside the grid without any
other symptom than a parity drift.  Here the checked library runs the small
cases of the parity tests -- random and steep geometries (z-driven rays),
ragged detectors, anisotropic and off-centre grids, tiny grids, w_spl, a
field-of-view cylinder, 16-bit storage, the gather / z-paired / prefetch /
batched forwards and the combined / scatter adjoints -- and must report no tap
outside the grid (gjp_stream_status == GJP_OK) and match the FP64 oracle.
A self-test shows the report path works: one thread records an
out-of-grid tap through the same check (indices only, no memory access)."""
import numpy as np
import pytest

import synth
from synth.geometry import VolumeGeometry
from tests.parity import all_rays, check_rays

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def gjp():
    """The package with the checked library swapped in for this module."""
    from paper_1609_00958_gb300 import build, _capi
    path = build.build_checked()
    saved = _capi._lib
    _capi._lib = _capi.load(path)
    import paper_1609_00958_gb300 as pkg
    assert pkg.library_path() is not None
    yield pkg
    import gc
    gc.collect()                   # geometries and batches made here are released by the checked library
    _capi._lib = saved


def _status(gjp):
    from paper_1609_00958_gb300 import _capi
    torch.cuda.synchronize()
    return _capi.gjp_stream_status(torch.cuda.current_stream().cuda_stream)


def _case(name):
    rng = np.random.default_rng(900 + len(name))
    if name == "c1_phantom":
        vg, cg = synth.c1_geometry()
        return synth.voxelize(vg, supersample=2), vg, cg, {}
    if name == "random_steep":                       # z-driven rays: the per-lane march
        vg = VolumeGeometry.centred((37, 29, 23), h=(0.8, 1.1, 1.3))
        return rng.random(vg.n, dtype=np.float32), vg, synth.random_geometry(rng, vg, 5, 45, 37, steep=True), {}
    if name == "random_flat":
        vg = VolumeGeometry.centred((33, 40, 27))
        return rng.random(vg.n, dtype=np.float32), vg, synth.random_geometry(rng, vg, 4, 50, 41), {}
    if name == "off_centre_ragged":
        vg = VolumeGeometry((40, 36, 33), (1.0, 1.0, 1.0), (-17.0, -20.5, -15.0))
        cg = synth.circular(5, 37, 45, 120.0, 240.0, 1.6, angles=[0.2, 1.1, 2.5, 3.9, 5.6])
        return rng.random(vg.n, dtype=np.float32), vg, cg, {}
    if name == "tiny_8":
        vg = VolumeGeometry.centred((8, 8, 8))
        cg = synth.circular(6, 11, 9, 30.0, 60.0, 1.9, angles=[0.0, 0.7, 1.571, 2.3, 3.1416, 4.9])
        return rng.random(vg.n, dtype=np.float32), vg, cg, {}
    if name == "spl":
        vg = VolumeGeometry.centred((30, 26, 34), h=(1.0, 1.2, 0.9))
        cg = synth.circular(4, 40, 52, 100.0, 200.0, 1.5, angles=[0.3, 1.2, 2.2, 4.0])
        return rng.random(vg.n, dtype=np.float32), vg, cg, {"weight": "spl"}
    if name == "fov":
        vg = VolumeGeometry.centred((40, 36, 24), h=(1.0, 1.1, 0.9))
        radius = 16.0
        x = (np.arange(vg.n[0]) - 0.5 * (vg.n[0] - 1)) * vg.h[0]
        y = (np.arange(vg.n[1]) - 0.5 * (vg.n[1] - 1)) * vg.h[1]
        mask = (x[:, None] ** 2 + y[None, :] ** 2 <= (radius - 2.5) ** 2)[:, :, None]
        cg = synth.circular(6, 47, 30, 90.0, 180.0, 1.3, angles=[0.05, 0.8, 1.57, 2.4, 3.9, 5.5])
        return (rng.random(vg.n) * mask).astype(np.float32), vg, cg, {"fov": radius}
    raise ValueError(name)


CASES = ["c1_phantom", "random_steep", "random_flat", "off_centre_ragged", "tiny_8", "spl", "fov"]


def _geometry(gjp, cg, opts):
    g = gjp.Geometry.from_cone(cg, weight=opts.get("weight", "lin"))
    if "fov" in opts:
        g.set_fov(opts["fov"])
    return g


def _oracle_opts(opts):
    return {"wfun": 1 if opts.get("weight") == "spl" else 0, "fov": opts.get("fov", 0.0)}


def test_selftest_reports_a_tap_outside_the_grid(gjp):
    from paper_1609_00958_gb300 import _capi
    s = torch.cuda.current_stream().cuda_stream
    assert _status(gjp) == _capi.GJP_OK
    assert _capi.gjp_selftest_tap_check(s) == _capi.GJP_OK
    assert _capi.gjp_stream_status(s) == _capi.GJP_ERR_INTERNAL
    assert _capi.gjp_stream_status(s) == _capi.GJP_OK          # reported once, then cleared


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("path", ["auto", "prefetch", "pairs"])
def test_checked_forward_stays_in_the_grid(gjp, case, path):
    import oracle
    from paper_1609_00958_gb300 import _capi
    vol, vg, cg, opts = _case(case)
    if path == "prefetch" and opts:
        pytest.skip("the prefetch family implements w_lin without clipping")
    if path == "pairs":                           # the z-paired copy serves 16-bit storage
        vol = torch.from_numpy(vol).to(torch.bfloat16).float().numpy()
    g = _geometry(gjp, cg, opts)
    dv = torch.from_numpy(vol).cuda()
    try:
        out = gjp.forward(dv.to(torch.bfloat16) if path == "pairs" else dv, g, vg.h, vg.origin, path=path)
    except gjp.GjpError as e:
        if e.status == _capi.GJP_ERR_UNSUPPORTED:      # e.g. TMA needs a 16-byte aligned z extent
            pytest.skip(f"{path} does not take this grid")
        raise
    assert _status(gjp) == _capi.GJP_OK
    ref = oracle.forward(vol, vg, cg, **_oracle_opts(opts))
    got = out.cpu().numpy()
    if opts:                       # circular views without driving-axis ties
        assert np.abs(got - ref).max() <= TOL32 * np.abs(ref).max()
    else:                          # either axis of a near-tie is a valid integral (reading C2)
        v, iu, iv = all_rays(cg)
        check_rays(got[v, iv, iu], vol, vg, cg, v, iu, iv, np.abs(ref).max(), TOL32, ref=ref[v, iv, iu])


@pytest.mark.parametrize("case", ["c1_phantom", "random_steep", "off_centre_ragged"])
def test_checked_bf16_forward_stays_in_the_grid(gjp, case):
    import oracle
    from paper_1609_00958_gb300 import _capi
    vol, vg, cg, opts = _case(case)
    g = _geometry(gjp, cg, opts)
    v16 = torch.from_numpy(vol).cuda().to(torch.bfloat16)
    out = gjp.forward(v16, g, vg.h, vg.origin).cpu().numpy().astype(np.float64)
    assert _status(gjp) == _capi.GJP_OK
    ref = oracle.forward(v16.float().cpu().numpy(), vg, cg)     # the stored values
    assert np.abs(out - ref).max() <= TOL32 * np.abs(ref).max()


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("path", ["combine", "gather"])
def test_checked_adjoint_stays_in_the_grid(gjp, case, path):
    import oracle
    from paper_1609_00958_gb300 import _capi
    vol, vg, cg, opts = _case(case)
    g = _geometry(gjp, cg, opts)
    y = np.random.default_rng(5).random((cg.n_views, cg.nv, cg.nu)).astype(np.float32)
    back = gjp.adjoint(torch.from_numpy(y).cuda(), g, vg.n, vg.h, vg.origin, path=path).cpu().numpy()
    assert _status(gjp) == _capi.GJP_OK
    ref = oracle.adjoint(y.astype(np.float64), vg, cg, **_oracle_opts(opts))
    assert np.abs(back - ref).max() <= TOL32 * np.abs(ref).max()


def test_checked_batch_stays_in_the_grid(gjp):
    import oracle
    from paper_1609_00958_gb300 import _capi
    items, refs = [], []
    for case in ("c1_phantom", "random_steep", "off_centre_ragged", "tiny_8"):
        vol, vg, cg, opts = _case(case)
        g = _geometry(gjp, cg, opts)
        items.append((torch.from_numpy(vol).cuda(), g, vg.h, vg.origin,
                      torch.empty(g.proj_shape, device="cuda")))
        refs.append(oracle.forward(vol, vg, cg))
    batch = gjp.Batch(items)
    batch.forward()
    assert _status(gjp) == _capi.GJP_OK
    for (vol, g, h, o, out), ref in zip(items, refs):
        assert np.abs(out.cpu().numpy() - ref).max() <= TOL32 * np.abs(ref).max()
