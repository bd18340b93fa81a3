"""gjp_forward_noalloc: the forward projection for callers that cannot let a
library allocate device memory while they run -- components handed a fixed
device-memory budget by their framework, real-time reconstruction loops
that forbid allocation once acquisition has started, plug-ins that must not
touch their host application's allocator.

The entry point keeps its per-view table in a fixed per-device array
instead of allocating one, and must produce what gjp_forward produces.
Both are called through the C ABI (ctypes), twice in a row with different
problems, so a table left over from the previous call cannot go unnoticed.
This file is collected last; it passes on its own in a fresh process as
well as after the other tests.
"""
import numpy as np
import pytest

import synth
from synth.geometry import VolumeGeometry

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5   # the parity tolerance used for float32 storage in the other GPU tests


@pytest.fixture(scope="module")
def capi():
    from paper_1609_00958_gb300 import build, _capi
    build.build()
    _capi.load()
    return _capi


def _problem(kind):
    if kind == "phantom64":
        vg, cg = synth.c1_geometry()
        vol = torch.from_numpy(synth.voxelize(vg, supersample=2)).cuda()
        return vg, cg, vol, 0
    rng = np.random.default_rng(31)
    vg = VolumeGeometry.centred((37, 29, 23), h=(0.8, 1.1, 1.3))
    cg = synth.random_geometry(rng, vg, 5, 45, 37, steep=True)
    vol = torch.from_numpy(rng.random(vg.n, dtype=np.float32)).cuda().to(torch.bfloat16)
    return vg, cg, vol, 1


def _run(capi, fn, vg, cg, vol, dtype_code):
    st, geom = capi.gjp_geometry_create(cg.n_views, cg.nu, cg.nv, cg.src, cg.det_origin, cg.det_u, cg.det_v)
    assert st == capi.GJP_OK
    try:
        out = torch.full((cg.n_views, cg.nv, cg.nu), float("nan"), device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        st = fn(vol.data_ptr(), dtype_code, *vg.n, vg.h, vg.origin, geom, out.data_ptr(), stream)
        assert st == capi.GJP_OK, capi.gjp_status_string(st)
        assert capi.gjp_stream_status(stream) == capi.GJP_OK
        return out.cpu().numpy().astype(np.float64)
    finally:
        capi.gjp_geometry_destroy(geom)


def test_noalloc_matches_forward_on_two_calls_in_a_row(capi):
    problems = [_problem("phantom64"), _problem("random_bf16")]
    refs = [_run(capi, capi.gjp_forward, *p) for p in problems]
    # two allocation-free calls back to back, each checked against gjp_forward
    outs = [_run(capi, capi.gjp_forward_noalloc, *p) for p in problems]
    for ref, out in zip(refs, outs):
        assert np.isfinite(out).all()
        scale = np.abs(ref).max()
        assert scale > 0
        assert np.abs(out - ref).max() <= TOL32 * scale
    # and once more in the opposite order: the shared table is rewritten each call
    again = _run(capi, capi.gjp_forward_noalloc, *problems[0])
    assert np.abs(again - refs[0]).max() <= TOL32 * np.abs(refs[0]).max()


def test_noalloc_rejects_more_views_than_its_table(capi):
    n = capi.GJP_NOALLOC_MAX_VIEWS + 1
    cg = synth.circular(n, 8, 8, 100.0, 200.0, 1.0)
    vg = VolumeGeometry.centred((16, 16, 16))
    st, geom = capi.gjp_geometry_create(cg.n_views, cg.nu, cg.nv, cg.src, cg.det_origin, cg.det_u, cg.det_v)
    assert st == capi.GJP_OK
    try:
        vol = torch.zeros(vg.n, device="cuda")
        out = torch.full((n, 8, 8), 7.0, device="cuda")
        st = capi.gjp_forward_noalloc(vol.data_ptr(), 0, *vg.n, vg.h, None, geom, out.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
        assert st == capi.GJP_ERR_UNSUPPORTED
        torch.cuda.synchronize()
        assert bool((out == 7.0).all())      # nothing was launched
    finally:
        capi.gjp_geometry_destroy(geom)
