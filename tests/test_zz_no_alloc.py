"""gjp_forward_noalloc: the forward projection for callers that cannot let a
library allocate device memory while they run -- components handed a fixed
device-memory budget by their framework, real-time reconstruction loops
that forbid allocation once acquisition has started, plug-ins that must not
touch their host application's allocator.

The entry point keeps its per-view table in a fixed per-device array
instead of allocating one.  It forms the same table and runs the same
kernels as gjp_forward, so its projections must be bitwise equal to
gjp_forward's.  Both are called through the C ABI (ctypes), several times
in a row with different problems (storage types, weight functions, a
field-of-view cylinder, more views than one table chunk), so a table left
over from the previous call cannot go unnoticed.  One case is also checked
against the FP64 oracle.  This file is collected last; it passes on its own
in a fresh process as well as after the other tests.
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
    """(volume geometry, cone geometry, device volume, dtype code, weight, fov radius)."""
    if kind == "phantom64":
        vg, cg = synth.c1_geometry()
        vol = torch.from_numpy(synth.voxelize(vg, supersample=2)).cuda()
        return vg, cg, vol, 0, 0, 0.0
    rng = np.random.default_rng(31)
    if kind == "random_bf16_steep":
        vg = VolumeGeometry.centred((37, 29, 23), h=(0.8, 1.1, 1.3))
        cg = synth.random_geometry(rng, vg, 5, 45, 37, steep=True)
        vol = torch.from_numpy(rng.random(vg.n, dtype=np.float32)).cuda().to(torch.bfloat16)
        return vg, cg, vol, 1, 0, 0.0
    if kind == "spl_f16":
        vg = VolumeGeometry.centred((24, 20, 28))
        cg = synth.random_geometry(rng, vg, 7, 33, 29)
        vol = torch.from_numpy(rng.random(vg.n, dtype=np.float32)).cuda().to(torch.float16)
        return vg, cg, vol, 2, 1, 0.0
    if kind == "fov_130_views":
        # more views than one chunk of the table upload, rays clipped to a cylinder
        vg = VolumeGeometry.centred((32, 32, 24))
        cg = synth.circular(130, 40, 30, 90.0, 180.0, 1.6)
        vol = torch.from_numpy(rng.random(vg.n, dtype=np.float32)).cuda()
        return vg, cg, vol, 0, 0, 12.5
    raise ValueError(kind)


def _run(capi, fn, vg, cg, vol, dtype_code, weight, fov):
    st, geom = capi.gjp_geometry_create(cg.n_views, cg.nu, cg.nv, cg.src, cg.det_origin, cg.det_u, cg.det_v)
    assert st == capi.GJP_OK
    try:
        assert capi.gjp_geometry_set_weight(geom, weight) == capi.GJP_OK
        assert capi.gjp_geometry_set_fov(geom, fov) == capi.GJP_OK
        out = torch.full((cg.n_views, cg.nv, cg.nu), float("nan"), device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        st = fn(vol.data_ptr(), dtype_code, *vg.n, vg.h, vg.origin, geom, out.data_ptr(), stream)
        assert st == capi.GJP_OK, capi.gjp_status_string(st)
        assert capi.gjp_stream_status(stream) == capi.GJP_OK
        return out.cpu().numpy()
    finally:
        capi.gjp_geometry_destroy(geom)


KINDS = ("phantom64", "random_bf16_steep", "spl_f16", "fov_130_views")


def test_noalloc_equals_forward_on_calls_in_a_row(capi):
    problems = [_problem(k) for k in KINDS]
    refs = [_run(capi, capi.gjp_forward, *p) for p in problems]
    # allocation-free calls back to back, each bitwise equal to gjp_forward
    outs = [_run(capi, capi.gjp_forward_noalloc, *p) for p in problems]
    for kind, ref, out in zip(KINDS, refs, outs):
        assert np.isfinite(out).all(), kind
        assert np.abs(ref).max() > 0, kind
        np.testing.assert_array_equal(out, ref, err_msg=kind)
    # and once more in the opposite order: the shared table is rewritten each call
    for kind, p, ref in reversed(list(zip(KINDS, problems, refs))):
        np.testing.assert_array_equal(_run(capi, capi.gjp_forward_noalloc, *p), ref, err_msg=kind)


def test_noalloc_matches_the_oracle(capi):
    import oracle
    vg, cg, vol, code, weight, fov = _problem("phantom64")
    out = _run(capi, capi.gjp_forward_noalloc, vg, cg, vol, code, weight, fov).astype(np.float64)
    ref = oracle.forward(vol.cpu().numpy(), vg, cg)
    assert np.abs(out - ref).max() <= TOL32 * np.abs(ref).max()


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
