"""Out-of-memory paths, injected on the host (gjp_debug_fail_allocations):
the library's next device allocation fails as if the device were full.  A
call that needs it returns GJP_ERR_OOM and leaves its output untouched, a
later call succeeds and computes what it would have computed, and nothing
is left half-built (no GPU fault is involved)."""
import numpy as np
import pytest

import synth
from synth.geometry import VolumeGeometry

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gjp():
    from paper_1609_00958_gb300 import build
    build.build()
    import paper_1609_00958_gb300 as m
    return m


@pytest.fixture
def capi(gjp):
    from paper_1609_00958_gb300 import _capi
    yield _capi
    _capi.gjp_debug_fail_allocations(0)


def _case():
    vg = VolumeGeometry.centred((24, 20, 16))
    cg = synth.circular(5, 30, 20, 80.0, 160.0, 1.6)
    vol = torch.from_numpy(np.random.default_rng(4).random(vg.n, dtype=np.float32)).cuda()
    return vg, cg, vol


def test_forward_table_allocation_failure(gjp, capi):
    vg, cg, vol = _case()
    ref = gjp.forward(vol, gjp.Geometry.from_cone(cg), vg.h)
    g = gjp.Geometry.from_cone(cg)                    # a fresh geometry: its table is not built yet
    out = torch.full(g.proj_shape, 7.0, device="cuda")
    assert capi.gjp_debug_fail_allocations(1) == capi.GJP_OK
    with pytest.raises(gjp.GjpError) as e:
        gjp.forward(vol, g, vg.h, out=out)
    assert e.value.status == capi.GJP_ERR_OOM
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())                   # nothing was launched
    gjp.forward(vol, g, vg.h, out=out)                # the next allocation succeeds
    gjp.stream_status()
    assert torch.equal(out, ref)


def test_adjoint_and_batch_allocation_failures(gjp, capi):
    vg, cg, vol = _case()
    g = gjp.Geometry.from_cone(cg)
    y = torch.rand(g.proj_shape, device="cuda")
    capi.gjp_debug_fail_allocations(1)
    with pytest.raises(gjp.GjpError) as e:
        gjp.adjoint(y, g, vg.n, vg.h)
    assert e.value.status == capi.GJP_ERR_OOM
    back = gjp.adjoint(y, g, vg.n, vg.h)
    assert torch.isfinite(back).all()
    g2 = gjp.Geometry.from_cone(cg)
    items = [(vol, g2, vg.h, None, torch.empty(g2.proj_shape, device="cuda"))]
    capi.gjp_debug_fail_allocations(1)                # the problem's per-view table
    with pytest.raises(gjp.GjpError) as e:
        gjp.Batch(items)
    assert e.value.status == capi.GJP_ERR_OOM
    gjp.forward(vol, g2, vg.h)                        # builds that table
    capi.gjp_debug_fail_allocations(1)                # now the batch's own queue
    with pytest.raises(gjp.GjpError) as e:
        gjp.Batch(items)
    assert e.value.status == capi.GJP_ERR_OOM
    batch = gjp.Batch(items)
    batch.forward()
    gjp.stream_status()
    assert torch.equal(items[0][4], gjp.forward(vol, g2, vg.h))


def test_texture_array_allocation_failure(gjp, capi):
    vg, cg, vol = _case()
    g = gjp.Geometry.from_cone(cg)
    ref = gjp.forward(vol, g, vg.h, path="texture")   # table and arrays built
    g2 = gjp.Geometry.from_cone(cg)
    gjp.forward(vol, g2, vg.h)                        # table built, texture arrays not yet
    capi.gjp_debug_fail_allocations(1)
    with pytest.raises(gjp.GjpError) as e:
        gjp.forward(vol, g2, vg.h, path="texture")
    assert e.value.status == capi.GJP_ERR_OOM
    out = gjp.forward(vol, g2, vg.h, path="texture")
    gjp.stream_status()
    assert torch.equal(out, ref)


def test_pairs_copy_allocation_failure(gjp, capi):
    """AUTO reads the volume directly when the z-paired copy of a 16-bit
    volume cannot be allocated; an explicit "pairs" call reports it."""
    vg, cg, vol = _case()
    g = gjp.Geometry.from_cone(cg)
    v16 = vol.to(torch.bfloat16)
    ref = gjp.forward(v16, g, vg.h, path="gather")   # the table exists from here on
    capi.gjp_debug_fail_allocations(1)
    got = gjp.forward(v16, g, vg.h)
    gjp.stream_status()
    assert torch.equal(got, ref)
    out = torch.full(g.proj_shape, 7.0, device="cuda")
    capi.gjp_debug_fail_allocations(1)
    with pytest.raises(gjp.GjpError) as e:
        gjp.forward(v16, g, vg.h, out=out, path="pairs")
    assert e.value.status == capi.GJP_ERR_OOM
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
    gjp.forward(v16, g, vg.h, out=out, path="pairs")
    gjp.stream_status()
    assert torch.equal(out, ref)
