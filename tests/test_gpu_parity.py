"""Parity of the CUDA projector (through the C ABI) with the FP64 oracle.

Bar: max |gpu - oracle| <= 1e-5 * max |oracle| for float32 storage; for
16-bit storage <= 1e-5 against the oracle on the stored (quantised) values
and <= 5e-3 against the unquantised float32 volume.  Driving-axis ties
follow reading C2 (see tests/parity.py).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from synth.geometry import ConeGeometry, VolumeGeometry
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 5e-3


@pytest.fixture(scope="module")
def gjp():
    from paper_1609_00958_gb300 import build
    build.build()
    import paper_1609_00958_gb300 as m
    return m


def _project(gjp, vol_np, vg, cg, dtype=torch.float32, path="auto"):
    vol = torch.from_numpy(np.ascontiguousarray(vol_np)).to("cuda").to(dtype)
    g = gjp.Geometry.from_cone(cg)
    out = gjp.forward(vol, g, voxel_size=vg.h, origin=vg.origin, path=path)
    gjp.stream_status()
    return out.cpu().numpy().astype(np.float64), vol


def _full_check(gjp, vol_np, vg, cg, tol=TOL32, dtype=torch.float32, path="auto"):
    gpu, _ = _project(gjp, vol_np, vg, cg, dtype, path)
    ref = oracle.forward(vol_np, vg, cg)
    views, ius, ivs = parity.all_rays(cg)
    return parity.check_rays(gpu[views, ivs, ius], vol_np, vg, cg, views, ius, ivs,
                             np.abs(ref).max(), tol, ref=ref[views, ivs, ius])


# --- c1: 64^3 Shepp-Logan-shaped phantom, 32 views, 64x64 -------------------

@pytest.mark.parametrize("path", ["gather", "slab", "prefetch"])
def test_c1_phantom_fp32_all_rays(gjp, path):
    vg, cg = synth.c1_geometry()
    vol = synth.voxelize(vg, supersample=2)
    r = _full_check(gjp, vol, vg, cg, path=path)
    assert r["n"] == 32 * 64 * 64


@pytest.mark.parametrize("path", ["gather", "slab", "prefetch"])
def test_c1_random_field_fp32_all_rays(gjp, path):
    vg, cg = synth.c1_geometry()
    _full_check(gjp, synth.random_field(vg.n, seed=0), vg, cg, path=path)


def test_c1_matches_analytic_phantom(gjp):
    """GJP of the rasterised phantom vs closed-form ellipsoid integrals
    (projection-quality experiment): same bounded discretisation error as
    the oracle's."""
    vg, cg = synth.c1_geometry()
    ell = synth.ellipsoids_world(vg)
    gpu, _ = _project(gjp, synth.voxelize(vg, ell, supersample=2), vg, cg)
    ana = oracle.ellipsoid_project(ell, cg, sub=8)
    assert np.abs(gpu - ana).sum() / np.abs(ana).sum() < 0.02


def test_linear_and_spline_weights_against_analytic_projections(gjp):
    """Projection quality of w_lin (Eq. 13) and w_spl (Eq. 14) on the GPU:
    l1 error of the rasterised phantom's projections against the closed-form
    ellipsoid integrals, for 64^3, 128^3 and 256^3 grids over the same
    64-unit cube (8 views, detectors as wide as the grid).  The paper finds
    GJP_lin the closer of the two; both errors must also shrink with the
    grid.  With GJP_REPORT_DIR set, the table is written there as JSON."""
    import json
    import os
    table = {}
    for n in (64, 128, 256):
        vg = VolumeGeometry.centred((n, n, n), h=(64.0 / n,) * 3)
        w = 64.0
        cg = synth.circular(8, n, n, 4 * w, 8 * w, synth.covering_pitch(w, 4 * w, 8 * w, n))
        ell = synth.ellipsoids_world(vg)
        vol = torch.from_numpy(synth.voxelize(vg, ell, supersample=2)).cuda()
        pa = oracle.ellipsoid_project(ell, cg, sub=8)
        row = {}
        for wname in ("lin", "spl"):
            g = gjp.Geometry.from_cone(cg, weight=wname)
            got = gjp.forward(vol, g, vg.h).double().cpu().numpy()
            gjp.stream_status()
            row[wname] = float(np.abs(got - pa).sum() / np.abs(pa).sum())
        table[n] = row
        assert row["lin"] < row["spl"], (n, row)
    for a, b in ((64, 128), (128, 256)):
        assert table[b]["lin"] < table[a]["lin"] and table[b]["spl"] < table[a]["spl"], table
    out_dir = os.environ.get("GJP_REPORT_DIR")
    if out_dir:
        with open(os.path.join(out_dir, "weights_l1.json"), "w") as f:
            json.dump(table, f, indent=1)


# --- arbitrary geometry: z-driven rays, anisotropic voxels, ragged tiles ----

@pytest.mark.parametrize("steep", [False, True])
def test_random_geometry_ragged_detector(gjp, steep):
    rng = np.random.default_rng(100 + steep)
    vg = VolumeGeometry.centred((37, 29, 23), h=(0.8, 1.1, 1.3))
    cg = synth.random_geometry(rng, vg, 5, 45, 37, steep=steep)
    vol = rng.random(vg.n, dtype=np.float32)
    r = _full_check(gjp, vol, vg, cg)
    if steep:
        m, _, _ = oracle.ray_info(vg, cg, *parity.all_rays(cg))
        assert (m == 2).sum() > 100


def test_off_centre_volume_origin(gjp):
    rng = np.random.default_rng(7)
    vg = VolumeGeometry((30, 34, 26), (1.0, 0.9, 1.2), (-12.0, -20.0, -9.0))
    cg = synth.random_geometry(rng, vg, 3, 33, 31)
    _full_check(gjp, rng.random(vg.n, dtype=np.float32), vg, cg)


# --- 16-bit storage: float32 weights and accumulation ------------------------

@pytest.mark.parametrize("path", ["gather", "slab", "prefetch"])
@pytest.mark.parametrize("dt", ["bfloat16", "float16"])
@pytest.mark.parametrize("content", ["phantom", "random"])
def test_16bit_storage(gjp, dt, content, path):
    vg, cg = synth.c1_geometry()
    vol = synth.voxelize(vg, supersample=2) if content == "phantom" else synth.random_field(vg.n, seed=3)
    tdt = getattr(torch, dt)
    gpu, tvol = _project(gjp, vol, vg, cg, tdt, path)
    stored = tvol.float().cpu().numpy()               # exact widening of the stored values
    views, ius, ivs = parity.all_rays(cg)
    ref_q = oracle.forward(stored, vg, cg)
    kernel = parity.check_rays(gpu[views, ivs, ius], stored, vg, cg, views, ius, ivs,
                               np.abs(ref_q).max(), TOL32, ref=ref_q[views, ivs, ius])
    ref = oracle.forward(vol, vg, cg)
    total = parity.check_rays(gpu[views, ivs, ius], vol, vg, cg, views, ius, ivs,
                              np.abs(ref).max(), TOL16, ref=ref[views, ivs, ius])
    assert kernel["max_rel"] < 1e-5 and total["max_rel"] < TOL16


# --- adjoint -----------------------------------------------------------------

def _adjoint_gpu(gjp, y_np, vg, cg, accumulate_into=None):
    g = gjp.Geometry.from_cone(cg)
    y = torch.from_numpy(np.ascontiguousarray(y_np, dtype=np.float32)).cuda()
    out = None if accumulate_into is None else torch.from_numpy(accumulate_into.astype(np.float32)).cuda()
    res = gjp.adjoint(y, g, vg.n, voxel_size=vg.h, origin=vg.origin, out=out,
                      accumulate=accumulate_into is not None)
    torch.cuda.synchronize()
    return res.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("steep", [False, True])
def test_adjoint_matches_oracle_transpose(gjp, steep):
    rng = np.random.default_rng(200 + steep)
    vg = VolumeGeometry.centred((40, 36, 33), h=(1.0, 0.9, 1.1))
    cg = synth.random_geometry(rng, vg, 4, 41, 35, steep=steep)
    y = rng.standard_normal((cg.n_views, cg.nv, cg.nu)).astype(np.float32)
    gpu = _adjoint_gpu(gjp, y, vg, cg)
    ref = oracle.adjoint(y.astype(np.float64), vg, cg)
    err = np.abs(gpu - ref).max() / np.abs(ref).max()
    assert err <= TOL32, err


@pytest.mark.parametrize("path", ["gather", "slab", "combine"])
@pytest.mark.parametrize("geom", ["circular", "diagonal"])
def test_adjoint_families_match_oracle_on_aligned_volume(gjp, path, geom):
    """Volume rows of 32 floats (TMA-compatible) so the slab adjoint runs;
    views near 45 degrees put the driving-axis tie line across the panel, so
    some tiles mix x- and y-driven rays (scatter fallback inside the kernel)."""
    rng = np.random.default_rng(300 + (geom == "diagonal"))
    vg = VolumeGeometry.centred((48, 40, 32), h=(1.0, 0.9, 1.1))
    if geom == "circular":
        cg = synth.cone_angle_geometry(48, 40, 6, 10.0)
    else:
        cg = synth.cone_angle_geometry(48, 41, 3, 10.0, angles=[math.radians(a) for a in (45.0, 43.0, 137.0)])
    y = rng.standard_normal((cg.n_views, cg.nv, cg.nu)).astype(np.float32)
    g = gjp.Geometry.from_cone(cg)
    out = gjp.adjoint(torch.from_numpy(y).cuda(), g, vg.n, voxel_size=vg.h, origin=vg.origin, path=path)
    gjp.stream_status()
    ref = oracle.adjoint(y.astype(np.float64), vg, cg)
    err = np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= TOL32, err


def test_adjoint_slab_equals_gather_full_size(gjp):
    """Both adjoint families on the 512^3 / 360-view workload agree to
    float32 summation-order rounding."""
    vg, cg = synth.c2_geometry()
    g = gjp.Geometry.from_cone(cg)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    y = torch.rand(cg.n_views, cg.nv, cg.nu, device="cuda", generator=gen)
    a = gjp.adjoint(y, g, vg.n, path="gather")
    b = gjp.adjoint(y, g, vg.n, path="slab")
    gjp.stream_status()
    assert ((a - b).abs().max() / a.abs().max()).item() < 1e-5


@pytest.mark.parametrize("case", ["random", "random_steep", "coarse_detector", "unaligned_rows", "dense_detector",
                                  "rows_along_minus_z", "ragged"])
@pytest.mark.parametrize("launch", [(4, 1), (8, 3), (1, 2)])
def test_adjoint_combine_matches_oracle(gjp, case, launch):
    """The warp-combined adjoint against the oracle's transpose on the cases
    that stress it: warps whose rays do not share a transverse row (random
    and z-driven views: per-tap scatter), rays several voxels apart (a
    coarse detector: no tap is shared), rays closer than a voxel (two rays
    per voxel), an odd z row length, a detector whose last warp is partly
    empty, under several launch shapes."""
    rng = np.random.default_rng(400 + len(case))
    if case.startswith("random"):
        vg = VolumeGeometry.centred((37, 29, 23), h=(0.8, 1.1, 1.3))
        cg = synth.random_geometry(rng, vg, 5, 45, 37, steep=case.endswith("steep"))
    elif case == "coarse_detector":
        vg = VolumeGeometry.centred((40, 40, 160))
        cg = synth.circular(4, 24, 40, 300.0, 600.0, 4.0, pitch_v=8.0)
    elif case == "unaligned_rows":
        vg = VolumeGeometry.centred((36, 30, 27))
        cg = synth.cone_angle_geometry(36, 40, 5, 12.0)
    elif case == "dense_detector":
        vg = VolumeGeometry.centred((30, 30, 24))
        cg = synth.circular(4, 33, 70, 90.0, 180.0, 0.55)
    elif case == "rows_along_minus_z":
        # detector rows run along -z: a warp's z indices decrease lane by lane
        vg = VolumeGeometry.centred((40, 36, 32))
        cg = synth.cone_angle_geometry(40, 38, 5, 12.0)
        cg.det_origin = cg.det_origin + (cg.nv - 1) * cg.det_v
        cg.det_v = -cg.det_v
    else:
        vg = VolumeGeometry.centred((33, 35, 44))
        cg = synth.circular(3, 37, 45, 120.0, 240.0, 1.6, angles=[0.3, 1.9, 4.0])
    y = rng.standard_normal((cg.n_views, cg.nv, cg.nu)).astype(np.float32)
    g = gjp.Geometry.from_cone(cg)
    g.set_launch(*launch)
    out = gjp.adjoint(torch.from_numpy(y).cuda(), g, vg.n, voxel_size=vg.h, origin=vg.origin, path="combine")
    gjp.stream_status()
    ref = oracle.adjoint(y.astype(np.float64), vg, cg)
    err = np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= TOL32, err


def test_adjoint_combine_spline_weight(gjp):
    rng = np.random.default_rng(73)
    vg = VolumeGeometry.centred((40, 36, 32), h=(1.0, 0.9, 1.1))
    cg = synth.cone_angle_geometry(40, 36, 5, 10.0)
    y = rng.standard_normal((cg.n_views, cg.nv, cg.nu)).astype(np.float32)
    g = gjp.Geometry.from_cone(cg, weight="spl")
    out = gjp.adjoint(torch.from_numpy(y).cuda(), g, vg.n, vg.h, vg.origin, path="combine")
    gjp.stream_status()
    ref = oracle.adjoint(y.astype(np.float64), vg, cg, wfun=1)
    assert np.abs(out.cpu().numpy() - ref).max() <= TOL32 * np.abs(ref).max()


def test_adjoint_combine_equals_gather_full_size(gjp):
    """Warp-combined and tap-by-tap adjoints on the 512^3 / 360-view workload
    agree to float32 summation-order rounding, in two launch orders."""
    vg, cg = synth.c2_geometry()
    g = gjp.Geometry.from_cone(cg)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(8)
    y = torch.rand(cg.n_views, cg.nv, cg.nu, device="cuda", generator=gen)
    a = gjp.adjoint(y, g, vg.n, path="gather")
    for launch in ((4, 1), (8, 8)):
        g.set_launch(*launch)
        b = gjp.adjoint(y, g, vg.n, path="combine")
        gjp.stream_status()
        assert ((a - b).abs().max() / a.abs().max()).item() < 1e-5


def test_launch_shape_changes_no_result(gjp):
    """tile_u and view_group reorder work only: gather forward results are
    bitwise equal (each ray is one thread with the same arithmetic, and a
    warp is always 32 rows of one column); the prefetch family sums its
    planes in another order and agrees to float32 rounding; invalid shapes
    are rejected."""
    rng = np.random.default_rng(12)
    vg = VolumeGeometry.centred((41, 38, 36))
    cg = synth.cone_angle_geometry(41, 45, 7, 10.0)
    vol = torch.from_numpy(rng.random(vg.n, dtype=np.float32)).cuda()
    g = gjp.Geometry.from_cone(cg)
    assert g.launch == (4, 16)
    base = gjp.forward(vol, g, vg.h, path="gather").clone()
    for launch in ((1, 1), (2, 5), (8, 7), (8, 64)):
        g.set_launch(*launch)
        assert g.launch == launch
        for path in ("gather", "prefetch") if launch[0] != 1 else ("gather",):
            try:
                out = gjp.forward(vol, g, vg.h, path=path)
            except gjp.GjpError:
                assert path == "prefetch"          # needs a TMA-aligned volume
                continue
            gjp.stream_status()
            if path == "gather":
                assert torch.equal(out, base), (launch, path)
            else:
                assert ((out - base).abs().max() / base.abs().max()).item() < 1e-6, (launch, path)
    for bad in ((3, 1), (16, 1), (4, 0), (4, 65)):
        with pytest.raises(gjp.GjpError):
            g.set_launch(*bad)


def test_default_view_group_follows_grid_and_scan(gjp):
    """Without set_launch, a launch takes its view group from the grid's
    longest edge and the scan's step between views (16 degrees of rotation
    at 512 voxels per edge, shrinking like the edge squared).  A long, thin
    grid (1024 voxels along x) scanned in 0.5 degree steps gets groups of
    8; that reorders blocks only, so the projections equal those of an
    explicit launch shape bitwise, and the adjoint agrees to float32
    rounding."""
    import math
    rng = np.random.default_rng(13)
    vg = VolumeGeometry.centred((1024, 40, 36))
    angles = [math.radians(0.5 * k) for k in range(20)]
    cg = synth.circular(20, 48, 40, 2000.0, 4000.0, 1.9, angles=angles)
    vol = torch.from_numpy(rng.random(vg.n, dtype=np.float32)).cuda()
    g = gjp.Geometry.from_cone(cg)
    assert g.launch == (4, 16)                  # the reported setting until set_launch
    auto = gjp.forward(vol, g, vg.h)
    back_auto = gjp.adjoint(auto, g, vg.n, vg.h)
    gjp.stream_status()
    for launch in ((4, 16), (4, 8), (4, 1)):
        g.set_launch(*launch)
        assert torch.equal(gjp.forward(vol, g, vg.h), auto), launch
        back = gjp.adjoint(auto, g, vg.n, vg.h)
        assert ((back - back_auto).abs().max() / back_auto.abs().max()).item() < 1e-6, launch


def test_adjoint_accumulate(gjp):
    rng = np.random.default_rng(5)
    vg = VolumeGeometry.centred((20, 18, 16))
    cg = synth.random_geometry(rng, vg, 2, 19, 17)
    y = rng.random((cg.n_views, cg.nv, cg.nu)).astype(np.float32)
    base = rng.random(vg.n).astype(np.float32)
    a = _adjoint_gpu(gjp, y, vg, cg)
    b = _adjoint_gpu(gjp, y, vg, cg, accumulate_into=base)
    np.testing.assert_allclose(b, a + base, rtol=1e-5, atol=1e-5 * np.abs(a).max())


def test_dot_test_differentiation_workload(gjp):
    """<A x, y> = <x, A^T y> on the 256^3 / 180-view / 256^2 workload with
    seeded Gaussian x and y.  The dot product is a sum of random-sign terms,
    so its float32 error is measured against S = sqrt(sum_r (Ax)_r^2 y_r^2),
    the natural scale of that sum; with positive (uniform) x, y there is no
    cancellation and the plain relative error is used."""
    vg, cg = synth.c4_geometry()
    g = gjp.Geometry.from_cone(cg)
    gen = torch.Generator(device="cuda")
    for kind in ("gauss", "uniform"):
        gen.manual_seed(1)
        if kind == "gauss":
            x = torch.randn(vg.n, device="cuda", generator=gen)
            y = torch.randn(cg.n_views, cg.nv, cg.nu, device="cuda", generator=gen)
        else:
            x = torch.rand(vg.n, device="cuda", generator=gen)
            y = torch.rand(cg.n_views, cg.nv, cg.nu, device="cuda", generator=gen)
        ax = gjp.forward(x, g, voxel_size=vg.h)
        aty = gjp.adjoint(y, g, vg.n, voxel_size=vg.h)
        lhs = torch.sum(ax.double() * y.double()).item()
        rhs = torch.sum(x.double() * aty.double()).item()
        if kind == "gauss":
            scale = torch.sqrt(torch.sum((ax.double() * y.double()) ** 2)).item()
        else:
            scale = abs(lhs)
        assert abs(lhs - rhs) <= 1e-5 * scale, (kind, lhs, rhs, scale)


def test_adjoint_rows_along_minus_z_full_size(gjp):
    """Detector rows along -z on the 256^3 / 180-view / 256^2 workload: each
    warp's z indices fall lane by lane, so the combined adjoint walks its
    runs against the lane order.  It must agree with the tap-by-tap scatter
    (the same transpose, summed in another order) and pass the dot test."""
    vg, cg = synth.c4_geometry()
    cg.det_origin = cg.det_origin + (cg.nv - 1) * cg.det_v
    cg.det_v = -cg.det_v
    g = gjp.Geometry.from_cone(cg)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    x = torch.rand(vg.n, device="cuda", generator=gen)
    y = torch.rand(cg.n_views, cg.nv, cg.nu, device="cuda", generator=gen)
    aty = gjp.adjoint(y, g, vg.n, voxel_size=vg.h, path="combine")
    ref = gjp.adjoint(y, g, vg.n, voxel_size=vg.h, path="gather")
    gjp.stream_status()
    assert ((aty - ref).abs().max() / ref.abs().max()).item() < 1e-5
    ax = gjp.forward(x, g, voxel_size=vg.h)
    lhs = torch.sum(ax.double() * y.double()).item()
    rhs = torch.sum(x.double() * aty.double()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_gradient_finite_differences_differentiation_workload(gjp):
    """L(x) = 1/2 |A x - b|^2 is quadratic, so central differences equal
    (A e_j)^T (A x - b) exactly; compare with the adjoint's A^T (A x - b) on
    64 seeded voxels of the 256^3 workload.  Both sides are float32 sums of
    ~10^3 signed terms, so the error is measured against the sum of the
    terms' magnitudes, (A^T |A x - b|)_j, not against the (possibly
    cancelling) gradient value."""
    vg, cg = synth.c4_geometry()
    g = gjp.Geometry.from_cone(cg)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2)
    x = torch.randn(vg.n, device="cuda", generator=gen)
    b = torch.randn(cg.n_views, cg.nv, cg.nu, device="cuda", generator=gen)
    res = gjp.forward(x, g, voxel_size=vg.h) - b
    grad = gjp.adjoint(res, g, vg.n, voxel_size=vg.h)
    mag = gjp.adjoint(res.abs(), g, vg.n, voxel_size=vg.h)
    rng = np.random.default_rng(2)
    # voxels inside the inscribed cylinder (seen by every view)
    picks = []
    while len(picks) < 64:
        i, j, k = rng.integers(32, 224, size=3)
        if (i - 127.5) ** 2 + (j - 127.5) ** 2 < 90 ** 2:
            picks.append((int(i), int(j), int(k)))
    eps = 1.0
    for (i, j, k) in picks:
        xp = x.clone(); xp[i, j, k] += eps
        xm = x.clone(); xm[i, j, k] -= eps
        rp = gjp.forward(xp, g, voxel_size=vg.h).double() - b.double()
        rm = gjp.forward(xm, g, voxel_size=vg.h).double() - b.double()
        fd = (0.5 * (rp ** 2).sum() - 0.5 * (rm ** 2).sum()).item() / (2 * eps)
        gv = grad[i, j, k].item()
        scale = mag[i, j, k].item()
        assert scale > 0
        assert abs(fd - gv) <= 1e-5 * scale, (i, j, k, fd, gv, scale)


# --- full-size workload (512^3, 360 views, 512^2), sampled outputs -----------

@pytest.mark.parametrize("path", ["gather", "slab", "prefetch"])
@pytest.mark.parametrize("content", ["phantom", "random"])
def test_c2_full_size_sampled(gjp, content, path):
    vg, cg = synth.c2_geometry()
    vol = synth.voxelize(vg, supersample=2) if content == "phantom" else synth.random_field(vg.n, seed=0)
    gpu, _ = _project(gjp, vol, vg, cg, path=path)
    # one whole view (45 degrees: contains driving-axis ties) plus 4000 random rays
    v45 = 45
    views = np.full(cg.nu * cg.nv, v45)
    iv, iu = np.meshgrid(np.arange(cg.nv), np.arange(cg.nu), indexing="ij")
    sv, su, sw = parity.sampled_rays(cg, 4000, seed=9)
    views = np.concatenate([views, sv]); ius = np.concatenate([iu.ravel(), su])
    ivs = np.concatenate([iv.ravel(), sw])
    ref = oracle.rays(vol, vg, cg, views, ius, ivs)
    parity.check_rays(gpu[views, ivs, ius], vol, vg, cg, views, ius, ivs, np.abs(ref).max(), TOL32, ref=ref)


def test_adjoint_full_size_against_oracle(gjp):
    """The 512^3 / 512^2 adjoint (combined family: row table, run form) of
    two whole views against the oracle's transpose of the same projections.
    Views 10 and 100 hold no driving-axis ties (their rays run within 20
    degrees of an axis), so every ray's taps are the oracle's."""
    vg, cg = synth.c2_geometry()
    sub = cg.subset([10, 100])
    g = gjp.Geometry.from_cone(sub)
    vol = synth.random_field(vg.n, seed=0)
    y = gjp.forward(torch.from_numpy(vol).cuda(), g, vg.h)
    back = gjp.adjoint(y, g, vg.n, vg.h).cpu().numpy()
    gjp.stream_status()
    ref = oracle.adjoint(y.cpu().numpy().astype(np.float64), vg, sub, max_bytes=16e9)
    err = np.abs(back - ref)
    scale = np.abs(ref).max()
    assert scale > 0
    assert err.max() <= TOL32 * scale, err.max() / scale


def test_exact_driving_axis_ties(gjp):
    """Rays with |r_x| == |r_y| exactly (reading C2: ties go to the lowest
    axis; either axis is accepted where float32 could see a near-tie)."""
    vg = VolumeGeometry.centred((16, 16, 16))
    src, org, du, dv = [], [], [], []
    for q in range(4):          # four exact quarter turns of one diagonal view
        rot = np.array([[[1, 0], [0, 1]], [[0, -1], [1, 0]], [[-1, 0], [0, -1]], [[0, 1], [-1, 0]]][q], dtype=float)
        def rz(x):
            return np.array([*(rot @ np.array(x[:2])), x[2]])
        src.append(rz([300.0, 300.0, 0.25]))
        du.append(rz([-1.0, 1.0, 0.0]))
        dv.append(rz([0.0, 0.0, 1.0]))
        org.append(rz([-300.0, -300.0, 0.0]) - 2.0 * du[-1] - 1.5 * dv[-1])
    cg = ConeGeometry(np.array(src), np.array(org), np.array(du), np.array(dv), 5, 4)
    vol = np.random.default_rng(3).random(vg.n, dtype=np.float32)
    r = _full_check(gjp, vol, vg, cg)
    assert r["ties"] >= 4 * 4        # the centre column of every view is an exact tie


# --- edge cases ----------------------------------------------------------------

def test_tiny_and_degenerate_grids(gjp):
    rng = np.random.default_rng(8)
    for shape in [(1, 1, 1), (2, 1, 3), (1, 5, 1), (3, 3, 1)]:
        vg = VolumeGeometry.centred(shape, h=(1.0, 1.5, 0.7))
        cg = synth.random_geometry(rng, VolumeGeometry.centred((8, 8, 8)), 3, 3, 2)
        vol = rng.random(shape, dtype=np.float32) + 0.5
        _full_check(gjp, vol, vg, cg)


def test_rays_missing_the_volume_are_exactly_zero(gjp):
    vg = VolumeGeometry.centred((16, 16, 16))
    cg = synth.circular(2, 64, 48, 60.0, 120.0, 3.0)     # panel much larger than the shadow
    vol = np.ones(vg.n, dtype=np.float32)
    gpu, _ = _project(gjp, vol, vg, cg)
    ref = oracle.forward(vol, vg, cg)
    assert (gpu[ref == 0.0] == 0.0).all() and (ref == 0.0).sum() > 1000
    _full_check(gjp, vol, vg, cg)


def test_axis_aligned_ray_column_sum(gjp):
    vg = VolumeGeometry.centred((12, 10, 8), h=(0.5, 1.0, 2.0))
    vol = np.random.default_rng(1).random(vg.n, dtype=np.float32)
    idx = np.array([0, 4, 5])
    centre = np.array(vg.origin) + idx * np.array(vg.h)
    src = (centre - [100.0, 0, 0])[None]
    cg = ConeGeometry(src, (centre + [100.0, 0, 0])[None], np.array([[0, 0, 1e-2]]),
                      np.array([[0, 1e-2, 0]]), 1, 1)
    gpu, _ = _project(gjp, vol, vg, cg)
    want = vg.h[0] * vol[:, 4, 5].astype(np.float64).sum()
    assert gpu[0, 0, 0] == pytest.approx(want, rel=2e-6)


def test_source_inside_volume_is_rejected(gjp):
    vg = VolumeGeometry.centred((300, 300, 300))
    cg = synth.circular(2, 8, 8, 100.0, 200.0, 1.0)
    vol = torch.zeros(vg.n, device="cuda")
    g = gjp.Geometry.from_cone(cg)
    with pytest.raises(gjp.GjpError) as e:
        gjp.forward(vol, g)
    assert e.value.status == 1


def test_repeated_calls_reuse_table_and_are_deterministic(gjp):
    vg, cg = synth.c1_geometry()
    vol = torch.from_numpy(synth.random_field(vg.n, seed=4)).cuda()
    g = gjp.Geometry.from_cone(cg)
    a = gjp.forward(vol, g).clone()
    b = gjp.forward(vol, g)
    assert torch.equal(a, b)
    # a different grid on the same geometry builds a second table
    c = gjp.forward(vol, g, voxel_size=(0.5, 0.5, 0.5))
    assert not torch.equal(a, c)


def test_int64_indexing_beyond_2_pow_31_elements(gjp):
    """Maximum-size path: a bfloat16 volume with more than 2^31 voxels uses
    64-bit offsets; sampled rays against the oracle."""
    free, _ = torch.cuda.mem_get_info()
    try:
        import os
        host_gb = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") / 2 ** 30
    except (ValueError, OSError):
        host_gb = 0
    if free < 12 * 2 ** 30 or host_gb < 48:
        pytest.skip("needs ~12 GB device and ~48 GB host memory")
    n = (1300, 1300, 1300)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    vol = torch.rand(n, device="cuda", generator=gen).to(torch.bfloat16)
    assert vol.numel() > 2 ** 31
    vg = VolumeGeometry.centred(n)
    cg = synth.cone_angle_geometry(1300, 96, 3, 10.0)
    g = gjp.Geometry.from_cone(cg)
    out = gjp.forward(vol, g).cpu().numpy().astype(np.float64)
    stored = vol.float().cpu().numpy()
    del vol
    views, ius, ivs = parity.sampled_rays(cg, 300, seed=12)
    ref = oracle.rays(stored, vg, cg, views, ius, ivs)
    parity.check_rays(out[views, ivs, ius], stored, vg, cg, views, ius, ivs, np.abs(ref).max(), TOL32,
                      ref=ref)


def test_slab_and_gather_agree_on_bf16_full_size(gjp):
    """Both kernel families on the 512^3 / 360-view workload with bfloat16
    storage: identical samples and weights; they differ only in the float32
    summation order (the gather family sums in two levels), so they agree
    within the float32 parity bound."""
    vg, cg = synth.c2_geometry()
    vol = torch.from_numpy(synth.random_field(vg.n, seed=5)).cuda().to(torch.bfloat16)
    g = gjp.Geometry.from_cone(cg)
    a = gjp.forward(vol, g, path="gather")
    b = gjp.forward(vol, g, path="slab")
    gjp.stream_status()
    assert ((a - b).abs().max() / a.abs().max()).item() < 1e-5


def test_slab_unsupported_for_unaligned_rows(gjp):
    vg = VolumeGeometry.centred((16, 16, 15))          # 15 floats per z row: not a TMA stride
    cg = synth.circular(2, 8, 8, 100.0, 200.0, 1.0)
    g = gjp.Geometry.from_cone(cg)
    vol = torch.zeros(vg.n, device="cuda")
    with pytest.raises(gjp.GjpError) as e:
        gjp.forward(vol, g, path="slab")
    assert e.value.status == 2
    gjp.forward(vol, g, path="auto")                  # falls back to the gather family


# --- w_spl weights (Eq. 14) -----------------------------------------------------

@pytest.mark.parametrize("case", ["c1_phantom", "random_steep"])
def test_spline_weight_forward_matches_oracle(gjp, case):
    if case == "c1_phantom":
        vg, cg = synth.c1_geometry()
        vol = synth.voxelize(vg, supersample=2)
    else:
        rng = np.random.default_rng(71)
        vg = VolumeGeometry.centred((37, 29, 23), h=(0.8, 1.1, 1.3))
        cg = synth.random_geometry(rng, vg, 5, 45, 37, steep=True)
        vol = rng.random(vg.n, dtype=np.float32)
    g = gjp.Geometry.from_cone(cg, weight="spl")
    out = gjp.forward(torch.from_numpy(vol).cuda(), g, vg.h, vg.origin)
    gjp.stream_status()
    gpu = out.cpu().numpy().astype(np.float64)
    ref = oracle.forward(vol, vg, cg, wfun=1)
    views, ius, ivs = parity.all_rays(cg)
    parity.check_rays(gpu[views, ivs, ius], vol, vg, cg, views, ius, ivs, np.abs(ref).max(), TOL32,
                      ref=ref[views, ivs, ius])
    lin = oracle.forward(vol, vg, cg, wfun=0)
    assert np.abs(ref - lin).max() > 1e-3 * np.abs(ref).max()   # the two weights differ


def test_spline_weight_adjoint_matches_oracle(gjp):
    rng = np.random.default_rng(72)
    vg = VolumeGeometry.centred((40, 36, 32), h=(1.0, 0.9, 1.1))
    cg = synth.cone_angle_geometry(40, 36, 5, 10.0)
    y = rng.standard_normal((cg.n_views, cg.nv, cg.nu)).astype(np.float32)
    g = gjp.Geometry.from_cone(cg, weight="spl")
    out = gjp.adjoint(torch.from_numpy(y).cuda(), g, vg.n, vg.h, vg.origin)
    gjp.stream_status()
    ref = oracle.adjoint(y.astype(np.float64), vg, cg, wfun=1)
    assert np.abs(out.cpu().numpy() - ref).max() <= TOL32 * np.abs(ref).max()
    for path in ("slab",):
        with pytest.raises(gjp.GjpError):
            gjp.adjoint(torch.from_numpy(y).cuda(), g, vg.n, vg.h, vg.origin, path=path)
    with pytest.raises(gjp.GjpError):
        gjp.forward(torch.zeros(vg.n, device="cuda"), g, vg.h, vg.origin, path="slab")


# --- texture families (texture memory and GJP_hwlin of the speed section) ----------

def _tex_case(case):
    rng = np.random.default_rng(500 + len(case))
    if case == "c1_phantom":
        vg, cg = synth.c1_geometry()
        return synth.voxelize(vg, supersample=2), vg, cg
    if case == "random_steep":                       # includes z-driven rays (global-memory march)
        vg = VolumeGeometry.centred((37, 29, 23), h=(0.8, 1.1, 1.3))
        return rng.random(vg.n, dtype=np.float32), vg, synth.random_geometry(rng, vg, 5, 45, 37, steep=True)
    vg = VolumeGeometry((40, 36, 33), (1.0, 1.0, 1.0), (-17.0, -20.5, -15.0))
    return rng.random(vg.n, dtype=np.float32), vg, synth.circular(5, 37, 45, 120.0, 240.0, 1.6,
                                                                    angles=[0.2, 1.1, 2.5, 3.9, 5.6])


@pytest.mark.parametrize("case", ["c1_phantom", "random_steep", "off_centre_ragged"])
@pytest.mark.parametrize("dt", ["float32", "float16"])
def test_texture_gather_family_matches_oracle(gjp, case, dt):
    """GJP_PATH_TEXTURE (one tld4 per sample, exact float32 weights) against
    the oracle on the stored values, every ray."""
    vol, vg, cg = _tex_case(case)
    stored = torch.from_numpy(vol).to(getattr(torch, dt)).float().numpy()
    gpu, _ = _project(gjp, vol, vg, cg, dtype=getattr(torch, dt), path="texture")
    ref = oracle.forward(stored, vg, cg)
    views, ius, ivs = parity.all_rays(cg)
    parity.check_rays(gpu[views, ivs, ius], stored, vg, cg, views, ius, ivs, np.abs(ref).max(), TOL32,
                      ref=ref[views, ivs, ius])


def test_texture_gather_spline_weight(gjp):
    vol, vg, cg = _tex_case("off_centre_ragged")
    g = gjp.Geometry.from_cone(cg, weight="spl")
    out = gjp.forward(torch.from_numpy(vol).cuda(), g, vg.h, vg.origin, path="texture")
    gjp.stream_status()
    ref = oracle.forward(vol, vg, cg, wfun=1)
    assert np.abs(out.cpu().numpy() - ref).max() <= TOL32 * np.abs(ref).max()


@pytest.mark.parametrize("content", ["phantom", "random"])
def test_texture_gather_full_size_sampled(gjp, content):
    vg, cg = synth.c2_geometry()
    vol = synth.voxelize(vg, supersample=1) if content == "phantom" else synth.random_field(vg.n, seed=3)
    gpu, _ = _project(gjp, vol, vg, cg, path="texture")
    rays = parity.sampled_rays(cg, 400, seed=11)
    ref = oracle.rays(vol, vg, cg, *rays)
    parity.check_rays(gpu[rays[0], rays[2], rays[1]], vol, vg, cg, *rays, np.abs(ref).max(), TOL32, ref=ref)


def test_texture_arrays_follow_volume_contents(gjp):
    """The cached texture arrays are refilled on every call: a second
    volume of the same grid projects to its own gather result."""
    rng = np.random.default_rng(7)
    vg = VolumeGeometry.centred((40, 36, 33))
    cg = synth.cone_angle_geometry(40, 37, 4, 10.0)
    g = gjp.Geometry.from_cone(cg)
    for _ in range(2):
        vol = torch.from_numpy(rng.random(vg.n, dtype=np.float32)).cuda()
        a = gjp.forward(vol, g, vg.h, path="texture")
        b = gjp.forward(vol, g, vg.h, path="gather")
        gjp.stream_status()
        assert ((a - b).abs().max() / b.abs().max()).item() < 1e-6


@pytest.mark.parametrize("case", ["c1_phantom", "off_centre_ragged"])
def test_hwlin_error_against_oracle(gjp, case):
    """GJP_hwlin: one hardware-filtered fetch per sample.  The filter's
    1/256 weight steps bound each sample's interpolation error by
    2^-9 (|dv_a| + |dv_b|) (plus float32 coordinates, far smaller), so the
    projection error stays well below 5e-3 of the maximum on these smooth
    and random volumes -- but, unlike every exact family, above 1e-6."""
    vol, vg, cg = _tex_case(case)
    gpu, _ = _project(gjp, vol, vg, cg, path="hwlin")
    ref = oracle.forward(vol, vg, cg)
    err = np.abs(gpu - ref).max() / np.abs(ref).max()
    assert 1e-6 < err < 5e-3, err


def test_texture_families_reject_what_they_cannot_do(gjp):
    vg = VolumeGeometry.centred((16, 16, 16))
    cg = synth.circular(2, 8, 8, 100.0, 200.0, 1.0)
    g = gjp.Geometry.from_cone(cg)
    for path in ("texture", "hwlin"):
        with pytest.raises(gjp.GjpError) as e:
            gjp.forward(torch.zeros(vg.n, device="cuda", dtype=torch.bfloat16), g, vg.h, path=path)
        assert e.value.status == 2
    gs = gjp.Geometry.from_cone(cg, weight="spl")
    with pytest.raises(gjp.GjpError):
        gjp.forward(torch.zeros(vg.n, device="cuda"), gs, vg.h, path="hwlin")
    y = torch.zeros(g.proj_shape, device="cuda")
    for path in ("texture", "hwlin"):
        with pytest.raises(gjp.GjpError):
            gjp.adjoint(y, g, vg.n, vg.h, path=path)


# --- field-of-view cylinder (the speed section's ray-cylinder sampling range) ----

def _fov_case():
    rng = np.random.default_rng(84)
    vg = VolumeGeometry.centred((40, 36, 24), h=(1.0, 1.1, 0.9))
    radius = 16.0
    x = (np.arange(vg.n[0]) - 0.5 * (vg.n[0] - 1)) * vg.h[0]
    y = (np.arange(vg.n[1]) - 0.5 * (vg.n[1] - 1)) * vg.h[1]
    mask = (x[:, None] ** 2 + y[None, :] ** 2 <= (radius - 2.5) ** 2)[:, :, None]
    vol = (rng.random(vg.n) * mask).astype(np.float32)
    cg = synth.circular(6, 47, 30, 90.0, 180.0, 1.3, angles=[0.05, 0.8, 1.57, 2.4, 3.9, 5.5])
    return vol, vg, cg, radius


@pytest.mark.parametrize("path", ["gather", "texture", "prefetch", "slab"])
def test_fov_clipped_forward_matches_oracle(gjp, path):
    """Rays clipped to the field-of-view cylinder: on a volume that is zero
    near and outside the cylinder wall the clipped projection equals the
    oracle's clipped projection and the unclipped one."""
    vol, vg, cg, radius = _fov_case()
    g = gjp.Geometry.from_cone(cg)
    g.set_fov(radius)
    try:
        out = gjp.forward(torch.from_numpy(vol).cuda(), g, vg.h, path=path)
    except gjp.GjpError as e:
        assert path in ("prefetch", "slab") and e.status == 2   # needs TMA-aligned rows
        pytest.skip("volume rows not TMA-aligned")
    gjp.stream_status()
    gpu = out.cpu().numpy().astype(np.float64)
    ref = oracle.forward(vol, vg, cg, fov=radius)
    assert np.abs(gpu - ref).max() <= TOL32 * np.abs(ref).max()
    full = oracle.forward(vol, vg, cg)
    assert np.abs(full - ref).max() <= 1e-12 * np.abs(full).max()


@pytest.mark.parametrize("path", ["combine", "gather", "slab"])
def test_fov_clipped_adjoint_matches_oracle(gjp, path):
    """The adjoint skips the same samples: against the oracle's clipped
    transpose with projections that are non-zero on every ray (so clipped
    samples would show)."""
    vol, vg, cg, radius = _fov_case()
    vg2 = VolumeGeometry.centred((40, 36, 32), h=vg.h)          # z rows of 32 floats: slab-aligned
    rng = np.random.default_rng(85)
    y = rng.standard_normal((cg.n_views, cg.nv, cg.nu)).astype(np.float32)
    g = gjp.Geometry.from_cone(cg)
    g.set_fov(radius)
    out = gjp.adjoint(torch.from_numpy(y).cuda(), g, vg2.n, vg2.h, path=path)
    gjp.stream_status()
    ref = oracle.adjoint(y.astype(np.float64), vg2, cg, fov=radius)
    assert np.abs(out.cpu().numpy() - ref).max() <= TOL32 * np.abs(ref).max()
    unclipped = oracle.adjoint(y.astype(np.float64), vg2, cg)
    assert np.abs(unclipped - ref).max() > 1e-2 * np.abs(ref).max()     # the clip matters here


def test_fov_phantom_full_size(gjp):
    """512^3 Shepp-Logan-shaped phantom (support within 0.93 of the half
    width) with rays clipped to a 250-voxel cylinder, the speed section's
    setting: same projections as without clipping, and sampled rays agree
    with the oracle's clipped rays."""
    vg, cg = synth.c2_geometry()
    vol = synth.voxelize(vg, supersample=1)
    d = torch.from_numpy(vol).cuda()
    g = gjp.Geometry.from_cone(cg)
    full = gjp.forward(d, g, vg.h)
    g.set_fov(250.0)
    clipped = gjp.forward(d, g, vg.h)
    gjp.stream_status()
    assert ((clipped - full).abs().max() / full.abs().max()).item() < 1e-6
    rays = parity.sampled_rays(cg, 300, seed=21)
    ref = oracle.rays(vol, vg, cg, *rays, fov=250.0)
    got = clipped.cpu().numpy()[rays[0], rays[2], rays[1]].astype(np.float64)
    assert np.abs(got - ref).max() <= TOL32 * np.abs(ref).max()


def test_fov_argument_checks(gjp):
    g = gjp.Geometry.from_cone(synth.circular(2, 8, 8, 100.0, 200.0, 1.0))
    for bad in (-1.0, float("inf"), float("nan")):
        with pytest.raises(gjp.GjpError):
            g.set_fov(bad)
    g.set_fov(0.0)


def test_bounded_wait_times_out_and_is_reported(gjp):
    """Failure detection without a fault: a kernel waits, through the
    library's bounded wait, on a barrier phase that nothing completes.  The
    wait gives up after its limit, gjp_stream_status reports
    GJP_ERR_TIMEOUT once (the flag is then cleared), and the context keeps
    working."""
    import time
    from paper_1609_00958_gb300 import _capi
    stream = torch.cuda.current_stream().cuda_stream
    gjp.stream_status()                                 # nothing pending
    t0 = time.perf_counter()
    assert _capi.gjp_selftest_wait_timeout(stream) == _capi.GJP_OK
    assert _capi.gjp_stream_status(stream) == _capi.GJP_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    assert _capi.gjp_stream_status(stream) == _capi.GJP_OK
    vg, cg = synth.c1_geometry()
    vol = synth.voxelize(vg, supersample=2)
    out = gjp.forward(torch.from_numpy(vol).cuda(), gjp.Geometry.from_cone(cg.subset([0, 9])), vg.h)
    gjp.stream_status()
    ref = oracle.forward(vol, vg, cg.subset([0, 9]))
    assert np.abs(out.cpu().numpy() - ref).max() <= TOL32 * np.abs(ref).max()


def test_adjoint_and_batch_with_64bit_offsets(gjp):
    """Volumes of more than 2^31 voxels take the 64-bit-offset kernels: the
    adjoint (both families) passes the dot test against the forward, the
    two families agree, and a batch that holds such a problem equals its
    separate projection bit for bit."""
    free, _ = torch.cuda.mem_get_info()
    if free < 40 * 2 ** 30:
        pytest.skip("needs ~40 GB of device memory")
    n = (1300, 1300, 1300)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(13)
    x = torch.rand(n, device="cuda", generator=gen)
    assert x.numel() > 2 ** 31
    cg = synth.cone_angle_geometry(1300, 96, 3, 10.0)
    g = gjp.Geometry.from_cone(cg)
    y = torch.rand(g.proj_shape, device="cuda", generator=gen)
    ax = gjp.forward(x, g)
    lhs = torch.sum(ax.double() * y.double()).item()
    aty = gjp.adjoint(y, g, n, path="combine")
    rhs = torch.sum(x.double() * aty.double()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    other = gjp.adjoint(y, g, n, path="gather")
    gjp.stream_status()
    assert ((aty - other).abs().max() / aty.abs().max()).item() < 1e-5
    del aty, other
    x16 = x.to(torch.bfloat16)
    del x
    small_vg = VolumeGeometry.centred((40, 36, 33))
    small = torch.rand(small_vg.n, device="cuda", generator=gen)
    gs = gjp.Geometry.from_cone(synth.cone_angle_geometry(40, 37, 4, 10.0))
    items = [(x16, g, (1.0, 1.0, 1.0), None, torch.empty(g.proj_shape, device="cuda")),
             (small, gs, small_vg.h, None, torch.empty(gs.proj_shape, device="cuda"))]
    gjp.Batch(items).forward()
    gjp.stream_status()
    for vol, geom, h, origin, out in items:
        assert torch.equal(out, gjp.forward(vol, geom, h, origin))


# --- warps sharing one row: the shared row-table march ----------------------

def _row_case(case):
    """Circular orbits about z, where the 32 rays of a detector column share
    their x/y row.  Every detector has a multiple of 32 rows (full warps)."""
    angles = [0.03, 0.7, 1.5708, 2.3, 3.2, 3.9, 4.75, 5.6]
    if case == "rays_missing":          # detector much taller than the volume: lanes without interior
        vg = VolumeGeometry.centred((40, 36, 24), h=(1.0, 1.1, 0.9))
        cg = synth.circular(8, 37, 64, 60.0, 120.0, 1.5, angles=angles, det_shift_v=0.3)
    elif case == "steep_odd":           # close source: lanes leave through z at different planes
        vg = VolumeGeometry.centred((45, 45, 45))
        cg = synth.circular(8, 29, 32, 50.0, 100.0, 2.8, angles=angles, z_shift=1.7)
    elif case == "short_axis":          # fewer planes than one 16-plane block
        vg = VolumeGeometry.centred((9, 7, 40))
        cg = synth.circular(8, 13, 32, 40.0, 80.0, 2.5, angles=angles)
    else:                               # "long": several 32-plane windows and a ragged last one
        vg = VolumeGeometry.centred((70, 66, 20), h=(0.7, 0.8, 1.2))
        cg = synth.circular(8, 21, 32, 90.0, 180.0, 1.1, angles=angles, det_shift_v=-0.4)
    return vg, cg


@pytest.mark.parametrize("case", ["rays_missing", "steep_odd", "short_axis", "long"])
@pytest.mark.parametrize("weight", ["lin", "spl"])
def test_shared_row_warps_match_oracle(gjp, case, weight):
    """Full warps on one row march from the warp's row table: all rays
    against the oracle, under every launch shape."""
    vg, cg = _row_case(case)
    vol = synth.random_field(vg.n, seed=71)
    wfun = 1 if weight == "spl" else 0
    ref = oracle.forward(vol, vg, cg, wfun=wfun)
    views, ius, ivs = parity.all_rays(cg)
    for launch in [(4, 8), (1, 1), (2, 3)]:
        g = gjp.Geometry.from_cone(cg, weight=weight)
        g.set_launch(*launch)
        out = gjp.forward(torch.from_numpy(vol).cuda(), g, vg.h, path="gather")
        gjp.stream_status()
        gpu = out.cpu().numpy().astype(np.float64)
        parity.check_rays(gpu[views, ivs, ius], vol, vg, cg, views, ius, ivs, np.abs(ref).max(), TOL32,
                          ref=ref[views, ivs, ius])


@pytest.mark.parametrize("dt", ["bfloat16", "float16"])
def test_shared_row_warps_16bit_and_fov(gjp, dt):
    """16-bit storage on the row-table march, unclipped and clipped to a
    field-of-view cylinder (on a volume that is zero near and outside the
    cylinder wall, so float32 and FP64 clipping decisions cannot differ on
    a non-zero sample)."""
    vg, cg = _row_case("steep_odd")
    radius = 17.5
    x = (np.arange(vg.n[0]) - 0.5 * (vg.n[0] - 1)) * vg.h[0]
    y = (np.arange(vg.n[1]) - 0.5 * (vg.n[1] - 1)) * vg.h[1]
    mask = (x[:, None] ** 2 + y[None, :] ** 2 <= (radius - 2.5) ** 2)[:, :, None]
    vol = (synth.random_field(vg.n, seed=72) * mask).astype(np.float32)
    xt = torch.from_numpy(vol).cuda().to(getattr(torch, dt))
    stored = xt.float().cpu().numpy()
    views, ius, ivs = parity.all_rays(cg)
    for fov in (0.0, radius):
        g = gjp.Geometry.from_cone(cg)
        if fov:
            g.set_fov(fov)
        gpu = gjp.forward(xt, g, vg.h).cpu().numpy().astype(np.float64)
        gjp.stream_status()
        ref = oracle.forward(stored, vg, cg, fov=fov)
        parity.check_rays(gpu[views, ivs, ius], stored, vg, cg, views, ius, ivs, np.abs(ref).max(), TOL32,
                          ref=ref[views, ivs, ius])
