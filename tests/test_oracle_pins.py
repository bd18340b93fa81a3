"""Pins of the FP64 oracle against facts that the paper and mathematics fix
(no GPU).  Each test names the property and the passage it comes from.

A plausible slip in the oracle -- a dropped tap, a swapped floor/ceil, a
transposed axis, a missing step factor, a sign error in the offset o --
breaks at least one of these.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from synth.geometry import ConeGeometry, VolumeGeometry
from tests import joseph_textbook as tb


def _single_ray_geometry(src, pix):
    """A one-pixel detector whose pixel centre is ``pix``."""
    src = np.asarray(src, dtype=np.float64)[None]
    pix = np.asarray(pix, dtype=np.float64)[None]
    du = np.array([[0.0, 0.0, 1e-3]])
    dv = np.array([[0.0, 1e-3, 0.0]])
    return ConeGeometry(src, pix.copy(), du, dv, 1, 1)


def _rng(seed):
    return np.random.default_rng(seed)


# --- Eq. 12: the branchless 4-tap form is 2-D interpolation in the plane
# perpendicular to the driving axis, for every m ----------------------------

@pytest.mark.parametrize("wfun", [0, 1])
@pytest.mark.parametrize("steep", [False, True])
def test_branchless_equals_textbook_joseph(wfun, steep):
    rng = _rng(11 + wfun + 2 * steep)
    vg = VolumeGeometry.centred((7, 9, 11), h=(0.9, 1.1, 0.7))
    vol = rng.standard_normal(vg.n)
    g = synth.random_geometry(rng, vg, 3, 6, 5, steep=steep)
    a = oracle.forward(vol, vg, g, wfun=wfun)
    b = tb.project(vol, vg, g, wfun=wfun)
    m, _, _ = oracle.ray_info(vg, g, *np.nonzero(np.ones((g.n_views, g.nu, g.nv))))
    if steep:
        assert (m == 2).any(), "steep geometry should produce z-driven rays"
    assert np.abs(a).max() > 1.0
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.abs(b).max())


# --- Eq. 7-12 special cases: integer transverse positions give duplicate
# taps with weights 1/0, so an axis-aligned ray through voxel centres is the
# column sum times the voxel size ---------------------------------------------

@pytest.mark.parametrize("axis", [0, 1, 2])
def test_axis_aligned_ray_is_column_sum(axis):
    rng = _rng(3 + axis)
    vg = VolumeGeometry.centred((6, 7, 8), h=(0.5, 1.25, 2.0))
    vol = rng.random(vg.n)
    idx = [3, 4, 5]
    centre = np.array(vg.origin) + np.array(idx) * np.array(vg.h)
    far = np.zeros(3)
    far[axis] = 100.0
    g = _single_ray_geometry(centre - far, centre + far)
    got = oracle.forward(vol, vg, g)[0, 0, 0]
    sl = [idx[0], idx[1], idx[2]]
    sl[axis] = slice(None)
    want = vg.h[axis] * vol[tuple(sl)].sum()
    assert got == pytest.approx(want, rel=1e-14, abs=0)


def _interior_rays(vg, g):
    """Rays whose transverse coordinates stay in [0, n_k - 1] on every plane
    0 .. n_m - 1 (so all four taps exist), evaluated independently here."""
    out = []
    h, o, n = np.array(vg.h), np.array(vg.origin), np.array(vg.n)
    for v in range(g.n_views):
        s = (g.src[v] - o) / h
        for iv in range(g.nv):
            for iu in range(g.nu):
                d = (g.det_origin[v] + iu * g.det_u[v] + iv * g.det_v[v] - o) / h
                r = d - s
                m = int(np.argmax(np.abs(r)))
                ok = True
                for plane in (0, n[m] - 1):
                    p = s + (plane - s[m]) / r[m] * r
                    for k in range(3):
                        if k != m and not (0.0 <= p[k] and math.ceil(p[k]) <= n[k] - 1):
                            ok = False
                if ok:
                    out.append((v, iu, iv, s, d, r, m))
    return out


# --- exact chord length through a constant volume --------------------------

def test_constant_volume_gives_exact_chord_length():
    vg = VolumeGeometry.centred((24, 20, 22), h=(1.0, 0.8, 1.3))
    c = 0.37
    vol = np.full(vg.n, c)
    # sources far away, pixels near the axis through the centre
    rng = _rng(5)
    srcs, pixs = [], []
    centre = np.array(vg.origin) + (np.array(vg.n) - 1) / 2 * np.array(vg.h)
    for _ in range(40):
        d = rng.normal(size=3)
        d[2] *= 0.3
        d /= np.linalg.norm(d)
        srcs.append(centre + 500 * d + rng.normal(size=3) * 0.5)
        pixs.append(centre - 500 * d + rng.normal(size=3) * 0.5)
    g = ConeGeometry(np.array(srcs), np.array(pixs), np.tile([[1e-3, 0, 0]], (40, 1)),
                     np.tile([[0, 1e-3, 0]], (40, 1)), 1, 1)
    rays = _interior_rays(vg, g)
    assert len(rays) > 20
    got = oracle.forward(vol, vg, g)[:, 0, 0]
    for (v, _, _, s, d, r, m) in rays:
        world = (d - s) * np.array(vg.h)
        # chord between the bounding planes p_m = -1/2 and n_m - 1/2
        length = vg.n[m] * vg.h[m] * np.linalg.norm(world) / abs(world[m])
        assert got[v] == pytest.approx(c * length, rel=1e-13)


# --- affine fields are reproduced exactly by bilinear interpolation and
# integrated exactly by the plane-midpoint rule ------------------------------

def test_affine_field_integral_closed_form():
    vg = VolumeGeometry.centred((20, 23, 21), h=(1.1, 0.9, 1.0))
    grad = np.array([0.3, -0.7, 0.45])
    bias = 2.5
    ii, jj, kk = np.meshgrid(*[np.arange(n) for n in vg.n], indexing="ij")
    vol = grad[0] * ii + grad[1] * jj + grad[2] * kk + bias
    rng = _rng(9)
    centre = np.array(vg.origin) + (np.array(vg.n) - 1) / 2 * np.array(vg.h)
    srcs, pixs = [], []
    for _ in range(60):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        srcs.append(centre + 400 * d + rng.normal(size=3) * 0.8)
        pixs.append(centre - 400 * d + rng.normal(size=3) * 0.8)
    g = ConeGeometry(np.array(srcs), np.array(pixs), np.tile([[1e-3, 0, 0]], (60, 1)),
                     np.tile([[0, 1e-3, 0]], (60, 1)), 1, 1)
    rays = _interior_rays(vg, g)
    assert len(rays) > 20
    assert len({m for *_, m in rays}) >= 2
    got = oracle.forward(vol, vg, g)[:, 0, 0]
    for (v, _, _, s, d, r, m) in rays:
        world = (d - s) * np.array(vg.h)
        length = vg.n[m] * vg.h[m] * np.linalg.norm(world) / abs(world[m])
        mid_plane = (vg.n[m] - 1) / 2.0
        mid = s + (mid_plane - s[m]) / r[m] * r          # index coordinates
        want = length * (grad @ mid + bias)
        assert got[v] == pytest.approx(want, rel=1e-12)


# --- system-matrix view g = A f: forward and adjoint are transposes --------

def test_system_matrix_brute_force_transpose():
    rng = _rng(21)
    vg = VolumeGeometry.centred((4, 5, 3), h=(1.0, 1.2, 0.8))
    g = synth.random_geometry(rng, vg, 2, 4, 3, steep=False)
    nvox = int(np.prod(vg.n))
    nray = g.n_views * g.nv * g.nu
    A = np.zeros((nray, nvox))
    for j in range(nvox):
        e = np.zeros(nvox)
        e[j] = 1.0
        A[:, j] = oracle.forward(e.reshape(vg.n), vg, g).reshape(-1)
    At = np.zeros((nvox, nray))
    for i in range(nray):
        e = np.zeros(nray)
        e[i] = 1.0
        At[:, i] = oracle.adjoint(e.reshape(g.n_views, g.nv, g.nu), vg, g, threads=1).reshape(-1)
    assert np.abs(A).max() > 0.1
    np.testing.assert_allclose(At, A.T, rtol=0, atol=1e-14)
    # every non-zero matrix entry is a product of w_lin factors and the step,
    # so a row sum over a constant volume is the chord (>= 0); linearity:
    x, y = rng.random(nvox), rng.random(nvox)
    fx = oracle.forward((2.0 * x - 3.0 * y).reshape(vg.n), vg, g).reshape(-1)
    np.testing.assert_allclose(fx, A @ (2.0 * x - 3.0 * y), rtol=1e-13, atol=1e-13)
    assert (A >= 0).all()


def test_dot_product_adjoint_fp64():
    rng = _rng(33)
    vg = VolumeGeometry.centred((12, 10, 14), h=(1.0, 1.0, 1.0))
    g = synth.random_geometry(rng, vg, 3, 9, 8, steep=True)
    x = rng.standard_normal(vg.n)
    y = rng.standard_normal((g.n_views, g.nv, g.nu))
    lhs = float(np.sum(oracle.forward(x, vg, g) * y))
    rhs = float(np.sum(x * oracle.adjoint(y, vg, g)))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_adjoint_threaded_equals_serial():
    rng = _rng(34)
    vg = VolumeGeometry.centred((10, 9, 8))
    g = synth.random_geometry(rng, vg, 3, 7, 6)
    y = rng.standard_normal((g.n_views, g.nv, g.nu))
    a = oracle.adjoint(y, vg, g, threads=1)
    b = oracle.adjoint(y, vg, g, threads=4)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_quadratic_loss_gradient_matches_central_differences():
    """L(f) = 1/2 |A f - b|^2 is quadratic, so central differences are exact
    up to rounding; grad L = A^T (A f - b)."""
    rng = _rng(44)
    vg = VolumeGeometry.centred((9, 8, 10))
    g = synth.random_geometry(rng, vg, 3, 6, 6)
    f = rng.standard_normal(vg.n)
    b = rng.standard_normal((g.n_views, g.nv, g.nu))

    def loss(v):
        r = oracle.forward(v, vg, g) - b
        return 0.5 * float(np.sum(r * r))

    grad = oracle.adjoint(oracle.forward(f, vg, g) - b, vg, g)
    flat = rng.choice(f.size, size=8, replace=False)
    eps = 1e-2
    for j in flat:
        e = np.zeros(f.size)
        e[j] = eps
        e = e.reshape(vg.n)
        fd = (loss(f + e) - loss(f - e)) / (2 * eps)
        assert fd == pytest.approx(grad.reshape(-1)[j], rel=1e-7, abs=1e-7)


# --- Fig. 1 caption: 1 <= |rt| <= sqrt(3), rt_m = 1 -------------------------

def test_increment_bounds():
    rng = _rng(55)
    vg = VolumeGeometry.centred((16, 16, 16))
    g = synth.random_geometry(rng, vg, 8, 7, 7, steep=True)
    views, ius, ivs = np.meshgrid(np.arange(g.n_views), np.arange(g.nu), np.arange(g.nv), indexing="ij")
    m, rt, margin = oracle.ray_info(vg, g, views.ravel(), ius.ravel(), ivs.ravel())
    norms = np.linalg.norm(rt, axis=1)
    assert (norms >= 1.0).all() and (norms <= math.sqrt(3.0) + 1e-15).all()
    assert np.all(rt[np.arange(len(m)), m] == 1.0)
    assert (margin >= 0).all()


def test_driving_axis_tie_goes_to_lowest_index():
    vg = VolumeGeometry.centred((8, 8, 8))
    g = _single_ray_geometry((-50.0, -50.0, 0.2), (50.0, 50.0, -0.3))  # |r_x| == |r_y|
    m, _, margin = oracle.ray_info(vg, g, [0], [0], [0])
    assert m[0] == 0 and margin[0] == 0.0
    vol = np.random.default_rng(1).random(vg.n)
    a_auto = oracle.rays(vol, vg, g, [0], [0], [0])[0]
    a_x = oracle.rays(vol, vg, g, [0], [0], [0], axis=0)[0]
    a_y = oracle.rays(vol, vg, g, [0], [0], [0], axis=1)[0]
    assert a_auto == a_x
    # both are valid Joseph integrals of the same ray; they differ slightly
    assert a_y == pytest.approx(a_x, rel=0.05)
    assert a_y == pytest.approx(tb.ray(vol, vg.h, vg.origin, g.src[0], g.det_origin[0], force_m=1), rel=1e-13)


def test_ray_missing_the_volume_is_zero():
    vg = VolumeGeometry.centred((8, 8, 8))
    g = _single_ray_geometry((-50.0, 30.0, 0.0), (50.0, 30.0, 0.0))
    vol = np.ones(vg.n)
    assert oracle.forward(vol, vg, g)[0, 0, 0] == 0.0


def test_zero_border_partial_contribution():
    """Reading of "p is in volume": a sample half a voxel outside the grid
    still interpolates with the zero border (weight 1/2 on the edge row)."""
    vg = VolumeGeometry.centred((5, 6, 7))
    vol = np.ones(vg.n)
    y_edge = vg.origin[1] - 0.5 * vg.h[1]   # transverse position -1/2 in index units
    z_mid = vg.origin[2] + 3 * vg.h[2]
    g = _single_ray_geometry((-40.0, y_edge, z_mid), (40.0, y_edge, z_mid))
    got = oracle.forward(vol, vg, g)[0, 0, 0]
    assert got == pytest.approx(0.5 * vg.n[0] * vg.h[0], rel=1e-14)


# --- symmetry: a 90-degree rotation about z maps the grid onto itself ------

def test_quarter_turn_symmetry():
    rng = _rng(66)
    n = 9
    vg = VolumeGeometry.centred((n, n, 6))
    vol = rng.random(vg.n)
    ang = [math.radians(17.0), math.radians(17.0) + math.pi / 2, 0.0, math.pi / 2]
    g = synth.circular(4, 7, 5, 40.0, 80.0, 2.0, angles=ang, det_shift_u=0.3, det_shift_v=-0.2)
    p = oracle.forward(vol, vg, g)
    rot = np.rot90(vol, 1, axes=(0, 1))
    pr = oracle.forward(rot, vg, g)
    np.testing.assert_allclose(pr[1], p[0], rtol=0, atol=1e-12 * np.abs(p).max())
    np.testing.assert_allclose(pr[3], p[2], rtol=0, atol=1e-12 * np.abs(p).max())
    assert np.abs(pr[0] - p[0]).max() > 1e-3   # not trivially equal


# --- analytic ellipsoid line integrals ---------------------------------------

def test_analytic_sphere_chord():
    """Closed form: a ray at distance b from a sphere's centre has chord
    2 sqrt(R^2 - b^2)."""
    ell = np.zeros((1, 16))
    ell[0, 0] = 2.0
    ell[0, 1:4] = (1.0, -2.0, 0.5)
    ell[0, 4:7] = 3.0
    ell[0, 7:16] = np.eye(3).reshape(-1)
    b = 1.7
    g = _single_ray_geometry((1.0 - 50.0, -2.0 + b, 0.5), (1.0 + 50.0, -2.0 + b, 0.5))
    got = oracle.ellipsoid_project(ell, g, sub=1)[0, 0, 0]
    assert got == pytest.approx(2.0 * 2.0 * math.sqrt(9.0 - b * b), rel=1e-13)


def test_voxelised_phantom_projection_converges_to_analytic():
    """Projection-quality experiment (rasterised vs analytic Shepp-Logan
    shaped phantom): the l1 residual ratio shrinks as the grid refines
    with the detector.  The paper prints no values for this metric, so only
    the trend and a loose bound are pinned."""
    errs = []
    for n in (32, 64, 128):
        vg = VolumeGeometry.centred((n, n, n), h=(64.0 / n,) * 3)
        w = 64.0
        pitch = synth.covering_pitch(w, 4 * w, 8 * w, n)
        g = synth.circular(3, n, n, 4 * w, 8 * w, pitch)
        ell = synth.ellipsoids_world(vg)
        vol = synth.voxelize(vg, ell, supersample=2)
        p = oracle.forward(vol, vg, g)
        pa = oracle.ellipsoid_project(ell, g, sub=8)
        errs.append(np.abs(p - pa).sum() / np.abs(pa).sum())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.012


def test_dense_sampling_of_smooth_field():
    """A smooth field sampled on the grid: the GJP line integral agrees with
    dense numerical integration (10^4 points) of the continuous field to
    second order in the voxel size."""
    vg = VolumeGeometry.centred((40, 40, 40), h=(0.5, 0.5, 0.5))
    c = np.array(vg.origin) + (np.array(vg.n) - 1) / 2 * np.array(vg.h)

    def field(x):
        return np.exp(-np.sum((x - c) ** 2, axis=-1) / (2 * 3.0 ** 2))

    idx = np.stack(np.meshgrid(*[np.arange(n) for n in vg.n], indexing="ij"), -1)
    vol = field(np.array(vg.origin) + idx * np.array(vg.h))
    rng = _rng(77)
    g = synth.random_geometry(rng, vg, 3, 4, 4)
    got = oracle.forward(vol, vg, g)
    for v in range(g.n_views):
        for iv in range(g.nv):
            for iu in range(g.nu):
                pix = g.det_origin[v] + iu * g.det_u[v] + iv * g.det_v[v]
                t = (np.arange(10000) + 0.5) / 10000
                pts = g.src[v] + t[:, None] * (pix - g.src[v])
                dense = field(pts).sum() * np.linalg.norm(pix - g.src[v]) / 10000
                assert got[v, iv, iu] == pytest.approx(dense, rel=2e-3, abs=2e-3 * 7.5)


def test_oracle_rejects_bad_arguments():
    vg = VolumeGeometry((0, 4, 4), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    g = _single_ray_geometry((-10, 0, 0), (10, 0, 0))
    with pytest.raises(ValueError):
        oracle.forward(np.zeros((0, 4, 4)), vg, g)


# --- regression fixture ------------------------------------------------------

def test_golden_c1_rays_regression():
    """Values written by tests/golden/make_golden.py (oracle only); guards the
    oracle's arithmetic against silent change."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "c1_rays.txt")
    rows = np.loadtxt(path, comments="#")
    vg, g = synth.c1_geometry()
    ell = synth.ellipsoids_world(vg)
    vol = synth.voxelize(vg, ell, supersample=2)
    views, ius, ivs = rows[:, 0].astype(int), rows[:, 1].astype(int), rows[:, 2].astype(int)
    got = oracle.rays(vol, vg, g, views, ius, ivs)
    np.testing.assert_allclose(got, rows[:, 3], rtol=1e-12, atol=1e-12)
    ana = oracle.ellipsoid_project(ell, g.subset(views), sub=8)[np.arange(len(views)), ivs, ius]
    np.testing.assert_allclose(ana, rows[:, 4], rtol=1e-12, atol=1e-12)
    # discretisation error of GJP_lin vs the analytic integrals stays small
    assert np.abs(got - ana).sum() / np.abs(ana).sum() < 0.03


def test_linear_weights_beat_spline_weights_against_analytic_projections():
    """Projection-quality experiment: the paper finds GJP_lin closer to the
    analytic projections than GJP_spl (qualitative; no values printed)."""
    for n in (64, 128):
        vg = VolumeGeometry.centred((n, n, n), h=(64.0 / n,) * 3)
        w = 64.0
        g = synth.circular(3, n, n, 4 * w, 8 * w, synth.covering_pitch(w, 4 * w, 8 * w, n))
        ell = synth.ellipsoids_world(vg)
        vol = synth.voxelize(vg, ell, supersample=2)
        pa = oracle.ellipsoid_project(ell, g, sub=8)
        e_lin = np.abs(oracle.forward(vol, vg, g, wfun=0) - pa).sum() / np.abs(pa).sum()
        e_spl = np.abs(oracle.forward(vol, vg, g, wfun=1) - pa).sum() / np.abs(pa).sum()
        assert e_lin < e_spl, (n, e_lin, e_spl)


# --- field-of-view cylinder of the speed section: sampling restricted to
# the ray-cylinder intersection instead of the bounding box ------------------

def _cylinder_mask(vg, radius):
    """True where a voxel centre lies within world distance `radius` of the
    axis through the volume centre parallel to z."""
    x = (np.arange(vg.n[0]) - 0.5 * (vg.n[0] - 1)) * vg.h[0]
    y = (np.arange(vg.n[1]) - 0.5 * (vg.n[1] - 1)) * vg.h[1]
    return (x[:, None] ** 2 + y[None, :] ** 2 <= radius ** 2)[:, :, None]


def test_fov_clipping_changes_nothing_inside_the_cylinder():
    """A volume that is zero farther than R - 2 voxels from the axis has no
    non-zero tap at a sample outside radius R (taps reach one voxel along
    each transverse axis), so clipping the rays to the cylinder of radius R
    changes no projection; a cylinder that contains the box changes none
    either, and a small one does change them."""
    rng = _rng(81)
    vg = VolumeGeometry.centred((24, 22, 10), h=(1.0, 1.1, 0.9))
    r = 9.0
    vol = rng.random(vg.n) * _cylinder_mask(vg, r - 2.5)
    g = synth.circular(5, 31, 12, 80.0, 160.0, 1.2, angles=[0.1, 0.9, 1.6, 2.8, 4.4])
    full = oracle.forward(vol, vg, g)
    np.testing.assert_allclose(oracle.forward(vol, vg, g, fov=r), full, rtol=0, atol=1e-12 * np.abs(full).max())
    np.testing.assert_allclose(oracle.forward(vol, vg, g, fov=100.0), full, rtol=0, atol=0)
    assert np.abs(oracle.forward(vol, vg, g, fov=r - 5.0) - full).max() > 1e-2 * np.abs(full).max()


def test_fov_clipped_constant_volume_counts_the_planes_in_the_cylinder():
    """An axis-aligned ray along x through voxel centres of a constant volume
    samples, with clipping, exactly the planes i with h_x |i - c_x| <= R:
    the result is h_x times that count (and the full column without it)."""
    vg = VolumeGeometry.centred((21, 9, 7), h=(0.5, 1.0, 1.0))
    vol = np.ones(vg.n)
    centre = np.array(vg.origin) + np.array([10, 4, 3]) * np.array(vg.h)
    g = _single_ray_geometry(centre - np.array([50.0, 0, 0]), centre + np.array([50.0, 0, 0]))
    for radius in (1.0, 2.26, 3.0, 20.0):
        count = sum(1 for i in range(vg.n[0]) if abs(vg.h[0] * (i - 10)) <= radius)
        got = oracle.forward(vol, vg, g, fov=radius)[0, 0, 0]
        assert got == pytest.approx(vg.h[0] * count, rel=1e-14), radius


def test_fov_clipped_adjoint_is_the_transpose():
    rng = _rng(82)
    vg = VolumeGeometry.centred((12, 11, 9))
    g = synth.random_geometry(rng, vg, 3, 9, 8)
    x = rng.standard_normal(vg.n)
    y = rng.standard_normal((g.n_views, g.nv, g.nu))
    lhs = np.sum(oracle.forward(x, vg, g, fov=4.5) * y)
    rhs = np.sum(x * oracle.adjoint(y, vg, g, fov=4.5))
    assert lhs == pytest.approx(rhs, rel=1e-12)
    assert abs(lhs - np.sum(oracle.forward(x, vg, g) * y)) > 1e-3 * abs(lhs)
