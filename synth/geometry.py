"""Seeded, synthetic cone-beam geometries (input generation only).

A geometry is four ``(n_views, 3)`` float64 arrays in world units:

* ``src``        -- X-ray focal spot of each view,
* ``det_origin`` -- centre of detector pixel ``(iu=0, iv=0)``,
* ``det_u``      -- world displacement for ``iu -> iu + 1``,
* ``det_v``      -- world displacement for ``iv -> iv + 1``,

plus ``nu``/``nv`` (detector columns/rows).  The circular trajectory rotates
about world ``z``, which is parallel to the fastest-varying index of the
``(nx, ny, nz)`` C-contiguous volume (the memory-order rule stated with
Algorithm 1 and in the projection-speed section of the paper).  Nothing in
this module computes a projection; it only places sources and detectors.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class ConeGeometry:
    src: np.ndarray
    det_origin: np.ndarray
    det_u: np.ndarray
    det_v: np.ndarray
    nu: int
    nv: int

    @property
    def n_views(self) -> int:
        return int(self.src.shape[0])

    def subset(self, views) -> "ConeGeometry":
        views = np.asarray(views, dtype=np.int64)
        return ConeGeometry(self.src[views].copy(), self.det_origin[views].copy(),
                            self.det_u[views].copy(), self.det_v[views].copy(),
                            self.nu, self.nv)


@dataclass
class VolumeGeometry:
    """Voxel grid: ``n = (nx, ny, nz)``, voxel size ``h`` and the world
    position of the centre of voxel ``(0, 0, 0)`` (``origin``).  Voxel
    centres sit on integer indices."""
    n: tuple
    h: tuple
    origin: tuple

    @staticmethod
    def centred(n, h=(1.0, 1.0, 1.0)) -> "VolumeGeometry":
        n = tuple(int(v) for v in n)
        h = tuple(float(v) for v in h)
        origin = tuple(-(n[k] - 1) / 2.0 * h[k] for k in range(3))
        return VolumeGeometry(n, h, origin)

    @property
    def extent(self):
        return tuple(self.n[k] * self.h[k] for k in range(3))


def exact_cos_sin(theta: float):
    """cos/sin that are exact at multiples of pi/2 (for symmetry pins)."""
    q = theta / (math.pi / 2.0)
    k = round(q)
    if abs(q - k) < 1e-12:
        return [(1.0, 0.0), (0.0, 1.0), (-1.0, 0.0), (0.0, -1.0)][k % 4]
    return math.cos(theta), math.sin(theta)


def circular(n_views: int, nu: int, nv: int, d_so: float, d_sd: float,
             pitch_u: float, pitch_v: float | None = None, angles=None,
             z_shift: float = 0.0, det_shift_u: float = 0.0,
             det_shift_v: float = 0.0) -> ConeGeometry:
    """Flat-panel circular cone beam about world z.

    View k sits at angle ``angles[k]`` (default ``2*pi*k/n_views``); the
    source is at distance ``d_so`` from the rotation axis and the detector
    centre at ``d_sd - d_so`` on the opposite side.  ``det_u`` is tangential,
    ``det_v`` is ``+z``.  ``det_shift_*`` offsets the panel centre (in
    pixels) to break symmetries in tests."""
    if pitch_v is None:
        pitch_v = pitch_u
    if angles is None:
        angles = [2.0 * math.pi * k / n_views for k in range(n_views)]
    angles = list(angles)
    src = np.zeros((len(angles), 3))
    org = np.zeros((len(angles), 3))
    du = np.zeros((len(angles), 3))
    dv = np.zeros((len(angles), 3))
    for k, th in enumerate(angles):
        c, s = exact_cos_sin(th)
        src[k] = (d_so * c, d_so * s, z_shift)
        centre = np.array((-(d_sd - d_so) * c, -(d_sd - d_so) * s, z_shift))
        eu = np.array((-s, c, 0.0)) * pitch_u
        ev = np.array((0.0, 0.0, 1.0)) * pitch_v
        centre = centre + det_shift_u * eu + det_shift_v * ev
        du[k] = eu
        dv[k] = ev
        org[k] = centre - (nu - 1) / 2.0 * eu - (nv - 1) / 2.0 * ev
    return ConeGeometry(src, org, du, dv, int(nu), int(nv))


def covering_pitch(width: float, d_so: float, d_sd: float, n_det: int) -> float:
    """Detector pitch such that every ray through a ``width``-cube centred
    on the axis lands on an ``n_det``-pixel panel: the larger of the
    horizontal half-width (tangent to the circumscribed cylinder) and the
    vertical half-width (top face corner nearest the source)."""
    r_c = width / math.sqrt(2.0)
    half_h = d_sd * math.tan(math.asin(r_c / d_so))
    half_v = d_sd * (width / 2.0) / (d_so - r_c)
    return 2.0 * max(half_h, half_v) / n_det


def cone_angle_geometry(n: int, n_det: int, n_views: int, half_angle_deg: float,
                        h: float = 1.0, angles=None) -> ConeGeometry:
    """Cone beam whose half-angle subtends the inscribed cylinder (radius
    W/2) of an ``n``-cube: ``d_so = (W/2)/sin(alpha)``, ``d_sd = 2 d_so``,
    square pixels of pitch ``2 d_sd tan(alpha) / n_det``."""
    a = math.radians(half_angle_deg)
    w = n * h
    d_so = (w / 2.0) / math.sin(a)
    d_sd = 2.0 * d_so
    pitch = 2.0 * d_sd * math.tan(a) / n_det
    return circular(n_views, n_det, n_det, d_so, d_sd, pitch, angles=angles)


# --- the named workloads ---------------------------------------------------

def c1_geometry():
    """64^3 voxels (h = 1), source-isocentre 4W, source-detector 8W, 64x64
    detector covering the magnified cube, 32 views over 360 degrees."""
    n = 64
    w = float(n)
    d_so, d_sd = 4.0 * w, 8.0 * w
    pitch = covering_pitch(w, d_so, d_sd, 64)
    return VolumeGeometry.centred((n, n, n)), circular(32, 64, 64, d_so, d_sd, pitch)


def c2_geometry(n_views: int = 360):
    """512^3 voxels, 10 degree cone half-angle on the inscribed cylinder,
    512x512 detector, 360 views over 360 degrees."""
    return VolumeGeometry.centred((512, 512, 512)), cone_angle_geometry(512, 512, n_views, 10.0)


def c3_geometry(n: int):
    """Precision form: 1024^3 / 1024^2 / 720 views and 2048^3 / 2048^2 / 64 views."""
    views = {1024: 720, 2048: 64}[n]
    return VolumeGeometry.centred((n, n, n)), cone_angle_geometry(n, n, views, 10.0)


def c4_geometry():
    """Differentiation form: 256^3, 256^2 detector, 180 views (10 degrees)."""
    return VolumeGeometry.centred((256, 256, 256)), cone_angle_geometry(256, 256, 180, 10.0)


def scaled_c2_geometry(n: int, n_det: int, n_views: int, half_angle_deg: float = 10.0):
    return VolumeGeometry.centred((n, n, n)), cone_angle_geometry(n, n_det, n_views, half_angle_deg)


def random_geometry(rng: np.random.Generator, vg: VolumeGeometry, n_views: int,
                    nu: int, nv: int, steep: bool = False) -> ConeGeometry:
    """Arbitrary (non-circular) cone views around a volume, for tests: the
    source is placed on a sphere of radius 2.5x the volume diagonal, the
    detector faces it through the volume centre with random in-plane
    rotation and tilt.  With ``steep`` the sources are near the poles so
    that some rays are driven by the z axis."""
    ext = np.array(vg.extent)
    centre = np.array(vg.origin) + (np.array(vg.n) - 1) / 2.0 * np.array(vg.h)
    radius = 2.5 * float(np.linalg.norm(ext))
    src = np.zeros((n_views, 3))
    org = np.zeros((n_views, 3))
    du = np.zeros((n_views, 3))
    dv = np.zeros((n_views, 3))
    for k in range(n_views):
        d = rng.normal(size=3)
        if steep:
            d[2] = abs(d[2]) * 4.0 * (1 if rng.random() < 0.5 else -1)
        d /= np.linalg.norm(d)
        s = centre + radius * d
        # orthonormal frame perpendicular to d, randomly rotated
        a = np.cross(d, rng.normal(size=3))
        a /= np.linalg.norm(a)
        b = np.cross(d, a)
        ang = rng.uniform(0, 2 * np.pi)
        eu = math.cos(ang) * a + math.sin(ang) * b
        ev = np.cross(d, eu)
        # slight tilt of the panel
        tilt = rng.uniform(-0.2, 0.2)
        eu = eu + tilt * d
        d_sd = 2.0 * radius
        # pitch so the panel covers the volume's projection (magnification 2)
        pitch_u = 2.2 * float(np.linalg.norm(ext)) / nu
        pitch_v = 2.2 * float(np.linalg.norm(ext)) / nv
        det_c = s - d_sd * d
        src[k] = s
        du[k] = eu * pitch_u
        dv[k] = ev * pitch_v
        org[k] = det_c - (nu - 1) / 2.0 * du[k] - (nv - 1) / 2.0 * dv[k]
    return ConeGeometry(src, org, du, dv, nu, nv)


# --- batching workload ---------------------------------------------------------

@dataclass
class BatchProblemSpec:
    """One problem of the batching workload: a centred volume of ``n``
    voxels (h = 1) stored as ``dtype``, projected on ``views`` views of a
    circular cone beam whose ``half_angle`` (degrees) subtends the inscribed
    cylinder of its in-plane extent, onto a ``det`` x ``det`` detector;
    contents are the phantom or a uniform field from ``seed``."""
    n: tuple
    dtype: str
    half_angle: float
    views: int
    det: int
    content: str
    seed: int

    def geometry(self):
        vg = VolumeGeometry.centred(self.n)
        return vg, cone_angle_geometry(max(self.n[0], self.n[1]), self.det, self.views, self.half_angle)


def c5_manifest(seed: int = 5, count: int = 16):
    """Batching form: ``count`` independent problems drawn from
    ``numpy.random.default_rng(seed)``: cubic volumes with edges 96 .. 768
    voxels (the first problem is the anisotropic 512 x 512 x 128), float32
    or bfloat16 storage, cone half-angle uniform in [5, 15] degrees,
    90 .. 720 views, square detectors of 128 .. 768 pixels (any size, so
    most detector tiles are ragged), phantom or random-field contents."""
    rng = np.random.default_rng(seed)
    edges = [96, 128, 160, 192, 256, 320, 384, 448, 512, 640, 768]
    out = []
    for k in range(count):
        n = (512, 512, 128) if k == 0 else (int(rng.choice(edges)),) * 3
        out.append(BatchProblemSpec(
            n=n,
            dtype=str(rng.choice(["float32", "bfloat16"])),
            half_angle=float(rng.uniform(5.0, 15.0)),
            views=int(rng.integers(90, 721)),
            det=int(rng.integers(128, 769)),
            content=str(rng.choice(["phantom", "random"])),
            seed=1000 + k))
    return out


def small_batch_manifest(seed: int = 6, count: int = 64):
    """Batching form, many small problems: ``count`` few-view problems from
    ``numpy.random.default_rng(seed)`` (tomosynthesis-like: 2 .. 16 views)
    with cubic volumes of 96 .. 192 voxels and square detectors of 96 .. 192
    pixels.  One problem's launch has 144 .. 4608 blocks of 128 rays, up to
    about four waves of a GB300's resident blocks and mostly less than one,
    so separate launches leave the GPU partly idle; float32 or bfloat16
    storage, cone half-angle in [5, 15] degrees, phantom or random-field
    contents."""
    rng = np.random.default_rng(seed)
    edges = [96, 128, 160, 192]
    out = []
    for k in range(count):
        e = int(rng.choice(edges))
        out.append(BatchProblemSpec(
            n=(e, e, e),
            dtype=str(rng.choice(["float32", "bfloat16"])),
            half_angle=float(rng.uniform(5.0, 15.0)),
            views=int(rng.integers(2, 17)),
            det=int(rng.integers(96, 193)),
            content=str(rng.choice(["phantom", "random"])),
            seed=2000 + k))
    return out
