"""Differentiation form: autograd through the projector and CGLS
reconstruction with the forward model and its matched adjoint."""
import json
import os

import numpy as np
import pytest

import oracle
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


def test_autograd_gradient_is_the_adjoint(gjp):
    from paper_1609_00958_gb300.autograd import project
    vg, cg = synth.c1_geometry()
    g = gjp.Geometry.from_cone(cg)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    x = torch.rand(vg.n, device="cuda", generator=gen).requires_grad_(True)
    b = torch.rand(cg.n_views, cg.nv, cg.nu, device="cuda", generator=gen)
    loss = 0.5 * ((project(x, g) - b) ** 2).sum()
    loss.backward()
    with torch.no_grad():
        res = gjp.forward(x.detach(), g) - b
        want = gjp.adjoint(res, g, vg.n)
    err = ((x.grad - want).abs().max() / want.abs().max()).item()
    assert err < 1e-5, err


def test_autograd_through_bfloat16_storage(gjp):
    from paper_1609_00958_gb300.autograd import project
    vg, cg = synth.c1_geometry()
    g = gjp.Geometry.from_cone(cg)
    x = torch.rand(vg.n, device="cuda").to(torch.bfloat16).requires_grad_(True)
    project(x, g).sum().backward()
    assert x.grad.dtype == torch.bfloat16 and torch.isfinite(x.grad.float()).all()


def test_cgls_reaches_dense_least_squares_solution(gjp):
    """Tiny full-rank problem: the system matrix is formed column by column
    from the FP64 oracle; CGLS on the GPU converges to the least-squares
    solution and its residual never increases (beyond float32 rounding)."""
    from paper_1609_00958_gb300.recon import cgls
    vg = VolumeGeometry.centred((8, 8, 8))
    cg = synth.circular(24, 12, 12, 40.0, 80.0, 1.6)     # cond(A) ~ 84
    nvox = int(np.prod(vg.n))
    A = np.zeros((cg.n_views * cg.nv * cg.nu, nvox))
    for j in range(nvox):
        e = np.zeros(nvox)
        e[j] = 1.0
        A[:, j] = oracle.forward(e.reshape(vg.n), vg, cg).reshape(-1)
    rng = np.random.default_rng(4)
    x_true = rng.random(nvox)
    bvec = A @ x_true + 0.01 * rng.standard_normal(A.shape[0])
    x_ls = np.linalg.lstsq(A, bvec, rcond=None)[0]
    g = gjp.Geometry.from_cone(cg)
    b = torch.from_numpy(bvec.reshape(cg.n_views, cg.nv, cg.nu).astype(np.float32)).cuda()
    x, hist = cgls(b, g, vg.n, n_iter=200)
    res = np.array(hist.residual)
    assert (np.diff(res) <= 1e-5 * res[0]).all()
    xv = x.cpu().numpy().reshape(-1).astype(np.float64)
    # CGLS minimises |b - A x|: the objective reaches the least-squares optimum
    r_cg = np.linalg.norm(bvec - A @ xv) ** 2
    r_ls = np.linalg.norm(bvec - A @ x_ls) ** 2
    assert (r_cg - r_ls) / r_ls < 1e-4, (r_cg, r_ls)
    err = np.linalg.norm(xv - x_ls) / np.linalg.norm(x_ls)
    assert err < 5e-3, err


def test_cgls_checkpoint_resume(gjp, tmp_path):
    from paper_1609_00958_gb300.recon import cgls
    vg, cg = synth.c1_geometry()
    g = gjp.Geometry.from_cone(cg)
    ell = synth.ellipsoids_world(vg)
    b = torch.from_numpy(oracle.ellipsoid_project(ell, cg, sub=2).astype(np.float32)).cuda()
    full_x, full = cgls(b, g, vg.n, n_iter=12)
    ck = str(tmp_path / "cgls.pt")
    cgls(b, g, vg.n, n_iter=6, checkpoint=ck, checkpoint_every=3)
    assert os.path.exists(ck)
    x, resumed = cgls(b, g, vg.n, n_iter=12, checkpoint=ck, checkpoint_every=3, resume=True)
    assert len(resumed.residual) == len(full.residual)
    np.testing.assert_allclose(resumed.residual, full.residual, rtol=1e-3)
    assert ((x - full_x).abs().max() / full_x.abs().max()).item() < 1e-2


def test_cgls_differentiation_workload_from_analytic_projections(gjp):
    """256^3 / 180 views / 256^2: 30 CGLS iterations from closed-form line
    integrals of the Shepp-Logan-shaped phantom (no inverse crime: the data
    are not produced by the projector).  The residual decreases
    monotonically and the reconstruction approaches the rasterised phantom."""
    from paper_1609_00958_gb300.recon import cgls
    vg, cg = synth.c4_geometry()
    g = gjp.Geometry.from_cone(cg)
    ell = synth.ellipsoids_world(vg)
    b = torch.from_numpy(oracle.ellipsoid_project(ell, cg, sub=2).astype(np.float32)).cuda()
    x_true = torch.from_numpy(synth.voxelize(vg, ell, supersample=2)).cuda()
    x, hist = cgls(b, g, vg.n, n_iter=30, x_true=x_true)
    res, rmse = np.array(hist.residual), np.array(hist.rmse)
    assert len(res) == 31
    assert (np.diff(res) <= 1e-5 * res[0]).all()
    assert res[-1] < 0.05 * res[0]
    assert rmse[-1] < 0.6 * rmse[0]
    out = os.environ.get("GJP_REPORT_DIR")
    if out:
        with open(os.path.join(out, "cgls_256.json"), "w") as f:
            json.dump({"residual": res.tolist(), "rmse": rmse.tolist()}, f)
