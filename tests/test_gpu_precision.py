"""Precision form: large Shepp-Logan-shaped volumes stored in float32,
bfloat16 and float16 (float32 weights and accumulation), projected on the
1024^3 / 1024^2 / 720-view and 2048^3 / 2048^2 / 64-view workloads.

Errors are measured against the FP64 oracle evaluated on the unquantised
float32 volume, on every view of an evenly spaced subset of (at most) 128
views, each on a strided 64 x 64 grid of its detector pixels (shifted from
view to view so that the views together take every residue of the
stride in u and in v): max error relative to the largest reference value (bound 1e-5 for
float32 storage, 5e-3 for 16-bit storage) and RMS error.  Rays whose two
largest direction components are within 1e-5 may take either driving axis
(reading C2).  Both phantoms are voxelised with 2x2x2 supersampling on
the host (about 5 s at 2048^3 on 16 cores).  With GJP_REPORT_DIR set, the
error table is written there as JSON.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUND = {"float32": 1e-5, "bfloat16": 5e-3, "float16": 5e-3}


@pytest.fixture(scope="module")
def gjp():
    from paper_1609_00958_gb300 import build
    build.build()
    import paper_1609_00958_gb300 as m
    return m


def _host_gb():
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") / 2 ** 30
    except (ValueError, OSError):
        return 0.0


def strided_rays(cg, m):
    """(views, ius, ivs) of an m x m grid of pixels on every view, the grid
    shifted by a view-dependent offset within the stride."""
    su, sv = max(1, cg.nu // m), max(1, cg.nv // m)
    vs, us, ws = [], [], []
    for k in range(cg.n_views):
        ou, ov = (7 * k) % su, (3 * k) % sv
        iv, iu = np.meshgrid(np.arange(ov, cg.nv, sv)[:m], np.arange(ou, cg.nu, su)[:m], indexing="ij")
        vs.append(np.full(iu.size, k))
        us.append(iu.ravel())
        ws.append(iv.ravel())
    return np.concatenate(vs), np.concatenate(us), np.concatenate(ws)


@pytest.mark.parametrize("n", [1024, 2048])
def test_precision_form(gjp, n):
    vol_gb = n ** 3 * 4 / 2 ** 30
    free, _ = torch.cuda.mem_get_info()
    if free < 2.2 * vol_gb * 2 ** 30 or _host_gb() < 2.5 * vol_gb:
        pytest.skip("not enough device or host memory for this size")
    vg, cg_all = synth.c3_geometry(n)
    views = np.unique(np.linspace(0, cg_all.n_views - 1, min(128, cg_all.n_views)).round().astype(int))
    cg = cg_all.subset(views)
    vol = synth.voxelize(vg, supersample=2)
    g = gjp.Geometry.from_cone(cg)
    rays = strided_rays(cg, 64)
    ref = oracle.rays(vol, vg, cg, *rays)
    scale = np.abs(ref).max()
    table = {}
    d32 = torch.from_numpy(vol).cuda()
    for name in ("float32", "bfloat16", "float16"):
        dv = d32 if name == "float32" else d32.to(getattr(torch, name))
        out = gjp.forward(dv, g, vg.h)
        gjp.stream_status()
        if name == "bfloat16" and n == 2048:
            # 64-bit element offsets: the z-paired copy is refused (AUTO above read the volume)
            with pytest.raises(gjp.GjpError) as e:
                gjp.forward(dv, g, vg.h, path="pairs")
            from paper_1609_00958_gb300 import _capi
            assert e.value.status == _capi.GJP_ERR_UNSUPPORTED
        got = out[torch.from_numpy(rays[0]).cuda(), torch.from_numpy(rays[2]).cuda(),
                  torch.from_numpy(rays[1]).cuda()].double().cpu().numpy()
        del out
        if name != "float32":
            del dv
        res = parity.check_rays(got, vol, vg, cg, *rays, scale, BOUND[name], ref=ref)
        table[name] = {"max_rel": res["max_rel"], "rms_rel": res["rms_rel"], "ties": res["ties"]}
    # 16-bit storage keeps most of the float32 accuracy budget: bf16 rounds
    # to 8 significant bits, fp16 to 11
    assert table["float16"]["max_rel"] < table["bfloat16"]["max_rel"]
    out_dir = os.environ.get("GJP_REPORT_DIR")
    if out_dir:
        with open(os.path.join(out_dir, f"precision_{n}.json"), "w") as f:
            json.dump({"n": n, "views": int(len(views)), "rays": int(rays[0].size), "errors": table}, f, indent=1)
