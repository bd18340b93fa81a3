"""Host-side logic of bench.py, on the CPU: the exact sample count that the
metric divides by, the guard that reports DRAM traffic only for the kernel
sources it was captured on, and the clock record that gates a run."""
import hashlib
import json
import os
import shutil

import numpy as np
import pytest

import bench
import synth
from synth.geometry import VolumeGeometry


def brute_force_counts(vg, cg):
    """Per view: (ray, plane) pairs with -1 < p_k < n_k on both transverse
    axes, plane by plane in float64 (the definition the metric counts)."""
    n = np.array(vg.n, dtype=np.float64)
    h = np.array(vg.h)
    o = np.array(vg.origin)
    out = []
    for k in range(cg.n_views):
        s = (cg.src[k] - o) / h
        total = 0
        for iv in range(cg.nv):
            for iu in range(cg.nu):
                d = (cg.det_origin[k] + iu * cg.det_u[k] + iv * cg.det_v[k] - o) / h
                r = d - s
                m = int(np.argmax(np.abs(r)))
                others = [a for a in range(3) if a != m]
                for i in range(int(n[m])):
                    t = (i - s[m]) / r[m]
                    p = s + t * r
                    if all(-1.0 < p[a] < n[a] for a in others):
                        total += 1
        out.append(total)
    return np.array(out)


@pytest.mark.parametrize("case", ["circular", "random", "off_centre"])
def test_sample_counts_equal_brute_force(case):
    rng = np.random.default_rng(7)
    if case == "circular":
        vg = VolumeGeometry.centred((12, 11, 9))
        cg = synth.circular(3, 9, 8, 30.0, 60.0, 1.9, angles=[0.1, 0.9, 2.2])
    elif case == "random":
        vg = VolumeGeometry.centred((10, 12, 8), h=(0.8, 1.1, 1.3))
        cg = synth.random_geometry(rng, vg, 3, 7, 6, steep=True)
    else:
        vg = VolumeGeometry((9, 10, 11), (1.0, 1.0, 1.0), (-3.0, -6.5, -4.0))
        cg = synth.circular(2, 8, 9, 25.0, 50.0, 1.7, angles=[0.4, 2.9], z_shift=1.3)
    ref = brute_force_counts(vg, cg)
    assert ref.sum() > 0
    np.testing.assert_array_equal(bench.sample_counts(vg, cg), ref)


def test_sample_counts_device_form_matches_host_form():
    torch = pytest.importorskip("torch")
    vg = VolumeGeometry.centred((20, 18, 16))
    cg = synth.circular(4, 15, 13, 40.0, 80.0, 1.6, angles=[0.0, 0.785398, 1.5, 4.0])
    np.testing.assert_array_equal(bench.sample_counts_device(vg, cg, torch.device("cpu")),
                                  bench.sample_counts(vg, cg))


def test_dram_traffic_only_for_the_captured_sources(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "dram_traffic.json")))
    root = tmp_path / "repo"
    for rel in rec["sources"]:
        dst = root / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), dst)
    (root / "profiles").mkdir()
    shutil.copy(os.path.join(bench.ROOT, "profiles", "dram_traffic.json"), root / "profiles")
    monkeypatch.setattr(bench, "ROOT", str(root))
    kernel = "gjp_adjoint_combine_kernel<int"
    same = all(hashlib.sha256((root / rel).read_bytes()).hexdigest() == sha for rel, sha in rec["sources"].items())
    if same:
        assert bench.dram_traffic(kernel) == pytest.approx(rec["kernels"][kernel]["bytes_per_launch"])
    rel = next(iter(rec["sources"]))
    with open(root / rel, "a") as f:
        f.write("\n// edited after the capture\n")
    assert bench.dram_traffic(kernel) is None
    assert bench.dram_traffic("no_such_kernel") is None


def test_clock_record_summary(tmp_path):
    """The clock record keeps the median SM clock and every throttle reason
    that was active in any sample."""
    path = tmp_path / "clocks.csv"
    rows = [
        "0, 2070, 2070, 650.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 700.4, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 690.0, 0x8, Active, Not Active, Not Active, Not Active",
    ]
    path.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler("0")
    cs.path = str(path)
    out = cs.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert out["power_w_max"] == pytest.approx(700.4)
    assert not path.exists()
    empty = bench.ClockSampler("0")
    empty.path = str(tmp_path / "missing.csv")
    assert empty.summary()["reasons"] == ["unavailable"]
