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


def test_counters_only_for_the_captured_sources(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, bench.COUNTERS)))
    root = tmp_path / "repo"
    for rel in rec["sources"]:
        dst = root / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), dst)
    (root / "profiles").mkdir()
    shutil.copy(os.path.join(bench.ROOT, bench.COUNTERS), root / "profiles")
    monkeypatch.setattr(bench, "ROOT", str(root))
    kernel = "gjp_adjoint_combine_kernel<int"
    same = all(hashlib.sha256((root / rel).read_bytes()).hexdigest() == sha for rel, sha in rec["sources"].items())
    if same:
        assert bench.dram_traffic(kernel) == pytest.approx(rec["kernels"][kernel]["bytes_per_launch"])
        assert bench.limiter(kernel)["unit"] == "L2 reduction sectors"
    rel = next(iter(rec["sources"]))
    with open(root / rel, "a") as f:
        f.write("\n// edited after the capture\n")
    assert bench.dram_traffic(kernel) is None
    assert bench.limiter(kernel) is None
    assert bench.dram_traffic("no_such_kernel") is None


def test_kernel_key():
    assert bench.kernel_key("void gjp_forward_kernel<float, int, 0>(const T1 *, VolParams, int *)") == \
        "gjp_forward_kernel<float"
    assert bench.kernel_key("void gjp_detail::gjp_adjoint_combine_kernel<int, 0, 0>(const float *)") == \
        "gjp_adjoint_combine_kernel<int"


def test_ncu_summary_reads_units_and_scales_traffic(tmp_path):
    """The long-format ncu --csv log: one row per (launch, metric), values in
    the unit of their row.  DRAM bytes are scaled from the captured views to
    a full launch; the sample count is the exact host count of those views."""
    head = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",' \
           '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"'
    rows = []
    for i, (kern, metric, unit, val) in enumerate([
            ("void gjp_forward_kernel<float, int, 0>(const T1 *)", "dram__bytes_read.sum", "Mbyte", "12.5"),
            ("void gjp_forward_kernel<float, int, 0>(const T1 *)", "dram__bytes_write.sum", "Kbyte", "500"),
            ("void gjp_forward_kernel<float, int, 0>(const T1 *)", "gpu__time_duration.sum", "usecond", "1.5"),
            ("void gjp_forward_kernel<float, int, 0>(const T1 *)", "l1tex__data_pipe_lsu_wavefronts.sum", "",
             "1,000"),
            ("void gjp_forward_kernel<float, int, 0>(const T1 *)",
             "l1tex__data_pipe_lsu_wavefronts.avg.pct_of_peak_sustained_elapsed", "%", "80.5"),
            ("void gjp_forward_kernel<float, int, 0>(const T1 *)", "not_a_recorded_metric", "", "3")]):
        rows.append(f'"{i}","1","python","h","{kern}","1","7","(32, 4, 1)","(8, 2, 1)","0","10.3","",'
                    f'"{metric}","{unit}","{val}"')
    path = tmp_path / "c.csv"
    path.write_text("==PROF== preamble\n" + head + "\n" + "\n".join(rows) + "\n")
    rec = bench.ncu_summary(str(path), views=2, command="ncu ...", n=16, n_views=8)
    e = rec["kernels"]["gjp_forward_kernel<float"]
    assert e["dram_bytes"] == pytest.approx(12.5e6 + 500e3)
    assert e["bytes_per_launch"] == pytest.approx(4 * (12.5e6 + 500e3))
    assert e["duration_ns"] == pytest.approx(1500.0)
    assert e["l1_wavefronts"] == 1000.0 and e["l1_wavefronts_pct"] == 80.5
    vg, cg = synth.scaled_c2_geometry(16, 16, 8, 10.0)
    assert e["samples_captured"] == int(bench.sample_counts(vg, cg.subset(range(2))).sum())
    assert set(rec["sources"]) == {"paper_1609_00958_gb300/csrc/gjp.cu", "paper_1609_00958_gb300/csrc/gjp_common.cuh"}


def test_limiter_figures(monkeypatch):
    rec = {"l2_red_sectors": 4.0e9, "samples_captured": 1.0e10, "l2_red_pct": 66.0, "issue_pct": 77.0}
    monkeypatch.setattr(bench, "ncu_record", lambda k: rec)
    lim = bench.limiter("gjp_adjoint_combine_kernel<int")
    assert lim["per_sample"] == pytest.approx(0.4)
    assert lim["min_per_sample"] == pytest.approx(10.0 / 32.0)
    assert lim["efficiency"] == pytest.approx(round((10.0 / 32.0) / 0.4, 3))
    assert lim["pct_of_peak"] == 66.0
    assert bench.limiter("unknown_kernel") is None


def test_oracle_views_are_evenly_spaced():
    v = bench.oracle_views(360, 12)
    assert v == list(range(0, 360, 30))
    assert bench.oracle_views(5, 12) == [0, 1, 2, 3, 4]
    assert len(set(bench.oracle_views(360, 92))) == 92


def test_reference_arm_on_a_small_scan(capsys):
    """The reference arm's procedure (blocks of views on the oracle, one
    call per kernel) on a 16^3 scan: one JSON line with a per-kernel split
    whose sum is the step rate."""
    bench.main(["--impl", "reference", "--n", "16", "--views", "12", "--steps", "2", "--warmup", "1"])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == bench.UNIT
    assert set(line["kernels"]) == {"forward_f32", "forward_bf16", "adjoint_f32"}
    t = sum(k["seconds"] for k in line["kernels"].values())
    assert line["ms_per_step"] == pytest.approx(1e3 * t / 2, rel=1e-2, abs=2e-3)
    assert line["e2e"]["value"] == line["value"]


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


def test_oracle_leg_child_on_a_small_scan(tmp_path, capsys):
    """The child process of the GPU arm's CPU baseline, run in-process on a
    16^3 scan with the oracle's own results standing in for the GPU's: the
    errors it reports are float32 rounding only, the rates are positive."""
    import oracle
    vg, cg = synth.scaled_c2_geometry(16, 16, 12, 10.0)
    vol = synth.random_field(vg.n, seed=0)
    blocks, warm = bench.baseline_blocks(cg.n_views, 2)
    assert all(len(b) == bench.ORACLE_BLOCK for b in blocks + warm)
    assert len({v for b in blocks + warm for v in b}) == bench.ORACLE_BLOCK * 3
    vol_w = bench.bf16_widened(vol)
    for bi, blk in enumerate(blocks):
        sub = cg.subset(blk)
        p = oracle.forward(vol, vg, sub).astype(np.float32)
        np.save(tmp_path / f"p32_{bi}.npy", p)
        np.save(tmp_path / f"p16_{bi}.npy", oracle.forward(vol_w, vg, sub).astype(np.float32))
        np.save(tmp_path / f"back_{bi}.npy", oracle.adjoint(p.astype(np.float64), vg, sub).astype(np.float32))
    (tmp_path / "blocks.json").write_text(json.dumps({"blocks": blocks, "warm": warm}))
    bench.main(["--oracle-leg", str(tmp_path), "--n", "16", "--views", "12"])
    leg = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert leg["value"] > 0 and set(leg["kernels"]) == {"forward_f32", "forward_bf16", "adjoint_f32"}
    err = leg["error_vs_oracle"]
    assert err["views"] == [v for b in blocks for v in b]
    assert err["forward_f32"]["max_rel"] < 1e-6 and err["adjoint_f32"]["max_rel"] < 1e-6
    assert err["forward_bf16_vs_stored_values"]["max_rel"] < 1e-6
    assert 0 < err["forward_bf16"]["max_rel"] < 5e-3            # the storage rounding
