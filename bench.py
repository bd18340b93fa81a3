#!/usr/bin/env python
"""Benchmark of the GB300 GJP projector on the 512^3 cone-beam workload.

Workload (default): 512^3 voxels (h = 1), circular cone beam at a 10 degree
half-angle on the inscribed cylinder (D_so = 256/sin 10deg, D_sd = 2 D_so),
512 x 512 detector, 360 views over 360 degrees; the volume is a seeded
uniform [0, 1) random field (numpy default_rng(seed = rank)).

One step is one pass of the whole hot path over that workload:
  1. forward projection, float32 volume storage     (360 views)
  2. forward projection, bfloat16 volume storage    (360 views)
  3. adjoint (matched transpose) of the float32 projections into a float32 volume
The metric is GJP samples per second (a sample is one (ray, plane) pair
with at least one in-range tap, counted exactly on the host) over the
whole step; per-kernel rates, bytes and roofline fractions are reported
alongside.  All inputs (512 MiB volume, 377 MB projections) are larger
than the 129 MB L2, so no L2 flush is inserted between iterations.

With the seeded random field as the timed content, the same three kernels
are also timed on the 512^3 Shepp-Logan-shaped phantom (the other content
of the workload), reported under ``kernels_phantom``.

    python bench.py [--steps K] [--warmup W] [--impl reference]
    torchrun --nproc-per-node N bench.py --gpus N     (one scan split by
        views: every rank projects its range of the 360 views from its own
        copy of the volume; the adjoint volumes are summed with one
        all-reduce; total work is fixed, so scaling is strong)
    python bench.py --ncu-summary counters.csv        (writes the committed
        ncu counter record profiles/ncu_counters.json from an ncu --csv
        metrics log of the first 16 views)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "GJP Gsamples/s and achieved GB/s vs HBM peak, FP32 vs BF16 storage at stated error"
UNIT = "Gsamples/s"
L2_BYTES = 129 * 2 ** 20


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["gjp", "reference"], default="gjp")
    p.add_argument("--workload", choices=["step", "batch", "cgls"], default="step",
                   help="step: the 512^3 hot-path step (default); batch: the batching workload; "
                        "cgls: the 256^3 differentiation form (CGLS and an autograd step)")
    p.add_argument("--batch-mix", choices=["c5", "small"], default="c5",
                   help="problems of --workload batch: the 16-problem c5 mix or 64 small problems")
    p.add_argument("--no-batch", action="store_true", help="skip the small-problem batching figures of the step")
    p.add_argument("--n", type=int, default=512, help="volume edge (workload is defined at 512)")
    p.add_argument("--views", type=int, default=360)
    p.add_argument("--first-views", type=int, default=0,
                   help="keep only the first K views of the --views geometry (small profiling captures)")
    p.add_argument("--forward-path", choices=["auto", "gather", "pairs", "slab", "prefetch", "texture", "hwlin"],
                   default="auto", help="forward kernel family of the step (profiling other families)")
    p.add_argument("--path16", choices=["gather", "pairs"], default=None,
                   help="forward family of the 16-bit forward only (default: --forward-path); a capture of the "
                        "first views of a many-view scan uses it to run the family AUTO takes for the whole scan")
    p.add_argument("--tile-u", type=int, default=None, help="detector columns per block (library default if unset)")
    p.add_argument("--view-group", type=int, default=None, help="views issued together (library default if unset)")
    p.add_argument("--content", choices=["random", "phantom"], default="random")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-phantom", action="store_true", help="skip the Shepp-Logan-shaped phantom timings")
    p.add_argument("--oracle-blocks", type=int, default=3,
                   help="CPU baseline sample: blocks of ORACLE_BLOCK evenly spaced views")
    p.add_argument("--oracle-leg", default=None, help=argparse.SUPPRESS)
    p.add_argument("--ncu-summary", default=None, help="ncu --csv metrics log to turn into profiles/ncu_counters.json")
    p.add_argument("--ncu-views", type=int, default=16, help="views of the workload the ncu capture covered")
    p.add_argument("--ncu-command", default="", help="the command line that made the ncu capture")
    return p.parse_args(argv)


# --- workload ----------------------------------------------------------------

def workload(args):
    vg, cg = synth.scaled_c2_geometry(args.n, args.n, args.views, 10.0)
    name = f"cone-beam GJP {args.n}^3 {args.content} volume, {args.n}^2 detector, {args.views} views, 10 deg half-angle"
    if args.first_views:
        cg = cg.subset(range(min(args.first_views, cg.n_views)))
        name += f" (first {cg.n_views} views)"
    return vg, cg, name


def make_volume(args, vg, seed):
    if args.content == "phantom":
        return synth.voxelize(vg, supersample=2)
    return synth.random_field(vg.n, seed=seed)


def sample_counts(vg, cg) -> np.ndarray:
    """Per view, the number of (ray, plane) pairs with at least one in-range
    tap: planes i in [0, n_m - 1] with -1 < p_k(i) < n_k for both transverse
    axes, evaluated in float64 from the geometry."""
    n = np.array(vg.n, dtype=np.float64)
    h = np.array(vg.h)
    o = np.array(vg.origin)
    iv, iu = np.meshgrid(np.arange(cg.nv, dtype=np.float64), np.arange(cg.nu, dtype=np.float64), indexing="ij")
    out = np.zeros(cg.n_views, dtype=np.int64)
    big = 1e18
    for k in range(cg.n_views):
        s = (cg.src[k] - o) / h
        d = (cg.det_origin[k] + iu[..., None] * cg.det_u[k] + iv[..., None] * cg.det_v[k] - o) / h
        r = d - s
        m = np.argmax(np.abs(r), axis=-1)
        rm = np.take_along_axis(r, m[..., None], -1)[..., 0]
        sm = s[m]
        lo = np.zeros(m.shape)
        hi = n[m] - 1
        for ax in range(3):
            sel = m != ax
            g = np.where(sel, r[..., ax] / rm, 0.0)
            with np.errstate(divide="ignore", invalid="ignore"):
                a = sm + (-1.0 - s[ax]) / g
                b = sm + (n[ax] - s[ax]) / g
            low = np.where(g > 0, a, b)
            upp = np.where(g > 0, b, a)
            inside0 = (s[ax] > -1.0) & (s[ax] < n[ax])
            low = np.where(g == 0, np.where(inside0, -big, big), low)
            upp = np.where(g == 0, np.where(inside0, big, -big), upp)
            low = np.where(sel, low, -big)
            upp = np.where(sel, upp, big)
            lo = np.maximum(lo, np.floor(low) + 1.0)
            hi = np.minimum(hi, np.ceil(upp) - 1.0)
        out[k] = int(np.maximum(hi - lo + 1.0, 0.0).sum())
    return out


def sample_counts_device(vg, cg, device):
    """sample_counts evaluated in float64 with torch on `device` (the same
    formula, for workloads with many large views)."""
    import torch
    f64 = torch.float64
    n = torch.tensor(vg.n, dtype=f64, device=device)
    h = torch.tensor(vg.h, dtype=f64, device=device)
    o = torch.tensor(vg.origin, dtype=f64, device=device)
    iv, iu = torch.meshgrid(torch.arange(cg.nv, dtype=f64, device=device),
                            torch.arange(cg.nu, dtype=f64, device=device), indexing="ij")
    big = 1e18
    out = np.zeros(cg.n_views, dtype=np.int64)
    for k in range(cg.n_views):
        s = (torch.tensor(cg.src[k], dtype=f64, device=device) - o) / h
        d = (torch.tensor(cg.det_origin[k], dtype=f64, device=device) + iu[..., None] *
             torch.tensor(cg.det_u[k], dtype=f64, device=device) + iv[..., None] *
             torch.tensor(cg.det_v[k], dtype=f64, device=device) - o) / h
        r = d - s
        m = torch.argmax(torch.abs(r), dim=-1)
        rm = torch.gather(r, -1, m[..., None])[..., 0]
        sm = s[m]
        lo = torch.zeros_like(rm)
        hi = n[m] - 1
        for ax in range(3):
            sel = m != ax
            g = torch.where(sel, r[..., ax] / rm, torch.zeros_like(rm))
            a = sm + (-1.0 - s[ax]) / g
            b = sm + (n[ax] - s[ax]) / g
            low = torch.where(g > 0, a, b)
            upp = torch.where(g > 0, b, a)
            inside0 = bool((s[ax] > -1.0) & (s[ax] < n[ax]))
            low = torch.where(g == 0, torch.full_like(low, -big if inside0 else big), low)
            upp = torch.where(g == 0, torch.full_like(upp, big if inside0 else -big), upp)
            low = torch.where(sel, low, torch.full_like(low, -big))
            upp = torch.where(sel, upp, torch.full_like(upp, big))
            lo = torch.maximum(lo, torch.floor(low) + 1.0)
            hi = torch.minimum(hi, torch.ceil(upp) - 1.0)
        out[k] = int(torch.clamp(hi - lo + 1.0, min=0.0).sum().item())
    return out


# --- clocks -------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


COUNTERS = os.path.join("profiles", "ncu_counters.json")
# the kernel each step entry runs (ncu kernel-name prefix)
KERNEL_NAMES = {"forward_f32": "gjp_forward_kernel<float", "forward_bf16": "gjp_forward_kernel<__nv_bfloat16",
                "forward_f16": "gjp_forward_tld4_kernel<__half", "adjoint_f32": "gjp_adjoint_combine_kernel<int"}
# ncu metric -> record field
NCU_FIELDS = {
    "gpu__time_duration.sum": "duration_ns",
    "dram__bytes_read.sum": "dram_read_bytes",
    "dram__bytes_write.sum": "dram_write_bytes",
    "smsp__inst_executed.sum": "warp_instructions",
    "l1tex__data_pipe_lsu_wavefronts.sum": "l1_wavefronts",
    "lts__t_sectors_srcunit_tex_op_red.sum": "l2_red_sectors",
    "smsp__inst_executed_op_global_red.sum": "red_instructions",
    "smsp__issue_active.avg.pct_of_peak_sustained_elapsed": "issue_pct",
    "l1tex__data_pipe_lsu_wavefronts.avg.pct_of_peak_sustained_elapsed": "l1_wavefronts_pct",
    "lts__t_sectors_srcunit_tex_op_red.avg.pct_of_peak_sustained_elapsed": "l2_red_pct",
    "sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_elapsed": "alu_pct",
    "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_elapsed": "fma_pct",
    "l1tex__t_sector_hit_rate.pct": "l1_hit_pct",
    "lts__t_sector_hit_rate.pct": "l2_hit_pct",
    "sm__warps_active.avg.pct_of_peak_sustained_active": "warps_active_pct",
}
_UNIT_SCALE = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "tbyte": 1e12,
               "ns": 1.0, "us": 1e3, "usecond": 1e3, "msecond": 1e6, "ms": 1e6, "nsecond": 1.0, "second": 1e9}
# The binding unit of each kernel and the fewest of its operations per warp-plane (32
# samples of one detector column) that the sample's tap pattern needs: every warp-plane
# touches two transverse rows over the z-span of 32 neighbouring rays, 33 voxels
# (132 bytes in float32: two 128-byte L1 lines and five 32-byte sectors; 66 bytes in
# 16-bit storage: one or two lines, 1.5 on average).
# A note names the binding resource where the unit's own fraction is not the largest.
LIMIT_MODEL = {
    "gjp_forward_kernel<float": ("l1_wavefronts", "l1_wavefronts_pct", "L1 data-pipe wavefronts", 2 * 2.0, None),
    "gjp_forward_kernel<__nv_bfloat16": ("l1_wavefronts", "l1_wavefronts_pct", "L1 data-pipe wavefronts",
                                         2 * 1.5, "z-paired taps: one 4-byte load per row; the L1 does not "
                                         "saturate, issue slots and load latency (long-scoreboard stalls) bind"),
    "gjp_adjoint_combine_kernel<int": ("l2_red_sectors", "l2_red_pct", "L2 reduction sectors", 2 * 5.0,
                                       "issue slots bind first, the L2 reduction units next"),
}


def kernel_key(name: str) -> str:
    """``gjp_forward_kernel<float`` from an ncu kernel name such as
    ``void gjp_detail::gjp_forward_kernel<float, int, 0>(const T1 *, ...)``."""
    import re
    base = name.split("(")[0].replace("void ", "").strip()
    m = re.search(r"(\w+<[^,>(]+)", base)
    return m.group(1) if m else base


def _sources_hash():
    out = {}
    for rel in ("paper_1609_00958_gb300/csrc/gjp.cu", "paper_1609_00958_gb300/csrc/gjp_common.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            out[rel] = hashlib.sha256(f.read()).hexdigest()
    return out


def ncu_summary(csv_path: str, views: int, command: str, n: int = 512, n_views: int = 360) -> dict:
    """The counter record of one ncu ``--metrics ... --csv`` log that covered
    the first ``views`` views (one view group) of the workload: per kernel
    the raw counters, DRAM bytes scaled to a full launch, and the samples the
    capture processed.  Written to profiles/ncu_counters.json."""
    import csv
    rows = list(csv.reader(open(csv_path)))
    head = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
    hdr = rows[head]
    ki, mi, ui, vi = (hdr.index(c) for c in ("Kernel Name", "Metric Name", "Metric Unit", "Metric Value"))
    kernels = {}
    for r in rows[head + 1:]:
        if len(r) <= vi or r[mi] not in NCU_FIELDS:
            continue
        key = kernel_key(r[ki])
        val = float(r[vi].replace(",", ""))
        val *= _UNIT_SCALE.get(r[ui].strip().lower(), 1.0)
        kernels.setdefault(key, {})[NCU_FIELDS[r[mi]]] = val   # the last launch of a kernel wins
    vg, cg = synth.scaled_c2_geometry(n, n, n_views, 10.0)
    samples = int(sample_counts(vg, cg.subset(range(views))).sum())
    for key, e in kernels.items():
        once = key.startswith("gjp_zpairs")              # once per forward call, whatever the view count
        if "dram_read_bytes" in e and "dram_write_bytes" in e:
            e["dram_bytes"] = e["dram_read_bytes"] + e["dram_write_bytes"]
            e["bytes_per_launch"] = e["dram_bytes"] * (1.0 if once else n_views / views)
        if not once:
            e["samples_captured"] = samples
    return {"sources": _sources_hash(), "kernels": kernels,
            "capture": {"views": views, "of_views": n_views, "volume": n, "command": command,
                        "note": f"one ncu capture of the first {views} views (one view group) of the {n_views}-view "
                                f"{n}^3 workload; DRAM bytes scaled x{n_views / views:g} to a full launch"}}


def ncu_record(kernel: str):
    """The committed ncu counters of `kernel`, or None if absent or taken on
    different kernel sources."""
    path = os.path.join(ROOT, COUNTERS)
    try:
        with open(path) as f:
            d = json.load(f)
        for rel, sha in d["sources"].items():
            with open(os.path.join(ROOT, rel), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != sha:
                    return None
        return d["kernels"].get(kernel)
    except (OSError, KeyError, ValueError, TypeError):
        return None


def dram_traffic(kernel: str, views: int | None = None):
    """Per-launch DRAM bytes of `kernel` from the committed ncu record (a
    launch over the workload's 360 views, or over `views` views), or None if
    absent or taken on different kernel sources."""
    e = ncu_record(kernel)
    try:
        if e is None:
            return None
        per = float(e["bytes_per_launch"])
        if views is not None:
            with open(os.path.join(ROOT, COUNTERS)) as f:
                per *= views / float(json.load(f)["capture"]["of_views"])
        return per
    except (OSError, KeyError, TypeError, ValueError):
        return None


def limiter(kernel: str):
    """The kernel's binding unit from the committed ncu counters: its
    utilisation (percent of its peak over the kernel), operations per sample
    and the fewest per sample that the tap pattern needs (LIMIT_MODEL)."""
    e = ncu_record(kernel)
    model = LIMIT_MODEL.get(kernel)
    if e is None or model is None:
        return None
    field, pct_field, unit, min_per_warp_plane, note = model
    try:
        per_sample = e[field] / e["samples_captured"]
        least = min_per_warp_plane / 32.0
        out = {"unit": unit, "pct_of_peak": round(e[pct_field], 2), "per_sample": round(per_sample, 4),
               "min_per_sample": round(least, 4), "efficiency": round(least / per_sample, 3),
               "issue_pct": round(e.get("issue_pct", float("nan")), 2),
               "source": COUNTERS}
        if note:
            out["note"] = note
        return out
    except (KeyError, TypeError, ZeroDivisionError):
        return None


# --- GPU arm -------------------------------------------------------------------

def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def gpu_id_for_smi(local):
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            return vis.split(",")[local]
        return str(local)


def kernel_entry(name, ms, samples, alg_bytes, hbm, peak_kind, kname):
    """Per-kernel figures of one timed kernel."""
    gbs = alg_bytes / (ms * 1e-3) / 1e9
    e = {"ms": round(ms, 4), "gsamples_s": round(samples / (ms * 1e-3) / 1e9, 2),
         "algorithmic_gb": round(alg_bytes / 1e9, 4), "achieved_gbs": round(gbs, 1),
         "frac_of_" + peak_kind + "_hbm": round(gbs / hbm, 4),
         "paper_logical_gbs": round(samples * (8 if "16" in name and "f32" not in name else 16)
                                    / (ms * 1e-3) / 1e9, 1)}
    lim = limiter(kname) if kname else None
    if lim is not None:
        e["limiter"] = lim
    return e


def run_gjp(args):
    import torch
    from paper_1609_00958_gb300 import build as libbuild
    libbuild.build()
    import paper_1609_00958_gb300 as gjp
    from paper_1609_00958_gb300 import dist as gdist

    rank, world, local = dist_setup(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    vg, cg_full, wname = workload(args)
    # one scan split by views across the ranks (the whole scan at N = 1)
    scan = gdist.ShardedScan(cg_full)
    cg = scan.local_cone
    geom = scan.geometry
    if args.tile_u is not None or args.view_group is not None:
        tu, vgp = geom.launch
        geom.set_launch(args.tile_u or tu, args.view_group or vgp)

    vol_np = make_volume(args, vg, seed=0)
    vol32 = torch.from_numpy(vol_np).to(dev)
    # the texture unit has no bfloat16 format: the texture families store the 16-bit form as float16
    tex = args.forward_path in ("texture", "hwlin")
    vol16 = vol32.to(torch.float16 if tex else torch.bfloat16)
    k16 = "forward_f16" if tex else "forward_bf16"
    proj32 = torch.empty(cg.n_views, cg.nv, cg.nu, device=dev)
    proj16 = torch.empty_like(proj32)
    back = torch.empty(vg.n, device=dev)
    stream = torch.cuda.current_stream(dev)

    counts = sample_counts(vg, cg)                     # this rank's views
    samples_per_kernel = int(counts.sum())
    foot = np.array(gjp.footprint_voxels(geom, vg.n, vg.h, device=dev), dtype=np.float64)
    proj_bytes = 4.0 * cg.n_views * cg.nu * cg.nv
    alg_bytes = {
        "forward_f32": 4.0 * foot.sum() + proj_bytes,
        k16: 2.0 * foot.sum() + proj_bytes,
        "adjoint_f32": 8.0 * foot.sum() + proj_bytes,    # read-modify-write of each touched voxel per view
    }

    names = ["forward_f32", k16, "adjoint_f32"] + (["allreduce"] if world > 1 else [])

    def step(ev=None, v32=vol32, v16=vol16):
        if ev is not None:
            ev[0].record(stream)
        gjp.forward(v32, geom, vg.h, out=proj32, path=args.forward_path)
        if ev is not None:
            ev[1].record(stream)
        gjp.forward(v16, geom, vg.h, out=proj16, path=args.path16 or args.forward_path)
        if ev is not None:
            ev[2].record(stream)
        gjp.adjoint(proj32, geom, vg.n, vg.h, out=back)
        if ev is not None:
            ev[3].record(stream)
        if world > 1:
            gdist.all_reduce_sum_(back)                  # A^T y of the whole scan on every rank
            if ev is not None:
                ev[4].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    nev = len(names) + 1
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nev)] for _ in range(args.steps)]
    gdist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_id_for_smi(local)) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(args.steps):
            step(evs[k])
        t_end.record(stream)
        torch.cuda.synchronize()
    gdist.barrier()
    clocks = clk.summary()
    total_ms = gdist.max_over_ranks(t_start.elapsed_time(t_end))
    ms_per_step = total_ms / args.steps
    per_kernel_ms = {n: statistics.mean(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps))
                     for i, n in enumerate(names)}
    # samples of the whole scan: every rank's views, three kernels each
    job_samples_per_step = gdist.sum_over_ranks(3 * samples_per_kernel)
    value = job_samples_per_step / (ms_per_step * 1e-3) / 1e9

    hbm, peak_kind = peaks()
    kernels = {n: kernel_entry(n, per_kernel_ms[n], samples_per_kernel, alg_bytes[n], hbm, peak_kind,
                               KERNEL_NAMES.get(n)) for n in names if n != "allreduce"}
    if world > 1:
        kernels["allreduce"] = {"ms": round(per_kernel_ms["allreduce"], 4),
                                "bytes": int(back.numel() * 4), "what": "sum of the adjoint volumes over the ranks"}
    projector = [n for n in names if n != "allreduce"]
    dominant = max(projector, key=lambda n: per_kernel_ms[n])
    kname = KERNEL_NAMES[dominant]
    traffic = dram_traffic(kname, cg.n_views)
    dmsec = per_kernel_ms[dominant] * 1e-3
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": kernels[dominant]["achieved_gbs"],
                "peak": hbm, "peak_kind": peak_kind + " (copy, MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured"
                else "fallback", "unit": "GB/s",
                "frac": round(kernels[dominant]["achieved_gbs"] / hbm, 4),
                "frac_algorithmic": round(kernels[dominant]["achieved_gbs"] / hbm, 4),
                "frac_note": "algorithmic bytes: per view, every voxel with a non-zero tap once (adjoint: read "
                             "and written), summed over the views; views issued together share the L2, so the "
                             "DRAM traffic is far lower (dram_frac)",
                "traffic": traffic,
                "dram_frac": None if traffic is None else round(traffic / dmsec / 1e9 / hbm, 4),
                "limiter": kernels[dominant].get("limiter")}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, gjp, geom, vg, cg, vol_np, dev, stream, job_samples_per_step, world)

    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
        "dtype": "f32 (weights/accumulation); volume storage f32 and bf16",
        "data": "synthetic (seeded uniform [0,1) random field)" if args.content == "random"
        else "synthetic (Shepp-Logan-shaped phantom, project-owned ellipsoids)",
        "config": {"workload": wname, "volume": list(vg.n), "detector": [cg.nv, cg.nu], "views": cg_full.n_views,
                   "launch": {"tile_u": geom.launch[0], "view_group": geom.launch[1]},
                   "forward_path": args.forward_path, **({"path16": args.path16} if args.path16 else {}),
                   "tap_source": {"forward_f32": "volume", k16: "z-paired copy, written per call"
                                  if launches_per_step(args.forward_path, args.path16, vg.n, cg.n_views) > 3 else "volume"},
                   "step": "forward f32 + forward bf16 + adjoint f32", "samples_per_kernel": samples_per_kernel,
                   "l2": "inputs larger than L2 (no flush)",
                   "parallelism": "one GPU" if world == 1 else
                   f"one scan split by views over {world} GPUs (rank views {scan.start}..{scan.stop - 1}), "
                   "adjoint volumes summed by one all-reduce"},
        "kernels": kernels, "roofline": roofline, "clocks": clocks,
        "gpu_launches": launches_per_step(args.forward_path, args.path16, vg.n, cg.n_views) * args.steps,
        "e2e": e2e,
    }
    if world == 1 and args.content == "random" and not args.no_phantom and not args.first_views:
        result["kernels_phantom"] = phantom_kernels(args, gjp, geom, vg, cg, dev, stream, hbm, peak_kind, k16)
    if world == 1 and not args.first_views:
        result["c1"] = c1_kernels(gjp, dev)
    if world == 1 and not args.no_batch and not args.first_views:
        name, make = BATCH_MIXES["small"]
        ms, counts, _, _ = batch_measure(make(), args.warmup, max(1, min(args.steps, 10)), dev)
        result["batching_small"] = {"workload": name, "samples": counts[0], **batch_summary(ms, counts)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args, gjp, vg, cg, proj32, proj16)
        if "error_vs_oracle" in result["cpu_baseline"]:
            result["error_vs_oracle"] = result["cpu_baseline"].pop("error_vs_oracle")
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def c1_kernels(gjp, dev, reps: int = 200):
    """The three kernels of the step on the c1 case (64^3 Shepp-Logan-shaped
    phantom, 2x2x2 supersampled, 64^2 detector, 32 views): samples/s only --
    the volume is cache-resident, so no roofline fraction applies.  CUDA
    events over ``reps`` back-to-back repetitions after a warm-up."""
    import torch
    vg, cg = synth.c1_geometry()
    g = gjp.Geometry.from_cone(cg)
    v32 = torch.from_numpy(synth.voxelize(vg, supersample=2)).to(dev)
    v16 = v32.to(torch.bfloat16)
    p32 = gjp.forward(v32, g, vg.h)
    p16 = torch.empty_like(p32)
    back = torch.empty(vg.n, device=dev)
    samples = int(sample_counts(vg, cg).sum())
    fns = {"forward_f32": lambda: gjp.forward(v32, g, vg.h, out=p32),
           "forward_bf16": lambda: gjp.forward(v16, g, vg.h, out=p16),
           "adjoint_f32": lambda: gjp.adjoint(p32, g, vg.n, vg.h, out=back)}
    out = {"workload": "c1: 64^3 phantom, 64^2 detector, 32 views (cache-resident; samples/s only)",
           "samples_per_kernel": samples}
    for k, f in fns.items():
        for _ in range(10):
            f()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            f()
        e.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(e) / reps
        out[k] = {"ms": round(ms, 5), "gsamples_s": round(samples / (ms * 1e-3) / 1e9, 2)}
    return out


def launches_per_step(path: str, path16, n, n_views: int) -> int:
    """The library's kernel launches in one step: forward f32, forward bf16
    and the adjoint, plus the z-paired copy that a "pairs" forward writes
    first (AUTO takes it for 16-bit storage over 32 or more views and 2^27
    view-voxels; both only where the element offsets fit 32 bits, the
    library's fits_int32 rule)."""
    nx, ny, nz = (int(v) for v in n)
    fits = nx * ny * nz + 2 * (ny * nz + nz + 1) < 2147483647
    p16 = path16 or path
    pays = n_views >= 32 and n_views * nx * ny * nz >= 2 ** 27      # the library's pairs_pay rule
    pairs16 = p16 == "pairs" or (p16 == "auto" and pays)
    return 3 + int(fits and pairs16) + int(fits and path == "pairs")


def phantom_kernels(args, gjp, geom, vg, cg, dev, stream, hbm, peak_kind, k16):
    """The three kernels of the step on the 512^3 Shepp-Logan-shaped
    phantom (2x2x2 supersampled), timed with CUDA events like the step
    (min(steps, 5) repetitions after the warm-up)."""
    import torch
    vol = torch.from_numpy(synth.voxelize(vg, supersample=2)).to(dev)
    v16 = vol.to(torch.float16 if k16 == "forward_f16" else torch.bfloat16)
    p32 = torch.empty(cg.n_views, cg.nv, cg.nu, device=dev)
    p16 = torch.empty_like(p32)
    bk = torch.empty(vg.n, device=dev)
    fns = {"forward_f32": lambda: gjp.forward(vol, geom, vg.h, out=p32, path=args.forward_path),
           k16: lambda: gjp.forward(v16, geom, vg.h, out=p16, path=args.path16 or args.forward_path),
           "adjoint_f32": lambda: gjp.adjoint(p32, geom, vg.n, vg.h, out=bk)}
    counts = sample_counts(vg, cg)
    foot = np.array(gjp.footprint_voxels(geom, vg.n, vg.h, device=dev), dtype=np.float64)
    proj_bytes = 4.0 * cg.n_views * cg.nu * cg.nv
    alg = {"forward_f32": 4.0 * foot.sum() + proj_bytes, k16: 2.0 * foot.sum() + proj_bytes,
           "adjoint_f32": 8.0 * foot.sum() + proj_bytes}
    out = {}
    reps = max(1, min(args.steps, 5))
    for name, fn in fns.items():
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        out[name] = kernel_entry(name, a.elapsed_time(b) / reps, int(counts.sum()), alg[name], hbm, peak_kind, None)
    out["content"] = "Shepp-Logan-shaped phantom (project-owned ellipsoids), 2x2x2 supersampled"
    return out


def run_e2e(args, gjp, geom, vg, cg, vol_np, dev, stream, job_samples_per_step, world=1):
    """Same step through the public API with host buffers.  Every step copies
    its inputs (float32 and bfloat16 volume) from pinned host memory to the
    GPU and its results (both projections and the adjoint volume) back to
    pinned host memory.  Steps are pipelined the way a caller of the
    stream-ordered API would run them: copies in, kernels and copies out
    each on their own stream, with two device buffer sets, so step k+1's
    input copy overlaps step k's kernels; with one event per tensor each
    kernel waits only for its own input and each result is copied out as
    soon as its kernel ends.  The timed region covers all steps, every copy
    included, and ends when the last results are on the host.  With the
    scan split over several GPUs, every rank copies the volume in and its
    own views' projections out, sums the adjoint volumes with the all-reduce
    and copies the whole adjoint out; the byte counts are the job's."""
    import torch
    from paper_1609_00958_gb300 import dist as gdist
    h_vol32 = torch.from_numpy(vol_np).pin_memory()
    h_vol16 = h_vol32.to(torch.bfloat16).pin_memory()
    pshape = (cg.n_views, cg.nv, cg.nu)
    h_out = [(torch.empty(pshape).pin_memory(), torch.empty(pshape).pin_memory(), torch.empty(vg.n).pin_memory())
             for _ in range(2)]
    d_set = [(torch.empty(vg.n, device=dev), torch.empty(vg.n, device=dev, dtype=torch.bfloat16),
              torch.empty(pshape, device=dev), torch.empty(pshape, device=dev), torch.empty(vg.n, device=dev))
             for _ in range(2)]
    s_in, s_comp, s_out = (torch.cuda.Stream(dev) for _ in range(3))
    ev = {name: [torch.cuda.Event() for _ in range(2)]
          for name in ("in32", "in16", "f32", "f16", "adj", "out")}
    for e in ev["f16"] + ev["out"]:
        e.record(stream)

    def step(k):
        # Per-tensor events: each kernel starts when its own input is on the
        # device, and each result leaves as soon as its kernel ends, so only
        # the first input copy and the last output copy are not overlapped.
        b = k % 2
        v32, v16, p32, p16, back = d_set[b]
        o32, o16, oback = h_out[b]
        with torch.cuda.stream(s_in):          # step k-2's forwards are done reading buffer b's volumes
            s_in.wait_event(ev["f16"][b])
            v32.copy_(h_vol32, non_blocking=True)
            ev["in32"][b].record(s_in)
            v16.copy_(h_vol16, non_blocking=True)
            ev["in16"][b].record(s_in)
        with torch.cuda.stream(s_comp):
            s_comp.wait_event(ev["out"][b])    # step k-2's results have left buffer b
            s_comp.wait_event(ev["in32"][b])
            gjp.forward(v32, geom, vg.h, out=p32, stream=s_comp)
            ev["f32"][b].record(s_comp)
            s_comp.wait_event(ev["in16"][b])
            gjp.forward(v16, geom, vg.h, out=p16, stream=s_comp)
            ev["f16"][b].record(s_comp)
            gjp.adjoint(p32, geom, vg.n, vg.h, out=back, stream=s_comp)
            if world > 1:
                gdist.all_reduce_sum_(back)
            ev["adj"][b].record(s_comp)
        with torch.cuda.stream(s_out):         # results of step k back to the host, each when ready
            s_out.wait_event(ev["f32"][b])
            o32.copy_(p32, non_blocking=True)
            s_out.wait_event(ev["f16"][b])
            o16.copy_(p16, non_blocking=True)
            s_out.wait_event(ev["adj"][b])
            oback.copy_(back, non_blocking=True)
            ev["out"][b].record(s_out)

    for k in range(max(1, args.warmup)):
        step(k)
    torch.cuda.synchronize()
    gdist.barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(k)
    torch.cuda.synchronize()                   # the host holds every step's results
    wall = gdist.max_over_ranks(time.perf_counter() - t0)
    bi = gdist.sum_over_ranks(h_vol32.numel() * 4 + h_vol16.numel() * 2)
    bo = gdist.sum_over_ranks((2 * int(np.prod(pshape)) + int(np.prod(vg.n))) * 4)
    return {"value": round(job_samples_per_step / (wall / args.steps) / 1e9, 3), "unit": UNIT,
            "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo),
            "ms_per_step": round(1e3 * wall / args.steps, 3),
            "pipelining": "copies in / kernels / copies out on three streams, two device buffer sets, "
                          "one event per tensor"}


# --- CPU oracle (baseline leg and reference arm) ----------------------------------
#
# Both legs time the oracle the same way: blocks of ORACLE_BLOCK evenly spaced
# views of the scan, each block in three calls -- forward of the float32
# volume, forward of the bfloat16-stored values, adjoint -- after one warm-up
# call.  The oracle's adjoint scatters into one private FP64 volume per thread
# and sums them once per call, so a call over a block of views pays that cost
# once per block; the adjoint figure includes it.

ORACLE_BLOCK = 4


def oracle_views(n_views: int, count: int) -> list:
    """``count`` views evenly spaced over the scan (distinct, ascending)."""
    count = max(1, min(count, n_views))
    return sorted({int(round(i * n_views / count)) % n_views for i in range(count)})


def oracle_threads():
    return os.cpu_count() or 1


def oracle_adjoint_bytes(vg, threads):
    """Room for every thread's private FP64 volume, within a quarter of the
    host's physical memory."""
    need = threads * float(np.prod(vg.n)) * 8.0 + 1.0
    try:
        phys = float(os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES"))
        return min(need, 0.25 * phys)
    except (ValueError, OSError, AttributeError):
        return need


def oracle_block(oracle, vg, cg, vol_np, vol_bf16w, views, threads, counts, y=None):
    """One block of views on the oracle: per kernel (seconds, samples) and
    the results.  The adjoint takes ``y`` (the projections of these views;
    the oracle's own float32-volume projections when None)."""
    import time as _t
    sub = cg.subset(views)
    samples = int(sum(int(counts[v]) for v in views))
    t0 = _t.perf_counter()
    p = oracle.forward(vol_np, vg, sub, threads=threads)
    t1 = _t.perf_counter()
    p16 = oracle.forward(vol_bf16w, vg, sub, threads=threads)
    t2 = _t.perf_counter()
    yy = p if y is None else np.asarray(y, dtype=np.float64)
    back = oracle.adjoint(yy, vg, sub, threads=threads, max_bytes=oracle_adjoint_bytes(vg, threads))
    t3 = _t.perf_counter()
    times = {"forward_f32": t1 - t0, "forward_bf16": t2 - t1, "adjoint_f32": t3 - t2}
    return times, samples, (p, p16, back)


def oracle_warmup(oracle, vg, cg, vol_np, threads):
    """Loads the library, starts the thread pool and pages the volume in."""
    oracle.forward(vol_np, vg, cg.subset([0]), threads=threads)


def oracle_rates(times_list, samples_list):
    """Per-kernel and whole-step rates over the timed blocks."""
    out = {}
    for k in ("forward_f32", "forward_bf16", "adjoint_f32"):
        t = sum(tm[k] for tm in times_list)
        out[k] = {"gsamples_s": round(sum(samples_list) / t / 1e9, 5), "seconds": round(t, 6)}
    total_t = sum(sum(tm.values()) for tm in times_list)
    return 3 * sum(samples_list) / total_t / 1e9, total_t, out


def bf16_widened(vol_np):
    """Round-to-nearest-even float32 -> bfloat16, widened back to float32
    (the values a bfloat16 volume stores)."""
    import torch
    return torch.from_numpy(vol_np).to(torch.bfloat16).float().numpy()


def _err(gpu, ref):
    d = np.abs(np.asarray(gpu, np.float64) - ref)
    m = max(float(np.abs(ref).max()), 1e-30)
    return {"max_rel": float(f"{d.max() / m:.3e}"), "rms_rel": float(f"{np.sqrt(np.mean(d * d)) / m:.3e}")}


def _worst(es):
    return {"max_rel": max(e["max_rel"] for e in es),
            "rms_rel": float(f"{np.sqrt(np.mean([e['rms_rel'] ** 2 for e in es])):.3e}")}


def oracle_leg(vg, cg, vol_np, counts, blocks, warm_blocks, gpu=None):
    """The oracle timed on the host cores: ``warm_blocks`` untimed blocks,
    then ``blocks`` timed, each block of views in three oracle calls.  With
    ``gpu`` (per block: GPU float32 and bfloat16 projections of the block's
    views and the GPU adjoint of those float32 projections), also the GPU's
    error against the oracle on those views; the oracle's adjoint then takes
    the GPU projections as its input, like the GPU adjoint."""
    import oracle
    threads = oracle_threads()
    vol_w = bf16_widened(vol_np)
    oracle_warmup(oracle, vg, cg, vol_np, threads)
    for blk in warm_blocks:
        oracle_block(oracle, vg, cg, vol_np, vol_w, blk, threads, counts)
    times, samples, e32, e16, e16s, eadj = [], [], [], [], [], []
    for bi, blk in enumerate(blocks):
        y = None if gpu is None else gpu[bi][0]
        tm, smp, (p, p16, back) = oracle_block(oracle, vg, cg, vol_np, vol_w, blk, threads, counts, y=y)
        times.append(tm)
        samples.append(smp)
        if gpu is not None:
            g32, g16, gback = gpu[bi]
            for j in range(len(blk)):
                e32.append(_err(g32[j], p[j]))
                e16.append(_err(g16[j], p[j]))
                e16s.append(_err(g16[j], p16[j]))
            eadj.append(_err(gback, back))
        del back
    value, total_t, per_kernel = oracle_rates(times, samples)
    out = {"value": value, "seconds": total_t, "kernels": per_kernel, "threads": threads}
    if gpu is not None:
        out["error_vs_oracle"] = {
            "views": [v for blk in blocks for v in blk], "forward_f32": _worst(e32), "forward_bf16": _worst(e16),
            "forward_bf16_vs_stored_values": _worst(e16s),
            "adjoint_f32": _worst(eadj) | {"what": f"A^T y of each block of {ORACLE_BLOCK} views, y = the GPU "
                                                   "projections; GPU against the FP64 oracle"},
            "bounds": {"f32": 1e-5, "bf16": 5e-3, "bf16_vs_stored_values": 1e-5, "adjoint_f32": 1e-5}}
    return out


def baseline_blocks(n_views, n_blocks):
    """``n_blocks`` blocks of ORACLE_BLOCK views, each spread over the scan,
    plus one further such block for the warm-up."""
    views = oracle_views(n_views, ORACLE_BLOCK * (n_blocks + 1))
    blocks = [views[i::n_blocks + 1][:ORACLE_BLOCK] for i in range(n_blocks + 1)]
    return blocks[1:], blocks[:1]


def cpu_baseline(args, gjp, vg, cg, proj32, proj16):
    """The oracle on the host cores over ``--oracle-blocks`` blocks of
    ORACLE_BLOCK views, after one warm-up block: the reference arm's
    procedure, run in a fresh child process (no CUDA) so that both legs time
    the oracle under the same conditions.  The GPU results for those views
    (float32 and bfloat16 projections, the adjoint of each block's float32
    projections) go to the child through files, which returns the oracle's
    rates and the GPU's error against it."""
    import shutil
    import subprocess as sp
    blocks, warm = baseline_blocks(cg.n_views, args.oracle_blocks)
    tmp = tempfile.mkdtemp(prefix="gjp_oracle_leg_")
    try:
        for bi, blk in enumerate(blocks):
            gsub = gjp.Geometry.from_cone(cg.subset(blk))
            gback = gjp.adjoint(proj32[blk].contiguous(), gsub, vg.n, vg.h)
            np.save(os.path.join(tmp, f"p32_{bi}.npy"), proj32[blk].cpu().numpy())
            np.save(os.path.join(tmp, f"p16_{bi}.npy"), proj16[blk].cpu().numpy())
            np.save(os.path.join(tmp, f"back_{bi}.npy"), gback.cpu().numpy())
            gsub.close()
            del gback
        with open(os.path.join(tmp, "blocks.json"), "w") as f:
            json.dump({"blocks": blocks, "warm": warm}, f)
        env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-leg", tmp, "--n", str(args.n),
               "--views", str(args.views), "--content", args.content]
        if args.first_views:
            cmd += ["--first-views", str(args.first_views)]
        res = sp.run(cmd, env=env, capture_output=True, text=True, check=True)
        leg = json.loads(res.stdout.strip().splitlines()[-1])
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    views = [v for blk in blocks for v in blk]
    return {"value": round(leg["value"], 5), "unit": UNIT, "cores": leg["threads"], "kind": "oracle",
            "sample": f"FP64 oracle (OpenMP, {leg['threads']} threads, fresh process) on {len(views)} of "
                      f"{cg.n_views} views in {len(blocks)} blocks of {ORACLE_BLOCK} spread over the scan, after "
                      "one warm-up block: per block one forward of the float32 volume, one of the bfloat16-stored "
                      "values and one adjoint; the adjoint includes summing its per-thread private volumes once "
                      "per block",
            "seconds": round(leg["seconds"], 3), "kernels": leg["kernels"],
            "c1": leg.get("c1"), "error_vs_oracle": leg["error_vs_oracle"]}


def run_oracle_leg(args):
    """Child process of cpu_baseline: times the oracle on the blocks named
    in ``--oracle-leg DIR`` and compares it with the GPU results there."""
    vg, cg, _ = workload(args)
    vol_np = make_volume(args, vg, seed=0)
    counts = sample_counts(vg, cg)
    with open(os.path.join(args.oracle_leg, "blocks.json")) as f:
        spec = json.load(f)
    gpu = [(np.load(os.path.join(args.oracle_leg, f"p32_{bi}.npy")),
            np.load(os.path.join(args.oracle_leg, f"p16_{bi}.npy")),
            np.load(os.path.join(args.oracle_leg, f"back_{bi}.npy"))) for bi in range(len(spec["blocks"]))]
    out = oracle_leg(vg, cg, vol_np, counts, spec["blocks"], spec["warm"], gpu=gpu)
    out["c1"] = oracle_c1()
    print(json.dumps(out), flush=True)


def oracle_c1():
    """The oracle on the whole c1 case (64^3 phantom, 32 views), the three
    calls of a step after one warm-up call."""
    import oracle
    vg, cg = synth.c1_geometry()
    vol = synth.voxelize(vg, supersample=2)
    threads = oracle_threads()
    counts = sample_counts(vg, cg)
    oracle_warmup(oracle, vg, cg, vol, threads)
    times, smp, _ = oracle_block(oracle, vg, cg, vol, bf16_widened(vol), list(range(cg.n_views)), threads, counts)
    value, total_t, per_kernel = oracle_rates([times], [smp])
    return {"value": value, "unit": UNIT, "seconds": total_t, "kernels": per_kernel, "threads": threads,
            "sample": "the whole c1 case: 32 views, forward f32, forward bf16-stored values, adjoint"}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, one block of
    ORACLE_BLOCK views spread over the scan per step (forward float32,
    forward of the bfloat16-stored values, adjoint), the procedure of the
    GPU arm's cpu_baseline."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vg, cg, wname = workload(args)
    vol_np = make_volume(args, vg, seed=0)
    counts = sample_counts(vg, cg)
    n_steps = args.steps + max(1, args.warmup)
    views = oracle_views(cg.n_views, ORACLE_BLOCK * n_steps)
    blocks = [views[i::n_steps][:ORACLE_BLOCK] for i in range(n_steps)]   # each block spans the scan
    warm = blocks[:n_steps - args.steps]
    leg = oracle_leg(vg, cg, vol_np, counts, blocks[len(warm):], warm)
    value, total_t, threads = leg["value"], leg["seconds"], leg["threads"]
    sample = (f"one block of {ORACLE_BLOCK} views per step (forward f32 + forward bf16-stored + adjoint, "
              f"one oracle call each), {args.steps} blocks spread over the scan after {len(warm)} warm-up "
              f"block(s), FP64 oracle with {threads} OpenMP threads; the adjoint includes summing its "
              "per-thread private volumes once per block")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * total_t / max(1, args.steps), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded uniform [0,1) random field)" if args.content == "random" else "synthetic phantom",
        "config": {"workload": wname, "volume": list(vg.n), "detector": [cg.nv, cg.nu], "views": cg.n_views,
                   "step": f"one block of {ORACLE_BLOCK} views: forward f32 + forward bf16 + adjoint (oracle)"},
        "kernels": leg["kernels"],
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def batch_measure(specs, warmup, steps, dev, clocks=False):
    """Times one set of independent problems (synth BatchProblemSpec) five
    ways, CUDA events over ``steps`` repetitions after ``warmup``:
    separate gjp_forward launches on one stream, the same launches replayed
    from a CUDA graph, one persistent batched launch with the geometries'
    default launch shapes, the same after gjp_batch_autotune, and that
    replayed from a CUDA graph.  Returns (ms per variant, samples, tunings,
    clock record or None)."""
    import torch
    import paper_1609_00958_gb300 as gjp
    items, samples, alg_bytes = [], 0, 0.0
    for sp in specs:
        vg, cg = sp.geometry()
        vol_np = (synth.voxelize(vg, supersample=2) if sp.content == "phantom"
                  else synth.random_field(vg.n, seed=sp.seed))
        vol = torch.from_numpy(vol_np).to(dev).to(getattr(torch, sp.dtype))
        g = gjp.Geometry.from_cone(cg)
        items.append((vol, g, vg.h, None, torch.empty(g.proj_shape, device=dev)))
        samples += int(sample_counts_device(vg, cg, dev).sum())
        # compulsory bytes: the footprint of up to 16 evenly spaced views,
        # scaled to all views, times the storage size, plus the projections
        pick = sorted({int(round(k * cg.n_views / min(16, cg.n_views))) % cg.n_views
                       for k in range(min(16, cg.n_views))})
        foot = float(np.mean(gjp.footprint_voxels(g, vg.n, vg.h, views=pick, device=dev)))
        alg_bytes += foot * cg.n_views * vol.element_size() + 4.0 * cg.n_views * cg.nu * cg.nv
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        for _ in range(max(1, warmup)):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def separate():
        for vol, g, h, origin, out in items:
            gjp.forward(vol, g, h, origin, out=out)

    side = [torch.cuda.Stream(dev) for _ in range(4)]

    def separate_streams():
        # the same launches spread round-robin over 4 streams, joined at the end
        for s_ in side:
            s_.wait_stream(stream)
        for k, (vol, g, h, origin, out) in enumerate(items):
            gjp.forward(vol, g, h, origin, out=out, stream=side[k % 4])
        for s_ in side:
            stream.wait_stream(s_)

    ms = {"separate_launches": timed(separate, steps), "separate_launches_4_streams": timed(separate_streams, steps)}
    sep_graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(sep_graph):
        separate()
    ms["separate_launches_graph"] = timed(sep_graph.replay, steps)
    batch = gjp.Batch(items)
    launches = batch.launches
    ms["batched"] = timed(batch.forward, steps)
    tunings = batch.autotune(reps=2)
    ms["batched_autotuned"] = timed(batch.forward, steps)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.forward()
    clk = None
    if clocks:
        with ClockSampler(gpu_id_for_smi(0)) as c:
            ms["batched_autotuned_graph"] = timed(graph.replay, steps)
        clk = c.summary()
    else:
        ms["batched_autotuned_graph"] = timed(graph.replay, steps)
    return {k: round(v, 3) for k, v in ms.items()}, (samples, alg_bytes, launches), tunings, clk


def batch_summary(ms, counts):
    samples, alg_bytes, launches = counts
    gsps = lambda m: round(samples / (m * 1e-3) / 1e9, 2)
    hbm, peak_kind = peaks()
    best = ms["batched_autotuned_graph"]
    return {"ms": ms, "gsamples_s": {k: gsps(v) for k, v in ms.items()},
            "algorithmic_gb": round(alg_bytes / 1e9, 3), "launches_per_batched_forward": launches,
            "frac_of_" + peak_kind + "_hbm": round(alg_bytes / (best * 1e-3) / 1e9 / hbm, 4),
            "speedup_vs_separate": round(ms["separate_launches"] / ms["batched_autotuned_graph"], 3),
            "speedup_vs_separate_graph": round(ms["separate_launches_graph"] / ms["batched_autotuned_graph"], 3),
            "speedup_vs_separate_4_streams": round(ms["separate_launches_4_streams"] / ms["batched_autotuned_graph"],
                                                   3)}


BATCH_MIXES = {
    "c5": ("batching form: 16 problems, 96^3..768^3 and 512x512x128, 90..720 views, 128^2..768^2 detectors, "
           "5..15 deg half-angles (synth.c5_manifest)", lambda: synth.c5_manifest()),
    "small": ("batching form, many small problems: 64 few-view problems, 96^3..192^3, 2..16 views, 96^2..192^2 "
              "detectors, 5..15 deg half-angles (synth.small_batch_manifest)", lambda: synth.small_batch_manifest()),
}


def run_batch(args):
    """The batching workload (``--batch-mix``): independent problems
    projected by separate launches (plain and from a CUDA graph) and by one
    persistent batched launch (default shapes, autotuned, autotuned from a
    CUDA graph).  One JSON line; ``value`` is the autotuned batched launch
    replayed from a CUDA graph, in Gsamples/s."""
    import torch
    from paper_1609_00958_gb300 import build as libbuild
    libbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    name, make = BATCH_MIXES[args.batch_mix]
    specs = make()
    ms, counts, tunings, clocks = batch_measure(specs, args.warmup, args.steps, dev, clocks=True)
    out = batch_summary(ms, counts)
    samples = counts[0]
    print(json.dumps({
        "metric": METRIC + " (batching form)", "value": out["gsamples_s"]["batched_autotuned_graph"], "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms["batched_autotuned_graph"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (weights/accumulation); volume storage f32 and bf16",
        "data": "synthetic (seeded problems: Shepp-Logan-shaped phantoms and uniform random fields)",
        "config": {"workload": name, "samples": samples, "problems": len(specs)},
        **out, "tuning": [{"tile_u": t, "view_group": v} for t, v in tunings],
        "clocks": clocks, "gpu_launches": counts[2] * args.steps,
    }), flush=True)


def run_cgls(args):
    """The differentiation form: 256^3 Shepp-Logan-shaped phantom, 256^2
    detector, 180 views (10 degree half-angle).  Times (a) 30 CGLS
    iterations (one forward and one adjoint each, plus the solver's dot
    products and updates) and (b) a gradient step through the autograd
    function (forward, squared-error loss, backward = adjoint).  The data
    are the GPU projections of the phantom itself: this times the solver;
    reconstruction quality from closed-form analytic projections is the
    tests' job.  One JSON line; ``value`` is (a) in Gsamples/s."""
    import torch
    from paper_1609_00958_gb300 import build as libbuild
    libbuild.build()
    import paper_1609_00958_gb300 as gjp
    from paper_1609_00958_gb300.autograd import project
    from paper_1609_00958_gb300.recon import cgls
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    vg, cg = synth.c4_geometry()
    g = gjp.Geometry.from_cone(cg)
    x_true = torch.from_numpy(synth.voxelize(vg, supersample=2)).to(dev)
    b = gjp.forward(x_true, g, vg.h)
    samples = int(sample_counts(vg, cg).sum())
    n_iter = 30
    # warm-up with the same arguments: the first call of each torch kernel of
    # the solver's bookkeeping can include its JIT compilation (seconds)
    cgls(b, g, vg.n, 2, vg.h, x_true=x_true)
    torch.cuda.synchronize()
    with ClockSampler(gpu_id_for_smi(0)) as clk:
        t0 = time.perf_counter()
        x, hist = cgls(b, g, vg.n, n_iter, vg.h, x_true=x_true)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    clocks = clk.summary()
    ms_iter = 1e3 * wall / n_iter
    # a training-style step: loss on the projections, gradient into the volume
    vol = torch.zeros(vg.n, device=dev, requires_grad=True)

    def grad_step():
        vol.grad = None
        loss = 0.5 * torch.sum((project(vol, g, vg.h) - b) ** 2)
        loss.backward()
        return loss

    for _ in range(max(1, args.warmup)):
        grad_step()
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        grad_step()
    e.record()
    torch.cuda.synchronize()
    ms_grad = a.elapsed_time(e) / args.steps
    pick = [0, 10, 20, 30]
    print(json.dumps({
        "metric": METRIC + " (differentiation form)", "value": round(2 * samples / (ms_iter * 1e-3) / 1e9, 2),
        "unit": UNIT, "n_gpus": 1, "steps": n_iter, "warmup": 2, "ms_per_step": round(ms_iter, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (Shepp-Logan-shaped phantom, its own GPU projections)",
        "config": {"workload": "differentiation form: 256^3 phantom, 256^2 detector, 180 views, 10 deg half-angle, "
                               "30 CGLS iterations", "samples_per_projection": samples},
        "cgls": {"ms_per_iteration": round(ms_iter, 3), "iterations": n_iter,
                 "residual": {str(k): float(f"{hist.residual[k]:.4e}") for k in pick if k < len(hist.residual)},
                 "rmse": {str(k): float(f"{hist.rmse[k]:.4e}") for k in pick if k < len(hist.rmse)}},
        "autograd_step_ms": round(ms_grad, 3),
        "clocks": clocks, "gpu_launches": 2 * n_iter,
    }), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.ncu_summary:
        rec = ncu_summary(args.ncu_summary, args.ncu_views, args.ncu_command, args.n, args.views)
        with open(os.path.join(ROOT, COUNTERS), "w") as f:
            json.dump(rec, f, indent=1)
            f.write("\n")
        print(json.dumps({k: sorted(v) for k, v in rec["kernels"].items()}))
    elif args.oracle_leg:
        run_oracle_leg(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "cgls":
        run_cgls(args)
    else:
        run_gjp(args)


if __name__ == "__main__":
    main()
