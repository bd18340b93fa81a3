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

    python bench.py [--steps K] [--warmup W] [--impl reference]
    torchrun --nproc-per-node N bench.py --gpus N     (weak scaling: every
        rank projects its own copy of the workload; no collective on the
        data path)
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
    p.add_argument("--workload", choices=["step", "batch"], default="step",
                   help="step: the 512^3 hot-path step (default); batch: the 16-problem batching workload")
    p.add_argument("--n", type=int, default=512, help="volume edge (workload is defined at 512)")
    p.add_argument("--views", type=int, default=360)
    p.add_argument("--first-views", type=int, default=0,
                   help="keep only the first K views of the --views geometry (small profiling captures)")
    p.add_argument("--forward-path", choices=["auto", "gather", "slab", "prefetch", "texture", "hwlin"],
                   default="auto", help="forward kernel family of the step (profiling other families)")
    p.add_argument("--tile-u", type=int, default=None, help="detector columns per block (library default if unset)")
    p.add_argument("--view-group", type=int, default=None, help="views issued together (library default if unset)")
    p.add_argument("--content", choices=["random", "phantom"], default="random")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="bound of the CPU baseline sample")
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


def dram_traffic(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or
    None if absent or taken on different kernel sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for rel, sha in d["sources"].items():
            with open(os.path.join(ROOT, rel), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != sha:
                    return None
        e = d["kernels"].get(kernel)
        return None if e is None else float(e["bytes_per_launch"])
    except (OSError, KeyError, ValueError, TypeError):
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


def run_gjp(args):
    import torch
    from paper_1609_00958_gb300 import build as libbuild
    libbuild.build()
    import paper_1609_00958_gb300 as gjp
    from paper_1609_00958_gb300 import dist as gdist

    rank, world, local = dist_setup(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    vg, cg, wname = workload(args)
    geom = gjp.Geometry.from_cone(cg)
    if args.tile_u is not None or args.view_group is not None:
        tu, vgp = geom.launch
        geom.set_launch(args.tile_u or tu, args.view_group or vgp)

    vol_np = make_volume(args, vg, seed=rank)
    vol32 = torch.from_numpy(vol_np).to(dev)
    # the texture unit has no bfloat16 format: the texture families store the 16-bit form as float16
    tex = args.forward_path in ("texture", "hwlin")
    vol16 = vol32.to(torch.float16 if tex else torch.bfloat16)
    k16 = "forward_f16" if tex else "forward_bf16"
    proj32 = torch.empty(cg.n_views, cg.nv, cg.nu, device=dev)
    proj16 = torch.empty_like(proj32)
    back = torch.empty(vg.n, device=dev)
    stream = torch.cuda.current_stream(dev)

    counts = sample_counts(vg, cg)
    samples_per_kernel = int(counts.sum())
    foot = np.array(gjp.footprint_voxels(geom, vg.n, vg.h, device=dev), dtype=np.float64)
    proj_bytes = 4.0 * cg.n_views * cg.nu * cg.nv
    alg_bytes = {
        "forward_f32": 4.0 * foot.sum() + proj_bytes,
        k16: 2.0 * foot.sum() + proj_bytes,
        "adjoint_f32": 8.0 * foot.sum() + proj_bytes,    # read-modify-write of each touched voxel per view
    }

    names = ["forward_f32", k16, "adjoint_f32"]

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        gjp.forward(vol32, geom, vg.h, out=proj32, path=args.forward_path)
        if ev is not None:
            ev[1].record(stream)
        gjp.forward(vol16, geom, vg.h, out=proj16, path=args.forward_path)
        if ev is not None:
            ev[2].record(stream)
        gjp.adjoint(proj32, geom, vg.n, vg.h, out=back)
        if ev is not None:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
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
    samples_per_step = 3 * samples_per_kernel
    job_samples_per_step = gdist.sum_over_ranks(samples_per_step)     # every rank projects its own workload
    value = job_samples_per_step / (ms_per_step * 1e-3) / 1e9

    hbm, peak_kind = peaks()
    kernels = {}
    for n in names:
        ms = per_kernel_ms[n]
        gbs = alg_bytes[n] / (ms * 1e-3) / 1e9
        kernels[n] = {"ms": round(ms, 4), "gsamples_s": round(samples_per_kernel / (ms * 1e-3) / 1e9, 2),
                      "algorithmic_gb": round(alg_bytes[n] / 1e9, 4), "achieved_gbs": round(gbs, 1),
                      "frac_of_" + peak_kind + "_hbm": round(gbs / hbm, 4),
                      "paper_logical_gbs": round(samples_per_kernel * (8 if "16" in n and "f32" not in n else 16)
                                                 / (ms * 1e-3) / 1e9, 1)}
    dominant = max(names, key=lambda n: per_kernel_ms[n])
    kmap = {"forward_f32": "gjp_forward_kernel<float", "forward_bf16": "gjp_forward_kernel<__nv_bfloat16",
            "forward_f16": "gjp_forward_tld4_kernel<__half",
            "adjoint_f32": "gjp_adjoint_combine_kernel<int"}
    traffic = dram_traffic(kmap[dominant])
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": kernels[dominant]["achieved_gbs"],
                "peak": hbm, "peak_kind": peak_kind + " (copy, MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured"
                else "fallback", "unit": "GB/s",
                "frac": round(kernels[dominant]["achieved_gbs"] / hbm, 4), "traffic": traffic}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, gjp, geom, vg, cg, vol_np, dev, stream, job_samples_per_step)

    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (weights/accumulation); volume storage f32 and bf16",
        "data": "synthetic (seeded uniform [0,1) random field)" if args.content == "random"
        else "synthetic (Shepp-Logan-shaped phantom, project-owned ellipsoids)",
        "config": {"workload": wname, "volume": list(vg.n), "detector": [cg.nv, cg.nu], "views": cg.n_views,
                   "launch": {"tile_u": geom.launch[0], "view_group": geom.launch[1]},
                   "forward_path": args.forward_path,
                   "step": "forward f32 + forward bf16 + adjoint f32", "samples_per_kernel": samples_per_kernel,
                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}"},
        "kernels": kernels, "roofline": roofline, "clocks": clocks,
        "gpu_launches": 3 * args.steps,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample_views = list(range(0, cg.n_views, max(1, cg.n_views // 36)))
        gpu_views = {v: (proj32[v].cpu().numpy(), proj16[v].cpu().numpy()) for v in sample_views}
        result["cpu_baseline"] = cpu_baseline(args, vg, cg, vol_np, counts, budget_s=args.cpu_seconds,
                                              gpu_views=gpu_views)
        if "error_vs_oracle" in result["cpu_baseline"]:
            result["error_vs_oracle"] = result["cpu_baseline"]["error_vs_oracle"]
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_e2e(args, gjp, geom, vg, cg, vol_np, dev, stream, job_samples_per_step):
    """Same step through the public API with host buffers.  Every step copies
    its inputs (float32 and bfloat16 volume) from pinned host memory to the
    GPU and its results (both projections and the adjoint volume) back to
    pinned host memory.  Steps are pipelined the way a caller of the
    stream-ordered API would run them: copies in, kernels and copies out
    each on their own stream, with two device buffer sets, so step k+1's
    input copy overlaps step k's kernels; with one event per tensor each
    kernel waits only for its own input and each result is copied out as
    soon as its kernel ends.  The timed region covers all steps, every copy
    included, and ends when the last results are on the host."""
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
    bi = h_vol32.numel() * 4 + h_vol16.numel() * 2
    bo = (2 * int(np.prod(pshape)) + int(np.prod(vg.n))) * 4
    return {"value": round(job_samples_per_step / (wall / args.steps) / 1e9, 3), "unit": UNIT,
            "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo),
            "ms_per_step": round(1e3 * wall / args.steps, 3),
            "pipelining": "copies in / kernels / copies out on three streams, two device buffer sets, "
                          "one event per tensor"}


# --- CPU oracle (baseline leg and reference arm) ----------------------------------

def oracle_step(oracle, vg, cg, vol_np, vol_bf16w, view, threads, counts, keep=None):
    """One view of the step on the oracle (forward f32, forward of the
    bfloat16-stored values, adjoint); `keep` collects the two projections."""
    sub = cg.subset([view])
    t0 = time.perf_counter()
    p = oracle.forward(vol_np, vg, sub, threads=threads)
    p16 = oracle.forward(vol_bf16w, vg, sub, threads=threads)
    oracle.adjoint(p, vg, sub, threads=threads, max_bytes=16e9)
    dt = time.perf_counter() - t0
    if keep is not None:
        keep[view] = (p[0], p16[0])
    return dt, 3 * int(counts[view])


def bf16_widened(vol_np):
    """Round-to-nearest-even float32 -> bfloat16, widened back to float32
    (the values a bfloat16 volume stores)."""
    import torch
    return torch.from_numpy(vol_np).to(torch.bfloat16).float().numpy()


def cpu_baseline(args, vg, cg, vol_np, counts, budget_s, gpu_views=None):
    """The oracle timed on the host cores over a time-bounded sample of
    views.  With `gpu_views` (view -> (float32 projection, bfloat16
    projection) from the timed GPU step), the same oracle projections also
    give the GPU results' error on those views: max and RMS |gpu - oracle|
    relative to the oracle maximum, against the float32 volume and, for
    bfloat16 storage, also against the stored (rounded) values."""
    import oracle
    threads = os.cpu_count() or 1
    vol_w = bf16_widened(vol_np)
    views = list(range(0, cg.n_views, max(1, cg.n_views // 36)))
    t_tot, s_tot, used, kept = 0.0, 0, [], {}
    for v in views:
        dt, s = oracle_step(oracle, vg, cg, vol_np, vol_w, v, threads, counts, keep=kept)
        t_tot += dt
        s_tot += s
        used.append(v)
        if t_tot >= budget_s:
            break
    out = {"value": round(s_tot / t_tot / 1e9, 5), "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"FP64 oracle (OpenMP, {threads} threads) on {len(used)} of {cg.n_views} views "
                     f"(views {used[0]}..{used[-1]} step {views[1] - views[0] if len(views) > 1 else 0}): "
                     "forward f32 + forward bf16-stored + adjoint per view, same volume and geometry"}
    if gpu_views:
        def err(gpu, ref):
            d = np.abs(np.asarray(gpu, np.float64) - ref)
            m = max(float(np.abs(ref).max()), 1e-30)
            return {"max_rel": float(f"{d.max() / m:.3e}"), "rms_rel": float(f"{np.sqrt(np.mean(d * d)) / m:.3e}")}
        e32 = [err(gpu_views[v][0], kept[v][0]) for v in used]
        e16 = [err(gpu_views[v][1], kept[v][0]) for v in used]
        e16s = [err(gpu_views[v][1], kept[v][1]) for v in used]
        worst = lambda es: {"max_rel": max(e["max_rel"] for e in es),
                            "rms_rel": float(f"{np.sqrt(np.mean([e['rms_rel'] ** 2 for e in es])):.3e}")}
        out["error_vs_oracle"] = {
            "views": used, "forward_f32": worst(e32), "forward_bf16": worst(e16),
            "forward_bf16_vs_stored_values": worst(e16s),
            "bounds": {"f32": 1e-5, "bf16": 5e-3, "bf16_vs_stored_values": 1e-5}}
    return out


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    vg, cg, wname = workload(args)
    vol_np = make_volume(args, vg, seed=0)
    vol_w = bf16_widened(vol_np)
    counts = sample_counts(vg, cg)
    threads = os.cpu_count() or 1
    stride = max(1, cg.n_views // max(1, args.steps + args.warmup))
    order = [(k * stride) % cg.n_views for k in range(args.steps + args.warmup)]
    for v in order[:args.warmup]:
        oracle_step(oracle, vg, cg, vol_np, vol_w, v, threads, counts)
    times, samples = [], 0
    for v in order[args.warmup:]:
        dt, s = oracle_step(oracle, vg, cg, vol_np, vol_w, v, threads, counts)
        times.append(dt)
        samples += s
    total = sum(times)
    value = samples / total / 1e9
    sample = (f"one view per step (forward f32 + forward bf16-stored + adjoint), views {order[args.warmup:]}, "
              f"FP64 oracle with {threads} OpenMP threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * total / max(1, len(times)), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded uniform [0,1) random field)" if args.content == "random" else "synthetic phantom",
        "config": {"workload": wname, "volume": list(vg.n), "detector": [cg.nv, cg.nu], "views": cg.n_views,
                   "step": "one view: forward f32 + forward bf16 + adjoint (oracle)"},
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_batch(args):
    """The batching workload: 16 independent problems (synth.c5_manifest)
    projected (a) by 16 separate gjp_forward launches, (b) by one persistent
    batched launch with the geometries' default launch shapes, (c) the same
    after gjp_batch_autotune, (d) (c) replayed from a CUDA graph.  One JSON
    line; `value` is (d) in Gsamples/s."""
    import torch
    from paper_1609_00958_gb300 import build as libbuild
    libbuild.build()
    import paper_1609_00958_gb300 as gjp
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    specs = synth.c5_manifest()
    items, samples = [], 0
    for sp in specs:
        vg, cg = sp.geometry()
        vol_np = (synth.voxelize(vg, supersample=2) if sp.content == "phantom"
                  else synth.random_field(vg.n, seed=sp.seed))
        vol = torch.from_numpy(vol_np).to(dev).to(getattr(torch, sp.dtype))
        g = gjp.Geometry.from_cone(cg)
        items.append((vol, g, vg.h, None, torch.empty(g.proj_shape, device=dev)))
        samples += int(sample_counts_device(vg, cg, dev).sum())
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        for _ in range(args.warmup):
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

    batch = gjp.Batch(items)
    ms_sep = timed(separate, args.steps)
    ms_batch = timed(batch.forward, args.steps)
    tunings = batch.autotune(reps=2)
    ms_tuned = timed(batch.forward, args.steps)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.forward()
    with ClockSampler(gpu_id_for_smi(0)) as clk:
        ms_graph = timed(graph.replay, args.steps)
    clocks = clk.summary()
    gsps = lambda ms: round(samples / (ms * 1e-3) / 1e9, 2)
    print(json.dumps({
        "metric": METRIC + " (batching form)", "value": gsps(ms_graph), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_graph, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (weights/accumulation); volume storage f32 and bf16",
        "data": "synthetic (16 seeded problems: Shepp-Logan-shaped phantoms and uniform random fields)",
        "config": {"workload": "batching form: 16 problems, 96^3..768^3 and 512x512x128, 90..720 views, "
                               "128^2..768^2 detectors, 5..15 deg half-angles (synth.c5_manifest)",
                   "samples": samples, "problems": len(items)},
        "ms": {"separate_launches": round(ms_sep, 3), "batched": round(ms_batch, 3),
               "batched_autotuned": round(ms_tuned, 3), "batched_autotuned_graph": round(ms_graph, 3)},
        "gsamples_s": {"separate_launches": gsps(ms_sep), "batched": gsps(ms_batch),
                       "batched_autotuned": gsps(ms_tuned), "batched_autotuned_graph": gsps(ms_graph)},
        "speedup_vs_separate": round(ms_sep / ms_graph, 3),
        "tuning": [{"tile_u": t, "view_group": v} for t, v in tunings],
        "clocks": clocks, "gpu_launches": args.steps,
    }), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_gjp(args)


if __name__ == "__main__":
    main()
