#!/usr/bin/env python
"""Benchmark of the 3DHEB bundling iteration on GB300.

A step is one full iteration of the loop (resample, histogram, box passes,
layer mix, advection with the halving step, Laplacian smoothing) over one
synthetic graph resident in HBM. The default workload is the criteria-driven
configuration the headline metric is quoted on: 5M edges between nodes of a
perturbed 2048 x 2048 lattice, 8 k-means groups on (origin, destination),
an 8 x 1024 x 1024 int64 histogram stack, r = 12, 4 passes, <= 64 samples per
edge (delta = 2 px). Metric: sample-point updates per second (points advected
per iteration x iterations / time).

Prints one JSON line. `--impl reference` times the FP64 CPU oracle instead
(bounded sample of the same workload, host cores).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sample_point_updates_per_s"
UNIT = "updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lattice",
                    choices=["lattice", "clustered", "small", "batch"])
    ap.add_argument("--graphs", type=int, default=64, help="graphs in the batch workload")
    ap.add_argument("--edges", type=int, default=0, help="override the edge count (testing)")
    ap.add_argument("--rho", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--split", action="store_true",
                    help="one graph's edges split over the ranks, histograms all-reduced each "
                         "iteration (strong scaling); default: an independent graph per rank")
    return ap.parse_args()


def make_workload(name, edges, seed_offset=0):
    from paper_1504_02687_gb300 import synth

    if name == "lattice":
        kw = dict(seed=synth.SEED_BASE + 3 + seed_offset)
        if edges:
            kw["n_edges"] = edges
        return synth.lattice_pattern(**kw)
    if name == "clustered":
        kw = dict(seed=synth.SEED_BASE + 2 + seed_offset)
        if edges:
            kw["n_edges"] = edges
        return synth.clustered(**kw)
    return synth.small(seed=synth.SEED_BASE + 1 + seed_offset)


def describe(w, rho):
    W, H = w.grid
    return {
        "workload": (f"{w.name}: {w.n_edges} edges, {w.n_groups} groups, {w.n_groups}x{H}x{W} "
                     f"histogram stack, r={w.radius}, k={w.passes}, "
                     + (f"{w.n_fixed} samples/edge" if w.n_fixed else
                        f"<= {w.n_max} samples/edge (delta={w.delta} px)")),
        "edges": w.n_edges, "groups": w.n_groups, "grid": [W, H], "radius": w.radius,
        "passes": w.passes, "n_max": w.n_max, "n_fixed": w.n_fixed, "rho_dtype": rho,
        "l2": "inputs larger than L2 (point buffers of the iteration exceed 129 MB)",
    }


def params_of(w, rho):
    import paper_1504_02687_gb300 as pkg

    return pkg.default_params(grid_w=w.grid[0], grid_h=w.grid[1], radius=w.radius,
                              passes=w.passes, n_fixed=w.n_fixed, n_max=w.n_max,
                              delta_px=w.delta,
                              rho_dtype={"f32": 0, "bf16": 1, "f16": 2}[rho])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(index)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons, busy = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz, smax, pw = float(f[1]), float(f[2]), float(f[3])
            except ValueError:
                continue
            sm.append(mhz)
            busy.append((pw, mhz))
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": sorted(reasons)}
        # under load: the samples at or above the median power draw
        pw_med = statistics.median(p for p, _ in busy)
        loaded = [m for p, m in busy if p >= pw_med] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(kind, N, E, GC, b_sum, b_rho, MC=None):
    """Bytes one launch of each kernel must move (its roofline numerator). GC: histogram
    cells (groups x H x W); MC: entries of the padded density map (groups x (H+4) x (W+4)).

    advect+resample: read and write every point (8 B each way), per-edge count in and out,
    group and weight (16 B), one read of the density stack, the histogram written once.
    """
    if kind == "advect_resample":
        return 16 * N + 16 * E + GC * b_rho + 4 * GC
    if kind == "resample":
        return 16 * N + 16 * E + 4 * GC
    if kind == "advect":
        return 16 * N + 12 * E + GC * b_rho
    if kind == "rowbox":
        return GC * (4 + b_sum)  # the histogram once (its copies are workspace) + the output
    if kind == "colbox":
        return 2 * GC * b_sum
    if kind == "mix_quads":
        # the sums once, the density quad map (four densities per quad) written once
        return GC * b_sum + 4 * (GC if MC is None else MC) * b_rho
    return 0


def kernel_source_hash():
    """Hash of the step kernel's code (its sources without // comments and blank lines: a
    comment edit does not change the kernel the counters were taken on)."""
    import re

    h = hashlib.sha256()
    for f in ("k_points.cu", "density.cuh", "internal.cuh"):  # the sources of k_step
        with open(os.path.join(ROOT, "paper_1504_02687_gb300", "csrc", f)) as fh:
            for line in fh:
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def measured_traffic(kind, algorithmic):
    """DRAM bytes per launch from the committed ncu capture, if the step kernel is unchanged:
    the captured launch's DRAM bytes per algorithmic byte, times this run's algorithmic bytes
    per launch. The capture is taken on the 1M-edge lattice case (same 8 x 1024^2 stack) and
    scaled to a full launch by the points it processes: traffic grows in proportion to them."""
    path = os.path.join(ROOT, "profiles", "k_step_lattice-1M-8groups.md")
    try:
        with open(path) as fh:
            text = fh.read()
        d = json.loads(text.split("```json", 1)[1].split("```", 1)[0])
    except Exception:
        return None
    ent = d.get(kind)
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return ent["dram_bytes_per_launch"] / ent["algorithmic_bytes_per_launch"] * algorithmic


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_baseline(w, sample_edges, iters=1):
    """The FP64 oracle as it stands, single-threaded, `iters` iterations on the first
    `sample_edges` edges of the same graph (same grid, groups, filter)."""
    import oracle

    oracle.build()
    E = min(sample_edges, w.n_edges)
    W_, H_, mp, sp, dp = oracle.grid_map(w.src_xy[:E], w.dst_xy[:E], w.grid[0], w.grid[1],
                                         margin=w.radius)
    off, xy = oracle.straight_polylines(sp, dp)
    prm = oracle.Params(radius=w.radius, passes=w.passes, n_fixed=w.n_fixed, n_max=w.n_max,
                        delta=w.delta)
    t0 = time.perf_counter()
    n = 0
    for it in range(iters):
        res = oracle.run(off, xy, w.group[:E], None if w.weight is None else w.weight[:E],
                         w.n_groups, H_, W_, prm, it, 1)
        off, xy = res.off, res.xy
        n += int(res.off[-1])  # points advected by this iteration
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": (f"{iters} iteration(s) of the FP64 oracle from straight edges on the first "
                       f"{E} of {w.n_edges} edges ({n} sample-point updates, full "
                       f"{w.n_groups}x{H_}x{W_} grid), {dt:.1f} s, single-threaded")}


def _oracle_job(job):
    """One FP64 oracle run in a worker process (spawned: no CUDA state is inherited)."""
    import oracle

    off, xy, group, weight, G, H, W, prm, iters = job
    r = oracle.run(off, xy, group, weight, G, H, W, oracle.Params(**prm), 0, iters)
    return r.off, r.xy


def precision_forms(w, pkg, stream, sample_edges=200_000, iters=30):
    """Precision form on a bounded sample of the workload (its first `sample_edges` edges on
    the full grid with the full workload's groups and filter): the GPU run with the density
    stack stored in FP32, BF16 and FP16 (histograms and sums integer, positions and gradients
    FP32) against the FP64 oracle from the same FP32 start after `iters` iterations. Errors
    are in units of the layout extent, measured on the polylines re-spaced to 9 points
    (resampled counts can differ after a near-tie), beside the FP64 method's own drift when
    its start moves by +-1 FP32 ulp (two seeds). The oracle runs in spawned worker
    processes after every GPU measurement of the line is done."""
    import multiprocessing as mp_

    import numpy as np

    import oracle

    oracle.build()
    E = min(sample_edges, w.n_edges)
    W_, H_ = w.grid
    g = w.group[:E]
    wt = None if w.weight is None else w.weight[:E]
    out = {"sample": f"first {E} of {w.n_edges} edges, {w.n_groups}x{H_}x{W_} grid, "
                     f"{iters} iterations", "forms": {}}
    start = None
    got = {}
    for name in ("f32", "bf16", "f16"):
        prm = params_of(w, name)
        ctx = pkg.bundle_init(prm, w.src_xy[:E], w.dst_xy[:E], g, w.n_groups, wt, stream=stream)
        try:
            off0, P0 = pkg.bundle_fetch(ctx, pixels=True)
            if start is None:
                start = (off0.astype(np.int64), P0.astype(np.float64), prm)
            pkg.bundle_iterate(ctx, iters)
            o, x = pkg.bundle_fetch(ctx, pixels=True)
            got[name] = (o.astype(np.int64), x.astype(np.float64))
        finally:
            pkg.bundle_destroy(ctx)
    off0, P0, prm = start
    op = dict(radius=prm.radius, passes=prm.passes, alpha_num=prm.alpha_num,
              alpha_den=prm.alpha_den, h_max_sigmas=prm.h_max_sigmas, lam=prm.lambda_,
              n_fixed=prm.n_fixed, n_max=prm.n_max, delta=float(prm.delta_px),
              beta=float(prm.laplace_beta), eps=float(prm.eps), tries=prm.step_tries)

    def perturbed(seed):
        rng = np.random.default_rng(seed)
        x32 = P0.astype(np.float32)
        d = rng.integers(-1, 2, x32.shape)
        up, dn = np.nextafter(x32, np.float32(1e9)), np.nextafter(x32, np.float32(-1e9))
        return np.where(d > 0, up, np.where(d < 0, dn, x32)).astype(np.float64)

    jobs = [(off0, xy, g, wt, w.n_groups, H_, W_, op, iters)
            for xy in (P0, perturbed(0), perturbed(1))]
    t0 = time.perf_counter()
    with mp_.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_oracle_job, jobs)
    out["oracle_seconds_wall"] = time.perf_counter() - t0
    ref_off, ref_xy = res[0]
    extent = float(max(W_, H_))
    o2, r2 = oracle.resample(ref_off, ref_xy, 9, 64, 2.0)

    def err(off, xy):
        o1, r1 = oracle.resample(off, xy, 9, 64, 2.0)
        e = np.hypot(*(r1 - r2).T) / extent
        return {"max": float(e.max()), "rms": float(np.sqrt((e ** 2).mean()))}

    for name, (o, x) in got.items():
        out["forms"][name] = {**err(o, x), "same_counts": bool(np.array_equal(o, ref_off))}
    out["fp64_ulp_envelope"] = [err(o, x) for o, x in res[1:]]
    out["units"] = "fraction of the layout extent (max(W, H) px)"
    return out


def run_reference(args):
    """The oracle arm: each step is one oracle iteration on a bounded sample of the workload."""
    import numpy as np

    import oracle

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "batch":
        # the batch's sample: its first graph (one graph of the batch is one oracle problem)
        from paper_1504_02687_gb300 import synth

        w = synth.batch(n_graphs=args.graphs)[0]
    else:
        w = make_workload(args.workload, args.edges)
    oracle.build()
    # a bounded sample: 500k edges keep the default 3 + 20 oracle iterations to a few
    # minutes on one core
    E = min(w.n_edges, 500_000)
    W_, H_, mp, sp, dp = oracle.grid_map(w.src_xy[:E], w.dst_xy[:E], w.grid[0], w.grid[1],
                                         margin=w.radius)
    off, xy = oracle.straight_polylines(sp, dp)
    prm = oracle.Params(radius=w.radius, passes=w.passes, n_fixed=w.n_fixed, n_max=w.n_max,
                        delta=w.delta)
    g = w.group[:E]
    wt = None if w.weight is None else w.weight[:E]
    it = 0
    for _ in range(args.warmup):
        r = oracle.run(off, xy, g, wt, w.n_groups, H_, W_, prm, it, 1)
        off, xy, it = r.off, r.xy, it + 1
    pts = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pts += int(off[-1]) if prm.n_fixed else 0
        r = oracle.run(off, xy, g, wt, w.n_groups, H_, W_, prm, it, 1, keep_last=True)
        if not prm.n_fixed:
            pts += int(r.res_off[-1])
        off, xy, it = r.off, r.xy, it + 1
    dt = time.perf_counter() - t0
    value = pts / dt
    cfg = describe(w, "f64")
    if E < w.n_edges:
        # the line names what the oracle times: the first E edges of the workload's graph
        cfg["workload"] = (f"{E}-edge sample (the first {E} of {w.n_edges} edges) of "
                           + cfg["workload"])
        cfg["sample_edges"] = E
    sample = (f"{args.steps} oracle iterations on the first {E} of {w.n_edges} edges of the "
              f"workload, single-threaded FP64")
    if args.workload == "batch":
        cfg["workload"] = f"batch of {args.graphs} graphs; the oracle runs its first graph"
        sample = f"{args.steps} oracle iterations on graph 0 of the batch ({w.name}), FP64"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def reduce_over_ranks(dist, ms: float, updates: float, device=None):
    """Whole-job figures over ranks: the slowest rank's time and the sum of the updates all
    ranks made (independent graphs per rank, weak scaling). `device` is where the collective's
    tensors live (CUDA for NCCL, CPU for gloo)."""
    if dist is None:
        return ms, updates
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([updates], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_ours(args):
    import numpy as np
    import torch

    import paper_1504_02687_gb300 as pkg
    from paper_1504_02687_gb300 import build as lib_build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev_index = torch.cuda.current_device()
    if rank == 0:
        lib_build.build()
    if dist:
        dist.barrier()
    lib_build.build()
    # every rank bundles its own graph of the same configuration (independent problems)
    w = make_workload(args.workload, args.edges, seed_offset=rank * 1000)
    # a dedicated stream: the library launches on it and the timing events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    p = params_of(w, args.rho)
    ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight, stream=stream)
    info = pkg.bundle_get_info(ctx)
    GC = info.n_groups * info.grid_w * info.grid_h
    MC = info.n_groups * (info.grid_w + 3) * (info.grid_h + 3)
    b_sum = info.sum_bits // 8
    b_rho = 4 if args.rho == "f32" else 2

    clocks = ClockSampler(dev_index)
    pkg.bundle_iterate(ctx, args.warmup)
    pkg.bundle_sync(ctx)
    done0 = pkg.bundle_get_info(ctx).points_processed
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    pkg.bundle_iterate(ctx, args.steps)  # the production path (CUDA graphs)
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = t_start.elapsed_time(t_end)
    info = pkg.bundle_get_info(ctx)
    updates = info.points_processed - done0
    # per-kernel CUDA-event times for the roofline: a second context run through the same
    # iterations with per-launch events (separate launches instead of graphs)
    pkg.bundle_destroy(ctx)
    ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight, stream=stream)
    pkg.bundle_iterate(ctx, args.warmup)
    pkg.bundle_sync(ctx)
    done1 = pkg.bundle_get_info(ctx).points_processed
    pkg.bundle_profile_enable(ctx, True)
    pkg.bundle_profile_read(ctx)  # clears
    pkg.bundle_iterate(ctx, args.steps)
    prof = pkg.bundle_profile_read(ctx)
    pkg.bundle_profile_enable(ctx, False)
    clk = clocks.stop()
    prof_updates = pkg.bundle_get_info(ctx).points_processed - done1
    E = info.n_edges
    N_avg = updates / max(args.steps, 1)
    ms, total_updates = reduce_over_ranks(dist, ms, float(updates), device="cuda")
    value = total_updates / (ms / 1e3)

    N_prof = prof_updates / max(args.steps, 1)
    kern = {k: v for k, v in prof.items() if v[1] > 0}
    # kernels of the timed call: the profiled pass launches the same kernels (+1 counter
    # kernel per iteration and 1 to set the counter), inside graphs in the timed call
    launches = sum(n for k, (t, n) in kern.items() if k != "hist_clear") + args.steps + 1
    dom = max((k for k in kern if k != "hist_clear"), key=lambda k: kern[k][0])
    dom_ms = kern[dom][0] / kern[dom][1]
    dom_bytes = algorithmic_bytes(dom, N_prof, E, GC, b_sum, b_rho, MC)
    peak, peak_src = peaks()
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    traffic = measured_traffic(dom, dom_bytes)
    per_kernel = {}
    for k, (tms, n) in kern.items():
        b = algorithmic_bytes(k, N_prof, E, GC, b_sum, b_rho, MC)
        per_kernel[k] = {"launches": n, "ms_per_launch": tms / n,
                         "share": tms / max(sum(v[0] for v in kern.values()), 1e-9),
                         "algorithmic_gbs": (b / (tms / n / 1e3) / 1e9) if b else None}
    step_bytes = (algorithmic_bytes("advect_resample", N_avg, E, GC, b_sum, b_rho)
                  + algorithmic_bytes("rowbox", N_avg, E, GC, b_sum, b_rho)
                  + algorithmic_bytes("colbox", N_avg, E, GC, b_sum, b_rho)
                  + algorithmic_bytes("mix_quads", N_avg, E, GC, b_sum, b_rho, MC))
    pkg.bundle_destroy(ctx)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded generator shaped like the paper's graphs)",
        "config": {**describe(w, args.rho), "parallelism": f"{world} independent graphs"
                   if world > 1 else "single GPU", "points_per_step": N_avg},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_src} hbm_gbs", "algorithmic_bytes_per_launch": dom_bytes,
                     "ms_per_launch": dom_ms},
        "step_roofline": {"algorithmic_bytes": step_bytes,
                          "achieved_gbs": step_bytes / (ms / args.steps / 1e3) / 1e9,
                          "frac": step_bytes / (ms / args.steps / 1e3) / 1e9 / peak},
        "kernels": per_kernel,
        "gpu_launches": launches,
        "clocks": clk,
    }

    if not args.no_variants and world == 1 and args.rho == "f32":
        def timed_variant(wl, prm, steps):
            c2 = pkg.bundle_init(prm, wl.src_xy, wl.dst_xy, wl.group, wl.n_groups, wl.weight,
                                 stream=stream)
            pkg.bundle_iterate(c2, max(args.warmup, 3))
            pkg.bundle_sync(c2)
            d0 = pkg.bundle_get_info(c2).points_processed
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pkg.bundle_iterate(c2, steps)
            b.record(stream)
            torch.cuda.synchronize()
            m2 = a.elapsed_time(b)
            u2 = pkg.bundle_get_info(c2).points_processed - d0
            pkg.bundle_destroy(c2)
            return {"value": u2 / (m2 / 1e3), "ms_per_step": m2 / steps}

        var = {"bf16": timed_variant(w, params_of(w, "bf16"), args.steps),
               "fp16": timed_variant(w, params_of(w, "f16"), args.steps)}
        # KDEEB's fixed step (Sec. 3.3) on the same workload: the cost of the density test
        pf = params_of(w, args.rho)
        pf.flags = pkg.FLAG_FIXED_STEP
        var["fixed_step"] = timed_variant(w, pf, args.steps)
        # Bresenham segment histogram (Eq. 1 as rasterised in Sec. 4) against the point splat
        # on the 1M-edge spatial-only workload (its int64 sums hold the segment mass; the
        # 8-group stack with r = 12, k = 4 does not)
        wc = make_workload("clustered", 0)
        pc = params_of(wc, args.rho)
        ps = params_of(wc, args.rho)
        ps.flags = pkg.FLAG_SEGMENT_HIST
        var["segment_hist"] = {"workload": wc.name, **timed_variant(wc, ps, args.steps),
                               "point_splat": timed_variant(wc, pc, args.steps)}
        # general interaction matrix (Eq. 3, Sec. 3.2): an ordinal 8 x 8 matrix on the same
        # workload as the headline, against Eq. 4's mix
        G = w.n_groups
        idx = np.arange(G)
        num = (4 - np.minimum(np.abs(idx[:, None] - idx[None, :]), 5)).astype(np.int64)
        cm = pkg.bundle_init(params_of(w, args.rho), w.src_xy, w.dst_xy, w.group, w.n_groups,
                             w.weight, stream=stream)
        pkg.bundle_set_interaction(cm, num, 4)
        pkg.bundle_iterate(cm, max(args.warmup, 3))
        pkg.bundle_sync(cm)
        d0 = pkg.bundle_get_info(cm).points_processed
        torch.cuda.synchronize()
        ea = torch.cuda.Event(enable_timing=True)
        eb = torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        pkg.bundle_iterate(cm, args.steps)
        eb.record(stream)
        torch.cuda.synchronize()
        mm = ea.elapsed_time(eb)
        var["interaction_matrix"] = {
            "value": (pkg.bundle_get_info(cm).points_processed - d0) / (mm / 1e3),
            "ms_per_step": mm / args.steps, "matrix": f"ordinal {G}x{G}, M(l,b) = (4 - min(|l-b|, 5)) / 4"}
        pkg.bundle_destroy(cm)
        # headless drawing (Sec. 3.4) of the 1M-edge workload after 20 iterations, 2x scale
        cr = pkg.bundle_init(pc, wc.src_xy, wc.dst_xy, wc.group, wc.n_groups, wc.weight,
                             stream=stream)
        pkg.bundle_iterate(cr, 20)
        inf = pkg.bundle_get_info(cr)
        rgba = torch.empty((inf.grid_h * 2, inf.grid_w * 2, 4), dtype=torch.uint8, device="cuda")
        pkg.bundle_render(cr, scale=2, alpha=0.05, width_max=4.0, rgba=rgba)  # warm-up
        torch.cuda.synchronize()
        t_r = time.perf_counter()
        pkg.bundle_render(cr, scale=2, alpha=0.05, width_max=4.0, rgba=rgba)
        t_r = time.perf_counter() - t_r
        var["render"] = {"workload": wc.name, "image": [inf.grid_w * 2, inf.grid_h * 2],
                         "ms": t_r * 1e3, "segments": int(inf.n_points - inf.n_edges),
                         "segments_per_s": (inf.n_points - inf.n_edges) / t_r,
                         "scope": "bundle_render into a device buffer, wall clock (one call)"}
        pkg.bundle_destroy(cr)
        # Fig. 3: ink of the segment-rasterised drawing entering each of 10 iterations,
        # optimised vs fixed step, on the 1,000-edge uniform graph
        from paper_1504_02687_gb300 import synth

        wsm = synth.small(n_edges=1000)
        conv = {"workload": "uniform-1000-edges-256sq", "measure": "occupied cells entering "
                "each iteration (segment histogram)"}
        for name, fl in (("optimised", 0), ("fixed", pkg.FLAG_FIXED_STEP)):
            pm = params_of(wsm, args.rho)
            pm.flags = fl | pkg.FLAG_SEGMENT_HIST | pkg.FLAG_INK_STATS
            c4 = pkg.bundle_init(pm, wsm.src_xy, wsm.dst_xy, wsm.group, wsm.n_groups, wsm.weight,
                                 stream=stream)
            pkg.bundle_iterate(c4, 10)
            conv[name] = pkg.bundle_fetch_ink(c4, 0, 10)[:, 0].tolist()
            pkg.bundle_destroy(c4)
        var["convergence"] = conv
        # the batched form (64 graphs, one graph launch per iteration, autotuned tiles)
        # against the same graphs bundled one after another
        var["batch"] = measure_batch(pkg, torch, stream, args.graphs, min(args.steps, 10),
                                     max(args.warmup, 3), args.rho)
        out["variants"] = var

    if not args.no_e2e:
        # the whole job through the public API: pinned host edges in, polylines back to host
        src = torch.from_numpy(w.src_xy).pin_memory()
        dst = torch.from_numpy(w.dst_xy).pin_memory()
        grp = torch.from_numpy(w.group).pin_memory()
        # the caller's pinned result buffers, sized for the largest polylines (E x cap points),
        # allocated once before the clock starts
        cap_pts = E * (w.n_fixed if w.n_fixed else w.n_max)
        off_h = torch.empty(E + 1, dtype=torch.int64).pin_memory()
        xy_all = torch.empty((cap_pts, 2), dtype=torch.float32).pin_memory()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c3 = pkg.bundle_init(p, src, dst, grp, w.n_groups, None, stream=stream)
        pkg.bundle_iterate(c3, args.steps)
        inf3 = pkg.bundle_get_info(c3)
        xy_h = xy_all[: inf3.n_points]
        pkg.bundle_fetch(c3, off=off_h, xy=xy_h)
        t1 = time.perf_counter()
        upd3 = inf3.points_processed
        pkg.bundle_destroy(c3)
        e2e_s, upd3 = reduce_over_ranks(dist, t1 - t0, float(upd3), device="cuda")
        h2d = w.n_edges * (8 + 8 + 4)
        d2h = (E + 1) * 8 + int(inf3.n_points) * 8
        out["e2e"] = {"value": upd3 / e2e_s, "unit": UNIT,
                      "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                      "scope": (f"bundle_init from pinned host edges + {args.steps} iterations + "
                                "bundle_fetch into pinned host buffers allocated beforehand, "
                                "wall clock")}

    if world == 1 and not args.no_cpu_baseline:
        # about 10-20 s of single-core oracle work: 2 iterations over the whole graph
        out["cpu_baseline"] = cpu_baseline(w, w.n_edges, iters=2 if args.workload != "small" else 10)
        if not args.no_variants and args.workload == "lattice" and args.rho == "f32":
            # the oracle's 30-iteration positions on a bounded sample against the GPU's
            # precision forms (after every timed measurement above)
            out.setdefault("variants", {})["precision"] = precision_forms(w, pkg, stream)
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def measure_batch(pkg, torch, stream, n_graphs, steps, warmup, rho):
    """Batched form: many independent graphs per iteration (one CUDA graph launch runs an
    iteration of all of them, tiles chosen by the autotuner), against the same batch with the
    size-rule tiles and against the same graphs bundled one after another."""
    from paper_1504_02687_gb300 import synth

    ws = synth.batch(n_graphs=n_graphs)
    ps = [params_of(w, rho) for w in ws]
    descs = [dict(src_xy=w.src_xy, dst_xy=w.dst_xy, group=w.group, n_groups=w.n_groups,
                  weight=w.weight) for w in ws]

    def timed_batch(tune):
        b = pkg.bundle_init_batch(descs, ps, stream=stream)
        t_tune, tiles = 0.0, {}
        if tune:
            t_tune = time.perf_counter()
            pkg.bundle_autotune(b)
            t_tune = time.perf_counter() - t_tune
            for k in range(pkg.bundle_batch_size(b)):
                inf = pkg.bundle_get_info(pkg.bundle_batch_member(b, k))
                key = f"eb{inf.tile_eb}/row{inf.tile_row}/strip{inf.tile_strip}"
                tiles[key] = tiles.get(key, 0) + 1
        pkg.bundle_iterate(b, warmup)
        pkg.bundle_sync(b)
        d0 = pkg.bundle_get_info(b).points_processed
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        pkg.bundle_iterate(b, steps)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        upd = pkg.bundle_get_info(b).points_processed - d0
        pkg.bundle_destroy(b)
        return ms, upd, t_tune, tiles

    ms, upd, t_tune, tiles = timed_batch(True)
    heur_ms, heur_upd, _, _ = timed_batch(False)
    seq_ms, seq_upd = 0.0, 0
    for w, p in zip(ws, ps):
        c = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight, stream=stream)
        pkg.bundle_iterate(c, warmup)
        pkg.bundle_sync(c)
        e0 = pkg.bundle_get_info(c).points_processed
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        pkg.bundle_iterate(c, steps)
        a1.record(stream)
        torch.cuda.synchronize()
        seq_ms += a0.elapsed_time(a1)
        seq_upd += pkg.bundle_get_info(c).points_processed - e0
        pkg.bundle_destroy(c)
    E = sum(w.n_edges for w in ws)
    return {
        "workload": (f"batch of {len(ws)} graphs, {E} edges in total (log-uniform 10k-500k), "
                     "1-16 groups, grids 256^2/512^2/1024^2, r 4-12, k=3, <= 64 samples/edge"),
        "graphs": len(ws), "edges": E, "steps": steps, "rho_dtype": rho,
        "value": upd / (ms / 1e3), "ms_per_step": ms / steps, "points_per_step": upd / steps,
        "autotune": {"seconds": t_tune, "tiles": tiles,
                     "untuned_batch": {"value": heur_upd / (heur_ms / 1e3),
                                       "ms_per_step": heur_ms / steps}},
        "sequential": {"value": seq_upd / (seq_ms / 1e3), "ms_per_step": seq_ms / steps},
        "speedup_over_sequential": (upd / ms) / (seq_upd / seq_ms),
    }


def run_split(args):
    """One graph split over the ranks (SURVEY's multi-GPU form, Sec. 4's edges over threads):
    rank r bundles edges [r E / N, (r + 1) E / N) and the splatted histograms are summed over
    the ranks each iteration (NCCL all-reduce of the int32 stack), so every rank advects on
    the whole graph's density. Strong scaling: the whole job is one graph."""
    import numpy as np
    import torch

    import paper_1504_02687_gb300 as pkg
    from paper_1504_02687_gb300 import build as lib_build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        lib_build.build()
    if dist:
        dist.barrier()
    lib_build.build()
    w = make_workload(args.workload, args.edges)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    p = params_of(w, args.rho)
    # the whole graph's grid map, pixel-unit straight edges and integer widths (a context over
    # all edges, destroyed before any iteration)
    full = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight, stream=stream)
    off0, xy0 = pkg.bundle_fetch(full, pixels=True)
    finfo = pkg.bundle_get_info(full)
    map5 = np.array(finfo.map)
    pkg.bundle_destroy(full)
    E = w.n_edges
    lo, hi = rank * E // world, (rank + 1) * E // world
    pp = params_of(w, args.rho)
    pp.sum_bits = finfo.sum_bits
    ctx = pkg.bundle_init_polylines(pp, off0[lo:hi + 1] - off0[lo], xy0[off0[lo]:off0[hi]],
                                    w.group[lo:hi], w.n_groups,
                                    None if w.weight is None else w.weight[lo:hi], map5=map5,
                                    stream=stream)
    reduce = (lambda t: dist.all_reduce(t)) if dist else (lambda t: None)
    clocks = ClockSampler(torch.cuda.current_device())
    pkg.bundle_iterate_split(ctx, args.warmup, reduce, on_device=True)
    pkg.bundle_sync(ctx)
    done0 = pkg.bundle_get_info(ctx).points_processed
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    pkg.bundle_iterate_split(ctx, args.steps, reduce, on_device=True)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = t0.elapsed_time(t1)
    updates = pkg.bundle_get_info(ctx).points_processed - done0
    clk = clocks.stop()
    pkg.bundle_destroy(ctx)
    ms, total = reduce_over_ranks(dist, ms, float(updates), device="cuda")
    if rank == 0:
        cfg = describe(w, args.rho)
        cfg["parallelism"] = (f"{world}-way edge split of one graph, int32 histogram all-reduce "
                              "per iteration" if world > 1 else
                              "one graph through the split-form entry points, no exchange")
        cfg["points_per_step"] = total / args.steps
        print(json.dumps({
            "metric": METRIC, "value": total / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded generator shaped like the paper's graphs)", "config": cfg,
            "clocks": clk}))
    if dist:
        dist.destroy_process_group()


def run_batch(args):
    """The batched form as the timed workload (`--workload batch`)."""
    import torch

    import paper_1504_02687_gb300 as pkg
    from paper_1504_02687_gb300 import build as lib_build

    torch.cuda.set_device(0)
    lib_build.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    clocks = ClockSampler(torch.cuda.current_device())
    r = measure_batch(pkg, torch, stream, args.graphs, args.steps, args.warmup, args.rho)
    clk = clocks.stop()
    print(json.dumps({
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded clustered graphs)",
        "config": {"workload": r["workload"], "graphs": r["graphs"], "edges": r["edges"],
                   "points_per_step": r["points_per_step"], "rho_dtype": args.rho},
        "autotune": r["autotune"],
        "sequential": {**r["sequential"], "speedup_of_batch": r["speedup_over_sequential"]},
        "clocks": clk,
    }))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.split:
        run_split(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
