#!/usr/bin/env python3
"""Throughput benchmark of 3D Richardson-Lucy deconvolution on GB300.

One step = one complete deconvolution of the workload volume (default
1024x1024x128 float32, 50 iterations, Gaussian PSF sigma_xy 2.5 / sigma_z 6),
i.e. every step of the hot path: flux sum and initial estimate, then per
iteration forward convolution, ratio, flipped-PSF correlation and update.
Metric: Gvoxel-iter/s = V * n_iter * steps / time / 1e9 (higher is better).

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and
torch.cuda.synchronize() on both sides, timed with CUDA events on the stream
the library launches on; the max over ranks is reported.  The inputs (512 MiB
volume, 2.1 GiB working set) are larger than the 129 MB L2, so no flush is
needed between steps.  Per-kernel device time comes from the library's own
event pairs around each launch in the same timed region.

Multi-GPU: a single volume does not shard, so ranks run independent replicas
(weak scaling); the only collectives are the host-side barrier and the max of
the elapsed time.

--impl reference times the FP64 CPU oracle (the reference arm) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_14143_gb300 import synth  # noqa: E402

METRIC = "3D RL Gvoxel-iter/s"
UNIT = "Gvoxel-iter/s"
FALLBACK_HBM_GBS = 6800.0


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Ranks:
    """The job's ranks (torchrun env): barrier and max-over-ranks of a scalar.

    With WORLD_SIZE > 1 a process group is created (nccl for the GPU run, gloo
    for host-only use); the only collectives are this barrier and this max.
    """

    def __init__(self, backend: str = "nccl"):
        self.rank, self.world, self.local = dist_env()
        self.backend = backend
        self.dist = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            kw = {}
            if backend == "nccl":
                kw["device_id"] = torch.device("cuda", self.local)
            dist.init_process_group(backend, **kw)
            self.dist = dist

    def _sync_device(self):
        if self.backend == "nccl":
            import torch
            torch.cuda.synchronize()

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()
        self._sync_device()

    def max(self, x: float) -> float:
        if self.dist is None:
            return float(x)
        import torch
        dev = torch.device("cuda", self.local) if self.backend == "nccl" else torch.device("cpu")
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput in G-units/s: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / (ms_max * 1e-3) / 1e9


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


_truth = {}


def make_inputs(w: synth.Workload):
    d, x_true = synth.workload_volume(w)
    _truth[w.name] = x_true      # the ground-truth object, for the metric legs
    return d


# ------------------------------------------------------------------ GPU arm

def run_ours(args, w: synth.Workload):
    import torch
    import paper_2510_14143_gb300 as cr

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ranks = Ranks("nccl")
    barrier = ranks.barrier
    max_over_ranks = ranks.max

    shape, V, n_iter, eps = w.shape, w.voxels, w.n_iter, 1e-6
    d_host = make_inputs(w)
    d = torch.from_numpy(d_host).cuda()
    psf = torch.empty(shape, dtype=torch.float32, device="cuda")
    cr.cubic_psf_gaussian(shape, w.psf_sigma_xy, w.psf_sigma_z, 1.0, psf)
    plan = cr.cubic_rl_plan(shape, psf)
    out = torch.empty_like(d)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    if args.variants:   # pinned launch shapes (a profiler distorts the tuner's timings)
        cr.cubic_rl_plan_set_variants(plan, *(int(v) for v in args.variants.split(",")))
    else:
        cr.cubic_rl_autotune(plan, d, out)      # untimed, like plan creation
    tune_s = time.perf_counter() - t0
    variants = cr.cubic_rl_plan_variants(plan)

    for _ in range(args.warmup):
        cr.cubic_rl_deconvolve(plan, d, n_iter, eps, out)
    barrier()

    # ---- device-resident timed region (per-kernel events inside)
    cr.cubic_rl_profile(plan, True, max_events=2 * (n_iter * 8 + 8) * args.steps + 64)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        cr.cubic_rl_deconvolve(plan, d, n_iter, eps, out)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    prof = cr.cubic_rl_profile_read(plan)
    cr.cubic_rl_profile(plan, False)
    ms = max_over_ranks(ms)
    flux_rel = abs(out.double().sum().item() / d.double().sum().item() - 1.0)

    # ---- end to end through the host-buffer entry point
    h_in = torch.from_numpy(d_host).pin_memory()
    h_out = torch.empty(shape, dtype=torch.float32).pin_memory()
    cr.cubic_rl_deconvolve_host(plan, h_in, n_iter, eps, h_out)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        cr.cubic_rl_deconvolve_host(plan, h_in, n_iter, eps, h_out)
    e1.record(stream)
    barrier()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1))

    units = V * n_iter * args.steps * world
    value = job_rate(V * n_iter * args.steps, world, ms)
    e2e = job_rate(V * n_iter * args.steps, world, ms_e2e)

    # roofline of the kernel instance with the largest share of device time
    kernels = {k: v for k, v in prof.items() if v["timed"] > 0}
    top, members, tk = top_instance(kernels)
    per_launch_bytes = tk["bytes"] / tk["launches"]
    avg_s = tk["ms"] / tk["timed"] * 1e-3
    peak, peak_src = hbm_peak()
    achieved = per_launch_bytes / avg_s / 1e9
    total_kernel_ms = sum(v["ms"] for v in kernels.values())
    launches = sum(v["launches"] for v in prof.values())
    traffic = load_traffic(members, w)
    # algorithmic bytes per voxel-iteration of the kernels that ran (80 with a real PSF
    # spectrum, 84 with a complex one), from the library's per-launch byte counts
    bpvi = sum(v["bytes"] for v in kernels.values()) / (V * n_iter * args.steps)

    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "xyz": list(w.xyz), "n_iter": n_iter, "eps": eps,
                   "psf_sigma_xy": w.psf_sigma_xy, "psf_sigma_z": w.psf_sigma_z,
                   "l2": "inputs larger than L2 (volume 512 MiB, working set ~2.1 GiB vs 129 MB L2), no flush",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": round(e2e, 3), "unit": UNIT, "h2d_bytes_per_step": V * 4, "d2h_bytes_per_step": V * 4},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": top, "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "peak_source": peak_src,
                     "bytes_per_launch": per_launch_bytes, "share": round(tk["ms"] / sum(
                         v["ms"] for v in kernels.values()), 4)},
        "model": {"bytes_per_voxel_iter": round(bpvi, 2), "frac": round(value * bpvi / peak, 4),
                  "note": "whole-step algorithmic bytes at the measured copy bandwidth"},
        "kernels": {k: {"share": round(v["ms"] / total_kernel_ms, 4),
                        "avg_us": round(v["ms"] / v["timed"] * 1e3, 2),
                        "GBps": round(v["bytes"] / v["launches"] / (v["ms"] / v["timed"] * 1e-3) / 1e9, 1)}
                    for k, v in sorted(kernels.items(), key=lambda kv: -kv[1]["ms"])},
        "flux_rel_err": flux_rel,
        "tuning": {"variants_xyz": list(variants[1]), "of": list(variants[0]), "seconds": round(tune_s, 2),
                   "pinned": bool(args.variants)},
        "clocks": clk,
    }
    if not args.no_accel:
        result["accel"] = run_accel(cr, args, plan, d, n_iter, eps, ms / args.steps / n_iter)
    if not args.no_metrics:
        result["metrics"] = run_metrics(cr, args, plan, d, w, ms / args.steps / n_iter)
    if not args.no_paper_shape:
        result["paper_shape"] = run_paper_shape(cr, args, keep_case=(rank == 0 and world == 1 and
                                                                     not args.no_accuracy))
    if not args.no_batched:
        result["batched"] = run_batched(cr, args, ranks)
    if not args.no_grad:
        result["fwd_bwd"] = run_fwd_bwd(cr, args)
    if not args.no_configs:
        result["configs"] = run_small_configs(cr, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w, d_host, args.cpu_sample)
    if rank == 0 and world == 1 and not args.no_accuracy:
        result["accuracy"] = accuracy(cr, plan, d, d_host, w, result.get("configs"))
    _small_plans.clear()
    _paper_case.clear()
    ranks.close()
    return rank, result


# the same kernel instance serves these pass kinds (same launch shape, a runtime mode)
INSTANCES = {"y_fwd": "y", "y_inv": "y", "z_conv": "z", "z_corr": "z"}


def top_instance(kernels):
    """(name, member kinds, summed profile) of the kernel instance with the most device time."""
    groups = {}
    for k, v in kernels.items():
        groups.setdefault(INSTANCES.get(k, k), []).append(k)
    def total(ks, f):
        return sum(kernels[k][f] for k in ks)
    name = max(groups, key=lambda g: total(groups[g], "ms"))
    ks = sorted(groups[name])
    tk = {f: total(ks, f) for f in ("ms", "timed", "launches", "bytes")}
    label = name if ks == [name] else f"{name} ({' + '.join(ks)}: one kernel instance)"
    return label, ks, tk


def run_small_configs(cr, args):
    """The two smaller plain workloads, each in its own tuned launch configuration: 64x64x32
    (20 iterations; launch-latency bound, so also replayed as a captured CUDA graph) and
    256x256x128 (100 iterations; its 176 MB working set sits mostly in the 129 MB L2)."""
    import torch
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for wl, reps in ((synth.SMALL, 50), (synth.MEDIUM, 5)):
        dh, _ = synth.workload_volume(wl)
        img = torch.from_numpy(dh).cuda()
        psf = torch.empty(wl.shape, dtype=torch.float32, device="cuda")
        cr.cubic_psf_gaussian(wl.shape, wl.psf_sigma_xy, wl.psf_sigma_z, 1.0, psf)
        plan = cr.cubic_rl_plan(wl.shape, psf)
        out = torch.empty_like(img)
        cr.cubic_rl_autotune(plan, img, out)
        n = wl.n_iter

        def call():
            cr.cubic_rl_deconvolve(plan, img, n, 1e-6, out)

        def timed(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        ms = timed(call)
        r = {"n_iter": n, "ms": round(ms, 4), "us_per_iter": round(ms * 1e3 / n, 2),
             "value": round(wl.voxels * n / (ms * 1e-3) / 1e9, 3), "unit": UNIT,
             "variants_xyz": list(cr.cubic_rl_plan_variants(plan)[1])}
        if wl is synth.SMALL:
            # the same call captured once into a CUDA graph and replayed
            g = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                call()
                with torch.cuda.graph(g, stream=side):
                    call()
            stream.wait_stream(side)
            ms_g = timed(g.replay)
            r["graph"] = {"ms": round(ms_g, 4), "us_per_iter": round(ms_g * 1e3 / n, 2),
                          "value": round(wl.voxels * n / (ms_g * 1e-3) / 1e9, 3)}
        res[wl.name] = r
        _small_plans[wl.name] = (plan, img, dh, psf)
    return res


_small_plans = {}   # workload name -> (plan, image on the device, image on the host, PSF)


def run_batched(cr, args, ranks=None):
    """64 uneven volumes (5-smooth axes in [48,160]) x 50 iterations: one graph vs 64 plain calls.
    Under several ranks each deconvolves its share of the volumes (balanced by voxels, no
    collective); the rate is all volumes' voxel-iterations over the slowest rank's time."""
    import torch
    all_shapes = synth.batch_shapes()
    rank, world = (ranks.rank, ranks.world) if ranks is not None else (0, 1)
    mine = cr.shard_volumes(all_shapes, world)[rank]
    shapes = [all_shapes[j] for j in mine]
    plans, imgs, outs = [], [], []
    for j, shape in zip(mine, shapes):
        d, _ = synth.batch_volume(j, shape)
        psf = torch.empty(shape, dtype=torch.float32, device="cuda")
        cr.cubic_psf_gaussian(shape, synth.SMALL.psf_sigma_xy, synth.SMALL.psf_sigma_z, 1.0, psf)
        plans.append(cr.cubic_rl_plan(shape, psf))
        imgs.append(torch.from_numpy(d).cuda())
        outs.append(torch.empty(shape, dtype=torch.float32, device="cuda"))
    n_iter, eps = synth.BATCH_ITERS, 1e-6
    vox = sum(int(np.prod(s)) for s in all_shapes)
    stream = torch.cuda.current_stream()
    sync = ranks.barrier if ranks is not None else torch.cuda.synchronize
    top = ranks.max if ranks is not None else (lambda x: x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        sync()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        sync()
        return top(e0.elapsed_time(e1) / reps)

    reps = max(1, min(args.steps, 5))
    ms_b = timed(lambda: cr.cubic_rl_deconvolve_batched(plans, imgs, n_iter, eps, outs), reps)
    nodes = cr.cubic_rl_batched_graph_nodes()

    def plain():
        for p, i, o in zip(plans, imgs, outs):
            cr.cubic_rl_deconvolve(p, i, n_iter, eps, o)

    ms_p = timed(plain, reps)
    # algorithmic bytes of one iteration of this rank's volumes (real H): the X ratio pass
    # 16 S + 4 V, the update 16 S + 8 V, four Y passes 64 S, two Z passes 2 (16 + 4) S, with
    # S = nz ny (nx / 2 + 1) spectrum elements and V voxels
    it_bytes = sum(136 * s[0] * s[1] * (s[2] // 2 + 1) + 12 * s[0] * s[1] * s[2] for s in shapes)
    peak, peak_src = hbm_peak()
    value = vox * n_iter / (ms_b * 1e-3) / 1e9
    return {"workload": f"{len(all_shapes)} volumes, axes drawn from the 5-smooth lengths in [48,160], {n_iter} iterations",
            "voxels": vox, "volumes_per_rank": [len(p) for p in cr.shard_volumes(all_shapes, world)], "value": round(value, 3), "unit": UNIT,
            "ms": round(ms_b, 3), "graph_kernel_nodes": nodes, "plain_calls_ms": round(ms_p, 3),
            "speedup_vs_plain_calls": round(ms_p / ms_b, 3),
            "model": {"bytes_per_voxel_iter": round(it_bytes / sum(int(np.prod(s)) for s in shapes), 2),
                      "frac": round(it_bytes * n_iter / (ms_b * 1e-3) / 1e9 / peak, 4), "peak_source": peak_src}}


def run_accel(cr, args, plan, d, n_iter: int, eps: float, plain_ms_per_iter: float):
    """Accelerated RL on the same volume and plan: time per iteration, and the plain-RL
    iteration count whose Poisson likelihood the accelerated n_iter iterations reach."""
    import torch
    stream = torch.cuda.current_stream()
    out = torch.empty_like(d)
    alpha = torch.empty(n_iter, dtype=torch.float32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        cr.cubic_rl_deconvolve_accel(plan, d, n_iter, eps, out, alpha)
    reps = max(1, min(args.steps, 5))
    cr.cubic_rl_profile(plan, True, max_events=2 * (n_iter * 10 + 8) * reps + 64)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        cr.cubic_rl_deconvolve_accel(plan, d, n_iter, eps, out, alpha)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    prof = cr.cubic_rl_profile_read(plan)
    cr.cubic_rl_profile(plan, False)
    kern = {k: {"avg_us": round(v["ms"] / v["timed"] * 1e3, 2),
                "GBps": round(v["bytes"] / v["launches"] / (v["ms"] / v["timed"] * 1e-3) / 1e9, 1)}
            for k, v in prof.items() if v["timed"] > 0 and k.startswith(("x_acc", "acc_"))}

    # evaluation only (not part of the timed path): NLL = sum(b - d ln b), b = h * x
    b = torch.empty_like(d)
    d64 = d.double()

    def nll(x):
        cr.cubic_rl_convolve(plan, x, 0, b)
        bb = b.double().clamp_min(eps)
        return float((bb - d64 * bb.log()).sum().item())

    nll_acc = nll(out)
    plain = torch.empty_like(d)
    match = None
    curve = {}
    lower = n_iter
    for n in (n_iter, 2 * n_iter, 4 * n_iter, 8 * n_iter, 16 * n_iter):   # doubling search
        cr.cubic_rl_deconvolve(plan, d, n, eps, plain)
        curve[n] = nll(plain)
        if curve[n] <= nll_acc:
            match = n
            break
        lower = n
    ms_it = ms / n_iter
    res = {"workload": f"the same volume, {n_iter} accelerated iterations (Biggs-Andrews)",
           "ms": round(ms, 3), "ms_per_iter": round(ms_it, 4), "plain_ms_per_iter": round(plain_ms_per_iter, 4),
           "value": round(int(d.numel()) * n_iter / (ms * 1e-3) / 1e9, 3), "unit": "Gvoxel-iter/s",
           "alpha_last": round(float(alpha[-1].item()), 4),
           "poisson_nll": {"accel": nll_acc, **{f"plain_{n}": v for n, v in curve.items()}},
           "plain_iters_to_match": [lower, match] if match is not None else f">{16 * n_iter}",
           "kernels": kern}
    if match is not None:
        # plain RL needs more than `lower` and at most `match` iterations for the same likelihood
        res["time_to_same_nll_speedup"] = [round(lower * plain_ms_per_iter / ms, 3),
                                           round(match * plain_ms_per_iter / ms, 3)]
    return res


def run_metrics(cr, args, plan, d, w: synth.Workload, plain_ms_per_iter: float):
    """The metric rows on the timed volume, against its ground-truth object: RL with
    metric-guided stopping on the scale-invariant PSNR (tol 0: stop once the PSNR falls),
    its cost per iteration next to plain RL's, and the FSC of the result and the truth."""
    import torch
    truth = torch.from_numpy(_truth[w.name]).cuda()
    out = torch.empty_like(d)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cr.cubic_rl_deconvolve_monitor(plan, d, 3, 1e-6, cr.METRIC_PSNR, -1.0, 1, out, truth)   # warm-up
    torch.cuda.synchronize()
    e0.record(stream)
    n, hist = cr.cubic_rl_deconvolve_monitor(plan, d, 200, 1e-6, cr.METRIC_PSNR, 0.0, 1, out, truth)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    psnr = [h[2] for h in hist]
    best = int(np.argmax(psnr))
    n_shells = 64
    fsc = torch.empty(n_shells, dtype=torch.float32, device="cuda")
    cr.cubic_fsc(plan, out, truth, n_shells, fsc)
    torch.cuda.synchronize()
    reps = 5
    e0.record(stream)
    for _ in range(reps):
        cr.cubic_fsc(plan, out, truth, n_shells, fsc)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fsc = e0.elapsed_time(e1) / reps
    f = fsc.cpu().numpy()
    below = np.nonzero(f < 1.0 / 7.0)[0]
    V = int(d.numel())
    return {"workload": f"the timed volume against its ground-truth object ({w.name})",
            "psnr_stop": {"iterations": n, "ms": round(ms, 3), "ms_per_iter": round(ms / max(n, 1), 4),
                          "plain_ms_per_iter": round(plain_ms_per_iter, 4), "best_psnr_db": round(psnr[best], 3),
                          "best_iteration": best + 1, "psnr_db_first": round(psnr[0], 3),
                          "rule": "stop at the first iteration whose scale-invariant PSNR falls"},
            "fsc": {"n_shells": n_shells, "ms": round(ms_fsc, 3), "Gvoxel_per_s": round(V / (ms_fsc * 1e-3) / 1e9, 3),
                    "first_shell_below_1_7": int(below[0]) if below.size else None}}


_paper_case = {}   # "case": (image, launch shapes, iterations) of the paper-shaped volume


def run_paper_shape(cr, args, keep_case: bool = False):
    """The paper's stack shape, ZYX 30 x 2160 x 2560 with a PSF of the same size (circular FFT
    convolution), 50 iterations: Gvoxel-iter/s and the top kernel's HBM fraction."""
    import torch
    w = synth.PAPER
    shape, V, n_iter, eps = w.shape, w.voxels, w.n_iter, 1e-6
    g = torch.Generator(device="cuda").manual_seed(w.seed)
    lam = 20.0 + 300.0 * torch.rand(shape, device="cuda", generator=g) ** 12
    d = torch.poisson(lam, generator=g)
    del lam
    psf = torch.empty(shape, dtype=torch.float32, device="cuda")
    cr.cubic_psf_gaussian(shape, w.psf_sigma_xy, w.psf_sigma_z, 1.0, psf)
    plan = cr.cubic_rl_plan(shape, psf)
    del psf
    out = torch.empty_like(d)
    cr.cubic_rl_autotune(plan, d, out)
    stream = torch.cuda.current_stream()
    cr.cubic_rl_deconvolve(plan, d, n_iter, eps, out)
    reps = 2
    cr.cubic_rl_profile(plan, True, max_events=2 * (n_iter * 8 + 8) * reps + 64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        cr.cubic_rl_deconvolve(plan, d, n_iter, eps, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    prof = cr.cubic_rl_profile_read(plan)
    cr.cubic_rl_profile(plan, False)
    kernels = {k: v for k, v in prof.items() if v["timed"] > 0}
    total = sum(v["ms"] for v in kernels.values())
    bpvi = sum(v["bytes"] for v in kernels.values()) / (V * n_iter * reps)
    peak, _ = hbm_peak()
    per = {k: {"share": round(v["ms"] / total, 4), "avg_us": round(v["ms"] / v["timed"] * 1e3, 2),
               "frac": round(v["bytes"] / v["launches"] / (v["ms"] / v["timed"] * 1e-3) / 1e9 / peak, 4)}
           for k, v in sorted(kernels.items(), key=lambda kv: -kv[1]["ms"])}
    value = V * n_iter / (ms * 1e-3) / 1e9
    flux = abs(out.double().sum().item() / d.double().sum().item() - 1.0)
    variants = list(cr.cubic_rl_plan_variants(plan)[1])
    if keep_case:
        # for the accuracy leg: the image and the timed launch shapes
        _paper_case["case"] = (d.cpu().numpy(), variants, 2)
    del plan

    # linear (zero-padded, same-mode) boundaries with a 31 x 33 x 33 PSF box, same data
    kb = (31, 33, 33)
    c = [k // 2 for k in kb]
    zz, yy, xx = np.meshgrid(*[np.arange(k) - cc for k, cc in zip(kb, c)], indexing="ij")
    g = np.exp(-(xx * xx + yy * yy) / (2 * w.psf_sigma_xy ** 2) - zz * zz / (2 * w.psf_sigma_z ** 2))
    box = torch.from_numpy((g / g.sum()).astype(np.float32)).cuda()
    lplan = cr.cubic_rl_plan_linear(shape, box)
    cr.cubic_rl_autotune(lplan, d, out)
    cr.cubic_rl_deconvolve(lplan, d, n_iter, eps, out)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        cr.cubic_rl_deconvolve(lplan, d, n_iter, eps, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_lin = e0.elapsed_time(e1) / reps
    linear = {"psf_box": list(kb), "transform_zyx": list(cr.cubic_rl_plan_dims(lplan)[1]),
              "value": round(V * n_iter / (ms_lin * 1e-3) / 1e9, 3), "unit": UNIT, "ms": round(ms_lin, 3),
              "variants_xyz": list(cr.cubic_rl_plan_variants(lplan)[1])}
    return {"workload": f"{w.name}: ZYX {shape[0]}x{shape[1]}x{shape[2]}, same-size Gaussian PSF "
                        f"(sigma {w.psf_sigma_xy}, {w.psf_sigma_z}), {n_iter} iterations, Poisson data generated "
                        "on the device",
            "value": round(value, 3), "unit": UNIT, "ms": round(ms, 3),
            "model": {"bytes_per_voxel_iter": round(bpvi, 2), "frac": round(value * bpvi / peak, 4)},
            "variants_xyz": variants,
            "flux_rel_err": flux,
            "kernels": per,
            "linear": linear}


def run_fwd_bwd(cr, args):
    """16 volumes 128x128x64, 30 iterations, checkpoints every 6: forward + backward of an MSE loss
    through the differentiable path, against 16 plain forwards."""
    import torch
    from paper_2510_14143_gb300.autograd import RLDeconvolve
    vols = [synth.grad_volume(j) for j in range(synth.GRAD_COUNT)]
    d = torch.from_numpy(np.stack([v[0] for v in vols])).cuda()
    xt = torch.from_numpy(np.stack([v[1] for v in vols])).cuda()
    sxy0, sz0, a0 = synth.GRAD_EVAL_PSF
    n_iter, ckpt = synth.GRAD_ITERS, synth.GRAD_CKPT
    shape = tuple(d.shape[1:])
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step():
        dd = d.clone().requires_grad_(True)
        p = [torch.tensor(v, device="cuda", requires_grad=True) for v in (sxy0, sz0, a0)]
        u = RLDeconvolve.apply(dd, p[0], p[1], p[2], n_iter, 1e-6, ckpt)
        loss = ((u - xt) ** 2).mean(dim=(1, 2, 3)).sum()
        loss.backward()
        return dd.grad, p

    psf = torch.empty(shape, dtype=torch.float32, device="cuda")
    cr.cubic_psf_gaussian(shape, sxy0, sz0, a0, psf)
    plan = cr.cubic_rl_plan(shape, psf)
    out = torch.empty_like(d)

    def fwd_only():
        for b in range(d.shape[0]):
            cr.cubic_rl_deconvolve(plan, d[b], n_iter, 1e-6, out[b])

    # the same forwards spread over the streams the differentiable path uses
    from paper_2510_14143_gb300.autograd import MAX_STREAMS, _fan_in, _fan_out, _streams
    ns = min(d.shape[0], MAX_STREAMS)
    plans = [cr.cubic_rl_plan(shape, psf) for _ in range(ns)]
    streams = _streams(ns, d.device)

    def fwd_streams():
        _fan_out(streams, (d, out))
        for b in range(d.shape[0]):
            with torch.cuda.stream(streams[b % ns]):
                cr.cubic_rl_deconvolve(plans[b % ns], d[b], n_iter, 1e-6, out[b])
        _fan_in(streams)

    def timed(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    reps = max(1, min(args.steps, 3))
    ms_fb = timed(step, reps)
    ms_f = timed(fwd_only, reps)
    ms_fs = timed(fwd_streams, reps)
    vox = int(d.numel())
    return {"workload": f"{d.shape[0]} volumes 128x128x64, {n_iter} iterations, checkpoint every {ckpt}, "
                        f"MSE loss, grads wrt image and (sigma_xy, sigma_z, amp); volumes over {ns} streams",
            "fwd_bwd_ms": round(ms_fb, 3), "fwd_plain_ms": round(ms_f, 3), "fwd_plain_streams_ms": round(ms_fs, 3),
            "fwd_bwd_over_fwd": round(ms_fb / ms_fs, 3),
            "fwd_bwd_over_sequential_fwd": round(ms_fb / ms_f, 3),
            "value": round(vox * n_iter / (ms_fb * 1e-3) / 1e9, 3), "unit": "Gvoxel-iter/s (fwd+bwd)"}


def load_traffic(kinds, w: synth.Workload):
    """DRAM bytes per launch of a kernel instance (the mean over the pass kinds it serves)
    from the committed ncu summary, if it covers this kernel build."""
    path = os.path.join(ROOT, "profiles", "ncu_dram_traffic.txt")
    if not os.path.exists(path):
        return None
    src_hash = source_hash()
    found = {}
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0] in kinds and parts[1] == w.name:
            if parts[3] != src_hash:
                return None
            found[parts[0]] = float(parts[2])
    if set(found) != set(kinds):
        return None
    return sum(found.values()) / len(found)


def source_hash() -> str:
    """Hash of the files the plain path's pass kernels compile from: the shard units and the
    headers they include (capi.cu, the host side and the small reduction kernels, and the
    batched path's all-lengths kernels are left out)."""
    import glob
    import hashlib
    from paper_2510_14143_gb300 import build as _build
    csrc = os.path.join(ROOT, "paper_2510_14143_gb300", "csrc")
    files = set()
    for src in glob.glob(os.path.join(csrc, "shard_*.cu")):
        files |= _build.source_files(src)
    h = hashlib.sha256()
    for f in sorted(files, key=os.path.basename):
        h.update(open(f, "rb").read())
    return h.hexdigest()[:12]


# ------------------------------------------------------------------ CPU oracle

def oracle_sample(w: synth.Workload, d_host, sample: str):
    """A bounded sample of the workload for the FP64 oracle: (d, psf) of the sample."""
    import oracle
    if sample == "full":
        dd = d_host
    else:  # "crop": a 5-smooth sub-volume of the workload's own data
        nz, ny, nx = w.shape
        dd = d_host[:min(nz, 64), :min(ny, 256), :min(nx, 256)]
    dd = np.ascontiguousarray(dd, dtype=np.float64)
    psf = oracle.psf_gaussian(dd.shape, w.psf_sigma_xy, w.psf_sigma_z)
    return dd, psf


def cpu_baseline(w: synth.Workload, d_host, sample: str, iters: int = 1):
    import oracle
    dd, psf = oracle_sample(w, d_host, sample)
    H = oracle.psf_spectrum(psf)                  # plan, excluded like the GPU plan
    u = np.full(dd.shape, oracle.initial_value(dd, 1e-6))
    t0 = time.perf_counter()
    for _ in range(iters):
        u, _, _, _ = oracle.rl_iterate(H, dd, u, 1e-6)
    dt = time.perf_counter() - t0
    vox = dd.size
    return {"value": round(vox * iters / dt / 1e9, 6), "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{iters} RL iteration(s) of the FP64 oracle on a {dd.shape[2]}x{dd.shape[1]}x{dd.shape[0]} "
                      f"{'volume' if sample == 'full' else 'crop'} of the workload (PSF spectrum precomputed), "
                      f"{dt:.1f} s"}


def err_stats(got, ref):
    """rel_l2 = ||got - ref|| / ||ref||; max_rel = max |got - ref| / max |ref| (the worst voxel
    against the volume's scale)."""
    got = np.asarray(got, np.float64)
    diff = got - ref
    return {"rel_l2": float(np.linalg.norm(diff) / np.linalg.norm(ref)),
            "max_rel": float(np.max(np.abs(diff)) / np.max(np.abs(ref)))}


def accuracy(cr, plan, d, d_host, w: synth.Workload, configs=None):
    """Error of the float32 GPU estimate against the FP64 oracle on the same inputs and PSF,
    for every workload at its stated iteration count: 64x64x32 at 20, 256x256x128 at 100, the
    timed volume (1024x1024x128) at its 50 in its benchmarked launch configuration.  Two stated
    subsets, where the oracle's Bluestein transforms of the non-power-of-two lengths are too
    slow for a bench run: the paper-shaped volume at 2 iterations, and 8 of the 64 batched
    volumes (every eighth, from the fifth) at their 50.  Both sides take the same PSF: the
    oracle's Gaussian, rounded to float32 (the GPU's own PSF generator is checked against it
    in the tests).  Each entry gives rel_l2, max_rel, the oracle's wall time on the host cores
    and, for the first two, the oracle's rate next to the GPU's."""
    import torch
    import oracle

    def host_psf(shape, sxy, sz):
        return oracle.psf_gaussian(shape, sxy, sz, 1.0).astype(np.float32)

    def plan_like(shape, psf32, variants=None):
        p = cr.cubic_rl_plan(shape, torch.from_numpy(psf32).cuda())
        if variants is not None:
            cr.cubic_rl_plan_set_variants(p, *variants)
        return p

    def run(plan_, img, n):
        out = torch.empty_like(img)
        cr.cubic_rl_deconvolve(plan_, img, n, 1e-6, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    def with_oracle(got, img_host, psf_host, n):
        t0 = time.perf_counter()
        ref = oracle.rl(img_host, psf_host, n, 1e-6)
        dt = time.perf_counter() - t0
        r = {"n_iter": n, **err_stats(got, ref), "oracle_s": round(dt, 1)}
        r["oracle_rate"] = round(img_host.size * n / dt / 1e9, 6)
        return r

    res = {}
    for wl in (synth.SMALL, synth.MEDIUM):
        psf32 = host_psf(wl.shape, wl.psf_sigma_xy, wl.psf_sigma_z)
        if wl.name in _small_plans:
            p0, img, dh, _ = _small_plans[wl.name]
            p = plan_like(wl.shape, psf32, cr.cubic_rl_plan_variants(p0)[1])
        else:
            dh, _ = synth.workload_volume(wl)
            img = torch.from_numpy(dh).cuda()
            p = plan_like(wl.shape, psf32)
        r = with_oracle(run(p, img, wl.n_iter), dh, psf32, wl.n_iter)
        if configs and wl.name in configs:
            r["gpu_rate"] = configs[wl.name]["value"]
        res[wl.name] = r
        del p
    psf32 = host_psf(w.shape, w.psf_sigma_xy, w.psf_sigma_z)
    shapes_xyz = list(cr.cubic_rl_plan_variants(plan)[1])
    p = plan_like(w.shape, psf32, shapes_xyz)
    res[w.name] = with_oracle(run(p, d, w.n_iter), d_host, psf32, w.n_iter)
    res[w.name]["launch_shapes_xyz"] = shapes_xyz
    del p
    if _paper_case:
        dh, variants, n = _paper_case["case"]
        wp = synth.PAPER
        psf32 = host_psf(wp.shape, wp.psf_sigma_xy, wp.psf_sigma_z)
        p = plan_like(wp.shape, psf32, variants)
        res[wp.name] = with_oracle(run(p, torch.from_numpy(dh).cuda(), n), dh, psf32, n)
        res[wp.name]["subset"] = f"{n} of {wp.n_iter} iterations"
        del p
    # batched workload: one batched call over the subset, each volume against the oracle
    all_shapes = synth.batch_shapes()
    picks = list(range(4, len(all_shapes), 8))
    plans, imgs, hosts = [], [], []
    for j in picks:
        shape = all_shapes[j]
        dh, _ = synth.batch_volume(j, shape)
        bpsf = host_psf(shape, synth.SMALL.psf_sigma_xy, synth.SMALL.psf_sigma_z)
        plans.append(plan_like(shape, bpsf))
        imgs.append(torch.from_numpy(dh).cuda())
        hosts.append((dh, bpsf))
    outs = [torch.empty_like(i) for i in imgs]
    cr.cubic_rl_deconvolve_batched(plans, imgs, synth.BATCH_ITERS, 1e-6, outs)
    torch.cuda.synchronize()
    per = []
    t_or = 0.0
    for j, (dh, bpsf), out in zip(picks, hosts, outs):
        t0 = time.perf_counter()
        ref = oracle.rl(dh, bpsf, synth.BATCH_ITERS, 1e-6)
        t_or += time.perf_counter() - t0
        per.append({"volume": j, "zyx": list(dh.shape), **err_stats(out.cpu().numpy(), ref)})
    res["batched"] = {"n_iter": synth.BATCH_ITERS, "subset": f"volumes {picks} of {len(all_shapes)}",
                      "rel_l2": max(v["rel_l2"] for v in per), "max_rel": max(v["max_rel"] for v in per),
                      "oracle_s": round(t_or, 1), "per_volume": per}
    res["reference"] = ("FP64 CPU oracle, same inputs and PSF (the oracle's Gaussian in float32); rel_l2 and "
                        "max_rel of the batched entry are the worst volume's")
    return res


def run_reference(args, w: synth.Workload):
    rank, world, _ = dist_env()
    if rank != 0:
        return rank, None
    import oracle
    d_host = make_inputs(w)
    dd, psf = oracle_sample(w, d_host, args.cpu_sample)
    H = oracle.psf_spectrum(psf)
    u = np.full(dd.shape, oracle.initial_value(dd, 1e-6))
    for _ in range(args.warmup):
        u, _, _, _ = oracle.rl_iterate(H, dd, u, 1e-6)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u, _, _, _ = oracle.rl_iterate(H, dd, u, 1e-6)
    dt = time.perf_counter() - t0
    value = dd.size * args.steps / dt / 1e9
    sample = (f"one FP64 oracle RL iteration per step on a {dd.shape[2]}x{dd.shape[1]}x{dd.shape[0]} "
              f"{'volume' if args.cpu_sample == 'full' else 'crop'} of the {w.name} workload")
    result = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "xyz": list(w.xyz), "n_iter": w.n_iter, "eps": 1e-6},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return rank, result


def run_ncu_target(args, w: synth.Workload):
    """Profiling target: plan + one RL iteration with pinned launch shapes; no timing, no line."""
    import torch
    import paper_2510_14143_gb300 as cr
    vx, vy, vz = (int(v) for v in args.ncu_target.split(","))
    g = torch.Generator(device="cuda").manual_seed(1)
    d = torch.rand(w.shape, device="cuda", generator=g) * 100 + 1
    psf = torch.empty(w.shape, dtype=torch.float32, device="cuda")
    cr.cubic_psf_gaussian(w.shape, w.psf_sigma_xy, w.psf_sigma_z, 1.0, psf)
    plan = cr.cubic_rl_plan(w.shape, psf)
    cr.cubic_rl_plan_set_variants(plan, vx, vy, vz)
    out = torch.empty_like(d)
    cr.cubic_rl_deconvolve(plan, d, args.ncu_iters, 1e-6, out)
    torch.cuda.synchronize()


def run_ncu_batched(args):
    """Profiling target: the batched leg's 64 plans, then three batched calls of
    --ncu-iters iterations (the first captures the graph); no timing, no line."""
    import torch
    import paper_2510_14143_gb300 as cr
    shapes = synth.batch_shapes()
    plans, imgs, outs = [], [], []
    for j, shape in enumerate(shapes):
        d, _ = synth.batch_volume(j, shape)
        psf = torch.empty(shape, dtype=torch.float32, device="cuda")
        cr.cubic_psf_gaussian(shape, synth.SMALL.psf_sigma_xy, synth.SMALL.psf_sigma_z, 1.0, psf)
        plans.append(cr.cubic_rl_plan(shape, psf))
        imgs.append(torch.from_numpy(d).cuda())
        outs.append(torch.empty(shape, dtype=torch.float32, device="cuda"))
    for _ in range(3):
        cr.cubic_rl_deconvolve_batched(plans, imgs, args.ncu_iters, 1e-6, outs)
    torch.cuda.synchronize()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=sorted(synth.PLAIN), default=synth.LARGE.name)
    ap.add_argument("--cpu-sample", choices=("crop", "full"), default="full")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-workload leg")
    ap.add_argument("--no-grad", action="store_true", help="skip the forward+backward leg")
    ap.add_argument("--no-accel", action="store_true", help="skip the accelerated-RL leg")
    ap.add_argument("--no-paper-shape", action="store_true", help="skip the 2560x2160x30 leg")
    ap.add_argument("--no-metrics", action="store_true", help="skip the stopping-metric and FSC leg")
    ap.add_argument("--no-configs", action="store_true", help="skip timing the 64x64x32 and 256x256x128 workloads")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the comparison with the FP64 oracle at the stated iteration counts (minutes of CPU)")
    ap.add_argument("--ncu-target", metavar="VX,VY,VZ",
                    help="profiling target only: plan + --ncu-iters RL iterations with these launch shapes")
    ap.add_argument("--ncu-batched", action="store_true",
                    help="profiling target only: the 64-volume batched workload, three calls of --ncu-iters iterations")
    ap.add_argument("--ncu-iters", type=int, default=1)
    ap.add_argument("--variants", metavar="VX,VY,VZ",
                    help="pin the launch shapes of the timed workload instead of autotuning")
    args = ap.parse_args()
    w = synth.PLAIN[args.workload]
    if args.ncu_target:
        run_ncu_target(args, w)
        return
    if args.ncu_batched:
        run_ncu_batched(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank, result = run_reference(args, w) if args.impl == "reference" else run_ours(args, w)
    if rank == 0 and result is not None:
        print(json.dumps(result), flush=True)


if __name__ == "__main__":
    main()
