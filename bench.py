#!/usr/bin/env python
"""Benchmark of the Gaussian-splatting CT hot path on one GB300 (or N replicas).

A step is one full reconstruction optimisation iteration (Eq. 5) at 75 cone-beam views of
512x512 pixels with 50,000 Gaussians: rasterizer forward, L1 + D-SSIM loss (fused), the
per-Gaussian rasterizer backward, voxelization of the 256^3 volume, its TV loss and voxelizer
backward, and the Adam update -- every stage a libgsct kernel.

Metric: in-cut Gaussian-pixel evaluations of the step's projection per second of the full
fwd+bwd step (higher is better); ms per step is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = {
    "workload": "recon step, 75 cone views x 512^2, 50k Gaussians, TV on 256^3",
    # tile 16: the autotuner's pick for this shape (autotune.tune_tile, forward + backward:
    # 4.45 / 2.90 / 3.14 ms for tiles 8 / 16 / 32), fixed here so that the step's launch
    # sequence, which the profiler commands count into, has no tuning runs in front of it
    "views": 75, "W": 512, "H": 512, "gaussians": 50000, "tv_volume": 256, "tile": 16,
    "model_seed": 21, "target_seed": 22, "scale_median": 0.012, "scale_sigma_log": 0.4,
}
# a reduced case of the same kernels for profiler captures (16 views, 128^3 TV volume)
SMALL = dict(WORKLOAD, workload="recon step, 16 cone views x 512^2, 50k Gaussians, TV on 128^3",
             views=16, tv_volume=128)
METRIC = "Gaussian-pixel evals/s (fwd+bwd step) at 75x512^2"
UNIT = "evals/s"

# The evaluation kernels' work per in-cut evaluation: one ex2 on the special-function unit and
# this many FP32 lane operations (raster_fwd: offset, two fma for the exponent, the
# accumulating fma; raster_bwd: two fma, G = g e, and three moment updates against the block's
# compile-time column offsets -- the y moments are folded per row; vox_fwd: the z offset fma,
# two fma, the accumulating fma; vox_bwd: the same offset and exponent, q = g e, q dz, three
# moment updates).  Their roofline is the slower of the two units at the rates the probe
# kernels measure.
FP32_OPS_PER_EVAL = {"raster_fwd": 4, "raster_bwd": 6, "vox_fwd": 4, "vox_bwd": 8}
# The per-evaluation figures of the hot-path scope's measurement plan, which count every FP32
# operation of an unpacked, unfolded evaluation: forward 2 adds (the pixel offset), 3 fma/mul
# (the quadratic form), 1 compare/select (the cut) and 1 fma (the accumulation) besides the
# ex2; backward about 20 FP32 operations besides the ex2.  The voxel passes take the same
# figures.  The line's frac uses these; the folded counts above give the stricter fraction.
SCOPE_OPS_PER_EVAL = {"raster_fwd": 7, "raster_bwd": 20, "vox_fwd": 7, "vox_bwd": 20}


def alu_peaks(device, blocks_per_sm=8, iters=2048):
    """Measured throughput of ex2.approx (SFU) and FP32 fma (ops/s) by the library's probe
    kernels, timed with CUDA events after warm-up; also per SM per clock at f_mhz."""
    import torch

    from paper_2604_01844_gb300 import binding as B

    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks = sms * blocks_per_sm
    sink = torch.empty(blocks * 256, dtype=torch.float32, device=device)
    out = {}
    for kind, name in ((0, "ex2"), (1, "fma")):
        for _ in range(3):
            B.check(B.lib().gs_probe_rate(kind, blocks, iters, B.ptr(sink), B.stream_handle()),
                    "gs_probe_rate")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.check(B.lib().gs_probe_rate(kind, blocks, iters, B.ptr(sink), B.stream_handle()),
                "gs_probe_rate")
        e1.record()
        e1.synchronize()
        out[name + "_per_s"] = blocks * 256 * 8 * iters / (e0.elapsed_time(e1) * 1e-3)
    out["sms"] = sms
    return out


# Unit counts per SM per clock: 128 FP32 lanes; 32 ex2 on the special-function unit (GB300
# doubles the 16 of earlier parts; the probe kernels measure 31.5 and 118 per SM per clock,
# 98 % and 92 % of these counts, and their rates are reported beside the roofline).
FP32_LANES_PER_SM = 128
EX2_PER_SM = 32


def eval_peak(kernel, sms, f_mhz, ops=None):
    """Roofline of an evaluation kernel in evaluations/s (SMs x clock x the binding unit's
    rate per evaluation) and the binding unit; ops: FP32 operations per evaluation (default
    the folded count)."""
    clk = sms * f_mhz * 1e6
    sfu = clk * EX2_PER_SM
    fp32 = clk * FP32_LANES_PER_SM / (ops or FP32_OPS_PER_EVAL)[kernel]
    return (sfu, "sfu") if sfu <= fp32 else (fp32, "fp32")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh)
    return None


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, window=None):
        """Stops sampling and summarises the samples whose timestamps fall in window = (t0, t1)
        (host epoch seconds around the timed region; all samples when none do or when the
        timestamps cannot be read)."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        return summarise_clocks(lines, window)


def _stamp(text):
    """nvidia-smi's local timestamp ('YYYY/MM/DD HH:MM:SS.mmm') as epoch seconds, or None."""
    import datetime

    try:
        return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
    except ValueError:
        return None


def summarise_clocks(lines, window=None):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            sm, mx = float(parts[2]), float(parts[3])
        except ValueError:
            continue
        active = {nm for nm, val in zip(names, parts[6:10]) if val.lower() == "active"}
        rows.append((_stamp(parts[0]), sm, mx, active))
    if not rows:
        return None
    inside = rows
    if window is not None:
        t0, t1 = window
        inside = [r for r in rows if r[0] is not None and t0 <= r[0] <= t1]
    scope = "timed region"
    if not inside:
        inside, scope = rows, "whole run of the sampler (no sample inside the timed region)"
    return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
            "samples": len(inside), "reasons": sorted(set().union(*(r[3] for r in inside))),
            "scope": scope}


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def build_problem(device, shard=None):
    """The headline step's reconstruction; shard = (rank, world) builds this process's part
    of the view-sharded step instead (its chunk of the views, one all-reduce per step)."""
    import numpy as np
    import torch

    import synth
    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300.recon import ReconConfig, Reconstruction
    from paper_2604_01844_gb300.sharded import ViewShardedReconstruction

    w = WORKLOAD
    views = synth.cone_views(w["views"], w["W"], w["H"])
    model = synth.gaussians(w["model_seed"], w["gaussians"], scale_median=w["scale_median"],
                            scale_sigma_log=w["scale_sigma_log"])
    tgt = synth.gaussians(w["target_seed"], w["gaussians"], scale_median=w["scale_median"],
                          scale_sigma_log=w["scale_sigma_log"])
    # target projections rendered once by the library (setup, outside the timed region)
    tproj = g.Projector(views, w["W"], w["H"], tile=w["tile"], device=device)
    target = tproj.forward(*[torch.from_numpy(a).to(device) for a in tgt]).clone()
    del tproj
    grid = synth.cube_grid(w["tv_volume"])
    cfg = ReconConfig(tile=w["tile"])
    if shard is not None:
        rec = ViewShardedReconstruction(views, w["W"], w["H"], target, grid, *model,
                                        rank=shard[0], world=shard[1], cfg=cfg, device=device)
    else:
        rec = Reconstruction(views, w["W"], w["H"], target, grid, *model, cfg=cfg, device=device)
    return rec, model, views


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300 import binding as B
    from paper_2604_01844_gb300 import build as gbuild
    from paper_2604_01844_gb300 import replicas as R

    gbuild.build()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=device)
    sharded = args.parallel == "views" and ws > 1
    rec, model, views = build_problem(device, shard=(rank, ws) if sharded else None)

    # algorithmic work of one step: in-cut Gaussian-pixel (and Gaussian-voxel) evaluations,
    # counted exactly by the counting kernels.  The parameters move as the steps optimise them,
    # so each timed phase is credited with the mean of the counts taken just before and just
    # after it.
    def count():
        return rec.projector.count_evals(*rec.act), rec.voxelizer.count_evals(*rec.act)

    def mean(a, b):
        return (a[0] + b[0]) // 2, (a[1] + b[1]) // 2

    rec.plan()
    for _ in range(args.warmup):
        rec.step()
    torch.cuda.synchronize()
    ev_a = count()
    if rec.overflowed():
        raise RuntimeError("a workspace of the step ran out of pair capacity")

    clocks = ClockSampler(local)
    stream = torch.cuda.current_stream()
    launches0 = B.launch_count()
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t_start = time.time()
    e0.record(stream)
    for _ in range(args.steps):
        rec.step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_end = time.time()
    clk = clocks.stop((t_start, t_end))
    if rec.overflowed():
        raise RuntimeError("a workspace of the step ran out of pair capacity during the timed "
                           "steps: the timing would credit work that was skipped")
    launches = B.launch_count() - launches0
    ms = R.slowest(e0.elapsed_time(e1) / args.steps, device)
    loss = float(rec.loss.item())
    ev_b = count()
    evals_px, evals_vox = mean(ev_a, ev_b)  # the timed steps

    # per-kernel breakdown: the same step in its serial form (one stream, views unchunked),
    # each launch bracketed by CUDA events on its stream, so that every kernel's time is its
    # own and one raster launch covers the step's evaluations
    rec.step(serial=True)
    torch.cuda.synchronize()
    B.timing_reset()
    B.timing_enable(True)
    for _ in range(args.steps):
        rec.step(serial=True)
    torch.cuda.synchronize()
    B.timing_enable(False)
    per_kernel = B.timing_read()
    pairs = int(rec.projector.status().pairs)  # (view, tile) pairs of the serial step
    ev_c = count()
    ser_px, ser_vox = mean(ev_b, ev_c)  # the serial per-kernel pass

    # end to end through the public API with host buffers: per step the parameters and the
    # target projections go host->device from pinned memory, the loss and the updated
    # parameters come back device->host.  The target copy runs on a copy stream (after the
    # previous step has finished reading the target) and only the image losses wait for it, so
    # it overlaps the projection forward.
    h_params = [t.detach().cpu().pin_memory() for t in rec.raw]
    h_target = rec.target.detach().cpu().pin_memory()
    h_out = [torch.empty_like(t, device="cpu").pin_memory() for t in rec.act]
    h_loss = torch.empty(1, dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * 4 for t in h_params) + h_target.numel() * 4
    d2h = sum(t.numel() * 4 for t in h_out) + 4
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    copy = torch.cuda.Stream(device=device)
    e2.record(stream)
    for _ in range(args.steps):
        for d, h in zip(rec.raw, h_params):
            d.copy_(h, non_blocking=True)
        copy.wait_stream(stream)
        with torch.cuda.stream(copy):
            rec.target.copy_(h_target, non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(copy)
        rec.activate()
        rec.step(target_ready=ready)
        for d, h in zip(rec.act, h_out):
            h.copy_(d, non_blocking=True)
        h_loss.copy_(rec.loss, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_e2e = R.slowest(e2.elapsed_time(e3) / args.steps, device)
    e2e_px = mean(ev_c, count())[0]  # the end-to-end steps
    if sharded:
        # every process evaluated its own views: the job's units are their sum (a collective,
        # so every rank takes part before the others leave)
        import torch.distributed as dist

        tot = torch.tensor([float(evals_px), float(e2e_px)], dtype=torch.float64, device=device)
        dist.all_reduce(tot)
        value = float(tot[0]) / (ms * 1e-3)
        e2e_value = float(tot[1]) / (ms_e2e * 1e-3)
    else:
        value = R.job_rate(evals_px, ms, ws)
        e2e_value = R.job_rate(e2e_px, ms_e2e, ws)

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel
    dom = max(per_kernel.items(), key=lambda kv: kv[1][1])
    name, (nl, tot_ms) = dom
    avg_ms = tot_ms / max(nl, 1)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mp = measured_peaks() or {}
    f_mhz = (clk or {}).get("sm_mhz") or mp.get("sm_max_mhz", 2070.0)
    roof = None
    peaks = alu_peaks(device)
    per_clk = {k: round(v / (sms * f_mhz * 1e6), 2) for k, v in peaks.items() if k != "sms"}
    if name in FP32_OPS_PER_EVAL:
        units = ser_px if name.startswith("raster") else ser_vox
        peak_s, unit_name = eval_peak(name, sms, f_mhz, SCOPE_OPS_PER_EVAL)
        peak = peak_s / 1e9
        peak_f = eval_peak(name, sms, f_mhz)[0] / 1e9
        ach = units / (avg_ms * 1e-3) / 1e9
        roof = {"kernel": name, "bound": "alu", "achieved": round(ach, 2), "peak": round(peak, 2),
                "unit": "Geval/s", "frac": round(ach / peak, 4), "traffic": read_traffic(name),
                "peak_basis": f"{sms} SMs x {f_mhz:.0f} MHz (median sampled) x min({EX2_PER_SM} "
                              f"ex2, {FP32_LANES_PER_SM} FP32 lanes / "
                              f"{SCOPE_OPS_PER_EVAL[name]} ops) per SM per clock: one ex2 and "
                              f"{SCOPE_OPS_PER_EVAL[name]} FP32 operations per evaluation (the "
                              f"scope's measurement figure), bound by the {unit_name}; the "
                              f"probe kernels measure {per_clk['ex2_per_s']} ex2 and "
                              f"{per_clk['fma_per_s']} fma per SM per clock",
                "peak_folded_count": round(peak_f, 2), "frac_folded_count": round(ach / peak_f, 4),
                "folded_count_basis": f"{FP32_OPS_PER_EVAL[name]} FP32 operations per "
                                      f"evaluation after packing and folding",
                "avg_launch_ms": round(avg_ms, 4), "launches": nl}
    else:
        roof = {"kernel": name, "bound": "hbm", "achieved": None, "peak": mp.get("hbm_gbs"),
                "unit": "GB/s", "frac": None, "traffic": read_traffic(name),
                "avg_launch_ms": round(avg_ms, 4), "launches": nl}

    # the same ALU roofline for every evaluation kernel of the step
    kernel_roofs = {}
    for kname in FP32_OPS_PER_EVAL:
        if kname not in per_kernel:
            continue
        kl, kt = per_kernel[kname]
        units = ser_px if kname.startswith("raster") else ser_vox
        kpeak = eval_peak(kname, sms, f_mhz, SCOPE_OPS_PER_EVAL)[0] / 1e9
        kpeak_f = eval_peak(kname, sms, f_mhz)[0] / 1e9
        kach = units / ((kt / max(kl, 1)) * 1e-3) / 1e9
        kernel_roofs[kname] = {"achieved": round(kach, 2), "peak": round(kpeak, 2),
                               "unit": "Geval/s", "frac": round(kach / kpeak, 4),
                               "peak_folded_count": round(kpeak_f, 2),
                               "frac_folded_count": round(kach / kpeak_f, 4),
                               "evals_per_launch": units}

    # HBM rooflines of the step's memory-heavy kernels from algorithmic bytes: a radix pass
    # reads and writes every (key, value) pair (16 B), the 2D SSIM passes read and write each
    # image or map pixel once.  The pairs sort over the tile bits of their keys in passes of
    # at most 8 bits (two passes of 5 bits for the 1024 tiles of 512^2 at tile 16).
    tiles = ((WORKLOAD["W"] + WORKLOAD["tile"] - 1) // WORKLOAD["tile"]) * \
        ((WORKLOAD["H"] + WORKLOAD["tile"] - 1) // WORKLOAD["tile"])
    passes = ((tiles - 1).bit_length() + 7) // 8
    px = int(WORKLOAD["views"]) * WORKLOAD["W"] * WORKLOAD["H"]
    step_bytes = {"radix_scatter": 16 * pairs * passes, "ssim2d_fwd": 20 * px,
                  "ssim2d_bwd": 24 * px}
    hbm_roofs = {}
    for k, nb in step_bytes.items():
        if k in per_kernel and mp.get("hbm_gbs"):
            kms = per_kernel[k][1] / args.steps  # ms per step
            gbs = nb / (kms * 1e-3) / 1e9
            hbm_roofs[k] = {"bytes_per_step": nb, "achieved_gbs": round(gbs, 1),
                            "peak_gbs": mp["hbm_gbs"], "frac": round(gbs / mp["hbm_gbs"], 3)}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD["workload"], "views": WORKLOAD["views"],
                   "detector": [WORKLOAD["W"], WORKLOAD["H"]], "gaussians": WORKLOAD["gaussians"],
                   "tv_volume": WORKLOAD["tv_volume"], "tile": WORKLOAD["tile"],
                   "evals_per_step": evals_px, "voxel_evals_per_step": evals_vox,
                   "evals_per_step_first_last": [ev_a[0], ev_b[0]],
                   "target": "projections of a second seeded Gaussian set",
                   "l2": "working set per step > 0.5 GB (images, SSIM maps, 256^3 volume) > L2",
                   "parallelism": (f"views sharded x{ws}" if sharded else f"replicas x{ws}")
                   if ws > 1 else "single GPU"},
        "roofline": roof, "kernel_rooflines": kernel_roofs, "hbm_rooflines": hbm_roofs,
        "pairs_per_step": pairs,
        "alu_peaks": {"ex2_per_s": round(peaks["ex2_per_s"]), "fma_per_s": round(peaks["fma_per_s"]),
                      "per_sm_per_clock": per_clk, "sm_mhz": f_mhz,
                      "note": "probe kernels gs_probe_rate, 8 CTAs of 256 threads per SM"},
        "kernels_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in
                                sorted(per_kernel.items(), key=lambda kv: -kv[1][1])},
        "kernels_note": "per-kernel times from the serial form of the step (one stream, views "
                        "unchunked); the timed step overlaps the TV branch and two view chunks "
                        "on three streams",
        "ms_per_step_serial": round(sum(v[1] for v in per_kernel.values()) / args.steps, 4),
        "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": ms_e2e,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "loss": loss,
    }
    if not args.no_extras:
        legs = {
            "time_to_psnr": lambda: time_to_psnr(device),
            "learned_init": lambda: learned_vs_plain(device),
            "batched": lambda: batched_learned_vs_plain(device),
            "fit_volume": lambda: fit_volume_rate(device, args.fit_side, args.fit_gaussians),
            "scale_up": lambda: scale_up(device),
            "warm_start": lambda: warm_start_study(device, side=args.warm_side,
                                                   det=args.warm_det),
            "adaptive_control": lambda: adaptive_control(device),
            "compression": lambda: compression(device),
            "gemm": lambda: gemm_rate(device),
            "batched_small": lambda: batched_small_step(device),
            "kernel_sweep": lambda: kernel_sweep(device),
        }
        chosen = list(legs) if args.extras == "all" else args.extras.split(",")
        for name in chosen:
            if name not in legs:
                raise SystemExit(f"unknown extra leg {name!r}; choose from {', '.join(legs)}")
            out[name] = legs[name]()
    if ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(model, views, target_s=args.cpu_seconds)
    print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


def time_to_psnr(device, target_db=35.0, max_iters=400, eval_every=5):
    """Plain single-instance reconstruction of the 40-ellipsoid phantom from 75 cone views of
    512^2 with 50k Gaussians (FDK-gradient init, L1 + D-SSIM + TV on the 256^3 volume): GPU
    time from the projections to the first evaluation at or above target_db."""
    import numpy as np
    import torch

    import synth
    from paper_2604_01844_gb300.recon import (PhantomProblem, ReconConfig, Reconstruction,
                                               fdk_volume, gradient_init, psnr_of,
                                               reconstruct_to_psnr)

    views = synth.cone_views(75, 512, 512)
    grid = synth.cube_grid(256)
    prob = PhantomProblem(synth.ellipsoid_phantom(1, 40), views, 512, 512, grid, device=device)
    u = np.random.default_rng(7).random((50000, 4)).astype(np.float32)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    fdk = fdk_volume(prob, grid)
    mr, sc, q = gradient_init(fdk, grid, 50000, u)
    e1.record()
    torch.cuda.synchronize()
    init_ms = e0.elapsed_time(e1)
    sse = torch.zeros(1, dtype=torch.float64, device=device)
    fdk_db = psnr_of(fdk, prob.gt, prob.peak, sse)
    cfg = ReconConfig(**LR_FAST, headroom=LONG_RUN_HEADROOM)
    rec = Reconstruction(views, 512, 512, prob.proj.clone(), grid, mr.cpu().numpy(),
                         sc.cpu().numpy(), q.cpu().numpy(), cfg=cfg, device=device)
    init_db = psnr_of(rec.voxelizer.forward(*rec.act), prob.gt, prob.peak, sse)
    hist, ok = reconstruct_to_psnr(rec, prob.gt, prob.peak, max_iters, target_db, eval_every)
    it, ms, db = hist[-1]
    return {"target_db": target_db, "reached": ok, "iters": it, "ms_optimise": round(ms, 2),
            "ms_fdk_and_init": round(init_ms, 2), "ms_total": round(ms + init_ms, 2),
            "psnr_fdk_db": round(fdk_db, 2), "psnr_init_db": round(init_db, 2),
            "psnr_final_db": round(db, 2), "eval_every": eval_every, "replans": rec.replans,
            "workload": "40-ellipsoid phantom, 75 cone views x 512^2, 50k Gaussians, 256^3",
            "note": "plain single-instance form; PSNR = 10 log10(max(V_gt)^2 / MSE) on 256^3"}


# Adam learning rates of the time-to-PSNR runs: FAST is the best of a sweep of the plain start
# (lr_mean 4e-4 / 8e-4 / 1.6e-3 x lr_scale 1e-2 / 2e-2); BASE the earlier setting.  Learned
# and plain starts are run with both and the faster is reported for each.
LR_FAST = dict(lr_mean=1.6e-3, lr_rho=2e-2, lr_scale=2e-2, lr_quat=2e-3)
LR_BASE = dict(lr_mean=4e-4, lr_rho=2e-2, lr_scale=1e-2, lr_quat=2e-3)

# pair capacity of the long reconstructions, as a multiple of the starting pair counts: the
# Gaussians grow as they are optimised, and a step that ran out of capacity does incomplete
# work (the runs count the re-plans they needed)
LONG_RUN_HEADROOM = 3.0

# learned start: the MLP on every brick above 5 % of the FDK volume's maximum, the largest-mass
# Gaussians up to the budget, any remainder gradient-sampled from the residual
LEARNED_INIT = dict(frac=0.05)


def _first_at(hist, target):
    """(iteration, gpu ms) of the first evaluation at or above target, or None."""
    return next(((it, ms) for it, ms, db in hist if db >= target), None)


def learned_vs_plain(device, ref_iters=200, max_iters=400, eval_every=5, n_fit=40,
                     train_steps=3000):
    """Per-brick MLP initializer against the FDK-gradient initialisation on the 40-ellipsoid
    phantom (75 cone views of 512^2, 50k Gaussians, 256^3).  The MLP is trained here on the
    voxelization of gs_fit_volume fits of n_fit phantoms with other seeds.  The plain form runs
    ref_iters iterations; its PSNR then is the reference the learned start must reach.
    Reported: PSNR of each start, GPU time (initialisation included) to 35 dB and to the
    reference."""
    import numpy as np
    import torch

    import synth
    from paper_2604_01844_gb300 import initializer as I
    from paper_2604_01844_gb300.mlp import BrickMLP
    from paper_2604_01844_gb300.recon import (PhantomProblem, ReconConfig, Reconstruction,
                                               fdk_volume, gradient_init, psnr_of,
                                               reconstruct_to_psnr)

    views = synth.cone_views(75, 512, 512)
    grid = synth.cube_grid(256)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    X, T, fit_db = I.fit_training_set([10 ** 6 + j for j in range(n_fit)], views, 512, 512,
                                      grid, 50000, fit_iters=100, device=device)
    mlp = BrickMLP(seed=0, device=device)
    hist = I.train(mlp, X, T, steps=train_steps, batch=1024, lr=1e-3)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    n_bricks = int(X.shape[0])
    del X, T
    prob = PhantomProblem(synth.ellipsoid_phantom(1, 40), views, 512, 512, grid, device=device)
    u = np.random.default_rng(7).random((50000, 4)).astype(np.float32)
    sse = torch.zeros(1, dtype=torch.float64, device=device)
    # warm the inference path once (module load, tensor-map set-up) outside the timing
    I.learned_init(mlp, fdk_volume(prob, grid), grid, 50000, u, **LEARNED_INIT)
    out = {"train_ms": round(train_ms, 1), "fits": n_fit, "train_bricks": n_bricks,
           "fit_psnr_db_min_mean": [round(min(fit_db), 2), round(float(np.mean(fit_db)), 2)],
           "train_loss_first_last": [round(hist[0], 5), round(hist[-1], 5)],
           "workload": "40-ellipsoid phantom, 75 cone views x 512^2, 50k Gaussians, 256^3",
           "learned_init": LEARNED_INIT, "ref_iters": ref_iters, "eval_every": eval_every}

    def start(kind):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fdk = fdk_volume(prob, grid)
        if kind == "plain":
            mr, sc, q = gradient_init(fdk, grid, 50000, u)
            n_mlp = 0
        else:
            mr, sc, q, n_mlp = I.learned_init(mlp, fdk, grid, 50000, u, **LEARNED_INIT)
        b.record()
        torch.cuda.synchronize()
        return (mr.cpu().numpy(), sc.cpu().numpy(), q.cpu().numpy()), a.elapsed_time(b), n_mlp

    def run(params, lrs, target, iters):
        rec = Reconstruction(views, 512, 512, prob.proj.clone(), grid, *params,
                             cfg=ReconConfig(**lrs, headroom=LONG_RUN_HEADROOM), device=device)
        p0 = psnr_of(rec.voxelizer.forward(*rec.act), prob.gt, prob.peak, sse)
        h, ok = reconstruct_to_psnr(rec, prob.gt, prob.peak, iters, target, eval_every)
        replans.append(rec.replans)
        return p0, h

    replans = []

    params, init_ms, _ = start("plain")
    p0, h = run(params, LR_FAST, float("inf"), ref_iters)
    ref_db = h[-1][2]
    at35 = _first_at(h, 35.0)
    out["plain"] = {"init_ms": round(init_ms, 2), "psnr_start_db": round(p0, 2),
                    "psnr_ref_db": round(ref_db, 2),
                    "ms_to_ref": round(h[-1][1] + init_ms, 2),
                    "ms_to_35db": round(at35[1] + init_ms, 2) if at35 else None,
                    "iters_to_35db": at35[0] if at35 else None}
    params, init_ms, n_mlp = start("learned")
    runs = []
    for lrs in (LR_FAST, LR_BASE):
        p0, h = run(params, lrs, ref_db, max_iters)
        at35, atref = _first_at(h, 35.0), _first_at(h, ref_db)
        runs.append({"lr_mean": lrs["lr_mean"], "psnr_start_db": round(p0, 2),
                     "ms_to_35db": round(at35[1] + init_ms, 2) if at35 else None,
                     "ms_to_ref": round(atref[1] + init_ms, 2) if atref else None,
                     "iters_to_ref": atref[0] if atref else None,
                     "psnr_last_db": round(h[-1][2], 2)})
    best = min(runs, key=lambda r: r["ms_to_ref"] if r["ms_to_ref"] else float("inf"))
    out["learned"] = {"init_ms": round(init_ms, 2), "gaussians_from_mlp": n_mlp, "runs": runs,
                      "ms_to_ref": best["ms_to_ref"]}
    out["learned_reaches_ref_faster"] = bool(best["ms_to_ref"] and
                                             best["ms_to_ref"] < out["plain"]["ms_to_ref"])
    out["replans"] = replans  # pair-capacity overflows met by the runs (0: every step complete)
    return out


def batched_small_step(device, n_inst=16, seq_steps=20):
    """Where batching pays: n_inst small reconstructions (volumes 64^3-128^3, 16-32 cone views
    of 128^2-192^2, 2k-6k Gaussians, FDK-gradient starts), one optimisation step each.  Times
    the batched step (one rasterizer and voxelizer launch per pass over all instances, the
    whole step in one CUDA graph) against the same instances stepped one by one, each in its
    own graph: a single small step leaves most SMs idle between its short launches."""
    import numpy as np
    import torch

    import synth
    from paper_2604_01844_gb300.batch import BatchGraphStep, BatchReconstruction
    from paper_2604_01844_gb300.recon import (GraphStep, PhantomProblem, ReconConfig,
                                               Reconstruction, fdk_volume, gradient_init)

    specs = synth.batch_specs(seeds=range(200, 200 + n_inst), sides=(64, 96, 128),
                              detectors=(128, 160, 192), views=(16, 32), gaussians=(2000, 6000))
    inst = []
    for sp in specs:
        v = synth.cone_views(sp["n_views"], sp["det"], sp["det"])
        g = synth.cube_grid(sp["side"])
        prob = PhantomProblem(synth.ellipsoid_phantom(sp["seed"], sp["n_ellipsoids"]), v,
                              sp["det"], sp["det"], g, device=device)
        u = np.random.default_rng(sp["seed"]).random((sp["n"], 4)).astype(np.float32)
        mr, sc, q = gradient_init(fdk_volume(prob, g), g, sp["n"], u)
        inst.append(dict(views=v, W=sp["det"], H=sp["det"], target=prob.proj, grid=g,
                         mean_rho=mr.cpu().numpy(), scale=sc.cpu().numpy(),
                         quat=q.cpu().numpy()))
    cfg = ReconConfig(**LR_FAST)

    def timed(step):
        step()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(seq_steps):
            step()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / seq_steps

    rec = BatchReconstruction(inst, cfg=cfg, device=device)
    batched = timed(BatchGraphStep(rec, warmup=1))
    del rec
    one_by_one = 0.0
    for x in inst:
        r = Reconstruction(x["views"], x["W"], x["H"], x["target"], x["grid"], x["mean_rho"],
                           x["scale"], x["quat"], cfg=cfg, device=device)
        one_by_one += timed(GraphStep(r, warmup=1))
        del r
    return {"workload": f"{n_inst} small reconstructions (seeds 200-{199 + n_inst}): volumes "
                        "64^3-128^3, 16-32 cone views of 128^2-192^2, 2k-6k Gaussians",
            "views_total": int(sum(sp["n_views"] for sp in specs)),
            "gaussians_total": int(sum(sp["n"] for sp in specs)),
            "step_ms_batched_graph": round(batched, 3),
            "step_ms_one_by_one_graphs": round(one_by_one, 3),
            "speedup": round(one_by_one / batched, 2)}


def batched_learned_vs_plain(device, ref_iters=200, max_iters=400, eval_every=5, n_fit=48,
                             train_steps=3000, seq_steps=5):
    """16 uneven reconstructions (synth.batch_specs: volumes 128^3-384^3, 25-75 views of
    256^2-512^2, 10k-80k Gaussians, 40-ellipsoid phantoms).  The plain single-instance form
    (FDK-gradient start, each instance stepped alone) runs ref_iters iterations per instance;
    each instance's PSNR then is its reference.  The batched, learned-initialised form (one
    batched rasterizer and voxelizer call per pass, the whole step in one CUDA graph, starts
    from the per-brick MLP trained here on gs_fit_volume fits of n_fit phantoms drawn like the
    instances, other seeds) runs until every instance reaches its reference.  GPU times include
    the initialisations.  Also: the graph step time against the same instances stepped one by
    one (each in its own graph), and the batched plain form to the same references."""
    import numpy as np
    import torch

    import synth
    from paper_2604_01844_gb300 import initializer as I
    from paper_2604_01844_gb300.batch import BatchGraphStep, BatchReconstruction, batch_to_psnr
    from paper_2604_01844_gb300.mlp import BrickMLP
    from paper_2604_01844_gb300.recon import (GraphStep, PhantomProblem, ReconConfig,
                                               Reconstruction, fdk_volume, gradient_init,
                                               reconstruct_to_psnr)

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        return e

    # training set: gs_fit_volume fits of phantoms drawn like the instances (other seeds)
    e0 = ev()
    Xs, Ts, fdb = [], [], []
    for sp in synth.batch_specs(seeds=[10 ** 6 + j for j in range(n_fit)]):
        v = synth.cone_views(sp["n_views"], sp["det"], sp["det"])
        X, T, db = I.fit_training_set([sp["seed"]], v, sp["det"], sp["det"],
                                      synth.cube_grid(sp["side"]), sp["n"], fit_iters=100,
                                      device=device)
        Xs.append(X)
        Ts.append(T)
        fdb += db
    X, T = torch.cat(Xs), torch.cat(Ts)
    del Xs, Ts
    mlp = BrickMLP(seed=0, device=device)
    hist = I.train(mlp, X, T, steps=train_steps, batch=1024, lr=1e-3)
    e1 = ev()
    torch.cuda.synchronize()
    out = {"workload": "16 uneven reconstructions (seeds 100-115): volumes 128^3-384^3, "
                       "25-75 cone views of 256^2-512^2, 10k-80k Gaussians",
           "train_ms": round(e0.elapsed_time(e1), 1), "fits": n_fit,
           "train_bricks": int(X.shape[0]),
           "fit_psnr_db_min_mean": [round(min(fdb), 2), round(float(np.mean(fdb)), 2)],
           "train_loss_first_last": [round(hist[0], 5), round(hist[-1], 5)],
           "ref_iters": ref_iters, "eval_every": eval_every}
    del X, T
    specs = synth.batch_specs()
    probs, grids, views = [], [], []
    for sp in specs:
        v = synth.cone_views(sp["n_views"], sp["det"], sp["det"])
        g = synth.cube_grid(sp["side"])
        probs.append(PhantomProblem(synth.ellipsoid_phantom(sp["seed"], sp["n_ellipsoids"]), v,
                                    sp["det"], sp["det"], g, device=device))
        grids.append(g)
        views.append(v)
    gts, peaks = [p.gt for p in probs], [p.peak for p in probs]
    us = [np.random.default_rng(sp["seed"]).random((sp["n"], 4)).astype(np.float32)
          for sp in specs]
    # warm the MLP inference path once outside the timing
    I.learned_init(mlp, fdk_volume(probs[0], grids[0]), grids[0], specs[0]["n"], us[0])

    def init(kind):
        torch.cuda.synchronize()
        a = ev()
        inst, n_mlp, ms_each = [], 0, []
        for sp, prob, g, v, u in zip(specs, probs, grids, views, us):
            c = ev()
            fdk = fdk_volume(prob, g)
            if kind == "plain":
                mr, sc, q = gradient_init(fdk, g, sp["n"], u)
            else:
                mr, sc, q, nm = I.learned_init(mlp, fdk, g, sp["n"], u, **LEARNED_INIT)
                n_mlp += nm
            d = ev()
            ms_each.append((c, d))
            inst.append(dict(views=v, W=sp["det"], H=sp["det"], target=prob.proj, grid=g,
                             mean_rho=mr, scale=sc, quat=q))
        b = ev()
        torch.cuda.synchronize()
        for x in inst:
            for key in ("mean_rho", "scale", "quat"):
                x[key] = x[key].cpu().numpy()
        return inst, a.elapsed_time(b), n_mlp, [c.elapsed_time(d) for c, d in ms_each]

    # step time: batched graph vs the same instances one by one (each its own graph)
    inst, _, _, _ = init("plain")
    rec = BatchReconstruction(inst, cfg=ReconConfig(**LR_FAST), device=device)
    g = BatchGraphStep(rec, warmup=1)
    g()
    torch.cuda.synchronize()
    a = ev()
    for _ in range(seq_steps):
        g()
    b = ev()
    torch.cuda.synchronize()
    out["step_ms_batched_graph"] = round(a.elapsed_time(b) / seq_steps, 3)
    out["pair_capacity"] = int(rec.projector.capacity)
    del rec, g
    seq_ms = 0.0
    for x in inst:
        r = Reconstruction(x["views"], x["W"], x["H"], x["target"], x["grid"], x["mean_rho"],
                           x["scale"], x["quat"], cfg=ReconConfig(**LR_FAST), device=device)
        gs = GraphStep(r, warmup=1)
        gs()
        torch.cuda.synchronize()
        a = ev()
        for _ in range(seq_steps):
            gs()
        b = ev()
        torch.cuda.synchronize()
        seq_ms += a.elapsed_time(b) / seq_steps
        del r, gs
    out["step_ms_one_by_one_graphs"] = round(seq_ms, 3)

    # the plain single-instance form, instance after instance: its references
    refs, plain_ms, plain35, plain_replans = [], 0.0, 0.0, 0
    for x, init_k, gt, pk in zip(inst, init("plain")[3], gts, peaks):
        r = Reconstruction(x["views"], x["W"], x["H"], x["target"], x["grid"], x["mean_rho"],
                           x["scale"], x["quat"],
                           cfg=ReconConfig(**LR_FAST, headroom=LONG_RUN_HEADROOM), device=device)
        h, _ = reconstruct_to_psnr(r, gt, pk, ref_iters, float("inf"), eval_every)
        plain_replans += r.replans
        refs.append(h[-1][2])
        plain_ms += h[-1][1] + init_k
        at35 = _first_at(h, 35.0)
        plain35 = plain35 + at35[1] + init_k if (at35 and plain35 is not None) else None
        del r
    out["plain_one_by_one"] = {"ms_to_ref": round(plain_ms, 1),
                               "ms_to_35db": round(plain35, 1) if plain35 else None,
                               "psnr_ref_db": [round(x, 2) for x in refs],
                               "replans": plain_replans}
    init("learned")  # first use of the learned start's buffers, outside the timing
    for kind, lr_sets in (("learned", [LR_FAST, LR_BASE]), ("plain", [LR_FAST])):
        inst, init_ms, n_mlp, _ = init(kind)
        runs = []
        for lrs in lr_sets:
            cfg = ReconConfig(**lrs, headroom=LONG_RUN_HEADROOM)
            # to each instance's reference, finished instances leaving the batch
            rec = BatchReconstruction(inst, cfg=cfg, device=device)
            hist = []
            reached, last, iters, ms = batch_to_psnr(rec, gts, peaks, max_iters, refs,
                                                     eval_every, history=hist, retire=True)
            ok = all(r is not None for r in reached)
            del rec
            # to 35 dB, the same way
            rec = BatchReconstruction(inst, cfg=cfg, device=device)
            h35 = []
            r35, _, it35, ms35 = batch_to_psnr(rec, gts, peaks, max_iters, 35.0, eval_every,
                                               history=h35, retire=True)
            ok35 = all(r is not None for r in r35)
            runs.append({"lr_mean": lrs["lr_mean"], "all_reached": ok, "iters": iters,
                         "ms_to_ref": round(ms + init_ms, 1) if ok else None,
                         "iters_per_instance": [r[0] if r else None for r in reached],
                         "psnr_last_min_margin_db": round(min(l - t for l, t in
                                                              zip(last, refs)), 2),
                         "ms_to_35db": round(ms35 + init_ms, 1) if ok35 else None,
                         "iters_to_35db_per_instance": [r[0] if r else None for r in r35],
                         "replans": hist[-1][4] + h35[-1][4]})
            del rec
        best = min(runs, key=lambda r: r["ms_to_ref"] if r["ms_to_ref"] else float("inf"))
        b35 = min((r["ms_to_35db"] for r in runs if r["ms_to_35db"]), default=None)
        out["batched_" + kind] = {"init_ms": round(init_ms, 1), "gaussians_from_mlp": n_mlp,
                                  "runs": runs, "ms_to_ref": best["ms_to_ref"],
                                  "ms_to_35db": b35}
    bl = out["batched_learned"]["ms_to_ref"]
    out["batched_learned_reaches_refs_faster"] = bool(bl and bl < plain_ms)
    b35 = out["batched_learned"]["ms_to_35db"]
    out["batched_learned_reaches_35db_faster"] = bool(b35 and plain35 and b35 < plain35)
    out["retire"] = ("an instance leaves the batch at the first evaluation at which it has "
                     "reached its target; the rest continue as a smaller batch (re-planned, "
                     "graph captured again, inside the timed span)")
    return out


def warm_start_study(device, side=512, det=1024, n_views=50, n=100000, fit_iters=50,
                     n_iter=400, eval_every=5, factor=5, seed=1, n_ell=120):
    """Prior-volume warm start against the cold (FDK-gradient) start, on the protocol of the
    paper's warm-start study: target = projections of a phantom (n_views cone views of det^2,
    side^3 grid), prior = the same phantom at a `factor` times coarser slice spacing resized to
    the grid, fit of n Gaussians to the prior for fit_iters iterations (Eq. 6), then n_iter
    reconstruction iterations (Eq. 5) from each start.  Reports both trajectories' best PSNR and
    3D SSIM and tau_iter, the fraction of the n_iter iterations the warm start needs to reach
    the cold start's best."""
    import numpy as np
    import torch

    import synth
    from paper_2604_01844_gb300.recon import (PhantomProblem, ReconConfig, Reconstruction,
                                               fdk_volume, gradient_init)
    from paper_2604_01844_gb300.warmstart import (VolumeScore, fit_prior, tau_iter,
                                                   trajectory)

    views = synth.cone_views(n_views, det, det)
    grid = synth.cube_grid(side)
    prob = PhantomProblem(synth.ellipsoid_phantom(seed, n_ell), views, det, det, grid,
                          device=device)
    prior = torch.from_numpy(synth.thick_slices(prob.gt.cpu().numpy(), factor)).to(device)
    score = VolumeScore(prob.gt, prob.peak)
    prior_db = score.psnr(prior)
    prior_ssim = score.ssim(prior)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    u = np.random.default_rng(7).random((n, 4)).astype(np.float32)
    ev[0].record()
    fdk = fdk_volume(prob, grid)
    cold0 = gradient_init(fdk, grid, n, u)
    ev[1].record()
    ev[2].record()
    (mr, sc, q), fit = fit_prior(prior, grid, n, fit_iters, torch.from_numpy(u).to(device))
    ev[3].record()
    torch.cuda.synchronize()
    fit_ok = fit.status().code == 0
    del fdk
    cfg = ReconConfig(**LR_FAST)
    res = {}
    for name, start in (("cold", cold0), ("warm", (mr, sc, q))):
        rec = Reconstruction(views, det, det, prob.proj, grid, *[t.cpu().numpy() for t in start],
                             cfg=cfg, device=device)
        traj, replans = trajectory(rec, score, n_iter, eval_every, graph=True)
        res[name] = traj
        res[name + "_replans"] = replans
        del rec
        torch.cuda.empty_cache()
    cold, warm = res["cold"], res["warm"]

    def best(t, c):
        return max(r[c] for r in t)

    def summary(t):
        return {"psnr_start_db": round(t[0][2], 2), "ssim_start": round(t[0][3], 4),
                "psnr_best_db": round(best(t, 2), 2), "ssim_best": round(best(t, 3), 4),
                "ms_per_iteration": round(t[-1][1] / n_iter, 3),
                "psnr_db_every": [round(r[2], 2) for r in t[::max(1, len(t) // 8)]]}

    return {"workload": f"{n_ell}-ellipsoid phantom, {n_views} cone views x {det}^2, {side}^3, "
                        f"{n} Gaussians; prior = the phantom at {factor}x slice spacing",
            "prior_psnr_db": round(prior_db, 2), "prior_ssim": round(prior_ssim, 4),
            "fit_iters": fit_iters, "fit_ms": round(ev[2].elapsed_time(ev[3]), 2),
            "fit_ok": fit_ok, "fdk_init_ms": round(ev[0].elapsed_time(ev[1]), 2),
            "n_iter": n_iter, "eval_every": eval_every, "cold": summary(cold),
            "warm": summary(warm), "replans": [res["cold_replans"], res["warm_replans"]],
            "tau_iter_psnr": tau_iter(cold, warm, n_iter, 2),
            "tau_iter_ssim": tau_iter(cold, warm, n_iter, 3),
            "note": "tau_iter = first evaluated warm iteration reaching the cold start's best "
                    "within n_iter, / n_iter; trajectories evaluated every eval_every iterations"}


def adaptive_control(device, n0=25000, budget=50000, iters=400, eval_every=50,
                     grad_threshold=7e-5):
    """Adaptive density control (prune / clone / split) on the 40-ellipsoid phantom, 75 cone
    views of 512^2, 256^3: n0 Gaussians from the FDK-gradient initialiser, densified every 100
    iterations from iteration 100 to 300 up to `budget`, against the same start kept at n0.
    Reports both PSNR trajectories, the events' counts and the gs_densify time at the budget."""
    import ctypes

    import numpy as np
    import torch

    import synth
    from paper_2604_01844_gb300 import binding as B
    from paper_2604_01844_gb300.density import DensifyConfig, DensityControl
    from paper_2604_01844_gb300.evaluate import VolumeScore, trajectory
    from paper_2604_01844_gb300.recon import (PhantomProblem, ReconConfig, Reconstruction,
                                               fdk_volume, gradient_init)

    views = synth.cone_views(75, 512, 512)
    grid = synth.cube_grid(256)
    prob = PhantomProblem(synth.ellipsoid_phantom(1, 40), views, 512, 512, grid, device=device)
    fdk = fdk_volume(prob, grid)
    score = VolumeScore(prob.gt, prob.peak)
    u = np.random.default_rng(7).random((n0, 4)).astype(np.float32)
    start = [t.cpu().numpy() for t in gradient_init(fdk, grid, n0, u)]
    cfg = DensifyConfig(start=100, interval=100, stop=301, max_gaussians=budget,
                        grad_threshold=grad_threshold)
    out = {}
    for name, dens in (("fixed", None), ("densified", cfg)):
        rec = Reconstruction(views, 512, 512, prob.proj, grid, *start,
                             cfg=ReconConfig(**LR_FAST), device=device)
        ctrl = DensityControl(rec, dens) if dens else None
        traj, _ = trajectory(rec, score, iters, eval_every, ssim=False, graph=True,
                             control=ctrl)
        out[name] = {"psnr_db_every_%d" % eval_every: [round(r[2], 2) for r in traj],
                     "ms": round(traj[-1][1], 1), "gaussians_final": rec.n}
        if ctrl:
            out[name]["events"] = ctrl.history
            # gs_densify alone on the final set (statistics of one more window), CUDA events
            for _ in range(3):
                rec.step()
            n = rec.n
            normals = torch.randn(n, 6, device=device)
            o = ctrl.opts
            cap = 2 * n
            bufs = [torch.empty((cap, 4), device=device) for _ in range(3)]
            om = torch.empty((3 * cap, 4), device=device)
            ov = torch.empty_like(om)
            ws = torch.empty(B.lib().gs_densify_workspace_size(n), dtype=torch.uint8,
                             device=device)

            def call():
                B.check(B.lib().gs_densify(
                    *[B.ptr(t) for t in rec.raw], B.ptr(rec.m), B.ptr(rec.v), B.ptr(ctrl.stat),
                    B.ptr(ctrl.vis), B.ptr(normals), n, ctypes.byref(o),
                    *[B.ptr(t) for t in bufs], B.ptr(om), B.ptr(ov), cap, B.ptr(ws), ws.numel(),
                    B.stream_handle()), "gs_densify")
            for _ in range(3):
                call()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(20):
                call()
            e1.record()
            e1.synchronize()
            out[name]["densify_call_ms"] = round(e0.elapsed_time(e1) / 20, 4)
        del rec, ctrl
        torch.cuda.empty_cache()
    out.update({"workload": f"40-ellipsoid phantom, 75 cone views x 512^2, 256^3; {n0} Gaussians "
                            f"(FDK-gradient init), densified up to {budget}",
                "rules": {"grad_threshold": grad_threshold, "split_scale": cfg.split_scale,
                          "split_factor": cfg.split_factor, "min_density": cfg.min_density,
                          "max_scale": cfg.max_scale, "schedule": "iterations 100, 200, 300"},
                "note": "PSNR evaluated right after each densification event (iterations 100, "
                        "200, 300) shows the event's immediate effect"})
    return out


def compression(device, side=256, n=40000, iters=500, seed=1, n_ell=40):
    """The paper's volume fitting and compression study on a synthetic volume: n Gaussians
    fitted to a side^3 phantom volume (gs_fit_volume, `iters` iterations), stored as the FP16
    codec (22 bytes per Gaussian) and voxelized on demand; size, PSNR and 3D SSIM against the
    volume, beside the FP32 Gaussians, the raw FP32 volume and a zlib-compressed uint8 volume.
    (The paper's JPEG-stack baseline needs a JPEG encoder, which this image does not have.)"""
    import zlib

    import numpy as np
    import torch

    import synth
    from paper_2604_01844_gb300 import codec
    from paper_2604_01844_gb300.evaluate import VolumeScore
    from paper_2604_01844_gb300.fit import VolumeFit, fit_opts
    from paper_2604_01844_gb300.recon import PhantomProblem
    from paper_2604_01844_gb300.voxelizer import Voxelizer

    grid = synth.cube_grid(side)
    prob = PhantomProblem(synth.ellipsoid_phantom(seed, n_ell), synth.cone_views(2, 16, 16), 16,
                          16, grid, device=device)
    gt = prob.gt
    score = VolumeScore(gt, prob.peak)
    u = torch.from_numpy(np.random.default_rng(11).random((n, 4)).astype(np.float32)).to(device)
    fit = VolumeFit(grid, n)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    params = fit.run(gt, iters, fit_opts(data_range=prob.peak), u)
    ev[1].record()
    torch.cuda.synchronize()
    fit_ok = fit.status().code == 0
    vol32 = Voxelizer(grid, device=device).forward(*params)
    bits = codec.encode(*params)
    cv = codec.CodecVoxelizer(grid, device=device)
    vol16 = cv.forward(bits)
    for _ in range(3):
        cv.forward(bits, out=vol16)
    ev[2].record()
    for _ in range(10):
        cv.forward(bits, out=vol16)
    ev[3].record()
    torch.cuda.synchronize()
    host = gt.cpu().numpy()
    lo, hi = float(host.min()), float(host.max())
    q8 = np.round((host - lo) / (hi - lo) * 255.0).astype(np.uint8)
    zipped = len(zlib.compress(q8.tobytes(), 9))
    deq = torch.from_numpy(q8.astype(np.float32) / 255.0 * (hi - lo) + lo).to(device)
    codec_zip = len(zlib.compress(bits.cpu().numpy().tobytes(), 9))
    mb = 1e-6
    rows = {
        "raw_float32": {"mb": round(gt.numel() * 4 * mb, 3)},
        "uint8_zlib": {"mb": round(zipped * mb, 3), "psnr_db": round(score.psnr(deq), 2),
                       "ssim": round(score.ssim(deq), 4)},
        "gaussians_fp32": {"mb": round(n * 44 * mb, 3), "psnr_db": round(score.psnr(vol32), 2),
                           "ssim": round(score.ssim(vol32), 4)},
        "gaussians_fp16_codec": {"mb": round(bits.numel() * 2 * mb, 3),
                                 "psnr_db": round(score.psnr(vol16), 2),
                                 "ssim": round(score.ssim(vol16), 4),
                                 "mb_zlib": round(codec_zip * mb, 3)},
        "jpeg_stack": "unavailable on this box: no JPEG encoder in the image",
    }
    return {"workload": f"{n_ell}-ellipsoid phantom sampled on {side}^3; {n} Gaussians fitted "
                        f"for {iters} iterations (L1 + 0.2 D-SSIM3D)",
            "fit_ms": round(ev[0].elapsed_time(ev[1]), 1), "fit_ok": fit_ok,
            "on_demand_voxelize_ms": round(ev[2].elapsed_time(ev[3]) / 10, 3),
            "formats": rows,
            "note": "sizes in 10^6 bytes; PSNR = 10 log10(max^2 / MSE), SSIM = 11^3 window"}


def scale_up(device, steps=5, warmup=3):
    """Reconstruction steps at the larger detector sizes: 75 cone views of 1024^2 with 200k
    Gaussians, TV on 512^3 and the sorted lists rebuilt in the backward; 75 views of 2048^2
    with 500k Gaussians, TV on the voxelized 1024^3 volume; raster tile chosen by the
    autotuner at both.  Gaussian scales give footprints of about 4 and 6 pixels (sigma)."""
    import numpy as np
    import torch

    import synth
    from paper_2604_01844_gb300.autotune import tune_tile
    from paper_2604_01844_gb300.projector import Projector
    from paper_2604_01844_gb300.recon import ReconConfig, Reconstruction

    out = {}
    for name, side, n, vol, median, recompute, tuned in (
            ("75x1024^2, 200k Gaussians, TV 512^3, lists rebuilt in backward, autotuned tile",
             1024, 200000, 512, 0.0123, True, True),
            ("75x2048^2, 500k Gaussians, TV 1024^3, autotuned tile", 2048, 500000, 1024,
             0.0088, False, True)):
        views = synth.cone_views(75, side, side)
        model = synth.gaussians(21, n, radius=0.8, scale_median=median, scale_sigma_log=0.4)
        tgt = synth.gaussians(22, n, radius=0.8, scale_median=median, scale_sigma_log=0.4)
        d_tgt = [torch.from_numpy(a).to(device) for a in tgt]
        tile, tune_ms = 16, None
        if tuned:
            d_model = [torch.from_numpy(a).to(device) for a in model]
            tile, tune_ms = tune_tile(views, side, side, *d_model, device=device)
            del d_model
        target = Projector(views, side, side, tile=tile, device=device).forward(*d_tgt).clone()
        del d_tgt
        cfg = ReconConfig(tile=tile, recompute_lists=recompute)
        rec = Reconstruction(views, side, side, target, synth.cube_grid(vol), *model, cfg=cfg,
                             device=device)
        evals = rec.projector.count_evals(*rec.act)
        rec.plan()
        for _ in range(warmup):
            rec.step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            rec.step()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        out[name] = {"ms_per_step": round(ms, 3), "evals_per_step": evals,
                     "value": evals / (ms * 1e-3), "unit": "evals/s", "tile": tile,
                     "tile_timings_ms": tune_ms, "status": 1 if rec.overflowed() else 0}
        del rec, target
        torch.cuda.empty_cache()
    return out


def fit_volume_rate(device, side=1024, n=500000, iters=4, warmup=2):
    """gs_fit_volume of n Gaussians to a side^3 ground truth (120-ellipsoid phantom):
    Gaussian-voxel evaluations per second of the fit iterations (forward voxelization's
    in-cut evaluations per iteration / ms per iteration)."""
    import numpy as np
    import torch

    import synth
    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300 import binding as B
    from paper_2604_01844_gb300.fit import VolumeFit, fit_opts

    grid = synth.cube_grid(side)
    ell = torch.from_numpy(synth.ellipsoid_phantom(3, 120).astype(np.float32)).to(device)
    gt = torch.empty((side, side, side), dtype=torch.float32, device=device)
    import ctypes

    B.check(B.lib().gs_phantom_voxelize(B.ptr(ell), 120, ctypes.byref(B.grid_struct(grid)),
                                        B.ptr(gt), B.stream_handle()), "gs_phantom_voxelize")
    u = torch.from_numpy(np.random.default_rng(11).random((n, 4)).astype(np.float32)).to(device)
    f = VolumeFit(grid, n, max_pairs=16 * n, device=device)
    opts = fit_opts(data_range=float(gt.abs().max()))
    f.run(gt, warmup, opts, u)  # init + warm-up iterations (16-voxel bricks)
    torch.cuda.synchronize()
    # the voxelizer's brick side chosen by the autotuner on the fit's current Gaussians
    from paper_2604_01844_gb300.autotune import tune_brick

    brick, brick_ms = tune_brick(grid, *f.params, device=device)
    opts.brick = brick
    opts.init = 0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    loss = torch.zeros(iters, device=device)
    e0.record()
    torch.cuda.nvtx.range_push("fit_volume_timed")  # lets a profiler select these launches
    f.run(gt, iters, opts, None, loss)
    torch.cuda.nvtx.range_pop()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    # per-kernel breakdown from one more (separately timed) pass of the same iterations
    B.timing_reset()
    B.timing_enable(True)
    f.run(gt, iters, opts, None, loss)
    per_kernel = {k: round(v[1] / iters, 3) for k, v in
                  sorted(B.timing_read().items(), key=lambda kv: -kv[1][1])}
    B.timing_enable(False)
    st = f.status()
    vox = g.Voxelizer(grid, device=device)
    evals = vox.count_evals(*f.params)
    del vox, f, gt
    torch.cuda.empty_cache()
    # the volume passes' HBM rooflines: algorithmic bytes per voxel (each input and output
    # volume once; halos and re-reads not counted) over the measured copy bandwidth
    nvox = side ** 3
    hbm = (measured_peaks() or {}).get("hbm_gbs")
    bytes_per_voxel = {
        "ssim3d_fwd": 20,     # fused streaming forward: X, Y in; three maps out
        "ssim3d_bwd": 24,     # fused streaming backward: three maps, X and Y in; the gradient out
        "ssim3d_z_fwd": 28,   # X, Y in; five moments out
        "ssim3d_z_bwd": 24,   # three maps in; three filtered maps out
        "ssim3d_xy_fwd": 32,  # five moments in; three maps out
        "ssim3d_xy_bwd": 24,  # three filtered maps, X and Y in; the gradient out
        "vox_fwd": 4,         # the volume out
        "vox_bwd": 4,         # dL/dV in
    }
    hbm_roofs = {}
    for k, bpv in bytes_per_voxel.items():
        if k in per_kernel and per_kernel[k] > 0 and hbm:
            gbs = bpv * nvox / (per_kernel[k] * 1e-3) / 1e9
            hbm_roofs[k] = {"bytes_per_voxel": bpv, "achieved_gbs": round(gbs, 1),
                            "peak_gbs": hbm, "frac": round(gbs / hbm, 3)}
    # the fused 3D SSIM kernels are bound by shared memory, not HBM: per output voxel they move
    # the TMA-staged boxes in, the y pass's loads and stores, the x pass's 11 loads of the
    # column's channels and the fused L1 term's x, y (forward 269 B, backward 259 B) through
    # the SM's 128 B/clock shared-memory pipe
    sms_ = torch.cuda.get_device_properties(device).multi_processor_count
    fmax_ = (measured_peaks() or {}).get("sm_max_mhz", 2070.0)
    smem_peak = 128.0 * sms_ * fmax_ * 1e6 / 1e9  # GB/s
    smem_roofs = {}
    for k, bpv in {"ssim3d_fwd": 269, "ssim3d_bwd": 259}.items():
        if k in per_kernel and per_kernel[k] > 0:
            gbs = bpv * nvox / (per_kernel[k] * 1e-3) / 1e9
            smem_roofs[k] = {"smem_bytes_per_voxel": bpv, "achieved_gbs": round(gbs, 1),
                             "peak_gbs": round(smem_peak, 1), "frac": round(gbs / smem_peak, 3)}
    # the voxel passes against their binding roofline: the larger of the HBM floor (the volume
    # or dL/dV streamed once, 4 B per voxel) and the ALU floor (in-cut evaluations at the
    # evaluation rate of the FP32 / ex2 unit counts at the maximum SM clock, with the scope's
    # per-evaluation figure; the folded count's floor beside it)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    f_max = (measured_peaks() or {}).get("sm_max_mhz", 2070.0)
    vox_roofs = {}
    for k in ("vox_fwd", "vox_bwd"):
        if k in per_kernel and per_kernel[k] > 0 and hbm:
            hbm_ms = 4.0 * nvox / (hbm * 1e9) * 1e3
            alu_ms = evals / eval_peak(k, sms, f_max, SCOPE_OPS_PER_EVAL)[0] * 1e3
            alu_f_ms = evals / eval_peak(k, sms, f_max)[0] * 1e3
            floor = max(hbm_ms, alu_ms)
            vox_roofs[k] = {"ms": per_kernel[k], "hbm_floor_ms": round(hbm_ms, 4),
                            "alu_floor_ms": round(alu_ms, 4),
                            "alu_floor_folded_count_ms": round(alu_f_ms, 4),
                            "frac_folded_count": round(max(hbm_ms, alu_f_ms) / per_kernel[k], 3),
                            "bound": "hbm" if hbm_ms >= alu_ms else "alu",
                            "frac": round(floor / per_kernel[k], 3),
                            "evals_per_s": evals / (per_kernel[k] * 1e-3)}
    return {"workload": f"gs_fit_volume, {n} Gaussians, {side}^3 ground truth",
            "brick": brick, "brick_timings_ms": {k: round(v, 3) for k, v in brick_ms.items()},
            "ms_per_iter": round(ms, 3), "voxel_evals_per_iter": evals,
            "value": evals / (ms * 1e-3), "unit": "Gaussian-voxel evals/s",
            "status": int(st.code), "loss_last": float(loss[-1].item()),
            "kernels_ms_per_iter": per_kernel,
            "hbm_rooflines": hbm_roofs, "smem_rooflines": smem_roofs, "vox_rooflines": vox_roofs,
            "hbm_note": "achieved = algorithmic bytes per voxel x voxels / kernel ms; the voxel "
                        "passes' frac is their binding floor (HBM or ALU) over their time"}


def gemm_rate(device, M=118016, reps=20, warmup=3):
    """CUDA-event throughput of the tcgen05 BF16 GEMM (gs_gemm_bf16) at the per-brick MLP's
    layer shapes for M bricks (forward layers, the first layer's weight gradient and a hidden
    layer's input gradient), against the measured bf16 peak.  2 M N K flops per call."""
    import torch

    from paper_2604_01844_gb300 import binding as B

    shapes = {"fwd_l1 (Mx256x4096)": (M, 256, 4096), "fwd_l2 (Mx256x256)": (M, 256, 256),
              "fwd_l4 (Mx384x256)": (M, 384, 256), "dW_l1 (256x4096xM)": (256, 4096, M),
              "dX_l4 (Mx256x384)": (M, 256, 384)}
    mp = measured_peaks() or {}
    peak = mp.get("bf16_tflops")
    err = torch.zeros(1, dtype=torch.int32, device=device)
    out = {}
    g = torch.Generator(device=device)
    g.manual_seed(0)
    for name, (m, n, k) in shapes.items():
        a = torch.randn((m, k), device=device, generator=g).to(torch.bfloat16)
        b = torch.randn((n, k), device=device, generator=g).to(torch.bfloat16)
        c = torch.empty((m, n), device=device, dtype=torch.bfloat16)
        s = B.stream_handle()

        def call():
            B.check(B.lib().gs_gemm_bf16(B.ptr(a), B.ptr(b), m, n, k, None, 0, None, B.ptr(c), n,
                                         B.ptr(err), s), "gs_gemm_bf16")

        for _ in range(warmup):
            call()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            call()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        tf = 2.0 * m * n * k / (ms * 1e-3) / 1e12
        out[name] = {"ms": round(ms, 4), "tflops": round(tf, 1),
                     "frac_of_measured_bf16": round(tf / peak, 3) if peak else None}
        del a, b, c
    out["status"] = int(err.item())
    out["peak_tflops"] = peak
    out["note"] = ("back-to-back calls of one shape (operands L2-resident for the smaller ones); "
                   "BF16 output, no bias")
    return out


SWEEP_SCALE = 0.01     # isotropic Gaussian scale of the kernel sweep (world units; cube side 2)
SWEEP_N = 20000        # Gaussians of the resolution sweep
SWEEP_SIDES = (256, 512, 1024, 2048)          # one cone view of side^2 pixels
SWEEP_VOL_SIDES = (64, 128, 256, 512, 1024)   # side^3 voxels
SWEEP_COUNTS = (5000, 10000, 20000, 40000, 80000, 160000, 320000)
SWEEP_PX_SIDE, SWEEP_VOX_SIDE = 1024, 96      # about 1e6 pixels / voxels (96: whole bricks)


def power_law(xs, ys):
    """Least-squares exponent k and prefactor a of y = a x^k on a log-log scale."""
    import numpy as np

    lx, ly = np.log(np.asarray(xs, float)), np.log(np.asarray(ys, float))
    k, c = np.polyfit(lx, ly, 1)
    return float(k), float(np.exp(c))


def _graph_ms(fn, reps=10, warmup=3, replays=5):
    """Device ms per call of fn: reps calls captured in one CUDA graph, the graph replayed and
    timed with CUDA events (no host launch overhead inside the timed region)."""
    import torch

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(warmup):
            fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(reps):
            fn()
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(replays):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / (reps * replays)


def kernel_sweep(device, seed=5):
    """The paper's kernel micro-benchmark (Sec. 3.5, Fig. 3): Gaussians with zero rotation and
    one isotropic scale (0.01 world units, the cube being [-1, 1]^3), centres uniform in the
    radius-0.8 ball, densities U(0.05, 1); (a) 20k Gaussians with the resolution varied: one
    cone view of side^2 pixels (the rasterizer) and a side^3 volume (the voxelizer); (b) about
    1e6 outputs (one 1024^2 view, a 96^3 volume) with the Gaussian count varied.  Per point:
    device ms of the forward (gs_project: projection, keys, sort, ranges, raster; gs_voxelize
    likewise) and of the backward with the forward's lists, from CUDA graphs of back-to-back
    calls; the in-cut evaluations; and the power-law exponent of each series (time ~ N^k)."""
    import torch

    import synth
    import paper_2604_01844_gb300 as g

    def gaussians(n):
        mr, sc, qt = synth.gaussians(seed, n, radius=0.8, scale_median=SWEEP_SCALE,
                                     scale_sigma_log=0.0, isotropic=True,
                                     identity_rotation=True)
        return [torch.from_numpy(a).to(device) for a in (mr, sc, qt)]

    def raster_point(side, d):
        proj = g.Projector(synth.cone_views(1, side, side), side, side, tile=16, device=device)
        img = proj.forward(*d)
        dimg = torch.randn(img.shape, device=device, generator=torch.Generator(
            device=device).manual_seed(side))
        grads = tuple(torch.empty_like(t) for t in d)
        fwd = _graph_ms(lambda: proj.forward(*d, out=img))
        bwd = _graph_ms(lambda: proj.backward(*d, dimg, grads=grads, reuse=True))
        evals = proj.count_evals(*d)
        ok = proj.status().code == 0
        del proj, img, dimg, grads
        return {"fwd_ms": round(fwd, 4), "bwd_ms": round(bwd, 4), "evals": evals,
                "evals_per_s_fwd": evals / (fwd * 1e-3), "status": 0 if ok else 1}

    def voxel_point(side, d):
        vox = g.Voxelizer(synth.cube_grid(side), device=device)
        vol = vox.forward(*d)
        dvol = torch.randn(vol.shape, device=device, generator=torch.Generator(
            device=device).manual_seed(side))
        grads = tuple(torch.empty_like(t) for t in d)
        fwd = _graph_ms(lambda: vox.forward(*d, out=vol))
        bwd = _graph_ms(lambda: vox.backward(*d, dvol, grads=grads, reuse=True))
        evals = vox.count_evals(*d)
        ok = vox.status().code == 0
        del vox, vol, dvol, grads
        torch.cuda.empty_cache()
        return {"fwd_ms": round(fwd, 4), "bwd_ms": round(bwd, 4), "evals": evals,
                "evals_per_s_fwd": evals / (fwd * 1e-3), "status": 0 if ok else 1}

    d = gaussians(SWEEP_N)
    by_res_r = {str(s): raster_point(s, d) for s in SWEEP_SIDES}
    by_res_v = {str(s): voxel_point(s, d) for s in SWEEP_VOL_SIDES}
    by_n_r, by_n_v = {}, {}
    for n in SWEEP_COUNTS:
        dn = gaussians(n)
        by_n_r[str(n)] = raster_point(SWEEP_PX_SIDE, dn)
        by_n_v[str(n)] = voxel_point(SWEEP_VOX_SIDE, dn)

    def fits(series, keys, xs):
        out = {}
        for key in ("fwd_ms", "bwd_ms"):
            k, a = power_law(xs, [series[str(x)][key] for x in keys])
            out[key] = {"exponent": round(k, 3), "prefactor_ms": a}
        return out

    return {
        "workload": f"kernel micro-benchmark: identity rotation, isotropic scale {SWEEP_SCALE}, "
                    "centres uniform in the radius-0.8 ball, rho U(0.05, 1); (a) "
                    f"{SWEEP_N} Gaussians, one cone view of side^2 / a side^3 volume; (b) one "
                    f"{SWEEP_PX_SIDE}^2 view / a {SWEEP_VOX_SIDE}^3 volume, Gaussian count varied",
        "raster_by_side": by_res_r, "voxel_by_side": by_res_v,
        "raster_by_gaussians": by_n_r, "voxel_by_gaussians": by_n_v,
        "power_laws": {
            "raster_vs_pixels": fits(by_res_r, SWEEP_SIDES, [s * s for s in SWEEP_SIDES]),
            "voxel_vs_voxels": fits(by_res_v, SWEEP_VOL_SIDES, [s ** 3 for s in SWEEP_VOL_SIDES]),
            "raster_vs_gaussians": fits(by_n_r, SWEEP_COUNTS, SWEEP_COUNTS),
            "voxel_vs_gaussians": fits(by_n_v, SWEEP_COUNTS, SWEEP_COUNTS),
        },
        "paper_context": "rasterizer on one 2K image with 20k Gaussians: 9.3 ms on an RTX 4070 "
                         "Ti SUPER (whether forward or forward + backward is not stated)",
        "note": "device time from CUDA graphs of 10 back-to-back calls, each forward including "
                "its projection, keys, sort and ranges; backward with the forward's lists",
    }


def read_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary (profiles/traffic.txt:
    lines '<kernel> <bytes per launch> <source>'), or None."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) >= 2 and parts[0] == kernel and not line.startswith("#"):
                try:
                    return float(parts[1])
                except ValueError:
                    return None
    return None


# ------------------------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and the reference arm)
# ------------------------------------------------------------------------------------------
def oracle_sample(model, views, n_views, nthreads=0):
    """Oracle forward + gradient (fwd+bwd) over the first n_views views with all Gaussians, on
    nthreads host threads (0: all); returns (in-cut evaluations, seconds)."""
    import numpy as np

    import oracle

    P = oracle.params64(*model)
    V = oracle.views64(views[:n_views])
    W, H = WORKLOAD["W"], WORKLOAD["H"]
    t0 = time.perf_counter()
    img, n_eval = oracle.project(P, V, W, H, nthreads=nthreads)
    dimg = np.sign(img - 0.5 * img.mean())  # an L1-style upstream gradient
    oracle.project_grad(P, V, W, H, dimg, nthreads=nthreads)
    return n_eval, time.perf_counter() - t0


def cpu_baseline(model, views, target_s=15.0):
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    n_eval, t = oracle_sample(model, views, 2)
    nv = int(min(len(views), max(2, round(2 * target_s / max(t, 1e-3)))))
    if nv > 2:
        n_eval, t = oracle_sample(model, views, nv)
    n1, t1 = oracle_sample(model, views, 1, nthreads=1)
    return {"value": n_eval / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle fwd + dual-number bwd of all {WORKLOAD['gaussians']} Gaussians "
                      f"on {nv} of the 75 views (512^2), {n_eval} in-cut evaluations in {t:.1f} s, "
                      f"OpenMP over {cores} host threads",
            "single_thread": {"value": n1 / t1, "unit": UNIT, "cores": 1,
                              "sample": f"the same on the first view, one host thread: {n1} "
                                        f"in-cut evaluations in {t1:.1f} s"}}


REF_BUDGET_S = 150.0  # seconds of timed oracle work in the reference arm


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import synth
    import oracle

    oracle.build()
    w = WORKLOAD
    views = synth.cone_views(w["views"], w["W"], w["H"])
    model = synth.gaussians(w["model_seed"], w["gaussians"], scale_median=w["scale_median"],
                            scale_sigma_log=w["scale_sigma_log"])
    per_step_views = 1
    # one step is the oracle on one view; when the K timed steps would take longer than
    # REF_BUDGET_S on these cores, each step takes the first n of the Gaussians instead
    # (evaluations are counted exactly either way)
    n_all = w["gaussians"]
    _, t1 = oracle_sample(model, views, per_step_views)
    n_sub = n_all
    if args.steps * t1 > REF_BUDGET_S:
        n_sub = max(1000, int(n_all * REF_BUDGET_S / (args.steps * t1)))
    sub = tuple(a[:n_sub] for a in model)
    for _ in range(max(args.warmup - 1, 0)):
        oracle_sample(sub, views, per_step_views)
    tot_e, tot_t = 0, 0.0
    for _ in range(args.steps):
        e, t = oracle_sample(sub, views, per_step_views)
        tot_e += e
        tot_t += t
    cores = os.cpu_count() or 1
    val = tot_e / tot_t
    which = f"all {n_all}" if n_sub == n_all else f"the first {n_sub} of the {n_all}"
    sample = (f"each step: FP64 oracle fwd + dual-number bwd of {which} Gaussians on "
              f"{per_step_views} of the 75 views (512^2)")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": w["workload"], "views": w["views"],
                      "detector": [w["W"], w["H"]], "gaussians": w["gaussians"]},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the time-to-PSNR and volume-fit measurements")
    ap.add_argument("--extras", default="all",
                    help="comma-separated study legs to run after the headline step "
                         "(time_to_psnr, learned_init, batched, fit_volume, scale_up, "
                         "warm_start, adaptive_control, compression, gemm, batched_small, "
                         "kernel_sweep) "
                         "or 'all'")
    ap.add_argument("--fit-side", type=int, default=1024)
    ap.add_argument("--fit-gaussians", type=int, default=500000)
    ap.add_argument("--warm-side", type=int, default=512)
    ap.add_argument("--warm-det", type=int, default=1024)
    ap.add_argument("--parallel", choices=["replicas", "views"], default="replicas",
                    help="N > 1: independent replicas of the step (weak scaling), or one "
                         "reconstruction with its views sharded over the processes and one "
                         "gradient all-reduce per step (strong scaling)")
    ap.add_argument("--workload", choices=["recon512", "small"], default="recon512",
                    help="small: 16-view case of the same kernels, for profiler captures")
    args = ap.parse_args()
    if args.workload == "small":
        WORKLOAD.clear()
        WORKLOAD.update(SMALL)
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        if args.warmup < 3:
            log("warning: fewer than 3 warm-up steps")
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
