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
    "views": 75, "W": 512, "H": 512, "gaussians": 50000, "tv_volume": 256, "tile": 16,
    "model_seed": 21, "target_seed": 22, "scale_median": 0.012, "scale_sigma_log": 0.4,
}
# a reduced case of the same kernels for profiler captures (16 views, 128^3 TV volume)
SMALL = dict(WORKLOAD, workload="recon step, 16 cone views x 512^2, 50k Gaussians, TV on 128^3",
             views=16, tv_volume=128)
METRIC = "Gaussian-pixel evals/s (fwd+bwd step) at 75x512^2"
UNIT = "evals/s"

# evaluations per SM clock at the ALU roofline of the evaluation kernels:
# forward: one ex2 per evaluation on 16 SFU lanes/SM/clk; backward: ~16 FP32 ops per
# evaluation on 128 FP32 lanes/SM/clk.
EVALS_PER_SM_CLK = {"raster_fwd": 16.0, "raster_bwd": 8.0, "vox_fwd": 16.0, "vox_bwd": 8.0}


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
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
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

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def build_problem(device):
    import numpy as np
    import torch

    import synth
    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300.recon import ReconConfig, Reconstruction

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
    rec = Reconstruction(views, w["W"], w["H"], target, grid, *model, cfg=cfg, device=device)
    return rec, model, views


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300 import binding as B
    from paper_2604_01844_gb300 import build as gbuild

    gbuild.build()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=device)
    rec, model, views = build_problem(device)
    # algorithmic work of one step: in-cut Gaussian-pixel evaluations of the projection
    evals_px = rec.projector.count_evals(*rec.act)
    evals_vox = rec.voxelizer.count_evals(*rec.act)
    rec.plan()
    for _ in range(args.warmup):
        rec.step()
    torch.cuda.synchronize()
    st = rec.projector.status()
    if st.code != 0:
        raise RuntimeError(f"projector workspace status {st.code}")

    clocks = ClockSampler(local)
    stream = torch.cuda.current_stream()
    B.timing_reset()
    B.timing_enable(True)
    launches0 = B.launch_count()
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        rec.step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    B.timing_enable(False)
    launches = B.launch_count() - launches0
    per_kernel = B.timing_read()
    ms = e0.elapsed_time(e1) / args.steps
    if ws > 1:
        import torch.distributed as dist

        t = torch.tensor([ms], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    loss = float(rec.loss.item())

    # end to end through the public API with host buffers: per step the parameters and the
    # target projections go host->device from pinned memory, the loss and the updated
    # parameters come back device->host
    h_params = [t.detach().cpu().pin_memory() for t in rec.raw]
    h_target = rec.target.detach().cpu().pin_memory()
    h_out = [torch.empty_like(t, device="cpu").pin_memory() for t in rec.act]
    h_loss = torch.empty(1, dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * 4 for t in h_params) + h_target.numel() * 4
    d2h = sum(t.numel() * 4 for t in h_out) + 4
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        for d, h in zip(rec.raw, h_params):
            d.copy_(h, non_blocking=True)
        rec.target.copy_(h_target, non_blocking=True)
        rec.activate()
        rec.step()
        for d, h in zip(rec.act, h_out):
            h.copy_(d, non_blocking=True)
        h_loss.copy_(rec.loss, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e2.elapsed_time(e3) / args.steps
    if ws > 1:
        import torch.distributed as dist

        t = torch.tensor([ms_e2e], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_e2e = float(t.item())

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
    if name in EVALS_PER_SM_CLK:
        units = evals_px if name.startswith("raster") else evals_vox
        peak = sms * f_mhz * 1e6 * EVALS_PER_SM_CLK[name] / 1e9
        ach = units / (avg_ms * 1e-3) / 1e9
        roof = {"kernel": name, "bound": "alu", "achieved": round(ach, 2), "peak": round(peak, 2),
                "unit": "Geval/s", "frac": round(ach / peak, 4), "traffic": read_traffic(name),
                "peak_basis": f"{sms} SMs x {f_mhz:.0f} MHz (median sampled) x "
                              f"{EVALS_PER_SM_CLK[name]:g} evals/SM/clk",
                "avg_launch_ms": round(avg_ms, 4), "launches": nl}
    else:
        roof = {"kernel": name, "bound": "hbm", "achieved": None, "peak": mp.get("hbm_gbs"),
                "unit": "GB/s", "frac": None, "traffic": read_traffic(name),
                "avg_launch_ms": round(avg_ms, 4), "launches": nl}

    value = evals_px / (ms * 1e-3) * ws
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD["workload"], "views": WORKLOAD["views"],
                   "detector": [WORKLOAD["W"], WORKLOAD["H"]], "gaussians": WORKLOAD["gaussians"],
                   "tv_volume": WORKLOAD["tv_volume"], "tile": WORKLOAD["tile"],
                   "evals_per_step": evals_px, "voxel_evals_per_step": evals_vox,
                   "target": "projections of a second seeded Gaussian set",
                   "l2": "working set per step > 0.5 GB (images, SSIM maps, 256^3 volume) > L2",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": roof,
        "kernels_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in
                                sorted(per_kernel.items(), key=lambda kv: -kv[1][1])},
        "e2e": {"value": evals_px / (ms_e2e * 1e-3) * ws, "unit": UNIT, "ms_per_step": ms_e2e,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "loss": loss,
    }
    if ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(model, views, target_s=args.cpu_seconds)
    print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


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
def oracle_sample(model, views, n_views):
    """Oracle forward + gradient (fwd+bwd) over the first n_views views with all Gaussians;
    returns (in-cut evaluations, seconds)."""
    import numpy as np

    import oracle

    P = oracle.params64(*model)
    V = oracle.views64(views[:n_views])
    W, H = WORKLOAD["W"], WORKLOAD["H"]
    t0 = time.perf_counter()
    img, n_eval = oracle.project(P, V, W, H)
    dimg = np.sign(img - 0.5 * img.mean())  # an L1-style upstream gradient
    oracle.project_grad(P, V, W, H, dimg)
    return n_eval, time.perf_counter() - t0


def cpu_baseline(model, views, target_s=15.0):
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    n_eval, t = oracle_sample(model, views, 2)
    nv = int(min(len(views), max(2, round(2 * target_s / max(t, 1e-3)))))
    if nv > 2:
        n_eval, t = oracle_sample(model, views, nv)
    return {"value": n_eval / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle fwd + dual-number bwd of all {WORKLOAD['gaussians']} Gaussians "
                      f"on {nv} of the 75 views (512^2), {n_eval} in-cut evaluations in {t:.1f} s, "
                      f"OpenMP over {cores} host threads"}


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
    for _ in range(args.warmup):
        oracle_sample(model, views, per_step_views)
    tot_e, tot_t = 0, 0.0
    for _ in range(args.steps):
        e, t = oracle_sample(model, views, per_step_views)
        tot_e += e
        tot_t += t
    cores = os.cpu_count() or 1
    val = tot_e / tot_t
    sample = (f"each step: FP64 oracle fwd + dual-number bwd of all {w['gaussians']} Gaussians on "
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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
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
