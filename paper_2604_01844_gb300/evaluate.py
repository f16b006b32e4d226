"""Scoring a reconstruction against its ground-truth volume along the optimisation: PSNR from
the library's FP64 SSE, 3D SSIM from its value-only SSIM call, and a stepping loop that
scores at fixed intervals, re-plans after a pair-capacity overflow and applies adaptive
density control on its schedule."""
from __future__ import annotations

import torch

from . import binding as B
from .recon import psnr_of


class VolumeScore:
    """PSNR and 3D SSIM of a volume against a fixed ground truth, from the library's FP64 SSE
    and its value-only 3D SSIM (both synchronise on the read-back)."""

    def __init__(self, gt: torch.Tensor, peak: float | None = None):
        self.gt = gt.contiguous()
        self.peak = float(peak if peak is not None else float(gt.max()))
        self.sse = torch.zeros(1, dtype=torch.float64, device=gt.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=gt.device)
        self.ws = torch.empty(B.lib().gs_ssim3d_workspace_size(gt.numel()), dtype=torch.uint8,
                              device=gt.device)

    def psnr(self, vol: torch.Tensor) -> float:
        return psnr_of(vol, self.gt, self.peak, self.sse)

    def ssim(self, vol: torch.Tensor) -> float:
        L = B.lib()
        s = B.stream_handle()
        dz, dy, dx = self.gt.shape
        B.check(L.gs_memset(B.ptr(self.loss), 0, 4, s), "gs_memset")
        B.check(L.gs_ssim3d_loss(B.ptr(vol), B.ptr(self.gt), dx, dy, dz, self.peak, 1.0,
                                 B.ptr(self.loss), None, 0, B.ptr(self.ws), self.ws.numel(), s),
                "gs_ssim3d_loss")
        return 1.0 - float(self.loss.item())


def trajectory(rec, score: VolumeScore, iters: int, eval_every: int = 5, ssim: bool = True,
               graph: bool = False, control=None):
    """Runs `iters` steps of rec (a recon.Reconstruction; graph = True replays the step as one
    CUDA graph) and scores its voxelized volume at iteration 0 and every eval_every
    iterations.  Returns ([(iteration, GPU ms of the steps so far, PSNR, SSIM or None)],
    re-plans): at each evaluation point a pair-capacity overflow of the steps since the last
    one is detected, and the workspaces are re-planned (and the graph captured again).
    control: a density.DensityControl, applied after the steps it is due (the graph is then
    captured again; its time is included).  The scoring itself is not timed."""
    from .recon import GraphStep

    step = GraphStep(rec, warmup=0) if graph else rec.step
    vol = rec.voxelizer.forward(*rec.act)
    out = [(0, 0.0, score.psnr(vol), score.ssim(vol) if ssim else None)]
    ms = 0.0
    it = 0
    replans = 0
    while it < iters:
        k = min(eval_every, iters - it)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            step()
            it += 1
            if control is not None and control.after_step(it) and graph:
                step = GraphStep(rec, warmup=0)
        e1.record()
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        if rec.overflowed():
            rec.plan()
            replans += 1
            if graph:
                step = GraphStep(rec, warmup=0)
        vol = rec.voxelizer.forward(*rec.act)
        out.append((it, ms, score.psnr(vol), score.ssim(vol) if ssim else None))
    return out, replans
