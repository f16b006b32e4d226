"""Warm start of a reconstruction from a volumetric prior (Sec. 3.6; the warm-start study of
the appendix).

A prior volume (an earlier or lower-resolution scan of the same object) is turned into a
Gaussian set by the voxelizer-based fit of Eq. 6 (gs_fit_volume: gradient sampling from the
prior, then voxelize -> L1 + alpha_ssim D-SSIM3D -> voxelizer backward -> Adam), and that set
is the starting point of the projection-domain reconstruction (Eq. 5) in place of the
FDK-gradient initialisation.  The Gaussians are continuous, so the prior's grid may differ from
the reconstruction's.

The study's measure is tau_iter: the fraction of the cold start's iteration budget that the
warm start needs to first reach the best score (PSNR, 3D SSIM) the cold start reached within
that budget.
"""
from __future__ import annotations

import torch

from . import binding as B
from .fit import VolumeFit, fit_opts
from .recon import psnr_of


def fit_prior(prior_vol: torch.Tensor, prior_grid, n: int, iters: int, uniforms: torch.Tensor,
              opts: B.GsFitOpts | None = None, max_pairs: int | None = None):
    """n Gaussians fitted to prior_vol ([z][y][x] on prior_grid) in `iters` iterations of
    Eq. 6, starting from gradient sampling of the prior (uniforms: (n, 4) device floats).
    Returns the activated (mean_rho, scale, quat) device tensors and the VolumeFit (whose
    status() reports a voxelizer capacity overflow)."""
    if opts is None:
        opts = fit_opts(data_range=float(prior_vol.abs().max()))
    if not opts.init:
        raise ValueError("a prior fit starts from gradient sampling (opts.init = 1)")
    fit = VolumeFit(prior_grid, n, max_pairs=max_pairs, device=prior_vol.device)
    params = fit.run(prior_vol, iters, opts, uniforms.contiguous())
    return params, fit


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
               graph: bool = False):
    """Runs `iters` steps of rec (a recon.Reconstruction; graph = True replays the step as one
    CUDA graph) and scores its voxelized volume at iteration 0 and every eval_every
    iterations.  Returns ([(iteration, GPU ms of the steps so far, PSNR, SSIM or None)],
    re-plans): at each evaluation point a pair-capacity overflow of the steps since the last
    one is detected, and the workspaces are re-planned (and the graph captured again).  The
    scoring itself is not timed."""
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
        e1.record()
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        it += k
        if rec.projector.status().code != B.GS_OK or rec.voxelizer.status().code != B.GS_OK:
            rec.plan()
            replans += 1
            if graph:
                step = GraphStep(rec, warmup=0)
        vol = rec.voxelizer.forward(*rec.act)
        out.append((it, ms, score.psnr(vol), score.ssim(vol) if ssim else None))
    return out, replans


def tau_iter(cold, warm, n_iter: int, col: int):
    """The study's normalised iteration ratio for score column `col` of two trajectories
    (2 = PSNR, 3 = SSIM): the first evaluated warm-start iteration whose score reaches the cold
    start's best within n_iter iterations, divided by n_iter; None if the warm start never
    reaches it within its trajectory."""
    best = max(r[col] for r in cold if r[0] <= n_iter)
    for r in warm:
        if r[col] >= best:
            return r[0] / n_iter
    return None


def first_reaching(traj, col: int, target: float):
    """(iteration, GPU ms) of the first trajectory entry whose score reaches target, or None."""
    for r in traj:
        if r[col] >= target:
            return r[0], r[1]
    return None
