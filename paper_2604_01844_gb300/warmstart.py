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
from .evaluate import VolumeScore, trajectory  # noqa: F401  (re-exported)


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
