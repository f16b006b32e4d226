"""Autotuners of the rasterizer's tile size (8, 16 or 32 pixels) and of the voxelizer's brick
size (16, 32 or 64 voxels): each times forward + backward of the actual inputs for every
candidate with CUDA events, discards candidates whose run reported an error status, and
caches the winner per shape class (views and detector size, or grid and region; Gaussian
count rounded to a power of two; device).  Neither choice changes the results: images do not
depend on the tile (per-pixel cut) and volumes do not depend on the brick (bit for bit)."""
from __future__ import annotations

import math

import torch

from . import binding as B
from .projector import Projector

_CACHE: dict = {}


def shape_class(n_views: int, W: int, H: int, n: int, device) -> tuple:
    name = torch.cuda.get_device_name(device)
    return (n_views, W, H, 1 << max(0, int(math.log2(max(n, 1)))), name)


def tune_tile(views, W: int, H: int, mean_rho, scale, quat, candidates=(8, 16, 32),
              repeats: int = 3, device="cuda", cut: float = 3.0) -> tuple[int, dict]:
    """Returns (best tile, {tile: ms of forward + backward})."""
    key = shape_class(len(views) if not isinstance(views, torch.Tensor) else views.shape[0],
                      W, H, mean_rho.shape[0], device)
    if key in _CACHE:
        return _CACHE[key]
    times = {}
    dimg = None
    for t in candidates:
        proj = Projector(views, W, H, tile=t, cut=cut, device=device)
        proj.ensure_capacity(mean_rho, scale, quat)
        img = proj.forward(mean_rho, scale, quat)
        if dimg is None:
            dimg = torch.randn_like(img)
        proj.backward(mean_rho, scale, quat, dimg)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(repeats):
            proj.forward(mean_rho, scale, quat, out=img)
            proj.backward(mean_rho, scale, quat, dimg, reuse=True)
        e1.record()
        torch.cuda.synchronize()
        if proj.status().code == B.GS_OK:  # a run that skipped work is no candidate
            times[t] = e0.elapsed_time(e1) / repeats
        del proj
    if not times:
        raise B.GsError("no raster tile size ran without error")
    best = min(times, key=times.get)
    _CACHE[key] = (best, times)
    return best, times


def tune_brick(grid, mean_rho, scale, quat, roi_lo=(0, 0, 0), roi_dim=None,
               candidates=(16, 32, 64), repeats: int = 3, device="cuda",
               cut: float = 3.0) -> tuple[int, dict]:
    """Returns (best brick side, {brick: ms of voxelizer forward + backward})."""
    import numpy as np

    from .voxelizer import Voxelizer

    dims = tuple(int(x) for x in np.asarray(grid["dims"]).ravel())
    key = ("brick", dims, tuple(roi_lo), tuple(roi_dim) if roi_dim is not None else None,
           1 << max(0, int(math.log2(max(int(mean_rho.shape[0]), 1)))),
           torch.cuda.get_device_name(device))
    if key in _CACHE:
        return _CACHE[key]
    times = {}
    dvol = None
    for b in candidates:
        vox = Voxelizer(grid, roi_lo, roi_dim, cut=cut, brick=b, device=device)
        vox.ensure_capacity(mean_rho, scale, quat)
        vol = vox.forward(mean_rho, scale, quat)
        if dvol is None:
            dvol = torch.randn_like(vol)
        grads = vox.backward(mean_rho, scale, quat, dvol)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(repeats):
            vox.forward(mean_rho, scale, quat, out=vol)
            vox.backward(mean_rho, scale, quat, dvol, grads=grads, reuse=True)
        e1.record()
        torch.cuda.synchronize()
        if vox.status().code == B.GS_OK:
            times[b] = e0.elapsed_time(e1) / repeats
        del vox, vol, grads
    del dvol
    if not times:
        raise B.GsError("no voxel brick size ran without error")
    best = min(times, key=times.get)
    _CACHE[key] = (best, times)
    return best, times
