"""Autotuner of the raster tile size (8, 16 or 32 pixels): times forward + backward of the
actual inputs for each candidate with CUDA events and caches the winner per shape class
(views, detector size, Gaussian count rounded to a power of two, device)."""
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
