"""Volume fit (Sec. 3.6, Eq. 6) through gs_fit_volume."""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import binding as B


def fit_opts(alpha_ssim=0.2, lr_mean=5e-4, lr_rho=2e-2, lr_scale=1e-2, lr_quat=5e-3,
             threshold_frac=0.05, density_k=0.15, data_range=0.0, init=True,
             min_scale=1e-4, max_scale=0.5, brick=16) -> B.GsFitOpts:
    o = B.GsFitOpts()
    o.alpha_ssim, o.lr_mean, o.lr_rho, o.lr_scale, o.lr_quat = alpha_ssim, lr_mean, lr_rho, lr_scale, lr_quat
    o.beta1, o.beta2, o.eps = 0.9, 0.999, 1e-15
    o.min_log_scale, o.max_log_scale = math.log(min_scale), math.log(max_scale)
    o.threshold_frac, o.density_k, o.data_range, o.cut = threshold_frac, density_k, data_range, 3.0
    o.init = 1 if init else 0
    o.brick = int(brick)
    return o


class VolumeFit:
    """Owns the workspace and parameter buffers of a fit of n Gaussians to a volume."""

    def __init__(self, grid, n: int, max_pairs: int | None = None, device="cuda"):
        self.device = torch.device(device)
        self.grid = B.grid_struct(grid)
        self.n = int(n)
        self.max_pairs = int(max_pairs if max_pairs is not None else 12 * n + 4096)
        nbytes = B.lib().gs_fit_volume_workspace_size(self.n, ctypes.byref(self.grid),
                                                      self.max_pairs)
        if nbytes == 0:
            raise B.GsError("invalid fit sizes")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.params = [torch.zeros((self.n, 4), dtype=torch.float32, device=self.device)
                       for _ in range(3)]

    def run(self, vol_gt: torch.Tensor, iters: int, opts: B.GsFitOpts, uniforms=None,
            loss: torch.Tensor | None = None):
        if opts.init and uniforms is None:
            raise ValueError("init = 1 needs 4n uniforms")
        B.check(B.lib().gs_fit_volume(
            B.ptr(vol_gt.contiguous()), ctypes.byref(self.grid), self.n, int(iters),
            ctypes.byref(opts), B.ptr(uniforms), *[B.ptr(t) for t in self.params], B.ptr(loss),
            B.ptr(self.ws), self.ws.numel(), B.stream_handle()), "gs_fit_volume")
        return self.params

    def status(self) -> B.GsStatus:
        st = B.GsStatus()
        B.check(B.lib().gs_fit_volume_status(B.ptr(self.ws), self.ws.numel(), self.n,
                                             ctypes.byref(self.grid), B.stream_handle(),
                                             ctypes.byref(st)), "gs_fit_volume_status")
        return st
