"""FP64 CPU oracle for the loss terms of the reconstruction and volume-fit objectives
(Eq. 5 and Eq. 6) -- TEST INFRASTRUCTURE ONLY.

Plain PyTorch float64 CPU ops; gradients come from torch.autograd of these definitions.

  * L1          : mean |a - b|                                   (Eq. 5, Eq. 6)
  * SSIM (2D)   : Wang et al. 2004 structural similarity with an 11x11 Gaussian window,
                  sigma 1.5, zero-padded 'same' filtering, C1 = (0.01 L)^2, C2 = (0.03 L)^2,
                  averaged over all pixels of all views; the loss term is 1 - SSIM (Eq. 5).
  * SSIM (3D)   : the same with an 11x11x11 window over a volume (Eq. 6).
  * TV (3D)     : anisotropic total variation with forward differences, summed over the three
                  axes where the neighbour exists and divided by the voxel count (Eq. 5).
  * PSNR        : 10 log10(max(gt)^2 / MSE) over the whole volume.
The paper does not print these formulas; the textbook definitions above are the readings.
"""
from __future__ import annotations

import math

import torch
import torch.nn.functional as F

WIN = 11
SIGMA = 1.5


def gaussian_window_1d(size: int = WIN, sigma: float = SIGMA) -> torch.Tensor:
    k = torch.arange(size, dtype=torch.float64) - (size - 1) / 2
    w = torch.exp(-(k * k) / (2 * sigma * sigma))
    return w / w.sum()


def l1(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    return (a - b).abs().mean()


def _ssim_map(mu_x, mu_y, sxx, syy, sxy, C1, C2):
    return ((2 * mu_x * mu_y + C1) * (2 * sxy + C2)) / ((mu_x ** 2 + mu_y ** 2 + C1) * (sxx + syy + C2))


def ssim2d(x: torch.Tensor, y: torch.Tensor, data_range: float) -> torch.Tensor:
    """Mean SSIM of x against y; x, y are (V, H, W) float64."""
    w1 = gaussian_window_1d()
    w2 = torch.outer(w1, w1)[None, None]
    pad = WIN // 2

    def filt(t):
        return F.conv2d(t[:, None], w2, padding=pad)[:, 0]

    C1 = (0.01 * data_range) ** 2
    C2 = (0.03 * data_range) ** 2
    mu_x, mu_y = filt(x), filt(y)
    sxx = filt(x * x) - mu_x ** 2
    syy = filt(y * y) - mu_y ** 2
    sxy = filt(x * y) - mu_x * mu_y
    return _ssim_map(mu_x, mu_y, sxx, syy, sxy, C1, C2).mean()


def ssim3d(x: torch.Tensor, y: torch.Tensor, data_range: float) -> torch.Tensor:
    """Mean SSIM of volume x against y; (D, H, W) float64."""
    w1 = gaussian_window_1d()
    w3 = (w1[:, None, None] * w1[None, :, None] * w1[None, None, :])[None, None]
    pad = WIN // 2

    def filt(t):
        return F.conv3d(t[None, None], w3, padding=pad)[0, 0]

    C1 = (0.01 * data_range) ** 2
    C2 = (0.03 * data_range) ** 2
    mu_x, mu_y = filt(x), filt(y)
    sxx = filt(x * x) - mu_x ** 2
    syy = filt(y * y) - mu_y ** 2
    sxy = filt(x * y) - mu_x * mu_y
    return _ssim_map(mu_x, mu_y, sxx, syy, sxy, C1, C2).mean()


def tv3d(v: torch.Tensor) -> torch.Tensor:
    """Anisotropic TV of a (D, H, W) volume, divided by the voxel count."""
    dz = (v[1:, :, :] - v[:-1, :, :]).abs().sum()
    dy = (v[:, 1:, :] - v[:, :-1, :]).abs().sum()
    dx = (v[:, :, 1:] - v[:, :, :-1]).abs().sum()
    return (dx + dy + dz) / v.numel()


def psnr(v: torch.Tensor, gt: torch.Tensor) -> float:
    mse = float(((v - gt) ** 2).mean())
    peak = float(gt.max())
    return 10.0 * math.log10(peak * peak / mse) if mse > 0 else float("inf")


def value_and_grad(fn, x, *args):
    """(value, d value / d x) of a scalar loss fn(x, *args), in float64."""
    xt = torch.as_tensor(x, dtype=torch.float64).clone().requires_grad_(True)
    out = fn(xt, *[torch.as_tensor(a, dtype=torch.float64) if not isinstance(a, (int, float)) else a
                   for a in args])
    (g,) = torch.autograd.grad(out, xt)
    return float(out), g.numpy()
