"""Learned initialisation with the per-brick MLP: training set from seeded phantoms (FDK bricks
as inputs, ground-truth bricks as targets, both scaled by 1 / max(FDK)), training, and the
inference that turns the FDK of a new scan into Gaussians (32 per non-empty 16^3 brick),
topped up by gradient sampling when the budget is not filled."""
from __future__ import annotations

import numpy as np
import torch

import synth

from . import binding as B
from .mlp import BrickMLP, brick_ids, extract
from .recon import PhantomProblem, fdk_volume, gradient_init


def _nonempty(vol: torch.Tensor, frac: float) -> np.ndarray:
    """Mask of 16^3 bricks whose max exceeds frac * max(vol) (vol dims multiple of 16)."""
    nz, ny, nx = vol.shape
    v = vol.reshape(nz // 16, 16, ny // 16, 16, nx // 16, 16).amax(dim=(1, 3, 5))
    return (v > frac * float(vol.max())).reshape(-1).cpu().numpy()


def training_set(seeds, views, W, H, grid, n_ell=(20, 60), device="cuda"):
    """Returns (x16 (n, 4096) bf16, target (n, 4096) f32) over the non-empty bricks."""
    xs, ts = [], []
    for s in seeds:
        rng = np.random.default_rng(s)
        ell = synth.ellipsoid_phantom(s, int(rng.integers(n_ell[0], n_ell[1] + 1)))
        prob = PhantomProblem(ell, views, W, H, grid, device=device)
        fdk = fdk_volume(prob, grid)
        scale = 1.0 / max(float(fdk.max()), 1e-6)
        nz, ny, nx = fdk.shape
        keep = _nonempty(fdk, 0.05)
        ids = torch.from_numpy(brick_ids((nx // 16, ny // 16, nz // 16), keep)).to(device)
        xs.append(extract(fdk, ids, scale, True))
        ts.append(extract(prob.gt, ids, scale, False))
    return torch.cat(xs), torch.cat(ts)


def train(mlp: BrickMLP, x16, target, steps=1500, batch=1024, lr=1e-3, seed=0):
    """Adam on random batches; returns the loss of every 100th step (synchronising there)."""
    n = x16.shape[0]
    batch = min(batch, n - n % 128)
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    loss = torch.zeros(1, device=x16.device)
    for it in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g).to(x16.device)
        if it % 100 == 0:
            loss.zero_()
        mlp.train_step(x16[idx].contiguous(), target[idx].contiguous(), loss, lr=lr)
        if it % 100 == 99:
            hist.append(float(loss.item()))
    return hist


def learned_init(mlp: BrickMLP, fdk: torch.Tensor, grid, budget: int, uniforms: np.ndarray,
                 frac=0.05, mlp_share: float = 1.0, min_rho_frac: float = 0.0):
    """Gaussians for a new scan: MLP on the non-empty bricks of its FDK volume (the
    `mlp_share * budget / 32` brightest bricks if there are more), dropping MLP Gaussians whose
    density is below `min_rho_frac` of the largest, topped up by gradient sampling."""
    dev = fdk.device
    nz, ny, nx = fdk.shape
    fmax = max(float(fdk.max()), 1e-6)
    nb = (nx // 16, ny // 16, nz // 16)
    vmax = fdk.reshape(nz // 16, 16, ny // 16, 16, nx // 16, 16).amax(dim=(1, 3, 5)).reshape(-1)
    order = torch.argsort(vmax, descending=True).cpu().numpy()
    keep_n = int(min((vmax > frac * fmax).sum().item(), int(budget * mlp_share) // 32))
    keep_n -= keep_n % 128  # the GEMM tiles 128 rows
    keep_n = max(keep_n, 128)
    sel = np.zeros(vmax.numel(), dtype=bool)
    sel[order[:keep_n]] = True
    ids_np = brick_ids(nb, sel)
    ids = torch.from_numpy(ids_np).to(dev)
    x16 = extract(fdk, ids, 1.0 / fmax, True)
    o = np.asarray(grid["origin"], dtype=np.float32).ravel()
    h = float(np.asarray(grid["voxel"]).ravel()[0])
    geo = np.stack([o[0] + ids_np[:, 0] * 16 * h, o[1] + ids_np[:, 1] * 16 * h,
                    o[2] + ids_np[:, 2] * 16 * h, np.full(len(ids_np), h)], 1).astype(np.float32)
    mr, sc, q = mlp.infer_gaussians(x16, torch.from_numpy(geo).to(dev), amp=fmax)
    if min_rho_frac > 0.0:
        keep = mr[:, 3] > min_rho_frac * mr[:, 3].max()
        mr, sc, q = mr[keep], sc[keep], q[keep]
    n_mlp = mr.shape[0]
    if n_mlp < budget:
        extra = gradient_init(fdk, grid, budget - n_mlp, uniforms[: budget - n_mlp])
        mr, sc, q = (torch.cat([a, b]) for a, b in zip((mr, sc, q), extra))
    return mr[:budget].contiguous(), sc[:budget].contiguous(), q[:budget].contiguous(), n_mlp
