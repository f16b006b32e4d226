"""Learned initialisation with the per-brick MLP: training sets from seeded phantoms (FDK
bricks as inputs; as targets the voxelization of a gs_fit_volume fit of the phantom, or the
ground-truth bricks themselves; both scaled by 1 / max(FDK)), training, and the inference that
turns the FDK of a new scan into Gaussians (32 per non-empty 16^3 brick), topped up by gradient
sampling when the budget is not filled."""
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


def fit_training_set(seeds, views, W, H, grid, n_gauss: int, fit_iters: int = 100,
                     n_ell=(20, 60), device="cuda"):
    """Training bricks whose targets come from gs_fit_volume: for every seeded phantom the
    ground-truth volume is fitted with n_gauss Gaussians (gradient initialisation, then
    fit_iters iterations of Eq. 6) and the fitted set is voxelized; inputs are the FDK bricks
    of the phantom's projections.  Returns (x16 (n, 4096) bf16, target (n, 4096) f32, fit
    PSNRs) over the non-empty bricks; one fit per seed."""
    from .fit import VolumeFit, fit_opts
    from .recon import psnr_of
    from .voxelizer import Voxelizer

    xs, ts, fit_db = [], [], []
    pairs = 16 * n_gauss
    fit = VolumeFit(grid, n_gauss, max_pairs=pairs, device=device)
    vox = Voxelizer(grid, device=device)
    sse = torch.zeros(1, dtype=torch.float64, device=device)
    for s in seeds:
        rng = np.random.default_rng(s)
        ell = synth.ellipsoid_phantom(s, int(rng.integers(n_ell[0], n_ell[1] + 1)))
        prob = PhantomProblem(ell, views, W, H, grid, device=device)
        fdk = fdk_volume(prob, grid)
        u = torch.from_numpy(rng.random((n_gauss, 4)).astype(np.float32)).to(device)
        for _ in range(4):
            fit.run(prob.gt, fit_iters, fit_opts(data_range=prob.peak), u)
            if fit.status().code == B.GS_OK:
                break
            # the Gaussians outgrew the fit's pair capacity: redo the fit with twice the room
            pairs *= 2
            fit = VolumeFit(grid, n_gauss, max_pairs=pairs, device=device)
        else:
            raise B.GsError("gs_fit_volume kept running out of pair capacity")
        vox.ensure_capacity(*fit.params)  # each fitted set has its own pair count
        fitted = vox.forward(*fit.params)
        fit_db.append(psnr_of(fitted, prob.gt, prob.peak, sse))
        scale = 1.0 / max(float(fdk.max()), 1e-6)
        nz, ny, nx = fdk.shape
        keep = _nonempty(fdk, 0.05)
        ids = torch.from_numpy(brick_ids((nx // 16, ny // 16, nz // 16), keep)).to(device)
        xs.append(extract(fdk, ids, scale, True))
        ts.append(extract(fitted, ids, scale, False))
    return torch.cat(xs), torch.cat(ts), fit_db


def train(mlp: BrickMLP, x16, target, steps=1500, batch=1024, lr=1e-3, seed=0, warmup=300):
    """Adam on random batches, the learning rate ramped linearly from lr / warmup to lr over
    the first `warmup` steps; returns the summed loss of every 100 steps (synchronising there).
    Adam's first steps move every weight by about lr whatever the gradient's size.  Without
    the ramp, at lr = 1e-3, half of the training sets that differ from one another only in the
    last bits of their targets (the fits' atomic sums) fell within 100 steps into one plateau
    (loss 1.32 against 0.43) and never left it.  With it none did, and the loss after 3000
    steps is unchanged."""
    n = x16.shape[0]
    batch = min(batch, n - n % 128)
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    loss = torch.zeros(1, device=x16.device)
    for it in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g).to(x16.device)
        if it % 100 == 0:
            loss.zero_()
        ramp = min(1.0, (it + 1) / warmup) if warmup > 0 else 1.0
        mlp.train_step(x16[idx].contiguous(), target[idx].contiguous(), loss, lr=lr * ramp)
        if it % 100 == 99:
            hist.append(float(loss.item()))
    return hist


def learned_init(mlp: BrickMLP, fdk: torch.Tensor, grid, budget: int, uniforms: np.ndarray,
                 frac: float = 0.05, mlp_share: float = 1.0, vox=None, min_scale: float = 1.5):
    """Gaussians for a new scan from its FDK volume: the MLP's 32 Gaussians for every 16^3
    brick whose maximum exceeds `frac` of the volume's (the brick list padded with the next
    brightest bricks to the GEMM's 128-row tile).  Over mlp_share of the budget, the Gaussians
    of largest mass (rho sx sy sz) are kept; the rest of the budget is sampled by the gradient
    initialisation from the residual max(FDK - voxelized MLP set, 0), so that it goes where the
    MLP's set falls short.  vox: a Voxelizer of `grid` to reuse for the residual.
    min_scale: every axis of the MLP's Gaussians is raised to at least this many voxels, the
    density lowered so that each Gaussian keeps its mass (rho sx sy sz).  The network, trained on
    16^3 bricks, puts out thin Gaussians (median minor axis 0.06 voxel); a reconstruction
    started from them converges more slowly.  Measured on the 40-ellipsoid phantom (75 views of
    512^2, 256^3, 50k Gaussians): the start 34.4 -> 34.7 dB, 400 iterations 39.9 -> 41.5 dB
    (floors of 1 and 2 voxels 41.4 dB, 3 voxels 40.8 dB).  Returns (mean_rho, scale, quat,
    Gaussians from the MLP)."""
    from .voxelizer import Voxelizer

    dev = fdk.device
    nz, ny, nx = fdk.shape
    fmax = max(float(fdk.max()), 1e-6)
    nb = (nx // 16, ny // 16, nz // 16)
    vmax = fdk.reshape(nz // 16, 16, ny // 16, 16, nx // 16, 16).amax(dim=(1, 3, 5)).reshape(-1)
    if vmax.numel() < 128:
        raise ValueError("the learned start needs a volume of at least 128 bricks of 16^3")
    order = torch.argsort(vmax, descending=True).cpu().numpy()
    n_sel = int((vmax > frac * fmax).sum().item())
    n_sel = min(max(128, -(-n_sel // 128) * 128), vmax.numel() - vmax.numel() % 128)
    sel = np.zeros(vmax.numel(), dtype=bool)
    sel[order[:n_sel]] = True
    ids_np = brick_ids(nb, sel)
    x16 = extract(fdk, torch.from_numpy(ids_np).to(dev), 1.0 / fmax, True)
    o = np.asarray(grid["origin"], dtype=np.float32).ravel()
    h = float(np.asarray(grid["voxel"]).ravel()[0])
    geo = np.stack([o[0] + ids_np[:, 0] * 16 * h, o[1] + ids_np[:, 1] * 16 * h,
                    o[2] + ids_np[:, 2] * 16 * h, np.full(len(ids_np), h)], 1).astype(np.float32)
    mr, sc, q = mlp.infer_gaussians(x16, torch.from_numpy(geo).to(dev), amp=fmax)
    if min_scale > 0:
        axes = sc[:, :3]
        floored = axes.clamp_min(min_scale * h)
        mr[:, 3] *= axes.prod(1) / floored.prod(1)
        sc[:, :3] = floored
    cap = int(budget * mlp_share)
    if mr.shape[0] > cap:
        mass = mr[:, 3] * sc[:, 0] * sc[:, 1] * sc[:, 2]
        keep = torch.topk(mass, cap).indices.sort().values
        mr, sc, q = mr[keep], sc[keep], q[keep]
    n_mlp = int(mr.shape[0])
    if n_mlp < budget:
        vox = vox if vox is not None else Voxelizer(grid, device=dev)
        mr, sc, q = mr.contiguous(), sc.contiguous(), q.contiguous()
        vox.ensure_capacity(mr, sc, q)
        resid = (fdk - vox.forward(mr, sc, q)).clamp_min(0)
        extra = gradient_init(resid, grid, budget - n_mlp, uniforms[: budget - n_mlp])
        mr, sc, q = (torch.cat([a, b]) for a, b in zip((mr, sc, q), extra))
    return mr.contiguous(), sc.contiguous(), q.contiguous(), n_mlp
