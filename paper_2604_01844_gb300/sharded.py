"""View-sharded reconstruction step over several processes, one GPU each.

The projection loss of Eq. 5 is a sum over views, and each view's image depends on all the
Gaussians but on no other view (Sec. 3.2: every view is rasterized on its own).  So the views
split into contiguous chunks, one per process: every process holds the whole Gaussian set and
its Adam state, projects only its views, takes their L1 + D-SSIM terms weighted by its share
of the views, and runs their per-Gaussian backward.  The 3D TV term (it needs the parameters
only) runs on one process.  One all-reduce (sum) of the gradient buffer -- 3 float4 per
Gaussian plus the loss, 48 N + 4 bytes -- then gives every process the full-problem gradient,
and every process applies the identical Adam step, so the parameters stay equal everywhere
without further exchange.

The collective is torch.distributed's all_reduce on the process group (NCCL on GPUs); it is
enqueued on the current stream after the backward, before Adam.  With one process nothing is
exchanged and the step is the single-process step.
"""
from __future__ import annotations

import dataclasses

import torch

from .recon import Reconstruction, ReconConfig


def view_range(n_views: int, rank: int, world: int) -> tuple[int, int]:
    """Views [a, b) of process `rank`: contiguous chunks that cover 0..n_views-1 once, sizes
    differing by at most one (the first n_views % world chunks take the extra view)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    if n_views < world:
        raise ValueError(f"{n_views} views cannot give each of {world} processes a view")
    q, r = divmod(n_views, world)
    a = rank * q + min(rank, r)
    return a, a + q + (1 if rank < r else 0)


def view_share(a: int, b: int, n_views: int) -> float:
    """Weight of views [a, b) in the all-view mean of an image term (every view has the same
    pixel count): the per-process means times these shares add up to the global mean."""
    return (b - a) / n_views


def allreduce_sum_(flat: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum of `flat` over the processes of `group` (identity without a process
    group or with one process)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    return flat


def allreduce_max(x: float, device, group=None) -> float:
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        t = torch.tensor([float(x)], dtype=torch.float32, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        return float(t.item())
    return float(x)


class ViewShardedReconstruction(Reconstruction):
    """Reconstruction of one problem with its views split over the processes of `group`.

    views, target: all n_views views of the problem and their target projections (each
    process reads only its own chunk of the target; passing only that chunk, with
    `target_is_local`, saves the memory).  The SSIM data range is the maximum over all views'
    targets (one all-reduce at construction).  tv_rank: the process that runs the TV term."""

    def __init__(self, views, W, H, target: torch.Tensor, grid, mean_rho, scale, quat,
                 rank: int, world: int, cfg: ReconConfig = ReconConfig(), device="cuda",
                 group=None, target_is_local: bool = False, tv_rank: int = 0,
                 data_range: float | None = None):
        n_views = len(views)
        a, b = view_range(n_views, rank, world)
        self.view_lo, self.view_hi, self.n_views_all = a, b, n_views
        self.group = group
        local = target if target_is_local else target[a:b]
        if local.shape[0] != b - a:
            raise ValueError("the local target must hold this process's views")
        if data_range is None:
            data_range = allreduce_max(float(local.max()), local.device, group)
        lcfg = dataclasses.replace(cfg, alpha_tv=cfg.alpha_tv if rank == tv_rank else 0.0)
        super().__init__(views[a:b], W, H, local, grid, mean_rho, scale, quat, cfg=lcfg,
                         device=device, data_range=data_range)
        self.view_share = view_share(a, b, n_views)
        self._flat_buffers()

    def _flat_buffers(self):
        """Gradients and loss as views into one buffer, so that one collective sums them."""
        n = self.n
        self.flat = torch.zeros(12 * n + 4, dtype=torch.float32, device=self.device)
        g = self.flat[:12 * n].view(3, n, 4)
        self.grads = [g[0], g[1], g[2]]
        self.loss = self.flat[12 * n:12 * n + 1]

    def replace_parameters(self, raw, m, v):
        super().replace_parameters(raw, m, v)
        self._flat_buffers()

    def _before_adam(self):
        allreduce_sum_(self.flat, self.group)
