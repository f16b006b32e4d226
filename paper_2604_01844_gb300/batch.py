"""Batched reconstruction: up to 32 independent reconstructions of uneven size advanced by one
optimisation step (Eq. 5 loop) at a time, with the rasterizer and the voxelizer each run as a
single batched call per pass, one Adam launch over all parameters, and the whole step captured
in one CUDA graph.

Per step: batched projection -> per-instance L1 + D-SSIM (loss kernels on each instance's
256-byte-aligned image block) -> batched per-Gaussian backward (accumulated) -> Adam, with the
TV branch (batched voxelization of every instance's full grid -> per-instance TV -> batched
voxelizer backward) on a second stream beside the projection, joined before the projection's
backward.  Instance k's loss lands in loss[k].
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import binding as B
from .projector import BatchProjector, views_to_device
from .recon import ReconConfig, inverse_softplus, psnr_of
from .voxelizer import BatchVoxelizer


class BatchReconstruction:
    """Device state of a batch of reconstructions.

    `instances`: list of dicts with keys views (VIEW_DTYPE array or device tensor), W, H,
    target ((V, H, W) device tensor), grid (GRID_DTYPE), mean_rho, scale, quat ((n, 4) arrays,
    activated), and optionally data_range.  All instances share `cfg`'s weights and learning
    rates.
    """

    def __init__(self, instances, cfg: ReconConfig = ReconConfig(), device="cuda"):
        if not 1 <= len(instances) <= B.MAX_INSTANCES:
            raise ValueError(f"1 .. {B.MAX_INSTANCES} instances")
        self.cfg = cfg
        self.device = dev = torch.device(device)
        self.K = len(instances)
        self.counts = [int(np.asarray(x["mean_rho"]).shape[0]) for x in instances]
        self.g_off = np.concatenate([[0], np.cumsum(self.counts)]).astype(int)
        self.n = int(self.g_off[-1])
        mr = np.concatenate([np.asarray(x["mean_rho"], np.float64) for x in instances])
        sc = np.concatenate([np.asarray(x["scale"], np.float64) for x in instances])
        qt = np.concatenate([np.asarray(x["quat"], np.float32) for x in instances])
        raw_mr = np.concatenate([mr[:, :3], inverse_softplus(mr[:, 3])[:, None]], 1)
        raw_sc = np.concatenate([np.log(np.maximum(sc[:, :3], 1e-12)), np.zeros((self.n, 1))], 1)
        self.raw = [torch.from_numpy(a.astype(np.float32)).to(dev) for a in (raw_mr, raw_sc, qt)]
        self.act = [torch.empty_like(t) for t in self.raw]
        self.grads = [torch.zeros_like(t) for t in self.raw]
        self.m = torch.zeros((3 * self.n, 4), dtype=torch.float32, device=dev)
        self.v = torch.zeros_like(self.m)
        self.step_count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.loss = torch.zeros(self.K, dtype=torch.float32, device=dev)

        views = [x["views"] if isinstance(x["views"], torch.Tensor)
                 else views_to_device(x["views"], dev) for x in instances]
        self.projector = BatchProjector([(v, x["W"], x["H"]) for v, x in zip(views, instances)],
                                        cut=cfg.cut, tile=cfg.tile, device=dev,
                                        headroom=cfg.headroom)
        self._geom = [(v, x["W"], x["H"]) for v, x in zip(views, instances)]
        self.grids = [x["grid"] for x in instances]
        self.voxelizer = BatchVoxelizer([(g, (0, 0, 0), None) for g in self.grids], cut=cfg.cut,
                                        device=dev, headroom=cfg.headroom)
        self.replans = 0  # workspaces re-planned after a pair-capacity overflow
        self.img = torch.zeros(self.projector.img_numel, dtype=torch.float32, device=dev)
        self.dimg = torch.zeros_like(self.img)
        self.target = torch.zeros_like(self.img)
        for t, x in zip(self.projector.split(self.target), instances):
            t.copy_(x["target"].reshape(t.shape))
        self.vol = torch.zeros(self.voxelizer.numel, dtype=torch.float32, device=dev)
        self.dvol = torch.zeros_like(self.vol)
        self.imgs = self.projector.split(self.img)
        self.dimgs = self.projector.split(self.dimg)
        self.targets = self.projector.split(self.target)
        self.vols = self.voxelizer.split(self.vol)
        self.dvols = self.voxelizer.split(self.dvol)
        self.data_range = [float(x.get("data_range") or float(t.max()))
                           for x, t in zip(instances, self.targets)]
        biggest = max(t.numel() for t in self.targets)
        self.ssim_ws = torch.empty(B.lib().gs_ssim_workspace_size(biggest), dtype=torch.uint8,
                                   device=dev)
        o = B.GsAdamOpts()
        o.lr_mean, o.lr_rho, o.lr_scale, o.lr_quat = cfg.lr_mean, cfg.lr_rho, cfg.lr_scale, cfg.lr_quat
        o.beta1, o.beta2, o.eps = cfg.beta1, cfg.beta2, cfg.eps
        o.min_log_scale, o.max_log_scale = cfg.min_log_scale, cfg.max_log_scale
        self.adam_opts = o
        self.activate()
        self.plan()

    def params(self, k: int):
        """Activated parameters of instance k (views into the concatenated arrays)."""
        a, b = int(self.g_off[k]), int(self.g_off[k + 1])
        return [t[a:b] for t in self.act]

    def subset(self, keep) -> "BatchReconstruction":
        """A batch of the instances `keep` (indices into this batch) that continues their
        optimisation where it stands: raw parameters, Adam moments and the step count are
        carried over.  The instances of a batch do not interact, so dropping the others
        changes nothing for these; the workspaces are planned for the smaller batch."""
        keep = [int(k) for k in keep]
        insts = []
        for k in keep:
            v, W, H = self._geom[k]
            mr, sc, q = (t.cpu().numpy() for t in self.params(k))
            insts.append(dict(views=v, W=W, H=H, target=self.targets[k], grid=self.grids[k],
                              mean_rho=mr, scale=sc, quat=q, data_range=self.data_range[k]))
        new = BatchReconstruction(insts, cfg=self.cfg, device=self.device)
        for j, k in enumerate(keep):
            a, b = int(self.g_off[k]), int(self.g_off[k + 1])
            c, d = int(new.g_off[j]), int(new.g_off[j + 1])
            for dst, src in zip(new.raw, self.raw):
                dst[c:d].copy_(src[a:b])
            new.m[3 * c:3 * d].copy_(self.m[3 * a:3 * b])
            new.v[3 * c:3 * d].copy_(self.v[3 * a:3 * b])
        new.step_count.copy_(self.step_count)
        new.replans = self.replans
        new.activate()
        new.plan()
        return new

    def activate(self):
        B.check(B.lib().gs_activate(*[B.ptr(t) for t in self.raw], *[B.ptr(t) for t in self.act],
                                    self.n, B.stream_handle()), "gs_activate")

    def plan(self):
        """Size both workspaces for the current parameters (synchronous)."""
        self.projector.ensure_capacity(*self.act, self.counts)
        self.voxelizer.ensure_capacity(*self.act, self.counts)

    def overflowed(self) -> bool:
        """True when the last step ran out of pair capacity (synchronises)."""
        return (B.read_status(self.projector.ws).code != B.GS_OK or
                B.read_status(self.voxelizer.ws).code != B.GS_OK)

    def _tv_branch(self, accumulate: bool):
        """Batched voxelization -> per-instance TV -> batched voxelizer backward."""
        L = B.lib()
        s = B.stream_handle()
        lp = self.loss.data_ptr()
        self.voxelizer.forward(*self.act, self.counts, out=self.vol)
        for k in range(self.K):
            dz, dy, dx = self.vols[k].shape
            B.check(L.gs_tv3d_loss(B.ptr(self.vols[k]), dx, dy, dz, self.cfg.alpha_tv, lp + 4 * k,
                                   B.ptr(self.dvols[k]), 0, s), "gs_tv3d_loss")
        self.voxelizer.backward(*self.act, self.counts, self.dvol, grads=self.grads,
                                accumulate=accumulate, reuse=True)

    def step(self):
        """One iteration of every instance; losses land in self.loss (device), no host sync."""
        L = B.lib()
        s = B.stream_handle()
        cfg = self.cfg
        B.check(L.gs_memset(B.ptr(self.loss), 0, 4 * self.K, s), "gs_memset")
        # the TV branch needs only the parameters: it runs on a second stream beside the
        # projection and writes the gradients first; the projection's backward adds to them
        branch = cfg.alpha_tv > 0 and cfg.overlap_tv
        if branch:
            main = torch.cuda.current_stream(self.device)
            if not hasattr(self, "_side"):
                self._side = torch.cuda.Stream(device=self.device)
            self._side.wait_stream(main)
            with torch.cuda.stream(self._side):
                self._tv_branch(accumulate=False)
        self.projector.forward(*self.act, self.counts, out=self.img)
        lp = self.loss.data_ptr()
        for k in range(self.K):
            img, tgt, dimg = self.imgs[k], self.targets[k], self.dimgs[k]
            nv, H, W = img.shape
            if cfg.alpha_ssim > 0:  # both terms in the two SSIM kernels
                B.check(L.gs_l1_ssim2d_loss(B.ptr(img), B.ptr(tgt), nv, H, W, self.data_range[k],
                                            1.0, cfg.alpha_ssim, lp + 4 * k, B.ptr(dimg), 0,
                                            B.ptr(self.ssim_ws), self.ssim_ws.numel(), s),
                        "gs_l1_ssim2d_loss")
            else:
                B.check(L.gs_l1_loss(B.ptr(img), B.ptr(tgt), img.numel(), 1.0, lp + 4 * k,
                                     B.ptr(dimg), 0, s), "gs_l1_loss")
        if branch:
            main.wait_stream(self._side)
        self.projector.backward(*self.act, self.counts, self.dimg, grads=self.grads,
                                accumulate=branch, reuse=True)
        if cfg.alpha_tv > 0 and not branch:
            self._tv_branch(accumulate=True)
        B.check(L.gs_adam_step(*[B.ptr(t) for t in self.raw], B.ptr(self.m), B.ptr(self.v),
                               *[B.ptr(t) for t in self.grads], *[B.ptr(t) for t in self.act],
                               self.n, B.ptr(self.step_count), ctypes.byref(self.adam_opts), s),
                "gs_adam_step")
        return self.loss

    def volumes(self):
        """Voxelizes every instance's full grid into self.vol (asynchronous)."""
        self.voxelizer.forward(*self.act, self.counts, out=self.vol)
        return self.vols


class BatchGraphStep:
    """BatchReconstruction.step captured once into a CUDA graph (one graph launch per step).
    Valid while the workspaces keep their capacity; re-plan and capture again otherwise."""

    def __init__(self, rec: BatchReconstruction, warmup: int = 2):
        self.rec = rec
        side = torch.cuda.Stream(device=rec.device)
        side.wait_stream(torch.cuda.current_stream(rec.device))
        with torch.cuda.stream(side):
            for _ in range(warmup):
                rec.step()
        torch.cuda.current_stream(rec.device).wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            rec.step()

    def __call__(self):
        self.graph.replay()
        return self.rec.loss


def batch_to_psnr(rec: BatchReconstruction, gts, peaks, max_iters: int, target_psnr,
                  eval_every: int = 5, graph: bool = True, history: list | None = None,
                  retire: bool = False):
    """Steps the batch until every instance's voxelized volume reaches target_psnr (one value
    for all, or one per instance) against its ground truth.  Returns (per instance the
    (iteration, gpu ms) at which it first reached its target, or None; per-instance PSNR at the
    last evaluation that stepped it; iterations run; total gpu ms).  retire: an instance that
    has reached its target leaves the batch at that evaluation (the rest continue as
    rec.subset(...), with the graph captured again), so that finished instances cost no more
    steps; the re-planning and capture are inside the timed span.  history, when given,
    receives (iteration, gpu ms, per-instance PSNRs, instances still stepped, re-plans) at
    every evaluation.  A step that ran out of pair capacity is detected at the evaluation
    points; the workspaces are then re-planned (and the graph captured again)."""
    sse = torch.zeros(1, dtype=torch.float64, device=rec.device)
    stepper = BatchGraphStep(rec, warmup=0) if graph else rec.step
    start = torch.cuda.Event(enable_timing=True)
    start.record()
    targets = list(target_psnr) if hasattr(target_psnr, "__len__") else [target_psnr] * rec.K
    reached = [None] * rec.K
    last = [float("-inf")] * rec.K
    active = list(range(rec.K))  # original index of each instance of the current batch
    it = 0
    ms = 0.0
    while it < max_iters:
        stepper()
        it += 1
        if it % eval_every and it != max_iters:
            continue
        if rec.overflowed():
            rec.plan()
            rec.replans += 1
            if graph:
                stepper = BatchGraphStep(rec, warmup=0)
        vols = rec.volumes()
        ev = torch.cuda.Event(enable_timing=True)
        ev.record()
        for j, k in enumerate(active):
            last[k] = psnr_of(vols[j], gts[k], peaks[k], sse)
        ms = start.elapsed_time(ev)
        if history is not None:
            history.append((it, ms, list(last), len(active), rec.replans))
        for k in active:
            if reached[k] is None and last[k] >= targets[k]:
                reached[k] = (it, ms)
        if all(r is not None for r in reached):
            break
        if retire:
            stay = [j for j, k in enumerate(active) if reached[k] is None]
            if len(stay) < len(active):
                rec = rec.subset(stay)
                active = [active[j] for j in stay]
                stepper = BatchGraphStep(rec, warmup=0) if graph else rec.step
    return reached, last, it, ms
