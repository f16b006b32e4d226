"""One optimisation step of Gaussian-splatting CT reconstruction (Eq. 5, Fig. 2 loop) through
libgsct calls only: project -> L1 + D-SSIM (fused fwd/bwd) -> per-Gaussian backward -> Adam
with activations, and beside the projection (second stream) voxelize -> TV (fused) ->
voxelizer backward, whose gradients the projection's backward adds to.

PyTorch only allocates the device buffers and provides the stream.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import binding as B
from .projector import Projector
from .voxelizer import Voxelizer


@dataclass
class ReconConfig:
    alpha_ssim: float = 0.25   # Eq. 5 weights; the paper gives no values
    alpha_tv: float = 0.05
    lr_mean: float = 2e-4
    lr_rho: float = 1e-2
    lr_scale: float = 5e-3
    lr_quat: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    min_log_scale: float = math.log(1e-4)
    max_log_scale: float = math.log(0.5)
    tile: int = 16
    cut: float = 3.0
    tv_roi: tuple | None = None  # (lo, dim) of the TV region; None = whole grid
    recompute_lists: bool = False  # backward rebuilds the sorted lists instead of reusing them
    overlap_tv: bool = True  # the TV branch runs on a second stream beside the projection
    view_streams: int = 2  # the views split into this many chunks, each on its own stream
    headroom: float = 1.5  # pair capacity planned as this multiple of the current pair counts


def inverse_softplus(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    return np.where(x > 20, x, np.log(np.expm1(np.maximum(x, 1e-12))))


class Reconstruction:
    """Holds the device state of one reconstruction: raw and activated parameters, Adam
    moments, the target projections, the workspaces and the loss accumulator."""

    def __init__(self, views, W, H, target: torch.Tensor, grid, mean_rho, scale, quat,
                 cfg: ReconConfig = ReconConfig(), device="cuda", data_range: float | None = None):
        self.cfg = cfg
        self.device = torch.device(device)
        self.n = int(mean_rho.shape[0])
        dev = self.device
        mr = np.asarray(mean_rho, dtype=np.float64)
        sc = np.asarray(scale, dtype=np.float64)
        raw_mr = np.concatenate([mr[:, :3], inverse_softplus(mr[:, 3])[:, None]], 1)
        raw_sc = np.concatenate([np.log(np.maximum(sc[:, :3], 1e-12)), np.zeros((self.n, 1))], 1)
        self.raw = [torch.from_numpy(a.astype(np.float32)).to(dev)
                    for a in (raw_mr, raw_sc, np.asarray(quat, dtype=np.float32))]
        self.act = [torch.empty_like(t) for t in self.raw]
        self.grads = [torch.zeros_like(t) for t in self.raw]
        self.m = torch.zeros((3 * self.n, 4), dtype=torch.float32, device=dev)
        self.v = torch.zeros_like(self.m)
        self.step_count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.target = target.contiguous()
        self.W, self.H = int(W), int(H)
        self.projector = Projector(views, W, H, cut=cfg.cut, tile=cfg.tile, device=dev,
                                   headroom=cfg.headroom)
        self.replans = 0  # workspaces re-planned after a pair-capacity overflow
        # view chunks of the pipelined step: (v0, v1, projector of those views)
        nv = int(self.target.shape[0])
        k = max(1, min(int(cfg.view_streams), nv))
        bounds = [round(i * nv / k) for i in range(k + 1)]
        self.vchunks = [] if k == 1 else [
            (a, b, Projector(self.projector.views[a:b], W, H, cut=cfg.cut, tile=cfg.tile,
                             device=dev, headroom=cfg.headroom))
            for a, b in zip(bounds[:-1], bounds[1:])]
        if cfg.tv_roi is None:
            self.voxelizer = Voxelizer(grid, cut=cfg.cut, device=dev, headroom=cfg.headroom)
        else:
            self.voxelizer = Voxelizer(grid, cfg.tv_roi[0], cfg.tv_roi[1], cut=cfg.cut, device=dev,
                                       headroom=cfg.headroom)
        self.img = torch.empty_like(self.target)
        self.dimg = torch.empty_like(self.target)
        self.vol = torch.empty(self.voxelizer.shape, dtype=torch.float32, device=dev)
        self.dvol = torch.empty_like(self.vol)
        self.ssim_ws = torch.empty(B.lib().gs_ssim_workspace_size(self.target.numel()),
                                   dtype=torch.uint8, device=dev)
        per_view = self.target[0].numel()
        self.chunk_ws = [torch.empty(B.lib().gs_ssim_workspace_size((b - a) * per_view),
                                     dtype=torch.uint8, device=dev) for a, b, _ in self.vchunks]
        self.chunk_grads = [[torch.zeros_like(t) for t in self.raw] for _ in self.vchunks[1:]]
        self._streams = [torch.cuda.Stream(device=dev) for _ in self.vchunks[1:]]
        self.data_range = float(data_range if data_range is not None else float(self.target.max()))
        o = B.GsAdamOpts()
        o.lr_mean, o.lr_rho, o.lr_scale, o.lr_quat = cfg.lr_mean, cfg.lr_rho, cfg.lr_scale, cfg.lr_quat
        o.beta1, o.beta2, o.eps = cfg.beta1, cfg.beta2, cfg.eps
        o.min_log_scale, o.max_log_scale = cfg.min_log_scale, cfg.max_log_scale
        self.adam_opts = o
        self.density_stats = None  # (grad_stat, vis) accumulated by the backward when set
        # weight of these views' image terms in the loss: the fraction of all the problem's
        # views they are (1 unless the views are sharded over several processes)
        self.view_share = 1.0
        self.activate()
        self.plan()

    def replace_parameters(self, raw, m, v):
        """Swaps in a new Gaussian set (raw parameters, Adam moments; e.g. after adaptive
        density control), re-activates it and re-plans the workspaces (synchronous).  The Adam
        step count is kept."""
        self.n = int(raw[0].shape[0])
        self.raw = [t.contiguous() for t in raw]
        self.act = [torch.empty_like(t) for t in self.raw]
        self.grads = [torch.zeros_like(t) for t in self.raw]
        self.m, self.v = m.contiguous(), v.contiguous()
        self.chunk_grads = [[torch.zeros_like(t) for t in self.raw] for _ in self.vchunks[1:]]
        self.activate()
        self.plan()

    def activate(self):
        L = B.lib()
        B.check(L.gs_activate(*[B.ptr(t) for t in self.raw], *[B.ptr(t) for t in self.act],
                              self.n, B.stream_handle()), "gs_activate")

    def plan(self):
        """Size the workspaces for the current parameters (synchronous)."""
        for _, _, pj in self.vchunks:
            pj.ensure_capacity(*self.act)
        if not self.vchunks:
            self.projector.ensure_capacity(*self.act)
        self.voxelizer.ensure_capacity(*self.act)

    def overflowed(self) -> bool:
        """True when the last step ran out of pair capacity somewhere (synchronises)."""
        pjs = [pj for _, _, pj in self.vchunks] or [self.projector]
        return any(pj.status().code != B.GS_OK for pj in pjs) or \
            self.voxelizer.status().code != B.GS_OK

    def _image_losses(self, a: int, b: int, ws: torch.Tensor):
        """L1 + D-SSIM of views a..b-1 (their share of the all-view means) into self.loss and
        self.dimg."""
        L = B.lib()
        s = B.stream_handle()
        img, tgt, dimg = self.img[a:b], self.target[a:b], self.dimg[a:b]
        share = self.view_share * (img.numel() / self.img.numel())
        if self.cfg.alpha_ssim > 0:  # both terms in the two SSIM kernels
            B.check(L.gs_l1_ssim2d_loss(B.ptr(img), B.ptr(tgt), b - a, self.H, self.W,
                                        self.data_range, share, self.cfg.alpha_ssim * share,
                                        B.ptr(self.loss), B.ptr(dimg), 0, B.ptr(ws), ws.numel(),
                                        s), "gs_l1_ssim2d_loss")
        else:
            B.check(L.gs_l1_loss(B.ptr(img), B.ptr(tgt), img.numel(), share, B.ptr(self.loss),
                                 B.ptr(dimg), 0, s), "gs_l1_loss")

    def _tv_branch(self, accumulate: bool):
        """Voxelize -> TV (fused value and gradient) -> voxelizer backward into self.grads."""
        L = B.lib()
        s = B.stream_handle()
        self.voxelizer.forward(*self.act, out=self.vol)
        dz, dy, dx = self.vol.shape
        B.check(L.gs_tv3d_loss(B.ptr(self.vol), dx, dy, dz, self.cfg.alpha_tv, B.ptr(self.loss),
                               B.ptr(self.dvol), 0, s), "gs_tv3d_loss")
        self.voxelizer.backward(*self.act, self.dvol, grads=self.grads, accumulate=accumulate,
                                reuse=True)

    def step(self, serial: bool = False, target_ready=None):
        """One full iteration; the loss lands in self.loss (device), no host synchronisation.

        With cfg.overlap_tv the TV branch (it needs only the parameters) runs on a second
        stream while the projection, its losses and its backward run on the current one; the
        branch writes the gradients first and the projection's backward adds to them.  With
        cfg.view_streams > 1 the views also run in chunks on their own streams.  serial = True
        runs everything on the current stream with the views unchunked (the same arithmetic
        per pixel and voxel; used to time each kernel on its own).  target_ready: a CUDA event
        after which self.target holds this step's projections (e.g. a host->device copy on
        another stream); only the image losses wait for it."""
        L = B.lib()
        s = B.stream_handle()
        cfg = self.cfg
        B.check(L.gs_memset(B.ptr(self.loss), 0, 4, s), "gs_memset")
        if self.vchunks and not serial:
            return self._step_pipelined(target_ready)
        branch = cfg.alpha_tv > 0 and cfg.overlap_tv and not serial
        if branch:
            main = torch.cuda.current_stream(self.device)
            if not hasattr(self, "_side"):
                self._side = torch.cuda.Stream(device=self.device)
            self._side.wait_stream(main)
            with torch.cuda.stream(self._side):
                self._tv_branch(accumulate=False)
        self.projector.forward(*self.act, out=self.img)
        if target_ready is not None:
            torch.cuda.current_stream(self.device).wait_event(target_ready)
        self._image_losses(0, self.img.shape[0], self.ssim_ws)
        if branch:
            main.wait_stream(self._side)
        self.projector.backward(*self.act, self.dimg, grads=self.grads, accumulate=branch,
                                reuse=not cfg.recompute_lists, stats=self.density_stats)
        if cfg.alpha_tv > 0 and not branch:
            self._tv_branch(accumulate=True)
        self._before_adam()
        B.check(L.gs_adam_step(*[B.ptr(t) for t in self.raw], B.ptr(self.m), B.ptr(self.v),
                               *[B.ptr(t) for t in self.grads], *[B.ptr(t) for t in self.act],
                               self.n, B.ptr(self.step_count), ctypes.byref(self.adam_opts), s),
                "gs_adam_step")
        return self.loss

    def _before_adam(self):
        """Runs on the current stream once the step's gradients and loss are complete, just
        before the Adam update (the view-sharded step sums them over processes here)."""

    def _step_pipelined(self, target_ready=None):
        """The step with the views in chunks, chunk 0 on the current stream and chunk k on
        stream k: each chunk projects, takes its losses and runs its backward independently, so
        that one chunk's binning and sorting overlap another's rasterization.  The TV branch
        (its own stream) writes self.grads first, chunk 0 adds to them, the other chunks write
        their own gradient buffers, which are added before Adam."""
        L = B.lib()
        cfg = self.cfg
        main = torch.cuda.current_stream(self.device)
        tv = cfg.alpha_tv > 0
        if tv:
            if not hasattr(self, "_side"):
                self._side = torch.cuda.Stream(device=self.device)
            self._side.wait_stream(main)
            with torch.cuda.stream(self._side):
                self._tv_branch(accumulate=False)
        for st in self._streams:
            st.wait_stream(main)
        for k, (a, b, pj) in enumerate(self.vchunks):
            st = main if k == 0 else self._streams[k - 1]
            with torch.cuda.stream(st):
                pj.forward(*self.act, out=self.img[a:b])
                if target_ready is not None:
                    st.wait_event(target_ready)
                self._image_losses(a, b, self.chunk_ws[k])
                if k == 0:
                    if tv:
                        main.wait_stream(self._side)
                    pj.backward(*self.act, self.dimg[a:b], grads=self.grads, accumulate=tv,
                                reuse=not cfg.recompute_lists, stats=self.density_stats)
                else:
                    pj.backward(*self.act, self.dimg[a:b], grads=self.chunk_grads[k - 1],
                                accumulate=False, reuse=not cfg.recompute_lists,
                                stats=self.density_stats)
        s = B.stream_handle()
        for st, g in zip(self._streams, self.chunk_grads):
            main.wait_stream(st)
            for dst, src in zip(self.grads, g):
                B.check(L.gs_add(B.ptr(dst), B.ptr(src), dst.numel(), s), "gs_add")
        self._before_adam()
        B.check(L.gs_adam_step(*[B.ptr(t) for t in self.raw], B.ptr(self.m), B.ptr(self.v),
                               *[B.ptr(t) for t in self.grads], *[B.ptr(t) for t in self.act],
                               self.n, B.ptr(self.step_count), ctypes.byref(self.adam_opts), s),
                "gs_adam_step")
        return self.loss


# ------------------------------------------------------------------------------------------
# End-to-end reconstruction of a synthetic phantom: projections -> FDK -> gradient-based
# initialisation (Sec. 3.1) -> optimisation (Eq. 5) until a target PSNR of the voxelized
# Gaussians against the ground-truth volume.
# ------------------------------------------------------------------------------------------
class PhantomProblem:
    """Ground truth of a random-ellipsoid phantom: cone-beam projections (exact line
    integrals) and the volume sampled at voxel centres, made on the device."""

    def __init__(self, ell: np.ndarray, views, W: int, H: int, grid, device="cuda"):
        from .projector import views_to_device

        self.device = torch.device(device)
        self.views = views
        self.W, self.H = int(W), int(H)
        self.grid = grid
        self.d_views = views_to_device(views, self.device)
        self.d_ell = torch.from_numpy(np.ascontiguousarray(ell, dtype=np.float32)).to(self.device)
        L = B.lib()
        s = B.stream_handle()
        nv = int(self.d_views.shape[0])
        self.proj = torch.empty((nv, H, W), dtype=torch.float32, device=self.device)
        B.check(L.gs_phantom_project(B.ptr(self.d_ell), ell.shape[0], B.ptr(self.d_views), nv,
                                     W, H, B.ptr(self.proj), s), "gs_phantom_project")
        dims = [int(x) for x in np.asarray(grid["dims"]).ravel()]
        self.gt = torch.empty((dims[2], dims[1], dims[0]), dtype=torch.float32, device=self.device)
        B.check(L.gs_phantom_voxelize(B.ptr(self.d_ell), ell.shape[0],
                                      ctypes.byref(B.grid_struct(grid)), B.ptr(self.gt), s),
                "gs_phantom_voxelize")
        self.peak = float(self.gt.max())


def fdk_volume(problem: PhantomProblem, grid) -> torch.Tensor:
    L = B.lib()
    nv = int(problem.d_views.shape[0])
    ws = torch.empty(L.gs_fdk_workspace_size(nv, problem.W, problem.H), dtype=torch.uint8,
                     device=problem.device)
    dims = [int(x) for x in np.asarray(grid["dims"]).ravel()]
    vol = torch.empty((dims[2], dims[1], dims[0]), dtype=torch.float32, device=problem.device)
    B.check(L.gs_fdk(B.ptr(problem.proj), B.ptr(problem.d_views), nv, problem.W, problem.H,
                     ctypes.byref(B.grid_struct(grid)), B.ptr(vol), B.ptr(ws), ws.numel(),
                     B.stream_handle()), "gs_fdk")
    return vol


def gradient_init(vol: torch.Tensor, grid, n: int, uniforms: np.ndarray, threshold_frac=0.05,
                  density_k=0.15, min_scale=None):
    """n Gaussians sampled from `vol` (Sec. 3.1); returns three (n, 4) device tensors."""
    L = B.lib()
    g = B.grid_struct(grid)
    if min_scale is None:
        min_scale = 0.5 * float(np.asarray(grid["voxel"]).min())
    out = [torch.empty((n, 4), dtype=torch.float32, device=vol.device) for _ in range(3)]
    du = torch.from_numpy(np.ascontiguousarray(uniforms, dtype=np.float32)).to(vol.device)
    ws = torch.empty(L.gs_grad_init_workspace_size(ctypes.byref(g), n), dtype=torch.uint8,
                     device=vol.device)
    B.check(L.gs_grad_init(B.ptr(vol), ctypes.byref(g), n, threshold_frac, density_k, min_scale,
                           B.ptr(du), *[B.ptr(t) for t in out], None, B.ptr(ws), ws.numel(),
                           B.stream_handle()), "gs_grad_init")
    return out


def psnr_of(vol: torch.Tensor, gt: torch.Tensor, peak: float, sse: torch.Tensor) -> float:
    """PSNR of vol against gt (peak = max of gt) from the library's FP64 SSE (synchronises)."""
    L = B.lib()
    B.check(L.gs_memset(B.ptr(sse), 0, 8, B.stream_handle()), "gs_memset")
    B.check(L.gs_sse(B.ptr(vol), B.ptr(gt), vol.numel(), B.ptr(sse), B.stream_handle()), "gs_sse")
    mse = float(sse.item()) / vol.numel()
    return 10.0 * math.log10(peak * peak / mse) if mse > 0 else float("inf")


def reconstruct_to_psnr(rec: "Reconstruction", gt: torch.Tensor, peak: float, max_iters: int,
                        target_psnr: float, eval_every: int = 25):
    """Runs rec.step() until the PSNR of its voxelized volume (the TV volume, which covers the
    ground-truth grid) reaches target_psnr.  Returns (history [(iter, gpu ms, psnr)], reached).
    At every evaluation the workspaces' status is read: when the growing Gaussians have run a
    step out of pair capacity, the workspaces are re-planned (rec.replans counts it; the steps
    since the last evaluation did incomplete work, so plan with enough cfg.headroom that this
    does not happen)."""
    sse = torch.zeros(1, dtype=torch.float64, device=gt.device)
    start = torch.cuda.Event(enable_timing=True)
    start.record()
    hist = []
    for it in range(1, max_iters + 1):
        rec.step()
        if it % eval_every == 0 or it == max_iters:
            ev = torch.cuda.Event(enable_timing=True)
            ev.record()
            if rec.overflowed():
                rec.plan()
                rec.replans += 1
            p = psnr_of(rec.vol, gt, peak, sse)
            hist.append((it, start.elapsed_time(ev), p))
            if p >= target_psnr:
                return hist, True
    return hist, False


class GraphStep:
    """The optimisation step captured once into a CUDA graph and replayed (one graph launch per
    step).  Valid while the workspaces keep their capacity; call Reconstruction.plan() and
    capture again after re-planning."""

    def __init__(self, rec: "Reconstruction", warmup: int = 2):
        self.rec = rec
        side = torch.cuda.Stream(device=rec.device)
        side.wait_stream(torch.cuda.current_stream(rec.device))
        with torch.cuda.stream(side):
            for _ in range(warmup):  # settle allocations outside the capture
                rec.step()
        torch.cuda.current_stream(rec.device).wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            rec.step()

    def __call__(self):
        self.graph.replay()
        return self.rec.loss
