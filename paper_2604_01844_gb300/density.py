"""Adaptive density control of a reconstruction: prune, clone and split (the optimisation loop
of Sec. 3.4) through gs_project_backward_stats and gs_densify.

The paper names the three operations only.  The rules are those of the 3D Gaussian splatting
lineage it builds on (Kerbl et al. 2023, via R2-Gaussian), restated for additive rendering:
the statistic is each Gaussian's detector-position gradient in normalised device
coordinates, averaged over the views and steps of a window; Gaussians whose mean reaches
grad_threshold are split (largest scale above split_scale) or cloned, faint or oversized ones
are pruned; clones and splits keep the integrated density (the quantity a projection sums).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import binding as B


@dataclass
class DensifyConfig:
    grad_threshold: float = 2e-4   # position-gradient threshold of Kerbl et al. (NDC units)
    split_scale: float = 0.02      # world units: 1 % of the [-1, 1]^3 volume's extent
    split_factor: float = 1.6      # children's scales = parent's / 1.6 (Kerbl et al.)
    min_density: float = 1e-3      # prune fainter Gaussians
    max_scale: float = 0.25        # prune Gaussians larger than 1/8 of the extent
    max_gaussians: int = 500000    # budget after densification
    start: int = 100               # first iteration that densifies
    stop: int = 10 ** 9            # no densification at or after this iteration
    interval: int = 100            # iterations per statistics window
    seed: int = 0                  # seed of the split children's normal draws
    inherit_moments: bool = False  # children start from the parent's Adam moments


def opts_struct(cfg: DensifyConfig, views_per_step: int, min_log_scale: float) -> B.GsDensifyOpts:
    o = B.GsDensifyOpts()
    o.grad_threshold, o.grad_scale = cfg.grad_threshold, float(views_per_step)
    o.split_scale, o.split_factor = cfg.split_scale, cfg.split_factor
    o.min_density, o.max_scale = cfg.min_density, cfg.max_scale
    o.min_log_scale, o.max_gaussians = min_log_scale, int(cfg.max_gaussians)
    o.inherit_moments = 1 if cfg.inherit_moments else 0
    return o


def densify(raw, m, v, stat, vis, normals, opts: B.GsDensifyOpts, ws=None):
    """One gs_densify call on device tensors: raw = [mean_rho, scale, quat] (n, 4) raw
    parameters, m / v (3n, 4) Adam moments, stat / vis (n,), normals (n, 6).  Returns the new
    ([raw x3], m, v) trimmed to the output count and the status block (synchronises)."""
    n = int(raw[0].shape[0])
    dev = raw[0].device
    cap = min(2 * n, max(n, int(opts.max_gaussians)))
    out = [torch.empty((max(cap, 1), 4), dtype=torch.float32, device=dev) for _ in range(3)]
    om = torch.empty((3 * max(cap, 1), 4), dtype=torch.float32, device=dev)
    ov = torch.empty_like(om)
    nbytes = B.lib().gs_densify_workspace_size(n)
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    B.check(B.lib().gs_densify(
        *[B.ptr(t) for t in raw], B.ptr(m), B.ptr(v), B.ptr(stat), B.ptr(vis), B.ptr(normals), n,
        ctypes.byref(opts), *[B.ptr(t) for t in out], B.ptr(om), B.ptr(ov), cap, B.ptr(ws),
        ws.numel(), B.stream_handle()), "gs_densify")
    st = B.read_status(ws)
    if st.code != B.GS_OK:
        raise B.GsError(f"gs_densify: output count {st.pairs} exceeds capacity {cap}")
    k = int(st.pairs)
    return [t[:k] for t in out], om[:3 * k], ov[:3 * k], st


class DensityControl:
    """Attaches the statistics to a recon.Reconstruction and densifies it on schedule."""

    def __init__(self, rec, cfg: DensifyConfig = DensifyConfig()):
        self.rec = rec
        self.cfg = cfg
        self.rng = np.random.default_rng(cfg.seed)
        self.views = int(rec.projector.n_views)
        self.opts = opts_struct(cfg, self.views, rec.cfg.min_log_scale)
        self.history = []
        self._reset()

    def _reset(self):
        n = self.rec.n
        dev = self.rec.device
        self.stat = torch.zeros(n, dtype=torch.float32, device=dev)
        self.vis = torch.zeros(n, dtype=torch.int32, device=dev)
        self.rec.density_stats = (self.stat, self.vis)

    def due(self, it: int) -> bool:
        c = self.cfg
        return c.start <= it < c.stop and (it - c.start) % c.interval == 0

    def apply(self, it: int | None = None):
        """Densifies the reconstruction now (synchronous); returns the counts."""
        rec = self.rec
        normals = torch.from_numpy(
            self.rng.standard_normal((rec.n, 6)).astype(np.float32)).to(rec.device)
        raw, m, v, st = densify(rec.raw, rec.m, rec.v, self.stat, self.vis, normals, self.opts)
        rec.replace_parameters([t.clone() for t in raw], m.clone(), v.clone())
        self._reset()
        rec_ = dict(iteration=it, n_before=int(normals.shape[0]), n_after=int(st.pairs),
                    pruned=int(st.reserved[0]), cloned=int(st.reserved[1]),
                    split=int(st.reserved[2]), candidates=int(st.reserved[3]))
        self.history.append(rec_)
        return rec_

    def after_step(self, it: int) -> bool:
        """Call after optimisation step `it` (1-based); True when the Gaussian set changed."""
        if self.due(it):
            self.apply(it)
            return True
        return False

