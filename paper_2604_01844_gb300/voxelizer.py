"""Voxelizer (Sec. 3.3, Eq. 2) over libgsct with workspace planning and autograd."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import binding as B
from .projector import _f4, block_offsets


class Voxelizer:
    """Voxelizes Gaussians into the region of interest roi_lo .. roi_lo + roi_dim - 1 of a
    grid (numpy GRID_DTYPE record); output volume [z][y][x] of shape roi_dim reversed."""

    def __init__(self, grid, roi_lo=(0, 0, 0), roi_dim=None, cut: float = 3.0, brick: int = 16,
                 device="cuda", headroom: float = 1.5):
        self.device = torch.device(device)
        self.grid = B.grid_struct(grid)
        dims = [self.grid.dims[k] for k in range(3)]
        self.roi_lo = B.i3(roi_lo)
        self.roi_dim = B.i3(roi_dim if roi_dim is not None else dims)
        self.shape = (self.roi_dim[2], self.roi_dim[1], self.roi_dim[0])
        self.opts = B.opts(cut=cut, brick=brick)
        self.headroom = float(headroom)
        self.ws = None
        self.ws_n = -1
        self.capacity = 0
        self._fwd_token = None

    def set_roi(self, roi_lo, roi_dim=None):
        self.roi_lo = B.i3(roi_lo)
        if roi_dim is not None:
            self.roi_dim = B.i3(roi_dim)
            self.shape = (self.roi_dim[2], self.roi_dim[1], self.roi_dim[0])
        self._fwd_token = None

    def workspace_bytes(self, n: int, pairs: int) -> int:
        b = B.lib().gs_voxelize_workspace_size(n, ctypes.byref(self.grid), self.roi_lo,
                                               self.roi_dim, ctypes.byref(self.opts), int(pairs))
        if b == 0:
            raise B.GsError("invalid voxelizer sizes")
        return int(b)

    def _alloc(self, n, pairs):
        self.ws = torch.empty(self.workspace_bytes(n, pairs), dtype=torch.uint8, device=self.device)
        self.ws_n = n
        self.capacity = pairs

    def count_pairs(self, mean_rho, scale, quat) -> int:
        n = mean_rho.shape[0]
        if self.ws is None or self.ws_n != n or self.workspace_bytes(n, 0) > self.ws.numel():
            self._alloc(n, 0)
        out = ctypes.c_int64(0)
        B.check(B.lib().gs_voxelize_count_pairs(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), n, ctypes.byref(self.grid), self.roi_lo,
            self.roi_dim, ctypes.byref(self.opts), B.ptr(self.ws), self.ws.numel(),
            B.stream_handle(), ctypes.byref(out)), "gs_voxelize_count_pairs")
        return int(out.value)

    def ensure_capacity(self, mean_rho, scale, quat) -> int:
        pairs = self.count_pairs(mean_rho, scale, quat)
        n = mean_rho.shape[0]
        if self.ws_n != n or pairs > self.capacity or \
                self.workspace_bytes(n, self.capacity) > self.ws.numel():
            self._alloc(n, int(pairs * self.headroom) + 1024)
        return pairs

    def status(self):
        return B.read_status(self.ws)

    def forward(self, mean_rho, scale, quat, out=None):
        mean_rho, scale, quat = _f4(mean_rho, "mean_rho"), _f4(scale, "scale"), _f4(quat, "quat")
        n = mean_rho.shape[0]
        if self.ws is None or self.ws_n != n or self.capacity == 0 or \
                self.workspace_bytes(n, self.capacity) > self.ws.numel():
            self.ensure_capacity(mean_rho, scale, quat)
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        B.check(B.lib().gs_voxelize(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), n, ctypes.byref(self.grid), self.roi_lo,
            self.roi_dim, ctypes.byref(self.opts), B.ptr(out), B.ptr(self.ws), self.ws.numel(),
            B.stream_handle()), "gs_voxelize")
        self._fwd_token = self._token(mean_rho, scale, quat)
        return out

    def backward(self, mean_rho, scale, quat, dvol, grads=None, accumulate=False, reuse=None):
        mean_rho, scale, quat = _f4(mean_rho, "mean_rho"), _f4(scale, "scale"), _f4(quat, "quat")
        dvol = dvol.contiguous()
        n = mean_rho.shape[0]
        if self.ws is None or self.ws_n != n or self.capacity == 0 or \
                self.workspace_bytes(n, self.capacity) > self.ws.numel():
            self.ensure_capacity(mean_rho, scale, quat)
        if reuse is None:
            reuse = self._fwd_token == self._token(mean_rho, scale, quat)
        if grads is None:
            grads = tuple(torch.empty_like(t) for t in (mean_rho, scale, quat))
            accumulate = False
        g_mr, g_sc, g_q = grads
        B.check(B.lib().gs_voxelize_backward(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), n, ctypes.byref(self.grid), self.roi_lo,
            self.roi_dim, ctypes.byref(self.opts), B.ptr(dvol), B.ptr(g_mr), B.ptr(g_sc),
            B.ptr(g_q), 1 if accumulate else 0, 1 if reuse else 0, B.ptr(self.ws),
            self.ws.numel(), B.stream_handle()), "gs_voxelize_backward")
        return g_mr, g_sc, g_q

    def count_evals(self, mean_rho, scale, quat) -> int:
        n = mean_rho.shape[0]
        self.ensure_capacity(mean_rho, scale, quat)
        B.check(B.lib().gs_voxelize_count_evals(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), n, ctypes.byref(self.grid), self.roi_lo,
            self.roi_dim, ctypes.byref(self.opts), B.ptr(self.ws), self.ws.numel(),
            B.stream_handle()), "gs_voxelize_count_evals")
        self._fwd_token = None
        return int(self.status().evals)

    def read_pairs(self):
        st = self.status()
        n = int(st.pairs)
        keys = np.zeros(max(n, 1), dtype=np.uint32)
        vals = np.zeros(max(n, 1), dtype=np.uint32)
        cnt = ctypes.c_int64(0)
        B.check(B.lib().gs_read_pairs(B.ptr(self.ws), self.ws.numel(), B.stream_handle(), n,
                                      keys.ctypes.data_as(ctypes.c_void_p),
                                      vals.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)),
                "gs_read_pairs")
        return keys[:n], vals[:n]

    @staticmethod
    def _token(*ts):
        return tuple((t.data_ptr(), t._version) for t in ts)


class BatchVoxelizer:
    """Voxelizes up to 32 independent instances (each its own Gaussians, grid and region of
    interest) with one kernel launch per pass.

    `instances` is a list of (grid, roi_lo, roi_dim) (roi_dim None: the whole grid).
    Parameters are the instances' (n_k, 4) arrays concatenated in order with `counts` = [n_k];
    the output is one flat float32 tensor holding each region [z][y][x] in order (`split`).
    """

    def __init__(self, instances, cut: float = 3.0, brick: int = 16, device="cuda",
                 headroom: float = 1.5):
        if not 1 <= len(instances) <= B.MAX_INSTANCES:
            raise ValueError(f"1 .. {B.MAX_INSTANCES} instances")
        self.device = torch.device(device)
        self.grids, self.rois = [], []
        for grid, lo, dim in instances:
            g = B.grid_struct(grid)
            dims = [g.dims[k] for k in range(3)]
            self.grids.append(g)
            self.rois.append((tuple(int(x) for x in lo),
                              tuple(int(x) for x in (dim if dim is not None else dims))))
        self.shapes = [(d[2], d[1], d[0]) for _, d in self.rois]
        self.offsets = block_offsets([a * b * c for a, b, c in self.shapes])
        self.numel = self.offsets[-1]
        self.opts = B.opts(cut=cut, brick=brick)
        self.headroom = float(headroom)
        self.ws = None
        self.ws_counts = None
        self.capacity = 0
        self._fwd_token = None

    def table(self, counts):
        if len(counts) != len(self.grids):
            raise ValueError("one Gaussian count per instance")
        t = (B.GsVoxelInstance * len(counts))()
        for k, n in enumerate(counts):
            t[k].n = int(n)
            t[k].grid = self.grids[k]
            lo, dim = self.rois[k]
            for a in range(3):
                t[k].roi_lo[a], t[k].roi_dim[a] = lo[a], dim[a]
        return t

    def split(self, flat):
        return [flat[o:o + a * b * c].view(a, b, c)
                for o, (a, b, c) in zip(self.offsets, self.shapes)]

    def _alloc(self, counts, pairs):
        t = self.table(counts)
        nbytes = int(B.lib().gs_voxelize_batch_workspace_size(
            t, len(counts), ctypes.byref(self.opts), int(pairs)))
        if nbytes == 0:
            raise B.GsError("invalid batch voxelizer sizes")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ws_counts = list(counts)
        self.capacity = pairs

    def count_pairs(self, mean_rho, scale, quat, counts) -> int:
        if self.ws is None or self.ws_counts != list(counts):
            self._alloc(counts, 0)
        out = ctypes.c_int64(0)
        B.check(B.lib().gs_voxelize_batch_count_pairs(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), self.table(counts), len(counts),
            ctypes.byref(self.opts), B.ptr(self.ws), self.ws.numel(), B.stream_handle(),
            ctypes.byref(out)), "gs_voxelize_batch_count_pairs")
        return int(out.value)

    def ensure_capacity(self, mean_rho, scale, quat, counts) -> int:
        pairs = self.count_pairs(mean_rho, scale, quat, counts)
        if self.ws_counts != list(counts) or pairs > self.capacity:
            self._alloc(counts, int(pairs * self.headroom) + 1024)
        return pairs

    def _ready(self, mean_rho, scale, quat, counts):
        if sum(counts) != mean_rho.shape[0]:
            raise ValueError("counts must add up to the number of Gaussians")
        if self.ws is None or self.ws_counts != list(counts) or self.capacity == 0:
            self.ensure_capacity(mean_rho, scale, quat, counts)

    def forward(self, mean_rho, scale, quat, counts, out=None):
        mean_rho, scale, quat = _f4(mean_rho, "mean_rho"), _f4(scale, "scale"), _f4(quat, "quat")
        self._ready(mean_rho, scale, quat, counts)
        if out is None:
            out = torch.empty(self.numel, dtype=torch.float32, device=self.device)
        B.check(B.lib().gs_voxelize_batch(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), self.table(counts), len(counts),
            ctypes.byref(self.opts), B.ptr(out), B.ptr(self.ws), self.ws.numel(),
            B.stream_handle()), "gs_voxelize_batch")
        self._fwd_token = tuple((t.data_ptr(), t._version) for t in (mean_rho, scale, quat)) + \
            (tuple(counts),)
        return out

    def backward(self, mean_rho, scale, quat, counts, dvol, grads=None, accumulate=False,
                 reuse: bool | None = None):
        mean_rho, scale, quat = _f4(mean_rho, "mean_rho"), _f4(scale, "scale"), _f4(quat, "quat")
        dvol = dvol.contiguous()
        self._ready(mean_rho, scale, quat, counts)
        if reuse is None:
            reuse = self._fwd_token == tuple((t.data_ptr(), t._version)
                                             for t in (mean_rho, scale, quat)) + (tuple(counts),)
        if grads is None:
            grads = tuple(torch.empty_like(x) for x in (mean_rho, scale, quat))
            accumulate = False
        g_mr, g_sc, g_q = grads
        B.check(B.lib().gs_voxelize_batch_backward(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), self.table(counts), len(counts),
            ctypes.byref(self.opts), B.ptr(dvol), B.ptr(g_mr), B.ptr(g_sc), B.ptr(g_q),
            1 if accumulate else 0, 1 if reuse else 0, B.ptr(self.ws), self.ws.numel(),
            B.stream_handle()), "gs_voxelize_batch_backward")
        return g_mr, g_sc, g_q

    def count_evals(self, mean_rho, scale, quat, counts) -> int:
        self.ensure_capacity(mean_rho, scale, quat, counts)
        B.check(B.lib().gs_voxelize_batch_count_evals(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), self.table(counts), len(counts),
            ctypes.byref(self.opts), B.ptr(self.ws), self.ws.numel(), B.stream_handle()),
            "gs_voxelize_batch_count_evals")
        self._fwd_token = None
        return int(B.read_status(self.ws).evals)


class VoxelizeFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mean_rho, scale, quat, vox: Voxelizer):
        vol = vox.forward(mean_rho, scale, quat)
        ctx.save_for_backward(mean_rho, scale, quat)
        ctx.vox = vox
        return vol

    @staticmethod
    def backward(ctx, dvol):
        mean_rho, scale, quat = ctx.saved_tensors
        g = ctx.vox.backward(mean_rho, scale, quat, dvol)
        return g[0], g[1], g[2], None


def voxelize(mean_rho, scale, quat, vox: Voxelizer):
    return VoxelizeFunction.apply(mean_rho, scale, quat, vox)
