"""FP16 Gaussian codec (22 bytes per Gaussian) and on-demand voxelization of encoded Gaussians
through gs_encode_fp16 / gs_decode_fp16 / gs_voxelize_fp16 (the paper's volume fitting and
compression study)."""
from __future__ import annotations

import ctypes

import torch

from . import binding as B

RECORD_BYTES = 22
PLANES = ("x", "y", "z", "sx", "sy", "sz", "qw", "qx", "qy", "qz", "rho")


def encode(mean_rho, scale, quat) -> torch.Tensor:
    """(11, n) int16 tensor of binary16 planes (22 n bytes) of activated parameters."""
    n = int(mean_rho.shape[0])
    out = torch.empty((11, n), dtype=torch.int16, device=mean_rho.device)
    B.check(B.lib().gs_encode_fp16(B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), n, B.ptr(out),
                                   B.stream_handle()), "gs_encode_fp16")
    return out


def decode(codec: torch.Tensor):
    """Activated (mean_rho, scale, quat) (n, 4) float32 tensors of an (11, n) codec."""
    n = int(codec.shape[1])
    out = [torch.empty((n, 4), dtype=torch.float32, device=codec.device) for _ in range(3)]
    B.check(B.lib().gs_decode_fp16(B.ptr(codec.contiguous()), n, *[B.ptr(t) for t in out],
                                   B.stream_handle()), "gs_decode_fp16")
    return out


class CodecVoxelizer:
    """Voxelizes encoded Gaussians on demand into a grid's region of interest."""

    def __init__(self, grid, roi_lo=(0, 0, 0), roi_dim=None, cut: float = 3.0, brick: int = 16,
                 device="cuda", headroom: float = 1.25):
        self.device = torch.device(device)
        self.grid = B.grid_struct(grid)
        dims = [self.grid.dims[k] for k in range(3)]
        self.roi_lo = B.i3(roi_lo)
        self.roi_dim = B.i3(roi_dim if roi_dim is not None else dims)
        self.shape = (self.roi_dim[2], self.roi_dim[1], self.roi_dim[0])
        self.opts = B.opts(cut=cut, brick=brick)
        self.headroom = float(headroom)
        self.ws = None
        self.key = None

    def _bytes(self, n, pairs):
        b = B.lib().gs_voxelize_fp16_workspace_size(n, ctypes.byref(self.grid), self.roi_lo,
                                                    self.roi_dim, ctypes.byref(self.opts),
                                                    int(pairs))
        if b == 0:
            raise B.GsError("invalid voxelizer sizes")
        return int(b)

    def plan(self, codec: torch.Tensor) -> int:
        """Sizes the workspace for this codec (synchronous); returns its pair count."""
        n = int(codec.shape[1])
        self.ws = torch.empty(self._bytes(n, 0), dtype=torch.uint8, device=self.device)
        out = ctypes.c_int64(0)
        B.check(B.lib().gs_voxelize_fp16_count_pairs(
            B.ptr(codec), n, ctypes.byref(self.grid), self.roi_lo, self.roi_dim,
            ctypes.byref(self.opts), B.ptr(self.ws), self.ws.numel(), B.stream_handle(),
            ctypes.byref(out)), "gs_voxelize_fp16_count_pairs")
        pairs = int(out.value)
        self.ws = torch.empty(self._bytes(n, int(pairs * self.headroom) + 1024),
                              dtype=torch.uint8, device=self.device)
        self.key = (codec.data_ptr(), codec._version, n)
        return pairs

    def forward(self, codec: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        codec = codec.contiguous()
        n = int(codec.shape[1])
        if self.key != (codec.data_ptr(), codec._version, n):
            self.plan(codec)
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        B.check(B.lib().gs_voxelize_fp16(
            B.ptr(codec), n, ctypes.byref(self.grid), self.roi_lo, self.roi_dim,
            ctypes.byref(self.opts), B.ptr(out), B.ptr(self.ws), self.ws.numel(),
            B.stream_handle()), "gs_voxelize_fp16")
        return out

    def status(self):
        return B.read_status(self.ws)
