"""X-ray rasterizer (Sec. 3.2, 3.5; Eq. 4) over libgsct, with workspace planning and a
torch.autograd.Function whose backward is the library's per-Gaussian backward kernels."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import binding as B


def _f4(t: torch.Tensor, name: str) -> torch.Tensor:
    if not (t.is_cuda and t.dtype == torch.float32 and t.dim() == 2 and t.shape[1] == 4):
        raise ValueError(f"{name} must be a CUDA float32 (N, 4) tensor")
    return t.contiguous()


def views_to_device(views, device) -> torch.Tensor:
    """gs_view records (numpy VIEW_DTYPE array) -> (V, 64) uint8 tensor on `device`."""
    v = np.ascontiguousarray(np.asarray(views).astype(B.VIEW_DTYPE, copy=False))
    raw = torch.from_numpy(v.view(np.uint8).reshape(len(v), 64).copy())
    return raw.to(device)


# One library call sorts at most 2^31 - 1 (view, tile) pairs (32-bit positions); the projector
# splits its views into chunks whose planned capacity stays below this.
MAX_PAIRS_PER_CALL = (1 << 31) - (1 << 24)


class Projector:
    """Projects Gaussians to a fixed set of views of a W x H detector.

    The workspace (device scratch owned by this object) is sized by counting the (view, tile)
    pairs of the parameters first seen, times `headroom`; `ensure_capacity` re-plans it.  When
    the views would need more pairs than one call can sort, they are split into chunks of
    consecutive views, each with its own workspace; the forward writes each chunk's images,
    the backward accumulates the chunks' gradients.
    """

    def __init__(self, views, W: int, H: int, cut: float = 3.0, eps: float = 0.0,
                 znear: float = 0.1, tile: int = 16, device="cuda", headroom: float = 1.5):
        self.device = torch.device(device)
        self.views = views if isinstance(views, torch.Tensor) else views_to_device(views, self.device)
        self.n_views = int(self.views.shape[0])
        self.W, self.H = int(W), int(H)
        self.opts = B.opts(cut=cut, eps=eps, znear=znear, tile=tile)
        self.headroom = float(headroom)
        self._kw = dict(cut=cut, eps=eps, znear=znear, tile=tile, device=device,
                        headroom=headroom)
        self.ws = None
        self.ws_n = -1
        self.capacity = 0
        self._fwd_token = None
        self.chunks = None  # [(v0, v1, Projector)] when the views are split

    def _split(self, mean_rho, scale, quat, pairs: int):
        """Splits the views into chunks of consecutive views whose capacity fits one call."""
        n_chunks = 2
        while True:
            bounds = np.linspace(0, self.n_views, n_chunks + 1).round().astype(int)
            chunks, ok = [], True
            for v0, v1 in zip(bounds[:-1], bounds[1:]):
                if v1 <= v0:
                    continue
                sub = Projector(self.views[v0:v1], self.W, self.H, **self._kw)
                p = sub.count_pairs(mean_rho, scale, quat)
                if p * self.headroom + 1024 > MAX_PAIRS_PER_CALL:
                    ok = False
                    break
                sub._alloc(mean_rho.shape[0], int(p * self.headroom) + 1024)
                chunks.append((int(v0), int(v1), sub))
            if ok:
                self.chunks = chunks
                self.ws = None
                return pairs
            if n_chunks >= self.n_views:
                raise B.GsError("a single view needs more pairs than one call can sort")
            n_chunks = min(self.n_views, n_chunks * 2)

    # -- workspace -----------------------------------------------------------------------
    def workspace_bytes(self, n: int, pairs: int) -> int:
        b = B.lib().gs_project_workspace_size(n, self.n_views, self.W, self.H,
                                              ctypes.byref(self.opts), int(pairs))
        if b == 0:
            raise B.GsError("invalid projector sizes")
        return int(b)

    def _alloc(self, n: int, pairs: int):
        nbytes = self.workspace_bytes(n, pairs)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ws_n = n
        self.capacity = pairs

    def count_pairs(self, mean_rho, scale, quat) -> int:
        """Exact number of (view, tile) pairs (synchronises the stream)."""
        n = mean_rho.shape[0]
        if self.ws is None or self.ws_n != n:
            self._alloc(n, 0)
        out = ctypes.c_int64(0)
        B.check(B.lib().gs_project_count_pairs(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), n, B.ptr(self.views), self.n_views,
            self.W, self.H, ctypes.byref(self.opts), B.ptr(self.ws), self.ws.numel(),
            B.stream_handle(), ctypes.byref(out)), "gs_project_count_pairs")
        return int(out.value)

    def ensure_capacity(self, mean_rho, scale, quat) -> int:
        """Re-plans the workspace if the current parameters need more pairs; returns the count."""
        if self.chunks is not None:
            return sum(sub.ensure_capacity(mean_rho, scale, quat) for _, _, sub in self.chunks)
        pairs = self.count_pairs(mean_rho, scale, quat)
        n = mean_rho.shape[0]
        if pairs * self.headroom + 1024 > MAX_PAIRS_PER_CALL:
            return self._split(mean_rho, scale, quat, pairs)
        if self.ws_n != n or pairs > self.capacity:
            self._alloc(n, int(pairs * self.headroom) + 1024)
        return pairs

    def status(self) -> B.GsStatus:
        """Status block of the last call (the first chunk reporting an error, if split)."""
        if self.chunks is not None:
            for _, _, sub in self.chunks:
                st = sub.status()
                if st.code != B.GS_OK:
                    return st
            return st
        return B.read_status(self.ws)

    # -- passes --------------------------------------------------------------------------
    def forward(self, mean_rho, scale, quat, out: torch.Tensor | None = None) -> torch.Tensor:
        mean_rho, scale, quat = _f4(mean_rho, "mean_rho"), _f4(scale, "scale"), _f4(quat, "quat")
        n = mean_rho.shape[0]
        if self.chunks is None and (self.ws is None or self.ws_n != n or self.capacity == 0):
            self.ensure_capacity(mean_rho, scale, quat)
        if out is None:
            out = torch.empty((self.n_views, self.H, self.W), dtype=torch.float32, device=self.device)
        if self.chunks is not None:
            for v0, v1, sub in self.chunks:
                sub.forward(mean_rho, scale, quat, out=out[v0:v1])
            self._fwd_token = self._token(mean_rho, scale, quat)
            return out
        B.check(B.lib().gs_project(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), n, B.ptr(self.views), self.n_views,
            self.W, self.H, ctypes.byref(self.opts), B.ptr(out), B.ptr(self.ws), self.ws.numel(),
            B.stream_handle()), "gs_project")
        self._fwd_token = self._token(mean_rho, scale, quat)
        return out

    def backward(self, mean_rho, scale, quat, dimg, grads=None, accumulate: bool = False,
                 reuse: bool | None = None, stats=None):
        """dL/d(mean_rho, scale, quat) from dL/dimg.  stats = (grad_stat float32 (n,),
        vis int32 (n,)) additionally accumulates the adaptive density control statistics
        (gs_project_backward_stats)."""
        mean_rho, scale, quat = _f4(mean_rho, "mean_rho"), _f4(scale, "scale"), _f4(quat, "quat")
        dimg = dimg.contiguous()
        n = mean_rho.shape[0]
        if self.chunks is None and (self.ws is None or self.ws_n != n or self.capacity == 0):
            self.ensure_capacity(mean_rho, scale, quat)
        if reuse is None:
            reuse = self._fwd_token == self._token(mean_rho, scale, quat)
        if grads is None:
            grads = tuple(torch.empty_like(t) for t in (mean_rho, scale, quat))
            accumulate = False
        if self.chunks is not None:
            for k, (v0, v1, sub) in enumerate(self.chunks):
                sub.backward(mean_rho, scale, quat, dimg[v0:v1], grads=grads,
                             accumulate=accumulate or k > 0, reuse=reuse, stats=stats)
            return grads
        g_mr, g_sc, g_q = grads
        if stats is None:
            B.check(B.lib().gs_project_backward(
                B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), n, B.ptr(self.views), self.n_views,
                self.W, self.H, ctypes.byref(self.opts), B.ptr(dimg), B.ptr(g_mr), B.ptr(g_sc),
                B.ptr(g_q), 1 if accumulate else 0, 1 if reuse else 0, B.ptr(self.ws),
                self.ws.numel(), B.stream_handle()), "gs_project_backward")
            return g_mr, g_sc, g_q
        stat, vis = stats
        if stat.dtype != torch.float32 or vis.dtype != torch.int32 or stat.numel() != n or \
                vis.numel() != n:
            raise ValueError("stats: float32 and int32 arrays of n entries")
        B.check(B.lib().gs_project_backward_stats(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), n, B.ptr(self.views), self.n_views,
            self.W, self.H, ctypes.byref(self.opts), B.ptr(dimg), B.ptr(g_mr), B.ptr(g_sc),
            B.ptr(g_q), B.ptr(stat), B.ptr(vis), 1 if accumulate else 0, 1 if reuse else 0,
            B.ptr(self.ws), self.ws.numel(), B.stream_handle()), "gs_project_backward_stats")
        return g_mr, g_sc, g_q

    def count_evals(self, mean_rho, scale, quat) -> int:
        """In-cut (pixel, Gaussian) evaluations of one forward (synchronises)."""
        n = mean_rho.shape[0]
        self.ensure_capacity(mean_rho, scale, quat)
        if self.chunks is not None:
            total = sum(sub.count_evals(mean_rho, scale, quat) for _, _, sub in self.chunks)
            self._fwd_token = None
            return total
        B.check(B.lib().gs_project_count_evals(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), n, B.ptr(self.views), self.n_views,
            self.W, self.H, ctypes.byref(self.opts), B.ptr(self.ws), self.ws.numel(),
            B.stream_handle()), "gs_project_count_evals")
        self._fwd_token = None
        return int(self.status().evals)

    def read_pairs(self):
        """Sorted (key, record) lists of the last binning (synchronises): key = (view << b) |
        tile with b = ceil(log2(tiles)), record = view * n + Gaussian, ordered by (tile, view,
        record), so every key's pairs are contiguous."""
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


def block_offsets(sizes):
    """Start of each instance's block in a batched image or volume (blocks start at multiples
    of 64 floats); the last entry is the total length."""
    out, off = [], 0
    for n in sizes:
        out.append(off)
        off += (int(n) + 63) // 64 * 64
    return out + [off]


class BatchProjector:
    """Projects up to 32 independent instances (each its own Gaussians, views and W x H
    detector) with one kernel launch per pass.

    `instances` is a list of (views, W, H).  Parameters are the instances' (n_k, 4) arrays
    concatenated in order, with `counts` = [n_k]; the image is one flat float32 tensor holding
    each instance's (V_k, H_k, W_k) block in order (`split` returns the blocks as views).
    """

    def __init__(self, instances, cut: float = 3.0, eps: float = 0.0, znear: float = 0.1,
                 tile: int = 16, device="cuda", headroom: float = 1.5):
        if not 1 <= len(instances) <= B.MAX_INSTANCES:
            raise ValueError(f"1 .. {B.MAX_INSTANCES} instances")
        self.device = torch.device(device)
        vs = [v if isinstance(v, torch.Tensor) else views_to_device(v, self.device)
              for v, _, _ in instances]
        self.views = torch.cat(vs, 0).contiguous()
        self.shapes = [(int(v.shape[0]), int(H), int(W)) for v, (_, W, H) in zip(vs, instances)]
        self.offsets = block_offsets([a * b * c for a, b, c in self.shapes])
        self.img_numel = self.offsets[-1]
        self.opts = B.opts(cut=cut, eps=eps, znear=znear, tile=tile)
        self.headroom = float(headroom)
        self.ws = None
        self.ws_counts = None
        self.capacity = 0
        self._fwd_token = None

    def table(self, counts):
        if len(counts) != len(self.shapes):
            raise ValueError("one Gaussian count per instance")
        t = (B.GsInstance * len(counts))()
        for k, (n, (nv, H, W)) in enumerate(zip(counts, self.shapes)):
            t[k].n, t[k].n_views, t[k].W, t[k].H = int(n), nv, W, H
        return t

    def split(self, flat: torch.Tensor):
        return [flat[o:o + nv * H * W].view(nv, H, W)
                for o, (nv, H, W) in zip(self.offsets, self.shapes)]

    def _alloc(self, counts, pairs):
        t = self.table(counts)
        nbytes = int(B.lib().gs_project_batch_workspace_size(t, len(counts),
                                                             ctypes.byref(self.opts), int(pairs)))
        if nbytes == 0:
            raise B.GsError("invalid batch sizes")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ws_counts = list(counts)
        self.capacity = pairs

    def count_pairs(self, mean_rho, scale, quat, counts) -> int:
        if self.ws is None or self.ws_counts != list(counts):
            self._alloc(counts, 0)
        out = ctypes.c_int64(0)
        t = self.table(counts)
        B.check(B.lib().gs_project_batch_count_pairs(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), B.ptr(self.views), t, len(counts),
            ctypes.byref(self.opts), B.ptr(self.ws), self.ws.numel(), B.stream_handle(),
            ctypes.byref(out)), "gs_project_batch_count_pairs")
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

    def forward(self, mean_rho, scale, quat, counts, out: torch.Tensor | None = None):
        mean_rho, scale, quat = _f4(mean_rho, "mean_rho"), _f4(scale, "scale"), _f4(quat, "quat")
        self._ready(mean_rho, scale, quat, counts)
        if out is None:
            out = torch.empty(self.img_numel, dtype=torch.float32, device=self.device)
        t = self.table(counts)
        B.check(B.lib().gs_project_batch(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), B.ptr(self.views), t, len(counts),
            ctypes.byref(self.opts), B.ptr(out), B.ptr(self.ws), self.ws.numel(),
            B.stream_handle()), "gs_project_batch")
        self._fwd_token = Projector._token(mean_rho, scale, quat) + (tuple(counts),)
        return out

    def backward(self, mean_rho, scale, quat, counts, dimg, grads=None, accumulate=False,
                 reuse: bool | None = None):
        mean_rho, scale, quat = _f4(mean_rho, "mean_rho"), _f4(scale, "scale"), _f4(quat, "quat")
        dimg = dimg.contiguous()
        self._ready(mean_rho, scale, quat, counts)
        if reuse is None:
            reuse = self._fwd_token == Projector._token(mean_rho, scale, quat) + (tuple(counts),)
        if grads is None:
            grads = tuple(torch.empty_like(x) for x in (mean_rho, scale, quat))
            accumulate = False
        g_mr, g_sc, g_q = grads
        t = self.table(counts)
        B.check(B.lib().gs_project_batch_backward(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), B.ptr(self.views), t, len(counts),
            ctypes.byref(self.opts), B.ptr(dimg), B.ptr(g_mr), B.ptr(g_sc), B.ptr(g_q),
            1 if accumulate else 0, 1 if reuse else 0, B.ptr(self.ws), self.ws.numel(),
            B.stream_handle()), "gs_project_batch_backward")
        return g_mr, g_sc, g_q

    def count_evals(self, mean_rho, scale, quat, counts) -> int:
        self.ensure_capacity(mean_rho, scale, quat, counts)
        t = self.table(counts)
        B.check(B.lib().gs_project_batch_count_evals(
            B.ptr(mean_rho), B.ptr(scale), B.ptr(quat), B.ptr(self.views), t, len(counts),
            ctypes.byref(self.opts), B.ptr(self.ws), self.ws.numel(), B.stream_handle()),
            "gs_project_batch_count_evals")
        self._fwd_token = None
        return int(B.read_status(self.ws).evals)


class ProjectFunction(torch.autograd.Function):
    """img = Project(mean_rho, scale, quat) with the hand-written backward kernels."""

    @staticmethod
    def forward(ctx, mean_rho, scale, quat, projector: Projector):
        img = projector.forward(mean_rho, scale, quat)
        ctx.save_for_backward(mean_rho, scale, quat)
        ctx.projector = projector
        return img

    @staticmethod
    def backward(ctx, dimg):
        mean_rho, scale, quat = ctx.saved_tensors
        g = ctx.projector.backward(mean_rho, scale, quat, dimg)
        return g[0], g[1], g[2], None


def project(mean_rho, scale, quat, projector: Projector):
    return ProjectFunction.apply(mean_rho, scale, quat, projector)
