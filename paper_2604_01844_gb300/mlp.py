"""Per-brick MLP initializer: a 16^3 FDK brick (4096 values) -> 3 hidden layers of 256 (ReLU)
-> 32 Gaussians x 11 raw parameters, BF16 weights and activations with FP32 accumulation on the
library's tcgen05 GEMM.  Trained through the fused brick render + L1 kernel (gs_brick_loss), so
that the unordered set of 32 Gaussians needs no matching.  The network's forward, backward,
training step and inference are single library calls (gs_mlp_*); this module allocates their
buffers and marshals the arguments.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import binding as B

K_IN = 4096
HIDDEN = 256
N_OUT = 352        # 32 Gaussians x 11
N_OUT_PAD = 384    # multiple of the GEMM's 128-column tile


def _s():
    return B.stream_handle()


class BrickMLP:
    """Device state of the network in the library's flat layout (gs_mlp_param_count FP32
    parameters W1..W4, b1..b4; BF16 weights; Adam moments; gradients) and the calls of its
    forward, backward, training step and inference."""

    def __init__(self, seed: int = 0, device="cuda"):
        self.device = torch.device(device)
        L = B.lib()
        n_par, n_w = int(L.gs_mlp_param_count()), int(L.gs_mlp_weight_count())
        rng = np.random.default_rng(seed)
        shapes = [(HIDDEN, K_IN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (N_OUT_PAD, HIDDEN)]
        flat = np.zeros(n_par, dtype=np.float32)
        off = 0
        ws, bs = [], []
        for li, (o, i) in enumerate(shapes):
            w = rng.standard_normal((o, i)) * np.sqrt(2.0 / i)
            b = np.zeros(o)
            if li == 3:
                w *= 0.1
                w[N_OUT:] = 0.0
                # start from the lattice (offsets 0, base scales) with densities about the
                # mean intensity of a normalised brick
                b[:N_OUT].reshape(32, 11)[:, 10] = -0.5
            ws.append(w)
            bs.append(b)
        for w in ws:
            flat[off:off + w.size] = w.ravel()
            off += w.size
        for b in bs:
            flat[off:off + b.size] = b
            off += b.size
        assert off == n_par and sum(w.size for w in ws) == n_w
        self.flat = torch.from_numpy(flat).to(self.device)
        self.flat16 = torch.empty(n_w, dtype=torch.bfloat16, device=self.device)
        self.flat_m = torch.zeros_like(self.flat)
        self.flat_v = torch.zeros_like(self.flat)
        self.flat_grad = torch.zeros_like(self.flat)
        # per-tensor views, [out][in] weights then biases
        self.W, self.b, self.W16, gw, gb = [], [], [], [], []
        off = 0
        for o, i in shapes:
            self.W.append(self.flat[off:off + o * i].view(o, i))
            self.W16.append(self.flat16[off:off + o * i].view(o, i))
            gw.append(self.flat_grad[off:off + o * i].view(o, i))
            off += o * i
        for o, _ in shapes:
            self.b.append(self.flat[off:off + o])
            gb.append(self.flat_grad[off:off + o])
            off += o
        self.params = self.W + self.b
        self.grads = gw + gb
        self.step_count = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.err = torch.zeros(1, dtype=torch.int32, device=self.device)
        self._ws = {}
        self._sync_bf16()

    def _sync_bf16(self):
        B.check(B.lib().gs_mlp_sync_bf16(B.ptr(self.flat), B.ptr(self.flat16), _s()),
                "gs_mlp_sync_bf16")

    def workspace(self, M: int) -> torch.Tensor:
        ws = self._ws.get(M)
        if ws is None:
            nbytes = int(B.lib().gs_mlp_workspace_size(M))
            if nbytes == 0:
                raise ValueError("the brick batch must be a positive multiple of 128")
            ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self._ws = {M: ws}
        return ws

    # -- forward ----------------------------------------------------------------------
    def forward(self, x16: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """x16: (M, 4096) bf16, M % 128 == 0 -> raw outputs (M, 384) float32."""
        M = x16.shape[0]
        ws = self.workspace(M)
        y = out if out is not None else torch.empty((M, N_OUT_PAD), dtype=torch.float32,
                                                    device=self.device)
        self.x16 = x16
        B.check(B.lib().gs_mlp_forward(B.ptr(self.flat), B.ptr(self.flat16), B.ptr(x16), M,
                                       B.ptr(y), B.ptr(ws), ws.numel(), B.ptr(self.err), _s()),
                "gs_mlp_forward")
        return y

    # -- backward ---------------------------------------------------------------------
    def backward(self, dy: torch.Tensor):
        """dy: (M, 384) float32 gradient of the raw outputs (padded columns zero); fills
        self.grads (W1..W4, b1..b4).  Uses the activations of the last forward."""
        M = dy.shape[0]
        ws = self.workspace(M)
        B.check(B.lib().gs_mlp_backward(B.ptr(self.flat16), B.ptr(self.x16), M,
                                        B.ptr(dy.contiguous()), B.ptr(self.flat_grad),
                                        B.ptr(ws), ws.numel(), B.ptr(self.err), _s()),
                "gs_mlp_backward")

    # -- training ---------------------------------------------------------------------
    def train_step(self, x16, target, loss, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        """One step on a batch: forward, brick render + L1 (loss += mean |render - target|),
        backward, Adam (gs_mlp_train_step)."""
        M = x16.shape[0]
        ws = self.workspace(M)
        B.check(B.lib().gs_mlp_train_step(
            B.ptr(self.flat), B.ptr(self.flat16), B.ptr(self.flat_m), B.ptr(self.flat_v),
            B.ptr(self.flat_grad), B.ptr(self.step_count), B.ptr(x16), B.ptr(target), M, lr,
            beta1, beta2, eps, B.ptr(loss), B.ptr(ws), ws.numel(), B.ptr(self.err), _s()),
            "gs_mlp_train_step")

    def infer_gaussians(self, x16, geo, amp: float):
        """World-space Gaussians (32 per brick) for the bricks in x16; geo (M, 4) float32 =
        origin and voxel size of each brick; densities times amp (gs_mlp_infer)."""
        M = x16.shape[0]
        ws = self.workspace(M)
        out = [torch.empty((M * 32, 4), dtype=torch.float32, device=self.device) for _ in range(3)]
        B.check(B.lib().gs_mlp_infer(B.ptr(self.flat), B.ptr(self.flat16), B.ptr(x16), M,
                                     B.ptr(geo), amp, *[B.ptr(t) for t in out], B.ptr(ws),
                                     ws.numel(), B.ptr(self.err), _s()), "gs_mlp_infer")
        return out


def brick_ids(nb: tuple, keep: np.ndarray | None = None) -> np.ndarray:
    """int32 (n, 4) brick coordinates (bx, by, bz, 0) of a grid of nb = (bx, by, bz) bricks."""
    bz, by, bx = np.meshgrid(np.arange(nb[2]), np.arange(nb[1]), np.arange(nb[0]), indexing="ij")
    ids = np.stack([bx.ravel(), by.ravel(), bz.ravel(), np.zeros(bx.size, dtype=np.int64)], 1)
    if keep is not None:
        ids = ids[keep]
    return np.ascontiguousarray(ids.astype(np.int32))


def extract(vol: torch.Tensor, ids: torch.Tensor, scale: float, as_bf16: bool):
    nz, ny, nx = vol.shape
    n = ids.shape[0]
    out = torch.empty((n, K_IN), dtype=torch.bfloat16 if as_bf16 else torch.float32,
                      device=vol.device)
    B.check(B.lib().gs_extract_bricks(B.ptr(vol), nx, ny, nz, B.ptr(ids), n, scale,
                                      B.ptr(out) if as_bf16 else None,
                                      None if as_bf16 else B.ptr(out), _s()), "gs_extract_bricks")
    return out
