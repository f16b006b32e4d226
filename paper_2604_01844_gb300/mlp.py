"""Per-brick MLP initializer: a 16^3 FDK brick (4096 values) -> 3 hidden layers of 256 (ReLU)
-> 32 Gaussians x 11 raw parameters, BF16 weights and activations with FP32 accumulation on the
library's tcgen05 GEMM.  Trained through the fused brick render + L1 kernel (gs_brick_loss), so
that the unordered set of 32 Gaussians needs no matching.  This module only orders the library
calls; every operation is a libgsct kernel.
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
    def __init__(self, seed: int = 0, device="cuda"):
        self.device = torch.device(device)
        rng = np.random.default_rng(seed)
        shapes = [(HIDDEN, K_IN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (N_OUT_PAD, HIDDEN)]
        self.W, self.b = [], []
        for li, (o, i) in enumerate(shapes):
            w = rng.standard_normal((o, i)) * np.sqrt(2.0 / i)
            b = np.zeros(o)
            if li == 3:
                w *= 0.1
                w[N_OUT:] = 0.0
                # start from the lattice (offsets 0, base scales) with densities about the
                # mean intensity of a normalised brick
                b[:N_OUT].reshape(32, 11)[:, 10] = -0.5
            self.W.append(torch.from_numpy(w.astype(np.float32)).to(self.device))
            self.b.append(torch.from_numpy(b.astype(np.float32)).to(self.device))
        self.W16 = [torch.empty(w.shape, dtype=torch.bfloat16, device=self.device) for w in self.W]
        self.params = self.W + self.b
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.grads = [torch.zeros_like(p) for p in self.params]
        self.step_count = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.err = torch.zeros(1, dtype=torch.int32, device=self.device)
        self._sync_bf16()
        self._bufs = {}

    def _sync_bf16(self):
        for w, w16 in zip(self.W, self.W16):
            B.check(B.lib().gs_f32_to_bf16(B.ptr(w), B.ptr(w16), w.numel(), _s()), "f32_to_bf16")

    def _buf(self, name, shape, dtype):
        t = self._bufs.get(name)
        if t is None or tuple(t.shape) != tuple(shape) or t.dtype != dtype:
            t = torch.empty(shape, dtype=dtype, device=self.device)
            self._bufs[name] = t
        return t

    def _gemm(self, a, b, M, N, K, bias=None, relu=False, c32=None, c16=None, ldc=None):
        B.check(B.lib().gs_gemm_bf16(B.ptr(a), B.ptr(b), M, N, K, B.ptr(bias), 1 if relu else 0,
                                     B.ptr(c32), B.ptr(c16), ldc or N, B.ptr(self.err), _s()),
                "gs_gemm_bf16")

    # -- forward ----------------------------------------------------------------------
    def forward(self, x16: torch.Tensor) -> torch.Tensor:
        """x16: (M, 4096) bf16, M % 128 == 0 -> raw outputs (M, 384) float32."""
        M = x16.shape[0]
        if M % 128:
            raise ValueError("the brick batch must be a multiple of 128")
        self.x16 = x16
        self.h = []
        a = x16
        K = K_IN
        for li in range(3):
            h = self._buf(f"h{li}", (M, HIDDEN), torch.bfloat16)
            self._gemm(a, self.W16[li], M, HIDDEN, K, bias=self.b[li], relu=True, c16=h)
            self.h.append(h)
            a, K = h, HIDDEN
        y = self._buf("y", (M, N_OUT_PAD), torch.float32)
        self._gemm(a, self.W16[3], M, N_OUT_PAD, HIDDEN, bias=self.b[3], c32=y)
        return y

    # -- backward ---------------------------------------------------------------------
    def backward(self, dy: torch.Tensor):
        """dy: (M, 384) float32 gradient of the raw outputs (padded columns zero); fills
        self.grads (W1..W4, b1..b4).  Uses the activations of the last forward."""
        L = B.lib()
        M = dy.shape[0]
        acts = [self.x16] + self.h  # inputs of layers 0..3
        g32 = dy
        g16 = self._buf("g16_out", (M, N_OUT_PAD), torch.bfloat16)
        B.check(L.gs_f32_to_bf16(B.ptr(g32), B.ptr(g16), g32.numel(), _s()), "f32_to_bf16")
        width = N_OUT_PAD
        for li in (3, 2, 1, 0):
            a_in = acts[li]
            k_in = a_in.shape[1]
            # bias gradient
            B.check(L.gs_colsum(B.ptr(g32), M, width, B.ptr(self.grads[4 + li]), _s()), "colsum")
            # weight gradient: dW = g^T a_in  (TN GEMM on the transposes, K = M)
            gT = self._buf(f"gT{li}", (width, M), torch.bfloat16)
            aT = self._buf(f"aT{li}", (k_in, M), torch.bfloat16)
            B.check(L.gs_transpose_bf16(B.ptr(g16), M, width, B.ptr(gT), _s()), "transpose")
            B.check(L.gs_transpose_bf16(B.ptr(a_in), M, k_in, B.ptr(aT), _s()), "transpose")
            self._gemm(gT, aT, width, k_in, M, c32=self.grads[li])
            if li == 0:
                break
            # gradient of the layer input: g W, then the ReLU of the previous layer
            WT = self._buf(f"WT{li}", (k_in, width), torch.bfloat16)
            B.check(L.gs_transpose_bf16(B.ptr(self.W16[li]), width, k_in, B.ptr(WT), _s()),
                    "transpose")
            g_prev = self._buf(f"gp{li}", (M, k_in), torch.float32)
            self._gemm(g16, WT, M, k_in, width, c32=g_prev)
            g16p = self._buf(f"g16_{li}", (M, k_in), torch.bfloat16)
            B.check(L.gs_relu_mask_bf16(B.ptr(g_prev), B.ptr(self.h[li - 1]), g_prev.numel(),
                                        B.ptr(g16p), _s()), "relu_mask")
            g32, g16, width = g_prev, g16p, k_in

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        L = B.lib()
        for i, (p, m, v, g) in enumerate(zip(self.params, self.m, self.v, self.grads)):
            p16 = self.W16[i] if i < 4 else None
            B.check(L.gs_adam_flat(B.ptr(p), B.ptr(m), B.ptr(v), B.ptr(g), p.numel(),
                                   B.ptr(self.step_count), lr, beta1, beta2, eps, B.ptr(p16),
                                   _s()), "adam_flat")
        B.check(L.gs_step_incr(B.ptr(self.step_count), _s()), "step_incr")

    # -- training ---------------------------------------------------------------------
    def train_step(self, x16, target, loss, lr=1e-3):
        """One step on a batch: forward, brick render + L1 (loss += mean |render - target|),
        backward, Adam."""
        y = self.forward(x16)
        M = x16.shape[0]
        dy = self._buf("dy", (M, N_OUT_PAD), torch.float32)
        B.check(B.lib().gs_memset(B.ptr(dy), 0, dy.numel() * 4, _s()), "memset")
        B.check(B.lib().gs_brick_loss(B.ptr(y), N_OUT_PAD, B.ptr(target), M, B.ptr(loss),
                                      B.ptr(dy), N_OUT_PAD, None, _s()), "gs_brick_loss")
        self.backward(dy)
        self.adam(lr=lr)

    def infer_gaussians(self, x16, geo, amp: float):
        """World-space Gaussians (32 per brick) for the bricks in x16; geo (M, 4) float32 =
        origin and voxel size of each brick; densities times amp."""
        y = self.forward(x16)
        M = x16.shape[0]
        out = [torch.empty((M * 32, 4), dtype=torch.float32, device=self.device) for _ in range(3)]
        B.check(B.lib().gs_brick_decode(B.ptr(y), N_OUT_PAD, B.ptr(geo), M, amp,
                                        *[B.ptr(t) for t in out], _s()), "gs_brick_decode")
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
