"""CPU reference of the per-brick MLP initializer -- TEST INFRASTRUCTURE ONLY.

float64 PyTorch; gradients by autograd.  The network's inputs, weights and hidden activations
are rounded to bfloat16 at the same points as the device path (the GEMM operands), so the
comparison isolates accumulation order.  The brick decoding and rendering follow the stated
parameterisation in brick-local voxel units.
"""
from __future__ import annotations

import torch

BRICK = 16


def bf16(t):
    return t.to(torch.bfloat16).to(torch.float64)


def mlp_forward(x, Ws, bs):
    """x (M, 4096); Ws[i] (out, in); bs[i] (out,).  Returns raw outputs (M, out4)."""
    h = bf16(x)
    for li in range(3):
        h = bf16(torch.relu(h @ bf16(Ws[li]).T + bs[li]))
    return h @ bf16(Ws[3]).T + bs[3]


def lattice():
    """Cell centre, half-cell size and base scale of the 32 Gaussians of a brick: Gaussian g
    in cell (g % 4, g / 4 % 4, g / 16) of a 4 x 4 x 2 lattice of 4 x 4 x 8-voxel cells."""
    g = torch.arange(32)
    base = torch.stack([((g % 4) + 0.5) * 4.0, (((g // 4) % 4) + 0.5) * 4.0,
                        ((g // 16) + 0.5) * 8.0], -1).to(torch.float64)
    half = torch.tensor([2.0, 2.0, 4.0], dtype=torch.float64)
    sbase = torch.tensor([1.2, 1.2, 2.4], dtype=torch.float64)
    return base, half, sbase


def decode(raw):
    """raw (B, 32, 11) -> centres (B,32,3), scales, unit quaternions, densities."""
    base, half, sbase = lattice()
    c = base + half * torch.tanh(raw[..., 0:3])
    s = sbase * torch.exp(torch.clamp(raw[..., 3:6], -3.0, 2.0))
    q = torch.cat([1 + raw[..., 6:7], raw[..., 7:10]], -1)
    q = q / torch.sqrt((q * q).sum(-1, keepdim=True) + 1e-20)
    rho = torch.nn.functional.softplus(raw[..., 10])
    return c, s, q, rho


def quat_rot(q):
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


MARGIN = 4


def render(raw, margin=MARGIN):
    """(B, 352) raw -> (B, S^3) renderings over the brick plus `margin` voxels on every side,
    S = 16 + 2 margin, [z][y][x], 3-sigma cut."""
    Bn = raw.shape[0]
    c, s, q, rho = decode(raw.reshape(Bn, 32, 11))
    R = quat_rot(q)
    Si = R @ torch.diag_embed(1.0 / (s * s)) @ R.transpose(-1, -2)  # (B, 32, 3, 3)
    ax = torch.arange(-margin, BRICK + margin, dtype=torch.float64) + 0.5
    zz, yy, xx = torch.meshgrid(ax, ax, ax, indexing="ij")
    X = torch.stack([xx, yy, zz], -1).reshape(-1, 3)
    d = X[None, None, :, :] - c[:, :, None, :]
    qf = torch.einsum("ngva,ngak,ngvk->ngv", d, Si, d)
    e = torch.where(qf < 9.0, torch.exp(-0.5 * qf), torch.zeros_like(qf))
    return (rho[:, :, None] * e).sum(1)


def brick_l1(raw, target, margin=MARGIN):
    """Mean |render - target| over the extended region; target (B, 4096) inside the brick, 0
    in the margin."""
    Bn = raw.shape[0]
    S = BRICK + 2 * margin
    full = torch.zeros(Bn, S, S, S, dtype=torch.float64)
    full[:, margin:margin + BRICK, margin:margin + BRICK, margin:margin + BRICK] = \
        target.reshape(Bn, BRICK, BRICK, BRICK)
    return (render(raw, margin) - full.reshape(Bn, -1)).abs().mean()
