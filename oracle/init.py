"""CPU reference of the initialisation (Sec. 3.1) -- TEST INFRASTRUCTURE ONLY.

fdk(): Feldkamp-Davis-Kress reconstruction written from the textbook algorithm (cosine weight
in the plane of the rotation axis, Ram-Lak ramp filter along detector rows by direct
convolution, back-projection with the D_so^2 / U^2 weight and bilinear detector
interpolation, scale pi / V for V views over a full circle), in float64 numpy.

grad_init(): sampling of Gaussian means proportional to the gradient magnitude of a volume
above a background threshold.  The per-voxel weight |grad V| is computed with plain IEEE
single-precision operations in a fixed order (the precision the kernel takes the sampling
decision in), the CDF in float64.  Densities use trilinear interpolation
(scipy.ndimage.map_coordinates, order 1, clamped), nearest-neighbour distances come from
scipy's cKDTree.
"""
from __future__ import annotations

import numpy as np


def _frame(view13):
    s = view13[0:3]
    c = view13[3:6]
    u = view13[6:9]
    v = view13[9:12]
    pu, pv = np.linalg.norm(u), np.linalg.norm(v)
    eu, ev = u / pu, v / pv
    d = c - s
    Dsd = np.linalg.norm(d)
    n = d / Dsd
    Dso = -(s @ n)
    return s, eu, ev, n, pu, pv, Dsd, Dso


def ramlak(W, tau):
    """h(k tau) for k = -(W-1) .. W-1."""
    k = np.arange(-(W - 1), W)
    h = np.zeros(2 * W - 1)
    h[k == 0] = 1.0 / (4.0 * tau * tau)
    odd = (k % 2) != 0
    h[odd] = -1.0 / (np.pi * np.pi * tau * tau * k[odd].astype(np.float64) ** 2)
    return h


def fdk(proj, V13, grid):
    """proj (V, H, W), V13 (V, 13) float64 views, grid record -> volume (nz, ny, nx)."""
    proj = np.asarray(proj, dtype=np.float64)
    nv, H, W = proj.shape
    dims = [int(x) for x in np.asarray(grid["dims"]).ravel()]
    o = np.asarray(grid["origin"], dtype=np.float64).ravel()
    h = np.asarray(grid["voxel"], dtype=np.float64).ravel()
    zz, yy, xx = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]),
                             indexing="ij")
    X = np.stack([o[0] + (xx + 0.5) * h[0], o[1] + (yy + 0.5) * h[1],
                  o[2] + (zz + 0.5) * h[2]], axis=-1)
    vol = np.zeros(dims[::-1])
    for k in range(nv):
        s, eu, ev, n, pu, pv, Dsd, Dso = _frame(V13[k])
        scale = Dso / Dsd
        tau = pu * scale
        us = ((np.arange(W) + 0.5 - 0.5 * W) * pu * scale)[None, :]
        vs = ((np.arange(H) + 0.5 - 0.5 * H) * pv * scale)[:, None]
        wgt = proj[k] * Dso / np.sqrt(Dso * Dso + us * us + vs * vs)
        hk = ramlak(W, tau)
        q = np.empty_like(wgt)
        for r in range(H):
            full = np.convolve(wgt[r], hk)
            q[r] = tau * full[W - 1:2 * W - 1]
        R = X - s
        U = R @ n
        ud = Dsd * (R @ eu) / U
        vd = Dsd * (R @ ev) / U
        cx = ud / pu + 0.5 * W - 0.5
        cy = vd / pv + 0.5 * H - 0.5
        fx, fy = np.floor(cx), np.floor(cy)
        ax, ay = cx - fx, cy - fy
        ix, iy = fx.astype(np.int64), fy.astype(np.int64)
        val = np.zeros_like(cx)
        for dxo, dyo, wt in ((0, 0, (1 - ax) * (1 - ay)), (1, 0, ax * (1 - ay)),
                             (0, 1, (1 - ax) * ay), (1, 1, ax * ay)):
            jx, jy = ix + dxo, iy + dyo
            ok = (jx >= 0) & (jx < W) & (jy >= 0) & (jy < H)
            val[ok] += wt[ok] * q[jy[ok], jx[ok]]
        good = U > 0
        vol[good] += (Dso * Dso / (U[good] ** 2)) * val[good]
    return vol * np.pi / nv


def grad_weights_f32(V, grid, frac):
    """|grad V| above the threshold in the kernel's single-precision operation order."""
    V = np.asarray(V, dtype=np.float32)
    nz, ny, nx = V.shape
    h = np.asarray(grid["voxel"], dtype=np.float32).ravel()
    thr = np.float32(frac) * np.float32(V.max())

    def diff(axis, hh):
        n_ax = V.shape[axis]
        idx = np.arange(n_ax)
        hi = np.minimum(idx + 1, n_ax - 1)
        lo = np.maximum(idx - 1, 0)
        num = np.take(V, hi, axis=axis) - np.take(V, lo, axis=axis)  # float32
        den = ((hi - lo).astype(np.float32) * np.float32(hh)).astype(np.float32)
        shape = [1, 1, 1]
        shape[axis] = n_ax
        den = den.reshape(shape)
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.where(den > 0, num / np.where(den > 0, den, np.float32(1)), np.float32(0))
        return g.astype(np.float32)

    gx, gy, gz = diff(2, h[0]), diff(1, h[1]), diff(0, h[2])
    s = (gx * gx + gy * gy).astype(np.float32) + (gz * gz).astype(np.float32)
    w = np.sqrt(s.astype(np.float32)).astype(np.float32)
    return np.where(V > thr, w, np.float32(0)).astype(np.float64)


def grad_init(V, grid, n, frac, k_density, min_scale, uniforms):
    """Returns (mean_rho (n,4), scale (n,4), quat (n,4), voxel index (n,), cdf margin (n,))."""
    from scipy import ndimage
    from scipy.spatial import cKDTree

    V32 = np.asarray(V, dtype=np.float32)
    nz, ny, nx = V32.shape
    o = np.asarray(grid["origin"], dtype=np.float64).ravel()
    h = np.asarray(grid["voxel"], dtype=np.float64).ravel()
    w = grad_weights_f32(V32, grid, frac).ravel()
    cdf = np.cumsum(w)
    total = cdf[-1]
    u = np.asarray(uniforms, dtype=np.float32).astype(np.float64).reshape(n, 4)
    target = u[:, 0] * total
    idx = np.searchsorted(cdf, target, side="right")  # first index with cdf > target
    idx = np.minimum(idx, cdf.size - 1)
    # distance of each target to the nearest CDF boundary (guard band for the decision)
    margin = np.minimum(np.abs(cdf[idx] - target),
                        np.abs(target - np.where(idx > 0, cdf[np.maximum(idx - 1, 0)], 0.0)))
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    cx, cy, cz = x + u[:, 1], y + u[:, 2], z + u[:, 3]
    P = np.stack([o[0] + cx * h[0], o[1] + cy * h[1], o[2] + cz * h[2]], axis=1)
    coords = np.stack([cz - 0.5, cy - 0.5, cx - 0.5])
    coords = np.stack([np.clip(coords[0], 0, nz - 1), np.clip(coords[1], 0, ny - 1),
                       np.clip(coords[2], 0, nx - 1)])
    rho = k_density * ndimage.map_coordinates(V32.astype(np.float64), coords, order=1,
                                              mode="nearest")
    d, _ = cKDTree(P).query(P, k=2)
    s = np.maximum(d[:, 1], min_scale)
    mean_rho = np.concatenate([P, rho[:, None]], axis=1)
    scale = np.stack([s, s, s, np.zeros(n)], axis=1)
    quat = np.zeros((n, 4))
    quat[:, 0] = 1.0
    return mean_rho, scale, quat, idx.astype(np.int64), margin / max(total, 1e-300)
