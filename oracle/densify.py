"""FP64 reference of adaptive density control -- TEST INFRASTRUCTURE ONLY (only tests/, the
smoke check and the benchmark's CPU legs may import it).

The paper's optimisation loop (Sec. 3.4) prunes, clones and splits Gaussians in the backward
pass and names no rule; the rules below are those of the 3D Gaussian splatting lineage it
builds on (Kerbl et al. 2023, via R2-Gaussian), restated for additive X-ray rendering:

* Statistic.  For every Gaussian, over the steps of a window, the detector-position gradient
  of every view in which the Gaussian has a listed tile, in normalised device coordinates
  (pixel coordinate px spans W pixels of [-1, 1], so dL/dndc_x = W/2 dL/dpx):
      stat += |(W/2 dL/dpx, H/2 dL/dpy)|,  vis += 1.
  The mean over the window is grad_scale * stat / vis; grad_scale (the views per step) turns
  the gradient of the all-views mean loss into that of a per-view loss.
* Prune when rho < min_density or the largest scale exceeds max_scale.
* Otherwise densify when the mean reaches grad_threshold: split when the largest scale
  exceeds split_scale, else clone.  With a Gaussian budget, only the highest-mean candidates
  (ties: lower index first) that fit under max_gaussians are densified.
* Clone: two copies of the Gaussian, each with density rho / 2 (the pair renders exactly as
  the parent).  The first keeps the Adam moments, the second starts from zero moments.
* Split: two children at p + R(q) diag(s) z_k (z_k standard normal draws, passed in), scales
  s / split_factor (log-scale clamped below at min_log_scale), and the density that conserves
  the integrated density rho (2 pi)^(3/2) s_x s_y s_z of the parent:
  rho' = rho split_factor^3 / 2.  Zero Adam moments.
* Option inherit_moments: every child (both clones, both split children) starts from its
  parent's Adam moments instead.
* Output order: Gaussian order, a densified Gaussian's two children consecutive.

Decisions (comparisons with the thresholds, the budget ranking) are taken in FP32, the
precision of the kernels that take them; children's parameters are computed in FP64.
"""
from __future__ import annotations

import numpy as np

from . import optim

PRUNE, KEEP, CLONE, SPLIT = 0, 1, 2, 3


def view_position_grads(fp, dimg):
    """d<dimg_v, I_v>/d(px, py) per (view, Gaussian) from footprint records fp (the dict of
    oracle.footprints): I_v = A exp(-q/2) over the pixels of the box with q < Q, q = ca dx^2 +
    2 cb dx dy + cc dy^2, dx = x - px, so dI/dpx = A exp(-q/2) (ca dx + cb dy) and
    dI/dpy = A exp(-q/2) (cb dx + cc dy).  Returns (V, N, 2)."""
    nv, n = fp["px"].shape
    out = np.zeros((nv, n, 2))
    for v in range(nv):
        for i in range(n):
            if fp["culled"][v, i]:
                continue
            x0, x1 = int(fp["ix0"][v, i]), int(fp["ix1"][v, i])
            y0, y1 = int(fp["iy0"][v, i]), int(fp["iy1"][v, i])
            if x0 > x1 or y0 > y1:
                continue
            ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1]
            dx = xs - fp["px"][v, i]
            dy = ys - fp["py"][v, i]
            ca, cb, cc = fp["ca"][v, i], fp["cb"][v, i], fp["cc"][v, i]
            q = ca * dx * dx + 2 * cb * dx * dy + cc * dy * dy
            m = q < fp["Q"][v, i]
            e = fp["A"][v, i] * np.exp(-0.5 * q) * dimg[v, ys, xs] * m
            out[v, i, 0] = np.sum(e * (ca * dx + cb * dy))
            out[v, i, 1] = np.sum(e * (cb * dx + cc * dy))
    return out


def grad_stats(fp, dimg, tile_counts, W, H):
    """(stat, vis) of one backward: tile_counts (V, N) = listed tiles per pair (oracle.keys)."""
    g = view_position_grads(fp, dimg)
    visible = tile_counts > 0
    norm = np.hypot(0.5 * W * g[:, :, 0], 0.5 * H * g[:, :, 1])
    return (norm * visible).sum(axis=0), visible.sum(axis=0).astype(np.int64)


def _f32(x):
    return np.asarray(x, dtype=np.float32)


def classify(raw_mr, raw_sc, stat, vis, opts):
    """Action per Gaussian (PRUNE / KEEP / CLONE / SPLIT) and the FP32 mean statistic.
    opts: dict with grad_threshold, grad_scale, split_scale, min_density, max_scale,
    max_gaussians.  stat (FP32) and vis are the accumulated statistics."""
    n = raw_mr.shape[0]
    rho = _f32(optim.softplus(_f32(raw_mr[:, 3]).astype(np.float64)))
    smax = _f32(np.exp(_f32(raw_sc[:, :3]).astype(np.float64).max(axis=1)))
    vis = np.asarray(vis, dtype=np.int64)
    avg = np.where(vis > 0, _f32(stat) / np.maximum(vis, 1).astype(np.float32), np.float32(0))
    avg = _f32(avg)
    prune = ~(rho >= np.float32(opts["min_density"])) | (smax > np.float32(opts["max_scale"]))
    cand = ~prune & (vis > 0) & (avg * np.float32(opts["grad_scale"]) >=
                                 np.float32(opts["grad_threshold"]))
    act = np.full(n, KEEP, dtype=np.int32)
    act[prune] = PRUNE
    idx = np.nonzero(cand)[0]
    budget = int(opts["max_gaussians"]) - (n - int(prune.sum()))
    if budget < idx.size:
        # highest mean first, ties by lower index
        order = sorted(idx.tolist(), key=lambda i: (-float(avg[i]), i))
        idx = np.array(sorted(order[:max(budget, 0)]), dtype=np.int64)
    split = smax[idx] > np.float32(opts["split_scale"])
    act[idx[split]] = SPLIT
    act[idx[~split]] = CLONE
    return act, avg, int(cand.sum())


def inverse_softplus(y):
    y = np.asarray(y, dtype=np.float64)
    return np.where(y > 20, y, np.log(np.expm1(np.minimum(y, 20))))


def densify(raw_mr, raw_sc, raw_q, m, v, stat, vis, normals, opts):
    """Applies the rules; raw_* (N, 4), m and v (N, 3, 4) Adam moments, normals (N, 6).
    Returns (out_raw_mr, out_raw_sc, out_raw_q, out_m, out_v, act, candidates)."""
    act, _, cands = classify(raw_mr, raw_sc, stat, vis, opts)
    phi = float(opts["split_factor"])
    inherit = bool(opts.get("inherit_moments", 0))
    outs = [[] for _ in range(5)]

    def put(a, b, c, mm, vv):
        for lst, x in zip(outs, (a, b, c, mm, vv)):
            lst.append(np.asarray(x, dtype=np.float64))

    zero = np.zeros((3, 4))
    for i in range(raw_mr.shape[0]):
        a, b, c = raw_mr[i].astype(np.float64), raw_sc[i].astype(np.float64), raw_q[i]
        if act[i] == PRUNE:
            continue
        if act[i] == KEEP:
            put(a, b, c, m[i], v[i])
            continue
        rho = float(optim.softplus(np.array(a[3])))
        if act[i] == CLONE:
            half = a.copy()
            half[3] = inverse_softplus(0.5 * rho)
            put(half, b, c, m[i], v[i])
            put(half, b, c, *((m[i], v[i]) if inherit else (zero, zero)))
            continue
        qn = np.asarray(c, dtype=np.float64)
        qn = qn / np.linalg.norm(qn)
        w, x, y, z = qn
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        s = np.exp(b[:3])
        child_sc = b.copy()
        child_sc[:3] = np.maximum(b[:3] - np.log(phi), float(opts["min_log_scale"]))
        for k in range(2):
            child = a.copy()
            child[:3] = a[:3] + R @ (s * normals[i, 3 * k:3 * k + 3])
            child[3] = inverse_softplus(rho * phi ** 3 / 2.0)
            put(child, child_sc, c, *((m[i], v[i]) if inherit else (zero, zero)))
    shapes = [(0, 4), (0, 4), (0, 4), (0, 3, 4), (0, 3, 4)]
    res = [np.stack(o) if o else np.zeros(sh) for o, sh in zip(outs, shapes)]
    return (*res, act, cands)


def mass(raw_mr, raw_sc):
    """Integrated density rho (2 pi)^(3/2) s_x s_y s_z of raw-form Gaussians."""
    rho = optim.softplus(np.asarray(raw_mr, dtype=np.float64)[:, 3])
    return rho * (2 * np.pi) ** 1.5 * np.exp(np.asarray(raw_sc, dtype=np.float64)[:, :3].sum(1))
