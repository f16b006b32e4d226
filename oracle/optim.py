"""FP64 reference of the optimiser step -- TEST INFRASTRUCTURE ONLY.

Adam (Kingma and Ba, 2015) with bias correction on raw parameters, and the activations the
library applies: mean raw, density = softplus(raw), scale = exp(raw) with the log-scale
clamped after the update, quaternion raw.  Gradients arrive with respect to the activated
parameters and are chained through the activations.
"""
from __future__ import annotations

import numpy as np


def softplus(x):
    return np.where(x > 20, x, np.log1p(np.exp(np.minimum(x, 20))))


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def activate(raw_mr, raw_sc, raw_q):
    mr = np.concatenate([raw_mr[:, :3], softplus(raw_mr[:, 3:4])], 1)
    sc = np.concatenate([np.exp(raw_sc[:, :3]), np.zeros((raw_sc.shape[0], 1))], 1)
    return mr, sc, raw_q.copy()


def adam_step(raw, m, v, grads_act, t, lr, beta1, beta2, eps, min_log_scale, max_log_scale):
    """raw, m, v: lists of three (N, 4) float64 arrays (mean_rho, scale, quat); m and v are
    updated in place, raw is returned updated; t = 1 for the first step.  lr = (mean, rho,
    scale, quat)."""
    raw_mr, raw_sc, raw_q = [a.copy() for a in raw]
    g_mr, g_sc, g_q = grads_act
    g_raw_mr = g_mr.copy()
    g_raw_mr[:, 3] = g_mr[:, 3] * sigmoid(raw_mr[:, 3])
    g_raw_sc = g_sc.copy()
    g_raw_sc[:, :3] = g_sc[:, :3] * np.exp(raw_sc[:, :3])
    g_raw_sc[:, 3] = 0.0
    lr_mean, lr_rho, lr_scale, lr_quat = lr
    lrs = [np.array([lr_mean, lr_mean, lr_mean, lr_rho]), np.array([lr_scale] * 3 + [0.0]),
           np.array([lr_quat] * 4)]
    out = []
    for p, g, mm, vv, lrv in zip((raw_mr, raw_sc, raw_q), (g_raw_mr, g_raw_sc, g_q), m, v, lrs):
        mm *= beta1
        mm += (1 - beta1) * g
        vv *= beta2
        vv += (1 - beta2) * g * g
        mhat = mm / (1 - beta1 ** t)
        vhat = vv / (1 - beta2 ** t)
        # a component whose gradients have all been zero has m = v = 0 and does not move
        # (with eps = 0 the quotient would read 0/0)
        den = np.sqrt(vhat) + eps
        step = np.divide(mhat, den, out=np.zeros_like(mhat), where=den > 0)
        out.append(p - lrv * step)
    out[1][:, :3] = np.clip(out[1][:, :3], min_log_scale, max_log_scale)
    out[1][:, 3] = raw_sc[:, 3]
    return out
