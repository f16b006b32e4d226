"""Shared helpers of the parity tests: device copies of the seeded inputs and the guard-band
tolerances of the FP32-vs-FP64 comparison."""
import numpy as np

# Guard band (FP32 path vs FP64 oracle).  A box edge decides ceil/floor of a pixel coordinate
# whose FP32 value carries an absolute error of a few ulp of the coordinate (<= max(W, H)):
# 1e-4 px plus 4e-6 * max(W, H) covers 30+ ulp at every size used.  The per-pixel cut q < Q is
# decided on an FP32 exponent with a relative error of a few 1e-7; 2e-5 * Q covers it.
REL_BAND = 2e-5


def px_band(W, H):
    return 1e-4 + 4e-6 * max(W, H)


IMG_TOL = 1e-4  # images: |gpu - oracle| <= 1e-4 * max|oracle| + guard-band allowance
GRAD_TOL = 1e-3  # gradients: |gpu - oracle| <= 1e-3 * (|oracle| + rms of that component)


def to_dev(mean_rho, scale, quat, device="cuda"):
    import torch

    return (torch.from_numpy(np.ascontiguousarray(mean_rho)).to(device),
            torch.from_numpy(np.ascontiguousarray(scale)).to(device),
            torch.from_numpy(np.ascontiguousarray(quat)).to(device))


def grads11(g_mr, g_sc, g_q):
    """(N, 11) = p[3], s[3], q[4], rho from the three float4 gradient tensors."""
    a, b, c = (t.detach().cpu().numpy().astype(np.float64) for t in (g_mr, g_sc, g_q))
    return np.concatenate([a[:, :3], b[:, :3], c[:, :4], a[:, 3:4]], axis=1)


ENTRY_TOL = 1e-2  # per entry: |gpu - oracle| <= 1e-2 |oracle| where |oracle| > 1e-2 rms


def assert_grads_close(got, want, rows, tol=GRAD_TOL, entry_tol=ENTRY_TOL):
    """Compare (N, 11) gradients on the selected rows, per parameter group: every entry within
    tol (|oracle| + rms of its group), and every entry larger than 1e-2 of the rms within
    entry_tol of its own magnitude (so that small entries are not hidden by the rms term)."""
    groups = [slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11)]
    for gsl in groups:
        w = want[rows][:, gsl]
        g = got[rows][:, gsl]
        rms = np.sqrt(np.mean(w * w)) + 1e-30
        err = np.abs(g - w)
        bound = tol * (np.abs(w) + rms)
        bad = err > bound
        assert not bad.any(), (gsl, int(bad.sum()), float((err / bound).max()))
        big = np.abs(w) > 1e-2 * rms
        rel = err[big] / np.abs(w[big])
        assert not (rel > entry_tol).any(), (gsl, "entry", int((rel > entry_tol).sum()),
                                             float(rel.max()))
