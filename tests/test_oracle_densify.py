"""Pins of the adaptive density control reference (oracle/densify.py) against facts it does not
compute itself: the dual-number parameter gradient, closed-form integrated densities, the
voxelizer, the distribution of a Gaussian, and order properties of the budget selection."""
import numpy as np
import pytest

import oracle
import synth
from oracle import densify as D
from oracle import optim as OO

OPTS = dict(grad_threshold=2e-4, grad_scale=1.0, split_scale=0.03, split_factor=1.6,
            min_density=1e-3, max_scale=0.4, min_log_scale=np.log(1e-4), max_gaussians=10 ** 9)


def _raw(n, seed, median=0.03):
    mr, sc, qt = synth.gaussians(seed, n, radius=0.5, scale_median=median)
    raw_mr = mr.astype(np.float64).copy()
    raw_mr[:, 3] = D.inverse_softplus(mr[:, 3])
    raw_sc = np.zeros((n, 4))
    raw_sc[:, :3] = np.log(sc[:, :3])
    return raw_mr.astype(np.float32), raw_sc.astype(np.float32), qt.astype(np.float32)


def test_position_gradient_matches_dual_number_gradient_in_parallel_beam():
    # parallel beam: px = (p - o) . u / |u|^2 + const and A, conic do not depend on p, so
    # dL/dp = dL/dpx u / |u|^2 + dL/dpy v / |v|^2 for one view
    W, H = 48, 40
    views = synth.parallel_views(1, W, H, angle0=0.3)
    mr, sc, qt = synth.gaussians(5, 20, radius=0.4, scale_median=0.06)
    P, V = oracle.params64(mr, sc, qt), oracle.views64(views)
    w = np.random.default_rng(1).standard_normal((1, H, W))
    g = D.view_position_grads(oracle.footprints(P, V, W, H), w)[0]
    u, v = V[0, 6:9], V[0, 9:12]
    want = oracle.project_grad(P, V, W, H, w)[:, 0:3]
    got = g[:, :1] * (u / u.dot(u)) + g[:, 1:2] * (v / v.dot(v))
    scale = np.abs(want).max()
    assert scale > 0
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9 * scale)


def test_grad_stats_visibility_is_listed_tiles():
    W, H = 40, 36
    views = synth.cone_views(3, W, H)
    mr, sc, qt = synth.gaussians(6, 30, radius=0.7, scale_median=0.03)
    P, V = oracle.params64(mr, sc, qt), oracle.views64(views)
    fp = oracle.footprints(P, V, W, H)
    _, _, counts = oracle.keys(P, V, W, H, 16)
    w = np.random.default_rng(2).standard_normal((3, H, W))
    stat, vis = D.grad_stats(fp, w, counts, W, H)
    assert np.array_equal(vis, (counts > 0).sum(0))
    g = D.view_position_grads(fp, w)
    # a Gaussian seen in one view only carries that view's NDC gradient norm
    one = np.nonzero(vis == 1)[0]
    for i in one:
        k = int(np.nonzero(counts[:, i] > 0)[0][0])
        assert np.isclose(stat[i], np.hypot(W / 2 * g[k, i, 0], H / 2 * g[k, i, 1]))
    assert np.all(stat[vis == 0] == 0)


def _act(raw_mr, raw_sc):
    return OO.softplus(raw_mr[:, 3].astype(np.float64)), np.exp(raw_sc[:, :3].astype(np.float64))


@pytest.mark.parametrize("kind", ["clone", "split"])
def test_children_conserve_integrated_density(kind):
    n = 40
    raw_mr, raw_sc, raw_q = _raw(n, 7)
    stat = np.full(n, 1.0, np.float32)
    vis = np.ones(n, np.int64)
    o = dict(OPTS, split_scale=(0.0 if kind == "split" else 10.0), max_scale=10.0,
             min_density=0.0)
    normals = np.random.default_rng(3).standard_normal((n, 6))
    m = np.random.default_rng(4).random((n, 3, 4))
    out = D.densify(raw_mr, raw_sc, raw_q, m, m, stat, vis, normals, o)
    act = out[5]
    assert np.all(act == (D.SPLIT if kind == "split" else D.CLONE))
    assert out[0].shape[0] == 2 * n
    parent = D.mass(raw_mr, raw_sc)
    kids = D.mass(out[0], out[1])
    np.testing.assert_allclose(kids[0::2] + kids[1::2], parent, rtol=1e-9)
    if kind == "clone":
        # the first copy keeps the moments, the second starts from zero
        np.testing.assert_array_equal(out[3][0::2], m)
        assert np.all(out[3][1::2] == 0)
    else:
        assert np.all(out[3] == 0) and np.all(out[4] == 0)
        np.testing.assert_allclose(np.exp(out[1][:, :3]),
                                   np.repeat(np.exp(raw_sc[:, :3].astype(np.float64)), 2, 0) / 1.6,
                                   rtol=1e-9)


def test_clone_renders_as_the_parent():
    n = 25
    raw_mr, raw_sc, raw_q = _raw(n, 8, median=0.05)
    o = dict(OPTS, split_scale=10.0, max_scale=10.0, min_density=0.0)
    out = D.densify(raw_mr, raw_sc, raw_q, np.zeros((n, 3, 4)), np.zeros((n, 3, 4)),
                    np.ones(n, np.float32), np.ones(n), np.zeros((n, 6)), o)
    grid = synth.cube_grid(24)

    def vox(rmr, rsc, rq):
        mr, sc, q = OO.activate(np.asarray(rmr, np.float64), np.asarray(rsc, np.float64),
                                np.asarray(rq, np.float64))
        return oracle.voxelize(oracle.params64(mr, sc, q), grid)[0]

    a, b = vox(raw_mr, raw_sc, raw_q), vox(*out[:3])
    np.testing.assert_allclose(b, a, rtol=1e-9, atol=1e-12 * np.abs(a).max())


def test_split_children_follow_the_parent_distribution():
    # one anisotropic rotated parent split many times: the child offsets p' - p = R diag(s) z
    # have covariance Sigma = R diag(s^2) R^T (a transposed R or a wrong scale fails)
    k = 20000
    s = np.array([0.05, 0.02, 0.01])
    q = np.array([0.8, 0.3, -0.4, 0.34])
    raw_mr = np.tile(np.array([[0.1, -0.2, 0.05, 1.0]], np.float32), (k, 1))
    raw_sc = np.tile(np.concatenate([np.log(s), [0]])[None].astype(np.float32), (k, 1))
    raw_q = np.tile(q[None].astype(np.float32), (k, 1))
    normals = np.random.default_rng(9).standard_normal((k, 6))
    o = dict(OPTS, split_scale=0.0, max_scale=10.0, min_density=0.0, min_log_scale=-30.0)
    out = D.densify(raw_mr, raw_sc, raw_q, np.zeros((k, 3, 4)), np.zeros((k, 3, 4)),
                    np.ones(k, np.float32), np.ones(k), normals, o)
    off = out[0][:, :3] - raw_mr[0, :3].astype(np.float64)
    R = oracle.rotation(raw_q[0].astype(np.float64))
    s32 = np.exp(raw_sc[0, :3].astype(np.float64))
    Sigma = R @ np.diag(s32 ** 2) @ R.T
    C = off.T @ off / off.shape[0]
    assert np.abs(C - Sigma).max() <= 0.03 * np.abs(Sigma).max(), (C, Sigma)


def test_prune_rules_and_budget_selection():
    rng = np.random.default_rng(10)
    n = 500
    raw_mr, raw_sc, raw_q = _raw(n, 11)
    raw_mr[:40, 3] = D.inverse_softplus(np.full(40, 1e-4))      # too faint
    raw_sc[40:60, :3] = np.log(0.6)                              # too large
    stat = rng.random(n).astype(np.float32) * 4e-4
    vis = rng.integers(0, 4, n)
    for budget in (10 ** 9, n + 50, n - 60 + 5, n - 100):
        o = dict(OPTS, max_gaussians=budget)
        act, avg, cands = D.classify(raw_mr, raw_sc, stat, vis, o)
        assert np.all(act[:60] == D.PRUNE)
        kept = n - int((act == D.PRUNE).sum())
        dense = np.isin(act, (D.CLONE, D.SPLIT))
        eligible = (act != D.PRUNE) & (vis > 0) & (avg >= np.float32(2e-4))
        assert cands == int(eligible.sum())
        assert int(dense.sum()) == min(cands, max(budget - kept, 0))
        # every densified candidate ranks at or above every left-out candidate
        left = eligible & ~dense
        if dense.any() and left.any():
            assert avg[dense].min() >= avg[left].max()
        # split versus clone by the largest scale
        smax = np.exp(raw_sc[:, :3].astype(np.float64).max(1))
        assert np.all(smax[act == D.SPLIT] > 0.03) and np.all(smax[act == D.CLONE] <= 0.03)
        out = D.densify(raw_mr, raw_sc, raw_q, np.zeros((n, 3, 4)), np.zeros((n, 3, 4)), stat,
                        vis, rng.standard_normal((n, 6)), o)
        assert out[0].shape[0] == kept + int(dense.sum())


def test_everything_pruned_and_empty():
    n = 10
    raw_mr, raw_sc, raw_q = _raw(n, 12)
    o = dict(OPTS, min_density=1e9)
    out = D.densify(raw_mr, raw_sc, raw_q, np.zeros((n, 3, 4)), np.zeros((n, 3, 4)),
                    np.ones(n, np.float32), np.ones(n), np.zeros((n, 6)), o)
    assert out[0].shape == (0, 4) and np.all(out[5] == D.PRUNE)
    e = D.densify(raw_mr[:0], raw_sc[:0], raw_q[:0], np.zeros((0, 3, 4)), np.zeros((0, 3, 4)),
                  np.zeros(0, np.float32), np.zeros(0), np.zeros((0, 6)), OPTS)
    assert e[0].shape == (0, 4)


def test_inherit_moments_copies_the_parent_moments_to_every_child():
    n = 30
    raw_mr, raw_sc, raw_q = _raw(n, 13)
    m = np.random.default_rng(5).random((n, 3, 4))
    v = np.random.default_rng(6).random((n, 3, 4))
    normals = np.random.default_rng(7).standard_normal((n, 6))
    for split_scale, kind in ((0.0, D.SPLIT), (10.0, D.CLONE)):
        o = dict(OPTS, split_scale=split_scale, max_scale=10.0, min_density=0.0,
                 inherit_moments=1)
        out = D.densify(raw_mr, raw_sc, raw_q, m, v, np.ones(n, np.float32), np.ones(n),
                        normals, o)
        assert np.all(out[5] == kind)
        for k in (0, 1):
            np.testing.assert_array_equal(out[3][k::2], m)
            np.testing.assert_array_equal(out[4][k::2], v)
        # the parameters do not depend on the moment rule
        base = D.densify(raw_mr, raw_sc, raw_q, m, v, np.ones(n, np.float32), np.ones(n),
                         normals, dict(o, inherit_moments=0))
        for a, b in zip(out[:3], base[:3]):
            np.testing.assert_array_equal(a, b)
