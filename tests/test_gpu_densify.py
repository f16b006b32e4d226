"""Adaptive density control on the GPU against the FP64 reference (oracle/densify.py): the
statistics the backward accumulates, and the prune / clone / split kernel."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import densify as OD
from tests.helpers import REL_BAND, px_band, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsct():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300 import build

    build.build()
    return g


def _stats_case(seed=40, n=400, nv=3, W=40, H=36):
    mr, sc, qt = synth.gaussians(seed, n, radius=0.7, scale_median=0.03)
    return mr, sc, qt, synth.cone_views(nv, W, H), W, H


@pytest.mark.parametrize("chunked", [False, True])
def test_stats_match_oracle(orc, gsct, chunked, monkeypatch):
    import torch

    from paper_2604_01844_gb300 import projector as P

    mr, sc, qt, views, W, H = _stats_case()
    d = to_dev(mr, sc, qt)
    if chunked:
        pairs = gsct.Projector(views, W, H).count_pairs(*d)
        # room for about half the pairs per call (with the projector's headroom): 2+ chunks
        monkeypatch.setattr(P, "MAX_PAIRS_PER_CALL", int(pairs * 1.5 * 0.5) + 1024 + 64)
    pj = gsct.Projector(views, W, H)
    img = pj.forward(*d)
    assert (pj.chunks is not None) == chunked
    w = np.random.default_rng(3).standard_normal(img.shape)
    n = mr.shape[0]
    stat = torch.zeros(n, dtype=torch.float32, device="cuda")
    vis = torch.zeros(n, dtype=torch.int32, device="cuda")
    dimg = torch.from_numpy(w.astype(np.float32)).cuda()
    for _ in range(2):  # accumulates over calls
        pj.backward(*d, dimg, stats=(stat, vis))
    P64, V64 = orc.params64(mr, sc, qt), orc.views64(views)
    fp = orc.footprints(P64, V64, W, H)
    _, _, counts = orc.keys(P64, V64, W, H, 16)
    want_s, want_v = OD.grad_stats(fp, w.astype(np.float32).astype(np.float64), counts, W, H)
    flags = orc.pair_flags(P64, V64, W, H, REL_BAND, px_band(W, H), tile=16)
    clean = ~(flags != 0).any(axis=0)
    assert clean.mean() > 0.85
    got_s, got_v = stat.cpu().numpy().astype(np.float64), vis.cpu().numpy()
    assert np.array_equal(got_v[clean], 2 * want_v[clean])
    scale = np.abs(want_s).max()
    assert scale > 0
    err = np.abs(got_s[clean] - 2 * want_s[clean])
    assert np.all(err <= 1e-3 * (2 * want_s[clean]) + 1e-5 * 2 * scale), float(err.max())


OPTS = dict(grad_threshold=2e-4, grad_scale=3.0, split_scale=0.03, split_factor=1.6,
            min_density=2e-3, max_scale=0.3, min_log_scale=float(np.log(1e-4)),
            max_gaussians=10 ** 9)


def _random_state(seed, n):
    rng = np.random.default_rng(seed)
    mr, sc, qt = synth.gaussians(seed, n, radius=0.6, scale_median=0.03)
    raw_mr = mr.astype(np.float64).copy()
    raw_mr[:, 3] = OD.inverse_softplus(mr[:, 3])
    k = n // 10
    raw_mr[:k, 3] = OD.inverse_softplus(rng.uniform(1e-5, 1e-3, k))      # faint: pruned
    raw_sc = np.zeros((n, 4))
    raw_sc[:, :3] = np.log(sc[:, :3])
    raw_sc[k:k + k // 2, :3] = np.log(rng.uniform(0.35, 0.5, (k // 2, 3)))  # oversized
    stat = (rng.random(n) * 3e-4).astype(np.float32)
    vis = rng.integers(0, 4, n).astype(np.int32)
    m = rng.standard_normal((n, 3, 4)).astype(np.float32)
    v = rng.random((n, 3, 4)).astype(np.float32)
    normals = rng.standard_normal((n, 6)).astype(np.float32)
    return (raw_mr.astype(np.float32), raw_sc.astype(np.float32), qt.astype(np.float32), m, v,
            stat, vis, normals)


def _margins_clear(raw_mr, raw_sc, stat, vis, o):
    """No decision within a relative 1e-5 of its threshold (FP32 transcendental rounding)."""
    rho = OD.optim.softplus(raw_mr[:, 3].astype(np.float64))
    smax = np.exp(raw_sc[:, :3].astype(np.float64).max(1))
    avg = np.where(vis > 0, stat.astype(np.float64) / np.maximum(vis, 1), 0) * o["grad_scale"]
    near = lambda x, t: np.abs(x - t) <= 1e-5 * abs(t)  # noqa: E731
    return not (near(rho, o["min_density"]).any() or near(smax, o["max_scale"]).any() or
                near(smax, o["split_scale"]).any() or near(avg, o["grad_threshold"]).any())


def _gpu_densify(gsct, state, o, cap=None):
    import torch

    from paper_2604_01844_gb300 import binding as B

    raw_mr, raw_sc, raw_q, m, v, stat, vis, normals = state
    n = raw_mr.shape[0]
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
           for a in (raw_mr, raw_sc, raw_q, m.reshape(-1, 4), v.reshape(-1, 4), stat, vis,
                     normals)]
    opts = B.GsDensifyOpts()
    for k, val in o.items():
        setattr(opts, k, val)
    if cap is None:
        cap = min(2 * n, max(n, o["max_gaussians"]))
    out = [torch.full((max(cap, 1), 4), -7.0, device="cuda") for _ in range(3)]
    om = torch.full((3 * max(cap, 1), 4), -7.0, device="cuda")
    ov = torch.full_like(om, -7.0)
    ws = torch.empty(max(B.lib().gs_densify_workspace_size(n), 256), dtype=torch.uint8,
                     device="cuda")
    B.check(B.lib().gs_densify(*[B.ptr(t) for t in dev], n, ctypes.byref(opts),
                               *[B.ptr(t) for t in out], B.ptr(om), B.ptr(ov), cap, B.ptr(ws),
                               ws.numel(), B.stream_handle()), "gs_densify")
    st = B.read_status(ws)
    k = int(st.pairs)
    res = [t.cpu().numpy() for t in out] + [om.cpu().numpy().reshape(-1, 3, 4),
                                            ov.cpu().numpy().reshape(-1, 3, 4)]
    return res, k, st


def _compare(got, k, want):
    g_mr, g_sc, g_q, g_m, g_v = [a[:k] for a in got]
    w_mr, w_sc, w_q, w_m, w_v = want[:5]
    assert k == w_mr.shape[0]
    np.testing.assert_array_equal(g_q, w_q.astype(np.float32))
    np.testing.assert_array_equal(g_m, w_m.astype(np.float32))
    np.testing.assert_array_equal(g_v, w_v.astype(np.float32))
    np.testing.assert_allclose(g_sc, w_sc, rtol=0, atol=2e-6)
    np.testing.assert_allclose(g_mr[:, :3], w_mr[:, :3], rtol=0, atol=2e-6)
    # densities compared activated (the raw inverse softplus is ill-conditioned near 0)
    sp = OD.optim.softplus
    np.testing.assert_allclose(sp(g_mr[:, 3].astype(np.float64)), sp(w_mr[:, 3]), rtol=2e-6,
                               atol=1e-9)


@pytest.mark.parametrize("budget,inherit", [(None, 0), ("binding", 0), ("zero", 0),
                                             (None, 1), ("binding", 1)])
def test_densify_matches_oracle(gsct, budget, inherit):
    n = 3000
    state = _random_state(50, n)
    o = dict(OPTS, inherit_moments=inherit)
    act0, _, cands0 = OD.classify(state[0], state[1], state[5], state[6], o)
    kept = n - int((act0 == OD.PRUNE).sum())
    if budget == "binding":
        o["max_gaussians"] = kept + cands0 // 3
    elif budget == "zero":
        o["max_gaussians"] = kept - 5
    assert _margins_clear(state[0], state[1], state[5], state[6], o)
    want = OD.densify(*state[:3], state[3].astype(np.float64), state[4].astype(np.float64),
                      state[5], state[6], state[7].astype(np.float64), o)
    act = want[5]
    got, k, st = _gpu_densify(gsct, state, o)
    assert st.code == 0
    assert int(st.reserved[0]) == int((act == OD.PRUNE).sum())
    assert int(st.reserved[1]) == int((act == OD.CLONE).sum())
    assert int(st.reserved[2]) == int((act == OD.SPLIT).sum())
    assert int(st.reserved[3]) == want[6]
    if budget == "binding":
        assert int((act >= OD.CLONE).sum()) == cands0 // 3
    if budget == "zero":
        assert int((act >= OD.CLONE).sum()) == 0
    assert int((act == OD.SPLIT).sum()) > 0 and int((act == OD.PRUNE).sum()) > 0 or \
        budget == "zero"
    _compare(got, k, want)


def test_densify_ties_rank_by_index(gsct):
    # equal statistics: the budget takes the lowest indices
    n = 600
    state = list(_random_state(51, n))
    state[5] = np.full(n, 1e-3, np.float32)
    state[6] = np.ones(n, np.int32)
    o = dict(OPTS, min_density=0.0, max_scale=10.0)
    o["max_gaussians"] = n + 37
    want = OD.densify(*state[:3], state[3].astype(np.float64), state[4].astype(np.float64),
                      state[5], state[6], state[7].astype(np.float64), o)
    assert np.all(want[5][:37] >= OD.CLONE) and np.all(want[5][37:] == OD.KEEP)
    got, k, st = _gpu_densify(gsct, state, o)
    assert k == n + 37
    _compare(got, k, want)


def test_densify_capacity_error_writes_nothing(gsct):
    n = 500
    state = _random_state(52, n)
    o = dict(OPTS, min_density=0.0, max_scale=10.0, grad_threshold=0.0)
    got, k, st = _gpu_densify(gsct, state, o, cap=n)
    assert st.code == -2 and k > n
    assert np.all(got[0] == -7.0) and np.all(got[3] == -7.0)


def test_densify_all_pruned_and_empty(gsct):
    n = 300
    state = _random_state(53, n)
    got, k, st = _gpu_densify(gsct, state, dict(OPTS, min_density=1e9))
    assert st.code == 0 and k == 0 and int(st.reserved[0]) == n
    empty = tuple(a[:0] for a in state)
    got, k, st = _gpu_densify(gsct, empty, OPTS, cap=0)
    assert st.code == 0 and k == 0


def test_reconstruction_with_density_control(gsct):
    """A reconstruction that densifies on schedule: the Gaussian set changes as counted, stays
    within the budget, and the loss keeps falling through the re-plans and graph captures."""
    import torch

    from paper_2604_01844_gb300.density import DensifyConfig, DensityControl
    from paper_2604_01844_gb300.evaluate import VolumeScore, trajectory
    from paper_2604_01844_gb300.recon import (PhantomProblem, ReconConfig, Reconstruction,
                                               fdk_volume, gradient_init)

    views = synth.cone_views(16, 64, 64)
    grid = synth.cube_grid(48)
    prob = PhantomProblem(synth.ellipsoid_phantom(90, 10), views, 64, 64, grid)
    u = np.random.default_rng(5).random((1500, 4)).astype(np.float32)
    mr, sc, q = gradient_init(fdk_volume(prob, grid), grid, 1500, u)
    rec = Reconstruction(views, 64, 64, prob.proj.clone(), grid, mr.cpu().numpy(),
                         sc.cpu().numpy(), q.cpu().numpy(), cfg=ReconConfig(lr_mean=1e-3,
                                                                           lr_rho=2e-2))
    # threshold 0: every visible Gaussian is a candidate, so the budget decides (top by stat)
    ctrl = DensityControl(rec, DensifyConfig(start=10, interval=10, stop=40, max_gaussians=2600,
                                             grad_threshold=0.0, seed=3))
    score = VolumeScore(prob.gt, prob.peak)
    traj, replans = trajectory(rec, score, 50, eval_every=10, ssim=False, graph=True,
                               control=ctrl)
    assert [h["iteration"] for h in ctrl.history] == [10, 20, 30]
    for h in ctrl.history:
        assert h["n_after"] == h["n_before"] - h["pruned"] + h["cloned"] + h["split"]
        assert h["n_after"] <= 2600 and h["candidates"] > 0
    assert ctrl.history[0]["n_after"] == 2600
    assert rec.n == ctrl.history[-1]["n_after"] and rec.n > 1500
    assert all(np.isfinite(r[2]) for r in traj)
    assert traj[-1][2] > traj[0][2] + 1.0, traj
    assert torch.isfinite(rec.loss).all()
