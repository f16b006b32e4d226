"""Prior-volume warm start: a Gaussian set fitted to a prior volume (gs_fit_volume) starts the
projection-domain reconstruction, and the value-only 3D SSIM used to score it."""
import numpy as np
import pytest
import torch

import synth
from oracle import losses as OL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300 import build

    build.build()
    return g


def test_value_only_ssim3d_matches_oracle_and_full_call(gsct):
    from paper_2604_01844_gb300.warmstart import VolumeScore

    rng = np.random.default_rng(11)
    y = rng.random((19, 23, 30)).astype(np.float32)
    x = np.clip(y + 0.1 * rng.standard_normal(y.shape), 0, None).astype(np.float32)
    sc = VolumeScore(torch.from_numpy(y).cuda(), peak=float(y.max()))
    got = sc.ssim(torch.from_numpy(x).cuda())
    want = float(OL.ssim3d(torch.from_numpy(x.astype(np.float64)),
                           torch.from_numpy(y.astype(np.float64)), float(y.max())))
    assert abs(got - want) <= 2e-5, (got, want)
    # the same value as the loss call that also writes the gradient
    B = gsct.binding
    L = B.lib()
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    loss = torch.zeros(1, device="cuda")
    grad = torch.empty_like(xd)
    ws = torch.empty(L.gs_ssim3d_workspace_size(xd.numel()), dtype=torch.uint8, device="cuda")
    B.check(L.gs_ssim3d_loss(B.ptr(xd), B.ptr(yd), 30, 23, 19, float(y.max()), 1.0, B.ptr(loss),
                             B.ptr(grad), 0, B.ptr(ws), ws.numel(), B.stream_handle()), "ssim3d")
    assert abs((1.0 - float(loss.item())) - got) <= 1e-6
    # neither a gradient nor a loss: rejected
    assert L.gs_ssim3d_loss(B.ptr(xd), B.ptr(yd), 30, 23, 19, 1.0, 1.0, None, None, 0, B.ptr(ws),
                            ws.numel(), B.stream_handle()) == B.GS_ERR_ARG


def _problem(gsct, seed=80, nv=16, det=64, side=48):
    from paper_2604_01844_gb300.recon import PhantomProblem

    views = synth.cone_views(nv, det, det)
    grid = synth.cube_grid(side)
    return PhantomProblem(synth.ellipsoid_phantom(seed, 10), views, det, det, grid), views, grid


def test_warm_start_from_thick_slice_prior(gsct):
    """The fitted prior is a better start than FDK-gradient sampling from sparse views, the
    reconstruction starts exactly from the fitted Gaussians, and it keeps improving."""
    from paper_2604_01844_gb300.recon import (ReconConfig, Reconstruction, fdk_volume,
                                               gradient_init)
    from paper_2604_01844_gb300.warmstart import VolumeScore, fit_prior, trajectory

    prob, views, grid = _problem(gsct)
    n = 2000
    prior = torch.from_numpy(synth.thick_slices(prob.gt.cpu().numpy(), 5)).cuda()
    u = torch.from_numpy(np.random.default_rng(3).random((n, 4)).astype(np.float32)).cuda()
    (mr, sc, q), fit = fit_prior(prior, grid, n, 40, u)
    assert fit.status().code == gsct.binding.GS_OK
    score = VolumeScore(prob.gt, prob.peak)
    fitted_vol = gsct.Voxelizer(grid).forward(mr, sc, q).clone()
    cfg = ReconConfig(lr_mean=1e-3, lr_rho=2e-2)
    warm = Reconstruction(views, 64, 64, prob.proj.clone(), grid, mr.cpu().numpy(),
                          sc.cpu().numpy(), q.cpu().numpy(), cfg=cfg)
    # the reconstruction's activated start reproduces the fitted set (raw -> activation round
    # trip in FP32), so its first volume is the fitted volume
    for a, b in zip(warm.act, (mr, sc, q)):
        torch.testing.assert_close(a, b, rtol=2e-5, atol=2e-6)
    v0 = warm.voxelizer.forward(*warm.act)
    assert float((v0 - fitted_vol).abs().max()) <= 1e-4 * float(fitted_vol.abs().max())

    u2 = np.random.default_rng(4).random((n, 4)).astype(np.float32)
    cmr, csc, cq = gradient_init(fdk_volume(prob, grid), grid, n, u2)
    cold = Reconstruction(views, 64, 64, prob.proj.clone(), grid, cmr.cpu().numpy(),
                          csc.cpu().numpy(), cq.cpu().numpy(), cfg=cfg)
    tw, rw = trajectory(warm, score, 20, eval_every=10, graph=True)
    tc, rc = trajectory(cold, score, 20, eval_every=10)
    assert rw == 0 and rc == 0
    assert tw[0][2] > tc[0][2] + 1.0, (tw, tc)    # the prior start is ahead at iteration 0
    assert tw[-1][2] > tw[0][2], tw                # and the projections still improve it
    assert tw[0][3] > tc[0][3], (tw, tc)
    assert all(r[1] >= 0 for r in tw) and tw[-1][1] > 0
