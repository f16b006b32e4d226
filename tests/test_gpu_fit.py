"""The volume fit (Sec. 3.6, Eq. 6) through gs_fit_volume.  The optimisation trajectory has no
closed form (parity unpinned); what is checked: the first iteration equals the composition of
the separately tested kernels, the loss falls, and the oracle's PSNR of the fitted Gaussians
(voxelized by the oracle itself) rises well above the initialisation's."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300 import build

    build.build()
    return g


def _problem(orc, n_side=40, n=3000, seed=0):
    grid = synth.cube_grid(n_side)
    ell = synth.ellipsoid_phantom(seed, 8)
    V = orc.phantom_voxelize(ell, grid).astype(np.float32)
    u = np.random.default_rng(seed).random((n, 4)).astype(np.float32)
    return grid, V, u


def test_fit_volume_improves_psnr(orc, gsct):
    from oracle import losses as OL
    from paper_2604_01844_gb300.fit import VolumeFit, fit_opts

    n = 3000
    grid, V, u = _problem(orc, n=n)
    dV, du = torch.from_numpy(V).cuda(), torch.from_numpy(u).cuda()
    f0 = VolumeFit(grid, n)
    p0 = [t.clone() for t in f0.run(dV, 0, fit_opts(), du)]  # initialisation only
    f = VolumeFit(grid, n)
    loss = torch.zeros(150, device="cuda")
    p = f.run(dV, 150, fit_opts(), du, loss)
    torch.cuda.synchronize()
    assert f.status().code == 0
    L = loss.cpu().numpy()
    assert L[-1] < 0.5 * L[0], (L[0], L[-1])
    Vt = torch.from_numpy(V.astype(np.float64))

    def psnr(params):
        P = orc.params64(*[t.cpu().numpy() for t in params])
        vol, _ = orc.voxelize(P, grid)
        return OL.psnr(torch.from_numpy(vol), Vt)

    a, b = psnr(p0), psnr(p)
    assert b > a + 5.0, (a, b)


def test_fit_first_iteration_is_the_composition(orc, gsct):
    """One iteration of gs_fit_volume from given parameters equals voxelize -> L1 + SSIM3D ->
    voxelizer backward -> Adam called one by one."""
    from paper_2604_01844_gb300.fit import VolumeFit, fit_opts
    from paper_2604_01844_gb300.recon import inverse_softplus

    B = gsct.binding
    n = 1000
    grid, V, u = _problem(orc, n_side=32, n=n, seed=1)
    mr, sc, qt = synth.gaussians(3, n, radius=0.6, scale_median=0.05)
    dV = torch.from_numpy(V).cuda()
    o = fit_opts(init=False, data_range=float(V.max()))
    f = VolumeFit(grid, n)
    for t, a in zip(f.params, (mr, sc, qt)):
        t.copy_(torch.from_numpy(a))
    f.run(dV, 1, o)
    got = [t.cpu().numpy() for t in f.params]
    # manual composition
    act = [torch.from_numpy(a).cuda() for a in (mr, sc, qt)]
    vox = gsct.Voxelizer(grid)
    vol = vox.forward(*act)
    loss = torch.zeros(1, device="cuda")
    dvol = torch.empty_like(vol)
    B.check(B.lib().gs_l1_loss(B.ptr(vol), B.ptr(dV), vol.numel(), 1.0, B.ptr(loss), B.ptr(dvol),
                               0, torch.cuda.current_stream().cuda_stream), "l1")
    ws = torch.empty(B.lib().gs_ssim3d_workspace_size(vol.numel()), dtype=torch.uint8, device="cuda")
    B.check(B.lib().gs_ssim3d_loss(B.ptr(vol), B.ptr(dV), 32, 32, 32, float(V.max()), o.alpha_ssim,
                                   B.ptr(loss), B.ptr(dvol), 1, B.ptr(ws), ws.numel(),
                                   torch.cuda.current_stream().cuda_stream), "ssim3d")
    g = vox.backward(*act, dvol)
    raw = [torch.from_numpy(np.concatenate([mr[:, :3], inverse_softplus(mr[:, 3])[:, None]], 1)
                            .astype(np.float32)).cuda(),
           torch.from_numpy(np.concatenate([np.log(sc[:, :3]), np.zeros((n, 1))], 1)
                            .astype(np.float32)).cuda(),
           torch.from_numpy(qt).cuda()]
    m = torch.zeros((3 * n, 4), device="cuda")
    v = torch.zeros_like(m)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    ao = B.GsAdamOpts()
    for k in ("lr_mean", "lr_rho", "lr_scale", "lr_quat", "beta1", "beta2", "eps",
              "min_log_scale", "max_log_scale"):
        setattr(ao, k, getattr(o, k))
    out = [torch.empty_like(t) for t in act]
    B.check(B.lib().gs_adam_step(*[B.ptr(t) for t in raw], B.ptr(m), B.ptr(v),
                                 *[B.ptr(t) for t in g], *[B.ptr(t) for t in out], n, B.ptr(step),
                                 ctypes.byref(ao), torch.cuda.current_stream().cuda_stream), "adam")
    for a, b in zip(got, out):
        np.testing.assert_allclose(a, b.cpu().numpy(), rtol=1e-5, atol=1e-6)
