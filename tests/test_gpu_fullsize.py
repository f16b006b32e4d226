"""Full-size parity on sampled outputs, in the launch configurations the benchmark times
(all 75 views; tile 16, and tile 32 where the autotuner picks it): the rasterizer at 75 cone views of 512^2 (50k Gaussians), 1024^2
(200k) and 2048^2 (500k), the voxelizer at 1024^3 (500k), each against the FP64 oracle
evaluated output by output with the same per-output guard-band allowance as the small tests
(1e-4 of the peak plus the contributions of pairs within the band of the cut or a box edge);
and the per-Gaussian gradient of sampled Gaussians at 512^2 and 1024^2 against the oracle's
dual-number gradient (a Gaussian's gradient needs only its own footprint, so the oracle runs
on the sampled Gaussians alone against the full dL/dI); the voxelizer's
per-Gaussian gradient at 1024^3 (the oracle on a region holding each sampled Gaussian's box);
the fused 3D SSIM's gradient at sampled voxels of a 1024^3 volume, the step's L1 + D-SSIM
gradient at sampled pixels of 75 views of 512^2 and TV at 512^3, against the oracle on a crop
around each."""
import numpy as np
import pytest
import torch

import synth
from tests.helpers import IMG_TOL, REL_BAND, assert_grads_close, grads11, px_band, to_dev

pytestmark = pytest.mark.gpu

IDX_BAND = 2e-4
N_SAMPLES = 1200


@pytest.fixture(scope="module")
def gsct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300 import build

    build.build()
    return g


def _gather(t, idx):
    ix = [torch.from_numpy(idx[:, k]).long().to(t.device) for k in range(3)]
    return t[ix[0], ix[1], ix[2]].cpu().numpy().astype(np.float64)


def _check(got, want, allow, min_nonzero=0.3):
    peak = float(np.abs(want).max())
    assert peak > 0 and (want != 0).mean() > min_nonzero
    bound = IMG_TOL * peak + allow
    err = np.abs(got - want)
    assert (err <= bound).all(), (float((err / bound).max()), int((err > bound).sum()))


# tile 16 at 512^2 (the reconstruction step's tile), 16 and 32 (the autotuner's pick for the
# 1024^2 and 2048^2 steps) at the larger detectors
@pytest.mark.parametrize("side,n,median,tile", [(512, 50000, 0.012, 16),
                                                (1024, 200000, 0.008, 16),
                                                (1024, 200000, 0.008, 32),
                                                (2048, 500000, 0.006, 16),
                                                (2048, 500000, 0.006, 32)])
def test_raster_full_size_sampled(orc, gsct, side, n, median, tile):
    mr, sc, qt = synth.gaussians(40 + side, n, radius=0.8, scale_median=median,
                                 scale_sigma_log=0.4)
    views = synth.cone_views(75, side, side)
    proj = gsct.Projector(views, side, side, tile=tile)
    img = proj.forward(*to_dev(mr, sc, qt))
    assert proj.status().code == 0
    pix = synth.pixel_samples(side, 75, side, side, N_SAMPLES)
    got = _gather(img, pix)
    del img, proj
    torch.cuda.empty_cache()
    P, V = orc.params64(mr, sc, qt), orc.views64(views)
    want, allow = orc.project_pixels_allow(P, V, side, side, pix, REL_BAND, px_band(side, side))
    _check(got, want, allow)


def test_voxelize_1024_sampled(orc, gsct):
    n = 500000
    mr, sc, qt = synth.gaussians(77, n, scale_median=0.004, scale_sigma_log=0.4)
    grid = synth.cube_grid(1024)
    d = to_dev(mr, sc, qt)
    vox = gsct.Voxelizer(grid)
    vol = vox.forward(*d)
    assert vox.status().code == 0
    idx = synth.voxel_samples(5, (1024, 1024, 1024), N_SAMPLES)
    got = _gather(vol, idx)
    # the 64-voxel bricks give the same volume bit for bit at full size
    vox64 = gsct.Voxelizer(grid, brick=64)
    assert torch.equal(vox64.forward(*d), vol)
    del vol, vox, vox64
    torch.cuda.empty_cache()
    want, allow = orc.voxelize_points_allow(orc.params64(mr, sc, qt), grid, idx, REL_BAND,
                                            IDX_BAND)
    _check(got, want, allow, min_nonzero=0.15)


# the 1024^2 step also runs at tile 32 with its lists rebuilt in the backward
@pytest.mark.parametrize("side,n,median,tile,reuse", [(512, 50000, 0.012, 16, True),
                                                      (1024, 200000, 0.008, 16, True),
                                                      (1024, 200000, 0.008, 32, False)])
def test_raster_gradients_full_size_sampled(orc, gsct, side, n, median, tile, reuse):
    mr, sc, qt = synth.gaussians(60 + side, n, radius=0.8, scale_median=median,
                                 scale_sigma_log=0.4)
    views = synth.cone_views(75, side, side)
    rng = np.random.default_rng(side)
    w = rng.standard_normal((75, side, side), dtype=np.float32)
    proj = gsct.Projector(views, side, side, tile=tile)
    d = to_dev(mr, sc, qt)
    proj.forward(*d)
    got = grads11(*proj.backward(*d, torch.from_numpy(w).cuda(), reuse=reuse))
    assert proj.status().code == 0
    del proj
    torch.cuda.empty_cache()
    # 200 sampled Gaussians with no guard-band pair in any of the 75 views (the oracle's
    # flags alone decide; with 75 views one Gaussian in 7 (512^2) to 55 (1024^2) has none)
    cand = np.sort(rng.choice(n, 30000, replace=False))
    V = orc.views64(views)
    flags = orc.pair_flags(orc.params64(mr, sc, qt)[cand], V, side, side, REL_BAND,
                           px_band(side, side))
    clean = cand[~(flags != 0).any(axis=0)]
    assert len(clean) >= 200, len(clean)
    sel = clean[:200]
    want = orc.project_grad(orc.params64(mr, sc, qt)[sel], V, side, side, w)
    assert_grads_close(got[sel], want, np.ones(len(sel), dtype=bool))


def _sweep_gaussians(n):
    import bench

    return synth.gaussians(5, n, radius=0.8, scale_median=bench.SWEEP_SCALE, scale_sigma_log=0.0,
                           isotropic=True, identity_rotation=True)


def test_kernel_sweep_largest_points_sampled(orc, gsct):
    """The kernel micro-benchmark's largest points (identity rotations, one isotropic scale):
    one cone view of 2048^2 and a 1024^3 volume of 20k Gaussians, sampled outputs against the
    oracle; and the per-Gaussian gradient of 200 sampled Gaussians at its 1024^2 view of 320k
    Gaussians (the rotation gradient of an isotropic Gaussian vanishes: rounding noise only)."""
    import bench

    mr, sc, qt = _sweep_gaussians(bench.SWEEP_N)
    P = orc.params64(mr, sc, qt)
    side = max(bench.SWEEP_SIDES)
    views = synth.cone_views(1, side, side)
    proj = gsct.Projector(views, side, side, tile=16)
    img = proj.forward(*to_dev(mr, sc, qt))
    assert proj.status().code == 0
    pix = synth.pixel_samples(9, 1, side, side, N_SAMPLES)
    got = _gather(img, pix)
    del img, proj
    want, allow = orc.project_pixels_allow(P, orc.views64(views), side, side, pix, REL_BAND,
                                           px_band(side, side))
    _check(got, want, allow, min_nonzero=0.2)

    vs = max(bench.SWEEP_VOL_SIDES)
    grid = synth.cube_grid(vs)
    vox = gsct.Voxelizer(grid)
    vol = vox.forward(*to_dev(mr, sc, qt))
    assert vox.status().code == 0
    idx = synth.voxel_samples(9, (vs, vs, vs), N_SAMPLES)
    got = _gather(vol, idx)
    del vol, vox
    torch.cuda.empty_cache()
    want, allow = orc.voxelize_points_allow(P, grid, idx, REL_BAND, IDX_BAND)
    _check(got, want, allow, min_nonzero=0.05)

    n = max(bench.SWEEP_COUNTS)
    mr, sc, qt = _sweep_gaussians(n)
    side = bench.SWEEP_PX_SIDE
    views = synth.cone_views(1, side, side)
    rng = np.random.default_rng(3)
    w = rng.standard_normal((1, side, side), dtype=np.float32)
    proj = gsct.Projector(views, side, side, tile=16)
    d = to_dev(mr, sc, qt)
    proj.forward(*d)
    got = grads11(*proj.backward(*d, torch.from_numpy(w).cuda(), reuse=True))
    assert proj.status().code == 0
    del proj
    torch.cuda.empty_cache()
    V = orc.views64(views)
    cand = np.sort(rng.choice(n, 5000, replace=False))
    P = orc.params64(mr, sc, qt)
    flags = orc.pair_flags(P[cand], V, side, side, REL_BAND, px_band(side, side))
    clean = cand[~(flags != 0).any(axis=0)]
    assert len(clean) >= 200, len(clean)
    sel = clean[:200]
    want = orc.project_grad(P[sel], V, side, side, w)
    # rotating an isotropic Gaussian changes nothing, so dL/dq vanishes (the oracle's is exactly
    # 0); the FP32 chain leaves rounding noise of order 1e-7 |dL/ds| s, bounded here by 1e-3 of
    # the scale gradient's rms times the scale, and the other groups keep the usual tolerance
    assert (want[:, 6:10] == 0).all()
    rms_s = np.sqrt(np.mean(want[:, 3:6] ** 2))
    assert np.abs(got[sel][:, 6:10]).max() <= 1e-3 * rms_s * bench.SWEEP_SCALE
    g = got[sel].copy()
    g[:, 6:10] = 0.0
    assert_grads_close(g, want, np.ones(len(sel), dtype=bool))


def test_ssim3d_1024_sampled_gradient(gsct):
    """The fused streaming 3D SSIM in the launch configuration of the 1024^3 volume fit: its
    gradient at sampled interior voxels against the oracle's SSIM on the 21^3 crop around each
    voxel (every voxel whose SSIM window holds the sampled one has its own window inside the
    crop, so the crop's gradient there is the full volume's times the voxel-count ratio); and
    the value at y = x, where every SSIM term is 1."""
    from oracle import losses as OL
    from paper_2604_01844_gb300 import binding as B

    n, weight = 1024, 0.25
    rng = np.random.default_rng(31)
    y = rng.random((n, n, n), dtype=np.float32)
    x = np.clip(y + 0.1 * rng.standard_normal((n, n, n), dtype=np.float32), 0, None)
    L = float(y.max())
    L_ = B.lib()
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ws = torch.empty(L_.gs_ssim3d_workspace_size(n ** 3), dtype=torch.uint8, device="cuda")
    loss = torch.zeros(1, device="cuda")
    grad = torch.empty_like(xd)
    s = torch.cuda.current_stream().cuda_stream
    B.check(L_.gs_ssim3d_loss(B.ptr(xd), B.ptr(yd), n, n, n, L, weight, B.ptr(loss), B.ptr(grad),
                              0, B.ptr(ws), ws.numel(), s), "gs_ssim3d_loss")
    same = torch.zeros(1, device="cuda")
    B.check(L_.gs_ssim3d_loss(B.ptr(xd), B.ptr(xd), n, n, n, L, weight, B.ptr(same), None, 0,
                              B.ptr(ws), ws.numel(), s), "gs_ssim3d_loss")
    torch.cuda.synchronize()
    assert abs(float(same.item())) <= 1e-5 * weight
    pts = rng.integers(10, n - 10, size=(16, 3))
    got = grad[torch.from_numpy(pts[:, 0]).cuda(), torch.from_numpy(pts[:, 1]).cuda(),
               torch.from_numpy(pts[:, 2]).cuda()].cpu().numpy().astype(np.float64)
    del xd, yd, ws, grad
    torch.cuda.empty_cache()
    want = np.empty(len(pts))
    ratio = 21.0 ** 3 / float(n) ** 3
    for k, (z, yy, xx) in enumerate(pts):
        cx = x[z - 10:z + 11, yy - 10:yy + 11, xx - 10:xx + 11].astype(np.float64)
        cy = y[z - 10:z + 11, yy - 10:yy + 11, xx - 10:xx + 11].astype(np.float64)
        _, g = OL.value_and_grad(lambda a, b: -weight * ratio * OL.ssim3d(a, b, L), cx, cy)
        want[k] = g[10, 10, 10]
    scale = np.abs(want).max()
    assert scale > 0
    assert np.abs(got - want).max() <= 1e-3 * scale, float(np.abs(got - want).max() / scale)
    big = np.abs(want) > 0.1 * scale
    assert (np.abs(got - want)[big] <= 1e-2 * np.abs(want[big])).all()


def test_l1_ssim2d_75x512_sampled_gradient(gsct):
    """The reconstruction step's image loss (L1 + D-SSIM over 75 views of 512^2, TMA-staged
    kernels): the gradient at sampled interior pixels against the oracle's SSIM on the 21^2
    crop around each (scaled by the pixel-count ratio) plus the L1 term's sign gradient."""
    from oracle import losses as OL
    from paper_2604_01844_gb300 import binding as B

    nv, n, l1w, sw = 75, 512, 0.8, 0.2
    rng = np.random.default_rng(41)
    y = rng.random((nv, n, n), dtype=np.float32)
    x = np.clip(y + 0.1 * rng.standard_normal((nv, n, n), dtype=np.float32), 0, None)
    L = float(y.max())
    L_ = B.lib()
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ws = torch.empty(L_.gs_ssim_workspace_size(x.size), dtype=torch.uint8, device="cuda")
    loss = torch.zeros(1, device="cuda")
    grad = torch.empty_like(xd)
    B.check(L_.gs_l1_ssim2d_loss(B.ptr(xd), B.ptr(yd), nv, n, n, L, l1w, sw, B.ptr(loss),
                                 B.ptr(grad), 0, B.ptr(ws), ws.numel(),
                                 torch.cuda.current_stream().cuda_stream), "gs_l1_ssim2d_loss")
    torch.cuda.synchronize()
    pts = np.stack([rng.integers(0, nv, 64), rng.integers(10, n - 10, 64),
                    rng.integers(10, n - 10, 64)], axis=1)
    got = grad[torch.from_numpy(pts[:, 0]).cuda(), torch.from_numpy(pts[:, 1]).cuda(),
               torch.from_numpy(pts[:, 2]).cuda()].cpu().numpy().astype(np.float64)
    N = float(x.size)
    want = np.empty(len(pts))
    for k, (v, yy, xx) in enumerate(pts):
        cx = x[v:v + 1, yy - 10:yy + 11, xx - 10:xx + 11].astype(np.float64)
        cy = y[v:v + 1, yy - 10:yy + 11, xx - 10:xx + 11].astype(np.float64)
        _, g = OL.value_and_grad(lambda a, b: -sw * (21.0 ** 2 / n ** 2 / nv) * OL.ssim2d(a, b, L),
                                 cx, cy)
        want[k] = g[0, 10, 10] + l1w * np.sign(float(x[v, yy, xx]) - float(y[v, yy, xx])) / N
    scale = np.abs(want).max()
    assert scale > 0
    assert np.abs(got - want).max() <= 1e-3 * scale, float(np.abs(got - want).max() / scale)
    big = np.abs(want) > 0.1 * scale
    assert (np.abs(got - want)[big] <= 1e-2 * np.abs(want[big])).all()


def test_tv3d_512_value_and_sampled_gradient(gsct):
    """TV on the 512^3 volume of the 1024^2 step: the value against the oracle's FP64 sum, the
    sub-gradient at sampled interior voxels against the oracle on the 3^3 crop around each
    (every difference that involves the voxel lies inside it)."""
    from oracle import losses as OL
    from paper_2604_01844_gb300 import binding as B

    n, weight = 512, 0.05
    rng = np.random.default_rng(51)
    v = rng.random((n, n, n), dtype=np.float32)
    vd = torch.from_numpy(v).cuda()
    loss = torch.zeros(1, device="cuda")
    grad = torch.empty_like(vd)
    B.check(B.lib().gs_tv3d_loss(B.ptr(vd), n, n, n, weight, B.ptr(loss), B.ptr(grad), 0,
                                 torch.cuda.current_stream().cuda_stream), "gs_tv3d_loss")
    torch.cuda.synchronize()
    want_v = weight * float(OL.tv3d(torch.from_numpy(v.astype(np.float64))))
    # FP32 partial sums of about a thousand differences per thread, then block sums and atomics
    assert abs(float(loss.item()) - want_v) <= 1e-4 * abs(want_v)
    pts = rng.integers(1, n - 1, size=(64, 3))
    got = grad[torch.from_numpy(pts[:, 0]).cuda(), torch.from_numpy(pts[:, 1]).cuda(),
               torch.from_numpy(pts[:, 2]).cuda()].cpu().numpy().astype(np.float64)
    want = np.empty(len(pts))
    for k, (z, y, x) in enumerate(pts):
        c = v[z - 1:z + 2, y - 1:y + 2, x - 1:x + 2].astype(np.float64)
        _, g = OL.value_and_grad(lambda a: weight * (27.0 / n ** 3) * OL.tv3d(a), c)
        want[k] = g[1, 1, 1]
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6 * np.abs(want).max())


def test_voxelize_backward_1024_sampled(orc, gsct):
    """The voxelizer backward in the 1024^3 volume fit's configuration (500k Gaussians, 16-voxel
    bricks, the forward's lists reused): the (N, 11) gradient of 100 sampled Gaussians outside
    the guard band against the oracle's, each computed on a region of interest that holds the
    Gaussian's whole 3-sigma box (so that it sees exactly the dL/dV the full volume gives it)."""
    n, side = 500000, 1024
    mr, sc, qt = synth.gaussians(77, n, scale_median=0.004, scale_sigma_log=0.4)
    grid = synth.cube_grid(side)
    rng = np.random.default_rng(61)
    w = rng.standard_normal((side, side, side), dtype=np.float32)
    vox = gsct.Voxelizer(grid)
    d = to_dev(mr, sc, qt)
    vox.forward(*d)
    got = grads11(*vox.backward(*d, torch.from_numpy(w).cuda(), reuse=True))
    assert vox.status().code == 0
    del vox
    torch.cuda.empty_cache()
    P = orc.params64(mr, sc, qt)
    cand = np.sort(rng.choice(n, 400, replace=False))
    flags = orc.voxel_flags(P[cand], grid, (0, 0, 0), (side, side, side), REL_BAND, IDX_BAND)
    sel = cand[flags == 0][:100]
    assert len(sel) == 100
    o, h = float(np.ravel(grid["origin"])[0]), float(np.ravel(grid["voxel"])[0])
    want = np.empty((len(sel), 11))
    for k, i in enumerate(sel):
        r = 3.05 * float(sc[i, :3].max())  # the 3-sigma ellipsoid lies in this ball
        lo = np.clip(np.floor((mr[i, :3] - r - o) / h - 1.0).astype(int), 0, side)
        hi = np.clip(np.ceil((mr[i, :3] + r - o) / h + 1.0).astype(int), 0, side)
        dim = hi - lo
        crop = w[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        want[k] = orc.voxelize_grad(P[i:i + 1], grid, crop, roi_lo=tuple(int(a) for a in lo),
                                    roi_dim=tuple(int(a) for a in dim))[0]
    assert_grads_close(got[sel], want, np.ones(len(sel), dtype=bool))
