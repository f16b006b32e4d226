"""Parity of the fused loss kernels (Eq. 5, Eq. 6) and the Adam step with the FP64 oracle."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import losses as OL
from oracle import optim as OO

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_01844_gb300 import binding, build

    build.build()
    return binding


def _s():
    return torch.cuda.current_stream().cuda_stream


def _run_loss(B, name, x, y, *extra, ws=None, weight=1.0, accumulate_into=None):
    L = B.lib()
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda() if y is not None else None
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros_like(xd) if accumulate_into is None else \
        torch.from_numpy(accumulate_into.astype(np.float32)).cuda()
    acc = 0 if accumulate_into is None else 1
    if name == "l1":
        rc = L.gs_l1_loss(B.ptr(xd), B.ptr(yd), xd.numel(), weight, B.ptr(loss), B.ptr(grad), acc, _s())
    elif name == "tv":
        dz, dy, dx = x.shape
        rc = L.gs_tv3d_loss(B.ptr(xd), dx, dy, dz, weight, B.ptr(loss), B.ptr(grad), acc, _s())
    elif name == "ssim2d":
        wsb = torch.empty(L.gs_ssim_workspace_size(xd.numel()), dtype=torch.uint8, device="cuda")
        n, H, W = x.shape
        rc = L.gs_ssim2d_loss(B.ptr(xd), B.ptr(yd), n, H, W, extra[0], weight, B.ptr(loss),
                              B.ptr(grad), acc, B.ptr(wsb), wsb.numel(), _s())
    elif name == "l1ssim2d":  # extra = (data range, L1 weight); weight = SSIM weight
        wsb = torch.empty(L.gs_ssim_workspace_size(xd.numel()), dtype=torch.uint8, device="cuda")
        n, H, W = x.shape
        rc = L.gs_l1_ssim2d_loss(B.ptr(xd), B.ptr(yd), n, H, W, extra[0], extra[1], weight,
                                 B.ptr(loss), B.ptr(grad), acc, B.ptr(wsb), wsb.numel(), _s())
    else:
        wsb = torch.empty(L.gs_ssim3d_workspace_size(xd.numel()), dtype=torch.uint8, device="cuda")
        dz, dy, dx = x.shape
        rc = L.gs_ssim3d_loss(B.ptr(xd), B.ptr(yd), dx, dy, dz, extra[0], weight, B.ptr(loss),
                              B.ptr(grad), acc, B.ptr(wsb), wsb.numel(), _s())
    B.check(rc, name)
    torch.cuda.synchronize()
    return float(loss.item()), grad.cpu().numpy().astype(np.float64)


def _x32(a):
    return a.astype(np.float32).astype(np.float64)


def test_l1(B):
    rng = np.random.default_rng(0)
    x, y = _x32(rng.standard_normal(100003)), _x32(rng.standard_normal(100003))
    val, g = _run_loss(B, "l1", x, y, weight=0.7)
    want, gw = OL.value_and_grad(lambda a, b: 0.7 * OL.l1(a, b), x, y)
    assert abs(val - want) <= 1e-5 * abs(want)
    np.testing.assert_allclose(g, gw, rtol=1e-6, atol=1e-12)
    val2, g2 = _run_loss(B, "l1", x, y, weight=0.7, accumulate_into=np.ones_like(x))
    np.testing.assert_allclose(g2, gw + 1.0, rtol=1e-6, atol=1e-7)


def test_tv3d(B):
    rng = np.random.default_rng(1)
    v = _x32(rng.random((13, 17, 20)))
    val, g = _run_loss(B, "tv", v, None, weight=0.3)
    want, gw = OL.value_and_grad(lambda a: 0.3 * OL.tv3d(a), v)
    assert abs(val - want) <= 1e-5 * abs(want)
    np.testing.assert_allclose(g, gw, rtol=1e-5, atol=1e-9)


# (3, 37, 53) and (1, 5, 7) take the register-staged kernels (width not a multiple of 4, or
# smaller than one box); the others the TMA-staged ones, (2, 45, 52) and (1, 70, 100) with
# ragged tiles, (2, 512, 512) at the reconstruction step's detector size
SSIM2D_SHAPES = [(3, 37, 53), (2, 64, 64), (1, 5, 7), (2, 45, 52), (1, 70, 100), (2, 512, 512)]


@pytest.mark.parametrize("shape", SSIM2D_SHAPES)
def test_ssim2d(B, shape):
    rng = np.random.default_rng(2)
    y = _x32(rng.random(shape))
    x = _x32(np.clip(y + 0.1 * rng.standard_normal(shape), 0, None))
    L = float(y.max())
    val, g = _run_loss(B, "ssim2d", x, y, L, weight=0.25)
    want, gw = OL.value_and_grad(lambda a, b: 0.25 * (1 - OL.ssim2d(a, b, L)), x, y)
    assert abs(val - want) <= 2e-5 * max(1.0, abs(want)), (val, want)
    scale = np.abs(gw).max()
    assert np.abs(g - gw).max() <= 1e-3 * scale, float(np.abs(g - gw).max() / scale)


@pytest.mark.parametrize("shape", SSIM2D_SHAPES)
def test_l1_ssim2d_fused(B, shape):
    """L1 + D-SSIM in the two SSIM kernels equals the oracle's sum of both terms, and the
    separate L1 and SSIM calls, value and gradient; accumulate adds onto the gradient."""
    rng = np.random.default_rng(5)
    y = _x32(rng.random(shape))
    x = _x32(np.clip(y + 0.1 * rng.standard_normal(shape), 0, None))
    x.flat[::7] = y.flat[::7]  # ties: sign(0) = 0 on both paths
    L = float(y.max())
    val, g = _run_loss(B, "l1ssim2d", x, y, L, 0.6, weight=0.25)
    want, gw = OL.value_and_grad(lambda a, b: 0.6 * OL.l1(a, b) + 0.25 * (1 - OL.ssim2d(a, b, L)),
                                 x, y)
    assert abs(val - want) <= 2e-5 * max(1.0, abs(want)), (val, want)
    scale = np.abs(gw).max()
    assert np.abs(g - gw).max() <= 1e-3 * scale, float(np.abs(g - gw).max() / scale)
    v1, g1 = _run_loss(B, "l1", x, y, weight=0.6)
    v2, g2 = _run_loss(B, "ssim2d", x, y, L, weight=0.25, accumulate_into=g1)
    assert abs(val - (v1 + v2)) <= 1e-5 * max(1.0, abs(val))
    np.testing.assert_allclose(g, g2, rtol=1e-5, atol=1e-6 * scale)
    va, ga = _run_loss(B, "l1ssim2d", x, y, L, 0.6, weight=0.25, accumulate_into=np.ones_like(x))
    np.testing.assert_allclose(ga, g + 1.0, rtol=1e-6, atol=1e-7)


def test_ssim2d_tma_equals_register_staging(B):
    """The TMA-staged 2D kernels equal the register-staged ones (taken when a buffer is not
    16-byte aligned) on the same images: L1 + D-SSIM value and the gradient accumulated onto
    a non-zero one."""
    L_ = B.lib()
    rng = np.random.default_rng(11)
    n, H, W = 3, 75, 136
    y = rng.random((n, H, W), dtype=np.float32)
    x = np.clip(y + 0.1 * rng.standard_normal((n, H, W)).astype(np.float32), 0, None)
    # a base of the gradient's own size, so that its rounding does not hide the comparison
    base = (1e-5 * rng.standard_normal((n, H, W))).astype(np.float32)
    out = []
    for off in (0, 1):  # a one-float offset breaks the 16-byte alignment
        bufs = [torch.zeros(n * H * W + 4, device="cuda") for _ in range(3)]
        xd, yd, gd = (t[off:off + n * H * W] for t in bufs)
        xd.copy_(torch.from_numpy(x.ravel()))
        yd.copy_(torch.from_numpy(y.ravel()))
        gd.copy_(torch.from_numpy(base.ravel()))
        loss = torch.zeros(1, device="cuda")
        ws = torch.empty(L_.gs_ssim_workspace_size(n * H * W), dtype=torch.uint8, device="cuda")
        B.check(L_.gs_l1_ssim2d_loss(B.ptr(xd), B.ptr(yd), n, H, W, float(y.max()), 0.6, 0.25,
                                     B.ptr(loss), B.ptr(gd), 1, B.ptr(ws), ws.numel(), _s()),
                "gs_l1_ssim2d_loss")
        torch.cuda.synchronize()
        out.append((float(loss.item()), gd.cpu().numpy().astype(np.float64)))
    (v0, g0), (v1, g1) = out
    assert abs(v0 - v1) <= 1e-6 * abs(v1)
    scale = np.abs(g1 - base.ravel()).max()
    assert np.abs(g0 - g1).max() <= 1e-5 * scale


@pytest.mark.parametrize("shape", [(21, 19, 35), (12, 16, 16), (4, 40, 33), (1, 9, 70)])
def test_ssim3d(B, shape):
    rng = np.random.default_rng(3)
    y = _x32(rng.random(shape))
    x = _x32(np.clip(y + 0.1 * rng.standard_normal(shape), 0, None))
    L = float(y.max())
    val, g = _run_loss(B, "ssim3d", x, y, L, weight=0.5)
    want, gw = OL.value_and_grad(lambda a, b: 0.5 * (1 - OL.ssim3d(a, b, L)), x, y)
    assert abs(val - want) <= 2e-5 * max(1.0, abs(want)), (val, want)
    scale = np.abs(gw).max()
    assert np.abs(g - gw).max() <= 1e-3 * scale, float(np.abs(g - gw).max() / scale)


@pytest.mark.parametrize("shape", [(37, 45, 52), (70, 26, 48), (16, 33, 96)])
def test_ssim3d_streaming(B, shape):
    """Volumes the fused streaming kernels take (x a multiple of 4, at least 48 x 18 columns):
    several 32 x 8 column tiles with ragged edges, z in one or more chunks (70 planes run as
    two chunks of 35), against the FP64 oracle; then accumulation onto a non-zero gradient and
    the value-only call."""
    rng = np.random.default_rng(5)
    y = _x32(rng.random(shape))
    x = _x32(np.clip(y + 0.1 * rng.standard_normal(shape), 0, None))
    L = float(y.max())
    val, g = _run_loss(B, "ssim3d", x, y, L, weight=0.5)
    want, gw = OL.value_and_grad(lambda a, b: 0.5 * (1 - OL.ssim3d(a, b, L)), x, y)
    assert abs(val - want) <= 2e-5 * max(1.0, abs(want)), (val, want)
    scale = np.abs(gw).max()
    assert np.abs(g - gw).max() <= 1e-3 * scale, float(np.abs(g - gw).max() / scale)
    base = _x32(rng.standard_normal(shape))
    val2, g2 = _run_loss(B, "ssim3d", x, y, L, weight=0.5, accumulate_into=base)
    assert abs(val2 - val) <= 1e-6 * abs(val)  # block sums meet in atomic order
    assert np.abs(g2 - (gw + base)).max() <= 1e-3 * scale + 1e-6 * np.abs(base).max()
    # value only: no gradient pointer
    Lb = B.lib()
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    loss = torch.zeros(1, device="cuda")
    ws = torch.empty(Lb.gs_ssim3d_workspace_size(xd.numel()), dtype=torch.uint8, device="cuda")
    dz, dy, dx = shape
    B.check(Lb.gs_ssim3d_loss(B.ptr(xd), B.ptr(yd), dx, dy, dz, L, 0.5, B.ptr(loss), None, 0,
                              B.ptr(ws), ws.numel(), _s()), "ssim3d value")
    torch.cuda.synchronize()
    assert abs(float(loss.item()) - val) <= 1e-6 * abs(val)


def test_ssim3d_streaming_equals_separable_passes(B):
    """The fused streaming kernels against the separable z + xy passes on one larger volume
    (the separable path taken by handing the library x and y at a 4-byte offset, which the
    streaming kernels' tile copies cannot start from): the same loss and accumulated gradient
    up to FP32 rounding order, at a size the FP64 oracle would take minutes for."""
    Lb = B.lib()
    shape = (100, 70, 96)  # z, y, x: three 32-column tiles, 9 ragged 8-row tiles, 2 z chunks
    g = torch.Generator(device="cuda").manual_seed(11)
    y = torch.rand(shape, device="cuda", generator=g)
    x = (y + 0.1 * torch.randn(shape, device="cuda", generator=g)).clamp_min(0)
    n = x.numel()
    ws = torch.empty(Lb.gs_ssim3d_workspace_size(n), dtype=torch.uint8, device="cuda")
    # the same values one float past a 16-byte boundary
    xs = torch.empty(n + 4, device="cuda")
    ys = torch.empty(n + 4, device="cuda")
    xs[1:n + 1] = x.reshape(-1)
    ys[1:n + 1] = y.reshape(-1)
    # a gradient to accumulate onto, of the size of the SSIM gradient itself (about 1e-6 here),
    # so that the FP32 sum keeps the SSIM part's digits
    base = 1e-6 * torch.randn(shape, device="cuda", generator=g)
    out = []
    for px, py in ((B.ptr(x), B.ptr(y)), (B.ptr(xs) + 4, B.ptr(ys) + 4)):
        loss = torch.zeros(1, device="cuda")
        grad = base.clone()
        dz, dy, dx = shape
        B.check(Lb.gs_ssim3d_loss(px, py, dx, dy, dz, 1.0, 0.5, B.ptr(loss), B.ptr(grad), 1,
                                  B.ptr(ws), ws.numel(), _s()), "ssim3d")
        torch.cuda.synchronize()
        out.append((float(loss.item()), (grad - base).double().cpu().numpy()))
    (l_f, g_f), (l_s, g_s) = out
    assert abs(l_f - l_s) <= 1e-5 * abs(l_s)
    assert np.abs(g_f - g_s).max() <= 1e-4 * np.abs(g_s).max()


def test_adam_matches_oracle(B):
    rng = np.random.default_rng(4)
    n = 1000
    raw = [_x32(rng.standard_normal((n, 4))) for _ in range(3)]
    raw[1][:, 3] = 0
    raw[1][:, :3] = np.log(0.02) + 0.3 * raw[1][:, :3]
    o = B.GsAdamOpts()
    o.lr_mean, o.lr_rho, o.lr_scale, o.lr_quat = 1e-3, 1e-2, 5e-3, 2e-3
    o.beta1, o.beta2, o.eps = 0.9, 0.999, 1e-15
    o.min_log_scale, o.max_log_scale = np.log(1e-4), np.log(0.5)
    d_raw = [torch.from_numpy(a.astype(np.float32)).cuda() for a in raw]
    d_act = [torch.empty_like(t) for t in d_raw]
    m = torch.zeros((3 * n, 4), device="cuda")
    v = torch.zeros_like(m)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    om = [np.zeros((n, 4)) for _ in range(3)]
    ov = [np.zeros((n, 4)) for _ in range(3)]
    cur = [a.copy() for a in raw]
    for t in range(1, 4):
        gr = [_x32(rng.standard_normal((n, 4))) for _ in range(3)]
        gr[1][:, 3] = 0
        d_g = [torch.from_numpy(a.astype(np.float32)).cuda() for a in gr]
        B.check(B.lib().gs_adam_step(*[B.ptr(x) for x in d_raw], B.ptr(m), B.ptr(v),
                                     *[B.ptr(x) for x in d_g], *[B.ptr(x) for x in d_act], n,
                                     B.ptr(step), ctypes.byref(o), _s()), "adam")
        cur = OO.adam_step(cur, om, ov, gr, t, (1e-3, 1e-2, 5e-3, 2e-3), 0.9, 0.999, 1e-15,
                           np.log(1e-4), np.log(0.5))
    torch.cuda.synchronize()
    assert int(step.item()) == 3
    for a, b in zip(d_raw, cur):
        np.testing.assert_allclose(a.cpu().numpy(), b, rtol=2e-5, atol=2e-6)
    act = OO.activate(*cur)
    for a, b in zip(d_act, act):
        np.testing.assert_allclose(a.cpu().numpy(), b, rtol=2e-5, atol=2e-6)


def test_recon_step_decreases_loss(B):
    """A small reconstruction (projections of a second Gaussian set as the target): the loss
    falls over the first iterations and the step's gradient equals the sum of its parts."""
    import synth
    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300.recon import ReconConfig, Reconstruction

    views = synth.cone_views(8, 64, 64)
    model = synth.gaussians(30, 1500, scale_median=0.03)
    tgt = synth.gaussians(31, 1500, scale_median=0.03)
    target = g.Projector(views, 64, 64).forward(*[torch.from_numpy(a).cuda() for a in tgt])
    rec = Reconstruction(views, 64, 64, target.clone(), synth.cube_grid(48), *model,
                         cfg=ReconConfig(lr_mean=1e-3, lr_rho=2e-2))
    losses = []
    for _ in range(30):
        losses.append(float(rec.step().item()))
    assert losses[-1] < 0.8 * losses[0], losses[::5]


@pytest.mark.parametrize("chunks", [2, 3])
def test_pipelined_step_equals_serial_step(B, chunks):
    """The step with the TV branch and view chunks on their own streams computes what the serial
    step computes: the same images and volume (bit-identical), the loss to rounding (its terms
    are summed in another order), the same parameter update up to Adam's sign flips of
    gradients near zero (unordered float atomics)."""
    import synth
    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300.recon import ReconConfig, Reconstruction

    views = synth.cone_views(9, 64, 56)
    model = synth.gaussians(40, 2000, scale_median=0.03)
    tgt = synth.gaussians(41, 2000, scale_median=0.03)
    target = g.Projector(views, 64, 56).forward(*[torch.from_numpy(a).cuda() for a in tgt])
    recs = [Reconstruction(views, 64, 56, target.clone(), synth.cube_grid(40), *model,
                           cfg=ReconConfig(lr_mean=1e-3, lr_rho=2e-2, view_streams=k))
            for k in (chunks, 1)]
    assert len(recs[0].vchunks) == chunks and not recs[1].vchunks
    la = float(recs[0].step().item())
    lb = float(recs[1].step(serial=True).item())
    torch.cuda.synchronize()
    assert torch.equal(recs[0].img, recs[1].img)
    assert torch.equal(recs[0].vol, recs[1].vol)
    assert abs(la - lb) <= 1e-5 * abs(lb), (la, lb)
    for x, y in zip(recs[0].act, recs[1].act):
        close = torch.isclose(x, y, rtol=1e-5, atol=1e-6).float().mean().item()
        assert close > 0.99, close
    # and over a few more steps the two runs stay together
    for _ in range(4):
        la = float(recs[0].step().item())
        lb = float(recs[1].step(serial=True).item())
    assert abs(la - lb) <= 1e-3 * abs(lb), (la, lb)
