"""The per-brick MLP initializer on the device against the float64 oracle: the fused brick
render + L1 kernel (value and gradient), the network's forward and its weight gradients, and a
training run whose loss falls."""
import numpy as np
import pytest
import torch

from oracle import mlp as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300 import build

    build.build()
    return g


def test_brick_loss_matches_oracle(gsct):
    B = gsct.binding
    rng = np.random.default_rng(0)
    nb = 6
    raw = rng.standard_normal((nb, 352)) * 0.6
    raw.reshape(nb, 32, 11)[:, :, 3:6] += 0.8
    target = rng.random((nb, 4096)) * 0.5
    raw32, tgt32 = raw.astype(np.float32), target.astype(np.float32)
    y = torch.zeros((nb, 384), device="cuda")
    y[:, :352] = torch.from_numpy(raw32).cuda()
    t = torch.from_numpy(tgt32).cuda()
    loss = torch.zeros(1, device="cuda")
    dy = torch.zeros((nb, 384), device="cuda")
    B.check(B.lib().gs_brick_loss(B.ptr(y), 384, B.ptr(t), nb, B.ptr(loss), B.ptr(dy), 384, None,
                                  torch.cuda.current_stream().cuda_stream), "brick_loss")
    torch.cuda.synchronize()
    rr = torch.from_numpy(raw32.astype(np.float64)).requires_grad_(True)
    want = OM.brick_l1(rr, torch.from_numpy(tgt32.astype(np.float64)))
    (g,) = torch.autograd.grad(want, rr)
    assert abs(float(loss) - float(want)) <= 1e-5 * abs(float(want))
    got = dy[:, :352].cpu().double()
    scale = float(g.abs().max())
    assert float((got - g).abs().max()) <= 2e-3 * scale, float((got - g).abs().max() / scale)


def _mlp_ref(m):
    Ws = [w.detach().cpu().double() for w in m.W]
    bs = [b.detach().cpu().double() for b in m.b]
    return Ws, bs


def test_mlp_forward_and_weight_gradients(gsct):
    from paper_2604_01844_gb300.mlp import BrickMLP

    m = BrickMLP(seed=3)
    rng = np.random.default_rng(1)
    M = 256
    x = torch.from_numpy(rng.random((M, 4096)).astype(np.float32))
    x16 = x.to(torch.bfloat16).cuda()
    y = m.forward(x16)
    Ws, bs = _mlp_ref(m)
    Ws = [w.requires_grad_(True) for w in Ws]
    bs = [b.requires_grad_(True) for b in bs]
    yref = OM.mlp_forward(x.double(), Ws, bs)
    got = y.cpu().double()
    assert float((got - yref).abs().max()) <= 2e-2 * float(yref.abs().max()) + 1e-3
    gy = torch.from_numpy(rng.standard_normal((M, 384)).astype(np.float32))
    gy[:, 352:] = 0
    m.backward(gy.cuda())
    (yref * gy.double()).sum().backward()
    torch.cuda.synchronize()
    for gw, ref in zip(m.grads, [w.grad for w in Ws] + [b.grad for b in bs]):
        g = gw.cpu().double()
        scale = float(ref.abs().max()) + 1e-12
        assert float((g - ref).abs().max()) <= 5e-2 * scale, float((g - ref).abs().max() / scale)


def test_mlp_training_reduces_brick_loss(gsct):
    """Bricks of smooth random blobs; 60 Adam steps roughly halve the render L1."""
    from paper_2604_01844_gb300.mlp import BrickMLP

    rng = np.random.default_rng(2)
    M = 256
    ax = np.arange(16) + 0.5
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    tgt = np.zeros((M, 4096), dtype=np.float32)
    for b in range(M):
        for _ in range(3):
            c = rng.uniform(3, 13, 3)
            s = rng.uniform(1.5, 4)
            tgt[b] += (rng.uniform(0.3, 1.0) * np.exp(-((xx - c[0]) ** 2 + (yy - c[1]) ** 2 +
                                                       (zz - c[2]) ** 2) / (2 * s * s))).ravel()
    noisy = tgt + 0.05 * rng.standard_normal(tgt.shape).astype(np.float32)
    x16 = torch.from_numpy(noisy).to(torch.bfloat16).cuda()
    t = torch.from_numpy(tgt).cuda()
    m = BrickMLP(seed=4)
    losses = []
    for it in range(60):
        loss = torch.zeros(1, device="cuda")
        m.train_step(x16, t, loss, lr=1e-3)
        losses.append(float(loss))
    assert int(m.err.item()) == 0
    assert losses[-1] < 0.6 * losses[0], losses[::10]


# ------------------------------------------------------------------------------------------
# The network entry points of the C ABI (gs_mlp_train_step, gs_mlp_infer) against the
# sequence of primitive library calls they stand for
# ------------------------------------------------------------------------------------------
def _primitive_train_step(B, m, x16, target, loss, lr, M):
    """Forward GEMMs -> gs_brick_loss -> transposes and backward GEMMs -> per-tensor Adam ->
    step increment, each a separate library call on the network's tensors."""
    L = B.lib()
    s = torch.cuda.current_stream().cuda_stream
    err = m.err

    def gemm(a, b, Mr, N, K, bias=None, relu=False, c32=None, c16=None):
        B.check(L.gs_gemm_bf16(B.ptr(a), B.ptr(b), Mr, N, K, B.ptr(bias), 1 if relu else 0,
                               B.ptr(c32), B.ptr(c16), N, B.ptr(err), s), "gemm")

    h = []
    a, K = x16, 4096
    for li in range(3):
        hb = torch.empty((M, 256), dtype=torch.bfloat16, device="cuda")
        gemm(a, m.W16[li], M, 256, K, bias=m.b[li], relu=True, c16=hb)
        h.append(hb)
        a, K = hb, 256
    y = torch.empty((M, 384), device="cuda")
    gemm(a, m.W16[3], M, 384, 256, bias=m.b[3], c32=y)
    dy = torch.zeros((M, 384), device="cuda")
    B.check(L.gs_brick_loss(B.ptr(y), 384, B.ptr(target), M, B.ptr(loss), B.ptr(dy), 384, None,
                            s), "brick_loss")
    acts = [x16] + h
    g32, width = dy, 384
    g16 = torch.empty((M, 384), dtype=torch.bfloat16, device="cuda")
    B.check(L.gs_f32_to_bf16(B.ptr(g32), B.ptr(g16), g32.numel(), s), "f32_to_bf16")
    for li in (3, 2, 1, 0):
        k_in = acts[li].shape[1]
        B.check(L.gs_colsum(B.ptr(g32), M, width, B.ptr(m.grads[4 + li]), s), "colsum")
        gT = torch.empty((width, M), dtype=torch.bfloat16, device="cuda")
        aT = torch.empty((k_in, M), dtype=torch.bfloat16, device="cuda")
        B.check(L.gs_transpose_bf16(B.ptr(g16), M, width, B.ptr(gT), s), "transpose")
        B.check(L.gs_transpose_bf16(B.ptr(acts[li]), M, k_in, B.ptr(aT), s), "transpose")
        gemm(gT, aT, width, k_in, M, c32=m.grads[li])
        if li == 0:
            break
        WT = torch.empty((k_in, width), dtype=torch.bfloat16, device="cuda")
        B.check(L.gs_transpose_bf16(B.ptr(m.W16[li]), width, k_in, B.ptr(WT), s), "transpose")
        gp = torch.empty((M, k_in), device="cuda")
        gemm(g16, WT, M, k_in, width, c32=gp)
        g16p = torch.empty((M, k_in), dtype=torch.bfloat16, device="cuda")
        B.check(L.gs_relu_mask_bf16(B.ptr(gp), B.ptr(h[li - 1]), gp.numel(), B.ptr(g16p), s),
                "relu_mask")
        g32, g16, width = gp, g16p, k_in
    # per-tensor Adam on views of the flat moments
    off = 0
    views = []
    for p in m.params:
        views.append((m.flat_m[off:off + p.numel()], m.flat_v[off:off + p.numel()]))
        off += p.numel()
    for i, (p, g, (mm, vv)) in enumerate(zip(m.params, m.grads, views)):
        B.check(L.gs_adam_flat(B.ptr(p), B.ptr(mm), B.ptr(vv), B.ptr(g), p.numel(),
                               B.ptr(m.step_count), lr, 0.9, 0.999, 1e-8,
                               B.ptr(m.W16[i]) if i < 4 else None, s), "adam_flat")
    B.check(L.gs_step_incr(B.ptr(m.step_count), s), "step_incr")


def test_exported_train_step_equals_primitive_sequence(gsct):
    """Three steps of gs_mlp_train_step and of the primitive call sequence from the same
    start: parameters, bf16 weights, Adam moments and gradients equal bit for bit."""
    from paper_2604_01844_gb300.mlp import BrickMLP

    B = gsct.binding
    rng = np.random.default_rng(9)
    M = 256
    x = torch.from_numpy(rng.random((3, M, 4096)).astype(np.float32))
    t = torch.from_numpy((rng.random((3, M, 4096)) * 0.4).astype(np.float32)).cuda()
    a, b = BrickMLP(seed=5), BrickMLP(seed=5)
    la, lb = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    for k in range(3):
        x16 = x[k].to(torch.bfloat16).cuda()
        a.train_step(x16, t[k], la, lr=1e-3)
        _primitive_train_step(B, b, x16, t[k], lb, 1e-3, M)
    torch.cuda.synchronize()
    assert int(a.err.item()) == 0 and int(b.err.item()) == 0
    assert int(a.step_count.item()) == 3 == int(b.step_count.item())
    for name, u, v in (("params", a.flat, b.flat), ("bf16 weights", a.flat16, b.flat16),
                       ("m", a.flat_m, b.flat_m), ("v", a.flat_v, b.flat_v),
                       ("grad", a.flat_grad, b.flat_grad)):
        assert torch.equal(u, v), (name, float((u.float() - v.float()).abs().max()))
    # the loss is summed over the bricks with float atomics: equal up to their order
    assert abs(float(la) - float(lb)) <= 1e-6 * abs(float(lb))


def test_infer_equals_forward_and_decode(gsct):
    from paper_2604_01844_gb300.mlp import BrickMLP

    B = gsct.binding
    rng = np.random.default_rng(10)
    M = 128
    m = BrickMLP(seed=6)
    x16 = torch.from_numpy(rng.random((M, 4096)).astype(np.float32)).to(torch.bfloat16).cuda()
    geo = torch.from_numpy(np.stack([rng.uniform(-1, 1, M), rng.uniform(-1, 1, M),
                                     rng.uniform(-1, 1, M), np.full(M, 2 / 256)],
                                    1).astype(np.float32)).cuda()
    got = m.infer_gaussians(x16, geo, 1.7)
    y = m.forward(x16)
    want = [torch.empty((M * 32, 4), device="cuda") for _ in range(3)]
    B.check(B.lib().gs_brick_decode(B.ptr(y), 384, B.ptr(geo), M, 1.7, *[B.ptr(w) for w in want],
                                    torch.cuda.current_stream().cuda_stream), "decode")
    torch.cuda.synchronize()
    for u, v in zip(got, want):
        assert torch.equal(u, v)
