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
