"""View-sharded reconstruction step, host logic on the CPU: the partition of the views, the
per-process loss shares and the gradient all-reduce, on two gloo processes with the FP64
oracle's gradients standing in for each process's GPU backward.  The all-reduced gradient of
the sharded L1 projection loss must equal the gradient of the loss over all views computed in
one process (Eq. 5 is a sum over views; Sec. 3.2 renders each view on its own)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import synth

W = H = 24
NV = 5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import oracle

    model = oracle.params64(*synth.gaussians(40, 60, radius=0.6, scale_median=0.08))
    tgt = oracle.params64(*synth.gaussians(41, 60, radius=0.6, scale_median=0.08))
    V = oracle.views64(synth.cone_views(NV, W, H))
    target, _ = oracle.project(tgt, V, W, H)
    return model, V, target


def _l1_terms(P, V, target, share):
    """Value and gradient of share * mean |I - target| over the given views (the weighting
    Reconstruction._image_losses applies to its views' L1 term)."""
    import oracle

    img, _ = oracle.project(P, V, W, H)
    d = img - target
    loss = share * np.abs(d).mean()
    dimg = share * np.sign(d) / d.size
    return loss, oracle.project_grad(P, V, W, H, dimg)


def _rank(rank, world, port, out):
    import torch.distributed as dist

    from paper_2604_01844_gb300 import sharded as S

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P, V, target = _problem()
        a, b = S.view_range(NV, rank, world)
        loss, g = _l1_terms(P, V[a:b], target[a:b], S.view_share(a, b, NV))
        flat = torch.from_numpy(np.concatenate([g.ravel(), [loss]]))
        S.allreduce_sum_(flat)
        peak = S.allreduce_max(float(target[a:b].max()), "cpu")
        out[rank] = (flat.numpy().copy(), peak, (a, b))
    finally:
        dist.destroy_process_group()


def test_two_process_view_shards_sum_to_the_full_gradient():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    P, V, target = _problem()
    loss, g = _l1_terms(P, V, target, 1.0)
    want = np.concatenate([g.ravel(), [loss]])
    assert np.abs(want[:-1]).max() > 0
    assert res[0][2] == (0, 3) and res[1][2] == (3, 5)
    for r in range(2):
        np.testing.assert_allclose(res[r][0], want, rtol=1e-12, atol=1e-15 * np.abs(want).max())
        assert res[r][1] == pytest.approx(float(target.max()), rel=1e-6)
    assert np.array_equal(res[0][0], res[1][0])  # every process applies the same update


def test_view_range_partitions():
    from paper_2604_01844_gb300 import sharded as S

    for nv in (1, 2, 7, 75, 128):
        for world in range(1, min(nv, 9) + 1):
            rs = [S.view_range(nv, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == nv
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
            assert sum(S.view_share(a, b, nv) for a, b in rs) == pytest.approx(1.0, abs=1e-15)
    with pytest.raises(ValueError):
        S.view_range(3, 0, 4)
    with pytest.raises(ValueError):
        S.view_range(8, 2, 2)


def test_single_process_allreduce_is_identity():
    from paper_2604_01844_gb300 import sharded as S

    x = torch.arange(5, dtype=torch.float32)
    assert torch.equal(S.allreduce_sum_(x.clone()), x)
    assert S.allreduce_max(2.5, "cpu") == 2.5
