"""Batched reconstruction step: several uneven reconstructions advanced together equal the same
reconstructions stepped one by one, eagerly and under CUDA-graph replay."""
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


# (seed, n, views, W, H, grid side): uneven detectors, view counts, grids and budgets
SPECS = [(70, 1500, 8, 64, 64, 32), (72, 800, 5, 48, 40, 40), (74, 2500, 12, 64, 56, 48)]


def _instances(gsct):
    out = []
    for seed, n, nv, W, H, side in SPECS:
        views = synth.cone_views(nv, W, H)
        model = synth.gaussians(seed, n, scale_median=0.03)
        tgt = synth.gaussians(seed + 1, n, scale_median=0.03)
        target = gsct.Projector(views, W, H).forward(*[torch.from_numpy(a).cuda() for a in tgt])
        out.append(dict(views=views, W=W, H=H, target=target.clone(),
                        grid=synth.cube_grid(side), mean_rho=model[0], scale=model[1],
                        quat=model[2]))
    return out


def _cfg():
    from paper_2604_01844_gb300.recon import ReconConfig

    return ReconConfig(lr_mean=1e-3, lr_rho=2e-2)


def _singles(inst):
    from paper_2604_01844_gb300.recon import Reconstruction

    return [Reconstruction(x["views"], x["W"], x["H"], x["target"].clone(), x["grid"],
                           x["mean_rho"], x["scale"], x["quat"], cfg=_cfg()) for x in inst]


def _close_fraction(a, b):
    return torch.isclose(a, b, rtol=1e-4, atol=1e-6).float().mean().item()


def test_batch_step_equals_single_steps(gsct):
    from paper_2604_01844_gb300.batch import BatchReconstruction

    inst = _instances(gsct)
    rec = BatchReconstruction(inst, cfg=_cfg())
    singles = _singles(inst)
    for it in range(4):
        lb = rec.step().cpu().numpy()
        ls = np.array([float(s.step().item()) for s in singles])
        np.testing.assert_allclose(lb, ls, rtol=1e-4)
        if it == 0:
            # the first step's images and volumes come from the same initial parameters through
            # the same per-pair arithmetic and order: identical block by block
            for k, s in enumerate(singles):
                assert torch.equal(rec.imgs[k], s.img)
                assert torch.equal(rec.vols[k], s.vol)
    # parameters agree (Adam's near-zero-gradient sign flips under unordered atomics aside)
    for k, s in enumerate(singles):
        for x, y in zip(rec.params(k), s.act):
            assert _close_fraction(x, y) > 0.99


def test_batch_graph_replay_matches_eager(gsct):
    from paper_2604_01844_gb300.batch import BatchGraphStep, BatchReconstruction

    inst = _instances(gsct)
    a = BatchReconstruction(inst, cfg=_cfg())
    b = BatchReconstruction(inst, cfg=_cfg())
    g = BatchGraphStep(b, warmup=0)
    for _ in range(6):
        la = a.step().cpu().numpy()
        lb = g().cpu().numpy()
        np.testing.assert_allclose(lb, la, rtol=1e-4)
    for x, y in zip(a.act, b.act):
        assert _close_fraction(x, y) > 0.99


def test_batch_to_psnr_improves_every_instance(gsct):
    from paper_2604_01844_gb300.batch import BatchReconstruction, batch_to_psnr
    from paper_2604_01844_gb300.recon import PhantomProblem, fdk_volume, gradient_init, psnr_of

    inst, gts, peaks, p0 = [], [], [], []
    sse = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed, n, nv, W, H, side in [(80, 3000, 16, 64, 64, 48), (81, 2000, 12, 48, 48, 32)]:
        views = synth.cone_views(nv, W, H)
        grid = synth.cube_grid(side)
        prob = PhantomProblem(synth.ellipsoid_phantom(seed, 10), views, W, H, grid)
        u = np.random.default_rng(seed).random((n, 4)).astype(np.float32)
        mr, sc, q = gradient_init(fdk_volume(prob, grid), grid, n, u)
        inst.append(dict(views=views, W=W, H=H, target=prob.proj, grid=grid,
                         mean_rho=mr.cpu().numpy(), scale=sc.cpu().numpy(), quat=q.cpu().numpy()))
        gts.append(prob.gt)
        peaks.append(prob.peak)
    rec = BatchReconstruction(inst, cfg=_cfg())
    for k, v in enumerate(rec.volumes()):
        p0.append(psnr_of(v, gts[k], peaks[k], sse))
    reached, last, iters, ms = batch_to_psnr(rec, gts, peaks, max_iters=40, target_psnr=1e9,
                                             eval_every=10)
    assert iters == 40 and all(r is None for r in reached) and ms > 0
    assert all(b > a + 1.0 for a, b in zip(p0, last)), (p0, last)


def test_subset_continues_where_the_batch_stands(gsct):
    """rec.subset(keep) carries the kept instances' raw parameters, Adam moments and step
    count over bit for bit; stepped on, they follow the full batch."""
    from paper_2604_01844_gb300.batch import BatchReconstruction

    rec = BatchReconstruction(_instances(gsct), cfg=_cfg())
    for _ in range(3):
        rec.step()
    keep = [0, 2]
    sub = rec.subset(keep)
    torch.cuda.synchronize()
    assert sub.K == 2 and int(sub.step_count.item()) == int(rec.step_count.item()) == 3
    for j, k in enumerate(keep):
        a, b = int(rec.g_off[k]), int(rec.g_off[k + 1])
        c, d = int(sub.g_off[j]), int(sub.g_off[j + 1])
        for x, y in zip(sub.raw, rec.raw):
            assert torch.equal(x[c:d], y[a:b])
        for x, y in zip(sub.params(j), rec.params(k)):
            assert torch.equal(x, y)
        assert torch.equal(sub.m[3 * c:3 * d], rec.m[3 * a:3 * b])
        assert torch.equal(sub.v[3 * c:3 * d], rec.v[3 * a:3 * b])
        assert torch.equal(sub.targets[j], rec.targets[k])
    for _ in range(3):
        lf = rec.step().cpu().numpy()
        ls = sub.step().cpu().numpy()
        np.testing.assert_allclose(ls, lf[keep], rtol=1e-4)
    for j, k in enumerate(keep):
        for x, y in zip(sub.params(j), rec.params(k)):
            assert _close_fraction(x, y) > 0.99


def test_batch_to_psnr_retires_finished_instances(gsct):
    """With retire=True an instance that reached its target is not stepped again: its PSNR
    stays at the value of the evaluation that retired it, and the batch shrinks."""
    from paper_2604_01844_gb300.batch import BatchReconstruction, batch_to_psnr

    inst = _instances(gsct)
    rec = BatchReconstruction(inst, cfg=_cfg())
    # ground truths: the starting volumes; instance 0's target (0 dB) is met at the first
    # evaluation, the others' never
    gts = [v.clone() for v in rec.volumes()]
    peaks = [float(g.max()) for g in gts]
    targets = [0.0, 1e9, 1e9]
    hist = []
    reached, last, iters, ms = batch_to_psnr(rec, gts, peaks, 10, targets, eval_every=5,
                                             history=hist, retire=True)
    assert reached[0] == (5, hist[0][1]) and reached[1] is None and reached[2] is None
    assert [h[3] for h in hist] == [3, 2]  # three instances stepped to 5, two to 10
    assert last[0] == hist[0][2][0] and iters == 10
    assert last[1] != hist[0][2][1]  # the others kept stepping
