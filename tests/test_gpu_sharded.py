"""View-sharded reconstruction step on one GPU: the shards' gradient buffers, summed (what the
all-reduce over processes does), equal the single-process step's gradient, and with one
process the sharded step is the single-process step."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_01844_gb300 import build

    build.build()
    import paper_2604_01844_gb300 as g

    views = synth.cone_views(7, 64, 48)
    model = synth.gaussians(50, 1500, scale_median=0.03)
    tgt = synth.gaussians(51, 1500, scale_median=0.03)
    target = g.Projector(views, 64, 48).forward(*[torch.from_numpy(a).cuda() for a in tgt])
    return views, model, target.clone()


def _grads_before_adam(rec):
    """Runs one serial step of `rec` and returns a copy of its gradients (and loss) as they
    stand just before the Adam update."""
    got = {}
    orig = rec._before_adam

    def hook():
        orig()
        got["g"] = [t.clone() for t in rec.grads]
        got["loss"] = rec.loss.clone()

    rec._before_adam = hook
    rec.step(serial=True)
    torch.cuda.synchronize()
    return got["g"], got["loss"]


def test_shards_sum_to_single_process_gradient(setup):
    from paper_2604_01844_gb300.recon import ReconConfig, Reconstruction
    from paper_2604_01844_gb300.sharded import ViewShardedReconstruction

    views, model, target = setup
    cfg = ReconConfig(view_streams=1)
    grid = synth.cube_grid(32)
    full = Reconstruction(views, 64, 48, target, grid, *model, cfg=cfg)
    gw, lw = _grads_before_adam(full)
    parts = []
    for r in range(3):
        sh = ViewShardedReconstruction(views, 64, 48, target, grid, *model, rank=r, world=3,
                                       cfg=cfg, data_range=full.data_range)
        parts.append(_grads_before_adam(sh))
    for k in range(3):
        tot = sum(p[0][k] for p in parts)
        scale = float(gw[k].abs().max())
        assert scale > 0
        assert float((tot - gw[k]).abs().max()) <= 1e-5 * scale, k
    ltot = sum(float(p[1]) for p in parts)
    assert ltot == pytest.approx(float(lw), rel=1e-5)


def test_one_process_sharded_step_is_the_step(setup):
    """world = 1: no exchange, the same gradient and loss as the single-process step (float
    atomics make the sums' rounding order vary, hence the relative bound)."""
    from paper_2604_01844_gb300.recon import ReconConfig, Reconstruction
    from paper_2604_01844_gb300.sharded import ViewShardedReconstruction

    views, model, target = setup
    cfg = ReconConfig(view_streams=1)
    grid = synth.cube_grid(32)
    a = Reconstruction(views, 64, 48, target, grid, *model, cfg=cfg)
    b = ViewShardedReconstruction(views, 64, 48, target, grid, *model, rank=0, world=1, cfg=cfg)
    assert a.data_range == b.data_range
    ga, la = _grads_before_adam(a)
    gb, lb = _grads_before_adam(b)
    for x, y in zip(ga, gb):
        assert float((x - y).abs().max()) <= 1e-5 * float(x.abs().max())
    assert float(lb) == pytest.approx(float(la), rel=1e-6)
