"""Parity of the CUDA rasterizer (C ABI through the Python binding) with the FP64 oracle."""
import numpy as np
import pytest

import synth
from tests.helpers import (IMG_TOL, REL_BAND, assert_grads_close, grads11, px_band, to_dev)

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


def _case(seed, n, nv, W, H, median=0.02, radius=0.8):
    mr, sc, qt = synth.gaussians(seed, n, radius=radius, scale_median=median)
    views = synth.cone_views(nv, W, H)
    return mr, sc, qt, views


def _image_parity(orc, gsct, mr, sc, qt, views, W, H, tile, cut=3.0, eps=0.0):
    P = orc.params64(mr, sc, qt)
    V = orc.views64(views)
    opts = orc.Opts(cut=cut, eps=eps)
    want, n_eval = orc.project(P, V, W, H, opts)
    allow = orc.project_ambiguity(P, V, W, H, REL_BAND, px_band(W, H), opts)
    proj = gsct.Projector(views, W, H, cut=cut, eps=eps, tile=tile)
    d = to_dev(mr, sc, qt)
    img = proj.forward(*d).cpu().numpy().astype(np.float64)
    st = proj.status()
    assert st.code == 0
    err = np.abs(img - want)
    bound = IMG_TOL * np.abs(want).max() + allow + 1e-30
    assert (err <= bound).all(), (float((err / bound).max()), np.unravel_index(np.argmax(err / bound), err.shape))
    return proj, d, P, V, want, n_eval


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_forward_tiny_config(orc, gsct, tile):
    """2,000 Gaussians, 8 cone views of 64x64 (the small workload): images within 1e-4 of peak."""
    mr, sc, qt, views = _case(0, 2000, 8, 64, 64)
    _image_parity(orc, gsct, mr, sc, qt, views, 64, 64, tile)


def test_forward_ragged_detector(orc, gsct):
    """Non-square detector that is not a multiple of the tile: partial tiles on two sides."""
    mr, sc, qt, views = _case(1, 1500, 5, 83, 45, median=0.03)
    for tile in (8, 16, 32):
        _image_parity(orc, gsct, mr, sc, qt, views, 83, 45, tile)


def test_forward_single_tile_views(orc, gsct):
    """Views that fit in one tile (tile 32: no tile bits, the lists need no sort pass) and in
    four (tile 16: a 2-bit sort)."""
    mr, sc, qt, views = _case(8, 600, 5, 24, 20, median=0.03)
    for tile in (32, 16):
        _image_parity(orc, gsct, mr, sc, qt, views, 24, 20, tile)


def test_forward_parallel_beam(orc, gsct):
    mr, sc, qt = synth.gaussians(2, 800, scale_median=0.03)
    views = synth.parallel_views(4, 48, 40)
    _image_parity(orc, gsct, mr, sc, qt, views, 48, 40, 16)


def test_forward_density_cut(orc, gsct):
    """Factored-in density (Sec. 3.5) with eps > 0."""
    mr, sc, qt, views = _case(3, 1000, 4, 64, 64)
    _image_parity(orc, gsct, mr, sc, qt, views, 64, 64, 16, eps=2e-3)


def test_forward_degenerate_inputs(orc, gsct):
    """Zero quaternion, Gaussians behind the near plane or off the detector, huge footprints."""
    mr, sc, qt, views = _case(4, 300, 3, 40, 40, median=0.03)
    qt[0] = 0.0                          # zero quaternion: culled
    mr[1, :3] = views[0]["src"] * 0.99   # just in front of view 0's source: behind near plane
    mr[2, :3] = (5.0, 5.0, 5.0)          # far off every detector
    sc[3, :3] = (0.6, 0.5, 0.7)          # footprint larger than the detector
    _image_parity(orc, gsct, mr, sc, qt, views, 40, 40, 16)


def test_empty_and_single(orc, gsct):
    import torch

    views = synth.cone_views(2, 32, 32)
    proj = gsct.Projector(views, 32, 32)
    z = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
    img = proj.forward(z, z, z)
    assert img.shape == (2, 32, 32) and float(img.abs().max()) == 0.0
    mr, sc, qt = synth.gaussians(5, 1, radius=0.1, scale_median=0.05)
    _image_parity(orc, gsct, mr, sc, qt, views, 32, 32, 16)


@pytest.mark.parametrize("tile", [8, 16])
def test_keys_and_sort_order_bit_exact(orc, gsct, tile):
    """Culling, key duplication and the sort order equal the oracle's on every (view, Gaussian)
    pair outside the guard band: the device groups the oracle's (key, Gaussian)-ordered list
    by tile, stably."""
    W = H = 64
    mr, sc, qt, views = _case(6, 2000, 8, W, H)
    P, V = orc.params64(mr, sc, qt), orc.views64(views)
    keys_o, vals_o, counts_o = orc.keys(P, V, W, H, tile)  # tight tile rule
    flags = orc.pair_flags(P, V, W, H, REL_BAND, px_band(W, H), tile=tile)
    amb = (flags & 21) != 0  # box-edge, near-plane or tile-rule ambiguity changes keys
    proj = gsct.Projector(views, W, H, tile=tile)
    proj.forward(*to_dev(mr, sc, qt))
    keys_g, recs_g = proj.read_pairs()
    TWH = ((W + tile - 1) // tile) * ((H + tile - 1) // tile)
    tb = (TWH - 1).bit_length()  # key = (view << tb) | tile
    n, nv = mr.shape[0], len(views)
    kd, rd = keys_g.astype(np.int64), recs_g.astype(np.int64)
    v_g, t_g = kd >> tb, kd & ((1 << tb) - 1)
    assert np.all(t_g < TWH) and np.all(v_g < nv)
    # the device's values are (view, Gaussian) record indices v * n + i of the key's view
    assert np.array_equal(rd // n, v_g)
    vals_g = rd % n
    # the list is ordered by (tile, view, Gaussian): keys contiguous, Gaussians ascending
    assert np.all(np.diff((t_g * nv + v_g) * n + vals_g) > 0)

    def strip(k, v):
        keep = ~amb[k // TWH, v]
        return k[keep], v[keep]

    # the oracle's list (by key, then Gaussian) regrouped by tile, stably
    ko, vo = strip(keys_o.astype(np.int64), vals_o.astype(np.int64))
    perm = np.argsort(ko % TWH, kind="stable")
    ko, vo = ko[perm], vo[perm]
    kg, vg = strip(v_g * TWH + t_g, vals_g)
    assert np.array_equal(ko, kg) and np.array_equal(vo, vg)
    assert int(amb.sum()) < 0.01 * amb.size  # the guard band is rare


def test_count_evals_matches_oracle(orc, gsct):
    W = H = 64
    mr, sc, qt, views = _case(7, 2000, 8, W, H)
    P, V = orc.params64(mr, sc, qt), orc.views64(views)
    _, n_or = orc.project(P, V, W, H)
    flags = orc.pair_flags(P, V, W, H, REL_BAND, px_band(W, H))
    proj = gsct.Projector(views, W, H)
    n_gpu = proj.count_evals(*to_dev(mr, sc, qt))
    assert abs(n_gpu - n_or) <= int((flags != 0).sum()) * 2


def test_tile_invariance(gsct):
    """The per-pixel cut makes the image independent of the tile size (up to FP32 order)."""
    import torch

    mr, sc, qt, views = _case(8, 3000, 6, 96, 80)
    d = to_dev(mr, sc, qt)
    imgs = [gsct.Projector(views, 96, 80, tile=t).forward(*d) for t in (8, 16, 32)]
    peak = float(imgs[0].abs().max())
    for im in imgs[1:]:
        assert float((im - imgs[0]).abs().max()) <= 2e-6 * peak
    torch.cuda.synchronize()


def test_permutation_invariance(gsct):
    import torch

    mr, sc, qt, views = _case(9, 2000, 4, 64, 64)
    perm = np.random.default_rng(0).permutation(2000)
    a = gsct.Projector(views, 64, 64).forward(*to_dev(mr, sc, qt))
    b = gsct.Projector(views, 64, 64).forward(*to_dev(mr[perm], sc[perm], qt[perm]))
    assert float((a - b).abs().max()) <= 2e-6 * float(a.abs().max())
    torch.cuda.synchronize()


def test_capacity_overflow_is_reported(gsct):
    """A workspace with too few pair slots reports GS_ERR_CAPACITY and the needed count."""
    import torch

    mr, sc, qt, views = _case(10, 2000, 4, 64, 64)
    d = to_dev(mr, sc, qt)
    proj = gsct.Projector(views, 64, 64)
    need = proj.count_pairs(*d)
    proj._alloc(2000, need // 2)
    img = torch.empty((4, 64, 64), device="cuda")
    proj.forward(*d, out=img)
    st = proj.status()
    assert st.code == gsct.binding.GS_ERR_CAPACITY and st.pairs == need
    proj.ensure_capacity(*d)
    proj.forward(*d, out=img)
    assert proj.status().code == 0


def _grad_case(orc, gsct, seed, n, nv, W, H, tile, median=0.03, mode="cone", reuse=True):
    mr, sc, qt = synth.gaussians(seed, n, radius=0.7, scale_median=median)
    views = synth.cone_views(nv, W, H) if mode == "cone" else synth.parallel_views(nv, W, H)
    P, V = orc.params64(mr, sc, qt), orc.views64(views)
    w = np.random.default_rng(seed).standard_normal((nv, H, W))
    want = orc.project_grad(P, V, W, H, w)
    flags = orc.pair_flags(P, V, W, H, REL_BAND, px_band(W, H))
    clean = ~(flags != 0).any(axis=0)
    proj = gsct.Projector(views, W, H, tile=tile)
    import torch

    d = to_dev(mr, sc, qt)
    if reuse:
        proj.forward(*d)
    g = proj.backward(*d, torch.from_numpy(w.astype(np.float32)).cuda(), reuse=reuse)
    got = grads11(*g)
    assert clean.mean() > 0.9
    assert_grads_close(got, want, clean)
    return got, want


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_backward_matches_oracle_adjoint(orc, gsct, tile):
    """Per-Gaussian backward vs the oracle's dual-number gradients (1e-3 relative)."""
    _grad_case(orc, gsct, 11, 600, 6, 64, 64, tile)


def test_backward_recompute_equals_reuse(orc, gsct):
    a, _ = _grad_case(orc, gsct, 12, 500, 4, 48, 48, 16, reuse=True)
    b, _ = _grad_case(orc, gsct, 12, 500, 4, 48, 48, 16, reuse=False)
    np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-7 * np.abs(a).max())


def test_backward_parallel_beam(orc, gsct):
    _grad_case(orc, gsct, 13, 400, 4, 48, 40, 16, mode="parallel")


def test_backward_accumulate_flag(gsct):
    import torch

    mr, sc, qt, views = _case(14, 500, 3, 48, 48, median=0.03)
    d = to_dev(mr, sc, qt)
    proj = gsct.Projector(views, 48, 48)
    proj.forward(*d)
    w = torch.randn(3, 48, 48, device="cuda")
    g1 = proj.backward(*d, w)
    acc = tuple(torch.ones_like(t) for t in d)
    proj.backward(*d, w, grads=acc, accumulate=True)
    for a, b in zip(acc, g1):
        assert torch.allclose(a, b + 1.0, rtol=1e-5, atol=1e-5)


def test_backward_against_fp64_finite_differences(orc, gsct):
    """GPU gradients vs FP64 central differences of the oracle forward (1e-2 relative), on a
    tiny case without truncation so that the mask cannot flip."""
    import torch

    W = H = 24
    mr, sc, qt = synth.gaussians(15, 4, radius=0.3, scale_median=0.07)
    views = synth.cone_views(3, W, H, det_len=1.6)
    P, V = orc.params64(mr, sc, qt), orc.views64(views)
    opts = orc.Opts(cut=20.0)
    w = np.random.default_rng(1).standard_normal((3, H, W))
    proj = gsct.Projector(views, W, H, cut=20.0, tile=8)
    g = grads11(*proj.backward(*to_dev(mr, sc, qt), torch.from_numpy(w.astype(np.float32)).cuda(),
                               reuse=False))
    for i in range(4):
        for t in range(11):
            h = 1e-6 * max(1.0, abs(P[i, t]))
            Pp = P.copy(); Pp[i, t] += h
            Pm = P.copy(); Pm[i, t] -= h
            fd = ((w * orc.project(Pp, V, W, H, opts)[0]).sum() -
                  (w * orc.project(Pm, V, W, H, opts)[0]).sum()) / (2 * h)
            assert abs(g[i, t] - fd) <= 1e-2 * (abs(fd) + np.abs(g[i]).max() * 0.01), (i, t, g[i, t], fd)


def test_autograd_function(gsct):
    import torch

    mr, sc, qt, views = _case(16, 400, 3, 40, 40, median=0.03)
    d = [t.clone().requires_grad_(True) for t in to_dev(mr, sc, qt)]
    proj = gsct.Projector(views, 40, 40)
    img = gsct.project(d[0], d[1], d[2], proj)
    w = torch.randn_like(img)
    (img * w).sum().backward()
    ref = proj.backward(*[t.detach() for t in d], w, reuse=False)
    # the two backward calls sum with float atomics in no fixed order: entries agree to a few
    # ulp of the terms summed, i.e. relative to the gradient's scale, not to each entry
    for t, r in zip(d, ref):
        assert torch.allclose(t.grad, r, rtol=1e-5, atol=1e-5 * float(r.abs().max()))


def test_view_chunking_matches_single_call(gsct, monkeypatch):
    """When the views need more pairs than one call can sort, the projector splits them into
    chunks: images are identical to the single call, gradients agree (unordered atomics)."""
    import torch

    from paper_2604_01844_gb300 import projector as P

    mr, sc, qt, views = _case(31, 3000, 12, 64, 64)
    d = to_dev(mr, sc, qt)
    one = gsct.Projector(views, 64, 64)
    img1 = one.forward(*d)
    w = torch.randn_like(img1)
    g1 = one.backward(*d, w)
    pairs = one.count_pairs(*d)
    monkeypatch.setattr(P, "MAX_PAIRS_PER_CALL", pairs // 3)
    many = gsct.Projector(views, 64, 64)
    img2 = many.forward(*d)
    assert many.chunks is not None and len(many.chunks) >= 3
    assert torch.equal(img1, img2)
    g2 = many.backward(*d, w)
    for a, b in zip(g1, g2):
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * float(a.abs().max()))
    assert many.count_evals(*d) == one.count_evals(*d)
    assert many.status().code == 0
