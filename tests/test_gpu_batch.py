"""Batched rasterizer: several independent instances (own Gaussians, views, detector) in one
launch per pass.  Each instance's image and gradients are checked against the FP64 oracle run
on that instance alone, and against the single-instance path (same per-pair arithmetic and
summation order, so the forward images are bit-identical)."""
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


# uneven instances: Gaussian counts, view counts and ragged detectors all differ; one is empty
SPECS = [(300, 3, 40, 40), (0, 2, 24, 17), (900, 5, 83, 45), (120, 1, 16, 16), (500, 4, 64, 48)]


def _instances(specs, seed=100, median=0.03):
    out = []
    for k, (n, nv, W, H) in enumerate(specs):
        mr, sc, qt = synth.gaussians(seed + k, max(n, 1), radius=0.7, scale_median=median)
        out.append((mr[:n], sc[:n], qt[:n], synth.cone_views(nv, W, H), W, H))
    return out


def _concat(inst):
    import torch

    parts = [to_dev(mr, sc, qt) for mr, sc, qt, *_ in inst]
    d = tuple(torch.cat([p[j] for p in parts], 0).contiguous() for j in range(3))
    return d, [x[0].shape[0] for x in inst]


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_batch_forward_matches_oracle_and_single(orc, gsct, tile):
    inst = _instances(SPECS)
    bp = gsct.BatchProjector([(v, W, H) for *_, v, W, H in inst], tile=tile)
    d, counts = _concat(inst)
    imgs = bp.split(bp.forward(*d, counts))
    for (mr, sc, qt, views, W, H), img in zip(inst, imgs):
        single = gsct.Projector(views, W, H, tile=tile).forward(*to_dev(mr, sc, qt))
        assert np.array_equal(img.cpu().numpy(), single.cpu().numpy())
        if mr.shape[0] == 0:
            assert float(img.abs().max()) == 0.0
            continue
        P, V = orc.params64(mr, sc, qt), orc.views64(views)
        want, _ = orc.project(P, V, W, H)
        allow = orc.project_ambiguity(P, V, W, H, REL_BAND, px_band(W, H))
        err = np.abs(img.cpu().numpy().astype(np.float64) - want)
        bound = IMG_TOL * max(np.abs(want).max(), 1e-30) + allow + 1e-30
        assert (err <= bound).all()


@pytest.mark.parametrize("reuse", [True, False])
def test_batch_backward_matches_oracle(orc, gsct, reuse):
    import torch

    inst = _instances(SPECS, seed=200)
    bp = gsct.BatchProjector([(v, W, H) for *_, v, W, H in inst])
    d, counts = _concat(inst)
    rng = np.random.default_rng(7)
    ws = [rng.standard_normal((len(v), H, W)) for *_, v, W, H in inst]
    dimg = torch.zeros(bp.img_numel, device="cuda")
    for o, w in zip(bp.offsets, ws):
        dimg[o:o + w.size] = torch.from_numpy(w.ravel().astype(np.float32)).cuda()
    if reuse:
        bp.forward(*d, counts)
    got = grads11(*bp.backward(*d, counts, dimg, reuse=reuse))
    off = 0
    for (mr, sc, qt, views, W, H), w in zip(inst, ws):
        n = mr.shape[0]
        if n:
            P, V = orc.params64(mr, sc, qt), orc.views64(views)
            want = orc.project_grad(P, V, W, H, w)
            flags = orc.pair_flags(P, V, W, H, REL_BAND, px_band(W, H))
            clean = ~(flags != 0).any(axis=0)
            assert clean.mean() > 0.85
            assert_grads_close(got[off:off + n], want, clean)
        off += n


def test_batch_keys_and_records(gsct):
    """Keys are (global view, tile), records are (instance offset + view * n + Gaussian); the
    sorted list is ordered by tile, then global view, then record."""
    import ctypes

    inst = _instances(SPECS[:3], seed=300)
    bp = gsct.BatchProjector([(v, W, H) for *_, v, W, H in inst])
    d, counts = _concat(inst)
    bp.forward(*d, counts)
    st = gsct.binding.read_status(bp.ws)
    n = int(st.pairs)
    keys = np.zeros(max(n, 1), np.uint32)
    vals = np.zeros(max(n, 1), np.uint32)
    cnt = ctypes.c_int64(0)
    gsct.binding.check(gsct.binding.lib().gs_read_pairs(
        gsct.binding.ptr(bp.ws), bp.ws.numel(), gsct.binding.stream_handle(), n,
        keys.ctypes.data_as(ctypes.c_void_p), vals.ctypes.data_as(ctypes.c_void_p),
        ctypes.byref(cnt)), "gs_read_pairs")
    k, r = keys[:n].astype(np.int64), vals[:n].astype(np.int64)
    T = 16
    tiles = [((W + T - 1) // T) * ((H + T - 1) // T) for *_, W, H in inst]
    tb = (max(tiles) - 1).bit_length()  # key = (global view << tb) | tile
    gv, t = k >> tb, k & ((1 << tb) - 1)
    # ordered by (tile, global view, record): every key's pairs contiguous, records ascending
    order = np.stack([t, gv, r])
    d = np.diff(order, axis=1)
    assert np.all((d[0] > 0) | ((d[0] == 0) & (d[1] > 0)) | ((d[0] == 0) & (d[1] == 0) & (d[2] > 0)))
    # each record's instance and view agree with its key's, and the tile lies in the instance
    v_off = rec_off = 0
    for (mr, _, _, views, W, H), nt in zip(inst, tiles):
        nv, nr = len(views), len(views) * mr.shape[0]
        sel = (gv >= v_off) & (gv < v_off + nv)
        assert np.all((r[sel] >= rec_off) & (r[sel] < rec_off + nr))
        assert np.all(t[sel] < nt)
        if mr.shape[0]:
            assert np.array_equal(gv[sel] - v_off, (r[sel] - rec_off) // mr.shape[0])
        v_off += nv
        rec_off += nr
    assert np.all(gv < v_off)


def test_batch_of_one_equals_single(gsct):
    mr, sc, qt = synth.gaussians(400, 700, radius=0.7, scale_median=0.03)
    views = synth.cone_views(3, 48, 40)
    d = to_dev(mr, sc, qt)
    bp = gsct.BatchProjector([(views, 48, 40)])
    a = bp.split(bp.forward(*d, [700]))[0]
    b = gsct.Projector(views, 48, 40).forward(*d)
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_batch_rejects_mismatched_counts(gsct):
    views = synth.cone_views(2, 16, 16)
    bp = gsct.BatchProjector([(views, 16, 16)])
    with pytest.raises(ValueError):
        bp.forward(*to_dev(*synth.gaussians(1, 3)), [2])


# ---- batched voxelizer -------------------------------------------------------------------
IDX_BAND = 2e-4  # index-space guard band of the voxel box edges

# uneven instances: grids, regions (ragged, off-origin) and Gaussian counts differ; one empty
VSPECS = [(400, 48, (0, 0, 0), (48, 48, 48)), (0, 32, (0, 0, 0), (32, 32, 32)),
          (900, 72, (5, 9, 13), (37, 50, 23)), (150, 40, (8, 8, 8), (16, 16, 16)),
          (700, 64, (0, 0, 0), (64, 64, 64))]


def _vinstances(specs, seed=500, median=0.04):
    out = []
    for k, (n, side, lo, dim) in enumerate(specs):
        mr, sc, qt = synth.gaussians(seed + k, max(n, 1), scale_median=median)
        out.append((mr[:n], sc[:n], qt[:n], synth.cube_grid(side), lo, dim))
    return out


def test_batch_voxelize_matches_oracle_and_single(orc, gsct):
    inst = _vinstances(VSPECS)
    bv = gsct.BatchVoxelizer([(g, lo, dim) for *_, g, lo, dim in inst])
    d, counts = _concat(inst)
    vols = bv.split(bv.forward(*d, counts))
    for (mr, sc, qt, grid, lo, dim), vol in zip(inst, vols):
        single = gsct.Voxelizer(grid, lo, dim).forward(*to_dev(mr, sc, qt))
        assert np.array_equal(vol.cpu().numpy(), single.cpu().numpy())
        if mr.shape[0] == 0:
            assert float(vol.abs().max()) == 0.0
            continue
        P = orc.params64(mr, sc, qt)
        want, _ = orc.voxelize(P, grid, lo, dim)
        allow = orc.voxelize_ambiguity(P, grid, lo, dim, REL_BAND, IDX_BAND)
        err = np.abs(vol.cpu().numpy().astype(np.float64) - want)
        assert (err <= IMG_TOL * np.abs(want).max() + allow + 1e-30).all()


@pytest.mark.parametrize("reuse", [True, False])
def test_batch_voxelize_backward_matches_oracle(orc, gsct, reuse):
    import torch

    inst = _vinstances(VSPECS, seed=600)
    bv = gsct.BatchVoxelizer([(g, lo, dim) for *_, g, lo, dim in inst])
    d, counts = _concat(inst)
    rng = np.random.default_rng(9)
    ws = [rng.standard_normal((dim[2], dim[1], dim[0])) for *_, dim in inst]
    dvol = torch.zeros(bv.numel, device="cuda")
    for o, w in zip(bv.offsets, ws):
        dvol[o:o + w.size] = torch.from_numpy(w.ravel().astype(np.float32)).cuda()
    if reuse:
        bv.forward(*d, counts)
    got = grads11(*bv.backward(*d, counts, dvol, reuse=reuse))
    off = 0
    for (mr, sc, qt, grid, lo, dim), w in zip(inst, ws):
        n = mr.shape[0]
        if n:
            P = orc.params64(mr, sc, qt)
            want = orc.voxelize_grad(P, grid, w, lo, dim)
            flags = orc.voxel_flags(P, grid, lo, dim, REL_BAND, IDX_BAND)
            clean = flags == 0
            assert clean.mean() > 0.85
            assert_grads_close(got[off:off + n], want, clean)
        off += n
