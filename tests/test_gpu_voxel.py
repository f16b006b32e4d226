"""Parity of the CUDA voxelizer with the FP64 oracle."""
import numpy as np
import pytest

import synth
from tests.helpers import IMG_TOL, REL_BAND, assert_grads_close, grads11, to_dev

pytestmark = pytest.mark.gpu

IDX_BAND = 2e-4  # index-space guard band of the voxel box edges (|index| <= 1024)


@pytest.fixture(scope="module")
def gsct():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300 import build

    build.build()
    return g


def _vox_parity(orc, gsct, mr, sc, qt, grid, lo, dim):
    P = orc.params64(mr, sc, qt)
    want, _ = orc.voxelize(P, grid, lo, dim)
    allow = orc.voxelize_ambiguity(P, grid, lo, dim, REL_BAND, IDX_BAND)
    vox = gsct.Voxelizer(grid, lo, dim)
    got = vox.forward(*to_dev(mr, sc, qt)).cpu().numpy().astype(np.float64)
    assert vox.status().code == 0
    err = np.abs(got - want)
    bound = IMG_TOL * np.abs(want).max() + allow + 1e-30
    assert (err <= bound).all(), float((err / bound).max())
    return vox


def test_voxelize_tiny_config(orc, gsct):
    """2,000 Gaussians of the small workload into 64^3."""
    mr, sc, qt = synth.gaussians(0, 2000)
    _vox_parity(orc, gsct, mr, sc, qt, synth.cube_grid(64), (0, 0, 0), (64, 64, 64))


def test_voxelize_ragged_roi(orc, gsct):
    """A region of interest that is not a multiple of the brick and starts off-origin."""
    mr, sc, qt = synth.gaussians(1, 1500, scale_median=0.04)
    _vox_parity(orc, gsct, mr, sc, qt, synth.cube_grid(72), (5, 9, 13), (37, 50, 23))


def test_voxelize_patch_32(orc, gsct):
    """The 32^3 TV patch of Eq. 5 inside a 256^3 grid."""
    mr, sc, qt = synth.gaussians(2, 3000, scale_median=0.01)
    _vox_parity(orc, gsct, mr, sc, qt, synth.cube_grid(256), (100, 120, 90), (32, 32, 32))


def test_voxel_keys_bit_exact(orc, gsct):
    mr, sc, qt = synth.gaussians(3, 2000)
    grid = synth.cube_grid(64)
    P = orc.params64(mr, sc, qt)
    ko, vo, _ = orc.voxel_keys(P, grid, (0, 0, 0), (64, 64, 64), 16)
    flags = orc.voxel_flags(P, grid, (0, 0, 0), (64, 64, 64), REL_BAND, IDX_BAND)
    amb = (flags & 1) != 0
    vox = gsct.Voxelizer(grid)
    vox.forward(*to_dev(mr, sc, qt))
    kg, vg = vox.read_pairs()
    keep_o = ~amb[vo]
    keep_g = ~amb[vg.astype(np.int64)]
    assert np.array_equal(ko[keep_o], kg[keep_g].astype(np.int32))
    assert np.array_equal(vo[keep_o], vg[keep_g].astype(np.int32))


def test_voxel_count_evals(orc, gsct):
    mr, sc, qt = synth.gaussians(4, 2000)
    grid = synth.cube_grid(64)
    P = orc.params64(mr, sc, qt)
    _, n_or = orc.voxelize(P, grid)
    flags = orc.voxel_flags(P, grid, (0, 0, 0), (64, 64, 64), REL_BAND, IDX_BAND)
    vox = gsct.Voxelizer(grid)
    n_gpu = vox.count_evals(*to_dev(mr, sc, qt))
    assert abs(n_gpu - n_or) <= 4 * int((flags != 0).sum())


def test_voxelize_backward_matches_oracle(orc, gsct):
    import torch

    mr, sc, qt = synth.gaussians(5, 800, scale_median=0.04)
    grid = synth.cube_grid(48)
    P = orc.params64(mr, sc, qt)
    w = np.random.default_rng(5).standard_normal((48, 48, 48))
    want = orc.voxelize_grad(P, grid, w)
    flags = orc.voxel_flags(P, grid, (0, 0, 0), (48, 48, 48), REL_BAND, IDX_BAND)
    clean = flags == 0
    vox = gsct.Voxelizer(grid)
    d = to_dev(mr, sc, qt)
    vox.forward(*d)
    got = grads11(*vox.backward(*d, torch.from_numpy(w.astype(np.float32)).cuda()))
    assert clean.mean() > 0.9
    assert_grads_close(got, want, clean)


def test_voxelize_backward_roi_recompute(orc, gsct):
    import torch

    mr, sc, qt = synth.gaussians(6, 1500, scale_median=0.03)
    grid = synth.cube_grid(64)
    lo, dim = (8, 20, 3), (40, 33, 45)
    P = orc.params64(mr, sc, qt)
    w = np.random.default_rng(6).standard_normal((dim[2], dim[1], dim[0]))
    want = orc.voxelize_grad(P, grid, w, lo, dim)
    flags = orc.voxel_flags(P, grid, lo, dim, REL_BAND, IDX_BAND)
    vox = gsct.Voxelizer(grid, lo, dim)
    got = grads11(*vox.backward(*to_dev(mr, sc, qt), torch.from_numpy(w.astype(np.float32)).cuda(),
                                reuse=False))
    assert_grads_close(got, want, flags == 0)


def test_voxel_mass_on_gpu(gsct):
    """A well-sampled Gaussian's voxel sum times h^3 equals its truncated mass."""
    import math

    from scipy import special

    grid = synth.cube_grid(64, half=0.6)
    h = float(grid["voxel"][0])
    mr = np.array([[0.02, -0.01, 0.03, 0.6]], dtype=np.float32)
    sc = np.array([[0.05, 0.07, 0.04, 0]], dtype=np.float32)
    qt = np.array([[0.9, -0.2, 0.35, 0.1]], dtype=np.float32)
    vol = gsct.Voxelizer(grid).forward(*to_dev(mr, sc, qt)).cpu().numpy().astype(np.float64)
    mass = 0.6 * (2 * math.pi) ** 1.5 * 0.05 * 0.07 * 0.04
    frac = special.erf(3 / math.sqrt(2)) - math.sqrt(2 / math.pi) * 3 * math.exp(-4.5)
    assert abs(vol.sum() * h ** 3 / (mass * frac) - 1) < 3e-3


def test_voxelize_full_size_sampled(orc, gsct):
    """256^3 grid with 50,000 Gaussians: sampled voxels against the oracle one by one."""
    mr, sc, qt = synth.gaussians(7, 50000, scale_median=0.012, scale_sigma_log=0.4)
    grid = synth.cube_grid(256)
    vox = gsct.Voxelizer(grid)
    vol = vox.forward(*to_dev(mr, sc, qt)).cpu().numpy()
    idx = synth.voxel_samples(2, (256, 256, 256), 1200)
    want, allow = orc.voxelize_points_allow(orc.params64(mr, sc, qt), grid, idx, REL_BAND,
                                            IDX_BAND)
    got = vol[idx[:, 0], idx[:, 1], idx[:, 2]].astype(np.float64)
    peak = float(np.abs(want).max())
    assert peak > 0
    assert np.all(np.abs(got - want) <= IMG_TOL * peak + allow)


# ------------------------------------------------------------------------------------------
# Brick sides 16, 32 and 64: keys against the oracle's key rule for that side, volumes equal to
# the oracle and bit-identical across sides, gradients against the oracle's adjoint
# ------------------------------------------------------------------------------------------
BRICK_CASE = dict(grid=72, lo=(5, 9, 13), dim=(61, 50, 47))


@pytest.mark.parametrize("brick", [16, 32, 64])
def test_voxel_keys_bit_exact_per_brick(orc, gsct, brick):
    mr, sc, qt = synth.gaussians(13, 2500, scale_median=0.03)
    grid = synth.cube_grid(BRICK_CASE["grid"])
    lo, dim = BRICK_CASE["lo"], BRICK_CASE["dim"]
    P = orc.params64(mr, sc, qt)
    ko, vo, _ = orc.voxel_keys(P, grid, lo, dim, brick)
    flags = orc.voxel_flags(P, grid, lo, dim, REL_BAND, IDX_BAND)
    amb = (flags & 1) != 0
    vox = gsct.Voxelizer(grid, lo, dim, brick=brick)
    vox.forward(*to_dev(mr, sc, qt))
    assert vox.status().code == 0
    kg, vg = vox.read_pairs()
    keep_o = ~amb[vo]
    keep_g = ~amb[vg.astype(np.int64)]
    assert keep_o.sum() > 0.99 * len(vo)
    assert np.array_equal(ko[keep_o], kg[keep_g].astype(np.int32))
    assert np.array_equal(vo[keep_o], vg[keep_g].astype(np.int32))


@pytest.mark.parametrize("brick", [32, 64])
def test_volume_is_brick_invariant(orc, gsct, brick):
    """A ragged region (not a multiple of any brick side, off-origin): the volume matches the
    oracle and equals the 16-voxel-brick volume bit for bit; the in-cut evaluation count is
    the same."""
    import torch

    mr, sc, qt = synth.gaussians(14, 2500, scale_median=0.03)
    grid = synth.cube_grid(BRICK_CASE["grid"])
    lo, dim = BRICK_CASE["lo"], BRICK_CASE["dim"]
    if brick == 32:
        _vox_parity(orc, gsct, mr, sc, qt, grid, lo, dim)
    d = to_dev(mr, sc, qt)
    ref = gsct.Voxelizer(grid, lo, dim, brick=16)
    other = gsct.Voxelizer(grid, lo, dim, brick=brick)
    a = ref.forward(*d)
    b = other.forward(*d)
    torch.cuda.synchronize()
    assert other.status().code == 0
    assert torch.equal(a, b)
    assert ref.count_evals(*d) == other.count_evals(*d)


@pytest.mark.parametrize("brick", [32, 64])
def test_voxelize_parity_per_brick(orc, gsct, brick):
    mr, sc, qt = synth.gaussians(15, 2000)
    grid = synth.cube_grid(64)
    P = orc.params64(mr, sc, qt)
    want, _ = orc.voxelize(P, grid)
    allow = orc.voxelize_ambiguity(P, grid, (0, 0, 0), (64, 64, 64), REL_BAND, IDX_BAND)
    vox = gsct.Voxelizer(grid, brick=brick)
    got = vox.forward(*to_dev(mr, sc, qt)).cpu().numpy().astype(np.float64)
    assert vox.status().code == 0
    bound = IMG_TOL * np.abs(want).max() + allow + 1e-30
    assert (np.abs(got - want) <= bound).all()


@pytest.mark.parametrize("brick", [16, 32, 64])
def test_voxelize_backward_per_brick(orc, gsct, brick):
    import torch

    mr, sc, qt = synth.gaussians(16, 1200, scale_median=0.035)
    grid = synth.cube_grid(BRICK_CASE["grid"])
    lo, dim = BRICK_CASE["lo"], BRICK_CASE["dim"]
    P = orc.params64(mr, sc, qt)
    w = np.random.default_rng(16).standard_normal((dim[2], dim[1], dim[0]))
    want = orc.voxelize_grad(P, grid, w, lo, dim)
    flags = orc.voxel_flags(P, grid, lo, dim, REL_BAND, IDX_BAND)
    clean = flags == 0
    vox = gsct.Voxelizer(grid, lo, dim, brick=brick)
    d = to_dev(mr, sc, qt)
    vox.forward(*d)
    got = grads11(*vox.backward(*d, torch.from_numpy(w.astype(np.float32)).cuda()))
    assert vox.status().code == 0
    assert clean.mean() > 0.9
    assert_grads_close(got, want, clean)


def test_brick_autotuner_picks_a_valid_side(gsct):
    from paper_2604_01844_gb300.autotune import tune_brick

    mr, sc, qt = synth.gaussians(17, 20000, scale_median=0.01)
    best, times = tune_brick(synth.cube_grid(128), *to_dev(mr, sc, qt))
    assert best in (16, 32, 64) and set(times) == {16, 32, 64}
    assert all(t > 0 for t in times.values())
