"""FP16 Gaussian codec on the GPU: encoding bit-exact with the reference (IEEE binary16,
round to nearest even), exact decoding, and on-demand voxelization of a codec equal to the
voxelization of its decoded parameters and to the FP64 oracle's."""
import numpy as np
import pytest

import synth
from oracle import codec as OC
from tests.helpers import IMG_TOL, REL_BAND, to_dev

pytestmark = pytest.mark.gpu

IDX_BAND = 2e-4


@pytest.fixture(scope="module")
def gsct():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300 import build

    build.build()
    return g


def _params(seed, n):
    mr, sc, qt = synth.gaussians(seed, n, scale_median=0.04)
    return mr, sc, qt


@pytest.mark.parametrize("n", [1, 37, 4099])
def test_encode_bit_exact_and_decode_exact(gsct, n):
    import torch

    from paper_2604_01844_gb300 import codec

    mr, sc, qt = _params(60, n)
    # edge values: overflow to inf, subnormals, signed zero, exact ties
    edge = np.array([7e4, -7e4, 2.0 ** -25, 3 * 2.0 ** -25, -0.0, 1 + 2.0 ** -11,
                     1 + 3 * 2.0 ** -11, 2.0 ** -20], np.float32)
    k = min(n, edge.size)
    mr[:k, 0] = edge[:k]
    qt[:k, 3] = edge[::-1][:k]
    d = to_dev(mr, sc, qt)
    bits = codec.encode(*d)
    assert bits.shape == (11, n) and bits.numel() * 2 == 22 * n
    want = OC.encode(mr, sc, qt)
    assert np.array_equal(bits.cpu().numpy().view(np.uint16), want)
    got = [t.cpu().numpy() for t in codec.decode(bits)]
    for a, b in zip(got, OC.decode(want)):
        assert np.array_equal(a.view(np.uint32), b.astype(np.float32).view(np.uint32))
    assert torch.isinf(codec.decode(bits)[0][:2, 0]).all() if n >= 2 else True


def test_empty_codec(gsct):
    import torch

    from paper_2604_01844_gb300 import codec

    z = torch.zeros((0, 4), device="cuda")
    assert codec.encode(z, z, z).shape == (11, 0)


def test_on_demand_voxelization(orc, gsct):
    from paper_2604_01844_gb300 import codec

    mr, sc, qt = _params(61, 1500)
    bits = codec.encode(*to_dev(mr, sc, qt))
    grid = synth.cube_grid(72)
    lo, dim = (5, 9, 13), (37, 50, 23)
    cv = codec.CodecVoxelizer(grid, lo, dim)
    vol = cv.forward(bits).cpu().numpy()
    assert cv.status().code == 0
    dmr, dsc, dq = codec.decode(bits)
    ref = gsct.Voxelizer(grid, lo, dim).forward(dmr, dsc, dq).cpu().numpy()
    assert np.array_equal(vol, ref)
    P = orc.params64(*OC.decode(bits.cpu().numpy().view(np.uint16)))
    want, _ = orc.voxelize(P, grid, lo, dim)
    allow = orc.voxelize_ambiguity(P, grid, lo, dim, REL_BAND, IDX_BAND)
    err = np.abs(vol.astype(np.float64) - want)
    assert (err <= IMG_TOL * np.abs(want).max() + allow + 1e-30).all()


def test_codec_keeps_a_fitted_volume(gsct):
    """A volume fit stored as FP16 and voxelized on demand loses little against FP32."""
    import torch

    from paper_2604_01844_gb300 import codec
    from paper_2604_01844_gb300.evaluate import VolumeScore
    from paper_2604_01844_gb300.fit import VolumeFit, fit_opts
    from paper_2604_01844_gb300.recon import PhantomProblem

    grid = synth.cube_grid(64)
    prob = PhantomProblem(synth.ellipsoid_phantom(95, 12), synth.cone_views(4, 32, 32), 32, 32,
                          grid)
    n = 4000
    u = torch.from_numpy(np.random.default_rng(2).random((n, 4)).astype(np.float32)).cuda()
    fit = VolumeFit(grid, n)
    params = fit.run(prob.gt, 80, fit_opts(data_range=prob.peak), u)
    score = VolumeScore(prob.gt, prob.peak)
    p32 = score.psnr(gsct.Voxelizer(grid).forward(*params))
    p16 = score.psnr(codec.CodecVoxelizer(grid).forward(codec.encode(*params)))
    assert p32 > 25.0 and abs(p32 - p16) < 0.5, (p32, p16)
