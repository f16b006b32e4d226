"""Full-size parity on sampled outputs: the rasterizer at 75 cone views of 1024^2 with 200k
Gaussians and of 2048^2 with 500k Gaussians, and the voxelizer at 1024^3 with 500k Gaussians,
each against the FP64 oracle evaluated pixel by pixel (voxel by voxel)."""
import numpy as np
import pytest
import torch

import synth
from tests.helpers import IMG_TOL, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01844_gb300 as g
    from paper_2604_01844_gb300 import build

    build.build()
    return g


@pytest.mark.parametrize("side,n,median", [(1024, 200000, 0.008), (2048, 500000, 0.006)])
def test_raster_full_size_sampled(orc, gsct, side, n, median):
    mr, sc, qt = synth.gaussians(40 + side, n, radius=0.8, scale_median=median,
                                 scale_sigma_log=0.4)
    views = synth.cone_views(75, side, side)
    proj = gsct.Projector(views, side, side, tile=16)
    img = proj.forward(*to_dev(mr, sc, qt))
    assert proj.status().code == 0
    pix = synth.pixel_samples(side, 75, side, side, 48)
    got = img[torch.from_numpy(pix[:, 0]).long().cuda(), torch.from_numpy(pix[:, 1]).long().cuda(),
              torch.from_numpy(pix[:, 2]).long().cuda()].cpu().numpy()
    peak = float(img.abs().max())
    del img, proj
    torch.cuda.empty_cache()
    P, V = orc.params64(mr, sc, qt), orc.views64(views)
    want = orc.project_pixels(P, V, side, side, pix)
    assert np.all(np.abs(got - want) <= IMG_TOL * peak + 2e-3 * np.abs(want)), \
        float(np.abs(got - want).max() / peak)


def test_voxelize_1024_sampled(orc, gsct):
    n = 500000
    mr, sc, qt = synth.gaussians(77, n, scale_median=0.004, scale_sigma_log=0.4)
    grid = synth.cube_grid(1024)
    vox = gsct.Voxelizer(grid)
    vol = vox.forward(*to_dev(mr, sc, qt))
    assert vox.status().code == 0
    idx = synth.voxel_samples(5, (1024, 1024, 1024), 64)
    got = vol[torch.from_numpy(idx[:, 0]).long().cuda(), torch.from_numpy(idx[:, 1]).long().cuda(),
              torch.from_numpy(idx[:, 2]).long().cuda()].cpu().numpy()
    peak = float(vol.abs().max())
    del vol, vox
    torch.cuda.empty_cache()
    want = orc.voxelize_points(orc.params64(mr, sc, qt), grid, idx)
    assert np.all(np.abs(got - want) <= IMG_TOL * peak + 2e-3 * np.abs(want))
