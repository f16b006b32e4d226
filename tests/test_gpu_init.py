"""Parity of the phantom generator, FDK and the gradient initialiser with the CPU oracle."""
import ctypes

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


def _s():
    return torch.cuda.current_stream().cuda_stream


def test_phantom_project_and_voxelize(orc, gsct):
    B = gsct.binding
    ell = synth.ellipsoid_phantom(1, 40)
    W = H = 64
    views = synth.cone_views(6, W, H)
    d_ell = torch.from_numpy(ell.astype(np.float32)).cuda()
    d_views = gsct.views_to_device(views, "cuda")
    img = torch.empty((6, H, W), device="cuda")
    B.check(B.lib().gs_phantom_project(B.ptr(d_ell), 40, B.ptr(d_views), 6, W, H, B.ptr(img),
                                       _s()), "phantom_project")
    want = orc.phantom_project(ell.astype(np.float32).astype(np.float64), orc.views64(views), W, H)
    got = img.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max()
    grid = synth.cube_grid(48)
    vol = torch.empty((48, 48, 48), device="cuda")
    B.check(B.lib().gs_phantom_voxelize(B.ptr(d_ell), 40, ctypes.byref(B.grid_struct(grid)),
                                        B.ptr(vol), _s()), "phantom_voxelize")
    want_v = orc.phantom_voxelize(ell.astype(np.float32).astype(np.float64), grid)
    diff = np.abs(vol.cpu().numpy() - want_v) > 1e-5
    # only voxel centres on an ellipsoid surface (FP32 vs FP64 inside test) may differ
    assert diff.mean() < 1e-3


def test_fdk_matches_oracle(orc, gsct):
    from oracle.init import fdk
    B = gsct.binding
    ell = synth.ellipsoid_phantom(2, 10)
    W, H, nv = 64, 48, 24
    views = synth.cone_views(nv, W, H)
    V = orc.views64(views)
    proj = orc.phantom_project(ell, V, W, H).astype(np.float32)
    grid = synth.cube_grid(40)
    want = fdk(proj.astype(np.float64), V, grid)
    d_proj = torch.from_numpy(proj).cuda()
    d_views = gsct.views_to_device(views, "cuda")
    ws = torch.empty(B.lib().gs_fdk_workspace_size(nv, W, H), dtype=torch.uint8, device="cuda")
    vol = torch.empty((40, 40, 40), device="cuda")
    B.check(B.lib().gs_fdk(B.ptr(d_proj), B.ptr(d_views), nv, W, H,
                           ctypes.byref(B.grid_struct(grid)), B.ptr(vol), B.ptr(ws), ws.numel(),
                           _s()), "gs_fdk")
    got = vol.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max(), \
        float(np.abs(got - want).max() / np.abs(want).max())


@pytest.mark.parametrize("n", [1, 500, 4000])
def test_grad_init_matches_oracle(orc, gsct, n):
    from oracle.init import grad_init
    B = gsct.binding
    rng = np.random.default_rng(n)
    grid = synth.cube_grid(32)
    ell = synth.ellipsoid_phantom(3, 12)
    V = orc.phantom_voxelize(ell, grid).astype(np.float32)
    V += (0.01 * rng.standard_normal(V.shape)).astype(np.float32)
    u = rng.random((n, 4)).astype(np.float32)
    mr, sc, q, idx, margin = grad_init(V, grid, n, 0.05, 0.15, 1e-4, u)
    d_V = torch.from_numpy(V).cuda()
    d_u = torch.from_numpy(u).cuda()
    out = [torch.empty((n, 4), device="cuda") for _ in range(3)]
    vox = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = torch.empty(B.lib().gs_grad_init_workspace_size(ctypes.byref(B.grid_struct(grid)), n),
                     dtype=torch.uint8, device="cuda")
    B.check(B.lib().gs_grad_init(B.ptr(d_V), ctypes.byref(B.grid_struct(grid)), n, 0.05, 0.15,
                                 1e-4, B.ptr(d_u), *[B.ptr(t) for t in out], B.ptr(vox),
                                 B.ptr(ws), ws.numel(), _s()), "gs_grad_init")
    got_idx = vox.cpu().numpy()
    safe = margin > 1e-12
    assert safe.mean() > 0.99
    assert np.array_equal(got_idx[safe], idx[safe])  # integer decision: bit-exact
    g_mr, g_sc, g_q = (t.cpu().numpy().astype(np.float64) for t in out)
    np.testing.assert_allclose(g_mr[safe, :3], mr[safe, :3], rtol=0, atol=1e-6)
    np.testing.assert_allclose(g_mr[safe, 3], mr[safe, 3], rtol=1e-5, atol=1e-6)
    if n > 1:
        np.testing.assert_allclose(g_sc[safe, 0], sc[safe, 0], rtol=1e-4, atol=1e-6)
    assert np.all(g_q[:, 0] == 1) and np.all(g_q[:, 1:] == 0)
