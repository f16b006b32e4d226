"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a, loads, and
exports every function include/*.h declares; struct layouts agree; argument errors are caught
on the host before any launch."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2604_01844_gb300 import build

    return build.build()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(gs_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(built):
    names = declared_functions()
    assert len(names) >= 15
    L = ctypes.CDLL(built)
    for n in sorted(names):
        assert hasattr(L, n), n


def test_binding_covers_header(built):
    from paper_2604_01844_gb300 import binding

    assert declared_functions() <= set(binding.SIGNATURES)


def test_build_arch_and_version(built):
    from paper_2604_01844_gb300 import binding

    L = binding.lib()
    assert L.gs_build_arch() == 103
    assert b"sm_103a" in L.gs_version()


def test_struct_layouts():
    import numpy as np

    import synth
    from paper_2604_01844_gb300 import binding

    assert binding.VIEW_DTYPE.itemsize == 64 and synth.VIEW_DTYPE == binding.VIEW_DTYPE
    assert np.dtype(synth.GRID_DTYPE).itemsize == ctypes.sizeof(binding.GsGrid)


def test_workspace_size_arithmetic(built):
    from paper_2604_01844_gb300 import binding

    L = binding.lib()
    o = binding.opts(tile=16)
    a = L.gs_project_workspace_size(1000, 8, 64, 64, ctypes.byref(o), 0)
    b = L.gs_project_workspace_size(1000, 8, 64, 64, ctypes.byref(o), 100000)
    assert a > 0 and b >= a + 100000 * 16
    bad = binding.opts(tile=12)
    assert L.gs_project_workspace_size(1000, 8, 64, 64, ctypes.byref(bad), 0) == 0
    g = binding.GsGrid()
    for k in range(3):
        g.dims[k], g.origin[k], g.voxel[k] = 64, -1.0, 2 / 64
    lo, dim = binding.i3((0, 0, 0)), binding.i3((64, 64, 64))
    assert L.gs_voxelize_workspace_size(1000, ctypes.byref(g), lo, dim, ctypes.byref(o), 0) > 0
    dim_bad = binding.i3((65, 64, 64))
    assert L.gs_voxelize_workspace_size(1000, ctypes.byref(g), lo, dim_bad, ctypes.byref(o), 0) == 0


def test_argument_errors_are_host_side(built):
    from paper_2604_01844_gb300 import binding

    L = binding.lib()
    o = binding.opts()
    # null parameter pointers with n > 0
    rc = L.gs_project(None, None, None, 10, None, 1, 8, 8, ctypes.byref(o), None, None, 0, None)
    assert rc == binding.GS_ERR_ARG
    # misaligned workspace pointer
    rc = L.gs_project(16, 16, 16, 10, 16, 1, 8, 8, ctypes.byref(o), 16, 17, 1 << 20, None)
    assert rc == binding.GS_ERR_ARG
    # image losses: null inputs, a non-positive data range, a workspace below the 3 maps
    rc = L.gs_l1_ssim2d_loss(None, 16, 1, 8, 8, 1.0, 1.0, 0.2, 16, 16, 0, 16, 1 << 20, None)
    assert rc == binding.GS_ERR_ARG
    rc = L.gs_l1_ssim2d_loss(16, 16, 1, 8, 8, 0.0, 1.0, 0.2, 16, 16, 0, 16, 1 << 20, None)
    assert rc == binding.GS_ERR_ARG
    rc = L.gs_l1_ssim2d_loss(16, 16, 1, 8, 8, 1.0, 1.0, 0.2, 16, 16, 0, 16, 64, None)
    assert rc == binding.GS_ERR_CAPACITY
    # TV: more than 2^31 - 1 (y, z) rows is refused before any launch
    rc = L.gs_tv3d_loss(16, 4, 65536, 32768, 1.0, 16, 16, 0, None)
    assert rc == binding.GS_ERR_ARG


def test_batch_table_validation(built):
    """The batched rasterizer rejects bad instance tables on the host; a batch of one sizes its
    workspace like the single-instance call."""
    from paper_2604_01844_gb300 import binding

    L = binding.lib()
    o = binding.opts()
    t = (binding.GsInstance * 33)()
    for i in range(33):
        t[i].n, t[i].n_views, t[i].W, t[i].H = 100, 2, 40, 30
    one = L.gs_project_workspace_size(100, 2, 40, 30, ctypes.byref(o), 5000)
    assert L.gs_project_batch_workspace_size(t, 1, ctypes.byref(o), 5000) == one > 0
    assert L.gs_project_batch_workspace_size(t, 32, ctypes.byref(o), 0) > one
    assert L.gs_project_batch_workspace_size(t, 33, ctypes.byref(o), 0) == 0
    assert L.gs_project_batch_workspace_size(t, 0, ctypes.byref(o), 0) == 0
    t[3].n = 0  # an empty instance is allowed
    assert L.gs_project_batch_workspace_size(t, 8, ctypes.byref(o), 0) > 0
    t[5].n_views = 0
    assert L.gs_project_batch_workspace_size(t, 8, ctypes.byref(o), 0) == 0
    t[5].n_views, t[6].W = 2, 40000
    assert L.gs_project_batch_workspace_size(t, 8, ctypes.byref(o), 0) == 0
    t[6].W = 40
    rc = L.gs_project_batch(None, None, None, None, t, 8, ctypes.byref(o), 16, 16, 1 << 20, None)
    assert rc == binding.GS_ERR_ARG


def test_voxel_batch_table_validation(built):
    from paper_2604_01844_gb300 import binding

    L = binding.lib()
    o = binding.opts()
    g = binding.GsGrid()
    for k in range(3):
        g.dims[k], g.origin[k], g.voxel[k] = 64, -1.0, 2 / 64
    t = (binding.GsVoxelInstance * 33)()
    for i in range(33):
        t[i].n, t[i].grid = 100, g
        for k in range(3):
            t[i].roi_lo[k], t[i].roi_dim[k] = 0, 64
    one = L.gs_voxelize_workspace_size(100, ctypes.byref(g), binding.i3((0, 0, 0)),
                                       binding.i3((64, 64, 64)), ctypes.byref(o), 777)
    assert L.gs_voxelize_batch_workspace_size(t, 1, ctypes.byref(o), 777) == one > 0
    assert L.gs_voxelize_batch_workspace_size(t, 33, ctypes.byref(o), 0) == 0
    t[2].roi_lo[1] = 1  # region leaves the grid
    assert L.gs_voxelize_batch_workspace_size(t, 4, ctypes.byref(o), 0) == 0
    t[2].roi_lo[1], t[2].n = 0, 0
    assert L.gs_voxelize_batch_workspace_size(t, 4, ctypes.byref(o), 0) > 0


def test_mlp_network_layout_and_host_errors(built):
    """The flat parameter layout's size, and the MLP entry points' argument checks (batch not
    a multiple of 128, workspace too small) answered on the host before any launch."""
    from paper_2604_01844_gb300 import binding as B

    L = B.lib()
    weights = 256 * 4096 + 2 * 256 * 256 + 384 * 256
    assert L.gs_mlp_weight_count() == weights
    assert L.gs_mlp_param_count() == weights + 3 * 256 + 384
    assert L.gs_mlp_workspace_size(100) == 0 and L.gs_mlp_workspace_size(0) == 0
    ws = L.gs_mlp_workspace_size(256)
    assert ws > 256 * 4096 * 2  # holds at least the transposed input of the first layer
    fake = 1 << 20  # never dereferenced: the checks fail first
    rc = L.gs_mlp_forward(fake, fake, fake, 100, fake, fake, ws, fake, None)
    assert rc == B.GS_ERR_ARG
    rc = L.gs_mlp_forward(fake, fake, fake, 256, fake, fake, ws - 1, fake, None)
    assert rc == B.GS_ERR_CAPACITY
    rc = L.gs_mlp_train_step(fake, fake, fake, fake, fake, fake, fake, None, 256, 1e-3, 0.9,
                             0.999, 1e-8, fake, fake, ws, fake, None)
    assert rc == B.GS_ERR_ARG
