"""ctypes binding of libgsct (include/gsct.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; PyTorch provides device memory
and the current stream.  Importing this module does not need a GPU; calling a compute entry
point without the built library raises immediately (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgsct.so")

GS_OK, GS_ERR_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA = 0, -1, -2, -3
GS_CONE, GS_PARALLEL = 0, 1

# numpy layouts matching the C structs
VIEW_DTYPE = np.dtype([("src", "<f4", (3,)), ("det_center", "<f4", (3,)), ("u", "<f4", (3,)),
                       ("v", "<f4", (3,)), ("mode", "<i4"), ("pad", "<i4", (3,))])
GRID_DTYPE = np.dtype([("dims", "<i4", (3,)), ("origin", "<f4", (3,)), ("voxel", "<f4", (3,))])


class GsGrid(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("origin", ctypes.c_float * 3),
                ("voxel", ctypes.c_float * 3)]


class GsOpts(ctypes.Structure):
    _fields_ = [("cut", ctypes.c_float), ("eps", ctypes.c_float), ("znear", ctypes.c_float),
                ("tile", ctypes.c_int32), ("brick", ctypes.c_int32), ("pad", ctypes.c_int32 * 3)]


class GsStatus(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int32), ("pad", ctypes.c_int32), ("pairs", ctypes.c_int64),
                ("capacity", ctypes.c_int64), ("evals", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 28)]


class GsAdamOpts(ctypes.Structure):
    _fields_ = [("lr_mean", ctypes.c_float), ("lr_rho", ctypes.c_float),
                ("lr_scale", ctypes.c_float), ("lr_quat", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("min_log_scale", ctypes.c_float), ("max_log_scale", ctypes.c_float),
                ("pad", ctypes.c_float * 3)]


class GsFitOpts(ctypes.Structure):
    _fields_ = [("alpha_ssim", ctypes.c_float), ("lr_mean", ctypes.c_float),
                ("lr_rho", ctypes.c_float), ("lr_scale", ctypes.c_float),
                ("lr_quat", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("min_log_scale", ctypes.c_float),
                ("max_log_scale", ctypes.c_float), ("threshold_frac", ctypes.c_float),
                ("density_k", ctypes.c_float), ("data_range", ctypes.c_float),
                ("cut", ctypes.c_float), ("init", ctypes.c_int32), ("brick", ctypes.c_int32)]


class GsInstance(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_views", ctypes.c_int32), ("W", ctypes.c_int32),
                ("H", ctypes.c_int32)]


class GsVoxelInstance(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("grid", GsGrid), ("roi_lo", ctypes.c_int32 * 3),
                ("roi_dim", ctypes.c_int32 * 3)]


class GsDensifyOpts(ctypes.Structure):
    _fields_ = [("grad_threshold", ctypes.c_float), ("grad_scale", ctypes.c_float),
                ("split_scale", ctypes.c_float), ("split_factor", ctypes.c_float),
                ("min_density", ctypes.c_float), ("max_scale", ctypes.c_float),
                ("min_log_scale", ctypes.c_float), ("max_gaussians", ctypes.c_int32),
                ("inherit_moments", ctypes.c_int32), ("pad", ctypes.c_int32 * 3)]


MAX_INSTANCES = 32

assert ctypes.sizeof(GsGrid) == 36 and ctypes.sizeof(GsOpts) == 32
assert ctypes.sizeof(GsInstance) == 16 and ctypes.sizeof(GsVoxelInstance) == 64
assert ctypes.sizeof(GsAdamOpts) == 48
assert ctypes.sizeof(GsDensifyOpts) == 48
assert ctypes.sizeof(GsStatus) == 256

_lib = None

# name -> (restype, argtypes)
_P, _I, _I64, _SZ, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
_OPTS = ctypes.POINTER(GsOpts)
_GRID = ctypes.POINTER(GsGrid)
_I3 = ctypes.POINTER(ctypes.c_int32)
_INST = ctypes.POINTER(GsInstance)
_VINST = ctypes.POINTER(GsVoxelInstance)
SIGNATURES = {
    "gs_version": (ctypes.c_char_p, []),
    "gs_build_arch": (_I, []),
    "gs_read_status": (_I, [_P, _P, ctypes.POINTER(GsStatus)]),
    "gs_last_error": (ctypes.c_char_p, []),
    "gs_memset": (_I, [_P, _I, _SZ, _P]),
    "gs_probe_rate": (_I, [_I, _I, _I, _P, _P]),
    "gs_project_workspace_size": (_SZ, [_I, _I, _I, _I, _OPTS, _I64]),
    "gs_project_count_pairs": (_I, [_P, _P, _P, _I, _P, _I, _I, _I, _OPTS, _P, _SZ, _P,
                                    ctypes.POINTER(ctypes.c_int64)]),
    "gs_project": (_I, [_P, _P, _P, _I, _P, _I, _I, _I, _OPTS, _P, _P, _SZ, _P]),
    "gs_project_backward": (_I, [_P, _P, _P, _I, _P, _I, _I, _I, _OPTS, _P, _P, _P, _P, _I, _I,
                                 _P, _SZ, _P]),
    "gs_project_backward_stats": (_I, [_P, _P, _P, _I, _P, _I, _I, _I, _OPTS, _P, _P, _P, _P,
                                       _P, _P, _I, _I, _P, _SZ, _P]),
    "gs_project_count_evals": (_I, [_P, _P, _P, _I, _P, _I, _I, _I, _OPTS, _P, _SZ, _P]),
    "gs_project_batch_workspace_size": (_SZ, [_INST, _I, _OPTS, _I64]),
    "gs_project_batch_count_pairs": (_I, [_P, _P, _P, _P, _INST, _I, _OPTS, _P, _SZ, _P,
                                          ctypes.POINTER(ctypes.c_int64)]),
    "gs_project_batch": (_I, [_P, _P, _P, _P, _INST, _I, _OPTS, _P, _P, _SZ, _P]),
    "gs_project_batch_backward": (_I, [_P, _P, _P, _P, _INST, _I, _OPTS, _P, _P, _P, _P, _I,
                                       _I, _P, _SZ, _P]),
    "gs_project_batch_backward_stats": (_I, [_P, _P, _P, _P, _INST, _I, _OPTS, _P, _P, _P, _P,
                                             _P, _P, _I, _I, _P, _SZ, _P]),
    "gs_project_batch_count_evals": (_I, [_P, _P, _P, _P, _INST, _I, _OPTS, _P, _SZ, _P]),
    "gs_voxelize_workspace_size": (_SZ, [_I, _GRID, _I3, _I3, _OPTS, _I64]),
    "gs_voxelize_count_pairs": (_I, [_P, _P, _P, _I, _GRID, _I3, _I3, _OPTS, _P, _SZ, _P,
                                     ctypes.POINTER(ctypes.c_int64)]),
    "gs_voxelize": (_I, [_P, _P, _P, _I, _GRID, _I3, _I3, _OPTS, _P, _P, _SZ, _P]),
    "gs_voxelize_backward": (_I, [_P, _P, _P, _I, _GRID, _I3, _I3, _OPTS, _P, _P, _P, _P, _I,
                                  _I, _P, _SZ, _P]),
    "gs_voxelize_count_evals": (_I, [_P, _P, _P, _I, _GRID, _I3, _I3, _OPTS, _P, _SZ, _P]),
    "gs_encode_fp16": (_I, [_P, _P, _P, _I, _P, _P]),
    "gs_decode_fp16": (_I, [_P, _I, _P, _P, _P, _P]),
    "gs_voxelize_fp16_workspace_size": (_SZ, [_I, _GRID, _I3, _I3, _OPTS, _I64]),
    "gs_voxelize_fp16": (_I, [_P, _I, _GRID, _I3, _I3, _OPTS, _P, _P, _SZ, _P]),
    "gs_voxelize_fp16_count_pairs": (_I, [_P, _I, _GRID, _I3, _I3, _OPTS, _P, _SZ, _P,
                                          ctypes.POINTER(ctypes.c_int64)]),
    "gs_voxelize_batch_workspace_size": (_SZ, [_VINST, _I, _OPTS, _I64]),
    "gs_voxelize_batch_count_pairs": (_I, [_P, _P, _P, _VINST, _I, _OPTS, _P, _SZ, _P,
                                           ctypes.POINTER(ctypes.c_int64)]),
    "gs_voxelize_batch": (_I, [_P, _P, _P, _VINST, _I, _OPTS, _P, _P, _SZ, _P]),
    "gs_voxelize_batch_backward": (_I, [_P, _P, _P, _VINST, _I, _OPTS, _P, _P, _P, _P, _I, _I,
                                        _P, _SZ, _P]),
    "gs_voxelize_batch_count_evals": (_I, [_P, _P, _P, _VINST, _I, _OPTS, _P, _SZ, _P]),
    "gs_read_pairs": (_I, [_P, _SZ, _P, _I64, _P, _P, ctypes.POINTER(ctypes.c_int64)]),
    "gs_l1_loss": (_I, [_P, _P, _I64, ctypes.c_float, _P, _P, _I, _P]),
    "gs_tv3d_loss": (_I, [_P, _I, _I, _I, ctypes.c_float, _P, _P, _I, _P]),
    "gs_sse": (_I, [_P, _P, _I64, _P, _P]),
    "gs_ssim_workspace_size": (_SZ, [_I64]),
    "gs_ssim3d_workspace_size": (_SZ, [_I64]),
    "gs_ssim2d_loss": (_I, [_P, _P, _I, _I, _I, ctypes.c_float, ctypes.c_float, _P, _P, _I, _P,
                            _SZ, _P]),
    "gs_l1_ssim2d_loss": (_I, [_P, _P, _I, _I, _I, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, _P, _P, _I, _P, _SZ, _P]),
    "gs_ssim3d_loss": (_I, [_P, _P, _I, _I, _I, ctypes.c_float, ctypes.c_float, _P, _P, _I, _P,
                            _SZ, _P]),
    "gs_ssim2d_loss_noalloc": (_I, [_P, _P, _I, _I, _I, ctypes.c_float, ctypes.c_float, _P, _P,
                                    _I, _P]),
    "gs_adam_step": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I, _P,
                          ctypes.c_void_p, _P]),
    "gs_densify_workspace_size": (_SZ, [_I]),
    "gs_densify": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _I, ctypes.POINTER(GsDensifyOpts), _P, _P,
                        _P, _P, _P, _I, _P, _SZ, _P]),
    "gs_add": (_I, [_P, _P, _I64, _P]),
    "gs_activate": (_I, [_P, _P, _P, _P, _P, _P, _I, _P]),
    "gs_phantom_project": (_I, [_P, _I, _P, _I, _I, _I, _P, _P]),
    "gs_phantom_voxelize": (_I, [_P, _I, _GRID, _P, _P]),
    "gs_fdk_workspace_size": (_SZ, [_I, _I, _I]),
    "gs_fdk": (_I, [_P, _P, _I, _I, _I, _GRID, _P, _P, _SZ, _P]),
    "gs_fit_volume_workspace_size": (_SZ, [_I, _GRID, _I64]),
    "gs_fit_volume": (_I, [_P, _GRID, _I, _I, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "gs_fit_volume_status": (_I, [_P, _SZ, _I, _GRID, _P, ctypes.POINTER(GsStatus)]),
    "gs_grad_init_workspace_size": (_SZ, [_GRID, _I]),
    "gs_grad_init": (_I, [_P, _GRID, _I, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P, _P,
                          _P, _P, _P, _P, _SZ, _P]),
    "gs_gemm_bf16": (_I, [_P, _P, _I, _I, _I, _P, _I, _P, _P, _I, _P, _P]),
    "gs_f32_to_bf16": (_I, [_P, _P, _I64, _P]),
    "gs_transpose_bf16": (_I, [_P, _I, _I, _P, _P]),
    "gs_relu_mask_bf16": (_I, [_P, _P, _I64, _P, _P]),
    "gs_colsum": (_I, [_P, _I, _I, _P, _P]),
    "gs_brick_loss": (_I, [_P, _I, _P, _I, _P, _P, _I, _P, _P]),
    "gs_brick_decode": (_I, [_P, _I, _P, _I, ctypes.c_float, _P, _P, _P, _P]),
    "gs_extract_bricks": (_I, [_P, _I, _I, _I, _P, _I, ctypes.c_float, _P, _P, _P]),
    "gs_adam_flat": (_I, [_P, _P, _P, _P, _I64, _P, ctypes.c_float, ctypes.c_float,
                          ctypes.c_float, ctypes.c_float, _P, _P]),
    "gs_step_incr": (_I, [_P, _P]),
    "gs_mlp_param_count": (_SZ, []),
    "gs_mlp_weight_count": (_SZ, []),
    "gs_mlp_workspace_size": (_SZ, [_I]),
    "gs_mlp_sync_bf16": (_I, [_P, _P, _P]),
    "gs_mlp_forward": (_I, [_P, _P, _P, _I, _P, _P, _SZ, _P, _P]),
    "gs_mlp_backward": (_I, [_P, _P, _I, _P, _P, _P, _SZ, _P, _P]),
    "gs_mlp_train_step": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _I, ctypes.c_float,
                               ctypes.c_float, ctypes.c_float, ctypes.c_float, _P, _P, _SZ, _P,
                               _P]),
    "gs_mlp_infer": (_I, [_P, _P, _P, _I, _P, ctypes.c_float, _P, _P, _P, _P, _SZ, _P, _P]),
    "gs_timing_enable": (None, [_I]),
    "gs_timing_reset": (None, []),
    "gs_timing_read": (_I, [_I, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(ctypes.c_double)]),
    "gs_launch_count": (_I64, []),
}


class GsError(RuntimeError):
    pass


def lib():
    """The loaded libgsct; raises if the CUDA library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GsError(f"libgsct.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc: int, what: str):
    if rc != GS_OK:
        msg = lib().gs_last_error().decode(errors="replace")
        names = {GS_ERR_ARG: "GS_ERR_ARG", GS_ERR_CAPACITY: "GS_ERR_CAPACITY",
                 GS_ERR_CUDA: "GS_ERR_CUDA"}
        raise GsError(f"{what} failed: {names.get(rc, rc)} {msg}")


def opts(cut: float = 3.0, eps: float = 0.0, znear: float = 0.1, tile: int = 16,
         brick: int = 16) -> GsOpts:
    o = GsOpts()
    o.cut, o.eps, o.znear, o.tile, o.brick = cut, eps, znear, tile, brick
    return o


def grid_struct(grid) -> GsGrid:
    g = np.asarray(grid)
    s = GsGrid()
    for k in range(3):
        s.dims[k] = int(g["dims"].ravel()[k])
        s.origin[k] = float(g["origin"].ravel()[k])
        s.voxel[k] = float(g["voxel"].ravel()[k])
    return s


def i3(x):
    a = (ctypes.c_int32 * 3)(*[int(v) for v in x])
    return a


def ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def stream_handle(stream=None) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def read_status(ws, stream=None) -> GsStatus:
    st = GsStatus()
    check(lib().gs_read_status(ptr(ws), stream_handle(stream), ctypes.byref(st)), "gs_read_status")
    return st


def timing_enable(on: bool):
    lib().gs_timing_enable(1 if on else 0)


def timing_reset():
    lib().gs_timing_reset()


def timing_read() -> dict:
    L = lib()
    n = L.gs_timing_read(0, None, None, None)
    names = (ctypes.c_char_p * max(n, 1))()
    launches = (ctypes.c_int64 * max(n, 1))()
    ms = (ctypes.c_double * max(n, 1))()
    n = L.gs_timing_read(n, names, launches, ms)
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(n)}


def launch_count() -> int:
    return int(lib().gs_launch_count())
