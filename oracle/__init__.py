"""FP64 CPU oracle for the FaCT-GS hot path (arXiv 2604.01844) -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may import this
package.  The CUDA product path (paper_2604_01844_gb300) shares no code with it.

The arithmetic lives in gs_oracle.cpp (projection, keys, voxelization, dual-number gradients,
phantom) and losses.py (L1, SSIM 2D/3D, TV, PSNR).  This module compiles the C++ file with g++
and wraps it with ctypes over numpy float64 arrays.

Parity status of each function (what pins it) is listed in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

FP_FIELDS = ["culled", "why", "px", "py", "ca", "cb", "cc", "A", "mu", "Q", "lo_x", "hi_x",
             "lo_y", "hi_y", "ix0", "ix1", "iy0", "iy1", "zc", "sxx", "sxy", "syy"]


def build(force: bool = False) -> str:
    """Compile gs_oracle.cpp into oracle/_build/liboracle.so (g++, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            d, i, ll, P = ctypes.c_double, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p
            sig = {
                "orc_footprints": (None, [i, P, i, P, i, i, d, d, d, P]),
                "orc_project": (ll, [i, P, i, P, i, i, d, d, d, P, i]),
                "orc_project_pixels": (None, [i, P, i, P, i, i, d, d, d, i, P, P, i]),
                "orc_project_ambiguity": (None, [i, P, i, P, i, i, d, d, d, d, d, P, i]),
                "orc_project_pixels_allow": (None, [i, P, i, P, i, i, d, d, d, d, d, i, P, P,
                                                    P, i]),
                "orc_voxelize_points_allow": (None, [i, P, P, d, d, d, i, P, P, P, i]),
                "orc_project_exact": (None, [i, P, i, P, i, i, P, i]),
                "orc_pair_flags": (None, [i, P, i, P, i, i, d, d, d, d, d, P, i, i]),
                "orc_min_q_rect": (d, [d, d, d, d, d, d, d, d, d]),
                "orc_voxel_flags": (None, [i, P, P, P, P, d, d, d, P]),
                "orc_pixel_ray": (None, [P, i, i, i, i, P, P]),
                "orc_keys": (ll, [i, P, i, P, i, i, d, d, d, i, ll, P, P, P, i]),
                "orc_project_grad": (None, [i, P, i, P, i, i, d, d, d, P, P, i]),
                "orc_voxelize": (ll, [i, P, P, P, P, d, P, i]),
                "orc_voxelize_points": (None, [i, P, P, d, i, P, P, i]),
                "orc_voxelize_ambiguity": (None, [i, P, P, P, P, d, d, d, P]),
                "orc_voxel_keys": (ll, [i, P, P, P, P, d, i, ll, P, P, P]),
                "orc_voxelize_grad": (None, [i, P, P, P, P, d, P, P, i]),
                "orc_phantom_project": (None, [i, P, i, P, i, i, P, i]),
                "orc_phantom_raymarch": (None, [i, P, P, i, i, i, i, d, d, ll, P]),
                "orc_phantom_voxelize": (None, [i, P, P, P, i]),
                "orc_rotation": (i, [P, P]),
                "orc_fp_stride": (i, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


# ------------------------------------------------------------------------------------------
# numpy helpers
# ------------------------------------------------------------------------------------------
def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def params64(mean_rho, scale, quat) -> np.ndarray:
    """(N, 11) float64 = p[3], s[3], q[4], rho from the float32 (N, 4) arrays."""
    mean_rho = np.asarray(mean_rho, dtype=np.float64)
    scale = np.asarray(scale, dtype=np.float64)
    quat = np.asarray(quat, dtype=np.float64)
    out = np.concatenate([mean_rho[:, :3], scale[:, :3], quat[:, :4], mean_rho[:, 3:4]], axis=1)
    return np.ascontiguousarray(out)


def views64(views) -> np.ndarray:
    """(V, 13) float64 = src[3], det_center[3], u[3], v[3], mode from the 64-byte view records."""
    v = np.asarray(views)
    out = np.concatenate([v["src"].astype(np.float64), v["det_center"].astype(np.float64),
                          v["u"].astype(np.float64), v["v"].astype(np.float64),
                          v["mode"].astype(np.float64)[:, None]], axis=1)
    return np.ascontiguousarray(out)


def grid64(grid) -> np.ndarray:
    g = np.asarray(grid)
    return np.ascontiguousarray(np.concatenate([g["dims"].astype(np.float64).ravel(),
                                                g["origin"].astype(np.float64).ravel(),
                                                g["voxel"].astype(np.float64).ravel()]))


def _i3(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32).reshape(3))


class Opts:
    def __init__(self, cut: float = 3.0, eps: float = 0.0, znear: float = 0.1):
        self.cut, self.eps, self.znear = float(cut), float(eps), float(znear)


def footprints(P, V, W, H, opts=Opts()):
    """Per (view, Gaussian) footprint record; returns dict of (V, N) arrays."""
    n, nv = P.shape[0], V.shape[0]
    L = lib()
    stride = L.orc_fp_stride()
    out = np.zeros((nv, n, stride))
    L.orc_footprints(n, _p(P), nv, _p(V), W, H, opts.cut, opts.eps, opts.znear, _p(out))
    return {name: out[:, :, k] for k, name in enumerate(FP_FIELDS)}


def project(P, V, W, H, opts=Opts(), nthreads=0):
    """Method (B) images (V, H, W) float64 and the in-cut evaluation count."""
    n, nv = P.shape[0], V.shape[0]
    img = np.zeros((nv, H, W))
    cnt = lib().orc_project(n, _p(P), nv, _p(V), W, H, opts.cut, opts.eps, opts.znear, _p(img),
                            nthreads)
    return img, int(cnt)


def project_pixels(P, V, W, H, pix, opts=Opts(), nthreads=0):
    pix = np.ascontiguousarray(pix, dtype=np.int32)
    out = np.zeros(pix.shape[0])
    lib().orc_project_pixels(P.shape[0], _p(P), V.shape[0], _p(V), W, H, opts.cut, opts.eps,
                             opts.znear, pix.shape[0], _p(pix), _p(out), nthreads)
    return out


def project_pixels_allow(P, V, W, H, pix, rel_band, px_band, opts=Opts(), nthreads=0):
    """Values and guard-band allowances at the pixels pix (view, row, col): what project() and
    project_ambiguity() give there, without whole images."""
    pix = np.ascontiguousarray(pix, dtype=np.int32)
    out = np.zeros(pix.shape[0])
    allow = np.zeros(pix.shape[0])
    lib().orc_project_pixels_allow(P.shape[0], _p(P), V.shape[0], _p(V), W, H, opts.cut,
                                   opts.eps, opts.znear, rel_band, px_band, pix.shape[0], _p(pix),
                                   _p(out), _p(allow), nthreads)
    return out, allow


def voxelize_points_allow(P, grid, idx, rel_band, idx_band, cut=3.0, nthreads=0):
    """Values and guard-band allowances at the voxels idx (z, y, x) of the whole grid: what
    voxelize() and voxelize_ambiguity() give there, without the whole volume."""
    G = grid64(grid)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.zeros(idx.shape[0])
    allow = np.zeros(idx.shape[0])
    lib().orc_voxelize_points_allow(P.shape[0], _p(P), _p(G), cut, rel_band, idx_band,
                                    idx.shape[0], _p(idx), _p(out), _p(allow), nthreads)
    return out, allow


def project_ambiguity(P, V, W, H, rel_band, px_band, opts=Opts(), nthreads=0):
    allow = np.zeros((V.shape[0], H, W))
    lib().orc_project_ambiguity(P.shape[0], _p(P), V.shape[0], _p(V), W, H, opts.cut, opts.eps,
                                opts.znear, rel_band, px_band, _p(allow), nthreads)
    return allow


def pair_flags(P, V, W, H, rel_band, px_band, opts=Opts(), nthreads=0, tile=0):
    """Guard-band flags per (view, Gaussian), (V, N) int32 (see gs_oracle.cpp); tile > 0 adds
    the tight tile rule's flag (16) for tiles of that side."""
    flags = np.zeros((V.shape[0], P.shape[0]), dtype=np.int32)
    lib().orc_pair_flags(P.shape[0], _p(P), V.shape[0], _p(V), W, H, opts.cut, opts.eps,
                         opts.znear, rel_band, px_band, _p(flags), nthreads, int(tile))
    return flags


def min_q_rect(ca, cb, cc, px, py, x0, x1, y0, y1):
    """Minimum of the footprint's quadratic form over a pixel-coordinate rectangle."""
    return lib().orc_min_q_rect(ca, cb, cc, px, py, x0, x1, y0, y1)


TILE_MARGIN = 1e-3  # the tight tile rule lists a tile if min q over it < (1 + margin) Q


def voxel_flags(P, grid, roi_lo, roi_dim, rel_band, idx_band, cut=3.0):
    G = grid64(grid)
    lo, dim = _i3(roi_lo), _i3(roi_dim)
    flags = np.zeros(P.shape[0], dtype=np.int32)
    lib().orc_voxel_flags(P.shape[0], _p(P), _p(G), _p(lo), _p(dim), cut, rel_band, idx_band,
                          _p(flags))
    return flags


def project_exact(P, V, W, H, nthreads=0):
    img = np.zeros((V.shape[0], H, W))
    lib().orc_project_exact(P.shape[0], _p(P), V.shape[0], _p(V), W, H, _p(img), nthreads)
    return img


def pixel_ray(view13, W, H, col, row):
    o, d = np.zeros(3), np.zeros(3)
    v = np.ascontiguousarray(view13, dtype=np.float64)
    lib().orc_pixel_ray(_p(v), W, H, col, row, _p(o), _p(d))
    return o, d


def keys(P, V, W, H, T, opts=Opts(), tight=True):
    """Sorted (key, gaussian) pairs and per-(view, Gaussian) tile counts (V, N); tight=False
    lists every tile of the bounding box."""
    n, nv = P.shape[0], V.shape[0]
    counts = np.zeros((nv, n), dtype=np.int32)
    L = lib()
    t = 1 if tight else 0
    total = L.orc_keys(n, _p(P), nv, _p(V), W, H, opts.cut, opts.eps, opts.znear, T, 0,
                       None, None, _p(counts), t)
    k = np.zeros(max(total, 1), dtype=np.int32)
    v = np.zeros(max(total, 1), dtype=np.int32)
    L.orc_keys(n, _p(P), nv, _p(V), W, H, opts.cut, opts.eps, opts.znear, T, total, _p(k), _p(v),
               _p(counts), t)
    return k[:total], v[:total], counts


def project_grad(P, V, W, H, dimg, opts=Opts(), nthreads=0):
    """d<dimg, I>/d theta, (N, 11) = p[3], s[3], q[4], rho."""
    dimg = np.ascontiguousarray(dimg, dtype=np.float64)
    g = np.zeros((P.shape[0], 11))
    lib().orc_project_grad(P.shape[0], _p(P), V.shape[0], _p(V), W, H, opts.cut, opts.eps,
                           opts.znear, _p(dimg), _p(g), nthreads)
    return g


def voxelize(P, grid, roi_lo=(0, 0, 0), roi_dim=None, cut=3.0, nthreads=0):
    """Volume (dz, dy, dx) float64 over the region of interest and the in-cut evaluation count."""
    G = grid64(grid)
    if roi_dim is None:
        roi_dim = tuple(int(x) for x in np.asarray(grid["dims"]).ravel())
    lo, dim = _i3(roi_lo), _i3(roi_dim)
    vol = np.zeros((dim[2], dim[1], dim[0]))
    cnt = lib().orc_voxelize(P.shape[0], _p(P), _p(G), _p(lo), _p(dim), cut, _p(vol), nthreads)
    return vol, int(cnt)


def voxelize_points(P, grid, idx, cut=3.0, nthreads=0):
    G = grid64(grid)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.zeros(idx.shape[0])
    lib().orc_voxelize_points(P.shape[0], _p(P), _p(G), cut, idx.shape[0], _p(idx), _p(out),
                              nthreads)
    return out


def voxelize_ambiguity(P, grid, roi_lo, roi_dim, rel_band, idx_band, cut=3.0):
    G = grid64(grid)
    lo, dim = _i3(roi_lo), _i3(roi_dim)
    allow = np.zeros((dim[2], dim[1], dim[0]))
    lib().orc_voxelize_ambiguity(P.shape[0], _p(P), _p(G), _p(lo), _p(dim), cut, rel_band,
                                 idx_band, _p(allow))
    return allow


def voxel_keys(P, grid, roi_lo, roi_dim, B, cut=3.0):
    G = grid64(grid)
    lo, dim = _i3(roi_lo), _i3(roi_dim)
    counts = np.zeros(P.shape[0], dtype=np.int32)
    L = lib()
    total = L.orc_voxel_keys(P.shape[0], _p(P), _p(G), _p(lo), _p(dim), cut, B, 0, None, None,
                             _p(counts))
    k = np.zeros(max(total, 1), dtype=np.int32)
    v = np.zeros(max(total, 1), dtype=np.int32)
    L.orc_voxel_keys(P.shape[0], _p(P), _p(G), _p(lo), _p(dim), cut, B, total, _p(k), _p(v),
                     _p(counts))
    return k[:total], v[:total], counts


def voxelize_grad(P, grid, dvol, roi_lo=(0, 0, 0), roi_dim=None, cut=3.0, nthreads=0):
    G = grid64(grid)
    if roi_dim is None:
        roi_dim = tuple(int(x) for x in np.asarray(grid["dims"]).ravel())
    lo, dim = _i3(roi_lo), _i3(roi_dim)
    dvol = np.ascontiguousarray(dvol, dtype=np.float64)
    g = np.zeros((P.shape[0], 11))
    lib().orc_voxelize_grad(P.shape[0], _p(P), _p(G), _p(lo), _p(dim), cut, _p(dvol), _p(g),
                            nthreads)
    return g


def phantom_project(ell, V, W, H, nthreads=0):
    ell = np.ascontiguousarray(ell, dtype=np.float64)
    img = np.zeros((V.shape[0], H, W))
    lib().orc_phantom_project(ell.shape[0], _p(ell), V.shape[0], _p(V), W, H, _p(img), nthreads)
    return img


def phantom_raymarch(ell, view13, W, H, col, row, t0, t1, nsteps):
    ell = np.ascontiguousarray(ell, dtype=np.float64)
    v = np.ascontiguousarray(view13, dtype=np.float64)
    out = np.zeros(1)
    lib().orc_phantom_raymarch(ell.shape[0], _p(ell), _p(v), W, H, col, row, t0, t1, nsteps,
                               _p(out))
    return float(out[0])


def phantom_voxelize(ell, grid, nthreads=0):
    ell = np.ascontiguousarray(ell, dtype=np.float64)
    G = grid64(grid)
    dims = np.asarray(grid["dims"]).ravel()
    vol = np.zeros((dims[2], dims[1], dims[0]))
    lib().orc_phantom_voxelize(ell.shape[0], _p(ell), _p(G), _p(vol), nthreads)
    return vol


def rotation(q) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    R = np.zeros(9)
    ok = lib().orc_rotation(_p(q), _p(R))
    return R.reshape(3, 3) if ok else None
