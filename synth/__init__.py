"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module only draws random numbers and lays out scanner geometry; it contains none of
the method's arithmetic (no projection, no Gaussian evaluation).  Both sides receive the
same float32 arrays produced here.

Layouts (the C ABI in include/gsct.h uses the same ones):
  mean_rho  float32 (N, 4)  = (x, y, z, rho)          -- Gaussian centre and density (Eq. 1)
  scale     float32 (N, 4)  = (sx, sy, sz, 0)         -- per-axis standard deviations, > 0
  quat      float32 (N, 4)  = (w, x, y, z)            -- rotation, not necessarily unit
  views     VIEW_DTYPE (V,)  = 64-byte records: src[3], det_center[3], u[3], v[3], mode, pad[3]
  grid      GRID_DTYPE       = dims (nx, ny, nz), origin[3], voxel[3]

Workload recipes (sizes and distributions) follow the paper's settings (Sec. 4.1, 4.2):
cone-beam views evenly spaced over 360 degrees, 75 views of 512^2 etc.
"""
from __future__ import annotations

import numpy as np

CONE = 0
PARALLEL = 1

VIEW_DTYPE = np.dtype(
    [
        ("src", "<f4", (3,)),
        ("det_center", "<f4", (3,)),
        ("u", "<f4", (3,)),
        ("v", "<f4", (3,)),
        ("mode", "<i4"),
        ("pad", "<i4", (3,)),
    ],
    align=False,
)
assert VIEW_DTYPE.itemsize == 64

# Geometry constants of the normalised scanner: volume box [-1, 1]^3, rotation axis z,
# source 4 units and detector 2 units from the axis, detector side 3 units.
D_SO = 4.0
D_OD = 2.0
DET_LEN = 3.0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_ball(rng: np.random.Generator, n: int, radius: float) -> np.ndarray:
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    return d * r[:, None]


def random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed unit quaternions (Shoemake's subgroup algorithm), as (w, x, y, z)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    x = a * np.sin(2 * np.pi * u2)
    y = a * np.cos(2 * np.pi * u2)
    z = b * np.sin(2 * np.pi * u3)
    w = b * np.cos(2 * np.pi * u3)
    return np.stack([w, x, y, z], axis=1)


def gaussians(
    seed: int,
    n: int,
    radius: float = 0.8,
    scale_median: float = 0.02,
    scale_sigma_log: float = 0.5,
    rho_range: tuple[float, float] = (0.05, 1.0),
    isotropic: bool = False,
    identity_rotation: bool = False,
):
    """Random anisotropic Gaussians: centres uniform in a ball, log-normal per-axis scales,
    uniformly random rotations, densities uniform in rho_range.  Returns float32 arrays
    (mean_rho, scale, quat), each (n, 4)."""
    rng = _rng(seed)
    p = uniform_ball(rng, n, radius)
    if isotropic:
        s1 = scale_median * np.exp(scale_sigma_log * rng.standard_normal(n))
        s = np.repeat(s1[:, None], 3, axis=1)
    else:
        s = scale_median * np.exp(scale_sigma_log * rng.standard_normal((n, 3)))
    q = random_quaternions(rng, n)
    if identity_rotation:
        q = np.zeros((n, 4))
        q[:, 0] = 1.0
    rho = rng.uniform(rho_range[0], rho_range[1], n)
    mean_rho = np.concatenate([p, rho[:, None]], axis=1).astype(np.float32)
    scale = np.concatenate([s, np.zeros((n, 1))], axis=1).astype(np.float32)
    quat = q.astype(np.float32)
    return mean_rho, scale, quat


def cone_views(n_views: int, W: int, H: int, d_so: float = D_SO, d_od: float = D_OD,
               det_len: float = DET_LEN, angle0: float = 0.0, span: float = 2 * np.pi) -> np.ndarray:
    """Circular cone-beam trajectory about the z axis: view k at angle angle0 + span*k/n_views
    (no endpoint), flat detector perpendicular to the central ray, square pixels of pitch
    det_len / max(W, H)."""
    pitch = det_len / max(W, H)
    out = np.zeros(n_views, dtype=VIEW_DTYPE)
    for k in range(n_views):
        th = angle0 + span * k / n_views
        c, s = np.cos(th), np.sin(th)
        out[k]["src"] = (d_so * c, d_so * s, 0.0)
        out[k]["det_center"] = (-d_od * c, -d_od * s, 0.0)
        out[k]["u"] = (-s * pitch, c * pitch, 0.0)
        out[k]["v"] = (0.0, 0.0, pitch)
        out[k]["mode"] = CONE
    return out


def parallel_views(n_views: int, W: int, H: int, det_len: float = 2.0 * 1.5,
                   angle0: float = 0.0, span: float = np.pi) -> np.ndarray:
    """Parallel-beam views: rays perpendicular to the detector plane."""
    pitch = det_len / max(W, H)
    out = np.zeros(n_views, dtype=VIEW_DTYPE)
    for k in range(n_views):
        th = angle0 + span * k / n_views
        c, s = np.cos(th), np.sin(th)
        out[k]["src"] = (-c, -s, 0.0)  # unused for parallel beams
        out[k]["det_center"] = (-2.0 * c, -2.0 * s, 0.0)
        out[k]["u"] = (-s * pitch, c * pitch, 0.0)
        out[k]["v"] = (0.0, 0.0, pitch)
        out[k]["mode"] = PARALLEL
    return out


GRID_DTYPE = np.dtype([("dims", "<i4", (3,)), ("origin", "<f4", (3,)), ("voxel", "<f4", (3,))])


def cube_grid(n: int, half: float = 1.0) -> np.ndarray:
    """n^3 voxels covering [-half, half]^3; voxel (ix, iy, iz) centre = origin + (idx + 1/2) * voxel."""
    g = np.zeros((), dtype=GRID_DTYPE)
    g["dims"] = (n, n, n)
    g["origin"] = (-half, -half, -half)
    g["voxel"] = (2 * half / n,) * 3
    return g


def ellipsoid_phantom(seed: int, n: int, centre_radius: float = 0.5,
                      axis_range: tuple[float, float] = (0.05, 0.35), max_radius: float = 0.85):
    """Random-ellipsoid phantom: centres uniform in a ball, semi-axes uniform in axis_range and
    shrunk so each ellipsoid lies inside a ball of max_radius, uniformly random rotations,
    attenuation U(0, 1).  Returns float64 (n, 11) rows = centre[3], semi-axes[3], quat(w,x,y,z), att."""
    rng = _rng(seed)
    c = uniform_ball(rng, n, centre_radius)
    ax = rng.uniform(axis_range[0], axis_range[1], (n, 3))
    room = max_radius - np.linalg.norm(c, axis=1)
    shrink = np.minimum(1.0, room / ax.max(axis=1))
    ax = ax * shrink[:, None]
    q = random_quaternions(rng, n)
    att = rng.uniform(0.0, 1.0, n)
    return np.concatenate([c, ax, q, att[:, None]], axis=1)


def pixel_samples(seed: int, n_views: int, W: int, H: int, count: int) -> np.ndarray:
    """Random (view, row, col) triples, int32 (count, 3)."""
    rng = _rng(seed)
    return np.stack([rng.integers(0, n_views, count), rng.integers(0, H, count),
                     rng.integers(0, W, count)], axis=1).astype(np.int32)


def voxel_samples(seed: int, dims, count: int) -> np.ndarray:
    """Random (z, y, x) triples, int32 (count, 3)."""
    rng = _rng(seed)
    return np.stack([rng.integers(0, dims[2], count), rng.integers(0, dims[1], count),
                     rng.integers(0, dims[0], count)], axis=1).astype(np.int32)


def tiny_config(seed: int = 0):
    """2,000 Gaussians in a radius-0.8 ball, log-normal scales (median 0.02, sigma_log 0.5),
    random rotations, densities U(0.05, 1); 8 cone views of 64x64; 64^3 grid."""
    g = gaussians(seed, 2000)
    return g, cone_views(8, 64, 64), cube_grid(64)


def batch_specs(seeds=range(100, 116), sides=(128, 192, 256, 320, 384),
                detectors=(256, 320, 384, 448, 512), views=(25, 75), gaussians=(10000, 80000),
                n_ellipsoids=40):
    """Uneven reconstructions for the batched form: per seed, a volume side, a detector side
    and a view count drawn uniformly from the given sets/ranges, a Gaussian budget uniform in
    the given range, and a random-ellipsoid phantom of that seed."""
    out = []
    for s in seeds:
        rng = _rng(s)
        out.append(dict(seed=int(s), side=int(rng.choice(sides)),
                        det=int(rng.choice(detectors)),
                        n_views=int(rng.integers(views[0], views[1] + 1)),
                        n=int(rng.integers(gaussians[0], gaussians[1] + 1)),
                        n_ellipsoids=int(n_ellipsoids)))
    return out


def perturbed_phantom(ell: np.ndarray, seed: int, att_jitter: float = 0.2,
                      shift: float = 0.01, axis_jitter: float = 0.05,
                      drop_frac: float = 0.1) -> np.ndarray:
    """A prior for a phantom (an earlier scan of the same object): every ellipsoid's
    attenuation scaled by U(1 - att_jitter, 1 + att_jitter), its centre shifted by
    N(0, shift^2) per axis, its semi-axes scaled by U(1 - axis_jitter, 1 + axis_jitter), and a
    fraction drop_frac of the ellipsoids removed.  Rows as in ellipsoid_phantom."""
    rng = _rng(seed)
    e = np.array(ell, dtype=np.float64, copy=True)
    n = e.shape[0]
    e[:, 10] *= rng.uniform(1.0 - att_jitter, 1.0 + att_jitter, n)
    e[:, 0:3] += rng.normal(0.0, shift, (n, 3))
    e[:, 3:6] *= rng.uniform(1.0 - axis_jitter, 1.0 + axis_jitter, (n, 3))
    keep = rng.random(n) >= drop_frac
    return e[keep]


def thick_slices(vol: np.ndarray, factor: int) -> np.ndarray:
    """A lower longitudinal resolution scan of the same volume ([z][y][x]), resized back to its
    grid: slices averaged in consecutive groups of `factor` (a trailing partial group over its
    own slices), then linearly interpolated in z from the groups' centres to every slice's
    centre (held constant beyond the first and last group centre).  Works slice by slice, so
    a 512^3 volume needs no more than its output's memory."""
    v = np.asarray(vol)
    nz = v.shape[0]
    starts = list(range(0, nz, factor))
    groups = [v[a:a + factor].astype(np.float64).mean(axis=0) for a in starts]
    centres = [a + (min(a + factor, nz) - a - 1) / 2.0 for a in starts]
    out = np.empty(v.shape, dtype=np.float32)
    g = 0
    for z in range(nz):
        while g + 2 < len(starts) and centres[g + 1] <= z:
            g += 1
        if len(starts) == 1 or z <= centres[0]:
            out[z] = groups[0]
        elif z >= centres[-1]:
            out[z] = groups[-1]
        else:
            t = (z - centres[g]) / (centres[g + 1] - centres[g])
            out[z] = (1.0 - t) * groups[g] + t * groups[g + 1]
    return out
