"""Reference of the FP16 Gaussian codec -- TEST INFRASTRUCTURE ONLY (only tests/, the smoke
check and the benchmark's CPU legs may import it).

Storage format of the paper's compression study (volume fitting and compression section):
each Gaussian's 11 parameters as IEEE 754 binary16, 22 bytes per Gaussian.  The layout is
11 planes of n values (plane k holds parameter k of every Gaussian) in the order
x, y, z, sx, sy, sz, qw, qx, qy, qz, rho; conversion rounds to nearest, ties to even
(numpy's float32 -> float16 conversion, pinned against IEEE bit patterns in the tests).
"""
from __future__ import annotations

import numpy as np

PLANES = ("x", "y", "z", "sx", "sy", "sz", "qw", "qx", "qy", "qz", "rho")
RECORD_BYTES = 2 * len(PLANES)


def planes_of(mean_rho, scale, quat) -> np.ndarray:
    """(11, n) float32 parameter planes of the (n, 4) float32 arrays."""
    mr, sc, q = (np.asarray(a, dtype=np.float32) for a in (mean_rho, scale, quat))
    return np.stack([mr[:, 0], mr[:, 1], mr[:, 2], sc[:, 0], sc[:, 1], sc[:, 2], q[:, 0],
                     q[:, 1], q[:, 2], q[:, 3], mr[:, 3]])


def encode(mean_rho, scale, quat) -> np.ndarray:
    """(11, n) uint16 binary16 bit patterns (values beyond the binary16 range become inf)."""
    with np.errstate(over="ignore"):
        return planes_of(mean_rho, scale, quat).astype(np.float16).view(np.uint16)


def decode(bits: np.ndarray):
    """(mean_rho, scale, quat) (n, 4) float32 from (11, n) uint16 planes; scale[:, 3] = 0."""
    p = np.asarray(bits, dtype=np.uint16).view(np.float16).astype(np.float32)
    n = p.shape[1]
    mr = np.stack([p[0], p[1], p[2], p[10]], 1)
    sc = np.stack([p[3], p[4], p[5], np.zeros(n, np.float32)], 1)
    q = np.stack([p[6], p[7], p[8], p[9]], 1)
    return mr, sc, q
