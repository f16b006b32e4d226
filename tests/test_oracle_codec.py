"""Pins of the FP16 codec reference against IEEE 754 binary16 facts (bit patterns fixed by the
standard: sign, 5 exponent bits with bias 15, 10 fraction bits)."""
import numpy as np

from oracle import codec as C

# (float32 value, binary16 bits): exact values, extremes, subnormals and ties to even
GOLDEN = [
    (1.0, 0x3C00), (-2.0, 0xC000), (0.5, 0x3800), (65504.0, 0x7BFF), (0.0, 0x0000),
    (-0.0, 0x8000), (2.0 ** -14, 0x0400),            # smallest normal
    (2.0 ** -24, 0x0001),                              # smallest subnormal
    (2.0 ** -25, 0x0000),                              # half of it: tie, rounds to even (0)
    (3 * 2.0 ** -25, 0x0002),                          # 1.5 x smallest: tie, rounds to even (2)
    (1.0 + 2.0 ** -11, 0x3C00),                        # tie between 1 and 1 + 2^-10: even
    (1.0 + 3 * 2.0 ** -11, 0x3C02),                    # tie between 1+2^-10 and 1+2^-9: even
    (1.0 + 2.0 ** -11 + 2.0 ** -20, 0x3C01),           # just above the tie: up
    (65520.0, 0x7C00),                                 # rounds past the largest finite: inf
    (0.1, 0x2E66), (0.3333333, 0x3555),
]


def _one(x):
    mr = np.array([[x, 0, 0, 0]], np.float32)
    z = np.zeros((1, 4), np.float32)
    return int(C.encode(mr, z, z)[0, 0])


def test_golden_bit_patterns():
    for x, bits in GOLDEN:
        assert _one(x) == bits, (x, hex(_one(x)), hex(bits))


def test_round_trip_error_bound_and_layout():
    rng = np.random.default_rng(0)
    n = 5000
    mr = rng.uniform(-1, 1, (n, 4)).astype(np.float32)
    mr[:, 3] = rng.uniform(0, 2, n)
    sc = np.exp(rng.uniform(np.log(1e-3), np.log(0.5), (n, 4))).astype(np.float32)
    q = rng.standard_normal((n, 4)).astype(np.float32)
    bits = C.encode(mr, sc, q)
    assert bits.shape == (11, n) and bits.nbytes == C.RECORD_BYTES * n == 22 * n
    dmr, dsc, dq = C.decode(bits)
    # normal binary16 values: relative rounding error at most 2^-11
    for a, b in ((mr, dmr), (sc[:, :3], dsc[:, :3]), (q, dq)):
        big = np.abs(a) >= 2.0 ** -14
        assert np.all(np.abs(b - a)[big] <= 2.0 ** -11 * np.abs(a)[big])
        assert np.all(np.abs(b - a)[~big] <= 2.0 ** -25)
    # plane order: x, y, z, sx, sy, sz, qw, qx, qy, qz, rho
    order = [mr[:, 0], mr[:, 1], mr[:, 2], sc[:, 0], sc[:, 1], sc[:, 2], q[:, 0], q[:, 1],
             q[:, 2], q[:, 3], mr[:, 3]]
    for k, col in enumerate(order):
        assert np.array_equal(bits[k], C.encode(np.stack([col, col, col, col], 1), sc, q)[0])
    assert np.all(dsc[:, 3] == 0)
    # decode is exact on representable values: a second round trip changes nothing
    assert np.array_equal(C.encode(dmr, dsc, dq), bits)


def _golden_sizes():
    import pathlib

    out = {}
    for line in (pathlib.Path(__file__).parent / "golden" / "compression_sizes.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_paper_storage_sizes():
    """The codec's byte count reproduces the sizes printed for the compression study: 22 bytes
    per Gaussian, 0.84 MB for 40,000 Gaussians, against 64 MB for the raw 256^3 float32 volume."""
    g = _golden_sizes()
    n = int(g["gaussians"])
    rng = np.random.default_rng(3)
    mr = rng.uniform(-1, 1, (n, 4)).astype(np.float32)
    sc = rng.uniform(1e-3, 0.1, (n, 4)).astype(np.float32)
    q = rng.standard_normal((n, 4)).astype(np.float32)
    bits = C.encode(mr, sc, q)
    assert bits.shape[0] == int(g["values_per_gaussian"])
    assert bits.nbytes == int(g["bytes_per_gaussian"]) * n
    assert round(bits.nbytes / 2 ** 20, 2) == g["gaussians_fp16_mb"]
    assert int(g["volume_side"]) ** 3 * 4 / 2 ** 20 == g["raw_float32_mb"]
