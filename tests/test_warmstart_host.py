"""Host-side pieces of the prior-volume warm start: the synthetic priors and the study's
iteration ratio (no GPU)."""
import numpy as np
import pytest

import synth
from paper_2604_01844_gb300 import warmstart as W


def test_thick_slices_factor_one_is_identity():
    v = np.random.default_rng(0).random((11, 4, 5))
    np.testing.assert_allclose(synth.thick_slices(v, 1), v, rtol=1e-6)


@pytest.mark.parametrize("nz,factor", [(23, 5), (20, 5), (17, 4), (9, 3)])
def test_thick_slices_reproduces_linear_profiles(nz, factor):
    # a profile linear in z survives group averaging (group mean = value at the group centre)
    # and linear interpolation between group centres; beyond the outer centres it is held
    z = np.arange(nz, dtype=np.float64)
    v = (0.3 * z + 1.0)[:, None, None] * np.ones((1, 3, 2))
    out = synth.thick_slices(v, factor)
    starts = np.arange(0, nz, factor)
    c0 = (min(factor, nz) - 1) / 2.0
    c1 = starts[-1] + (nz - starts[-1] - 1) / 2.0
    inner = (z >= c0) & (z <= c1)
    np.testing.assert_allclose(out[inner], v[inner], rtol=1e-6)
    np.testing.assert_allclose(out[z < c0], 0.3 * c0 + 1.0, rtol=1e-6)
    np.testing.assert_allclose(out[z > c1], 0.3 * c1 + 1.0, rtol=1e-6)


def test_thick_slices_blurs_a_thin_slab():
    v = np.zeros((20, 2, 2))
    v[7] = 1.0
    out = synth.thick_slices(v, 5)
    assert out[7, 0, 0] < 0.5 and out.sum() > 0
    # the slab's mass spreads over its group's neighbourhood and stays within two groups
    assert np.all(out[:2] == 0) and np.all(out[15:] == 0)


def test_perturbed_phantom_is_seeded_and_bounded():
    ell = synth.ellipsoid_phantom(1, 40)
    a = synth.perturbed_phantom(ell, 5)
    b = synth.perturbed_phantom(ell, 5)
    assert np.array_equal(a, b)
    assert 25 <= a.shape[0] <= 40 and a.shape[1] == ell.shape[1]
    none = synth.perturbed_phantom(ell, 5, att_jitter=0, shift=0, axis_jitter=0, drop_frac=0)
    np.testing.assert_array_equal(none, ell)


def _traj(scores):
    return [(5 * k, float(k), p, s) for k, (p, s) in enumerate(scores)]


def test_tau_iter():
    cold = _traj([(20, .5), (25, .7), (30, .8), (31, .85), (32, .9)])  # n_iter = 20
    warm = _traj([(28, .75), (31, .86), (32.5, .9), (33, .95)])
    assert W.tau_iter(cold, warm, 20, 2) == 10 / 20
    assert W.tau_iter(cold, warm, 20, 3) == 10 / 20
    # the cold start's best is taken within n_iter only
    assert W.tau_iter(cold, warm, 10, 2) == 5 / 10
    assert W.tau_iter(cold, warm, 5, 2) == 0.0
    assert W.tau_iter(cold, _traj([(10, .1), (11, .2)]), 20, 2) is None
    assert W.first_reaching(warm, 2, 31.0) == (5, 1.0)
    assert W.first_reaching(warm, 2, 40.0) is None
