"""The oracle's explicit store error (the noise-injection estimate of the second-order term
of Eq. 6), on the CPU: the draw is the stated transform of the Philox block (pinned by the
published Philox known answers), uniform with unit variance, antithetic pairs cancel
exactly, sigma scales per field, and a rollout with sign 0 is the plain FP64 rollout."""
import numpy as np
import pytest


def test_noise_is_the_stated_transform_of_the_philox_block(oracle):
    s = oracle.add_noise(3, "corotated", np.zeros((5, 24)), 7, 0xDEADBEEF12345678, [1.0] * 4, 1.0)
    key = (0x12345678, 0xDEADBEEF)
    for p in range(5):
        for c in range(24):
            blk = oracle.philox((p, 7, c // 4, 0xA5), key)
            k = blk[c % 4] >> 9
            xi = (2.0 * (k + 0.5) / 2.0 ** 23 - 1.0) * np.sqrt(3.0)
            assert s[p, c] == xi


def test_noise_is_uniform_with_unit_variance_and_antithetic(oracle):
    # 2D fluid: x (2), v (2), C (4), J (1) = 9 components
    a = oracle.add_noise(2, "fluid", np.zeros((100_000, 9)), 3, 9, [1.0] * 4, 1.0)
    n = a.size
    assert abs(a.mean()) <= 4 / np.sqrt(n)
    assert abs(a.var() - 1.0) <= 4 * np.sqrt(0.8 / n)  # var of xi^2 for a unit-variance uniform: 4/5
    assert np.abs(a).max() < np.sqrt(3.0)
    hist, _ = np.histogram(a, bins=10, range=(-np.sqrt(3), np.sqrt(3)))
    assert np.all(np.abs(hist - n / 10) <= 5 * np.sqrt(n / 10))
    s0 = np.random.default_rng(1).normal(size=(50, 9))
    sigma = [0.1, 0.2, 0.3, 0.4]
    p = oracle.add_noise(2, "fluid", s0, 4, 5, sigma, 1.0)
    m = oracle.add_noise(2, "fluid", s0, 4, 5, sigma, -1.0)
    assert np.allclose((p + m) / 2, s0, rtol=0, atol=1e-15)
    u = oracle.add_noise(2, "fluid", np.zeros((50, 9)), 4, 5, [1.0] * 4, 1.0)
    ratio = (p - s0) / u
    for lo, hi, sg in ((0, 2, 0.1), (2, 4, 0.2), (4, 8, 0.3), (8, 9, 0.4)):
        assert np.allclose(ratio[:, lo:hi], sg, rtol=1e-12)


def test_noise_free_rollout_is_the_fp64_rollout(oracle):
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.block2d_scene(n_strata=(8, 4))
    z = oracle.noise_rollout_z(sc, s0, 5, [1.0] * 4, 3, 0.0)
    states = oracle.rollout_fp64(oracle.make_phys(sc), s0, 5)
    assert z == oracle.mean_sq_pos(2, states[-1])


def test_matched_noise_has_the_dithered_variance(oracle):
    """Matched errors: a value on the lattice gets none, a value at fraction Y gets
    Delta sqrt(Y (1 - Y)) times the unit draw (the dithered store's standard deviation)."""
    delta = 2.0 ** -4
    n = 20_000
    Y = np.random.default_rng(2).uniform(0, 1, n)
    s0 = np.zeros((n, 9))
    s0[:, 8] = (7 + Y) * delta  # J of a 2D fluid, fraction Y
    s0[:, 0] = 3 * delta        # x on the lattice
    unit = oracle.add_noise(2, "fluid", np.zeros((n, 9)), 2, 11, [1.0] * 4, 1.0)
    m = oracle.add_noise(2, "fluid", s0, 2, 11, [delta] * 4, 1.0, matched=True)
    assert np.array_equal(m[:, 0], s0[:, 0])
    assert np.allclose(m[:, 8] - s0[:, 8], delta * np.sqrt(Y * (1 - Y)) * unit[:, 8], rtol=1e-9, atol=1e-15)
    # averaged over uniform fractions the variance is Delta^2 / 6, as for uniform errors of sd Delta / sqrt 6
    assert abs(((m[:, 8] - s0[:, 8]) ** 2).mean() / delta ** 2 - 1 / 6) < 0.01
