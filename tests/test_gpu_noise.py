"""The device's noise-injection moments (qmpm_noise_moments: the second-order shift and the
first-order spread of z under explicit store errors) against the oracle's FP64 runs with
the same errors (same Philox counters, particles keyed by the handle's slot order).
Bars: z0 within 1e-5 relative; the spread within 1e-3 relative; the shift within 2 % plus
FP32 rounding of z (5e-6 z0): the shift is about 3e-4 z0 at these noise levels."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,material,matched", [(2, "neohookean", False), (3, "corotated", False),
                                                  (2, "fluid", False), (3, "corotated", True)])
def test_noise_moments_match_the_oracle(oracle, dim, material, matched):
    import torch
    from paper_2207_04658_b300 import qmpm
    from test_gpu_adjoint import small
    assert torch.cuda.is_available()
    sc, s0 = small(dim, material, N_side=10, seed=3)
    T, seed0, pairs = 20, 11, 3
    # matched: the resolutions (powers of two), each store's error of its dithered variance
    sigma = [2.0 ** -8, 0.5, 64.0, 2.0 ** -5] if matched else [2e-3, 0.2, 20.0, 2e-2]
    g = qmpm.Scene(sc, None, s0)
    ids = g.readback(state=False, ids=True)["ids"]
    m = qmpm.qmpm_noise_moments(g.h, T, qmpm.MEASURE_MEAN_SQ_POS | (qmpm.NOISE_MATCHED if matched else 0), sigma,
                                seed0, pairs)
    g.close()
    s_slot = s0[ids]  # particle p of the device runs is slot p
    z0 = oracle.noise_rollout_z(sc, s_slot, T, sigma, 0, 0.0)
    sh, sp = [], []
    for k in range(pairs):
        zp = oracle.noise_rollout_z(sc, s_slot, T, sigma, seed0 + k, 1.0, matched=matched)
        zm = oracle.noise_rollout_z(sc, s_slot, T, sigma, seed0 + k, -1.0, matched=matched)
        sh.append(0.5 * (zp + zm) - z0)
        sp.append(0.25 * (zp - zm) ** 2)
    assert m["pairs"] == pairs
    assert abs(m["z0"] - z0) <= 1e-5 * abs(z0), (m, z0)
    # matched errors scale with each value's fraction on its lattice, which FP32 and FP64
    # runs see a few units apart: 5e-3 for the spread there, 1e-3 otherwise
    assert abs(m["spread"] - np.mean(sp)) <= (5e-3 if matched else 1e-3) * np.mean(sp), (m, np.mean(sp))
    assert abs(m["shift"] - np.mean(sh)) <= 2e-2 * abs(np.mean(sh)) + 5e-6 * abs(z0), (m, np.mean(sh))


def test_noise_moments_arguments():
    import torch
    from paper_2207_04658_b300 import qmpm, scenes
    assert torch.cuda.is_available()
    sc, s0 = scenes.block2d_scene(n_strata=(8, 4))
    g = qmpm.Scene(sc, None, s0)
    try:
        with pytest.raises(qmpm.QmpmError):
            qmpm.qmpm_noise_moments(g.h, 5, qmpm.MEASURE_MEAN_SQ_POS, [0.1] * 4, 1, 1)  # n_pairs < 2
        with pytest.raises(qmpm.QmpmError):
            qmpm.qmpm_noise_moments(g.h, 5, qmpm.MEASURE_MEAN_SQ_POS, [-0.1, 0, 0, 0], 1, 2)
        m = qmpm.qmpm_noise_moments(g.h, 5, qmpm.MEASURE_KINETIC_ENERGY, [0.0] * 4, 1, 2)
        assert m["shift"] == 0.0 and m["spread"] == 0.0  # no noise: every run is the noise-free one
    finally:
        g.close()


def test_position_noise_moments_match_the_oracle(oracle):
    """The vector evaluation (final positions): |b|^2 of the bias vector and the summed
    first-order spread, against the same estimates from the oracle's FP64 runs."""
    import torch
    from paper_2207_04658_b300 import qmpm
    from test_gpu_adjoint import small
    assert torch.cuda.is_available()
    sc, s0 = small(3, "corotated", N_side=10, seed=3)
    T, sigma, seed0, K = 20, [2e-3, 0.2, 20.0, 2e-2], 11, 3
    g = qmpm.Scene(sc, None, s0)
    ids = g.readback(state=False, ids=True)["ids"]
    m = qmpm.qmpm_noise_moments(g.h, T, qmpm.MEASURE_POSITIONS, sigma, seed0, K)
    g.close()
    s_slot = s0[ids]
    x0 = oracle.noise_rollout_state(sc, s_slot, T, sigma, 0, 0.0)[:, :3]
    ms, sq, sp = [], [], []
    for k in range(K):
        xp = oracle.noise_rollout_state(sc, s_slot, T, sigma, seed0 + k, 1.0)[:, :3]
        xm = oracle.noise_rollout_state(sc, s_slot, T, sigma, seed0 + k, -1.0)[:, :3]
        mk = 0.5 * (xp + xm) - x0
        ms.append(mk)
        sq.append((mk ** 2).sum())
        sp.append((0.25 * (xp - xm) ** 2).sum())
    mean = np.mean(ms, axis=0)
    b2 = (K * (mean ** 2).sum() - np.mean(sq)) / (K - 1)
    assert abs(m["z0"] - (x0 ** 2).sum(1).mean()) <= 1e-5 * m["z0"]
    assert abs(m["spread"] - np.mean(sp)) <= 1e-3 * np.mean(sp), (m, np.mean(sp))
    # |b|^2 is a difference of two close sums: compare within FP32 rounding of the positions
    assert abs(m["shift"] - b2) <= 5e-2 * abs(b2) + 1e-3 * np.mean(sq), (m, b2, np.mean(sq))
