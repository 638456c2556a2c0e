"""The device's noise-injection moments (qmpm_noise_moments: the second-order shift and the
first-order spread of z under explicit store errors) against the oracle's FP64 runs with
the same errors (same Philox counters, particles keyed by the handle's slot order).
Bars: z0 within 1e-5 relative; the spread within 1e-3 relative; the shift within 2 % plus
FP32 rounding of z (5e-6 z0): the shift is about 3e-4 z0 at these noise levels."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,material", [(2, "neohookean"), (3, "corotated"), (2, "fluid")])
def test_noise_moments_match_the_oracle(oracle, dim, material):
    import torch
    from paper_2207_04658_b300 import qmpm
    from test_gpu_adjoint import small
    assert torch.cuda.is_available()
    sc, s0 = small(dim, material, N_side=10, seed=3)
    T, sigma, seed0, pairs = 20, [2e-3, 0.2, 20.0, 2e-2], 11, 3
    g = qmpm.Scene(sc, None, s0)
    ids = g.readback(state=False, ids=True)["ids"]
    m = qmpm.qmpm_noise_moments(g.h, T, qmpm.MEASURE_MEAN_SQ_POS, sigma, seed0, pairs)
    g.close()
    s_slot = s0[ids]  # particle p of the device runs is slot p
    z0 = oracle.noise_rollout_z(sc, s_slot, T, sigma, 0, 0.0)
    sh, sp = [], []
    for k in range(pairs):
        zp = oracle.noise_rollout_z(sc, s_slot, T, sigma, seed0 + k, 1.0)
        zm = oracle.noise_rollout_z(sc, s_slot, T, sigma, seed0 + k, -1.0)
        sh.append(0.5 * (zp + zm) - z0)
        sp.append(0.25 * (zp - zm) ** 2)
    assert m["pairs"] == pairs
    assert abs(m["z0"] - z0) <= 1e-5 * abs(z0), (m, z0)
    assert abs(m["spread"] - np.mean(sp)) <= 1e-3 * np.mean(sp), (m, np.mean(sp))
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
