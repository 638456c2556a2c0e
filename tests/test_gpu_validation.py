"""The statistical protocol of the paper's error-bound experiments (Sec. 8.1) on solved
schemes: repeated dithered rollouts against the FP64 oracle's z.  Bars: the runs stay
within the paper's 3 eps band in at least 80 % of cases (the paper reports 19/20 and
20/20), the observed spread of z is within a factor 3 of the prediction of Eq. 8 (the
linearisation holds), the mean deviation is within 4 standard errors of zero (the
dithered store is unbiased), and tighter bounds cost more bits."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_error_bound_protocol(oracle):
    import torch
    from paper_2207_04658_b300 import qmpm, validation
    assert torch.cuda.is_available()
    qmpm.lib()
    sc, s0 = validation.impact_block()
    T = 300
    f = oracle.Fp64Rollout(sc, s0)
    f.step(T)
    z_ref = oracle.kinetic_energy(oracle.make_phys(sc), f.s)
    res = validation.error_bound_protocol(sc, s0, T, [0.01, 0.001], runs=12, z_ref=z_ref)
    for r in res:
        assert r["success_3eps"] >= 0.8, r
        assert r["pred_sigma"] / 3 <= r["obs_rms"] <= 3 * r["pred_sigma"], r
        assert abs(r["bias"]) <= 4 * r["bias_stderr"] + 1e-12 * abs(z_ref), r
    assert sum(res[1]["bits"]) > sum(res[0]["bits"])
    assert res[1]["obs_rms"] < res[0]["obs_rms"]
