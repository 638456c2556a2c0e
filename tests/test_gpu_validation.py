"""The statistical protocol of the paper's error-bound experiments (Sec. 8.1) on solved
schemes: repeated dithered rollouts against the FP64 oracle's z.  Bars: the runs stay
within the paper's 3 eps band in at least 80 % of cases (the paper reports 19/20 and
20/20), the observed spread of z is within a factor 3 of the prediction of Eq. 8 (the
linearisation holds), and tighter bounds cost more bits.

The mean deviation has two sources, checked apart.  (1) The kernels: each run r is paired
with the oracle's quantized rollout of the same scheme and dither seed (the same store
rule and draws, in FP64), and the mean of the paired differences of z must be within 4
standard errors of zero.  (2) The method: each dithered store is unbiased, but z is not
linear in the state, so zero-mean store errors shift the mean of z at second order (the
part of Eq. 6 that Eq. 8 drops).  That shift is predicted by antithetic noise injection
(errors of the dithered variance Delta_h^2 / 6 at every store) and the observed bias must
match the prediction within 4 combined standard errors, at both bounds."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def oracle_quantized_z(oracle, sc, s0, scheme, T, seed):
    ro = oracle.QuantRollout(dict(sc, seed=seed), scheme, s0)
    ro.step(T)
    return oracle.kinetic_energy(ro.ph, ro.state())


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
    res = validation.error_bound_protocol(sc, s0, T, [0.01, 0.001], runs=12, z_ref=z_ref, noise_pairs=24)
    for r in res:
        assert r["success_3eps"] >= 0.8, r
        assert r["pred_sigma"] / 3 <= r["obs_rms"] <= 3 * r["pred_sigma"], r
        # (1) the kernels against the oracle, run by run
        zo = np.array([oracle_quantized_z(oracle, sc, s0, r["scheme"], T, r["seed0"] + i) for i in range(r["runs"])])
        d = np.asarray(r["z_runs"]) - zo
        se_d = d.std(ddof=1) / np.sqrt(len(d))
        assert abs(d.mean()) <= 4 * se_d + 1e-9 * abs(z_ref), (r["eps"], d.mean(), se_d)
        # (2) the method's second-order bias against its prediction
        se = np.hypot(r["bias_stderr"], r["pred_bias_se"])
        assert abs(r["bias"] - r["pred_bias"]) <= 4 * se + 1e-12 * abs(z_ref), r
    assert sum(res[1]["bits"]) > sum(res[0]["bits"])
    assert res[1]["obs_rms"] < res[0]["obs_rms"]


def test_optimality_check_and_dithering():
    """Sec. 8.1's optimality check on the eps = 0.01 scheme of the impact block: taking bits
    away from every field quickly breaks the bound (the scheme sits near the critical
    point), and the error grows with the bits taken.  The dithering experiment on the
    eps = 0.1 scheme: dithered stores round up as often as down in every field, while
    round-to-nearest stores of the slowly changing velocity are skewed to one side."""
    import torch
    from paper_2207_04658_b300 import qmpm, validation
    assert torch.cuda.is_available()
    qmpm.lib()
    sc, s0 = validation.impact_block()
    T = 300
    g = qmpm.Scene(sc, None, s0)
    g.step(T)
    z_ref = validation.kinetic_energy(sc, g.readback(state=True, ids=False)["state"])
    g.close()
    opt = validation.optimality_check(sc, s0, T, z_ref, runs=12, takes=(1, 2), move_runs=6)
    assert opt["base"]["success_3eps"] >= 0.8, opt["base"]
    assert opt["reduce_all"][2]["success_3eps"] <= 0.5, opt["reduce_all"]
    assert opt["base"]["obs_rms"] < opt["reduce_all"][1]["obs_rms"] < opt["reduce_all"][2]["obs_rms"], opt
    assert set(opt["move"]) == {"x->v", "v->x", "C->F", "F->C"}
    info = qmpm.sensitivities(sc, s0, T, 25, qmpm.MEASURE_KINETIC_ENERGY)
    bold, _ = qmpm.solve_scheme(info, 0.1, material=sc["material"])
    dith = validation.dithering_effectiveness(sc, s0, T, z_ref, bold, runs=3)
    assert all(0.9 < r < 1.1 for r in dith["dithered"]["up_down_ratio"]), dith
    v_ratio = dith["nearest"]["up_down_ratio"][1]
    assert v_ratio > 2.0 or v_ratio < 0.5, dith


def test_memory_bound_protocol():
    """Sec. 8.1's memory-bounded experiment on the 2D fluid dam break (shortened to 2048
    steps): the memory-bound solve meets each target fraction of the FP32 bits, and the
    error metric e_mem stays within a few times the FP32 runs' own run-to-run spread (the
    grid's atomic sums make FP32 rollouts differ, and the sloshing fluid amplifies that)."""
    import torch
    from paper_2207_04658_b300 import qmpm, scenes, validation
    assert torch.cuda.is_available()
    qmpm.lib()
    sc, s0 = scenes.dambreak2d_scene(steps=2048)
    T = sc["steps"]
    g = qmpm.Scene(sc, None, s0)
    g.step(T)
    z_ref = validation.kinetic_energy(sc, g.readback(state=True, ids=False)["state"])
    g.close()
    res = validation.memory_bound_protocol(sc, s0, T, [0.6, 0.5, 0.4], z_ref, runs=5)
    floor = res[0]
    assert floor.get("fp32") and floor["real_fraction"] == 1.0
    for r in res[1:]:
        assert r["eps_mem"] - 0.12 <= r["real_fraction"] <= r["eps_mem"] + 1e-9, r
        assert r["e_mem"] <= max(4 * floor["e_mem"], 0.05), (r, floor)


def test_scaling_procedure_small():
    """The scaling procedure of Sec. 8.3 at small sizes: a memory-bound scheme (half the FP32
    bits) from the gradients of a 20,000-particle 3D fluid column on 32^3, with ranges
    recorded on the 160,000-particle configuration, applied unchanged to both: the mean
    height stays within 1 % of the FP32 run's."""
    import torch
    from paper_2207_04658_b300 import qmpm, validation
    assert torch.cuda.is_available()
    qmpm.lib()
    res = validation.scaling_protocol(sizes=[(20_000, 5, 4e-4, 512), (160_000, 6, 2e-4, 1024)], runs=2,
                                      range_every=256)
    bits = {k: v["bits"] for k, v in res["scheme"].items()}
    assert 3 * bits["x"] + 3 * bits["v"] + 9 * bits["C"] + bits["J"] <= 0.5 * 32 * 16
    for c in res["configs"]:
        assert c["rel_err"] < 1e-2, c
