"""Statistical validation of solved schemes (the protocol of the paper's Sec. 8.1 error-bound
experiments): for each error bound eps, solve the scheme (Algorithm 1), run R quantized
rollouts that differ only in their dither seed, and compare

  * the predicted variance of z, E[dz] = (1/12) sum_h Delta_h^2 g_h (Eq. 8), with the
    observed mean square deviation of the runs' z from the reference z;
  * the mean deviation (bias; dithering makes the store unbiased, Sec. 5);
  * the success rate: runs within the paper's band |z~ - z| <= 3 eps z (Sec. 8.1), and
    within eps z;
  * the memory of the scheme (bits per particle vs FP32).

Everything runs through the library (adjoint, solve, rollouts).  The reference z is
supplied by the caller (the FP64 oracle in the tests); the command line uses the FP32 run
of the same kernels.

    python -m paper_2207_04658_b300.validation [--runs 20] [--steps 300] [--smoke]
"""
import argparse
import json

import numpy as np

from . import qmpm, scenes


def kinetic_energy(scene, state):
    d = scene["dim"]
    m = scene["p_vol"] * scene.get("rho", 1.0)
    return 0.5 * m * float((state[:, d:2 * d] ** 2).sum())


def impact_block(n_strata=(64, 32)):
    """The 2D neo-Hookean block driven into the floor (the impact couples every field into
    the final kinetic energy, the evaluation function of the paper's MPM experiments)."""
    sc, s0 = scenes.block2d_scene(n_strata=n_strata)
    s0[:, 1] -= 0.4 - 3.6 / 128
    s0[:, 3] = -0.5
    return dict(sc, resort_every=8), s0


def error_bound_protocol(scene, state0, T, eps_list, runs, z_ref, ckpt_every=25, seed0=1000):
    """Per eps: the solved scheme, predicted and observed spread of z, bias, success rates."""
    info = qmpm.sensitivities(scene, state0, T, ckpt_every, qmpm.MEASURE_KINETIC_ENERGY)
    out = []
    for eps in eps_list:
        scheme, res = qmpm.solve_scheme(info, eps, material=scene["material"])
        zs = []
        for r in range(runs):
            g = qmpm.Scene(dict(scene, seed=seed0 + r), scheme, state0)
            g.step(T)
            zs.append(kinetic_energy(scene, g.readback(state=True, ids=False)["state"]))
            g.close()
        zs = np.asarray(zs)
        dev = zs - z_ref
        ms = float((dev ** 2).mean())
        out.append({
            "eps": eps, "bits": res["bits"], "frac": res["frac"], "capped": res.get("capped", []),
            "words_per_particle": qmpm.make_scheme_struct(scheme, scene["dim"], scene["material"]).n_words,
            "pred_sigma": float(np.sqrt(res["pred_err"])), "obs_rms": float(np.sqrt(ms)),
            "bias": float(dev.mean()), "bias_stderr": float(dev.std(ddof=1) / np.sqrt(runs)) if runs > 1 else 0.0,
            "success_3eps": float((np.abs(dev) <= 3 * eps * abs(z_ref)).mean()),
            "success_eps": float((np.abs(dev) <= eps * abs(z_ref)).mean()),
            "z_ref": z_ref, "runs": runs,
        })
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", type=int, default=20)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--smoke", action="store_true", help="the 2D smoke plume instead of the MPM block")
    args = ap.parse_args()
    if args.smoke:
        from . import smoke
        sc = scenes.smoke_scene()
        res = smoke.error_bound_protocol(sc, sc["steps"], [0.1, 0.01, 1e-3, 1e-4], args.runs)
        print(json.dumps({"scene": "2D smoke plume, 256^2, 64 Jacobi sweeps, 100 steps",
                          "reference": "FP32 run of the same kernels", **res}))
        return
    sc, s0 = impact_block()
    g = qmpm.Scene(sc, None, s0)
    g.step(args.steps)
    z_ref = kinetic_energy(sc, g.readback(state=True, ids=False)["state"])
    g.close()
    res = error_bound_protocol(sc, s0, args.steps, [0.1, 0.01, 1e-3, 1e-4], args.runs, z_ref)
    print(json.dumps({"scene": "2D neo-Hookean impact block, 2048 particles, 128^2",
                      "reference": "FP32 run of the same kernels", "results": res}))


if __name__ == "__main__":
    main()
