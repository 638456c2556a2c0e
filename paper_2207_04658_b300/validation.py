"""Statistical validation of solved schemes (the protocol of the paper's Sec. 8.1 error-bound
experiments): for each error bound eps, solve the scheme (Algorithm 1), run R quantized
rollouts that differ only in their dither seed, and compare

  * the predicted variance of z, E[dz] = (1/12) sum_h Delta_h^2 g_h (Eq. 8), with the
    observed mean square deviation of the runs' z from the reference z;
  * the mean deviation (bias; dithering makes the store unbiased, Sec. 5);
  * the success rate: runs within the paper's band |z~ - z| <= 3 eps z (Sec. 8.1), and
    within eps z;
  * the memory of the scheme (bits per particle vs FP32);

and, with --optimality, the optimality check (bits taken from all or half of the fields,
bits moved between fields) and the dithering experiment (with and without dithered stores,
round-up / round-down ratios); with --memory, the memory-bounded experiment (a 2D fluid dam
break at target fractions of the FP32 bits); with --checkpointing, the adjoint's memory and
time with every state kept, uniform and bisection checkpoints; with --layouts, the step
time of bit-packed against bit-struct records; with --scaling, the scaling procedure (one
scheme from the smallest of four 3D fluid configurations applied up to 5M particles).

Everything runs through the library (adjoint, solve, rollouts).  The reference z is
supplied by the caller (the FP64 oracle in the tests); the command line uses the FP32 run
of the same kernels.

    python -m paper_2207_04658_b300.validation [--runs 20] [--steps 300]
        [--smoke | --optimality | --memory | --checkpointing | --layouts | --scaling]
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


def predicted_moments(scene, state0, T, scheme, pairs=16, seed=4242, measure=qmpm.MEASURE_KINETIC_ENERGY):
    """The mean shift and the spread of z that dithered stores of `scheme` cause, predicted by
    antithetic noise injection (qmpm_noise_moments, matched): at every store of type h an
    error with the dithered store's own variance there, Delta_h^2 Y (1 - Y) for a value at
    fraction Y of its lattice.  The shift is the second-order term that Eq. 8 leaves out."""
    names = ("x", "v", "C", "J" if scene["material"] == "fluid" else "F")
    deltas = [2.0 ** -scheme[k]["frac"] for k in names]
    g = qmpm.Scene(dict(scene, resort_every=0), None, state0)
    try:
        m = qmpm.qmpm_noise_moments(g.h, T, measure | qmpm.NOISE_MATCHED, deltas, seed, pairs)
    finally:
        g.close()
    return m


def error_bound_protocol(scene, state0, T, eps_list, runs, z_ref, ckpt_every=25, seed0=1000, noise_pairs=16):
    """Per eps: the solved scheme, predicted and observed spread of z, predicted (second
    order) and observed bias, success rates, and each run's z (run r has dither seed
    seed0 + r)."""
    info = qmpm.sensitivities(scene, state0, T, ckpt_every, qmpm.MEASURE_KINETIC_ENERGY)
    out = []
    for eps in eps_list:
        scheme, res = qmpm.solve_scheme(info, eps, material=scene["material"])
        mom = predicted_moments(scene, state0, T, scheme, pairs=noise_pairs) if noise_pairs >= 2 else None
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
            "z_ref": z_ref, "runs": runs, "z_runs": zs.tolist(), "seed0": seed0, "scheme": scheme,
        })
        if mom is not None:
            out[-1].update(pred_bias=mom["shift"], pred_bias_se=mom["shift_se"],
                           pred_sigma_dither=float(np.sqrt(max(mom["spread"], 0.0))), noise_pairs=mom["pairs"])
    return out


def _rollouts(scene, state0, T, scheme, runs, seed0, dither=True, stats=False):
    """z of `runs` quantized rollouts differing only in their dither seed, and the summed
    round-up / round-down counters per field when `stats`."""
    zs, ups, dns = [], np.zeros(4, np.int64), np.zeros(4, np.int64)
    for r in range(runs):
        g = qmpm.Scene(dict(scene, seed=seed0 + r, dither=dither), scheme, state0, stats=stats)
        g.step(T)
        rb = g.readback(state=True, ids=False)
        zs.append(kinetic_energy(scene, rb["state"]))
        if stats:
            ups += np.asarray(rb["stats"]["round_ups"], np.int64)
            dns += np.asarray(rb["stats"]["round_downs"], np.int64)
        g.close()
    return np.asarray(zs), ups, dns


def shift_bits(scheme, material, names, k):
    """The scheme with k fewer bits (k < 0: more) for each type in names, each over its same
    window (qmpm_scheme_shift by -k): the resolution doubles per bit taken."""
    for n in names:
        scheme = qmpm.scheme_shift(scheme, material, n, -k)
    return scheme


def optimality_check(scene, state0, T, z_ref, eps=0.01, runs=20, takes=(1, 2, 3), move_runs=10, seed=7,
                     ckpt_every=25, seed0=3000):
    """The optimality check of Sec. 8.1 on the scheme Algorithm 1 solves at eps: take k bits
    from every field, or from a random half of the fields, and move one bit between fields
    (x <-> v, C <-> F); success = |z~ - z| <= 3 eps z over repeated dithered rollouts."""
    info = qmpm.sensitivities(scene, state0, T, ckpt_every, qmpm.MEASURE_KINETIC_ENERGY)
    base, res = qmpm.solve_scheme(info, eps, material=scene["material"])
    names = [k for k in ("x", "v", "C", "F", "J") if k in base]
    gen = np.random.default_rng(seed)

    def trial(scheme, n):
        zs, _, _ = _rollouts(scene, state0, T, scheme, n, seed0)
        dev = zs - z_ref
        return {"bits": [scheme[k]["bits"] for k in names], "success_3eps": float(np.mean(np.abs(dev) <= 3 * eps * abs(z_ref))),
                "z_mean": float(zs.mean()), "z_std": float(zs.std(ddof=1)) if n > 1 else 0.0,
                "obs_rms": float(np.sqrt(np.mean(dev ** 2)))}

    mat = scene["material"]
    out = {"eps": eps, "fields": names, "base": trial(base, runs), "reduce_all": {}, "reduce_half": {}, "move": {}}
    for k in takes:
        out["reduce_all"][k] = trial(shift_bits(base, mat, [f for f in names if base[f]["bits"] > k], k), runs)
        half = set(gen.choice(names, size=len(names) // 2, replace=False).tolist())
        red = shift_bits(base, mat, [f for f in names if f in half and base[f]["bits"] > k], k)
        out["reduce_half"][k] = dict(trial(red, runs), fields_reduced=sorted(half))
    pairs = [(names[0], names[1]), (names[1], names[0]), (names[2], names[3]), (names[3], names[2])]
    for a, b in pairs:
        moved = shift_bits(shift_bits(base, mat, [a], 1), mat, [b], -1)
        out["move"][f"{a}->{b}"] = trial(moved, move_runs)
    return out


def dithering_effectiveness(scene, state0, T, z_ref, scheme, runs=5, seed0=5000):
    """Sec. 8.1's dithering experiment: the same scheme with and without dithered stores;
    z against the reference and the ratio of round-ups to round-downs per field (about 1
    when dithered; skewed by the rounding of systematically placed values otherwise)."""
    out = {}
    for name, dither in (("dithered", True), ("nearest", False)):
        zs, ups, dns = _rollouts(scene, state0, T, scheme, runs if dither else 1, seed0, dither=dither, stats=True)
        out[name] = {"z_mean": float(zs.mean()), "rel_err": float(abs(zs.mean() - z_ref) / abs(z_ref)),
                     "up_down_ratio": [float(u) / max(float(d), 1.0) for u, d in zip(ups, dns)]}
    out["z_ref"] = z_ref
    return out


def memory_bound_protocol(scene, state0, T, eps_list, z_ref, runs=10, ckpt_every=0, seed0=7000):
    """The memory-bounded experiment of Sec. 8.1: per target fraction eps_mem of the FP32
    bits, the scheme of the memory-bound solve (Eq. 7), its real compression, and z over
    `runs` dithered rollouts: mean, spread and e_mem = sqrt(sigma^2 + (mu - z)^2) / z."""
    info = qmpm.sensitivities(scene, state0, T, ckpt_every, qmpm.MEASURE_KINETIC_ENERGY)
    # the floor: FP32 rollouts differ from one another through the order of the grid's
    # floating-point atomic sums, and a long fluid run amplifies that like any other noise
    z32, _, _ = _rollouts(scene, state0, T, None, runs, seed0)
    out = [{"eps_mem": 1.0, "bits": [32] * 4, "real_fraction": 1.0, "compression": 1.0, "z_mean": float(z32.mean()),
            "z_std": float(z32.std(ddof=1)) if runs > 1 else 0.0,
            "e_mem": float(np.sqrt(z32.var(ddof=1) + (z32.mean() - z_ref) ** 2) / abs(z_ref)) if runs > 1 else 0.0,
            "z_ref": z_ref, "runs": runs, "fp32": True}]
    for eps in eps_list:
        scheme, res = qmpm.solve_scheme(info, eps, mode="memory", material=scene["material"])
        zs, _, _ = _rollouts(scene, state0, T, scheme, runs, seed0)
        names = [k for k in ("x", "v", "C", "F", "J") if k in scheme]
        d = scene["dim"]
        n_comp = {"x": d, "v": d, "C": d * d, "F": d * d, "J": 1}
        bits = sum(scheme[f]["bits"] * n_comp[f] for f in names)
        fp32 = 32 * sum(n_comp[f] for f in names)
        mu, sd = float(zs.mean()), float(zs.std(ddof=1)) if runs > 1 else 0.0
        out.append({"eps_mem": eps, "bits": [scheme[f]["bits"] for f in names], "real_fraction": bits / fp32,
                    "compression": fp32 / bits, "z_mean": mu, "z_std": sd,
                    "e_mem": float(np.sqrt(sd ** 2 + (mu - z_ref) ** 2) / abs(z_ref)), "z_ref": z_ref, "runs": runs})
    return out


def checkpointing_cost(scene, state0, Ts=(256, 1024, 4096)):
    """The cost of the adjoint's checkpointing (Sec. 6; the paper's comparison of bisection
    with the unfolded tape): per horizon T, the states held, the forward steps run and the
    wall time of one adjoint pass with every state kept (ckpt_every 1), uniform checkpoints
    every sqrt(T) steps, and bisection checkpoints."""
    import time
    import torch
    N, nc = state0.shape
    out = []
    for T in Ts:
        row = {"T": T}
        for name, every in (("unfolded", 1), ("uniform", int(round(T ** 0.5))), ("bisection", qmpm.CKPT_BISECTION)):
            g = qmpm.Scene(dict(scene, resort_every=0), None, state0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = qmpm.qmpm_adjoint(g.h, T, every, qmpm.MEASURE_KINETIC_ENERGY)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            g.close()
            row[name] = {"ckpt_every": every, "state_buffers": info["state_buffers"],
                         "state_mb": info["state_buffers"] * N * nc * 4 / 1e6,
                         "forward_steps": info["forward_steps"], "seconds": el, "g": info["g"]}
        out.append(row)
    return out


def layout_cost(widths=(16, 20, 24), steps=20, warmup=3):
    """The layout experiment of Sec. 8.2 (bit pack vs bit struct): the 3D elastic cubes
    (8,192,000 particles) with every component stored in w bits, packed across word
    boundaries (components straddle words when 32 is not a multiple of w) or in 64-bit
    containers (whole components per container, the rest of a container unused); words per
    particle and the step kernel's device time per step."""
    import torch
    sc, s0 = scenes.cubes3d_scene()
    out = []
    for w in widths:
        row = {"bits": w}
        for name, cont in (("bit_pack", 0), ("bit_struct", 64)):
            sch = scenes.fixed_scheme_3d("corotated", x_bits=w, v=(w, -8.0, 8.0), C=(w, -512.0, 512.0),
                                         F=(w, -0.5, 1.5), x_container=cont)
            for f in sch.values():
                f["container"] = cont
            g = qmpm.Scene(dict(sc, resort_every=8), sch, s0, profile=True)
            g.step(warmup)
            torch.cuda.synchronize()
            g.profile(reset=True)
            g.step(steps)
            prof = g.profile(reset=True)
            row[name] = {"words": g.n_words, "step_kernel_ms": prof["step_ms"] / max(1, prof["step_launches"])}
            g.close()
        out.append(row)
    return out


def mean_height(state):
    return float(state[:, 1].mean())


def scaling_protocol(sizes=None, eps_mem=0.5, runs=3, range_every=1024, seed0=9000):
    """The scaling procedure of Sec. 8.3 on a 3D fluid column: g_h from the adjoint of the
    smallest configuration (mean height as z, bisection checkpoints), ranges recorded from
    the FP32 run of the largest one (the state read back every `range_every` steps), one
    memory-bound scheme (eps_mem of the FP32 bits) applied unchanged to every
    configuration; per configuration the FP32 z and the quantized z over `runs` dither
    seeds."""
    import torch
    sizes = sizes or scenes.SCALING_CONFIGS
    sc0, s00 = scenes.fluid3d_column_scene(*sizes[0])
    N0, nc = s00.shape
    seed = torch.zeros((N0, nc), dtype=torch.float32, device="cuda")
    seed[:, 1] = 1.0 / N0  # dz/dy of the mean height
    g = qmpm.Scene(dict(sc0, resort_every=0), None, s00)
    info = qmpm.qmpm_adjoint(g.h, sizes[0][3], qmpm.CKPT_BISECTION, qmpm.MEASURE_USER, seed.data_ptr())
    g.close()
    # ranges from the largest configuration's FP32 run
    scL, sL = scenes.fluid3d_column_scene(*sizes[-1])
    comps = [[0, 1, 2], [3, 4, 5], list(range(6, 15)), [15]]
    lo, hi = np.full(4, np.inf), np.full(4, -np.inf)
    g = qmpm.Scene(scL, None, sL)
    fp32_last = None
    for t0 in range(0, sizes[-1][3] + 1, range_every):
        if t0 > 0:
            g.step(range_every)
        st = g.readback(state=True, ids=False)["state"]
        for h in range(4):
            lo[h] = min(lo[h], float(st[:, comps[h]].min()))
            hi[h] = max(hi[h], float(st[:, comps[h]].max()))
        fp32_last = st
    g.close()
    info = dict(info, lo=list(lo), hi=list(hi))
    scheme, res = qmpm.solve_scheme(info, eps_mem, mode="memory", material="fluid")
    out = {"scheme": scheme, "g": info["g"], "lo": list(lo), "hi": list(hi), "configs": []}
    for k, cfg in enumerate(sizes):
        sc, s0 = scenes.fluid3d_column_scene(*cfg)
        if k == len(sizes) - 1:
            z32 = mean_height(fp32_last)
        else:
            g = qmpm.Scene(sc, None, s0)
            g.step(cfg[3])
            z32 = mean_height(g.readback(state=True, ids=False)["state"])
            g.close()
        zq = []
        for r in range(runs):
            g = qmpm.Scene(dict(sc, seed=seed0 + r), scheme, s0)
            g.step(cfg[3])
            zq.append(mean_height(g.readback(state=True, ids=False)["state"]))
            g.close()
        zq = np.asarray(zq)
        out["configs"].append({"particles": s0.shape[0], "grid": f"{1 << cfg[1]}^3", "dt": cfg[2], "steps": cfg[3],
                               "z_fp32": z32, "z_quant_mean": float(zq.mean()),
                               "z_quant_std": float(zq.std(ddof=1)) if runs > 1 else 0.0,
                               "rel_err": float(abs(zq.mean() - z32) / abs(z32))})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", type=int, default=20)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--smoke", action="store_true", help="the 2D smoke plume instead of the MPM block")
    ap.add_argument("--optimality", action="store_true", help="the optimality check and the dithering experiment")
    ap.add_argument("--memory", action="store_true", help="the memory-bounded 2D fluid dam break")
    ap.add_argument("--checkpointing", action="store_true", help="adjoint memory and time by checkpointing")
    ap.add_argument("--layouts", action="store_true", help="bit pack vs bit struct step time")
    ap.add_argument("--scaling", action="store_true", help="one scheme from 0.2M particles applied up to 5M")
    args = ap.parse_args()
    if args.scaling:
        print(json.dumps({"scene": "3D fluid column (K 200), mean height", "reference": "FP32 runs",
                          **scaling_protocol()}, default=float))
        return
    if args.layouts:
        print(json.dumps({"scene": "3D fixed-corotated cubes, 8,192,000 particles, 256^3", "results": layout_cost()}))
        return
    if args.checkpointing:
        sc, s0 = impact_block()
        print(json.dumps({"scene": "2D neo-Hookean impact block, 2,048 particles, 128^2",
                          "results": checkpointing_cost(sc, s0)}))
        return
    if args.memory:
        sc, s0 = scenes.dambreak2d_scene()
        T = sc["steps"]
        g = qmpm.Scene(sc, None, s0)
        g.step(T)
        z_ref = kinetic_energy(sc, g.readback(state=True, ids=False)["state"])
        g.close()
        res = memory_bound_protocol(sc, s0, T, [0.6, 0.5, 0.4], z_ref, runs=min(args.runs, 10))
        print(json.dumps({"scene": "2D fluid dam break, 10,000 particles, 128^2, 16,384 steps",
                          "reference": "FP32 run of the same kernels", "results": res}))
        return
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
    if args.optimality:
        opt = optimality_check(sc, s0, args.steps, z_ref, runs=args.runs)
        info = qmpm.sensitivities(sc, s0, args.steps, 25, qmpm.MEASURE_KINETIC_ENERGY)
        bold, _ = qmpm.solve_scheme(info, 0.1, material=sc["material"])
        dith = dithering_effectiveness(sc, s0, args.steps, z_ref, bold)
        print(json.dumps({"scene": "2D neo-Hookean impact block, 2,048 particles, 128^2",
                          "reference": "FP32 run of the same kernels", "optimality": opt,
                          "dithering": dict(dith, scheme=bold)}, default=str))
        return
    res = error_bound_protocol(sc, s0, args.steps, [0.1, 0.01, 1e-3, 1e-4], args.runs, z_ref)
    print(json.dumps({"scene": "2D neo-Hookean impact block, 2048 particles, 128^2",
                      "reference": "FP32 run of the same kernels", "results": res}))


if __name__ == "__main__":
    main()
