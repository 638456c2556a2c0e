"""Algorithm 1 end to end: a quantization scheme for a scene from its sensitivities.

The paper's workflow (Sec. 4, Algorithm 1; scaling procedure of Sec. 8.3): run the
full-precision simulation at low resolution, record each field's range, back-propagate
the evaluation function to get the accumulated squared sensitivities g_h (Eq. 8), solve
Eq. 10 (or its memory-bound form) for the bit widths, and apply the scheme to the
high-resolution run.  Forward and backward passes run in the library's FP32 adjoint;
the solve is the library's host solver.
"""
import os

from . import qmpm, scenes


def scheme_from_run(scene, state0, T, eps, mode="error", measure=qmpm.MEASURE_MEAN_SQ_POS,
                    ckpt_every=32, containers=(0, 0, 0, 0), rounding="paper", kappa=2.0):
    """Sensitivities of ``scene`` over T steps, then the scheme at tolerance ``eps``
    (error mode) or compression rate ``eps`` (memory mode).  Returns (scheme, report)."""
    info = qmpm.sensitivities(scene, state0, T, ckpt_every, measure)
    scheme, res = qmpm.solve_scheme(info, eps, mode=mode, rounding=rounding, kappa=kappa,
                                    containers=containers, material=scene["material"])
    return scheme, {"solve": res, "sensitivities": info}


def position_sensitivities(scene, state0, T, samples=2, ckpt_every=32, seed=0, reference="position"):
    """Sensitivities of the final particle positions as a whole: the evaluation is the
    vector of final positions x_T, and Eq. 8 summed over its N d outputs gives
    G_h = sum_m sum_t sum_i (d x_T,m / d e_{t,i})^2, the trace of J J^T over the
    variables of type h.  It is estimated with ``samples`` adjoint runs seeded with
    independent standard normal vectors u on x_T (E[(u^T J)^2] = trace(J J^T)).
    Returns the adjoint report with g replaced by G and z by sqrt(sum_m |x_T,m|^2)
    (so that (eps z)^2 bounds the summed squared position error, i.e. the RMS position
    error stays below eps times the RMS position), or with reference="displacement" by
    sqrt(sum_m |x_T,m - x_0,m|^2) (the RMS error below eps times the RMS displacement)."""
    import numpy as np
    import torch
    dim = scene["dim"]
    g = qmpm.Scene(dict(scene, resort_every=0), None, state0)
    N, nc = g.N, g.n_comp
    gen = np.random.default_rng(seed)
    acc = np.zeros(4)
    info = None
    for _ in range(samples):
        u = np.zeros((N, nc), dtype=np.float32)
        u[:, :dim] = gen.standard_normal((N, dim)).astype(np.float32)
        d_seed = torch.from_numpy(u).cuda()
        info = qmpm.qmpm_adjoint(g.h, T, ckpt_every, qmpm.MEASURE_USER, d_seed.data_ptr())
        acc += np.asarray(info["g"])
    out = dict(info)
    out["g"] = list(acc / samples)
    if reference == "displacement":
        g.step(T)
        xT = g.state_by_id()[:, :dim]
        out["z"] = float(np.sqrt(((xT - state0[:, :dim]) ** 2).sum()))
    else:
        out["z"] = float(np.sqrt(N * info["z"]))  # info["z"] is the mean square position of x_T
    g.close()
    out["samples"] = samples
    out["reference"] = reference
    return out


def cubes3d_scheme(eps=0.01, T=None, samples=2, ckpt_every=32, material="corotated"):
    """Scheme for the 3D elastic cubes at relative error ``eps`` on the final particle
    positions (RMS position error <= eps x RMS position): sensitivities of the same 16
    cubes at half resolution (20-cell cubes on a 128^3 grid, 1,024,000 particles), the
    scheme applied unchanged at full resolution (Sec. 8.3); x in one 64-bit container,
    the rest bit-packed."""
    sc, s0 = scenes.cubes3d_scene(cube_cells=20, grid_log2=7, material=material)
    steps = T if T is not None else sc["steps"]
    info = position_sensitivities(sc, s0, steps, samples=samples, ckpt_every=ckpt_every)
    scheme, res = qmpm.solve_scheme(info, eps, containers=(64, 0, 0, 0), material=material)
    return scheme, {"solve": res, "sensitivities": info}


def _margin_windows(scheme, material, info, margins, kappa=2.0, grow_only=False):
    """The windows of the types in margins = {h: (src, gain)} re-derived at their current
    resolution by qmpm_scheme_window: the solve's window of the recorded range [lo_h,
    hi_h] widened by gain times the resolution of type src (the solve's window-margin
    option, here applied after every change of resolution); grow_only keeps the union with
    the type's current window."""
    for h, (src, gain) in (margins or {}).items():
        scheme = qmpm.scheme_window(scheme, material, h, info["lo"][h], info["hi"][h], kappa, src, gain, grow_only)
    return scheme


def fill_word_slack(scheme, dim, material, types=("v", "C", "F", "J")):
    """Spend the unused bits of the last packed word on wider windows
    (qmpm_scheme_fill_words): each of the given types in turn gets its window doubled (one
    more bit, same resolution) while the packed layout keeps its number of words, until none
    fits.  A dithered run's values spread past the full-precision run's ranges (the noise of
    the stores feeds back through the grid), and this headroom costs no memory traffic."""
    return qmpm.scheme_fill_words(scheme, dim, material, types)[0]


def second_order_scheme(scene, state0, T, eps, info, pairs=2, iters=8, max_step=2, containers=(0, 0, 0, 0),
                        seed=100, margins=None, accept_seeds=(None, 777, 1001, 1002), accept_rounds=6, log=None):
    """Algorithm 1's scheme for the vector evaluation (the final particle positions),
    refined with the second-order term of the error at the resolution it will run at.

    Eq. 6 bounds the second moment of the error; Eq. 8 keeps its linear part.  For the
    position vector the second moment is |b|^2 + tr(Cov) with b the bias vector of the
    final positions, and zero-mean dithered stores of the deformation gradient (a random
    walk over the rollout) or of the positions shift the positions systematically.  Per
    round, for each type h: qmpm_noise_moments of the final positions with errors matched to
    the dithered stores (variance Delta_h^2 Y (1 - Y) at fraction Y, whose average over
    the fraction is sigma_h^2 = Delta_h^2 / 6) at the stores of type h only gives |b_h|^2 and
    the first-order spread; then beta_h = |b_h| / sigma_h^2 (the combined bias |sum_h b_h|
    is at most sum_h |b_h|), g_h = spread_h / sigma_h^2, and the solve's second-order
    refinement of Algorithm 1's scheme adds fraction bits until (sum_h beta_h Delta_h^2 /
    6)^2 + sum_h g_h Delta_h^2 / 6 <= (eps z)^2.  The moments are re-estimated at the
    refined scheme's own noise level (the shift is not quadratic in it; a resolution at which
    a field's runs blow up becomes a lower bound for that field) until the scheme repeats
    or after `iters` rounds, each round moving a type's resolution by at most
    max_step bits (a damped fixed-point iteration), and keeping the finer fraction per type
    where the last two differ.  margins (the solve's window option, {h: (src, gain)}) are
    re-applied at every resolution.  The last packed word's free bits then widen the windows
    (fill_word_slack), and _accept checks the scheme with quantized rollouts against the FP32
    rollout at this resolution, refining it where they miss the bound or saturate.  info:
    the sensitivities and ranges of Algorithm 1 (g_h, lo, hi; the run the ranges come from).
    Returns (scheme, report)."""
    import numpy as np
    material = scene["material"]
    dim = scene["dim"]
    names = ["x", "v", "C", "J" if material == "fluid" else "F"]
    N = state0.shape[0]
    per = [dim, dim, dim * dim, 1 if material == "fluid" else dim * dim]
    P = [float(N * k) for k in per]
    base, res0 = qmpm.solve_scheme(info, eps, containers=containers, material=material, margins=margins)
    g = qmpm.Scene(dict(scene, resort_every=0), None, state0)
    rounds = []
    # a noise level at which a field's runs blow up (non-finite moments) bounds that field's
    # resolution from below (floor) until the end; the field's last finite coefficients
    # stand in for the missing ones
    floor = {n: -(10 ** 9) for n in names}
    last_beta, last_g = [1e30] * 4, [1e30] * 4
    try:
        scheme, prev = base, None
        z = None
        for it in range(iters):
            # errors matched to the dithered stores (variance Delta_h^2 Y (1 - Y) at fraction
            # Y); sigma_h^2 = Delta_h^2 / 6 is its average over the fraction, the scale the
            # solve's moments take
            deltas = [2.0 ** -scheme[n]["frac"] for n in names]
            sig = [d / np.sqrt(6.0) for d in deltas]
            mom = []
            for h in range(4):
                d_h = [deltas[k] if k == h else 0.0 for k in range(4)]
                mom.append(qmpm.qmpm_noise_moments(g.h, T, qmpm.MEASURE_POSITIONS | qmpm.NOISE_MATCHED, d_h,
                                                   seed + 10 * it + h, pairs))
            z = float(np.sqrt(N * mom[0]["z0"])) if np.isfinite(mom[0]["z0"]) else z
            beta, geff = [], []
            for h, m in enumerate(mom):
                if np.isfinite(m["shift"]) and np.isfinite(m["spread"]):
                    last_beta[h] = float(np.sqrt(max(m["shift"], 0.0))) / sig[h] ** 2
                    last_g[h] = float(m["spread"]) / sig[h] ** 2
                else:
                    floor[names[h]] = max(floor[names[h]], scheme[names[h]]["frac"] + 1)
                beta.append(last_beta[h])
                geff.append(last_g[h])
            sol = dict(info, g=geff, P=P, z=z)
            want, res = qmpm.solve_scheme(sol, eps, containers=containers, material=material, beta=beta,
                                          margins=margins)
            nxt = dict(scheme)
            for n in names:
                # the current window, the resolution moved toward the solve's (not below the
                # field's floor) by at most max_step bits, and never past the 24 bits FP32
                # compute decodes exactly
                target = max(want[n]["frac"], floor[n])
                k = max(-max_step, min(max_step, target - scheme[n]["frac"]))
                k = min(k, 24 - scheme[n]["bits"])
                k = max(k, 1 - scheme[n]["bits"])
                nxt = qmpm.scheme_shift(nxt, material, n, k)
            nxt = _margin_windows(nxt, material, info, margins)
            rounds.append({"scheme": scheme, "sigma": sig, "moments": mom, "beta": beta, "g": geff, "solve": want,
                           "next": nxt, "pred_bias": res["pred_bias"], "pred_var": res["pred_var_dither"],
                           "floor": dict(floor)})
            if log:
                log(it, {k: v["bits"] for k, v in nxt.items()}, res["pred_bias"], res["pred_var_dither"], z)
            # each round refines Algorithm 1's scheme with the moments measured at the current
            # one, moving at most max_step bits per type
            seen = [r["scheme"] for r in rounds]
            prev, scheme = scheme, nxt
            if scheme in seen:  # a fixed point, or a cycle: keep the finer of the last two
                break
        if prev is not None and scheme != prev:
            scheme = {n: (scheme[n] if scheme[n]["frac"] >= prev[n]["frac"] else prev[n]) for n in names}
            scheme = _margin_windows(scheme, material, info, margins)
    finally:
        g.close()
    last = rounds[-1] if rounds else None
    scheme = fill_word_slack(scheme, dim, material)
    scheme, accepted = _accept(scene, state0, T, eps, z, scheme, names, last, info, margins, accept_seeds,
                               accept_rounds, log)
    return scheme, {"algorithm1": base, "algorithm1_solve": res0, "rounds": rounds, "z": z, "eps": eps,
                    "acceptance": accepted}


def _accept(scene, state0, T, eps, z, scheme, names, last, info, margins, seeds, max_rounds, log):
    """The acceptance check of a solved scheme at the resolution it runs at: the quantized
    rollouts (one per dither seed in seeds) against the FP32 rollout of the same scene.
    The scheme is accepted when the mean over the seeds of the summed squared error of
    the final positions is within (eps z)^2 (Eq. 6 for the position vector) and no store
    saturated.  Otherwise a type that saturated gets its window doubled about its middle,
    and while the error is above the bound the type with the largest share of the
    predicted second moment (beta_h sigma_h^2 sum_k beta_k sigma_k^2 + g_h sigma_h^2, the
    coefficients of the last round) gets one more fraction bit; at most max_rounds times.
    Returns (scheme, history)."""
    import numpy as np
    dim = scene["dim"]
    material = scene["material"]
    history = []
    if not seeds or max_rounds <= 0 or z is None:
        return scheme, history
    ref = qmpm.Scene(dict(scene), None, state0)
    ref.step(T)
    x32 = ref.state_by_id()[:, :dim]
    ref.close()
    for r in range(max_rounds + 1):
        err2, sat = [], np.zeros(4, dtype=np.int64)
        for sd in seeds:
            q = qmpm.Scene(dict(scene, seed=sd) if sd is not None else dict(scene), scheme, state0, stats=True)
            q.step(T)
            x = q.state_by_id()[:, :dim]
            sat += np.asarray(q.readback(state=False, ids=False)["stats"]["saturations"][:4], dtype=np.int64)
            q.close()
            err2.append(float(((x - x32) ** 2).sum()) if np.isfinite(x).all() else float("inf"))
        rel = float(np.sqrt(np.mean(err2))) / z
        history.append({"scheme": scheme, "rel_err": rel, "saturations": sat.tolist(),
                        "seeds": [sd for sd in seeds]})
        if log:
            log("accept", {n: scheme[n]["bits"] for n in names}, rel, sat.tolist())
        if rel <= eps and not sat.any():
            break
        if r == max_rounds:
            break
        nxt = dict(scheme)
        for h, n in enumerate(names):
            if sat[h] > 0:
                nxt = qmpm.scheme_widen(nxt, material, n)
        if rel > eps:
            sig2 = [2.0 ** (-2 * scheme[n]["frac"]) / 6.0 for n in names]
            beta = last["beta"] if last else [0.0] * 4
            gg = last["g"] if last else [1.0] * 4
            B = sum(b * s2 for b, s2 in zip(beta, sig2))
            share = [beta[h] * sig2[h] * B + gg[h] * sig2[h] if scheme[names[h]]["bits"] < 24 else -1.0
                     for h in range(4)]
            h = int(np.argmax(share))
            nxt = qmpm.scheme_shift(nxt, material, names[h], 1)
        scheme = _margin_windows(nxt, material, info, margins, grow_only=True)
    return scheme, history


def c_noise_margin(grid_log2):
    """The solve's window margin for C (type 2) from the velocity noise (type 1): the
    recorded C range comes from the unquantized run, where C of a rigidly moving body is
    nearly zero; in the quantized run the dithered velocities (resolution Delta_v) make the
    grid velocities noisy, and C = D^-1 sum_i w_i v_i (x_i - x_p)^T picks that noise up with
    a gain of about 6 n (sum_i w_i |x_i - x_p| <= 1.5 dx, D^-1 = 4 / dx^2).  The solve keeps
    C's resolution and widens its window by 6 n Delta_v on each side."""
    return {2: (1, 6.0 * (1 << grid_log2))}


def serving_schemes(eps_list=scenes.SERVING_EPS, n_rep=20000, samples=2, seed=11, reference="displacement",
                    kappa=4.0):
    """Schemes for the serving workload: for every class (2D/3D x elastic/fluid) and grid,
    the sensitivities of the final positions of a representative scene of that class and
    grid (about n_rep particles, the serving step count), then Eq. 10 at each error bound,
    relative to the RMS displacement over the rollout (the bodies move a few cells in 200
    steps; measured from the origin, the bound would allow errors of many cells).  The x
    window is the unit domain (every request's body lies in it), the other windows the
    representative's recorded ranges widened by kappa (4: a request's body differs from the
    representative in size, so its fields spread further), C's also by the velocity noise it
    picks up (c_noise_margin).  Returns {(dim, material, grid_log2, eps): scheme}."""
    out = {}
    for dim, material in scenes.SERVING_CLASSES:
        for grid_log2 in scenes.SERVING_GRIDS[dim]:
            sc, s0 = scenes.serving_scene(dim, material, n_rep, grid_log2, seed)
            info = position_sensitivities(sc, s0, sc["steps"], samples=samples, ckpt_every=25,
                                          reference=reference)
            info["lo"][0], info["hi"][0] = 0.5 - 0.5 / kappa, 0.5 + 0.5 / kappa  # widened: [0, 1]
            for eps in eps_list:
                scheme, _ = qmpm.solve_scheme(info, eps, material=material, kappa=kappa,
                                              margins=c_noise_margin(grid_log2))
                out[(dim, material, grid_log2, eps)] = scheme
    return out


def iterate_scheme(scene, state0, T, eps, measure=qmpm.MEASURE_KINETIC_ENERGY, max_iter=6, ckpt_every=32,
                   kappa=2.0, containers=(0, 0, 0, 0)):
    """Algorithm 1 with the iterative re-linearisation the paper discusses (Sec. 4): the
    first solve linearises at the full-precision run; every further round re-runs the
    adjoint along the quantized trajectory of the current scheme (gradients and ranges at
    the quantized solution) and solves again, keeping the error budget (eps z)^2 of the
    full-precision z, until the scheme repeats (a fixed point or a two-cycle) or max_iter
    rounds.  Returns (scheme, history), history a list of per-round dicts with the bits,
    fractions and g_h."""
    material = scene["material"]
    info0 = qmpm.sensitivities(scene, state0, T, ckpt_every, measure)
    z_ref = info0["z"]
    scheme, res = qmpm.solve_scheme(info0, eps, kappa=kappa, containers=containers, material=material)
    history = [{"bits": res["bits"], "frac": res["frac"], "g": info0["g"], "quantized_forward": False}]
    seen = [scheme]
    for _ in range(1, max_iter):
        g = qmpm.Scene(dict(scene, resort_every=0), scheme, state0)
        info = qmpm.qmpm_adjoint(g.h, T, ckpt_every, measure | qmpm.ADJ_QUANTIZED_FORWARD)
        g.close()
        info["z"] = z_ref
        scheme, res = qmpm.solve_scheme(info, eps, kappa=kappa, containers=containers, material=material)
        history.append({"bits": res["bits"], "frac": res["frac"], "g": info["g"], "quantized_forward": True})
        if scheme in seen[-2:]:
            break
        seen.append(scheme)
    return scheme, history


def cubes3d_second_order_scheme(eps=0.01, cube_cells=40, grid_log2=8, T=None, pairs=2, iters=8, log=None):
    """The cubes' scheme at relative error eps on the final positions, Algorithm 1 plus the
    second-order refinement: the sensitivities g_h come from the same 16 cubes at half
    resolution (the scaling procedure of Sec. 8.3), the ranges from the FP32 run at the
    resolution the scheme runs at (so C's window holds its full-resolution values), and
    second_order_scheme refines the scheme there.  Returns (scheme, report)."""
    sc_lo, s0_lo = scenes.cubes3d_scene(cube_cells=cube_cells // 2, grid_log2=grid_log2 - 1)
    sc, s0 = scenes.cubes3d_scene(cube_cells=cube_cells, grid_log2=grid_log2)
    steps = T if T is not None else sc["steps"]
    info_lo = position_sensitivities(sc_lo, s0_lo, steps)
    rng_hi = qmpm.sensitivities(sc, s0, steps)  # the forward records the ranges
    info = dict(info_lo, lo=rng_hi["lo"], hi=rng_hi["hi"])
    scheme, rep = second_order_scheme(sc, s0, steps, eps, info, pairs=pairs, iters=iters,
                                      containers=(64, 0, 0, 0), margins=c_noise_margin(grid_log2), log=log)
    rep["sensitivities"] = {k: info_lo[k] for k in ("g", "z", "P")}
    rep["ranges"] = {"lo": list(rng_hi["lo"]), "hi": list(rng_hi["hi"])}
    return scheme, rep


SCHEME_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "schemes")


def cached_scheme_path(name, eps):
    return os.path.join(SCHEME_DIR, f"{name}_eps{eps:g}.json")


def load_cubes3d_scheme(eps=0.01):
    """The cubes' second-order scheme as written by `python -m paper_2207_04658_b300.autoquant
    cubes3d --eps EPS` (it takes several minutes to compute), with the hash of the scene it
    was computed for; None when absent or computed for another scene."""
    import json
    path = cached_scheme_path("cubes3d", eps)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    sc, s0 = scenes.cubes3d_scene()
    if d.get("scene_hash") != scene_hash(sc, s0):
        return None
    return d


def scene_hash(sc, s0):
    import hashlib
    import json
    import numpy as np
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(s0, dtype=np.float64).tobytes())
    h.update(json.dumps({k: sc[k] for k in sorted(sc) if k not in ("resort_every",)}, sort_keys=True,
                        default=str).encode())
    return h.hexdigest()


def _summary(rep):
    rounds = []
    for r in rep["rounds"]:
        rounds.append({"scheme": r["scheme"], "beta": r["beta"], "g": r["g"], "pred_bias": r["pred_bias"],
                       "pred_var": r["pred_var"], "floor": r["floor"],
                       "moments": [{k: m[k] for k in ("shift", "spread", "z0")} for m in r["moments"]]})
    return {"algorithm1": rep["algorithm1"], "rounds": rounds, "z": rep["z"], "eps": rep["eps"],
            "sensitivities": rep["sensitivities"], "ranges": rep["ranges"],
            "acceptance": rep.get("acceptance", [])}


def main():
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(description="solve and cache a workload's second-order scheme")
    ap.add_argument("workload", choices=["cubes3d"])
    ap.add_argument("--eps", type=float, default=0.01)
    args = ap.parse_args()
    t0 = time.time()
    scheme, rep = cubes3d_second_order_scheme(args.eps, log=lambda *a: print(f"[{time.time() - t0:6.0f}s]", *a,
                                                                               flush=True))
    sc, s0 = scenes.cubes3d_scene()
    out = {"what": "3D fixed-corotated cubes (8,192,000 particles, 256^3): Algorithm 1 from half-resolution "
                   "sensitivities, refined with the second-order term at full resolution and accepted by FP32-referenced "
                   "rollouts there",
           "eps": args.eps, "scheme": scheme, "scene_hash": scene_hash(sc, s0), "report": _summary(rep),
           "seconds": time.time() - t0}
    os.makedirs(SCHEME_DIR, exist_ok=True)
    path = cached_scheme_path(args.workload, args.eps)
    with open(path, "w") as f:
        json.dump(out, f, indent=1, default=float)
    print(path, {k: (v["bits"], v["frac"]) for k, v in scheme.items()})



def dambreak3d_schemes(eps_list=(0.1, 0.01), cells=256, grid_log2=9, factor=4, T=None, samples=2):
    """Schemes of Algorithm 1 for the 3D dam break at the given relative error bounds on the
    final particle positions (the scaling procedure of Sec. 8.3): the sensitivities and
    ranges of the column at 1/factor resolution (cells / factor cells on a grid factor times
    coarser, same dt and step count), the affine field C's window scaled by the resolution
    ratio (C is a velocity gradient: it grows like 1 / dx), bit pack, the last word's free
    bits spent on wider windows of v, C and J (fill_word_slack: the dithered J wanders
    past the range of the full-precision run).  Returns
    {eps: (scheme, solve report)} and the sensitivity report."""
    k = factor.bit_length() - 1
    sc_lo, s0_lo = scenes.dambreak3d_scene(column_cells=cells // factor, grid_log2=grid_log2 - k)
    steps = T if T is not None else sc_lo["steps"]
    info = position_sensitivities(sc_lo, s0_lo, steps, samples=samples)
    lo, hi = list(info["lo"]), list(info["hi"])
    mid, half = 0.5 * (lo[2] + hi[2]), 0.5 * (hi[2] - lo[2]) * factor
    lo[2], hi[2] = mid - half, mid + half
    info_hi = dict(info, lo=lo, hi=hi)
    out = {}
    for eps in eps_list:
        scheme, res = qmpm.solve_scheme(info_hi, eps, material="fluid")
        out[eps] = (fill_word_slack(scheme, 3, "fluid"), res)
    return out, info


if __name__ == "__main__":
    main()
