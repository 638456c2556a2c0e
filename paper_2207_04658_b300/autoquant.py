"""Algorithm 1 end to end: a quantization scheme for a scene from its sensitivities.

The paper's workflow (Sec. 4, Algorithm 1; scaling procedure of Sec. 8.3): run the
full-precision simulation at low resolution, record each field's range, back-propagate
the evaluation function to get the accumulated squared sensitivities g_h (Eq. 8), solve
Eq. 10 (or its memory-bound form) for the bit widths, and apply the scheme to the
high-resolution run.  Forward and backward passes run in the library's FP32 adjoint;
the solve is the library's host solver.
"""
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
