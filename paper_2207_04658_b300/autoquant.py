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


def position_sensitivities(scene, state0, T, samples=2, ckpt_every=32, seed=0):
    """Sensitivities of the final particle positions as a whole: the evaluation is the
    vector of final positions x_T, and Eq. 8 summed over its N d outputs gives
    G_h = sum_m sum_t sum_i (d x_T,m / d e_{t,i})^2, the trace of J J^T over the
    variables of type h.  It is estimated with ``samples`` adjoint runs seeded with
    independent standard normal vectors u on x_T (E[(u^T J)^2] = trace(J J^T)).
    Returns the adjoint report with g replaced by G and z by sqrt(sum_m |x_T,m|^2)
    (so that (eps z)^2 bounds the summed squared position error, i.e. the RMS position
    error stays below eps times the RMS position)."""
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
    g.close()
    out = dict(info)
    out["g"] = list(acc / samples)
    out["z"] = float(np.sqrt(N * info["z"]))  # info["z"] is the mean square position of x_T
    out["samples"] = samples
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
