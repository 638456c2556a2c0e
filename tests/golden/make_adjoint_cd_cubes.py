#!/usr/bin/env python
"""Write FP64 central differences for the full-size adjoint case, computed by the CPU
oracle alone: the 3D fixed-corotated elastic cubes with 1,024,000 particles on a 128^3 grid,
256 steps, z = mean |x_T|^2 (Sec. 6, Eq. 12-13).

    python tests/golden/make_adjoint_cd_cubes.py [--workers 6] [--steps 256] [--count 64]

64 injected errors (step t, particle p by initial index, component c) are drawn with seed 4.
An error injected into the stored state s_t moves z by dz/ds_t (the quantized store of
Eq. 1 is s_t = F(s_{t-1}) + e_t, so dz/de_t = dz/ds_t).  For each injection the
unquantized FP64 oracle step is applied T - t times from s_t + h e and from s_t - h e, and
    fd = sum_p (|x+_p|^2 - |x-_p|^2) / (2 h N),
summed particle by particle so that the particles the injection never reaches cancel
exactly.  The base states s_t come from one FP64 rollout from the scene's seeded initial
state.  The sequential oracle is used (one process per injection): its P2G sums run in
particle order, so both runs of a pair differ only where the injection reaches.
Nothing here touches the CUDA library.
"""
import argparse
import json
import multiprocessing as mp
import os
import shutil
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

NAME = "adjoint_cd_cubes_n128_T256.json"
# step per field (x, v, C, F), times max(1, |s|): small for x and v, larger for the weakly
# coupled C and F so that the difference of z stands above FP64 rounding
H_FIELD = (1e-6, 1e-5, 1e-3, 1e-4)


def scene():
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.cubes3d_scene(n_cubes=2, cube_cells=40, ppc_axis=2, grid_log2=7, seed=4,
                                  material="corotated", dt=5e-5)
    return dict(sc, resort_every=0), s0


def field_of(c):
    return 0 if c < 3 else 1 if c < 6 else 2 if c < 15 else 3


def injections(N, T, count, seed=4):
    gen = np.random.default_rng(seed)
    t = gen.integers(0, T, count)
    p = gen.integers(0, N, count)
    c = gen.integers(0, 24, count)
    return [(int(a), int(b), int(d)) for a, b, d in zip(t, p, c)]


def _job(args):
    tdir, t, p, c, T = args
    import oracle
    sc, _ = scene()
    ph = oracle.make_phys(sc)
    base = np.load(os.path.join(tdir, f"s{t}.npy"))
    h = H_FIELD[field_of(c)] * max(1.0, abs(base[p, c]))
    grid = np.zeros(oracle.n_nodes(ph) * (1 + ph.dim))
    xs = []
    for sgn in (1.0, -1.0):
        st = base.copy()
        st[p, c] += sgn * h
        for _ in range(T - t):
            st = oracle.step_fp64(ph, st, grid)
        xs.append(st[:, :3].copy())
    dp = (xs[0] ** 2).sum(1) - (xs[1] ** 2).sum(1)
    N = base.shape[0]
    fd = float(dp.sum() / (2.0 * h * N))
    return {"t": t, "p": p, "c": c, "h": h, "fd": fd, "reached": int(np.count_nonzero(dp)),
            "z_plus": float((xs[0] ** 2).sum() / N), "z_minus": float((xs[1] ** 2).sum() / N)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 2))
    ap.add_argument("--steps", type=int, default=256)
    ap.add_argument("--count", type=int, default=64)
    args = ap.parse_args()
    import oracle
    sys.path.insert(0, HERE)
    import make_cubes3d_fp64 as mk
    sc, s0 = scene()
    N, T = s0.shape[0], args.steps
    inj = injections(N, T, args.count)
    need = sorted(set(t for t, _, _ in inj))
    tdir = tempfile.mkdtemp(prefix="qmpm_cd_")
    t0 = time.time()
    try:
        ph = oracle.make_phys(sc)
        grid = np.zeros(oracle.n_nodes(ph) * (1 + ph.dim))
        s = np.ascontiguousarray(s0, dtype=np.float64).copy()
        for t in range(T + 1):
            if t in need:
                np.save(os.path.join(tdir, f"s{t}.npy"), s)
            if t == T:
                break
            s = oracle.step_fp64(ph, s, grid)
        z_T = float((s[:, :3] ** 2).sum() / N)
        print(f"base rollout {time.time() - t0:.0f} s, z_T {z_T:.12g}", flush=True)
        jobs = sorted(((tdir, t, p, c, T) for t, p, c in inj), key=lambda j: j[1])  # longest first
        ctx = mp.get_context("spawn")
        with ctx.Pool(args.workers) as pool:
            res = []
            for r in pool.imap_unordered(_job, jobs):
                res.append(r)
                print(f"{len(res)}/{len(jobs)} t={r['t']} p={r['p']} c={r['c']} fd={r['fd']:.6g} "
                      f"({time.time() - t0:.0f} s)", flush=True)
    finally:
        shutil.rmtree(tdir, ignore_errors=True)
    order = {j: i for i, j in enumerate(inj)}
    res.sort(key=lambda r: order[(r["t"], r["p"], r["c"])])
    out = {
        "what": "FP64 oracle central differences dz/ds_t of z = mean |x_T|^2 for injected errors "
                "(Sec. 6, Eq. 12-13) on the 3D fixed-corotated cubes, 1,024,000 particles, 128^3",
        "scene": {k: (list(v) if isinstance(v, tuple) else v) for k, v in sc.items()},
        "particles": N, "steps": T, "state_hash": mk.state_hash(sc, s0), "z_T": z_T,
        "seed": 4, "h_field": list(H_FIELD), "injections": res, "seconds": time.time() - t0,
    }
    path = os.path.join(HERE, NAME)
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print(path)


if __name__ == "__main__":
    main()
