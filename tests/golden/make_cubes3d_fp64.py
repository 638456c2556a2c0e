#!/usr/bin/env python
"""Write the FP64 reference rollout of the 3D elastic cubes (the stand-in for the falling
elastic blocks of Sec. 8.1) computed by the CPU oracle alone.

    python tests/golden/make_cubes3d_fp64.py [--half] [--steps 1000] [--threads N]

The unquantized FP64 oracle step (threaded build of the same C sources; its P2G sums are
atomic, so the last bits vary between runs) is applied ``steps`` times from the scene's
seeded initial state.  The fixture holds z = mean |x|^2 every 100 steps, the final
z and sum |x|^2, and the final positions of every ``sample_every``-th particle (by
initial index), with the hash of the initial state it was computed from.  Nothing here
touches the CUDA library.
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2207_04658_b300 import scenes  # noqa: E402


def scene_for(half):
    if half:
        return scenes.cubes3d_scene(cube_cells=20, grid_log2=7)
    return scenes.cubes3d_scene()


def state_hash(sc, s0):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(s0, dtype=np.float64).tobytes())
    h.update(json.dumps({k: sc[k] for k in sorted(sc) if k != "steps"}, sort_keys=True,
                        default=str).encode())
    return h.hexdigest()


def fixture_name(half, steps):
    return f"cubes3d_fp64_{'n128' if half else 'n256'}_T{steps}.json"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--half", action="store_true", help="the 1,024,000-particle 128^3 scene")
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--sample-every", type=int, default=None)
    args = ap.parse_args()
    sc, s0 = scene_for(args.half)
    N = s0.shape[0]
    every = args.sample_every or max(1, N // 2048)
    ro = oracle.Fp64Rollout(sc, s0, threaded=True)
    z_hist = [[0, oracle.mean_sq_pos(3, s0)]]
    t0 = time.time()
    for t in range(1, args.steps + 1):
        ro.step(1)
        if t % 100 == 0 or t == args.steps:
            z_hist.append([t, oracle.mean_sq_pos(3, ro.s)])
            print(f"step {t} z {z_hist[-1][1]:.12g} ({time.time() - t0:.0f} s)", flush=True)
    assert np.all(np.isfinite(ro.s))
    pos = np.empty((N, 3))
    pos[ro.ids] = ro.s[:, :3]
    ids = np.arange(0, N, every)
    out = {
        "what": "FP64 oracle rollout (unquantized MLS-MPM, Sec. 8.1 simulator) of the 3D "
                "fixed-corotated cubes; positions of sampled particles by initial index",
        "scene": {k: (list(v) if isinstance(v, tuple) else v) for k, v in sc.items()},
        "particles": N, "steps": args.steps, "state_hash": state_hash(sc, s0),
        "z_history": z_hist, "z": z_hist[-1][1], "sum_sq_pos": float((pos ** 2).sum()),
        "sample_every": every, "sample_ids": ids.tolist(),
        "sample_pos": [[float(v) for v in p] for p in pos[ids]],
        "seconds": time.time() - t0,
    }
    path = os.path.join(HERE, fixture_name(args.half, args.steps))
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print(path)


if __name__ == "__main__":
    main()
