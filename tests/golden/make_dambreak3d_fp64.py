#!/usr/bin/env python
"""Write the FP64 reference rollout of a reduced 3D dam break (the weakly compressible fluid
column of Sec. 8.3's scaling experiment, at reduced size) computed by the CPU oracle alone.

    python tests/golden/make_dambreak3d_fp64.py [--cells 32] [--grid-log2 6] [--steps 500]

The unquantized FP64 oracle step (threaded build of the same C sources) is applied `steps`
times from the scene's seeded initial state.  The fixture holds z = mean |x|^2 every 100
steps, the final z, and the final positions of every k-th particle (by initial index, about
2,048 of them), with the hash of the initial state.  Nothing here touches the CUDA library.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from make_cubes3d_fp64 import state_hash  # noqa: E402
from paper_2207_04658_b300 import scenes  # noqa: E402


def fixture_name(cells, grid_log2, steps):
    return f"dambreak3d_fp64_c{cells}_n{1 << grid_log2}_T{steps}.json"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cells", type=int, default=32)
    ap.add_argument("--grid-log2", type=int, default=6)
    ap.add_argument("--steps", type=int, default=500)
    args = ap.parse_args()
    sc, s0 = scenes.dambreak3d_scene(column_cells=args.cells, grid_log2=args.grid_log2)
    N = s0.shape[0]
    every = max(1, N // 2048)
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
        "what": "FP64 oracle rollout (unquantized MLS-MPM, weakly compressible fluid) of a reduced 3D dam "
                "break; positions of sampled particles by initial index",
        "scene": {k: (list(v) if isinstance(v, tuple) else v) for k, v in sc.items()},
        "particles": N, "steps": args.steps, "state_hash": state_hash(sc, s0),
        "z_history": z_hist, "z": z_hist[-1][1], "sample_every": every, "sample_ids": ids.tolist(),
        "sample_pos": [[float(v) for v in p] for p in pos[ids]], "seconds": time.time() - t0,
    }
    path = os.path.join(HERE, fixture_name(args.cells, args.grid_log2, args.steps))
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print(path)


if __name__ == "__main__":
    main()
