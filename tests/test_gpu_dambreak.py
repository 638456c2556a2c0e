"""The 3D dam break (the weakly compressible fluid of Sec. 8.3's scaling experiment) at
reduced size: a 64^3-cell column on a 128^3 grid (2,097,152 particles), 500 steps, with the
schemes Algorithm 1 solves at relative error bounds 0.1 and 0.01 on the final positions from
the column at quarter resolution (the scaling procedure), against the FP64 oracle rollout
stored in tests/golden/dambreak3d_fp64_c64_n128_T500.json (written by
make_dambreak3d_fp64.py with the oracle alone).  Bars, for dithered stores and two seeds:
z within eps of the FP64 run and the RMS position error within the paper's 3 eps band
(Sec. 8.1); the FP32 run within 1e-3 of the FP64 one.  Round-to-nearest stores of the
same schemes are run and reported beside them."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def case():
    import sys
    import torch
    from paper_2207_04658_b300 import autoquant, qmpm, scenes
    assert torch.cuda.is_available()
    path = os.path.join(GOLDEN, "dambreak3d_fp64_c64_n128_T500.json")
    if not os.path.exists(path):
        pytest.skip("dambreak3d_fp64_c64_n128_T500.json has not been generated")
    with open(path) as f:
        ref = json.load(f)
    sys.path.insert(0, GOLDEN)
    import make_cubes3d_fp64 as mk
    sc, s0 = scenes.dambreak3d_scene(column_cells=64, grid_log2=7)
    assert ref["state_hash"] == mk.state_hash(sc, s0)
    schemes, info = autoquant.dambreak3d_schemes((0.1, 0.01), cells=64, grid_log2=7, factor=4)
    return qmpm, sc, s0, ref, schemes


def run(qmpm, sc, s0, scheme, T):
    g = qmpm.Scene(sc, scheme, s0, stats=scheme is not None)
    g.step(T)
    st = g.state_by_id()
    stats = g.readback(state=False, ids=False)["stats"]
    g.close()
    return st, stats


def errors(st, ref):
    ids = np.asarray(ref["sample_ids"])
    xr = np.asarray(ref["sample_pos"])
    dx = float(np.sqrt(((st[ids, :3] - xr) ** 2).sum(1).mean()) / np.sqrt((xr ** 2).sum(1).mean()))
    z = float((st[:, :3] ** 2).sum(1).mean())
    return abs(z - ref["z"]) / ref["z"], dx


def test_fp32_dambreak_matches_fp64(case):
    qmpm, sc, s0, ref, _ = case
    st, _ = run(qmpm, sc, s0, None, ref["steps"])
    dz, dx = errors(st, ref)
    assert dz <= 1e-3 and dx <= 1e-3, (dz, dx)


@pytest.mark.parametrize("eps", [0.1, 0.01])
def test_solved_dambreak_schemes_within_the_bound(case, eps):
    qmpm, sc, s0, ref, schemes = case
    scheme, res = schemes[eps]
    report = {}
    for seed in (None, 4242):
        st, stats = run(qmpm, dict(sc, seed=seed) if seed else sc, s0, scheme, ref["steps"])
        assert np.isfinite(st).all()
        dz, dx = errors(st, ref)
        report[seed] = (dz, dx, stats["saturations"])
        assert dz <= eps and dx <= 3 * eps, (eps, seed, dz, dx, res["bits"], stats["saturations"])
    st, stats = run(qmpm, dict(sc, dither=False), s0, scheme, ref["steps"])
    report["nearest"] = errors(st, ref)
    print(eps, res["bits"], report)
