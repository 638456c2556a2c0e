"""Full rollouts of the 3D elastic cubes against the FP64 oracle rollout stored in
tests/golden/cubes3d_fp64_*.json (written by tests/golden/make_cubes3d_fp64.py, which calls
only the oracle).

The evaluation function is the vector of final positions (relative error bound eps on the
positions: RMS position error <= eps x RMS position) with z = mean |x|^2 reported beside it.
Bars: the FP32 run of the library's kernels matches the FP64 oracle to 1e-3 relative in z
and RMS position (both integrate the same explicit scheme; FP32 rounding in a stiff,
colliding scene grows to that size over 1000 steps).  The quantized runs keep z within eps
of the FP64 run and the RMS position error within the paper's success band (Sec. 8.1:
3 eps), for two dither seeds:
  * Algorithm 1 alone, from the half-resolution sensitivities, on the half-resolution scene
    (its linear error model holds there within a factor of about 3);
  * the second-order scheme (Algorithm 1 refined with the bias and spread that noise
    injection measures at the resolution the scheme runs at) at both resolutions: the one
    committed for the full-resolution benchmark, and one solved here for the
    half-resolution scene.  Algorithm 1 alone reaches 2.6 eps at full resolution, where the
    dithered deformation gradient's random walk shifts the positions systematically; its
    saturations are counted and must be zero for the second-order schemes.
Positions are compared on the stored sample of particles (every k-th particle by initial
index)."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def q():
    import torch
    from paper_2207_04658_b300 import qmpm
    assert torch.cuda.is_available()
    qmpm.lib()
    return qmpm


def load(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} has not been generated")
    with open(path) as f:
        return json.load(f)


def scene_of(half):
    from paper_2207_04658_b300 import scenes
    if half:
        return scenes.cubes3d_scene(cube_cells=20, grid_log2=7)
    return scenes.cubes3d_scene()


def check_fixture(ref, sc, s0):
    import sys
    sys.path.insert(0, GOLDEN)
    import make_cubes3d_fp64 as mk
    assert ref["state_hash"] == mk.state_hash(sc, s0)
    assert ref["particles"] == s0.shape[0]


def rollout(q, sc, s0, scheme, T):
    g = q.Scene(sc, scheme, s0, stats=True)
    g.step(T)
    st = g.state_by_id()
    stats = g.readback(state=False, ids=False)["stats"]
    g.close()
    return st, stats


def compare(st, ref):
    ids = np.asarray(ref["sample_ids"])
    xr = np.asarray(ref["sample_pos"])
    x = st[ids, :3]
    rms_err = float(np.sqrt(((x - xr) ** 2).sum(1).mean()))
    rms_pos = float(np.sqrt((xr ** 2).sum(1).mean()))
    z = float((st[:, :3] ** 2).sum(1).mean())
    return abs(z - ref["z"]) / ref["z"], rms_err / rms_pos


@pytest.mark.parametrize("half", [True, False])
def test_fp32_rollout_matches_fp64_oracle(q, half):
    ref = load(f"cubes3d_fp64_{'n128' if half else 'n256'}_T1000.json")
    sc, s0 = scene_of(half)
    check_fixture(ref, sc, s0)
    st, stats = rollout(q, sc, s0, None, ref["steps"])
    dz, dx = compare(st, ref)
    assert dz <= 1e-3 and dx <= 1e-3, (dz, dx)


@pytest.fixture(scope="module")
def solved():
    from paper_2207_04658_b300 import autoquant
    scheme, rep = autoquant.cubes3d_scheme(0.01)
    return scheme, rep


def test_algorithm1_scheme_rollout_within_the_error_bound(q, solved):
    ref = load("cubes3d_fp64_n128_T1000.json")
    sc, s0 = scene_of(True)
    check_fixture(ref, sc, s0)
    scheme, rep = solved
    eps = 0.01
    # the predicted error (Eq. 8) of the solved scheme is within the bound by construction
    assert rep["solve"]["pred_err"] <= (eps * rep["sensitivities"]["z"]) ** 2
    for seed in (None, 777):
        st, stats = rollout(q, dict(sc, seed=seed) if seed else sc, s0, scheme, ref["steps"])
        assert np.isfinite(st).all()
        dz, dx = compare(st, ref)
        assert dz <= eps and dx <= 3 * eps, (seed, dz, dx)


@pytest.fixture(scope="module")
def second_order():
    from paper_2207_04658_b300 import autoquant
    full = autoquant.load_cubes3d_scheme(0.01)
    full = full["scheme"] if full is not None else autoquant.cubes3d_second_order_scheme(0.01)[0]
    half, rep = autoquant.cubes3d_second_order_scheme(0.01, cube_cells=20, grid_log2=7)
    return {False: full, True: half}


@pytest.mark.parametrize("half", [True, False])
def test_second_order_scheme_rollout_within_the_error_bound(q, second_order, half):
    ref = load(f"cubes3d_fp64_{'n128' if half else 'n256'}_T1000.json")
    sc, s0 = scene_of(half)
    check_fixture(ref, sc, s0)
    scheme = second_order[half]
    eps = 0.01
    for seed in (None, 777):
        st, stats = rollout(q, dict(sc, seed=seed) if seed else sc, s0, scheme, ref["steps"])
        assert np.isfinite(st).all()
        dz, dx = compare(st, ref)
        assert dz <= eps and dx <= 3 * eps, (half, seed, dz, dx, scheme)
        assert stats["saturations"] == [0, 0, 0, 0], stats["saturations"]
