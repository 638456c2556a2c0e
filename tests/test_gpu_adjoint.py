"""Device adjoint (Sec. 6, Eq. 12-13) and the sensitivities of Eq. 8, through the C ABI.

Bars: FP32 device reverse mode vs the FP64 oracle reverse mode and FP64 central
differences within 2e-3 of each field's scale (the adjoint sums thousands of FP32
products over several steps); g_h within 2e-3 relative; the error-bound scheme solved
from these sensitivities keeps a quantized rollout's measurement within 3 eps z of the FP64
run (the paper's success criterion, Sec. 8.1)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    from paper_2207_04658_b300 import qmpm
    assert torch.cuda.is_available()
    qmpm.lib()
    return qmpm


def small(dim, material, N_side=12, seed=0, grid_log2=None):
    from paper_2207_04658_b300 import scenes
    gen = np.random.default_rng(seed)
    n = 1 << (grid_log2 or (6 if dim == 2 else 5))
    lo = np.full(dim, 0.45)
    x = scenes.jitter_box(gen, lo, np.full(dim, 0.1), (N_side,) * dim)
    s0 = scenes.initial_state(dim, material, x, v0=gen.normal(0, 0.3, dim))
    N = s0.shape[0]
    s0[:, 2 * dim:2 * dim + dim * dim] = gen.normal(0, 1.0, (N, dim * dim))
    off = 2 * dim + dim * dim
    if material == "fluid":
        s0[:, off] = 1.0 + gen.uniform(-0.02, 0.02, N)
    else:
        s0[:, off:] += 0.03 * gen.normal(0, 1, (N, dim * dim))
    sc = dict(dim=dim, material=material, grid_log2=int(np.log2(n)), bound=3, dt=2e-4, E=2e3, nu=0.3,
              bulk=300.0, rho=1.0, p_vol=(0.1 ** dim) / N, gravity=(0.5, -9.8, 1.0), seed=1, dither=True,
              resort_every=0)
    return sc, s0


def device_grad0(q, sc, s0, T, k):
    import torch
    g = q.Scene(sc, None, s0)
    ids = g.readback(state=False, ids=True)["ids"]
    d = torch.empty((s0.shape[0], s0.shape[1]), dtype=torch.float32, device="cuda")
    info = q.qmpm_adjoint(g.h, T, k, q.MEASURE_MEAN_SQ_POS, 0, d.data_ptr())
    g.close()
    grad = np.empty((s0.shape[0], s0.shape[1]))
    grad[ids] = d.cpu().numpy()
    return grad, info


def field_slices(dim, nc):
    b = [0, dim, 2 * dim, 2 * dim + dim * dim, nc]
    return [slice(b[h], b[h + 1]) for h in range(4)]


def close_by_field(got, ref, dim, rel=2e-3):
    for sl in field_slices(dim, ref.shape[1]):
        scale = np.abs(ref[:, sl]).max() + 1e-30
        err = np.abs(got[:, sl] - ref[:, sl]).max()
        assert err <= rel * scale, (sl, err, scale)


CASES = [(2, "neohookean"), (2, "corotated"), (2, "fluid"), (3, "corotated"), (3, "fluid"), (3, "neohookean")]


@pytest.mark.parametrize("dim,material", CASES)
def test_adjoint_matches_oracle_reverse_mode(q, oracle, dim, material):
    sc, s0 = small(dim, material, N_side=16 if dim == 2 else 8, seed=dim)
    T = 6
    grad, info = device_grad0(q, sc, s0, T, 4)
    ph = oracle.make_phys(sc)
    z, adj, g = oracle.rollout_adjoint(ph, s0, T)
    assert abs(info["z"] - z) <= 1e-5 * abs(z)
    close_by_field(grad, adj[0], dim)
    assert np.allclose(info["g"], g, rtol=2e-3)
    # recorded ranges of the forward states (Algorithm 1's range update)
    states = oracle.rollout_fp64(ph, s0, T)
    allst = np.concatenate(states)
    for h, sl in enumerate(field_slices(dim, s0.shape[1])):
        assert abs(info["lo"][h] - allst[:, sl].min()) <= 1e-4 * (np.abs(allst[:, sl]).max() + 1e-6)
        assert abs(info["hi"][h] - allst[:, sl].max()) <= 1e-4 * (np.abs(allst[:, sl]).max() + 1e-6)
    assert info["P"] == [s0.shape[0] * k for k in (dim, dim, dim * dim, s0.shape[1] - 2 * dim - dim * dim)]


def test_injected_errors_against_fp64_central_differences(q, oracle):
    # 64 (step, particle, component) errors injected into the FP64 rollout; the device
    # adjoint from the state at that step gives dz/de = dz/ds_t (Eq. 1)
    sc, s0 = small(3, "corotated", N_side=8, seed=9)
    T = 12
    ph = oracle.make_phys(sc)
    states = oracle.rollout_fp64(ph, s0, T)
    gen = np.random.default_rng(5)
    steps = sorted(set(int(t) for t in gen.integers(0, T, 8)))
    checked = 0
    for t in steps:
        grad_t, _ = device_grad0(q, sc, states[t], T - t, 4)
        scales = [np.abs(grad_t[:, sl]).max() for sl in field_slices(3, s0.shape[1])]
        for _ in range(64 // len(steps) + 1):
            if checked == 64:
                break
            p = int(gen.integers(0, s0.shape[0]))
            c = int(gen.integers(0, s0.shape[1]))
            fld = 0 if c < 3 else 1 if c < 6 else 2 if c < 15 else 3
            # step per field: large enough that the difference of z rises above FP64
            # rounding for the weakly coupled fields (C, F), small for x and v
            h = (1e-6, 1e-5, 1e-3, 1e-4)[fld] * max(1.0, abs(states[t][p, c]))
            zs = []
            for sgn in (1.0, -1.0):
                st = states[t].copy()
                st[p, c] += sgn * h
                for _ in range(T - t):
                    st = oracle.step_fp64(ph, st)
                zs.append(oracle.mean_sq_pos(3, st))
            fd = (zs[0] - zs[1]) / (2 * h)
            noise = 1e-14 * abs(zs[0]) / h
            assert abs(fd - grad_t[p, c]) <= 2e-3 * scales[fld] + 1e-3 * abs(fd) + noise, (t, p, c, fd, grad_t[p, c])
            checked += 1
    assert checked == 64


@pytest.mark.parametrize("dim,material", [(2, "neohookean"), (3, "corotated")])
def test_kinetic_energy_adjoint_matches_oracle(q, oracle, dim, material):
    import torch
    sc, s0 = small(dim, material, N_side=16 if dim == 2 else 8, seed=20 + dim)
    T = 6
    g = q.Scene(sc, None, s0)
    ids = g.readback(state=False, ids=True)["ids"]
    d = torch.empty((s0.shape[0], s0.shape[1]), dtype=torch.float32, device="cuda")
    info = q.qmpm_adjoint(g.h, T, 3, q.MEASURE_KINETIC_ENERGY, 0, d.data_ptr())
    g.close()
    grad = np.empty((s0.shape[0], s0.shape[1]))
    grad[ids] = d.cpu().numpy()
    ph = oracle.make_phys(sc)
    z, adj, gg = oracle.rollout_adjoint(ph, s0, T, seed_fn="kinetic")
    assert abs(info["z"] - z) <= 1e-5 * abs(z)
    close_by_field(grad, adj[0], dim)
    assert np.allclose(info["g"], gg, rtol=2e-3)


def test_checkpoint_interval_does_not_change_the_gradient(q):
    sc, s0 = small(3, "corotated", N_side=8, seed=4)
    T = 16
    ref, info_ref = device_grad0(q, sc, s0, T, T)
    for k in (1, 3, 8):
        got, info = device_grad0(q, sc, s0, T, k)
        # only the order of FP32 atomic additions differs between the runs
        close_by_field(got, ref, 3, rel=1e-3)
        assert np.allclose(info["g"], info_ref["g"], rtol=1e-3)


@pytest.mark.parametrize("T", [16, 37])
def test_bisection_checkpointing_gives_the_same_gradient(q, T):
    # Sec. 6: checkpoints on the bisection tree instead of uniform segments; O(log T)
    # states held, the gradient unchanged (only FP32 atomic order differs)
    import math
    sc, s0 = small(3, "corotated", N_side=8, seed=4)
    ref, info_ref = device_grad0(q, sc, s0, T, T)
    got, info = device_grad0(q, sc, s0, T, q.CKPT_BISECTION)
    close_by_field(got, ref, 3, rel=1e-3)
    assert np.allclose(info["g"], info_ref["g"], rtol=1e-3)
    depth = int(math.floor(math.log2(T)))
    assert info["state_buffers"] == (depth + 1) + 2  # tree slots, the first-pass pair (one is scratch)
    assert T < info["forward_steps"] <= T + math.ceil(T / 2) * (depth + 1)
    assert info_ref["forward_steps"] == 2 * T - 1  # uniform, one segment: forward + recompute


def test_rollout_autograd_function(q):
    import torch
    sc, s0 = small(2, "neohookean", N_side=16, seed=2)
    T = 8
    x0 = torch.tensor(s0, dtype=torch.float64, requires_grad=True)
    sT = q.Rollout.apply(x0, sc, T, 4)
    loss = (sT[:, :2] ** 2).sum(dim=1).mean()
    loss.backward()
    grad, info = device_grad0(q, sc, s0, T, 4)
    close_by_field(x0.grad.numpy(), grad, 2, rel=1e-4)
    assert q.Rollout.last is not None and len(q.Rollout.last["g"]) == 4
    assert abs(loss.item() - info["z"]) <= 1e-5 * abs(info["z"])


def impact_block():
    # the 2D block driven into the floor: the impact couples every field into the final
    # kinetic energy, the evaluation function of the paper's MPM experiments (Sec. 8.1)
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.block2d_scene(n_strata=(64, 32))
    s0[:, 1] -= 0.4 - 3.6 / 128
    s0[:, 3] = -0.5
    return dict(sc, resort_every=8), s0


@pytest.mark.parametrize("eps", [0.01, 0.003])
def test_error_bound_scheme_holds_the_bound(q, oracle, eps):
    # Algorithm 1 end to end: FP32 adjoint -> g_h, ranges, z -> Eq. 10 -> a quantized
    # dithered rollout whose kinetic energy stays within 3 eps z of the FP64 run
    sc, s0 = impact_block()
    T = 300
    info = q.sensitivities(sc, s0, T, ckpt_every=25, measure=q.MEASURE_KINETIC_ENERGY)
    scheme, res = q.solve_scheme(info, eps, material="neohookean")
    assert res["pred_err"] <= (eps * info["z"]) ** 2
    assert max(res["bits"]) <= 24
    g = q.Scene(sc, scheme, s0, stats=True)
    g.step(T)
    st = g.readback(state=True, ids=False)
    ph = oracle.make_phys(sc)
    zq = oracle.kinetic_energy(ph, st["state"])
    f = oracle.Fp64Rollout(sc, s0)
    f.step(T)
    z64 = oracle.kinetic_energy(ph, f.s)
    assert abs(zq - z64) <= 3 * eps * z64, (zq, z64, res["bits"], res["frac"], st["stats"]["saturations"])
    # the scheme compresses the state below the 12 FP32 words of a 2D elastic particle
    assert g.n_words < 12


def test_full_size_adjoint_against_fp64_central_differences(q):
    """3D elastic, 1,024,000 particles, 128^3 grid, 256 steps, checkpoint every 32: the
    device adjoint's dz/ds_t at 64 injected (step, particle, component) errors drawn with
    seed 4 against FP64 central differences of the oracle (tests/golden/
    adjoint_cd_cubes_n128_T256.json, written by make_adjoint_cd_cubes.py with the oracle
    alone).  dz/ds_t comes from the adjoint over the remaining T - t steps started from the
    device's own FP32 state at step t.  Bar as in the small case: 2e-3 of the field's largest
    sensitivity at that step plus 1e-3 relative plus the FD rounding floor."""
    import json
    import os
    import sys
    import torch
    from paper_2207_04658_b300 import scenes
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "adjoint_cd_cubes_n128_T256.json")
    if not os.path.exists(path):
        pytest.skip("adjoint_cd_cubes_n128_T256.json has not been generated")
    with open(path) as f:
        ref = json.load(f)
    sys.path.insert(0, os.path.dirname(path))
    import make_adjoint_cd_cubes as mk
    import make_cubes3d_fp64 as mk3
    sc, s0 = mk.scene()
    assert ref["state_hash"] == mk3.state_hash(sc, s0) and ref["particles"] == s0.shape[0] == 1_024_000
    T = ref["steps"]
    assert T == 256 and len(ref["injections"]) == 64
    by_t = {}
    for r in ref["injections"]:
        by_t.setdefault(r["t"], []).append(r)
    g = q.Scene(sc, None, s0)  # the device's FP32 trajectory, fixed particle order
    done, worst = 0, 0.0
    t_now = 0
    for t in sorted(by_t):
        g.step(t - t_now)
        t_now = t
        st = g.state_by_id()
        gt = q.Scene(sc, None, st)
        ids = gt.readback(state=False, ids=True)["ids"]
        d = torch.empty(st.shape, dtype=torch.float32, device="cuda")
        info = q.qmpm_adjoint(gt.h, T - t, 32, q.MEASURE_MEAN_SQ_POS, 0, d.data_ptr())
        gt.close()
        grad = np.empty(st.shape)
        grad[ids] = d.cpu().numpy()
        assert np.all(np.isfinite(grad)) and all(np.isfinite(info["g"]))
        scales = [np.abs(grad[:, sl]).max() for sl in field_slices(3, st.shape[1])]
        for r in by_t[t]:
            p, c, fd = r["p"], r["c"], r["fd"]
            fld = 0 if c < 3 else 1 if c < 6 else 2 if c < 15 else 3
            noise = 1e-14 * abs(r["z_plus"]) / r["h"]
            tol = 2e-3 * scales[fld] + 1e-3 * abs(fd) + noise
            err = abs(fd - grad[p, c])
            worst = max(worst, err / tol)
            assert err <= tol, (t, p, c, fd, grad[p, c], scales[fld])
            done += 1
    g.close()
    assert done == 64, done


def test_quantized_forward_adjoint_and_iterative_relinearisation(q):
    # Sec. 4: the linearisation can be re-taken at the quantized solution; the paper finds
    # the iteration converges within six rounds and within about one bit of the first solve
    import torch
    from paper_2207_04658_b300 import autoquant
    sc, s0 = impact_block()
    T = 200
    scheme, hist = autoquant.iterate_scheme(sc, s0, T, 0.01, measure=q.MEASURE_KINETIC_ENERGY, ckpt_every=25)
    assert 2 <= len(hist) <= 6
    assert all(np.isfinite(h["g"]).all() and min(h["g"]) > 0 for h in hist)
    last, prev = hist[-1]["bits"], hist[-2]["bits"]
    converged = last == prev or (len(hist) >= 3 and last == hist[-3]["bits"])
    assert converged or len(hist) == 6
    assert max(abs(a - b) for a, b in zip(hist[0]["bits"], last)) <= 2
    # the quantized-forward adjoint needs a quantized handle
    g = q.Scene(sc, None, s0)
    with pytest.raises(q.QmpmError):
        q.qmpm_adjoint(g.h, 4, 2, q.MEASURE_KINETIC_ENERGY | q.ADJ_QUANTIZED_FORWARD)
    g.close()
