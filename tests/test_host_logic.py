"""Host-only logic of the library, on the CPU: the bisection reverse schedule (Sec. 6), the
device footprint used for admission, the serving workload generator and the scheme capping.
No GPU: only pure-host entry points are called."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def q():
    from paper_2207_04658_b300 import build, qmpm
    build.build()
    qmpm.lib()
    return qmpm


def simulate(ops, T):
    """Run a schedule on symbolic states (a slot holds the index t of the state in it) and
    check every op's preconditions: an advance starts from the state it claims, a reverse
    finds s_t and dz/ds_(t+1).  Returns (forward steps, slots used)."""
    slots = {0: 0}
    lam = T  # dz/ds_lam is known
    fwd = 0
    for kind, frm, to, t0, t1 in ops:
        assert slots.get(frm) == t0, (kind, frm, to, t0, t1, slots)
        if kind == 0:
            assert t1 > t0 and to != frm
            slots[to] = t1
            fwd += t1 - t0
        else:
            assert kind == 1 and t1 == t0 + 1 and lam == t1
            lam = t0
    assert lam == 0
    return fwd, max(slots) + 1


@pytest.mark.parametrize("T", [1, 2, 3, 4, 5, 7, 8, 31, 32, 33, 100, 256, 1000, 4097])
def test_bisection_schedule_reverses_every_step_in_log_memory(q, T):
    ops, n_slots = q.qmpm_bisection_schedule(T)
    fwd, used = simulate(ops, T)
    assert used == n_slots
    depth = int(math.floor(math.log2(T)))
    assert n_slots == depth + 1  # O(log T) states: one per tree level
    assert sum(1 for o in ops if o[0] == 1) == T
    # each level of the tree recomputes at most the states of its half intervals
    assert fwd <= math.ceil(T / 2) * (depth + 1) + T


def test_bisection_matches_the_paper_illustration(q):
    # Fig. 7's tree over s_0..s_4 reversed: checkpoints halve the distance to the state
    # being recovered; s_3 comes from s_2, a checkpoint made halfway from s_0 to s_4
    ops, slots = q.qmpm_bisection_schedule(4)
    assert ops[0] == (0, 0, 1, 0, 2)  # s_2 from s_0
    assert ops[1] == (0, 1, 2, 2, 3)  # s_3 from s_2
    assert ops[2] == (1, 2, 2, 3, 4)  # reverse step 3
    assert ops[3] == (1, 1, 1, 2, 3)  # reverse step 2 from the s_2 checkpoint
    assert slots == 3


def test_footprint_counts_the_buffers(q):
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.cubes3d_scene(n_cubes=2, cube_cells=16, grid_log2=7)
    N = s0.shape[0]
    ss = q.make_scene_struct(sc, N)
    r32, p32 = q.qmpm_footprint(ss, q.make_scheme_struct(None))
    rq, pq = q.qmpm_footprint(ss, q.make_scheme_struct(scenes.fixed_scheme_3d("corotated"), 3, "corotated"))
    ld = (N + 31) // 32 * 32
    assert r32 - rq == 2 * 4 * ld * (24 - 13)  # word planes: 24 FP32 words vs 13 packed
    assert p32 - r32 == 8 * N * 24 and pq - rq == 8 * N * 24  # the FP64 initial state
    nb = 128 // 4 + 2
    assert r32 > 2 * nb ** 3 * 64 * 16  # two grid buffers


def test_serving_requests_follow_the_workload_definition():
    from paper_2207_04658_b300 import scenes
    reqs = scenes.serving_requests(rate=20.0, duration=50.0, seed=5)
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] <= 50.0
    assert abs(len(reqs) / 50.0 - 20.0) < 3.0  # Poisson count: 1000 +- 3 sigma
    n = np.array([r["n"] for r in reqs])
    assert n.min() >= 1e4 * 0.99 and n.max() <= 4e6 * 1.01
    # log-uniform: the median of log N sits mid-range
    assert abs(np.median(np.log(n)) - 0.5 * (math.log(1e4) + math.log(4e6))) < 0.4
    for r in reqs:
        assert r["grid_log2"] in scenes.SERVING_GRIDS[r["dim"]] and r["eps"] in (0.1, 0.01)
    classes = {(r["dim"], r["material"]) for r in reqs}
    assert classes == set(scenes.SERVING_CLASSES)


def test_serving_scene_fits_the_grid():
    from paper_2207_04658_b300 import scenes
    for dim, material in scenes.SERVING_CLASSES:
        for g in scenes.SERVING_GRIDS[dim]:
            sc, s0 = scenes.serving_scene(dim, material, 30000, g, 3)
            dx = 1.0 / (1 << g)
            x = s0[:, :dim]
            assert x.min() >= 3 * dx and x.max() <= 1 - 4 * dx
            assert sc["dt"] <= 0.3 * dx / (math.sqrt(400.0) if material == "fluid" else 1.0) + 1e-12


def test_scheme_cap_keeps_the_window(q):
    info = {"P": [300.0, 300.0, 900.0, 900.0], "g": [1e12, 1.0, 1e-6, 1.0],
            "lo": [0.0, -1.0, -10.0, 0.5], "hi": [1.0, 1.0, 10.0, 1.5], "z": 1.0}
    scheme, res = q.solve_scheme(info, 1e-4, material="corotated")
    assert res["capped"] == ["x"] and scheme["x"]["bits"] == 24
    d = 2.0 ** -scheme["x"]["frac"]
    lo = scheme["x"]["offset"] * d
    hi = (scheme["x"]["offset"] + 2 ** 24 - 1) * d
    assert lo <= -0.5 and hi >= 1.5  # the kappa = 2 window of [0, 1]


def test_margin_windows_match_the_solve(q):
    """The second-order iteration re-derives a margin type's window after every change of
    resolution; at the solve's own resolutions it gives the solve's window option."""
    from paper_2207_04658_b300 import autoquant
    info = {"P": [300.0, 300.0, 900.0, 900.0], "g": [1e6, 1e2, 1e-4, 1e3],
            "lo": [0.1, -11.7, -3044.5, -2.06], "hi": [0.9, 14.1, 3871.5, 2.07], "z": 1.0}
    names = ["x", "v", "C", "F"]
    margins = {2: (1, 6.0 * 256)}
    for eps in (1e-2, 1e-3, 1e-4):
        plain, _ = q.solve_scheme(info, eps, material="corotated")
        wide, _ = q.solve_scheme(info, eps, material="corotated", margins=margins)
        assert wide["C"]["frac"] == plain["C"]["frac"]
        got = autoquant._margin_windows(plain, "corotated", info, margins)
        assert got["C"] == wide["C"] and got["x"] == plain["x"]
        # grow_only keeps a wider current window, and the new one holds the old
        big = dict(wide, C=dict(wide["C"], bits=wide["C"]["bits"] + 1,
                                offset=wide["C"]["offset"] - (1 << (wide["C"]["bits"] - 1))))
        kept = autoquant._margin_windows(big, "corotated", info, margins, grow_only=True)
        assert kept["C"] == big["C"]
        finer = q.scheme_shift(wide, "corotated", "C", 1)["C"]
        grown = autoquant._margin_windows(dict(wide, C=finer), "corotated", info, margins, grow_only=True)
        d = 2.0 ** -finer["frac"]
        assert grown["C"]["offset"] * d <= finer["offset"] * d
        assert (grown["C"]["offset"] + 2 ** grown["C"]["bits"] - 1) * d >= (finer["offset"] + 2 ** finer["bits"] - 1) * d


def test_fill_word_slack_keeps_words_and_resolution(q):
    from paper_2207_04658_b300 import autoquant
    sch = {"x": {"bits": 16, "frac": 15, "offset": -9688, "container": 64},
           "v": {"bits": 4, "frac": -2, "offset": -7, "container": 0},
           "C": {"bits": 4, "frac": -11, "offset": -7, "container": 0},
           "F": {"bits": 11, "frac": 7, "offset": -536, "container": 0}}
    words = q.make_scheme_struct(sch, 3, "corotated").n_words
    got = autoquant.fill_word_slack(sch, 3, "corotated")
    assert q.make_scheme_struct(got, 3, "corotated").n_words == words
    assert got["x"] == sch["x"]
    for n in "vCF":
        a, b = sch[n], got[n]
        assert a["frac"] == b["frac"] and b["bits"] >= a["bits"]
        assert b["offset"] <= a["offset"] and b["offset"] + 2 ** b["bits"] >= a["offset"] + 2 ** a["bits"]
        # no type can take one more window bit without another word
        wider = q.scheme_widen(got, "corotated", n)
        assert q.make_scheme_struct(wider, 3, "corotated").n_words > words
    # 3 v components and 9 of C take the 13 free bits of the last word: one bit each
    assert (got["v"]["bits"], got["C"]["bits"], got["F"]["bits"]) == (5, 5, 11)


def test_acceptance_loop_refines_until_the_bound_holds(monkeypatch):
    # the acceptance check of the second-order scheme against a fake scene: the quantized
    # run's position error scales with the velocity resolution, and C saturates while its
    # window is narrower than 6 bits; the loop adds velocity fraction bits (the type with
    # the largest predicted share) and widens C until both hold
    import numpy as np
    from paper_2207_04658_b300 import autoquant

    class FakeScene:
        def __init__(self, scene, scheme, state0, stats=False):
            self.scheme, self.s0, self.seed = scheme, np.asarray(state0, float), scene.get("seed")

        def step(self, n=1):
            pass

        def state_by_id(self):
            if self.scheme is None:
                return self.s0.copy()
            err = 2.0 ** -self.scheme["v"]["frac"]
            return self.s0 + err

        def readback(self, state=False, ids=False):
            sat = [0, 0, 5 if self.scheme["C"]["bits"] < 6 else 0, 0]
            return {"stats": {"saturations": sat}}

        def close(self):
            pass

    monkeypatch.setattr(autoquant.qmpm, "Scene", FakeScene)
    names = ["x", "v", "C", "F"]
    s0 = np.zeros((10, 24))
    f = lambda bits, frac, off: {"bits": bits, "frac": frac, "offset": off, "container": 0}
    scheme = {"x": f(16, 15, 0), "v": f(4, 2, -8), "C": f(4, -8, -8), "F": f(11, 7, -536)}
    last = {"beta": [0.0] * 4, "g": [0.0, 1.0, 0.0, 0.0]}
    out, hist = autoquant._accept({"dim": 3, "material": "corotated"}, s0, 10, 0.5, 1.0, scheme, names, last, {}, None,
                                  (None, 7), 6, None)
    # error: sqrt(30) 2^-frac_v relative to z = 1: 1.37 at frac 2, 0.68 at 3, 0.34 at 4
    assert [round(h["rel_err"], 2) for h in hist] == [1.37, 0.68, 0.34]
    assert hist[0]["saturations"] == [0, 0, 10, 0] and hist[-1]["saturations"] == [0, 0, 0, 0]
    assert out["v"]["frac"] == 4 and out["v"]["bits"] == 6 and out["v"]["offset"] == -32
    assert out["C"]["frac"] == -8 and out["C"]["bits"] == 6 and out["C"]["offset"] == -8 - 8 - 16
    assert out["x"] == scheme["x"] and out["F"] == scheme["F"]
    # a bound that is already met returns the scheme after one check
    out2, hist2 = autoquant._accept({"dim": 3, "material": "corotated"}, s0, 10, 5.0, 1.0, dict(scheme, C=f(6, -8, -8)), names, last,
                                    {}, None, (None,), 6, None)
    assert len(hist2) == 1 and out2["v"] == scheme["v"]


def test_second_order_iteration_damps_floors_and_stops(monkeypatch, q):
    # the second-order refinement against fake noise moments (no device): per field h,
    # shift = (beta_h sigma_h^2)^2 and spread = g_h sigma_h^2, except that the velocity's
    # runs blow up (non-finite moments) while its resolution is coarser than 2^-7.  Checks:
    # every round moves a field by at most max_step bits; after the blow-up the velocity is
    # held at or above its floor; the result meets the refined bound of the coefficients
    import numpy as np
    from paper_2207_04658_b300 import autoquant

    class FakeScene:
        def __init__(self, scene, scheme, state0, stats=False):
            self.h = 1

        def close(self):
            pass

    N = 1000
    beta = [2e3, 5.0, 1e-9, 50.0]
    g = [4e3, 20.0, 1e-10, 3e2]

    def fake_moments(h, T, measure, sigma, seed0=1, n_pairs=16):
        k = [i for i, s in enumerate(sigma) if s > 0][0]
        s2 = sigma[k] ** 2 / 6.0
        if k == 1 and sigma[k] > 2.0 ** -7:
            return {"z0": 1.0 / N, "shift": float("nan"), "spread": float("nan")}
        return {"z0": 1.0 / N, "shift": (beta[k] * s2) ** 2, "spread": g[k] * s2}

    monkeypatch.setattr(autoquant.qmpm, "Scene", FakeScene)
    monkeypatch.setattr(autoquant.qmpm, "qmpm_noise_moments", fake_moments)
    info = {"P": [3.0 * N, 3.0 * N, 9.0 * N, 9.0 * N], "g": [1e3, 10.0, 1e-10, 1e2],
            "lo": [0.1, -2.0, -50.0, -1.5], "hi": [0.9, 2.0, 50.0, 1.5], "z": 1.0}
    scene = {"dim": 3, "material": "corotated"}
    eps = 0.05
    scheme, rep = autoquant.second_order_scheme(scene, np.zeros((N, 24)), 10, eps, info, iters=8, max_step=2,
                                                accept_seeds=())
    names = ["x", "v", "C", "F"]
    rounds = rep["rounds"]
    assert 1 <= len(rounds) <= 8
    for r in rounds:
        for n in names:
            assert abs(r["next"][n]["frac"] - r["scheme"][n]["frac"]) <= 2
    # the velocity blew up in the first round (Algorithm 1 left it at 2^-6) and is floored
    # one bit finer for the rest of the iteration
    assert rounds[0]["scheme"]["v"]["frac"] == 6 and rounds[0]["floor"]["v"] == 7
    assert scheme["v"]["frac"] >= rounds[-1]["floor"]["v"]
    # the result meets the second-order bound of the true coefficients (z^2 = N z0 = 1)
    s2 = [2.0 ** (-2 * scheme[n]["frac"]) / 6.0 for n in names]
    bias = sum(b * s for b, s in zip(beta, s2))
    var = sum(gg * s for gg, s in zip(g, s2))
    assert bias ** 2 + var <= eps ** 2 * 1.0001


def test_scheme_edits_through_the_abi(q):
    # the edits of one type of a scheme (qmpm_scheme_shift / widen / window / fill_words):
    # exact integer results, the other types kept, and the refusals
    f = lambda b, fr, o, c=0: {"bits": b, "frac": fr, "offset": o, "container": c}
    sch = {"x": f(16, 15, -9688, 64), "v": f(4, -2, -7), "C": f(4, -11, -7), "F": f(11, 7, -536)}
    s2 = q.scheme_shift(sch, "corotated", "v", 2)
    assert s2["v"] == f(6, 0, -28) and {k: s2[k] for k in "xCF"} == {k: sch[k] for k in "xCF"}
    assert q.scheme_shift(sch, "corotated", "v", -1)["v"] == f(3, -3, -4)  # floor(-7 / 2)
    assert q.scheme_widen(sch, "corotated", "C")["C"] == f(5, -11, -15)
    # the window of the solve for [-2, 2] (kappa 2: [-4, 4]) at resolution 2^-frac = 4
    assert q.scheme_window(sch, "corotated", "v", -2.0, 2.0)["v"] == f(2, -2, -1)
    # a margin of 3 resolutions of v (Delta_v = 4) on each side: [-16, 16]
    assert q.scheme_window(sch, "corotated", "v", -2.0, 2.0, 2.0, "v", 3.0)["v"] == f(4, -2, -4)
    filled, n = q.scheme_fill_words(sch, 3, "corotated", ("v", "C", "F"))
    assert n == 2 and filled["x"] == sch["x"]
    assert q.scheme_fill_words(sch, 3, "corotated", ())[1] == 0
    with pytest.raises(q.QmpmError) as ei:
        q.scheme_shift(sch, "corotated", "F", 14)  # 25 bits
    assert ei.value.code == -3
    with pytest.raises(q.QmpmError) as ei:
        q.scheme_window(sch, "corotated", "v", 2.0, -2.0)
    assert ei.value.code == -1
