"""The quantized 2D smoke kernels (Sec. 8.1's advection-reflection solver) against the FP64
smoke oracle, through the C ABI.

  - FP32 stores: state after 1 and 8 steps within FP32 rounding of the FP64 oracle;
  - quantized stores (dithered and nearest): every stored code of every store of two steps
    equals the oracle's, except at near-ties of the rounding threshold, where the oracle
    takes the kernel's code (follow mode); the final velocities are then identical and the
    density within FP32 rounding;
  - antithetic noise runs: z+ and z- of each pair equal the oracle's noise runs, so the
    sensitivity estimate g_h equals the oracle's;
  - batch invariance: a scene's result does not depend on the other scenes of its batch,
    and graph replay equals plain launches bit for bit;
  - edge cases: zero Jacobi sweeps, an empty source, saturation counts."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sm():
    import torch
    from paper_2207_04658_b300 import qmpm, smoke
    assert torch.cuda.is_available()
    qmpm.lib()
    return smoke


def plume(n=64, jacobi=16, **kw):
    sc = dict(n=n, jacobi=jacobi, dt=0.01, buoyancy=1.0, v_in=1.0, src=(0.35, 0.05, 0.65, 0.17), seed=11)
    sc.update(kw)
    return sc


SCHEME = {"v": dict(bits=16, frac=12, offset=-(1 << 15)), "p": dict(bits=16, frac=18, offset=-(1 << 15))}


def oracle_run(oracle, sc, T, scheme=None, state=None):
    r = oracle.SmokeRollout(sc, scheme, *(state or ()))
    r.step(T)
    return r


def scale(a):
    return max(float(np.abs(a).max()), 1e-30)


@pytest.mark.parametrize("T", [1, 8])
def test_fp32_matches_fp64_oracle(sm, oracle, T):
    sc = plume()
    with sm.Smoke(sc) as g:
        g.step(T)
        st = g.readback(0)
        z = g.measure()[0]
    o = oracle_run(oracle, sc, T)
    for k, ref in (("u", o.u), ("v", o.v), ("d", o.d), ("q", o.q)):
        err = np.abs(st[k] - ref).max() / scale(ref)
        assert err < 2e-5 * T, (k, err)
    assert abs(z - o.measure()) / o.measure() < 1e-5 * T


def taus(oracle, sc, scheme, T, state=None, ulps=16):
    """Near-tie tolerances in quanta of each type: the kernel computes a stored value in FP32
    from values of its field's magnitude, so it differs from the FP64 value by a few units
    in the last place of that magnitude (the largest |value| of the type in an FP64 run)."""
    r = oracle.SmokeRollout(sc, None, *(state or ()))
    mv, mq = 0.0, 0.0
    for _ in range(T):
        r.step(1)
        mv = max(mv, np.abs(r.u).max(), np.abs(r.v).max())
        mq = max(mq, np.abs(r.q).max())
    ulp = 2.0 ** -23
    return (ulps * ulp * 2 * mv * 2.0 ** scheme["v"]["frac"], ulps * ulp * 2 * mq * 2.0 ** scheme["p"]["frac"])


def trace_run(sm, sc, scheme, T, state=None):
    import torch
    with sm.Smoke(sc, scheme, 1, seeds=[sc["seed"]]) as g:
        if state is not None:
            g.set_state(*state)
        tr = torch.zeros(g.trace_len(T), dtype=torch.int32, device="cuda")
        g.step(T, trace=tr)
        st = g.readback(0)
        lo, hi, sat = g.ranges()
    return tr.cpu().numpy().view(np.uint32), st, sat[0]


@pytest.mark.parametrize("dither", [True, False])
@pytest.mark.parametrize("n,jacobi", [(64, 16), (96, 64)])
def test_quantized_codes_match_oracle(sm, oracle, dither, n, jacobi):
    sc = plume(n=n, jacobi=jacobi, dither=dither)
    T = 2
    codes, st, sat = trace_run(sm, sc, SCHEME, T)
    assert codes.size == len(oracle.smoke_store_events(n, jacobi, T))
    o = oracle.SmokeRollout(sc, SCHEME)
    tv, tp = taus(oracle, sc, SCHEME, T)
    assert tv < 0.05 and tp < 0.05  # the tolerance is a small fraction of a quantum
    with oracle.smoke_follow(codes, tv, tp) as f:
        o.step(T)
    stores, adopted, violations, max_dist = f.report
    assert stores == codes.size and violations == 0, (f.report, f.first, locate(n, jacobi, f.first))
    assert adopted <= 1e-4 * stores, f.report
    assert o.saturations == int(sat.sum())
    # the kernel's codes are the oracle's run: velocities identical, density within rounding
    assert np.array_equal(st["u"].astype(np.float64), o.u)
    assert np.array_equal(st["v"].astype(np.float64), o.v)
    assert np.array_equal(st["q"].astype(np.float64), o.q)
    assert np.abs(st["d"] - o.d).max() < 1e-5


def locate(n, jacobi, first):
    """(step, stage, field, sample) of a store position, for failure messages."""
    if not first:
        return None
    V, Pq = 2 * n * (n + 1), n * n
    per = 5 * V + 2 * jacobi * Pq
    t, r = divmod(first["pos"], per)
    bounds = [("s1", V), ("jac1", jacobi * Pq), ("s2", V), ("s3", V), ("s4", V), ("jac2", jacobi * Pq), ("s5", V)]
    for name, size in bounds:
        if r < size:
            return (t + 1, name, r)
        r -= size
    return None


def test_quantized_from_a_generic_state(sm, oracle):
    """Nonzero velocities everywhere, set through the C ABI (rounded to the lattice)."""
    n = 64
    gen = np.random.default_rng(3)
    u0 = np.round(gen.normal(0, 0.3, (n, n + 1)) * 4096) / 4096
    v0 = np.round(gen.normal(0, 0.3, (n + 1, n)) * 4096) / 4096
    u0[:, 0] = u0[:, -1] = 0.0
    v0[0, :] = v0[-1, :] = 0.0
    d0 = gen.uniform(0, 1, (n, n)).astype(np.float32).astype(np.float64)
    sc = plume(n=n, jacobi=16)
    codes, st, sat = trace_run(sm, sc, SCHEME, 2, state=(u0, v0, d0))
    o = oracle.SmokeRollout(sc, SCHEME, u0, v0, d0)
    with oracle.smoke_follow(codes, *taus(oracle, sc, SCHEME, 2, (u0, v0, d0))) as f:
        o.step(2)
    assert f.report[2] == 0 and f.report[1] <= 1e-4 * f.report[0], (f.report, f.first)
    assert np.array_equal(st["u"].astype(np.float64), o.u)
    assert np.abs(st["d"] - o.d).max() < 1e-5


def test_noise_runs_match_oracle(sm, oracle):
    sc = plume(n=64, jacobi=8)
    T, pairs = 3, 8
    for h, sigma in ((0, (1e-2, 0.0)), (1, (0.0, 1e-4))):
        ns = np.repeat(np.arange(pairs, dtype=np.uint64) + np.uint64(5), 2)
        signs = np.tile(np.array([1.0, -1.0], np.float32), pairs)
        with sm.Smoke(sc, None, 2 * pairs) as g:
            g.set_noise(sigma, ns, signs)
            g.step(T)
            z = g.measure()
        zo = []
        for k in range(2 * pairs):
            with oracle.smoke_noise(sigma, int(ns[k]), float(signs[k])):
                zo.append(oracle_run(oracle, sc, T).measure())
        zo = np.array(zo)
        z0 = oracle_run(oracle, sc, T).measure()
        assert np.abs(z - zo).max() < 2e-6 * z0
        # the halved pair differences are the linear response to the injected noise; FP32
        # rounding of z (about 1e-6 of it) is far below their spread
        dz, dzo = (z[0::2] - z[1::2]) / 2, (zo[0::2] - zo[1::2]) / 2
        rms = np.sqrt(np.mean(dzo ** 2))
        assert rms > 1e-4 * z0, (h, rms, z0)
        assert np.abs(dz - dzo).max() < 0.02 * rms, (h, dz, dzo)
        g_gpu, g_or = np.mean(dz ** 2) / sigma[h] ** 2, np.mean(dzo ** 2) / sigma[h] ** 2
        assert abs(g_gpu / g_or - 1) < 0.05, (h, g_gpu, g_or)


def test_batch_invariance_and_graph_replay(sm):
    import torch
    sc = plume(n=64, jacobi=8)
    seeds = [11, 12, 13, 14, 15]
    with sm.Smoke(sc, SCHEME, len(seeds), seeds=seeds) as g:
        g.step(4)
        zb = g.measure()
        sb = g.readback(3)
    with sm.Smoke(sc, SCHEME, 1, seeds=[14]) as g:
        g.step(4)
        zs = g.measure()
        ss = g.readback(0)
    assert zb[3] == zs[0]
    for k in "uvdq":
        assert np.array_equal(sb[k], ss[k])
    # different seeds give different dither decisions
    assert len(set(zb.tolist())) == len(seeds)
    # plain launches (trace mode) equal the graph replay
    with sm.Smoke(sc, SCHEME, 1, seeds=[14]) as g:
        tr = torch.zeros(g.trace_len(4), dtype=torch.int32, device="cuda")
        g.step(4, trace=tr)
        st = g.readback(0)
        info = g.info()
    for k in "uvdq":
        assert np.array_equal(st[k], ss[k])
    assert info["steps"] == 4 and info["launches_per_step"] == 10 + 2 * 2


def test_edge_cases(sm, oracle):
    # zero sweeps: no projection, q stays zero
    sc = plume(n=32, jacobi=0)
    codes, st, sat = trace_run(sm, sc, SCHEME, 2)
    o = oracle.SmokeRollout(sc, SCHEME)
    with oracle.smoke_follow(codes, *taus(oracle, sc, SCHEME, 2)) as f:
        o.step(2)
    assert f.report[2] == 0
    assert np.array_equal(st["u"].astype(np.float64), o.u) and not st["q"].any()
    # an empty source and no buoyancy: rest stays at rest, bit for bit
    sc = plume(n=32, jacobi=4, src=(1.0, 1.0, -1.0, -1.0), v_in=0.0, buoyancy=0.0)
    with sm.Smoke(sc, SCHEME) as g:
        g.step(3)
        st = g.readback(0)
    assert not st["u"].any() and not st["v"].any() and not st["d"].any()
    # a pressure window too narrow saturates, and both sides count the same saturations
    narrow = {"v": SCHEME["v"], "p": dict(bits=8, frac=18, offset=-128)}
    sc = plume(n=32, jacobi=8)
    codes, st, sat = trace_run(sm, sc, narrow, 1)
    o = oracle.SmokeRollout(sc, narrow)
    with oracle.smoke_follow(codes, *taus(oracle, sc, narrow, 1)) as f:
        o.step(1)
    assert sat[1] > 0 and o.saturations == int(sat.sum()) and f.report[2] == 0


def test_invalid_arguments_fail_loudly(sm):
    from paper_2207_04658_b300.qmpm import QmpmError
    with pytest.raises(QmpmError):
        sm.Smoke(plume(n=48))          # not a multiple of 32
    with pytest.raises(QmpmError):
        sm.Smoke(plume(jacobi=600))
    with pytest.raises(QmpmError):
        sm.Smoke(plume(), {"v": dict(bits=30, frac=10, offset=0), "p": SCHEME["p"]})
    with sm.Smoke(plume(), SCHEME) as g:
        with pytest.raises(QmpmError):
            g.set_noise((1e-3, 0.0), [1], [1.0])  # quantized handle


def test_bias_aware_schemes_meet_the_error_bound(sm):
    """The error-bounded protocol of Sec. 8.1 on a 128^2 plume (50 steps): for eps = 1e-2
    and 1e-3 the bias-aware scheme keeps at least 17 of 20 dithered runs within 3 eps z of
    the FP32 run (the paper's band), and its observed spread is of the predicted size."""
    from paper_2207_04658_b300 import scenes
    sc = scenes.smoke_scene(n=128, steps=50)
    res = sm.error_bound_protocol(sc, sc["steps"], [1e-2, 1e-3], runs=20, variants=(True,))
    assert all(b > 0 for b in res["g"])
    for r in res["results"]:
        assert r["saturations"] == 0, r
        assert r["success_3eps"] >= 0.85, r
        assert 0.3 < r["z_std"] / r["pred_sigma_dither"] < 3.0, r
        # the scheme still compresses the quantized fields
        assert r["compression"] > 1.5, r


def test_largest_grid_fp32_matches_fp64(sm, oracle):
    """The largest grid the C ABI accepts (4096^2, 16.8 M cells), one step against the FP64
    oracle: the tiles, the packed-row padding and the index arithmetic at full size."""
    sc = plume(n=4096, jacobi=8)
    with sm.Smoke(sc) as g:
        g.step(1)
        st = g.readback(0)
    o = oracle_run(oracle, sc, 1)
    for k, ref in (("u", o.u), ("v", o.v), ("d", o.d), ("q", o.q)):
        err = np.abs(st[k] - ref).max() / scale(ref)
        assert err < 2e-5, (k, err)


@pytest.mark.parametrize("n", [160, 1024])
def test_quantized_codes_match_oracle_ragged_and_large(sm, oracle, n):
    """A grid whose width is not a multiple of the 128-cell tile (160: one full and one
    32-cell tile per row) and a 1024^2 grid, every store of one step against the oracle."""
    sc = plume(n=n, jacobi=8)
    codes, st, sat = trace_run(sm, sc, SCHEME, 1)
    o = oracle.SmokeRollout(sc, SCHEME)
    with oracle.smoke_follow(codes, *taus(oracle, sc, SCHEME, 1)) as f:
        o.step(1)
    assert f.report[0] == codes.size and f.report[2] == 0, (f.report, f.first)
    assert f.report[1] <= 1e-4 * f.report[0]
    assert np.array_equal(st["u"].astype(np.float64), o.u)
    assert np.array_equal(st["v"].astype(np.float64), o.v)
    assert np.abs(st["d"] - o.d).max() < 1e-5


def test_bench_configuration_against_oracle(sm, oracle):
    """The benchmark's configuration (the 256^2 plume, 64 sweeps, the bias-aware eps 1e-3
    scheme: v 13 bits, p 14 bits) in a batch of scenes: every store of scene 0's first two
    steps against the oracle, and another scene's state after two steps against the oracle
    with that scene's seed (the batch stores what single runs store)."""
    import torch
    from paper_2207_04658_b300 import scenes
    sc = scenes.smoke_scene()
    sch = {"v": dict(bits=13, frac=10, offset=-3616), "p": dict(bits=14, frac=18, offset=-4288)}
    T = 2
    seeds = [sc["seed"], 1234, 99]
    with sm.Smoke(sc, sch, len(seeds), seeds=seeds) as g:
        tr = torch.zeros(g.trace_len(T), dtype=torch.int32, device="cuda")
        g.step(T, trace=tr)
        st0, st2 = g.readback(0), g.readback(2)
        _, _, sat = g.ranges()
    codes = tr.cpu().numpy().view(np.uint32)
    o = oracle.SmokeRollout(sc, sch)
    with oracle.smoke_follow(codes, *taus(oracle, sc, sch, T)) as f:
        o.step(T)
    assert f.report[0] == codes.size and f.report[2] == 0, (f.report, f.first)
    assert f.report[1] <= 1e-4 * f.report[0]
    assert o.saturations == int(sat[0].sum()) == 0
    assert np.array_equal(st0["u"].astype(np.float64), o.u)
    assert np.array_equal(st0["v"].astype(np.float64), o.v)
    assert np.abs(st0["d"] - o.d).max() < 1e-5
    # scene 2 (no trace): same dither rule with its own seed; near-ties may flip a code, so
    # compare in quanta
    o2 = oracle.SmokeRollout(dict(sc, seed=99), sch)
    o2.step(T)
    dq = np.abs(st2["u"] - o2.u).max() / 2.0 ** -10
    assert dq <= 2.0 and np.abs(st2["d"] - o2.d).max() < 1e-3, dq


def test_batch_state_transfers(sm):
    """qmpm_smoke_get_states / set_states move every scene at once: the batch read equals
    the per-scene reads, writing it back stores the same codes (the values are on the
    lattice), and a scene stepped from the written state matches one that was never read."""
    import torch
    sc = plume(n=64, jacobi=8)
    S, n = 3, 64
    with sm.Smoke(sc, SCHEME, S, seeds=[5, 6, 7]) as g:
        g.step(3)
        hu = torch.zeros((S, n, n + 1), dtype=torch.float32).pin_memory()
        hv = torch.zeros((S, n + 1, n), dtype=torch.float32).pin_memory()
        hd = torch.zeros((S, n, n), dtype=torch.float32)  # pageable works too
        g.get_states(hu, hv, hd)
        for s in range(S):
            r = g.readback(s)
            assert np.array_equal(hu[s].numpy(), r["u"]) and np.array_equal(hv[s].numpy(), r["v"])
            assert np.array_equal(hd[s].numpy(), r["d"])
        z_before = g.measure()
        g.set_states(hu, hv, hd)
        assert np.array_equal(g.measure(), z_before)
        g.step(2)
        z_round_trip = g.measure()
    with sm.Smoke(sc, SCHEME, S, seeds=[5, 6, 7]) as g:
        g.step(5)
        assert np.array_equal(g.measure(), z_round_trip)
