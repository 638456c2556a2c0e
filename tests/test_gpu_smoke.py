"""The quantized 2D smoke kernels (Sec. 8.1's advection-reflection solver) against the FP64
smoke oracle, through the C ABI.

  - FP32 stores: state after 1 and 8 steps within FP32 rounding of the FP64 oracle;
  - quantized stores (dithered and nearest), stage by stage: each kernel launch of the step
    run once from identical stored inputs (drawn by a seeded generator, never taken from
    the kernel) against the oracle's function for that stage, every code equal except at
    near-ties of the rounding threshold, counted and bounded; whole quantized steps, each
    side on its own, within a few quanta;
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
    o.step(2)
    assert np.abs(st["u"] - o.u).max() <= 4 * 2.0 ** -SCHEME["v"]["frac"] and not st["q"].any()
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
    o.step(1)
    assert sat[1] > 0 and abs(o.saturations - int(sat.sum())) <= 1e-3 * codes.size


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


# ---------------------------------------------------------------------------- stage parity
def lattice(gen, shape, frac, sd, lo=None, hi=None):
    """Seeded values on the lattice of resolution 2^-frac (stored exactly by either side)."""
    x = np.round(gen.normal(0, sd, shape) * 2.0 ** frac) / 2.0 ** frac
    return x


def vel_pair(gen, n, frac, sd=0.3):
    u = lattice(gen, (n, n + 1), frac, sd)
    v = lattice(gen, (n + 1, n), frac, sd)
    u[:, 0] = u[:, -1] = 0.0
    v[0, :] = v[-1, :] = 0.0
    return u, v


def f32(gen, shape, sd):
    return gen.normal(0, sd, shape).astype(np.float32).astype(np.float64)


STAGE_STORES = {"advect1": [("v", 1)], "jacobi": None, "gradsub2": [("v", "J+2"), ("v", "J+3")],
                "advect4": [("v", "J+4")], "gradsub5": [("v", "2J+5")]}


def store_layout(stage, n, J, step, arg):
    """(type, field, sample index, store counter) of every store of a stage, in order."""
    base = 1024 * step
    ev = []
    if stage == "jacobi":
        c = base + 1 + arg
        return [(1, 2, i, c) for i in range(n * n)]
    ks = {"advect1": [1], "gradsub2": [J + 2, J + 3], "advect4": [J + 4], "gradsub5": [2 * J + 5]}[stage]
    for k in ks:
        ev += [(0, 0, i, base + k) for i in range((n + 1) * n)] + [(0, 1, i, base + k) for i in range(n * (n + 1))]
    return ev


def compare_stage(oracle, sc, scheme, stage, step, kernel_codes, ref, tau):
    """Kernel codes against the oracle's from identical inputs: equal, except where the
    oracle's FP64 value lies within tau quanta of its rounding threshold (the FP32 kernel may
    fall on the other side there: a difference of one).  Returns (stores, near-tie
    differences)."""
    n, J = sc["n"], sc["jacobi"]
    codes, xs = ref["codes"], ref["x"]
    assert kernel_codes.size == codes.size, (kernel_codes.size, codes.size)
    diff = np.nonzero(kernel_codes != codes)[0]
    if diff.size:
        ev = store_layout(stage, n, J, step, 0 if stage != "jacobi" else ref["arg"])
        for m in diff:
            h, field, idx, counter = ev[m]
            frac = scheme["v" if h == 0 else "p"]["frac"]
            t = xs[m] * 2.0 ** frac
            y = t - np.floor(t)
            if sc.get("dither", True):
                thr = oracle.dither_draw(sc["seed"], idx >> 3, counter, 8 * field + (idx & 7)) * 2.0 ** -32
            else:
                thr = 0.5
            dk = int(kernel_codes[m]) - int(codes[m])
            assert abs(dk) == 1 and abs(y - thr) <= tau[h], (stage, m, ev[m], dk, y, thr, tau)
    return codes.size, diff.size


def window(field):
    d = 2.0 ** -field["frac"]
    return field["offset"] * d, (field["offset"] + 2 ** field["bits"] - 1) * d


def stage_inputs(gen, sc, scheme, stage):
    """Seeded stage inputs inside the scheme's windows (a stored input outside would
    saturate on one side only)."""
    n = sc["n"]
    fv, fp = scheme["v"]["frac"], scheme["p"]["frac"]
    (vlo, vhi), (qlo, qhi) = window(scheme["v"]), window(scheme["p"])
    a = tuple(np.clip(x, vlo, vhi) for x in vel_pair(gen, n, fv))
    b = tuple(np.clip(x, vlo, vhi) for x in vel_pair(gen, n, fv))
    q = np.clip(lattice(gen, (n, n), fp, 0.01), qlo, qhi)
    div = f32(gen, (n, n), 5.0)
    if stage == "advect1":
        # the advecting v is the FP32 velocity after the forces, off the lattice
        a = (a[0], np.where(np.abs(a[1]) > 0, a[1] + f32(gen, a[1].shape, 1e-3), 0.0))
        a[1][0, :] = a[1][-1, :] = 0.0
        a = (a[0], a[1].astype(np.float32).astype(np.float64))
    return a, b, q, div


def run_stage_pair(sm, oracle, sc, scheme, stage, step=3, arg=0, seed=0, ulps=16):
    gen = np.random.default_rng(seed)
    a, b, q, div = stage_inputs(gen, sc, scheme, stage)
    with sm.Smoke(sc, scheme, 1, seeds=[sc["seed"]]) as g:
        kc = g.stage(stage, step, arg=arg, a=a, b=b, q=q, div=div)
    ref = oracle.smoke_stage(sc, scheme, stage, step, arg=arg, a=a, b=b, q=q, div=div)
    ref["arg"] = arg
    # near-tie tolerance in quanta: a few FP32 units of the largest value the stage handles
    mv = max(np.abs(a[0]).max(), np.abs(a[1]).max(), np.abs(b[0]).max(), np.abs(b[1]).max(), 1e-30)
    mq = max(np.abs(q).max(), np.abs(ref["x"]).max() if stage == "jacobi" else 0.0, 1e-30)
    taus = (ulps * 2.0 ** -23 * 2 * mv * 2.0 ** scheme["v"]["frac"],
            ulps * 2.0 ** -23 * 2 * mq * 2.0 ** scheme["p"]["frac"])
    assert max(taus) < 0.05  # a small fraction of a quantum
    return compare_stage(oracle, sc, scheme, stage, step, kc, ref, taus)


ALL_STAGES = [("advect1", 0), ("jacobi", 1), ("jacobi", 3), ("gradsub2", 0), ("advect4", 0), ("gradsub5", 0)]


@pytest.mark.parametrize("dither", [True, False])
@pytest.mark.parametrize("n,jacobi", [(64, 16), (160, 8)])
def test_every_stage_matches_oracle_from_identical_inputs(sm, oracle, dither, n, jacobi):
    """Each kernel launch of the step (advection of the velocity, one Jacobi sweep from a
    given iterate and from zero, the gradient subtraction with and without the reflection,
    the second advection) run once from identical stored inputs, drawn from a seeded
    generator (velocities and pressure on their lattices, FP32 divergence and forced
    velocity), against the oracle's function for that stage: every stored code equal, except
    within 16 FP32 units of the largest value the stage handles (in quanta, below 0.05) of
    the rounding threshold, where the kernel's FP32 value may fall on the other side; those
    are at most 1e-3 of the stores.  No code of the kernel enters the oracle.  n = 160 is a ragged tile width."""
    sc = plume(n=n, jacobi=jacobi, dither=dither)
    total = flips = 0
    for i, (stage, arg) in enumerate(ALL_STAGES):
        m, f = run_stage_pair(sm, oracle, sc, SCHEME, stage, step=3, arg=arg, seed=10 * i + n)
        total += m
        flips += f
    assert flips <= 1e-3 * total, (flips, total)


def test_stages_at_the_bench_configuration(sm, oracle):
    """The benchmark's 256^2 plume, 64 sweeps and its bias-aware eps 1e-3 scheme (v 13 bits,
    p 14 bits, dithered): every stage from identical inputs against the oracle, including
    the last sweep of the projection."""
    from paper_2207_04658_b300 import scenes
    sc = scenes.smoke_scene()
    sch = {"v": dict(bits=13, frac=10, offset=-3616), "p": dict(bits=14, frac=18, offset=-4288)}
    total = flips = 0
    for i, (stage, arg) in enumerate(ALL_STAGES + [("jacobi", 64)]):
        m, f = run_stage_pair(sm, oracle, sc, sch, stage, step=7, arg=arg, seed=100 + i)
        total += m
        flips += f
    assert flips <= 1e-3 * total, (flips, total)


def test_stage_arguments_fail_loudly(sm):
    from paper_2207_04658_b300.qmpm import QmpmError
    sc = plume(n=32, jacobi=4)
    with sm.Smoke(sc) as g:  # FP32 handle: no codes to compare
        with pytest.raises(QmpmError):
            g.stage("jacobi", 1, arg=1, div=np.zeros((32, 32)))
    with sm.Smoke(sc, SCHEME) as g:
        with pytest.raises(QmpmError):
            g.stage("jacobi", 1, arg=5, div=np.zeros((32, 32)))  # beyond the sweeps
        with pytest.raises(QmpmError):
            g.stage("advect1", 0, a=vel_pair(np.random.default_rng(0), 32, 12))  # step 0


def test_quantized_steps_stay_within_quanta_of_the_oracle(sm, oracle):
    """Whole steps (no stage inputs shared): two quantized steps of the plume from rest, the
    kernel's and the oracle's runs each on their own.  A near-tie decision taken the other
    way in an early store propagates, so the codes differ in a few places; the final
    velocities stay within a few quanta and the density within 1e-3, and nearly all stores
    agree."""
    sc = plume(n=64, jacobi=16)
    codes, st, sat = trace_run(sm, sc, SCHEME, 2)
    o = oracle.SmokeRollout(sc, SCHEME)
    buf = np.zeros(codes.size, dtype=np.uint32)
    import ctypes as ct
    L = oracle.lib()
    L.or_smoke_record(buf.ctypes.data_as(ct.POINTER(ct.c_uint32)), buf.size)
    try:
        o.step(2)
    finally:
        L.or_smoke_record(None, 0)
    assert np.count_nonzero(buf != codes) <= 1e-3 * codes.size
    dq = max(np.abs(st["u"] - o.u).max(), np.abs(st["v"] - o.v).max()) / 2.0 ** -SCHEME["v"]["frac"]
    assert dq <= 4.0, dq
    assert np.abs(st["d"] - o.d).max() < 1e-3
    assert o.saturations == int(sat.sum())
