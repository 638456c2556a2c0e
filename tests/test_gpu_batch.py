"""Multi-scene launches (qmpm_batch_*), the autotuner and the serving engine, through the
C ABI.

A scene stepped in a batch goes through the same stores, dither draws and re-sorts as the
same scene stepped alone; only the order of the floating-point atomic additions that flush
P2G tiles into the grid differs -- as it does between two runs of the scene alone.  Such a
rounding difference may flip a dither decision: one stored velocity then differs by one
quantum q_v, which moves the grid velocities around it by up to q_v and so the APIC C of
its neighbours by up to about 6 n q_v (C = D^-1 sum_i w_i v_i (x_i - x_p)^T), and through
F = (I + dt C) F and x += dt v the other fields.  The bar between a batch (or serving-mix)
result and an alone run A1, per field: four quanta plus that propagation over the T steps
(x: 4 dt q_v T, C: 12 n q_v, F: 12 n q_v dt T max|F|) plus twice the spread of a second
alone run A2 (for stiff scenes where such differences have grown); FP32 state: 1e-5 of the
field's natural scale plus twice the spread.  The measurement z and the RMS position must
agree to 1e-6 (plus twice the spread)."""
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


def mixed_scenes():
    """Scenes of four launch classes and uneven sizes (2D and 3D, elastic and fluid,
    quantized and FP32)."""
    from paper_2207_04658_b300 import scenes
    out = []
    sc, s0 = scenes.block2d_scene(n_strata=(64, 32), resort_every=8)
    out.append((sc, s0, scenes.block2d_scheme()))
    sc, s0 = scenes.block2d_scene(n_strata=(48, 48), seed=7, resort_every=8)
    s0[:, 3] = 0.5
    out.append((sc, s0, None))
    sc, s0 = scenes.cubes3d_scene(n_cubes=2, cube_cells=8, grid_log2=6, seed=5, steps=100)
    out.append((sc, s0, scenes.fixed_scheme_3d("corotated")))
    sc, s0 = scenes.dambreak3d_scene(column_cells=12, grid_log2=6, seed=6)
    out.append((sc, s0, scenes.fixed_scheme_3d("fluid", C=(16, -2048.0, 2048.0))))
    sc, s0 = scenes.cubes3d_scene(n_cubes=1, cube_cells=6, grid_log2=5, seed=8, steps=100)
    out.append((sc, s0, scenes.fixed_scheme_3d("corotated")))
    return out


def large_scene():
    """A member large enough for a launch of its own (314,432 particles, 1,229 chunks)."""
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.cubes3d_scene(n_cubes=1, cube_cells=34, grid_log2=7, seed=9, steps=100)
    return sc, s0, scenes.fixed_scheme_3d("corotated")


def quanta(scheme, dim, material, n_comp):
    from paper_2207_04658_b300 import scenes
    if scheme is None:
        return None
    widths = [dim, dim, dim * dim, n_comp - 2 * dim - dim * dim]
    names = ["x", "v", "C", "J" if material == "fluid" else "F"]
    return np.concatenate([np.full(w, 2.0 ** -scheme[n]["frac"]) for w, n in zip(widths, names)])


def field_scales(ref, sc):
    d = sc["dim"]
    n = 2 ** sc["grid_log2"]
    vmax = np.abs(ref[:, d:2 * d]).max() + 1e-3
    fj = np.abs(ref[:, 2 * d + d * d:]).max()
    widths = [d, d, d * d, ref.shape[1] - 2 * d - d * d]
    return np.concatenate([np.full(w, s) for w, s in zip(widths, (1.0, vmax, n * vmax, fj))])


def field_slices(sc, nc):
    d = sc["dim"]
    b = [0, d, 2 * d, 2 * d + d * d, nc]
    return [slice(b[h], b[h + 1]) for h in range(4)]


def assert_close(got, ref, scheme, sc, ref2=None, T=1):
    """got vs the alone run ref after T steps, with ref2 a second alone run."""
    from paper_2207_04658_b300 import scenes
    nc = scenes.n_comp(sc["dim"], sc["material"])
    qt = quanta(scheme, sc["dim"], sc["material"], nc)
    sl = field_slices(sc, nc)
    n = 2 ** sc["grid_log2"]
    if qt is not None:
        qv = qt[sl[1]][0]
        prop = [4 * sc["dt"] * qv * T, 0.0, 12 * n * qv, 12 * n * qv * sc["dt"] * T * np.abs(ref[:, sl[3]]).max()]
        tol = 4.0 * qt
        for h in range(4):
            tol[sl[h]] += prop[h]
    else:
        tol = 1e-5 * field_scales(ref, sc)
    spread = np.abs(ref2 - ref).max(axis=0) if ref2 is not None else np.zeros(nc)
    for h in range(4):
        tol[sl[h]] += 2.0 * spread[sl[h]].max()
    bad = np.abs(got - ref) > tol[None]
    assert not bad.any(), (int(bad.sum()), np.argwhere(bad)[:5].tolist())
    d = sc["dim"]
    rms = float(np.sqrt(((got[:, :d] - ref[:, :d]) ** 2).sum(1).mean()))
    rms_spread = float(np.sqrt(((ref2[:, :d] - ref[:, :d]) ** 2).sum(1).mean())) if ref2 is not None else 0.0
    assert rms <= 1e-6 + 2 * rms_spread, (rms, rms_spread)
    z = lambda s: float((s[:, :d] ** 2).sum(1).mean())
    zs = abs(z(ref2) - z(ref)) if ref2 is not None else 0.0
    assert abs(z(got) - z(ref)) <= 1e-6 * z(ref) + 2 * zs


def alone(q, spec, steps):
    """Two runs of the scene alone (its run-to-run spread)."""
    sc, s0, sch = spec
    out = []
    for _ in range(2):
        g = q.Scene(sc, sch, s0)
        g.step(steps)
        out.append(g.state_by_id())
        g.close()
    return out


@pytest.mark.parametrize("graphs", [False, True])
def test_batch_matches_scenes_stepped_alone(q, graphs):
    specs = mixed_scenes() + [large_scene()]
    T = 28
    refs = [alone(q, spec, T) for spec in specs]
    members = [q.Scene(sc, sch, s0) for sc, s0, sch in specs]
    b = q.Batch(resort_every=8, graphs=graphs)
    for m in members:
        b.add(m)
    b.step(8)   # a new membership runs direct launches
    b.step(20)  # then two graph replays of a half period (8 steps) and 4 direct steps
    info = b.info()
    assert info["n_members"] == len(specs) and info["steps"] == T
    assert info["n_classes"] == 4  # the two small 3D quantized corotated scenes share one launch
    assert info["n_solo"] == 1     # the large one has its own
    assert info["graph_launches"] == (2 if graphs else 0)
    for m, (sc, s0, sch), (r1, r2) in zip(members, specs, refs):
        assert_close(m.state_by_id(), r1, sch, sc, r2, T)
    b.close()
    for m in members:
        m.close()


def test_batch_membership_changes(q):
    # scenes join and leave between batch steps; each ends where it would have alone
    specs = mixed_scenes()
    plan = {0: (0, 36), 1: (8, 28), 2: (0, 16), 3: (16, 36), 4: (8, 36)}  # member: (join, leave)
    b = q.Batch(resort_every=8, graphs=True)
    members = {}
    for t in range(0, 36, 4):
        for i, (j, l) in plan.items():
            if j == t:
                sc, s0, sch = specs[i]
                members[i] = q.Scene(sc, sch, s0)
                b.add(members[i])
            if l == t and i in members:
                b.remove(members[i])
        b.step(4)
    for i, (j, l) in plan.items():
        sc, s0, sch = specs[i]
        r1, r2 = alone(q, specs[i], min(l, 36) - j)
        assert_close(members[i].state_by_id(), r1, sch, sc, r2, min(l, 36) - j)
    b.close()
    for m in members.values():
        m.close()


def test_member_stepped_alone_between_batch_steps(q):
    specs = mixed_scenes()[:3]
    members = [q.Scene(sc, sch, s0) for sc, s0, sch in specs]
    b = q.Batch(resort_every=8, graphs=True)
    for m in members:
        b.add(m)
    b.step(8)
    members[1].step(3)  # the batch notices and rebuilds its tables
    b.step(8)
    for k, (m, (sc, s0, sch)) in enumerate(zip(members, specs)):
        r1, r2 = alone(q, specs[k], 19 if k == 1 else 16)
        assert_close(m.state_by_id(), r1, sch, sc, r2, 19 if k == 1 else 16)
    b.close()


def test_autotune(q):
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.cubes3d_scene(n_cubes=2, cube_cells=16, grid_log2=7, seed=3)
    sch = scenes.fixed_scheme_3d("corotated")
    ss = q.make_scene_struct(sc, s0.shape[0])
    sk = q.make_scheme_struct(sch, 3, "corotated")
    r = q.qmpm_autotune(ss, sk, s0, trial_steps=16, use_cache=False)
    assert len(r["candidates"]) == 16 and not r["from_cache"]
    times = [t for _, _, t in r["candidates"]]
    assert all(t > 0 for t in times)
    assert r["best_ms_per_step"] == min(times)
    best = [c for c in r["candidates"] if c[2] == min(times)][0]
    assert (r["chunk"], r["resort_every"]) == best[:2]
    again = q.qmpm_autotune(ss, sk, s0, trial_steps=16, use_cache=True)
    assert again["from_cache"] and (again["chunk"], again["resort_every"]) == (r["chunk"], r["resort_every"])
    # a scene built with the tuned parameters steps and matches the oracle's ordering rules
    g = q.Scene(dict(sc, chunk=r["chunk"], resort_every=r["resort_every"]), sch, s0)
    g.step(r["resort_every"] * 2)
    assert np.isfinite(g.state_by_id()).all()
    g.close()


def run_engine(q, reqs, budget=8 * 2 ** 30, max_active=8, stagger=0):
    """Submit (scene, scheme, state, steps) requests, `stagger` engine iterations apart, run
    the engine in this thread until idle; returns (records by id, final states by id)."""
    e = q.Engine(budget_bytes=budget, resort_every=8, max_active=max_active)
    ids = []
    for k, (sc, s0, sch, steps) in enumerate(reqs):
        ids.append(e.submit(sc, sch, s0, steps, keep_state=True))
        for _ in range(stagger):
            e.run(1)
    recs = {}
    peak_bytes = 0
    import time
    t_end = time.time() + 300
    while time.time() < t_end:
        busy = e.run(1)
        peak_bytes = max(peak_bytes, e.stats()["bytes_in_use"])
        for r in e.poll():
            recs[r["id"]] = r
        if not busy:
            break
    for r in e.poll():
        recs[r["id"]] = r
    finals = {}
    from paper_2207_04658_b300 import scenes
    for rid, (sc, s0, sch, steps) in zip(ids, reqs):
        if recs[rid]["status"] == q.REQ_DONE:
            finals[rid] = e.result(rid, s0.shape[0], scenes.n_comp(sc["dim"], sc["material"]))
            e.release(rid)
    stats = e.stats()
    e.close()
    return ids, recs, finals, stats, peak_bytes


def test_engine_result_same_alone_and_in_the_mix(q):
    specs = mixed_scenes()
    target = specs[2]
    sc, s0, sch = target
    ids_a, recs_a, fin_a, _, _ = run_engine(q, [(sc, s0, sch, 48)])
    mix = [(s[0], s[1], s[2], n) for s, n in zip(specs, (40, 56, 48, 24, 64))]
    ids_b, recs_b, fin_b, stats, _ = run_engine(q, mix, stagger=1)
    assert all(recs_b[i]["status"] == q.REQ_DONE for i in ids_b)
    for i in ids_b:
        r = recs_b[i]
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
    r1, r2 = alone(q, target, 48)
    # alone in the engine, in the mix, and outside the engine: one spread
    assert_close(fin_a[ids_a[0]], r1, sch, sc, r2, 48)
    assert_close(fin_b[ids_b[2]], r1, sch, sc, r2, 48)
    za, zb = recs_a[ids_a[0]]["z"], recs_b[ids_b[2]]["z"]
    z1 = float((r1[:, :3] ** 2).sum(1).mean())
    z2 = float((r2[:, :3] ** 2).sum(1).mean())
    assert abs(za - zb) <= 1e-6 * abs(za) + 2 * abs(z1 - z2) + 1e-12
    assert stats["particle_steps"] == sum(s[1].shape[0] * n for s, n in zip(specs, (40, 56, 48, 24, 64)))
    assert stats["graph_launches"] > 0


def test_engine_admission_respects_the_budget(q):
    from paper_2207_04658_b300 import scenes
    specs = mixed_scenes()
    sizes = []
    for sc, s0, sch in specs:
        r, p = q.qmpm_footprint(q.make_scene_struct(sc, s0.shape[0]),
                                q.make_scheme_struct(sch, sc["dim"], sc["material"]))
        sizes.append(p)
    budget = 2 * max(sizes)  # at most a couple of scenes at a time
    reqs = [(sc, s0, sch, 16) for sc, s0, sch in specs] * 2
    # one request that can never fit
    big_sc, big_s0 = scenes.cubes3d_scene(n_cubes=1, cube_cells=8, grid_log2=9, seed=1)
    reqs.append((big_sc, big_s0, None, 8))
    big_peak = q.qmpm_footprint(q.make_scene_struct(big_sc, big_s0.shape[0]), q.make_scheme_struct(None))[1]
    assert big_peak > budget
    ids, recs, finals, stats, peak = run_engine(q, reqs, budget=budget)
    assert peak <= budget
    assert [recs[i]["status"] for i in ids[:-1]] == [q.REQ_DONE] * (len(reqs) - 1)
    assert recs[ids[-1]]["status"] == q.REQ_FAILED and recs[ids[-1]]["error"] == -2


def test_engine_background_thread(q):
    import time
    specs = mixed_scenes()
    e = q.Engine(budget_bytes=8 * 2 ** 30, resort_every=8, max_active=16)
    e.start()
    ids = []
    gen = np.random.default_rng(5)
    for k in range(12):
        sc, s0, sch = specs[k % len(specs)]
        ids.append(e.submit(sc, sch, s0, 24))
        time.sleep(float(gen.exponential(0.005)))
    e.stop(drain=True)
    recs = {r["id"]: r for r in e.poll()}
    assert sorted(recs) == sorted(ids)
    assert all(r["status"] == q.REQ_DONE and r["t_done"] >= r["t_submit"] for r in recs.values())
    assert all(np.isfinite(r["z"]) and r["z"] > 0 for r in recs.values())
    e.close()
