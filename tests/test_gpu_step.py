"""Device MLS-MPM step vs the oracle, through the C ABI.

Bars (floating point, FP32 device vs FP64 oracle):
  - initial encode + tile sort: bit-exact words and slot order;
  - one quantized step from the same packed state: every packed component within
    2 quantization steps (atomic ordering and FP32 rounding can move a value across a
    rounding or dither threshold);
  - FP32 state, one step: |gpu - oracle| <= 1e-5 (|oracle| + scale of the field);
  - rollouts: the position measurement z within the error bound of the oracle's."""

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


def small_scenes():
    from paper_2207_04658_b300 import scenes
    out = []
    sc, s0 = scenes.block2d_scene(n_strata=(64, 32))
    out.append(("block2d", sc, s0, scenes.block2d_scheme()))
    sc, s0 = scenes.cubes3d_scene(n_cubes=2, cube_cells=10, ppc_axis=2, grid_log2=6, seed=5)
    out.append(("cubes3d", sc, s0, scenes.fixed_scheme_3d("corotated")))
    sc, s0 = scenes.cubes3d_scene(n_cubes=2, cube_cells=8, ppc_axis=2, grid_log2=5, seed=6,
                                  material="neohookean", dt=1e-4)
    out.append(("nh3d", sc, s0, scenes.fixed_scheme_3d("neohookean", x_container=0)))
    sc, s0 = scenes.dambreak3d_scene(column_cells=12, ppc_axis=2, grid_log2=6, dt=5e-5)
    out.append(("dam3d", sc, s0, scenes.fixed_scheme_3d("fluid", C=(16, -2048.0, 2048.0))))
    return out


SCENES = small_scenes()
IDS = [s[0] for s in SCENES]


def quanta(oracle, scene, scheme):
    cd = oracle.make_codec(scene, scheme)
    return np.array([2.0 ** -cd.frac[c] for c in range(cd.n_comp)])


@pytest.mark.parametrize("case", range(len(SCENES)), ids=IDS)
def test_init_encode_and_sort_bit_exact(q, oracle, case):
    name, sc, s0, sch = SCENES[case]
    g = q.Scene(sc, sch, s0)
    r = g.readback(state=False, words=True, ids=True)
    o = oracle.QuantRollout(sc, sch, s0)
    assert np.array_equal(r["ids"], o.ids)
    assert np.array_equal(r["words"].T, o.words)
    g.close()


@pytest.mark.parametrize("spec", [False, True], ids=["library", "specialized"])
@pytest.mark.parametrize("case", range(len(SCENES)), ids=IDS)
def test_one_quantized_step_within_two_quanta(q, oracle, case, spec):
    name, sc, s0, sch = SCENES[case]
    g = q.Scene(sc, sch, s0, stats=True, specialize=spec)
    assert q.qmpm_step_kernel_info(g.h)["specialized"] == spec
    o = oracle.QuantRollout(sc, sch, s0)
    g.step(1)
    o.step(1)
    r = g.readback(state=True, ids=True)
    assert np.array_equal(r["ids"], o.ids)
    d = np.abs(r["state"] - o.state()) / quanta(oracle, sc, sch)[None]
    assert d.max() <= 2.0 + 1e-9, f"max {d.max()} quanta at {np.unravel_index(d.argmax(), d.shape)}"
    # most components agree exactly
    assert (d == 0).mean() > 0.95
    assert sum(r["stats"]["saturations"]) == 0
    g.close()


@pytest.mark.parametrize("dither", [True, False], ids=["dithered", "nearest"])
@pytest.mark.parametrize("case", range(len(SCENES)), ids=IDS)
def test_specialized_step_matches_the_library_kernel(q, oracle, case, dither):
    # the kernel compiled for the scheme does the library kernel's arithmetic.  The grid a
    # step starts from is summed by FP32 atomics from the overlapping tiles, in an order
    # that varies from run to run, and the two compilations may contract a multiply-add
    # differently; either moves a value by an FP32 rounding, so a code can land one quantum
    # apart where the value sits at a rounding threshold; nearly all are equal
    name, sc, s0, sch = SCENES[case]
    sc = dict(sc, dither=dither)
    a = q.Scene(sc, sch, s0)
    b = q.Scene(sc, sch, s0, specialize=True)
    info = q.qmpm_step_kernel_info(b.h)
    assert info["specialized"] and not q.qmpm_step_kernel_info(a.h)["specialized"]
    assert info["compile_seconds"] >= 0.0
    a.step(1)
    b.step(1)
    ra = a.readback(state=True, words=True, ids=True)
    rb = b.readback(state=True, words=True, ids=True)
    assert np.array_equal(ra["ids"], rb["ids"])
    d = np.abs(ra["state"] - rb["state"]) / quanta(oracle, sc, sch)[None]
    assert d.max() <= 1.0 + 1e-9 and (d > 0).mean() <= 1e-2, (d.max(), (d > 0).mean())
    # FP32 state: the kernel compiled with its word count as a constant gives the library
    # kernel's state but for FP32 roundings of the grid sums
    c = q.Scene(sc, None, s0, specialize=True)
    e = q.Scene(sc, None, s0)
    assert q.qmpm_step_kernel_info(c.h)["specialized"] and not q.qmpm_step_kernel_info(e.h)["specialized"]
    c.step(1)
    e.step(1)
    sc_, se = c.readback(state=True, ids=True), e.readback(state=True, ids=True)
    assert np.array_equal(sc_["ids"], se["ids"])
    # scale: each field's natural magnitude (x: 1; v: its largest speed; C, a velocity
    # gradient: n times that; F or J: its largest entry), so that the near-zero C and
    # off-diagonal F of a nearly rigid body are held to the rounding of the fields
    # they come from
    d = sc["dim"]
    st = se["state"]
    vmax = np.abs(st[:, d:2 * d]).max() + 1e-3
    widths = [d, d, d * d, st.shape[1] - 2 * d - d * d]
    field = [1.0, vmax, (1 << sc["grid_log2"]) * vmax, np.abs(st[:, 2 * d + d * d:]).max()]
    scale = np.concatenate([np.full(w, f) for w, f in zip(widths, field)])[None]
    assert (np.abs(sc_["state"] - se["state"]) <= 1e-5 * (np.abs(se["state"]) + scale)).all()
    for g in (a, b, c, e):
        g.close()


@pytest.mark.parametrize("case", range(len(SCENES)), ids=IDS)
def test_fp32_step_matches_fp64(q, oracle, case):
    name, sc, s0, sch = SCENES[case]
    sc = dict(sc, resort_every=0)
    g = q.Scene(sc, None, s0)
    o = oracle.Fp64Rollout(sc, s0)
    for _ in range(2):
        g.step(1)
        o.step(1)
    r = g.readback(state=True, ids=True)
    ref = np.empty_like(o.s)
    ref[o.ids] = o.s
    got = np.empty_like(r["state"])
    got[r["ids"]] = r["state"]
    dim = sc["dim"]
    nc = got.shape[1]
    n = 1 << sc["grid_log2"]
    vmax = np.abs(ref[:, dim:2 * dim]).max()
    # field scales: the domain for x, the largest speed for v, the velocity-gradient unit
    # |v| / dx (times D^-1 dx^2 = 4) for C, and 1 for F or J
    bounds = [0, dim, 2 * dim, 2 * dim + dim * dim, nc]
    scales = [1.0, vmax + 1e-30, max(np.abs(ref[:, 2 * dim:2 * dim + dim * dim]).max(), 4 * vmax * n), 1.0]
    # stiffness floor: the stress is K (J - 1) J or mu (F F^T - I) + ..., so an FP32
    # rounding of J or F near 1 (2^-24) is amplified into a pressure error of about
    # stiffness * 2^-24, which one step turns into a velocity error of dt * n * that
    # (impulse over one cell) and a C error of 4 n times the velocity error
    mu = sc.get("E", 0.0) / (2 * (1 + sc.get("nu", 0.0)))
    lam = sc.get("E", 0.0) * sc.get("nu", 0.0) / ((1 + sc.get("nu", 0.0)) * (1 - 2 * sc.get("nu", 0.0)))
    stiff = sc.get("bulk", 0.0) if sc["material"] == "fluid" else 2 * mu + abs(lam)
    dv = 4 * sc["dt"] * n * stiff * 2.0 ** -24
    floors = [0.0, dv, 4 * n * dv, 0.0]
    for (a, b), scale, floor in zip(zip(bounds[:-1], bounds[1:]), scales, floors):
        err = np.abs(got[:, a:b] - ref[:, a:b])
        tol = 1e-5 * (np.abs(ref[:, a:b]) + scale) + floor
        assert np.all(err <= tol), (name, a, b, err.max(), scale, floor)
    g.close()


@pytest.mark.parametrize("spec", [False, True], ids=["library", "specialized"])
@pytest.mark.parametrize("case", [0, 1, 3], ids=[IDS[0], IDS[1], IDS[3]])
def test_quantized_rollout_tracks_oracle(q, oracle, case, spec):
    name, sc, s0, sch = SCENES[case]
    steps = 40
    g = q.Scene(sc, sch, s0, stats=True, specialize=spec)
    o = oracle.QuantRollout(sc, sch, s0)
    g.step(steps)
    o.step(steps)
    r = g.readback(state=True, ids=True)
    got = np.empty_like(r["state"])
    got[r["ids"]] = r["state"]
    ref = np.empty_like(got)
    ref[o.ids] = o.state()
    dim = sc["dim"]
    zg, zo = oracle.mean_sq_pos(dim, got), oracle.mean_sq_pos(dim, ref)
    assert abs(zg - zo) <= 1e-4 * abs(zo)
    assert abs(g.measure() - zg) <= 1e-12 * abs(zg)
    # positions stay within a few position quanta of the oracle's
    dq = np.abs(got[:, :dim] - ref[:, :dim]) / quanta(oracle, sc, sch)[None, :dim]
    assert np.percentile(dq, 99) <= 8
    g.close()


def test_drift_out_of_tile_slow_path(q, oracle):
    # no re-sort after initialisation: particles leave their tiles and take the slow
    # path; the result still matches the oracle's identical ordering
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.cubes3d_scene(n_cubes=1, cube_cells=8, ppc_axis=2, grid_log2=5, seed=8,
                                  material="corotated", dt=1e-4)
    s0[:, 3:6] = np.array([30.0, -20.0, 25.0])  # fast uniform motion: ~3 cells in 30 steps
    sc = dict(sc, resort_every=0)
    sch = scenes.fixed_scheme_3d("corotated", v=(16, -64.0, 64.0))
    g = q.Scene(sc, sch, s0, stats=True)
    o = oracle.QuantRollout(sc, sch, s0)
    for _ in range(30):
        g.step(1)
        o.step(1)
    r = g.readback(state=True, ids=True)
    assert r["stats"]["out_of_tile"] > 0
    assert np.array_equal(r["ids"], o.ids)
    d = np.abs(r["state"] - o.state()) / quanta(oracle, sc, sch)[None]
    assert np.percentile(d, 99.9) <= 8


def test_walls_stop_particles(q, oracle):
    # a block driven into the floor: sticky wall nodes carry zero velocity.  After 100
    # quantized oracle steps the block's bottom row is in contact (its stencils reach the
    # wall band); one step from that state matches the oracle within two quanta.  After 100
    # more steps the bottom row has been stopped and the block as a whole decelerated,
    # while free fall would have sped it up to -0.5 - 9.8 * 0.02 = -0.696
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.block2d_scene(n_strata=(32, 16))
    s0[:, 1] -= 0.4 - 3.6 / 128  # the block's bottom row sits 0.6 cells above the wall band
    s0[:, 3] = -0.5
    sch = scenes.block2d_scheme()
    sch["C"] = dict(bits=16, frac=6, offset=-512 * 2 ** 6, container=0)  # [-512, 512]
    sch["F"] = dict(bits=16, frac=14, offset=-2 * 2 ** 14, container=0)  # [-2, 2]: signed shear
    o = oracle.QuantRollout(sc, sch, s0)
    o.step(100)
    s100 = o.state()  # exactly representable: re-encoding it reproduces the words
    dx = 1.0 / 128
    assert s100[:, 1].min() < 3.5 * dx
    g = q.Scene(sc, sch, s100, stats=True)
    o = oracle.QuantRollout(sc, sch, s100)
    qt = quanta(oracle, sc, sch)[None]
    g.step(1)
    o.step(1)
    r = g.readback(state=True, ids=True)
    assert np.array_equal(r["ids"], o.ids)
    assert (np.abs(r["state"] - o.state()) / qt).max() <= 2.0
    g.step(99)
    o.step(99)
    r = g.readback(state=True, ids=True)
    got = np.empty_like(r["state"])
    got[r["ids"]] = r["state"]
    ref = np.empty_like(got)
    ref[o.ids] = o.state()
    assert sum(r["stats"]["saturations"]) == 0 and o.stats[:4].sum() == 0
    d = np.abs(got[:, :2] - ref[:, :2]) / qt[:, :2]
    assert np.percentile(d, 99) <= 32
    for st in (got, ref):
        assert st[:, 1].min() >= 2.5 * dx  # nothing is pushed into the wall band
        low = st[:, 1] <= np.percentile(st[:, 1], 5)  # the bottom row of the block
        assert low.sum() > 10 and st[low, 3].mean() > -0.1
        assert st[:, 3].mean() > -0.3


def test_empty_and_single_particle(q, oracle):
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.block2d_scene(n_strata=(4, 4))
    sch = scenes.block2d_scheme()
    g = q.Scene(sc, sch, s0[:0])
    g.step(3)
    r = g.readback(state=True, words=True, ids=True)
    assert r["state"].shape == (0, 12) and g.measure() == 0.0
    g.close()
    g = q.Scene(sc, sch, s0[:1])
    o = oracle.QuantRollout(sc, sch, s0[:1])
    g.step(5)
    o.step(5)
    d = np.abs(g.readback()["state"] - o.state()) / quanta(oracle, sc, sch)[None]
    assert d.max() <= 2


def test_strict_mode_reports_saturation(q):
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.block2d_scene(n_strata=(16, 8))
    sch = scenes.block2d_scheme()
    sch["v"] = dict(bits=4, frac=13, offset=-8, container=0)  # |v| < 1e-3 only
    s0[:, 2:4] = 1.0
    g = q.Scene(sc, sch, s0, stats=True, strict=True)
    with pytest.raises(q.QmpmError) as ei:
        g.readback()
    assert ei.value.code == -6


def test_step_host_round_trip(q, oracle):
    # the end-to-end entry point (host words in and out) gives the resident result
    import torch
    from paper_2207_04658_b300 import scenes
    name, sc, s0, sch = SCENES[1]
    a = q.Scene(sc, sch, s0)
    b = q.Scene(sc, sch, s0)
    w = a.readback(state=False, words=True, ids=False)["words"]
    hin = torch.from_numpy(w.copy()).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    q.qmpm_step_host(b.h, 1, hin.data_ptr(), hout.data_ptr())
    a.step(1)
    wa = a.readback(state=True, words=True, ids=False)
    sb = b.readback(state=True, ids=False)["state"]
    d = np.abs(wa["state"] - sb) / quanta(oracle, sc, sch)[None]
    assert d.max() <= 2
    assert np.array_equal(hout.numpy(), b.readback(state=False, words=True, ids=False)["words"])


@pytest.mark.parametrize("chunks", [1, 3, 64])
def test_step_host_stream_matches_step_by_step_host_calls(q, oracle, chunks):
    # the pipelined end-to-end rollout (copies in particle ranges on two streams) gives the
    # state of one qmpm_step_host call per step, and leaves the final state in the host words
    import torch
    name, sc, s0, sch = SCENES[1]
    a = q.Scene(sc, sch, s0)
    b = q.Scene(sc, sch, s0)
    w = a.readback(state=False, words=True, ids=False)["words"]
    hin = torch.from_numpy(w.copy()).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    steps = 5
    for _ in range(steps):
        q.qmpm_step_host(a.h, 1, hin.data_ptr(), hout.data_ptr())
        hin, hout = hout, hin
    hb = torch.from_numpy(w.copy()).pin_memory()
    q.qmpm_step_host_stream(b.h, steps, hb.data_ptr(), chunks)
    sa = a.readback(state=True, ids=False)["state"]
    rb = b.readback(state=True, words=True, ids=False)
    d = np.abs(sa - rb["state"]) / quanta(oracle, sc, sch)[None]
    assert d.max() <= 2
    assert np.array_equal(hb.numpy(), rb["words"])
    # nothing to do, and bad arguments
    q.qmpm_step_host_stream(b.h, 0, 0, chunks)
    for bad in ((b.h, -1, hb.data_ptr(), 1), (b.h, 1, hb.data_ptr(), 65), (b.h, 1, 0, 1)):
        with pytest.raises(q.QmpmError) as ei:
            q.qmpm_step_host_stream(*bad)
        assert ei.value.code == -1
    a.close()
    b.close()


@pytest.mark.parametrize("dim,grid_log2", [(2, 11), (3, 10)])
def test_largest_grids_free_fall(q, dim, grid_log2):
    # the largest grids the ABI accepts (2048^2, 1024^3: 35 GB of 3D grid buffers): a small
    # body far from the walls in free fall keeps its shape, falls with v = g t exactly in
    # FP32 state (a uniform velocity field is reproduced by P2G + G2P) and touches only the
    # blocks around it
    from paper_2207_04658_b300 import scenes
    n = 1 << grid_log2
    dx = 1.0 / n
    gen = np.random.default_rng(3)
    x = scenes.jitter_box(gen, np.full(dim, 0.5), np.full(dim, 6 * dx), (12,) * dim)
    s0 = scenes.initial_state(dim, "neohookean", x)
    # dt large enough that each step's displacement is well above the FP32 resolution of x
    # near 0.5; a soft material keeps the step within its CFL limit
    sc = dict(dim=dim, material="neohookean", grid_log2=grid_log2, bound=3, dt=1e-4, E=1.0, nu=0.2,
              bulk=0.0, rho=1.0, p_vol=(6 * dx) ** dim / x.shape[0], gravity=(0.0, -9.8, 0.0), seed=1,
              dither=True, resort_every=8)
    g = q.Scene(sc, None, s0, stats=True)
    T = 100
    g.step(T)
    st = g.state_by_id()
    stats = g.readback(state=False, ids=False)["stats"]
    g.close()
    vy = st[:, dim + 1]
    assert np.allclose(vy, -9.8 * sc["dt"] * T, rtol=1e-4)
    dy = st[:, 1] - s0[:, 1]
    assert np.allclose(dy, -9.8 * sc["dt"] ** 2 * T * (T + 1) / 2, rtol=2e-3)
    assert np.allclose(st[:, 0], s0[:, 0], atol=1e-6)
    assert stats["out_of_grid"] == 0 and stats["out_of_tile"] == 0
    assert 0 < stats["active_blocks"] <= 4 ** dim
