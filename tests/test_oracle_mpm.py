"""Pins of the oracle's MLS-MPM step (the simulator the paper quantizes, Sec. 8.1) and of
its quantized form (Sec. 3.1 Eq. 1).  Invariants and special cases fixed by the
mathematics of the quadratic B-spline APIC transfer.  CPU only."""
import math

import numpy as np
import pytest

SCENE_BASE = dict(bound=3, dt=1e-4, E=1e3, nu=0.2, bulk=400.0, rho=1.0, p_vol=1e-5,
                  gravity=(0.0, 0.0, 0.0))


def scene(dim, material, **kw):
    s = dict(SCENE_BASE, dim=dim, material=material, grid_log2=5 if dim == 3 else 6)
    s.update(kw)
    return s


def random_state(gen, dim, material, N, lo=0.3, hi=0.7, vscale=1.0, cscale=5.0, fscale=0.1):
    nc = 2 * dim + dim * dim + (1 if material == "fluid" else dim * dim)
    s = np.zeros((N, nc))
    s[:, :dim] = gen.uniform(lo, hi, (N, dim))
    s[:, dim:2 * dim] = gen.normal(0, vscale, (N, dim))
    s[:, 2 * dim:2 * dim + dim * dim] = gen.normal(0, cscale, (N, dim * dim))
    off = 2 * dim + dim * dim
    if material == "fluid":
        s[:, off] = 1.0 + gen.uniform(-0.1, 0.1, N)
    else:
        F = np.eye(dim)[None] + fscale * gen.normal(0, 1, (N, dim, dim))
        s[:, off:] = F.reshape(N, -1)
    return s


def node_positions(dim, n):
    ax = np.arange(n) / n
    return np.stack(np.meshgrid(*([ax] * dim), indexing="ij"), -1).reshape(-1, dim)


CASES = [(2, "neohookean"), (2, "corotated"), (2, "fluid"),
         (3, "neohookean"), (3, "corotated"), (3, "fluid")]


def cross2(a, b):
    return a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]


@pytest.mark.parametrize("dim,material", CASES)
def test_p2g_conserves_mass_and_momenta(oracle, dim, material):
    gen = np.random.default_rng(dim * 10 + len(material))
    sc = scene(dim, material)
    ph = oracle.make_phys(sc)
    s = random_state(gen, dim, material, 300)
    grid, oog = oracle.p2g(ph, s)
    assert oog == 0
    n = 1 << sc["grid_log2"]
    mp = ph.p_mass
    x, v = s[:, :dim], s[:, dim:2 * dim]
    C = s[:, 2 * dim:2 * dim + dim * dim].reshape(-1, dim, dim)
    m_i, mv_i = grid[:, 0], grid[:, 1:]
    # mass
    assert abs(m_i.sum() - mp * len(s)) <= 1e-12 * mp * len(s)
    # linear momentum (sum_i w_ip (x_i - x_p) = 0 kills the affine term)
    P = mp * v.sum(0)
    assert np.allclose(mv_i.sum(0), P, rtol=0, atol=1e-12 * np.abs(mp * v).sum())
    # angular momentum: sum_i x_i x mv_i = sum_p m_p [x_p x v_p + (dx^2/4) eps:C_p^T];
    # the stress part drops out because tau is symmetric
    dx = 1.0 / n
    xi = node_positions(dim, n)
    if dim == 2:
        L_grid = cross2(xi, mv_i).sum()
        L_part = (mp * cross2(x, v)).sum() + mp * dx * dx / 4 * (C[:, 1, 0] - C[:, 0, 1]).sum()
        scale = np.abs(mp * cross2(x, v)).sum() + mp * dx * dx * np.abs(C).sum()
    else:
        L_grid = np.cross(xi, mv_i).sum(0)
        eps_C = np.stack([C[:, 2, 1] - C[:, 1, 2], C[:, 0, 2] - C[:, 2, 0],
                          C[:, 1, 0] - C[:, 0, 1]], -1)
        L_part = (mp * np.cross(x, v)).sum(0) + mp * dx * dx / 4 * eps_C.sum(0)
        scale = np.abs(mp * np.cross(x, v)).sum() + mp * dx * dx * np.abs(C).sum()
    assert np.allclose(L_grid, L_part, rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("dim", [2, 3])
def test_g2p_reproduces_affine_field(oracle, dim):
    # v_i = v0 + G x_i on the nodes  =>  v_p = v0 + G x_p and C_p = G (D_p = dx^2/4 I)
    gen = np.random.default_rng(40 + dim)
    sc = scene(dim, "neohookean")
    ph = oracle.make_phys(sc)
    n = 1 << sc["grid_log2"]
    v0 = gen.normal(0, 1, dim)
    G = gen.normal(0, 1, (dim, dim))
    xi = node_positions(dim, n)
    grid = np.zeros((n ** dim, 1 + dim))
    grid[:, 0] = 1.0
    grid[:, 1:] = v0 + xi @ G.T
    s = random_state(gen, dim, "neohookean", 200)
    s2 = oracle.g2p(ph, grid, s)
    xp = s[:, :dim]
    vp = v0 + xp @ G.T
    assert np.allclose(s2[:, dim:2 * dim], vp, rtol=0, atol=1e-12)
    Cp = s2[:, 2 * dim:2 * dim + dim * dim].reshape(-1, dim, dim)
    assert np.allclose(Cp, G[None], rtol=0, atol=1e-9)
    assert np.allclose(s2[:, :dim], xp + sc["dt"] * vp, rtol=0, atol=1e-14)
    # F <- (I + dt C) F with the new C
    F0 = s[:, 2 * dim + dim * dim:].reshape(-1, dim, dim)
    F1 = s2[:, 2 * dim + dim * dim:].reshape(-1, dim, dim)
    assert np.allclose(F1, (np.eye(dim) + sc["dt"] * G)[None] @ F0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("dim,material", CASES)
def test_rigid_translation_stays_rigid(oracle, dim, material):
    gen = np.random.default_rng(50 + dim)
    sc = scene(dim, material)
    ph = oracle.make_phys(sc)
    N = 400
    s = random_state(gen, dim, material, N)
    vel = gen.normal(0, 1, dim)
    s[:, dim:2 * dim] = vel
    s[:, 2 * dim:] = 0.0
    off = 2 * dim + dim * dim
    if material == "fluid":
        s[:, off] = 1.0
    else:
        s[:, off:] = np.eye(dim).ravel()
    s2 = oracle.step_fp64(ph, s)
    assert np.allclose(s2[:, dim:2 * dim], vel[None], rtol=0, atol=1e-13)
    assert np.allclose(s2[:, 2 * dim:off], 0.0, rtol=0, atol=1e-9)
    assert np.allclose(s2[:, :dim], s[:, :dim] + sc["dt"] * vel, rtol=0, atol=1e-15)
    assert np.allclose(s2[:, off:], s[:, off:], rtol=0, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_free_fall_one_step(oracle, dim):
    # at rest, no stress: the grid gains dt g, the particles v = dt g, x += dt^2 g
    g = (0.0, -9.8, 0.0)
    sc = scene(dim, "corotated", gravity=g)
    ph = oracle.make_phys(sc)
    gen = np.random.default_rng(60)
    s = random_state(gen, dim, "corotated", 100)
    s[:, dim:] = 0.0
    s[:, 2 * dim + dim * dim:] = np.eye(dim).ravel()
    s2 = oracle.step_fp64(ph, s)
    gv = np.array(g[:dim])
    assert np.allclose(s2[:, dim:2 * dim], sc["dt"] * gv, rtol=0, atol=1e-15)
    assert np.allclose(s2[:, :dim], s[:, :dim] + sc["dt"] ** 2 * gv, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim,material", CASES)
def test_step_momentum_balance(oracle, dim, material):
    # sum_p m_p v_p' = sum_i m_i v_i = P + M dt g, away from the walls
    g = (0.3, -9.8, 1.1)
    sc = scene(dim, material, gravity=g)
    ph = oracle.make_phys(sc)
    gen = np.random.default_rng(70 + dim)
    s = random_state(gen, dim, material, 300)
    s2 = oracle.step_fp64(ph, s)
    P0 = ph.p_mass * s[:, dim:2 * dim].sum(0)
    P1 = ph.p_mass * s2[:, dim:2 * dim].sum(0)
    M = ph.p_mass * len(s)
    expect = P0 + M * sc["dt"] * np.array(g[:dim])
    assert np.allclose(P1, expect, rtol=0, atol=1e-12 * (np.abs(ph.p_mass * s[:, dim:2 * dim]).sum() + M))


def test_sticky_walls(oracle):
    sc = scene(2, "neohookean", gravity=(0.0, -9.8, 0.0))
    ph = oracle.make_phys(sc)
    n = 1 << sc["grid_log2"]
    grid = np.zeros((n * n, 3))
    grid[:, 0] = 2.0
    grid[:, 1] = 4.0
    grid[:, 2] = -6.0
    out = oracle.grid_update(ph, grid).reshape(n, n, 3)
    B = sc["bound"]
    interior = out[B:n - B, B:n - B]
    assert np.allclose(interior[..., 1], 2.0)
    assert np.allclose(interior[..., 2], -3.0 + sc["dt"] * -9.8)
    for sl in [out[:B], out[n - B:], out[:, :B], out[:, n - B:]]:
        assert np.all(sl[..., 1:] == 0.0)
    # empty nodes carry no velocity
    grid[:, 0] = 0.0
    assert np.all(oracle.grid_update(ph, grid)[:, 1:] == 0.0)


def psi(material, F, mu, la, K):
    d = F.shape[0]
    J = np.linalg.det(F)
    if material == "neohookean":
        return mu / 2 * (np.trace(F.T @ F) - d) - mu * math.log(J) + la / 2 * math.log(J) ** 2
    U, S, Vt = np.linalg.svd(F)
    R = U @ Vt
    return mu * np.sum((F - R) ** 2) + la / 2 * (J - 1) ** 2


@pytest.mark.parametrize("dim,material", [(2, "neohookean"), (3, "neohookean"),
                                          (2, "corotated"), (3, "corotated")])
def test_stress_is_energy_derivative(oracle, dim, material):
    # tau = (d psi / d F) F^T for the hyperelastic energies the materials are named after
    sc = scene(dim, material, E=1000.0, nu=0.3)
    ph = oracle.make_phys(sc)
    mu = sc["E"] / (2 * (1 + sc["nu"]))
    la = sc["E"] * sc["nu"] / ((1 + sc["nu"]) * (1 - 2 * sc["nu"]))
    gen = np.random.default_rng(80 + dim)
    for _ in range(5):
        F = np.eye(dim) + 0.2 * gen.normal(0, 1, (dim, dim))
        if np.linalg.det(F) <= 0.2:
            continue
        h = 1e-6
        P = np.zeros((dim, dim))
        for a in range(dim):
            for b in range(dim):
                Fp, Fm = F.copy(), F.copy()
                Fp[a, b] += h
                Fm[a, b] -= h
                P[a, b] = (psi(material, Fp, mu, la, 0) - psi(material, Fm, mu, la, 0)) / (2 * h)
        tau = oracle.kirchhoff(ph, F)
        assert np.allclose(tau, P @ F.T, rtol=1e-6, atol=1e-5)
    # zero stress at rest
    assert np.allclose(oracle.kirchhoff(ph, np.eye(dim)), 0.0, atol=1e-12)


def test_fluid_pressure(oracle):
    # psi(J) = K/2 (J-1)^2: tau = J psi'(J) I, zero at J = 1
    for dim in (2, 3):
        sc = scene(dim, "fluid", bulk=400.0)
        ph = oracle.make_phys(sc)
        for J in [0.9, 1.0, 1.05]:
            h = 1e-7
            dpsi = (200.0 * (J + h - 1) ** 2 - 200.0 * (J - h - 1) ** 2) / (2 * h)
            assert np.allclose(oracle.kirchhoff(ph, np.array([J])), J * dpsi * np.eye(dim),
                               rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("dim", [2, 3])
def test_polar_decomposition(oracle, dim):
    gen = np.random.default_rng(90 + dim)
    for _ in range(20):
        F = np.eye(dim) + 0.5 * gen.normal(0, 1, (dim, dim))
        if np.linalg.det(F) <= 0.05:
            continue
        R = oracle.polar(F)
        assert np.allclose(R.T @ R, np.eye(dim), atol=1e-12)
        assert abs(np.linalg.det(R) - 1.0) < 1e-12
        S = R.T @ F
        assert np.allclose(S, S.T, atol=1e-12)
        assert np.all(np.linalg.eigvalsh((S + S.T) / 2) > 0)
        U, _, Vt = np.linalg.svd(F)
        assert np.allclose(R, U @ Vt, atol=1e-10)


@pytest.mark.parametrize("dim,material", [(2, "neohookean"), (3, "corotated"), (3, "fluid")])
def test_tile_keys_cover_stencil(oracle, dim, material):
    # the tile of blocks T..T+1 (4 nodes each, padded grid) holds every stencil node with
    # one node of slack on both sides
    sc = scene(dim, material)
    ph = oracle.make_phys(sc)
    n = 1 << sc["grid_log2"]
    nb = n // 4 + 2
    gen = np.random.default_rng(100 + dim)
    s = random_state(gen, dim, material, 2000, lo=0.6 / n, hi=1.0 - 1.6 / n)
    keys = oracle.tile_keys(ph, s)
    ncell = 4 ** dim
    assert keys.min() >= 0 and keys.max() < oracle.n_keys(ph) == nb ** dim * ncell
    T = np.stack(np.unravel_index(keys // ncell, (nb,) * dim), -1)
    cell = np.stack(np.unravel_index(keys % ncell, (4,) * dim), -1)
    base = np.floor(s[:, :dim] * n - 0.5).astype(int)
    lo_node = 4 * (T - 1)  # first node of the tile
    assert np.all(base - 1 >= lo_node)
    assert np.all(base + 2 + 1 <= lo_node + 7)
    # the cell part orders particles by their base inside the tile
    assert np.array_equal(base, lo_node + 1 + cell)


def test_stable_sort_is_stable(oracle):
    gen = np.random.default_rng(110)
    keys = gen.integers(0, 50, 5000)
    perm = oracle.stable_sort(keys, 50)
    assert list(perm) == sorted(range(len(keys)), key=lambda i: keys[i])


def test_quantized_step_is_step_then_store(oracle):
    # Eq. 1: s~_t = F(s~_{t-1}) + e_t with |e_t| < Delta per component (dithered store)
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.block2d_scene(n_strata=(32, 16))
    sch = scenes.block2d_scheme()
    ph = oracle.make_phys(sc)
    cd = oracle.make_codec(sc, sch)
    w0 = oracle.encode_state(cd, s0, 0)
    sq = oracle.decode_state(cd, w0)
    ref = oracle.step_fp64(ph, sq)
    w1 = w0.copy()
    stats = np.zeros(oracle.N_STATS, dtype=np.int64)
    scratch_s = np.zeros_like(sq)
    grid = np.zeros(oracle.n_nodes(ph) * 3)
    import ctypes as ct
    oracle.lib().or_step_quant(ct.byref(ph), ct.byref(cd), len(sq), oracle._p(w1, ct.c_uint32), 1,
                               oracle._p(scratch_s, ct.c_double), oracle._p(grid, ct.c_double),
                               oracle._p(stats, ct.c_int64))
    got = oracle.decode_state(cd, w1)
    delta = np.array([2.0 ** -cd.frac[c] for c in range(cd.n_comp)])
    assert np.all(np.abs(got - ref) < delta[None])
    assert stats[:4].sum() == 0  # no saturation


def test_quantized_rollout_tracks_fp64(oracle):
    # a fine scheme keeps the quantized rollout close to the FP64 rollout (same ordering)
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.block2d_scene(n_strata=(32, 16), steps=40)
    sch = scenes.block2d_scheme()
    q = oracle.QuantRollout(sc, sch, s0)
    f = oracle.Fp64Rollout(sc, s0)
    q.step(40)
    f.step(40)
    sq = np.zeros_like(f.s)
    sq[q.ids] = q.state()
    sf = np.zeros_like(f.s)
    sf[f.ids] = f.s
    zq = oracle.mean_sq_pos(2, sq)
    zf = oracle.mean_sq_pos(2, sf)
    assert abs(zq - zf) / zf < 1e-4
    assert np.abs(sq[:, :2] - sf[:, :2]).max() < 1e-3


def test_threaded_build_matches_sequential(oracle):
    # the OpenMP build (used only for full-size reference runs) sums P2G in another order:
    # FP64 results agree to rounding, quantized ones to at most a quantum where that
    # rounding crosses a dither threshold
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.cubes3d_scene(n_cubes=1, cube_cells=8, grid_log2=5, seed=8)
    sch = scenes.fixed_scheme_3d("corotated")
    a = oracle.Fp64Rollout(sc, s0)
    b = oracle.Fp64Rollout(sc, s0, threaded=True)
    a.step(3)
    b.step(3)
    assert np.array_equal(a.ids, b.ids)
    assert np.allclose(a.s, b.s, rtol=1e-12, atol=1e-12)
    qa = oracle.QuantRollout(sc, sch, s0)
    qb = oracle.QuantRollout(sc, sch, s0, threaded=True)
    qa.step(3)
    qb.step(3)
    assert np.array_equal(qa.ids, qb.ids)
    d = np.abs(qa.state() - qb.state())
    fields = oracle.comp_fields(3, "corotated")
    quanta = np.array([2.0 ** -sch[["x", "v", "C", "F"][h]]["frac"] for h in fields])
    assert (d <= quanta[None] * (1 + 1e-9)).all()
    assert (d == 0).mean() > 0.999


def test_polar_decomposition_inverted_and_singular(oracle):
    """An inverted F (det < 0) gets the orthogonal factor of the SVD (det R = -1, U V^T); a
    (nearly) singular one, |det F| < 1e-6, has no unique factor and gets R = I (the reading
    both the oracle and the kernels take)."""
    gen = np.random.default_rng(17)
    for _ in range(20):
        F = np.eye(3) + 0.5 * gen.normal(0, 1, (3, 3))
        F[0] *= -1.0  # invert
        if np.linalg.det(F) > -0.05:
            continue
        R = oracle.polar(F)
        U, _, Vt = np.linalg.svd(F)
        assert np.allclose(R, U @ Vt, atol=1e-10) and np.linalg.det(R) == pytest.approx(-1.0, abs=1e-12)
    for F in (np.zeros((3, 3)), np.diag([1.0, 1.0, 0.0]), np.outer([1.0, 2.0, 3.0], [0.5, -1.0, 2.0])):
        assert np.array_equal(oracle.polar(F), np.eye(3))
