"""Pins of the oracle's reverse mode (Sec. 6, Eq. 12-13): the adjoint of a short FP64
rollout equals central finite differences of the measurement, both with respect to the
initial state and to errors injected into intermediate states (the sensitivities that
Eq. 8 accumulates).  CPU only."""
import numpy as np
import pytest

CASES = [(2, "neohookean"), (2, "corotated"), (2, "fluid"),
         (3, "neohookean"), (3, "corotated"), (3, "fluid")]


def small(oracle, dim, material, N=40, seed=0):
    gen = np.random.default_rng(seed + 10 * dim + len(material))
    sc = dict(dim=dim, material=material, grid_log2=5 if dim == 2 else 4, bound=3, dt=2e-4,
              E=2e3, nu=0.3, bulk=300.0, rho=1.0, p_vol=2e-5, gravity=(0.5, -9.8, 1.0))
    ph = oracle.make_phys(sc)
    nc = oracle.n_comp(dim, material)
    s = np.zeros((N, nc))
    s[:, :dim] = gen.uniform(0.4, 0.6, (N, dim))
    s[:, dim:2 * dim] = gen.normal(0, 0.5, (N, dim))
    s[:, 2 * dim:2 * dim + dim * dim] = gen.normal(0, 2.0, (N, dim * dim))
    off = 2 * dim + dim * dim
    if material == "fluid":
        s[:, off] = 1.0 + gen.uniform(-0.05, 0.05, N)
    else:
        F = np.eye(dim)[None] + 0.05 * gen.normal(0, 1, (N, dim, dim))
        s[:, off:] = F.reshape(N, -1)
    return sc, ph, s


def z_from(oracle, ph, s, T):
    for _ in range(T):
        s = oracle.step_fp64(ph, s)
    return oracle.mean_sq_pos(ph.dim, s)


@pytest.mark.parametrize("dim,material", CASES)
def test_adjoint_matches_central_differences(oracle, dim, material):
    sc, ph, s0 = small(oracle, dim, material)
    T = 3
    z, adj, g = oracle.rollout_adjoint(ph, s0, T)
    sb0 = adj[0]
    gen = np.random.default_rng(7)
    scale = np.abs(sb0).max()
    checked = 0
    for _ in range(24):
        p = int(gen.integers(0, s0.shape[0]))
        c = int(gen.integers(0, s0.shape[1]))
        h = 1e-6 * max(1.0, abs(s0[p, c]))
        sp, sm = s0.copy(), s0.copy()
        sp[p, c] += h
        sm[p, c] -= h
        fd = (z_from(oracle, ph, sp, T) - z_from(oracle, ph, sm, T)) / (2 * h)
        assert abs(fd - sb0[p, c]) <= 1e-5 * (abs(sb0[p, c]) + 1e-3 * scale), (p, c, fd, sb0[p, c])
        checked += 1
    assert checked == 24


@pytest.mark.parametrize("dim,material", [(2, "corotated"), (3, "corotated"), (3, "fluid")])
def test_injected_error_sensitivities(oracle, dim, material):
    # dz/de_t = dz/ds_t for an error e_t injected into the state after step t (Eq. 1)
    sc, ph, s0 = small(oracle, dim, material, seed=3)
    T = 4
    z, adj, g = oracle.rollout_adjoint(ph, s0, T)
    states = oracle.rollout_fp64(ph, s0, T)
    gen = np.random.default_rng(11)
    for _ in range(16):
        t = int(gen.integers(0, T + 1))
        p = int(gen.integers(0, s0.shape[0]))
        c = int(gen.integers(0, s0.shape[1]))
        h = 1e-6 * max(1.0, abs(states[t][p, c]))
        zs = []
        for sgn in (1.0, -1.0):
            st = states[t].copy()
            st[p, c] += sgn * h
            zs.append(z_from(oracle, ph, st, T - t))
        fd = (zs[0] - zs[1]) / (2 * h)
        scale = np.abs(adj[t]).max()
        assert abs(fd - adj[t][p, c]) <= 1e-5 * (abs(adj[t][p, c]) + 1e-3 * scale), (t, p, c)
    # g_h of Eq. 8 is the sum over steps and variables of the squared sensitivities
    fields = oracle.comp_fields(dim, material)
    g2 = np.zeros(4)
    for a in adj:
        for c in range(a.shape[1]):
            g2[fields[c]] += (a[:, c] ** 2).sum()
    assert np.allclose(g, g2, rtol=1e-12)


def test_seed_of_mean_square_position(oracle):
    sc, ph, s0 = small(oracle, 3, "fluid")
    g = oracle.mean_sq_pos_seed(3, s0)
    h = 1e-6
    for p, c in [(0, 0), (5, 2), (7, 4)]:
        sp, sm = s0.copy(), s0.copy()
        sp[p, c] += h
        sm[p, c] -= h
        fd = (oracle.mean_sq_pos(3, sp) - oracle.mean_sq_pos(3, sm)) / (2 * h)
        assert abs(fd - g[p, c]) < 1e-9
