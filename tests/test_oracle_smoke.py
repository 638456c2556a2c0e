"""Pins of the oracle's 2D advection-reflection smoke (Sec. 8.1) against what the
mathematics fixes, CPU only:
  - a state at rest with no source stays exactly at rest (the step adds nothing);
  - a uniform flow translates a linear density exactly (RK-3 of a constant field is the
    straight path and bilinear interpolation is exact for linear fields), and interior
    velocities stay uniform (reflection of a divergence-free uniform field is itself);
  - a solid rotation follows third-order paths in closed form (velocity advected by
    itself, reflected, advected again; density advected by the projected half-step
    velocity);
  - with enough Jacobi sweeps the step's final velocity is discretely divergence-free up
    to the one checkerboard mode that undamped Jacobi cannot remove (the sign and the h^2
    scaling of the Poisson solve and of the gradient);
  - a quantized store with a fine scheme lands within its quanta of the FP64 value;
  - the store-event enumeration and injection hook: central differences over every
    store, combined with the dither's rounding variance Delta^2 / 6 (Sec. 5), predict the
    variance of z over dither seeds (Eq. 8's linear error propagation);
  - single stages: the step's stores up to the second advection, rebuilt from or_smoke_stage's
    stages, equal or_smoke_step's codes;
  - antithetic noise injection estimates the FD sensitivities g_h, and the mean shift of
    z under dithered stores equals that under noise of the same variance."""
import numpy as np


def scene(**kw):
    sc = dict(n=16, jacobi=16, dt=0.02, buoyancy=0.0, v_in=0.0, src=(1.0, 1.0, -1.0, -1.0), seed=5)
    sc.update(kw)
    return sc


def divergence(u, v):
    n = u.shape[0]
    return (u[:, 1:] - u[:, :-1] + v[1:, :] - v[:-1, :]) * n


def test_rest_stays_at_rest(oracle):
    gen = np.random.default_rng(0)
    n = 16
    d0 = gen.uniform(0, 1, (n, n))
    r = oracle.SmokeRollout(scene(), None, d0=d0)
    r.step(3)
    assert np.array_equal(r.d, d0)
    assert not r.u.any() and not r.v.any() and not r.q.any()


def test_uniform_flow_translates_linear_density(oracle):
    n, cu, cv, dt = 32, 0.5, -0.3, 0.02
    h = 1.0 / n
    u0 = np.full((n, n + 1), cu)
    v0 = np.full((n + 1, n), cv)
    u0[:, 0] = u0[:, -1] = 0.0
    v0[0, :] = v0[-1, :] = 0.0
    xc = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(xc, xc)  # [row = y][col = x]
    a, b, c = 0.2, 1.5, -0.7
    d0 = a + b * X + c * Y
    r = oracle.SmokeRollout(scene(n=n, jacobi=0, dt=dt), None, u0=u0, v0=v0, d0=d0)
    r.step(1)
    inner = slice(8, 24)
    want = a + b * (X - cu * dt) + c * (Y - cv * dt)
    assert np.abs(r.d[inner, inner] - want[inner, inner]).max() < 1e-12
    assert np.abs(r.u[inner, inner] - cu).max() < 1e-12
    assert np.abs(r.v[inner, inner] - cv).max() < 1e-12


def p3(M):
    """Third-order Taylor polynomial of exp(M): what any third-order Runge-Kutta method
    (Ralston's included) computes for a linear autonomous ODE."""
    I = np.eye(2)
    return I + M + M @ M / 2 + M @ M @ M / 6


def test_rotation_follows_third_order_paths(oracle):
    """A solid rotation w = A (x - c) with no projection (0 sweeps): the backtrace of a
    linear field is x_b - c = P3(-s A) (x - c), bilinear interpolation of linear fields is
    exact, and the reflection of an unprojected field is the field itself.  So the step
    makes u~ = u' = B (x - c) with B = A P3(-dt/2 A), the final velocity
    B P3(-dt/2 B) (x - c), and moves the density along P3(-dt B) (the step advects it by
    u', not by the final velocity)."""
    n, dt, om = 32, 0.02, 1.3
    h = 1.0 / n
    A = om * np.array([[0.0, -1.0], [1.0, 0.0]])
    c = np.array([0.5, 0.5])

    def lin(M, x, y):  # field M (p - c) at points (x, y): returns its two components
        return M[0, 0] * (x - c[0]) + M[0, 1] * (y - c[1]), M[1, 0] * (x - c[0]) + M[1, 1] * (y - c[1])

    ux, uy = np.meshgrid(np.arange(n + 1) * h, (np.arange(n) + 0.5) * h)  # u faces
    vx, vy = np.meshgrid((np.arange(n) + 0.5) * h, np.arange(n + 1) * h)  # v faces
    cx, cy = np.meshgrid((np.arange(n) + 0.5) * h, (np.arange(n) + 0.5) * h)
    u0 = lin(A, ux, uy)[0]
    v0 = lin(A, vx, vy)[1]
    u0[:, 0] = u0[:, -1] = 0.0
    v0[0, :] = v0[-1, :] = 0.0
    a, b, e = 0.3, 1.1, -0.6
    d0 = a + b * cx + e * cy
    r = oracle.SmokeRollout(scene(n=n, jacobi=0, dt=dt), None, u0=u0, v0=v0, d0=d0)
    r.step(1)
    B = A @ p3(-dt / 2 * A)
    F = B @ p3(-dt / 2 * B)
    inner = slice(8, 24)
    assert np.abs(r.u[inner, inner] - lin(F, ux, uy)[0][inner, inner]).max() < 1e-12
    assert np.abs(r.v[inner, inner] - lin(F, vx, vy)[1][inner, inner]).max() < 1e-12
    xb, yb = lin(p3(-dt * B), cx, cy)
    want = a + b * (xb + c[0]) + e * (yb + c[1])
    assert np.abs(r.d[inner, inner] - want[inner, inner]).max() < 1e-12
    # a second-order path (Taylor to dt^2) is off by far more than the tolerance
    P2 = np.eye(2) - dt * B + (dt * B) @ (dt * B) / 2
    xb2, yb2 = lin(P2, cx, cy)
    off = a + b * (xb2 + c[0]) + e * (yb2 + c[1])
    assert np.abs(off - want)[inner, inner].max() > 1e-8


def checkerboard_residual(D):
    """Divergence with its component along (-1)^(i+j) cnt_ij removed: undamped Jacobi on the
    Neumann Laplacian (a cell divides by its cnt interior neighbours) has iteration
    eigenvalue -1 on the bipartite grid, so that one mode of the divergence is never
    removed; every other mode converges."""
    n = D.shape[0]
    cnt = np.full((n, n), 4.0)
    cnt[0, :] -= 1
    cnt[-1, :] -= 1
    cnt[:, 0] -= 1
    cnt[:, -1] -= 1
    w = np.fromfunction(lambda j, i: (-1.0) ** (i + j), (n, n)) * cnt
    return D - (D * w).sum() / (w * w).sum() * w


def test_converged_projection_is_divergence_free(oracle):
    gen = np.random.default_rng(1)
    n = 12
    u0 = gen.normal(0, 0.3, (n, n + 1))
    v0 = gen.normal(0, 0.3, (n + 1, n))
    u0[:, 0] = u0[:, -1] = 0.0
    v0[0, :] = v0[-1, :] = 0.0
    d_before = np.abs(divergence(u0, v0)).max()
    r = oracle.SmokeRollout(scene(n=n, jacobi=3000, dt=0.01), None, u0=u0, v0=v0)
    r.step(1)
    d_after = np.abs(checkerboard_residual(divergence(r.u, r.v))).max()
    assert d_before > 1.0
    assert d_after < 1e-12 * d_before, (d_before, d_after)
    assert not r.u[:, 0].any() and not r.u[:, -1].any()
    assert not r.v[0, :].any() and not r.v[-1, :].any()
    # thirty sweeps leave a visible residual: the iteration is what converges
    r2 = oracle.SmokeRollout(scene(n=n, jacobi=30, dt=0.01), None, u0=u0, v0=v0)
    r2.step(1)
    assert np.abs(checkerboard_residual(divergence(r2.u, r2.v))).max() > 1e-4 * d_before


def plume(n=16, jacobi=16, T=4, **kw):
    return scene(n=n, jacobi=jacobi, dt=0.02, buoyancy=1.0, v_in=1.0, src=(0.35, 0.05, 0.65, 0.2), **kw), T


def test_fine_scheme_tracks_fp64(oracle):
    sc, T = plume()
    ref = oracle.SmokeRollout(sc)
    ref.step(1)
    fine = {"v": dict(bits=32, frac=28, offset=-(1 << 31)), "p": dict(bits=32, frac=34, offset=-(1 << 31))}
    q = oracle.SmokeRollout(sc, fine)
    q.step(1)
    assert q.saturations == 0
    # each store is within one quantum; the pressure's error reaches the velocity through
    # the gradient (n / Delta_p) and the Jacobi sweeps average, not grow, their errors
    assert np.abs(q.u - ref.u).max() < 64 * 2.0 ** -28
    assert np.abs(q.v - ref.v).max() < 64 * 2.0 ** -28
    assert np.abs(q.d - ref.d).max() < 64 * 2.0 ** -28


def generic_state(n, seed=7):
    """A state with every interior value generic (nonzero velocities, spread density), so
    that the stored values' fractions Y are spread and their rounding variances Y (1 - Y)
    Delta^2 average to Delta^2 / 6."""
    gen = np.random.default_rng(seed)
    u0 = gen.normal(0, 0.3, (n, n + 1))
    v0 = gen.normal(0, 0.3, (n + 1, n))
    u0[:, 0] = u0[:, -1] = 0.0
    v0[0, :] = v0[-1, :] = 0.0
    return u0, v0, gen.uniform(0, 1, (n, n))


def is_wall_face(n, field, idx):
    """Wall faces store an exact zero: no rounding error is made there."""
    if field == 0:
        return idx % (n + 1) in (0, n)
    if field == 1:
        return idx // n in (0, n)
    return False


def fd_sensitivities(oracle, sc, T, state, step=1e-6):
    """Sum over the stores of each type (0 velocity, 1 pressure) of (dz/d store)^2 by
    central differences through the injection hook, on the unquantized run.  Left out: the
    wall faces (an exact zero is stored) and the reflected velocity 2 u' - u~ (an integer
    combination of two stored values of the same lattice is stored exactly)."""
    n, J = sc["n"], sc["jacobi"]
    G = np.zeros(2)
    for (h, field, idx, ctr) in oracle.smoke_store_events(n, J, T):
        if is_wall_face(n, field, idx) or (h == 0 and ctr % 1024 == J + 3):
            continue
        zs = []
        for sgn in (1.0, -1.0):
            oracle.smoke_inject(1, field, idx, ctr, sgn * step)
            r = oracle.SmokeRollout(sc, None, *state)
            r.step(T)
            zs.append(r.measure())
        oracle.smoke_inject(0)
        G[h] += ((zs[0] - zs[1]) / (2 * step)) ** 2
    return G


def test_predicted_variance_matches_dither_runs(oracle):
    # n = 12 (not a power of two) keeps the stored values off each other's lattices: with
    # n = 2^k the gradient n (q_r - q_l) of stored pressures lands on the velocity lattice
    # and some stores are then exact, which the linear prediction does not know
    sc, T = plume(n=12, jacobi=8, T=2)
    state = generic_state(12)
    G = fd_sensitivities(oracle, sc, T, state)
    sch = {"v": dict(bits=16, frac=8, offset=-(1 << 15)), "p": dict(bits=16, frac=11, offset=-(1 << 15))}
    dv, dp = 2.0 ** -8, 2.0 ** -11
    parts = np.array([G[0] * dv * dv, G[1] * dp * dp]) / 6.0
    # both types carry a sizeable share, so a dropped store kind shows
    assert parts.min() > 0.3 * parts.max(), parts
    z = []
    for s in range(800):
        r = oracle.SmokeRollout(dict(sc, seed=1000 + s), sch, *state)
        r.step(T)
        assert r.saturations == 0
        z.append(r.measure())
    obs = float(np.var(z, ddof=1))
    # 800 samples: the variance estimate's relative sd is 5%
    assert 0.75 < obs / parts.sum() < 1.2, (obs, parts)


def test_antithetic_noise_estimates_the_sensitivities(oracle):
    """Over random +-sigma_h injections at every store of type h, E[((z+ - z-) / 2)^2] is
    sigma_h^2 g_h (the FD sum over the same stores): the estimator the kernels use for
    Eq. 8's linear term."""
    sc, T = plume(n=12, jacobi=8, T=2)
    state = generic_state(12)
    G = fd_sensitivities(oracle, sc, T, state)
    pairs = 300
    for h, sigma in ((0, (1e-5, 0.0)), (1, (0.0, 1e-5))):
        est = []
        for k in range(pairs):
            zs = []
            for sign in (1.0, -1.0):
                with oracle.smoke_noise(sigma, 1 + k, sign):
                    r = oracle.SmokeRollout(sc, None, *state)
                    r.step(T)
                zs.append(r.measure())
            est.append(((zs[0] - zs[1]) / 2) ** 2 / sigma[h] ** 2)
        est = np.array(est)
        se = est.std(ddof=1) / np.sqrt(pairs)
        assert abs(est.mean() - G[h]) < 4 * se, (h, est.mean(), G[h], se)
        assert se < 0.15 * G[h]


def test_dither_bias_has_the_sign_and_size_of_equal_variance_noise(oracle):
    """The premise of the second-order term: a dithered store errs by zero-mean noise of
    variance Delta^2 / 6 on average (Sec. 5), so the mean shift of z under dithered stores
    has the sign and the order of magnitude of the shift under +-Delta/sqrt(6) noise at the
    same stores.  Only that: where a stored value's fraction is not uniform (values on a
    coarser lattice, exact zeros) the dither errs less than the noise, and the advection's
    piecewise-bilinear sampling makes the shift depend on the noise scale, which is why the
    kernels estimate it at each scheme's own scale."""
    sc, T = plume(n=24, jacobi=8, T=8)
    state = generic_state(24)
    r0 = oracle.SmokeRollout(sc, None, *state)
    r0.step(T)
    z0 = r0.measure()
    fv, fp = 5, 8
    sch = {"v": dict(bits=16, frac=fv, offset=-(1 << 15)), "p": dict(bits=16, frac=fp, offset=-(1 << 15))}
    sig = (2.0 ** -fv / 6 ** 0.5, 2.0 ** -fp / 6 ** 0.5)
    K = 300
    zq, zn = [], []
    for k in range(K):
        r = oracle.SmokeRollout(dict(sc, seed=5000 + k), sch, *state)
        r.step(T)
        assert r.saturations == 0
        zq.append(r.measure() - z0)
        with oracle.smoke_noise(sig, 9000 + k, 1.0):
            r = oracle.SmokeRollout(sc, None, *state)
            r.step(T)
        zn.append(r.measure() - z0)
    zq, zn = np.array(zq), np.array(zn)
    se_q, se_n = zq.std(ddof=1) / np.sqrt(K), zn.std(ddof=1) / np.sqrt(K)
    assert zq.mean() < -5 * se_q and zn.mean() < -5 * se_n, (zq.mean(), zn.mean(), se_q, se_n)
    assert 0.5 < zq.mean() / zn.mean() < 2.0, (zq.mean(), zn.mean())
    assert 0.6 < zq.std() / zn.std() < 1.25


def test_stages_rebuild_the_step(oracle):
    """Advection, the first projection's sweeps, the gradient subtraction with the
    reflection and the second advection, each from or_smoke_stage with the previous stage's
    stored output, give exactly the codes or_smoke_step stores (no source, no buoyancy: the
    forces change nothing)."""
    import ctypes as ct
    n, J, step = 32, 6, 2
    sc = dict(n=n, jacobi=J, dt=0.01, buoyancy=0.0, v_in=0.0, src=(1.0, 1.0, -1.0, -1.0), seed=5)
    sch = {"v": dict(bits=16, frac=12, offset=-(1 << 15)), "p": dict(bits=16, frac=18, offset=-(1 << 15))}
    gen = np.random.default_rng(4)
    u = np.round(gen.normal(0, 0.3, (n, n + 1)) * 4096) / 4096
    v = np.round(gen.normal(0, 0.3, (n + 1, n)) * 4096) / 4096
    u[:, 0] = u[:, -1] = 0.0
    v[0, :] = v[-1, :] = 0.0
    # the whole step, recording every store
    total = 5 * 2 * n * (n + 1) + 2 * J * n * n
    rec = np.zeros(total, dtype=np.uint32)
    L = oracle.lib()
    L.or_smoke_record(rec.ctypes.data_as(ct.POINTER(ct.c_uint32)), total)
    try:
        o = oracle.SmokeRollout(sc, sch, u, v, np.zeros((n, n)))
        o.t = step - 1
        o.step(1)
    finally:
        L.or_smoke_record(None, 0)
    # the same from single stages
    parts = []
    r = oracle.smoke_stage(sc, sch, "advect1", step, a=(u, v))
    parts.append(r["codes"])
    ut, vt = r["u"], r["v"]
    div = (ut[:, 1:] - ut[:, :-1] + vt[1:, :] - vt[:-1, :]) * n
    q = np.zeros((n, n))
    for it in range(1, J + 1):
        r = oracle.smoke_stage(sc, sch, "jacobi", step, arg=it, q=q, div=div)
        parts.append(r["codes"])
        q = r["q"]
    r = oracle.smoke_stage(sc, sch, "gradsub2", step, a=(ut, vt), q=q)
    parts.append(r["codes"])
    r = oracle.smoke_stage(sc, sch, "advect4", step, a=(r["u2"], r["v2"]), b=(r["u"], r["v"]))
    parts.append(r["codes"])
    built = np.concatenate(parts)
    assert np.array_equal(built, rec[:built.size])
