"""Pins of the oracle's bit-allocation solve (Sec. 4: Eq. 6-10, Algorithm 1): the
analytic Lagrange optimum against a numerical optimizer, and the integer schemes
against exhaustive enumeration.  CPU only."""
import math

import numpy as np
import pytest
from scipy.optimize import minimize


def random_problem(gen, H):
    P = gen.integers(1000, 100000, H).astype(float)
    g = 10.0 ** gen.uniform(-6, 2, H)
    lo = gen.uniform(-5, 0, H)
    hi = lo + 10.0 ** gen.uniform(-1, 1.5, H)
    z = float(10.0 ** gen.uniform(-2, 3))
    return P, g, lo, hi, z


@pytest.mark.parametrize("seed", range(6))
def test_error_bound_lagrange_matches_optimizer(oracle, seed):
    gen = np.random.default_rng(seed)
    H = int(gen.integers(2, 6))
    P, g, lo, hi, z = random_problem(gen, H)
    eps = 0.01
    out = oracle.scheme_solve(P, g, lo, hi, z, eps, mode="error")
    # numerical optimum of the continuous problem of Eq. 9 in y = log2(Delta)
    R = 2.0 * (hi - lo)
    target = (eps * z) ** 2

    def obj(y):
        return -np.sum(P * (y - np.log2(R))) / P.sum()

    def con(y):
        return 1.0 - np.sum(np.exp2(2 * y) * g) / 12.0 / target

    y0 = np.log2(np.asarray(out["delta_cont"])) - 1.0
    res = minimize(obj, y0, constraints=[{"type": "ineq", "fun": con}], method="SLSQP",
                   options={"ftol": 1e-14, "maxiter": 500})
    assert res.success
    assert np.allclose(np.exp2(res.x), out["delta_cont"], rtol=1e-5)
    # the optimum sits on the constraint: E[dz] = (eps z)^2
    d = np.asarray(out["delta_cont"])
    assert abs(np.sum(d * d * g) / 12.0 / target - 1.0) < 1e-12
    # Algorithm 1's bit count
    assert out["bits_paper"] == [max(1, math.ceil(-math.log2(d[h] / R[h]))) for h in range(H)]


@pytest.mark.parametrize("seed", range(6))
def test_memory_bound_lagrange_matches_optimizer(oracle, seed):
    gen = np.random.default_rng(100 + seed)
    H = int(gen.integers(2, 6))
    P, g, lo, hi, z = random_problem(gen, H)
    eps = float(gen.uniform(0.3, 0.7))
    out = oracle.scheme_solve(P, g, lo, hi, z, eps, mode="memory")
    R = 2.0 * (hi - lo)
    B = eps * 32 * P.sum()

    def obj(y):
        return np.sum(np.exp2(2 * y) * g) / 12.0

    def con(y):
        return (B - np.sum(P * (np.log2(R) - y))) / P.sum()

    y0 = np.log2(np.asarray(out["delta_cont"])) + 0.5
    scale = obj(y0)
    res = minimize(lambda y: obj(y) / scale, y0, constraints=[{"type": "ineq", "fun": con}],
                   method="SLSQP", options={"ftol": 1e-15, "maxiter": 1000})
    assert res.success
    assert np.allclose(np.exp2(res.x), out["delta_cont"], rtol=1e-4)


@pytest.mark.parametrize("seed", range(8))
def test_error_bound_exact_integer_equals_bruteforce(oracle, seed):
    gen = np.random.default_rng(200 + seed)
    H = int(gen.integers(1, 5))
    P, g, lo, hi, z = random_problem(gen, H)
    eps = float(10.0 ** gen.uniform(-3, -1))
    exact = oracle.scheme_solve(P, g, lo, hi, z, eps, mode="error", rounding="exact")
    paper = oracle.scheme_solve(P, g, lo, hi, z, eps, mode="error", rounding="paper")
    brute = oracle.scheme_bruteforce(P, g, lo, hi, z, eps, mode="error", frac_lo=-10, frac_hi=45)
    target = (eps * z) ** 2
    assert exact["total_bits"] == brute["total_bits"]
    assert exact["pred_err"] <= target and paper["pred_err"] <= target
    assert paper["total_bits"] >= brute["total_bits"]
    # the ceil solution is at most one bit per variable above the optimum's power-of-two
    # rounding plus the window rounding
    assert paper["total_bits"] <= brute["total_bits"] + 2 * P.sum()


@pytest.mark.parametrize("seed", range(8))
def test_memory_bound_integer_equals_bruteforce(oracle, seed):
    gen = np.random.default_rng(300 + seed)
    H = int(gen.integers(1, 4))
    P, g, lo, hi, z = random_problem(gen, H)
    eps = float(gen.uniform(0.3, 0.7))
    exact = oracle.scheme_solve(P, g, lo, hi, z, eps, mode="memory", rounding="exact")
    greedy = oracle.scheme_solve(P, g, lo, hi, z, eps, mode="memory", rounding="paper")
    brute = oracle.scheme_bruteforce(P, g, lo, hi, z, eps, mode="memory")
    budget = eps * 32 * P.sum()
    assert exact["total_bits"] <= budget and greedy["total_bits"] <= budget
    assert math.isclose(exact["pred_err"], brute["pred_err"], rel_tol=1e-12)
    assert greedy["pred_err"] >= brute["pred_err"] * (1 - 1e-12)


def test_equal_types_get_equal_resolution(oracle):
    # symmetric problem: the Lagrange condition gives one Delta for all types (Eq. 10)
    P = [1000.0] * 3
    g = [2.0] * 3
    out = oracle.scheme_solve(P, g, [0, 0, 0], [1, 1, 1], 5.0, 0.01)
    d = out["delta_cont"]
    assert max(d) == pytest.approx(min(d), rel=1e-15)
    assert d[0] == pytest.approx(math.sqrt(12 * 1000 * (0.05) ** 2 / (2.0 * 3000)), rel=1e-15)


def test_windows_cover_the_widened_range(oracle):
    gen = np.random.default_rng(9)
    for mode in ("error", "memory"):
        P, g, lo, hi, z = random_problem(gen, 4)
        out = oracle.scheme_solve(P, g, lo, hi, z, 0.4 if mode == "memory" else 0.01, mode=mode)
        for h in range(4):
            d = 2.0 ** -out["frac"][h]
            mid, R = (lo[h] + hi[h]) / 2, 2.0 * (hi[h] - lo[h])
            assert out["offset"][h] * d <= mid - R / 2
            assert (out["offset"][h] + 2 ** out["bits"][h] - 1) * d >= mid + R / 2


def test_resolution_never_coarser_than_half_the_range(oracle):
    # Algorithm 1's b_h = ceil(-log2(Delta_h / R_h)) >= 1: a type whose error hardly matters
    # (tiny g_h) still gets a resolution of at most R_h / 2, not Eq. 10's huge Delta_h
    P = [1000.0, 1000.0]
    g = [1.0, 1e-20]
    out = oracle.scheme_solve(P, g, [0.0, -1e-4], [1.0, 1e-4], 1.0, 0.01)
    assert out["delta_cont"][1] > 1e6
    assert out["bits_paper"][1] == 1
    R = 2.0 * 2e-4
    assert 2.0 ** -out["frac"][1] <= R / 2


# ---------------------------------------------------------------------------- options
def test_options_cap_keeps_the_window(oracle):
    # x would need more than 12 bits: held at 12 over (at least) the same window
    P, g, lo, hi = [1000.0, 1000.0], [1e8, 1e-6], [0.0, -1.0], [1.0, 1.0]
    plain = oracle.scheme_solve(P, g, lo, hi, 1.0, 1e-4)
    capped = oracle.scheme_solve(P, g, lo, hi, 1.0, 1e-4, max_bits=12)
    assert plain["bits"][0] > 12 and capped["bits"][0] == 12 and capped["capped_mask"] == 1
    drop = plain["bits"][0] - 12
    assert capped["frac"][0] == plain["frac"][0] - drop
    d = 2.0 ** -capped["frac"][0]
    assert capped["offset"][0] * d <= -0.5 and (capped["offset"][0] + 2 ** 12 - 1) * d >= 1.5  # kappa 2 window
    assert capped["bits"][1] == plain["bits"][1] and capped["frac"][1] == plain["frac"][1]


def test_options_refinement_worked_example(oracle):
    # Two types with equal P; the paper solve gives Delta_1 = Delta_2 = D.  With a bias
    # coefficient on type 0 only, bias^2 + var = (beta0 D0^2/6)^2 + (g0 D0^2 + g1 D1^2)/6 must
    # drop below (eps z)^2 = 1e-4.  Taking g = (1, 1), z = 1, eps = 1e-2: Eq. 10 gives
    # Delta_h = sqrt(12 * 1e-4 / 2) = 0.02449, frac = ceil(-log2 0.02449) = 6 (D = 1/64,
    # var = 2 D^2 / 6 = 8.14e-5 <= 1e-4 without bias).  beta0 = 400: bias = 400 D^2 / 6 =
    # 0.01628, bias^2 = 2.65e-4: too large.  Refining type 0 (frac 7): bias = 4.07e-3,
    # bias^2 = 1.66e-5, var = (D^2/4 + D^2)/6 = 5.09e-5, total 6.75e-5 <= 1e-4: one bit, on
    # type 0 (type 1 would leave the bias untouched).
    res = oracle.scheme_solve([100.0, 100.0], [1.0, 1.0], [-1.0, -1.0], [1.0, 1.0], 1.0, 1e-2, beta=[400.0, 0.0])
    assert res["frac"] == [7, 6] and res["refined"] == 1
    assert res["pred_bias"] == pytest.approx(400.0 * 2.0 ** -14 / 6.0, rel=1e-14)
    assert res["pred_var_dither"] == pytest.approx((2.0 ** -14 + 2.0 ** -12) / 6.0, rel=1e-14)
    assert res["pred_bias"] ** 2 + res["pred_var_dither"] <= 1e-4
    # one fraction bit doubles the code range over the same window
    plain = oracle.scheme_solve([100.0, 100.0], [1.0, 1.0], [-1.0, -1.0], [1.0, 1.0], 1.0, 1e-2)
    assert res["bits"][0] == plain["bits"][0] + 1 and res["offset"][0] == 2 * plain["offset"][0]


def test_options_refinement_is_feasible_and_stops_at_once(oracle):
    gen = np.random.default_rng(8)
    for _ in range(50):
        H = 3
        P = list(gen.integers(100, 10000, H).astype(float))
        g = list(10.0 ** gen.uniform(-2, 2, H))
        beta = list(gen.normal(0, 1, H) * 10.0 ** gen.uniform(1, 4, H))
        lo, hi, z, eps = [-1.0] * H, [1.0] * H, 1.0, 1e-2
        res = oracle.scheme_solve(P, g, lo, hi, z, eps, beta=beta)
        d2 = [2.0 ** (-2 * f) / 6.0 for f in res["frac"]]
        bias = sum(b * d for b, d in zip(beta, d2))
        var = sum(gg * d for gg, d in zip(g, d2))
        assert bias ** 2 + var <= (eps * z) ** 2 or max(res["bits"]) >= 24
        plain = oracle.scheme_solve(P, g, lo, hi, z, eps)
        assert sum(res["frac"]) - sum(plain["frac"]) == res["refined"]
        if res["refined"] > 0:
            # it stopped at once: one fraction bit fewer (undoing any single added bit) fails
            for h in range(H):
                if res["frac"][h] > plain["frac"][h]:
                    f = list(res["frac"])
                    f[h] -= 1
                    d2 = [2.0 ** (-2 * ff) / 6.0 for ff in f]
                    b2 = sum(b * d for b, d in zip(beta, d2))
                    v2 = sum(gg * d for gg, d in zip(g, d2))
                    assert b2 ** 2 + v2 > (eps * z) ** 2 or res["refined"] > 1


def test_options_margin_covers_the_widened_window(oracle):
    P, g, lo, hi = [1000.0, 1000.0, 1000.0], [1.0, 10.0, 1e-3], [0.0, -1.0, -0.1], [1.0, 1.0, 0.1]
    res = oracle.scheme_solve(P, g, lo, hi, 1.0, 1e-2, margins={2: (1, 384.0)})
    plain = oracle.scheme_solve(P, g, lo, hi, 1.0, 1e-2)
    k, L, n = res["frac"][2], res["offset"][2], res["bits"][2]
    assert k == plain["frac"][2]  # resolution kept
    m = 384.0 * 2.0 ** -res["frac"][1]
    want_lo, want_hi = -0.2 - m, 0.2 + m  # kappa 2 window of [-0.1, 0.1], widened by m
    assert L * 2.0 ** -k <= want_lo and (L + 2 ** n - 1) * 2.0 ** -k >= want_hi
    assert (L + 2 ** (n - 1) - 1) * 2.0 ** -k < want_hi  # one bit fewer would not cover it
    assert res["bits"][:2] == plain["bits"][:2]
