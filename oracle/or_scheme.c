/*
 * or_scheme.c -- oracle: the bit-allocation solve of Sec. 4 and Algorithm 1, plus a
 * brute-force enumeration used to check it.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Error bound (Eq. 6, 9): minimise sum_h P_h b_h  s.t.  (1/12) sum_h Delta_h^2 g_h < (eps z)^2,
 *   Lagrange optimum (Eq. 10): Delta_h = sqrt(12 P_h (eps z)^2 / (g_h sum_h P_h)),
 *   Algorithm 1: b_h = ceil(-log2(Delta_h / R_h)).
 * Memory bound (Eq. 7): minimise (1/12) sum_h Delta_h^2 g_h  s.t.  sum_h P_h b_h <= eps M,
 *   with M = 32 sum_h P_h bits.  Stationarity gives Delta_h^2 g_h = c P_h, and the budget
 *   sum_h P_h log2(R_h / Delta_h) = B fixes
 *   log2 c = (2 sum P log2 R - sum P log2(P / g) - 2B) / sum P.
 * Ranges: the recorded [lo, hi] widened by the factor kappa about its midpoint (Sec. 3.1).
 * Power-of-two resolution: Delta_h = 2^-frac_h; the integer window starts at
 * L = floor(lo' 2^frac) and needs n bits with L + 2^n - 1 >= ceil(hi' 2^frac).
 */
#include "oracle.h"

#include <math.h>
#include <string.h>

static void window(const or_solve_in_t *in, int h, double *lo, double *hi, double *R)
{
    const double mid = 0.5 * (in->lo[h] + in->hi[h]);
    double r = in->kappa * (in->hi[h] - in->lo[h]);
    if (!(r > 0.0)) r = ldexp(1.0, -30);
    *R = r;
    *lo = mid - 0.5 * r;
    *hi = mid + 0.5 * r;
}

static int bits_for_frac(int k, double lo, double hi)
{
    const double L = floor(ldexp(lo, k));
    const double top = ceil(ldexp(hi, k));
    const double span = top - L;
    int n = 1;
    while (n < 64 && ldexp(1.0, n) < span + 1.0) ++n;
    return n;
}

static int64_t offset_for_frac(int k, double lo)
{
    return (int64_t)floor(ldexp(lo, k));
}

static int frac_for_bits(int n, double lo, double hi)
{
    int k = (int)floor((double)n - log2(hi - lo)) + 4;
    while (k > -200 && bits_for_frac(k, lo, hi) > n) --k;
    return k;
}

static double err_of(const or_solve_in_t *in, const int *frac)
{
    double e = 0.0;
    for (int h = 0; h < in->H; ++h) e += ldexp(1.0, -2 * frac[h]) * in->g[h];
    return e / 12.0;
}

static void finish(const or_solve_in_t *in, const int *frac, const int *bits, or_solve_out_t *out)
{
    double tb = 0.0;
    for (int h = 0; h < in->H; ++h) {
        double lo, hi, R;
        window(in, h, &lo, &hi, &R);
        out->frac[h] = frac[h];
        out->bits[h] = bits[h];
        out->offset[h] = offset_for_frac(frac[h], lo);
        tb += in->P[h] * (double)bits[h];
    }
    out->pred_err = err_of(in, frac);
    out->total_bits = tb;
}

int or_scheme_solve(const or_solve_in_t *in, or_solve_out_t *out)
{
    const int H = in->H;
    if (H < 1 || H > 8) return -1;
    memset(out, 0, sizeof(*out));
    double SP = 0.0;
    for (int h = 0; h < H; ++h) SP += in->P[h];
    double lo[8], hi[8], R[8];
    for (int h = 0; h < H; ++h) window(in, h, &lo[h], &hi[h], &R[h]);
    int frac[8], bits[8];

    if (in->mode == 0) {
        const double target = (in->eps * in->z) * (in->eps * in->z);
        int frac0[8], fixed[8];
        for (int h = 0; h < H; ++h) {
            fixed[h] = 0;
            if (in->g[h] > 0.0) {
                const double d = sqrt(12.0 * in->P[h] * target / (in->g[h] * SP));
                out->delta_cont[h] = d;
                out->bits_paper[h] = (int)ceil(-log2(d / R[h]));
                if (out->bits_paper[h] < 1) out->bits_paper[h] = 1;
                /* b_h >= 1 bounds the resolution by half the widened range */
                frac0[h] = (int)ceil(-log2(fmin(d, 0.5 * R[h])));
            } else {
                out->delta_cont[h] = INFINITY;
                out->bits_paper[h] = 1;
                frac0[h] = frac_for_bits(1, lo[h], hi[h]);
                fixed[h] = 1;
            }
        }
        if (in->rounding == 0) {
            for (int h = 0; h < H; ++h) {
                frac[h] = frac0[h];
                bits[h] = bits_for_frac(frac[h], lo[h], hi[h]);
            }
            finish(in, frac, bits, out);
            return 0;
        }
        /* exact integer search around the ceil solution */
        int best_frac[8];
        double best_bits = INFINITY, best_err = INFINITY;
        int cur[8];
        for (int h = 0; h < H; ++h) cur[h] = fixed[h] ? frac0[h] : frac0[h] - 3;
        for (;;) {
            const double e = err_of(in, cur);
            if (e <= target) {
                double tb = 0.0;
                for (int h = 0; h < H; ++h) tb += in->P[h] * bits_for_frac(cur[h], lo[h], hi[h]);
                if (tb < best_bits || (tb == best_bits && e < best_err)) {
                    best_bits = tb;
                    best_err = e;
                    memcpy(best_frac, cur, sizeof(cur));
                }
            }
            int h = 0;
            while (h < H) {
                if (!fixed[h] && cur[h] < frac0[h] + 3) { ++cur[h]; break; }
                cur[h] = fixed[h] ? frac0[h] : frac0[h] - 3;
                ++h;
            }
            if (h == H) break;
        }
        if (best_bits == INFINITY) return -2;
        for (int h = 0; h < H; ++h) {
            frac[h] = best_frac[h];
            bits[h] = bits_for_frac(frac[h], lo[h], hi[h]);
        }
        finish(in, frac, bits, out);
        return 0;
    }

    /* memory bound */
    double B = in->eps * 32.0 * SP;
    double SPg = 0.0, s1 = 0.0, s2 = 0.0;
    for (int h = 0; h < H; ++h) {
        if (in->g[h] > 0.0) {
            SPg += in->P[h];
            s1 += in->P[h] * log2(R[h]);
            s2 += in->P[h] * log2(in->P[h] / in->g[h]);
        } else {
            B -= in->P[h];
        }
    }
    double bcont[8];
    const double log2c = SPg > 0.0 ? (2.0 * s1 - s2 - 2.0 * B) / SPg : 0.0;
    for (int h = 0; h < H; ++h) {
        if (in->g[h] > 0.0) {
            const double d = sqrt(exp2(log2c) * in->P[h] / in->g[h]);
            out->delta_cont[h] = d;
            bcont[h] = log2(R[h] / d);
        } else {
            out->delta_cont[h] = INFINITY;
            bcont[h] = 1.0;
        }
        int b = (int)floor(bcont[h]);
        if (b < 1) b = 1;
        out->bits_paper[h] = b;
    }
    const double budget = in->eps * 32.0 * SP;
    if (in->rounding == 0) {
        double tb = 0.0;
        for (int h = 0; h < H; ++h) {
            bits[h] = out->bits_paper[h];
            tb += in->P[h] * bits[h];
        }
        for (;;) {
            int pick = -1;
            double best = 0.0;
            for (int h = 0; h < H; ++h) {
                if (in->g[h] <= 0.0 || bits[h] >= 32 || tb + in->P[h] > budget) continue;
                const int f0 = frac_for_bits(bits[h], lo[h], hi[h]);
                const int f1 = frac_for_bits(bits[h] + 1, lo[h], hi[h]);
                const double gain = (ldexp(1.0, -2 * f0) - ldexp(1.0, -2 * f1)) * in->g[h] / 12.0 / in->P[h];
                if (gain > best) { best = gain; pick = h; }
            }
            if (pick < 0) break;
            bits[pick] += 1;
            tb += in->P[pick];
        }
    } else {
        int cur[8], lo_b[8], hi_b[8], best_b[8];
        double best_err = INFINITY, best_tb = INFINITY;
        for (int h = 0; h < H; ++h) {
            lo_b[h] = out->bits_paper[h] - 3; if (lo_b[h] < 1) lo_b[h] = 1;
            hi_b[h] = out->bits_paper[h] + 3; if (hi_b[h] > 32) hi_b[h] = 32;
            if (in->g[h] <= 0.0) lo_b[h] = hi_b[h] = 1;
            cur[h] = lo_b[h];
        }
        for (;;) {
            double tb = 0.0;
            int fr[8];
            for (int h = 0; h < H; ++h) {
                tb += in->P[h] * cur[h];
                fr[h] = frac_for_bits(cur[h], lo[h], hi[h]);
            }
            if (tb <= budget) {
                const double e = err_of(in, fr);
                if (e < best_err || (e == best_err && tb < best_tb)) {
                    best_err = e;
                    best_tb = tb;
                    memcpy(best_b, cur, sizeof(cur));
                }
            }
            int h = 0;
            while (h < H) {
                if (cur[h] < hi_b[h]) { ++cur[h]; break; }
                cur[h] = lo_b[h];
                ++h;
            }
            if (h == H) break;
        }
        if (best_err == INFINITY) return -2;
        memcpy(bits, best_b, sizeof(int) * (size_t)H);
    }
    for (int h = 0; h < H; ++h) frac[h] = frac_for_bits(bits[h], lo[h], hi[h]);
    finish(in, frac, bits, out);
    return 0;
}

/* Exhaustive enumeration (H <= 4).  Error mode: frac_h over [frac_lo, frac_hi], minimum
 * total bits subject to the error bound (ties: smaller error).  Memory mode: bits_h over
 * [1, 32], minimum error subject to the budget (ties: fewer bits). */
int or_scheme_bruteforce(const or_solve_in_t *in, int frac_lo, int frac_hi, or_solve_out_t *out)
{
    const int H = in->H;
    if (H < 1 || H > 4) return -1;
    memset(out, 0, sizeof(*out));
    double lo[4], hi[4], R[4], SP = 0.0;
    for (int h = 0; h < H; ++h) {
        window(in, h, &lo[h], &hi[h], &R[h]);
        SP += in->P[h];
    }
    int cur[4], best[4], frac[4], bits[4];
    double best_a = INFINITY, best_b = INFINITY;
    const int mlo = in->mode == 0 ? frac_lo : 1, mhi = in->mode == 0 ? frac_hi : 32;
    for (int h = 0; h < H; ++h) cur[h] = mlo;
    const double target = (in->eps * in->z) * (in->eps * in->z);
    const double budget = in->eps * 32.0 * SP;
    for (;;) {
        double tb = 0.0;
        int fr[4];
        for (int h = 0; h < H; ++h) {
            if (in->mode == 0) {
                fr[h] = cur[h];
                tb += in->P[h] * bits_for_frac(cur[h], lo[h], hi[h]);
            } else {
                fr[h] = frac_for_bits(cur[h], lo[h], hi[h]);
                tb += in->P[h] * cur[h];
            }
        }
        const double e = err_of(in, fr);
        if (in->mode == 0) {
            if (e <= target && (tb < best_a || (tb == best_a && e < best_b))) {
                best_a = tb; best_b = e; memcpy(best, cur, sizeof(cur));
            }
        } else {
            if (tb <= budget && (e < best_a || (e == best_a && tb < best_b))) {
                best_a = e; best_b = tb; memcpy(best, cur, sizeof(cur));
            }
        }
        int h = 0;
        while (h < H) {
            if (cur[h] < mhi) { ++cur[h]; break; }
            cur[h] = mlo;
            ++h;
        }
        if (h == H) break;
    }
    if (best_a == INFINITY) return -2;
    for (int h = 0; h < H; ++h) {
        if (in->mode == 0) {
            frac[h] = best[h];
            bits[h] = bits_for_frac(best[h], lo[h], hi[h]);
        } else {
            bits[h] = best[h];
            frac[h] = frac_for_bits(best[h], lo[h], hi[h]);
        }
    }
    finish(in, frac, bits, out);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Options on a solved scheme (see oracle.h): the cap, the second-order refinement (the
 * bound of Eq. 6 on the second moment with the shift that Eq. 8's linear term leaves
 * out, for dithered stores of variance Delta^2 / 6) and widened windows.
 * ---------------------------------------------------------------------------------- */
static double sq_moment(const or_solve_in_t *in, const double *beta, const int *frac, double *bias, double *var)
{
    double b = 0.0, v = 0.0;
    for (int h = 0; h < in->H; ++h) {
        const double d2 = pow(2.0, -2.0 * frac[h]) / 6.0;
        b += beta[h] * d2;
        v += in->g[h] * d2;
    }
    if (bias) *bias = b;
    if (var) *var = v;
    return b * b + v;
}

int or_scheme_options(const or_solve_in_t *in, const or_solve_opt_t *opt, or_solve_out_t *out)
{
    const int H = in->H;
    int frac[8], bits[8];
    int64_t off[8];
    for (int h = 0; h < H; ++h) {
        frac[h] = out->frac[h];
        bits[h] = out->bits[h];
        off[h] = out->offset[h];
    }
    out->capped = 0;
    out->refined = 0;
    if (opt->max_bits > 0) {
        for (int h = 0; h < H; ++h) {
            while (bits[h] > opt->max_bits) {
                /* one bit fewer over the same window: half the resolution */
                bits[h] -= 1;
                frac[h] -= 1;
                off[h] = (int64_t)floor((double)off[h] / 2.0);
                out->capped |= 1 << h;
            }
        }
    }
    const int top = opt->max_bits > 0 ? opt->max_bits : 24;
    if (opt->refine && in->mode == 0) {
        const double target = (in->eps * in->z) * (in->eps * in->z);
        while (out->refined < 64) {
            const double now = sq_moment(in, opt->beta, frac, NULL, NULL);
            if (now <= target) break;
            int best = -1;
            double best_drop = 0.0;
            for (int h = 0; h < H; ++h) {
                if (bits[h] >= top) continue;
                frac[h] += 1;
                const double drop = (now - sq_moment(in, opt->beta, frac, NULL, NULL)) / in->P[h];
                frac[h] -= 1;
                if (drop > best_drop) {
                    best_drop = drop;
                    best = h;
                }
            }
            if (best >= 0) {
                frac[best] += 1;
                bits[best] += 1;
                off[best] = 2 * off[best];
                out->refined += 1;
                continue;
            }
            /* biases of opposite signs: no single bit helps, every type gets one (both
             * moments fall by 4) */
            int moved = 0;
            for (int h = 0; h < H; ++h) {
                if (bits[h] >= top) continue;
                frac[h] += 1;
                bits[h] += 1;
                off[h] = 2 * off[h];
                out->refined += 1;
                moved = 1;
            }
            if (!moved) break;
        }
    }
    for (int h = 0; h < H; ++h) {
        if (!(opt->margin_gain[h] > 0.0)) continue;
        const int src = opt->margin_src[h];
        if (src < 0 || src >= H) return -1;
        double lo, hi, R;
        window(in, h, &lo, &hi, &R);
        const double m = opt->margin_gain[h] * pow(2.0, -frac[src]);
        lo -= m;
        hi += m;
        int k = frac[h];
        while (opt->max_bits > 0 && bits_for_frac(k, lo, hi) > opt->max_bits) {
            --k;
            out->capped |= 1 << h;
        }
        frac[h] = k;
        bits[h] = bits_for_frac(k, lo, hi);
        off[h] = offset_for_frac(k, lo);
    }
    double tb = 0.0;
    for (int h = 0; h < H; ++h) {
        out->frac[h] = frac[h];
        out->bits[h] = bits[h];
        out->offset[h] = off[h];
        tb += in->P[h] * (double)bits[h];
    }
    out->total_bits = tb;
    out->pred_err = err_of(in, frac);
    sq_moment(in, opt->beta, frac, &out->pred_bias, &out->pred_var_dither);
    return 0;
}
