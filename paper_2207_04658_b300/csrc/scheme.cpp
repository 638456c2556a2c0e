// scheme.cpp -- host side of libqmpm: record layout (bit pack / bit struct, Sec. 7),
// per-component codec constants, and the bit-allocation solve (Sec. 4, Algorithm 1).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "qmpm_internal.h"

namespace qmpm {

int n_comp(int dim, int material)
{
    return 2 * dim + dim * dim + (material == QMPM_FLUID ? 1 : dim * dim);
}

int comp_field(int dim, int comp)
{
    if (comp < dim) return QMPM_FIELD_X;
    if (comp < 2 * dim) return QMPM_FIELD_V;
    if (comp < 2 * dim + dim * dim) return QMPM_FIELD_C;
    return QMPM_FIELD_F;
}

int layout(int dim, int material, qmpm_scheme_t *s, std::string &err)
{
    if ((dim != 2 && dim != 3) || material < 0 || material > 2) {
        err = "dim must be 2 or 3 and material 0..2";
        return QMPM_ERR_INVALID_ARG;
    }
    const int nc = n_comp(dim, material);
    if (!s->quantized) {
        s->n_words = nc;
        for (int c = 0; c < nc; ++c) s->bitpos[c] = 32 * c;
        return QMPM_OK;
    }
    for (int h = 0; h < 4; ++h) {
        const qmpm_field_t &f = s->field[h];
        if (f.bits < 1 || f.bits > QMPM_MAX_FIELD_BITS) {
            err = "field " + std::to_string(h) + ": bits must be in 1..24 for FP32 compute";
            return QMPM_ERR_SCHEME;
        }
        if (f.offset <= -(int64_t(1) << 24) || f.offset >= (int64_t(1) << 24)) {
            err = "field " + std::to_string(h) + ": |offset| must be below 2^24";
            return QMPM_ERR_SCHEME;
        }
        if (f.frac < -100 || f.frac > 100) {
            err = "field " + std::to_string(h) + ": frac out of range";
            return QMPM_ERR_SCHEME;
        }
        if (f.container != 0 && f.container != 32 && f.container != 64) {
            err = "field " + std::to_string(h) + ": container must be 0, 32 or 64";
            return QMPM_ERR_SCHEME;
        }
    }
    int64_t cursor = 0;  // next free record bit
    int c = 0;
    for (int h = 0; h < 4; ++h) {
        const int bits = s->field[h].bits;
        const int cw = s->field[h].container;
        int last = c;
        while (last < nc && comp_field(dim, last) == h) ++last;
        if (cw == 0) {
            // bit pack: the stream simply continues
            for (; c < last; ++c) {
                s->bitpos[c] = (int32_t)cursor;
                cursor += bits;
            }
        } else {
            // bit struct: fill containers of cw bits starting on a word boundary
            int64_t box = (cursor + 31) & ~int64_t(31);
            int fill = 0;
            for (; c < last; ++c) {
                if (fill + bits > cw) {
                    box += cw;
                    fill = 0;
                }
                s->bitpos[c] = (int32_t)(box + fill);
                fill += bits;
            }
            cursor = box + cw;
        }
    }
    s->n_words = (int32_t)((cursor + 31) / 32);
    return QMPM_OK;
}

void build_codec(const qmpm_scheme_t &s, int dim, int material, CompCodec *cc)
{
    const int nc = n_comp(dim, material);
    for (int c = 0; c < nc; ++c) {
        CompCodec &k = cc[c];
        const int h = comp_field(dim, c);
        k.field = h;
        if (!s.quantized) {
            k.word = c;
            k.shift = 0;
            k.straddle = 0;
            k.mask = 0xFFFFFFFFu;
            k.offset = 0;
            k.umax = 0xFFFFFFFFu;
            k.enc_scale = k.dec_scale = 1.0f;
            k.dec_bias = 0.0f;
            continue;
        }
        const qmpm_field_t &f = s.field[h];
        k.word = s.bitpos[c] >> 5;
        k.shift = s.bitpos[c] & 31;
        k.straddle = (k.shift + f.bits > 32) ? 1 : 0;
        k.mask = (f.bits >= 32) ? 0xFFFFFFFFu : ((1u << f.bits) - 1u);
        k.offset = (int32_t)f.offset;
        k.umax = k.mask;
        k.enc_scale = std::ldexp(1.0f, f.frac);
        k.dec_scale = std::ldexp(1.0f, -f.frac);
        k.dec_bias = (float)std::ldexp((double)f.offset, -f.frac);
    }
}

// ---------------------------------------------------------------------------------
// Bit-allocation solve.  R_h = kappa (hi - lo), the window [mid - R/2, mid + R/2].
// With resolution 2^-k the window needs L = floor(lo' 2^k) and the fewest n such that
// 2^n - 1 >= ceil(hi' 2^k) - L.
// ---------------------------------------------------------------------------------
namespace {

struct Window {
    double lo, hi, R;
};

Window window_of(const qmpm_solve_in_t &in, int h)
{
    const double mid = 0.5 * (in.lo[h] + in.hi[h]);
    double R = in.kappa * (in.hi[h] - in.lo[h]);
    if (!(R > 0.0)) R = std::ldexp(1.0, -30);
    return {mid - 0.5 * R, mid + 0.5 * R, R};
}

int bits_at(int k, const Window &w)
{
    const double L = std::floor(std::ldexp(w.lo, k));
    const double need = std::ceil(std::ldexp(w.hi, k)) - L + 1.0;
    int n = 1;
    while (n < 64 && std::ldexp(1.0, n) < need) ++n;
    return n;
}

int finest_frac(int n, const Window &w)
{
    int k = (int)std::floor((double)n - std::log2(w.hi - w.lo)) + 4;
    while (k > -200 && bits_at(k, w) > n) --k;
    return k;
}

double predicted(const qmpm_solve_in_t &in, const int *frac)
{
    double e = 0.0;
    for (int h = 0; h < in.H; ++h) e += std::ldexp(1.0, -2 * frac[h]) * in.g[h];
    return e / 12.0;
}

// floor(v / 2^k) for any sign (an arithmetic shift)
int64_t floor_shift(int64_t v, int k)
{
    return v >= 0 ? (v >> k) : -((-v + (int64_t(1) << k) - 1) >> k);
}

// Visit every integer vector v with lo[h] <= v[h] <= hi[h].
template <class F>
void odometer(int H, const int *lo, const int *hi, F &&visit)
{
    int v[8];
    for (int h = 0; h < H; ++h) v[h] = lo[h];
    for (;;) {
        visit(v);
        int h = 0;
        for (; h < H; ++h) {
            if (v[h] < hi[h]) {
                ++v[h];
                break;
            }
            v[h] = lo[h];
        }
        if (h == H) return;
    }
}

}  // namespace

}  // namespace qmpm

using namespace qmpm;

extern "C" int qmpm_scheme_solve_impl(const qmpm_solve_in_t *in, qmpm_solve_out_t *out, std::string &err)
{
    if (!in || !out || in->H < 1 || in->H > 8 || !(in->eps > 0.0)) {
        err = "qmpm_scheme_solve: need 1 <= H <= 8 and eps > 0";
        return QMPM_ERR_INVALID_ARG;
    }
    if (in->max_bits < 0 || in->max_bits > 64) {
        err = "qmpm_scheme_solve: max_bits must be in 0..64";
        return QMPM_ERR_INVALID_ARG;
    }
    for (int h = 0; h < in->H; ++h)
        if (in->margin_gain[h] > 0.0 && (in->margin_src[h] < 0 || in->margin_src[h] >= in->H)) {
            err = "qmpm_scheme_solve: margin_src names no type";
            return QMPM_ERR_INVALID_ARG;
        }
    std::memset(out, 0, sizeof(*out));
    const int H = in->H;
    std::array<Window, 8> win{};
    double sumP = 0.0;
    for (int h = 0; h < H; ++h) {
        win[h] = window_of(*in, h);
        sumP += in->P[h];
    }
    int frac[8], bits[8];

    if (in->mode == 0) {
        // Eq. 10 and Algorithm 1
        const double bound = (in->eps * in->z) * (in->eps * in->z);
        int k0[8], lo[8], hi[8];
        for (int h = 0; h < H; ++h) {
            if (in->g[h] > 0.0) {
                const double d = std::sqrt(12.0 * in->P[h] * bound / (in->g[h] * sumP));
                out->delta_cont[h] = d;
                out->bits_paper[h] = std::max(1, (int)std::ceil(-std::log2(d / win[h].R)));
                // at least one bit (Algorithm 1): the resolution is at most half the range
                k0[h] = (int)std::ceil(-std::log2(std::min(d, 0.5 * win[h].R)));
                lo[h] = k0[h] - 3;
                hi[h] = k0[h] + 3;
            } else {
                out->delta_cont[h] = std::numeric_limits<double>::infinity();
                out->bits_paper[h] = 1;
                k0[h] = lo[h] = hi[h] = finest_frac(1, win[h]);
            }
        }
        if (in->rounding == 0) {
            std::copy(k0, k0 + H, frac);
        } else {
            double best_bits = std::numeric_limits<double>::infinity(), best_err = best_bits;
            int best[8];
            odometer(H, lo, hi, [&](const int *v) {
                const double e = predicted(*in, v);
                if (e > bound) return;
                double tb = 0.0;
                for (int h = 0; h < H; ++h) tb += in->P[h] * bits_at(v[h], win[h]);
                if (tb < best_bits || (tb == best_bits && e < best_err)) {
                    best_bits = tb;
                    best_err = e;
                    std::copy(v, v + H, best);
                }
            });
            if (best_bits == std::numeric_limits<double>::infinity()) {
                err = "qmpm_scheme_solve: no feasible scheme in the search window";
                return QMPM_ERR_SCHEME;
            }
            std::copy(best, best + H, frac);
        }
        for (int h = 0; h < H; ++h) bits[h] = bits_at(frac[h], win[h]);
    } else {
        // memory bound: Delta_h^2 g_h = c P_h, c from the bit budget
        const double budget = in->eps * 32.0 * sumP;
        double B = budget, Pg = 0.0, a = 0.0, b = 0.0;
        for (int h = 0; h < H; ++h) {
            if (in->g[h] > 0.0) {
                Pg += in->P[h];
                a += in->P[h] * std::log2(win[h].R);
                b += in->P[h] * std::log2(in->P[h] / in->g[h]);
            } else {
                B -= in->P[h];
            }
        }
        const double log2c = Pg > 0.0 ? (2.0 * a - b - 2.0 * B) / Pg : 0.0;
        for (int h = 0; h < H; ++h) {
            double bc = 1.0;
            if (in->g[h] > 0.0) {
                const double d = std::sqrt(std::exp2(log2c) * in->P[h] / in->g[h]);
                out->delta_cont[h] = d;
                bc = std::log2(win[h].R / d);
            } else {
                out->delta_cont[h] = std::numeric_limits<double>::infinity();
            }
            out->bits_paper[h] = std::max(1, (int)std::floor(bc));
        }
        auto err_at_bits = [&](int h, int n) {
            return std::ldexp(1.0, -2 * finest_frac(n, win[h])) * in->g[h] / 12.0;
        };
        if (in->rounding == 0) {
            double used = 0.0;
            for (int h = 0; h < H; ++h) {
                bits[h] = out->bits_paper[h];
                used += in->P[h] * bits[h];
            }
            for (;;) {
                int pick = -1;
                double gain_best = 0.0;
                for (int h = 0; h < H; ++h) {
                    if (in->g[h] <= 0.0 || bits[h] >= 32 || used + in->P[h] > budget) continue;
                    const double gain = (err_at_bits(h, bits[h]) - err_at_bits(h, bits[h] + 1)) / in->P[h];
                    if (gain > gain_best) {
                        gain_best = gain;
                        pick = h;
                    }
                }
                if (pick < 0) break;
                bits[pick] += 1;
                used += in->P[pick];
            }
        } else {
            int lo[8], hi[8], best[8];
            for (int h = 0; h < H; ++h) {
                lo[h] = std::max(1, out->bits_paper[h] - 3);
                hi[h] = std::min(32, out->bits_paper[h] + 3);
                if (in->g[h] <= 0.0) lo[h] = hi[h] = 1;
            }
            double best_err = std::numeric_limits<double>::infinity(), best_used = best_err;
            odometer(H, lo, hi, [&](const int *v) {
                double used = 0.0, e = 0.0;
                for (int h = 0; h < H; ++h) {
                    used += in->P[h] * v[h];
                    e += err_at_bits(h, v[h]);
                }
                if (used > budget) return;
                if (e < best_err || (e == best_err && used < best_used)) {
                    best_err = e;
                    best_used = used;
                    std::copy(v, v + H, best);
                }
            });
            if (best_err == std::numeric_limits<double>::infinity()) {
                err = "qmpm_scheme_solve: no scheme fits the memory budget";
                return QMPM_ERR_SCHEME;
            }
            std::copy(best, best + H, bits);
        }
        for (int h = 0; h < H; ++h) frac[h] = finest_frac(bits[h], win[h]);
    }
    int64_t offset[8];
    for (int h = 0; h < H; ++h) offset[h] = (int64_t)std::floor(std::ldexp(win[h].lo, frac[h]));
    const int cap = in->max_bits > 0 ? in->max_bits : 0;
    // option 1: hold every type at max_bits, coarser by one power of two per bit dropped
    if (cap > 0)
        for (int h = 0; h < H; ++h)
            if (bits[h] > cap) {
                const int drop = bits[h] - cap;
                frac[h] -= drop;
                offset[h] = floor_shift(offset[h], drop);
                bits[h] = cap;
                out->capped |= 1 << h;
            }
    // option 2: the second-order refinement (error mode)
    auto moments = [&](const int *fr, double &bias, double &var) {
        bias = 0.0;
        var = 0.0;
        for (int h = 0; h < H; ++h) {
            const double d2 = std::ldexp(1.0, -2 * fr[h]) / 6.0;
            bias += in->beta[h] * d2;
            var += in->g[h] * d2;
        }
    };
    if (in->refine && in->mode == 0) {
        const double target = (in->eps * in->z) * (in->eps * in->z);
        const int limit = cap > 0 ? cap : QMPM_MAX_FIELD_BITS;
        for (int it = 0; it < 64; ++it) {
            double b, v;
            moments(frac, b, v);
            if (b * b + v <= target) break;
            int pick = -1;
            double best = 0.0;
            for (int h = 0; h < H; ++h) {
                if (bits[h] >= limit) continue;
                int f2[8];
                std::copy(frac, frac + H, f2);
                f2[h] += 1;
                double b2, v2;
                moments(f2, b2, v2);
                const double gain = (b * b + v - b2 * b2 - v2) / in->P[h];
                if (gain > best) {
                    best = gain;
                    pick = h;
                }
            }
            if (pick >= 0) {
                frac[pick] += 1;
                bits[pick] += 1;
                offset[pick] *= 2;
                out->refined += 1;
                continue;
            }
            // no single bit lowers bias^2 + var (biases of opposite signs cancel): refine
            // every type at once, which divides both moments by 4
            bool any = false;
            for (int h = 0; h < H; ++h) {
                if (bits[h] >= limit) continue;
                frac[h] += 1;
                bits[h] += 1;
                offset[h] *= 2;
                out->refined += 1;
                any = true;
            }
            if (!any) break;
        }
    }
    // option 3: windows widened by another type's noise, at the type's own resolution
    for (int h = 0; h < H; ++h) {
        const int src = in->margin_src[h];
        if (!(in->margin_gain[h] > 0.0) || src < 0 || src >= H) continue;
        const double m = in->margin_gain[h] * std::ldexp(1.0, -frac[src]);
        const Window w{win[h].lo - m, win[h].hi + m, win[h].R + 2.0 * m};
        int k = frac[h];
        int n = bits_at(k, w);
        if (cap > 0 && n > cap) {
            while (n > cap) {
                --k;
                n = bits_at(k, w);
            }
            out->capped |= 1 << h;
        }
        frac[h] = k;
        bits[h] = n;
        offset[h] = (int64_t)std::floor(std::ldexp(w.lo, k));
    }
    double tb = 0.0;
    for (int h = 0; h < H; ++h) {
        out->bits[h] = bits[h];
        out->frac[h] = frac[h];
        out->offset[h] = offset[h];
        tb += in->P[h] * bits[h];
    }
    out->pred_err = predicted(*in, frac);
    out->total_bits = tb;
    moments(frac, out->pred_bias, out->pred_var_dither);
    return QMPM_OK;
}

// ---------------------------------------------------------------------------------
// Edits of one type of a scheme (the second-order refinement and its acceptance check).
// A type's fixed point is its resolution 2^-frac and its window [offset 2^-frac,
// (offset + 2^bits - 1) 2^-frac] (Sec. 3.1); each edit keeps the other types.
// ---------------------------------------------------------------------------------
namespace {

int edit_check(const qmpm_scheme_t *s, int h, const char *what, std::string &err)
{
    if (!s || !s->quantized) {
        err = std::string(what) + ": no quantized scheme";
        return QMPM_ERR_INVALID_ARG;
    }
    if (h < 0 || h > 3) {
        err = std::string(what) + ": type index out of 0..3";
        return QMPM_ERR_INVALID_ARG;
    }
    return QMPM_OK;
}

int field_check(const qmpm_field_t &f, const char *what, std::string &err)
{
    if (f.bits < 1 || f.bits > 24 || f.offset <= -(int64_t(1) << 24) || f.offset >= (int64_t(1) << 24)) {
        err = std::string(what) + ": the edited type leaves 1..24 bits or |offset| < 2^24";
        return QMPM_ERR_SCHEME;
    }
    return QMPM_OK;
}

}  // namespace

extern "C" int qmpm_scheme_shift_impl(qmpm_scheme_t *s, int32_t h, int32_t k, std::string &err)
{
    int rc = edit_check(s, h, "qmpm_scheme_shift", err);
    if (rc != QMPM_OK) return rc;
    qmpm_field_t f = s->field[h];
    f.bits += k;
    f.frac += k;
    f.offset = k >= 0 ? f.offset * (int64_t(1) << std::min(k, 40)) : qmpm::floor_shift(f.offset, -k);
    rc = field_check(f, "qmpm_scheme_shift", err);
    if (rc != QMPM_OK) return rc;
    s->field[h] = f;
    return QMPM_OK;
}

extern "C" int qmpm_scheme_widen_impl(qmpm_scheme_t *s, int32_t h, std::string &err)
{
    int rc = edit_check(s, h, "qmpm_scheme_widen", err);
    if (rc != QMPM_OK) return rc;
    qmpm_field_t f = s->field[h];
    f.offset -= int64_t(1) << (f.bits - 1);
    f.bits += 1;
    rc = field_check(f, "qmpm_scheme_widen", err);
    if (rc != QMPM_OK) return rc;
    s->field[h] = f;
    return QMPM_OK;
}

extern "C" int qmpm_scheme_window_impl(qmpm_scheme_t *s, int32_t h, double lo, double hi, double kappa,
                                       int32_t src, double gain, int32_t grow, std::string &err)
{
    int rc = edit_check(s, h, "qmpm_scheme_window", err);
    if (rc != QMPM_OK) return rc;
    if (!(lo <= hi) || !(kappa > 0.0) || !(gain >= 0.0) || src > 3) {
        err = "qmpm_scheme_window: need lo <= hi, kappa > 0, gain >= 0, src < 4";
        return QMPM_ERR_INVALID_ARG;
    }
    qmpm_field_t f = s->field[h];
    // the solve's window of the recorded range, widened by the margin (its option 3)
    const double mid = 0.5 * (lo + hi);
    double R = kappa * (hi - lo);
    if (!(R > 0.0)) R = std::ldexp(1.0, -30);
    const double m = src >= 0 ? gain * std::ldexp(1.0, -s->field[src].frac) : 0.0;
    qmpm::Window w{mid - 0.5 * R - m, mid + 0.5 * R + m, R + 2.0 * m};
    if (grow) {
        w.lo = std::min(w.lo, std::ldexp((double)f.offset, -f.frac));
        w.hi = std::max(w.hi, std::ldexp((double)(f.offset + (int64_t(1) << f.bits) - 1), -f.frac));
        w.R = w.hi - w.lo;
    }
    f.offset = (int64_t)std::floor(std::ldexp(w.lo, f.frac));
    f.bits = qmpm::bits_at(f.frac, w);
    rc = field_check(f, "qmpm_scheme_window", err);
    if (rc != QMPM_OK) return rc;
    s->field[h] = f;
    return QMPM_OK;
}

extern "C" int qmpm_scheme_fill_words_impl(int32_t dim, int32_t material, qmpm_scheme_t *s, int32_t type_mask,
                                           int32_t *widened, std::string &err)
{
    if (!s || !s->quantized) {
        err = "qmpm_scheme_fill_words: no quantized scheme";
        return QMPM_ERR_INVALID_ARG;
    }
    qmpm_scheme_t cur = *s;
    int rc = qmpm::layout(dim, material, &cur, err);
    if (rc != QMPM_OK) return rc;
    const int32_t words = cur.n_words;
    int n = 0;
    for (bool grew = true; grew;) {
        grew = false;
        for (int h = 0; h < 4; ++h) {
            if (!(type_mask >> h & 1) || cur.field[h].bits >= 24) continue;
            qmpm_scheme_t trial = cur;
            std::string e2;
            if (qmpm_scheme_widen_impl(&trial, h, e2) != QMPM_OK) continue;
            if (qmpm::layout(dim, material, &trial, e2) != QMPM_OK || trial.n_words != words) continue;
            cur = trial;
            grew = true;
            ++n;
        }
    }
    *s = cur;
    if (widened) *widened = n;
    return QMPM_OK;
}
