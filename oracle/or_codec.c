/*
 * or_codec.c -- oracle: counter-based dither generator, fixed-point codec and the
 * bit pack / bit struct placement.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 * The OpenMP pragmas only matter in the threaded build used for full-size reference runs
 * (particles are independent there); the default build ignores them.
 */
#include "oracle.h"

#include <math.h>
#include <stdint.h>
#include <string.h>

/* ------------------------------------------------------------------------------------
 * Philox4x32-R (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy as
 * 1, 2, 3", SC 2011).  R rounds of the 4x32 Philox S-box; between rounds the two key
 * words are bumped by the Weyl constants (golden ratio, sqrt(3)-1 in 32-bit).  The
 * published known answers are for R = 10; the authors report that R = 7 already passes
 * their Crush batteries, and the dither draws use R = 7 (OR_DITHER_ROUNDS).
 * ---------------------------------------------------------------------------------- */
void or_philox4x32(const uint32_t ctr[4], const uint32_t key[2], int rounds, uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < rounds; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    or_philox4x32(ctr, key, 10, out);
}

/* The dither threshold of Sec. 5 for one stored component, compared with the 32-bit
 * fraction f of the value (round up when f > r).  A 16-bit uniform draw q is taken from the
 * Philox4x32-7 block with counter (slot, step, comp / 8, 0) and key = the 64-bit scene seed:
 * the low (comp even) or high (comp odd) half of word (comp / 2) % 4, so one call serves
 * eight consecutive components.  The threshold sits in the middle of q's bucket of 2^16
 * fractions, r = q 2^16 + 2^15, so P(round up) is the fraction rounded to 16 bits: exact
 * to 2^-17, and zero-mean over the fraction. */
uint32_t or_dither_draw(uint64_t seed, uint32_t slot, uint32_t step, int comp)
{
    uint32_t ctr[4] = {slot, step, (uint32_t)(comp >> 3), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32(ctr, key, OR_DITHER_ROUNDS, out);
    const uint32_t w = out[(comp >> 1) & 3];
    const uint32_t q = (comp & 1) ? (w >> 16) : (w & 0xFFFFu);
    return (q << 16) | 0x8000u;
}

/* ------------------------------------------------------------------------------------
 * Fixed-point encode (Sec. 3.1 Eq. 3, Sec. 5 Eq. 11).
 *
 * The resolution is Delta = 2^-frac and the stored integer u in [0, 2^bits) represents
 * (u + offset) * Delta.  With t = v / Delta, I = floor(t) and the fraction Y = t - I
 * truncated to 32 bits, f = floor(Y * 2^32):
 *   round to nearest (Eq. 3, ties up):  up = [f >= 2^31]
 *   dithered (Eq. 11):                   up = [f > r],  r uniform in [0, 2^32)
 * so that the probability of rounding up is Y (Sec. 5), to 2^-32.  Then
 * u = I - offset + up, clamped to [0, 2^bits - 1]; a clamp is a saturation.
 * NaN saturates to u = 0.
 * ---------------------------------------------------------------------------------- */
uint32_t or_encode(double v, int bits, int frac, int64_t offset, int dither, uint32_t r,
                   int *flags)
{
    const int64_t umax = (bits >= 32) ? (int64_t)0xFFFFFFFFu : (((int64_t)1 << bits) - 1);
    const double t = ldexp(v, frac);
    *flags = 0;
    if (isnan(t)) {
        *flags = OR_FLAG_SAT;
        return 0u;
    }
    /* far outside the window the clamp is decided without forming floor(t) */
    if (t < (double)offset - 1.0) {
        *flags = OR_FLAG_SAT;
        return 0u;
    }
    if (t >= (double)offset + (double)umax + 1.0) {
        *flags = OR_FLAG_SAT;
        return (uint32_t)umax;
    }
    const double I = floor(t);
    const double Y = t - I;                         /* exact */
    const uint64_t f = (uint64_t)floor(ldexp(Y, 32)); /* < 2^32 */
    int up;
    if (dither)
        up = f > (uint64_t)r;
    else
        up = f >= (uint64_t)0x80000000u;
    int64_t u = (int64_t)I - offset + up;
    if (u < 0) {
        *flags = OR_FLAG_SAT;
        return 0u;
    }
    if (u > umax) {
        *flags = OR_FLAG_SAT;
        return (uint32_t)umax;
    }
    if (up)
        *flags = OR_FLAG_UP;
    else if (f != 0)
        *flags = OR_FLAG_DOWN;
    return (uint32_t)u;
}

/* Decode phi^{-1}(u) = (u + offset) * Delta: lossless in FP64 (Sec. 3.1). */
double or_decode(uint32_t u, int frac, int64_t offset)
{
    return ldexp((double)((int64_t)u + offset), -frac);
}

/* ------------------------------------------------------------------------------------
 * Component bookkeeping: x[d], v[d], C[d*d], then F[d*d] or J.
 * ---------------------------------------------------------------------------------- */
int or_n_comp(int dim, int material)
{
    return 2 * dim + dim * dim + (material == OR_FLUID ? 1 : dim * dim);
}

int or_comp_field(int dim, int material, int comp)
{
    (void)material;
    if (comp < dim) return OR_FIELD_X;
    if (comp < 2 * dim) return OR_FIELD_V;
    if (comp < 2 * dim + dim * dim) return OR_FIELD_C;
    return OR_FIELD_F;
}

/* ------------------------------------------------------------------------------------
 * Placement (Sec. 7).  Fields are placed in canonical order.
 *   container 0  (bit pack): components follow each other bit by bit and may straddle
 *                a 32-bit word boundary (Fig. 7); consecutive bit-pack fields form one
 *                stream.
 *   container 32/64 (bit struct): a field starts a new container at a 32-bit boundary;
 *                components fill the container in order and never cross it; a component
 *                that does not fit opens the next container (Fig. 6).  A field's last
 *                container is occupied in full.
 * ---------------------------------------------------------------------------------- */
int or_layout(int dim, int material, const int *bits, const int container[4], int *bitpos,
              int *n_words)
{
    const int nc = or_n_comp(dim, material);
    int64_t pos = 0;
    int c = 0;
    for (int h = 0; h < 4; ++h) {
        int c_end = c;
        while (c_end < nc && or_comp_field(dim, material, c_end) == h) ++c_end;
        if (container[h] == 0) {
            for (; c < c_end; ++c) {
                if (bits[c] < 1 || bits[c] > 32) return -1;
                bitpos[c] = (int)pos;
                pos += bits[c];
            }
        } else if (container[h] == 32 || container[h] == 64) {
            const int cw = container[h];
            int64_t cstart = (pos + 31) / 32 * 32;
            int used = 0;
            for (; c < c_end; ++c) {
                if (bits[c] < 1 || bits[c] > 32) return -1;
                if (used + bits[c] > cw) {
                    cstart += cw;
                    used = 0;
                }
                bitpos[c] = (int)(cstart + used);
                used += bits[c];
            }
            pos = cstart + cw;
        } else {
            return -1;
        }
    }
    *n_words = (int)((pos + 31) / 32);
    return 0;
}

static uint32_t or_mask(int bits)
{
    return bits >= 32 ? 0xFFFFFFFFu : ((1u << bits) - 1u);
}

void or_pack(int n_comp, const int *bits, const int *bitpos, int n_words, const uint32_t *u,
             uint32_t *words)
{
    memset(words, 0, sizeof(uint32_t) * (size_t)n_words);
    for (int c = 0; c < n_comp; ++c) {
        const uint32_t val = u[c] & or_mask(bits[c]);
        const int w = bitpos[c] >> 5, s = bitpos[c] & 31;
        words[w] |= val << s;
        if (s + bits[c] > 32) words[w + 1] |= val >> (32 - s);
    }
}

void or_unpack(int n_comp, const int *bits, const int *bitpos, const uint32_t *words,
               uint32_t *u)
{
    for (int c = 0; c < n_comp; ++c) {
        const int w = bitpos[c] >> 5, s = bitpos[c] & 31;
        uint32_t val = words[w] >> s;
        if (s + bits[c] > 32) val |= words[w + 1] << (32 - s);
        u[c] = val & or_mask(bits[c]);
    }
}

/* ------------------------------------------------------------------------------------
 * Whole-state encode / decode.  The dither counter of particle slot p at step `step`
 * is (p, step, comp); the initial state is encoded with step 0 and the store of the
 * step that produces state t+1 uses step t+1.
 * ---------------------------------------------------------------------------------- */
void or_encode_state(const or_codec_t *cd, int64_t N, const double *s, uint32_t step,
                     uint32_t *words, int64_t *stats)
{
    const int nc = cd->n_comp;
    int64_t acc[OR_N_STATS] = {0};
#pragma omp parallel for schedule(static) reduction(+ : acc[:OR_N_STATS])
    for (int64_t p = 0; p < N; ++p) {
        uint32_t u[OR_MAX_COMP];
        for (int c = 0; c < nc; ++c) {
            uint32_t r = cd->dither ? or_dither_draw(cd->seed, (uint32_t)p, step, c) : 0u;
            int flags = 0;
            u[c] = or_encode(s[p * nc + c], cd->bits[c], cd->frac[c], cd->offset[c],
                             cd->dither, r, &flags);
            const int h = cd->field[c];
            if (flags & OR_FLAG_SAT) acc[OR_STAT_SAT(h)] += 1;
            if (flags & OR_FLAG_UP) acc[OR_STAT_UP(h)] += 1;
            if (flags & OR_FLAG_DOWN) acc[OR_STAT_DOWN(h)] += 1;
        }
        or_pack(nc, cd->bits, cd->bitpos, cd->n_words, u, words + p * cd->n_words);
    }
    if (stats)
        for (int i = 0; i < OR_N_STATS; ++i) stats[i] += acc[i];
}

void or_decode_state(const or_codec_t *cd, int64_t N, const uint32_t *words, double *s)
{
    const int nc = cd->n_comp;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        uint32_t u[OR_MAX_COMP];
        or_unpack(nc, cd->bits, cd->bitpos, words + p * cd->n_words, u);
        for (int c = 0; c < nc; ++c)
            s[p * nc + c] = or_decode(u[c], cd->frac[c], cd->offset[c]);
    }
}
