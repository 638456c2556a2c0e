/*
 * or_smoke.c -- oracle: the 2D Eulerian smoke simulator of the paper's experiments
 * (Sec. 8.1: an advection-reflection solver, semi-Lagrangian advection with RK-3 path
 * integration, 64 Jacobi iterations for the Poisson equation, evaluation = the sum of
 * squared smoke density over the grid, quantized pressure and velocity), in FP64, and its
 * quantized form: every store of a velocity or pressure value goes through the dithered
 * fixed-point codec.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Grid: n x n cells of size h = 1/n; MAC layout: u on vertical faces (n+1 columns x n rows,
 * u[j*(n+1)+i] at (i h, (j+1/2) h)), v on horizontal faces (n columns x n+1 rows, v[j*n+i]
 * at ((i+1/2) h, j h)), density d and pressure q at cell centres ((i+1/2) h, (j+1/2) h).
 * Walls on all four sides: the boundary faces' normal velocity is zero; the pressure has
 * zero normal derivative there.
 *
 * One step of size dt (advection-reflection, Zehnder, Narain, Thomaszewski 2018):
 *   0. forces: inside the source box, d = 1 and v = v_in; buoyancy v += dt b d (faces
 *      average the two adjacent cells' density);
 *   1. u~ = A(u; u, dt/2)           velocity advected by itself for half a step
 *   2. u' = P(u~)                   projection
 *   3. u^ = 2 u' - u~               reflection
 *   4. u~2 = A(u^; u', dt/2)        the reflected field advected by u' for half a step
 *   5. u'' = P(u~2)                 projection: the new velocity
 *   6. d = A(d; u', dt)             density advected by u' for the whole step
 * A(f; w, s): semi-Lagrangian, for each sample point x of f trace back x_b = RK3(x, w, s)
 * (Ralston: k1 = w(x), k2 = w(x - s/2 k1), k3 = w(x - 3s/4 k2), x_b = x - s (2 k1 + 3 k2 +
 * 4 k3) / 9) and take f(x_b) by bilinear interpolation with the sample point clamped into
 * the sample lattice.
 * P(w): divergence D = (div w) (face differences over h); 64 Jacobi sweeps from q = 0 of
 * the Poisson problem lap(q) = D with zero normal derivative at the walls (a neighbour
 * outside the domain is not counted, so a cell divides by its number of interior
 * neighbours); then w -= grad q on the interior faces.
 * Quantized stores (the codec's step index is the store counter of the step, Q7): the
 * velocity after 1, 2, 3, 4, 5 (stores 1..5 of u and v) and every Jacobi iterate of q
 * (pressure stores); the density stays FP64.  The store counter of a step's k-th store is
 * 1024 * step + k.  The dither threshold of the store of sample i of field f (0 = u, 1 = v,
 * 2 = q) with store counter c is the codec's 16-bit draw for slot i / 8, step c and
 * component 8 f + i % 8: one Philox block (counter (i / 8, c, f, 0)) serves eight
 * consecutive samples of a field.
 *
 * Single stages (or_smoke_stage) run one stage from given stored inputs, so that kernels
 * can be compared with it stage by stage; record mode returns every store's code and the
 * value it was offered.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* bilinear sample of a lattice of nx x ny values at (gx, gy) in lattice units */
static double sample(const double *f, int nx, int ny, double gx, double gy)
{
    gx = clampd(gx, 0.0, (double)(nx - 1));
    gy = clampd(gy, 0.0, (double)(ny - 1));
    int i = (int)floor(gx), j = (int)floor(gy);
    if (i > nx - 2) i = nx - 2;
    if (j > ny - 2) j = ny - 2;
    if (i < 0) i = 0;
    if (j < 0) j = 0;
    const double fx = gx - i, fy = gy - j;
    const double a = f[j * nx + i], b = f[j * nx + i + 1], c = f[(j + 1) * nx + i], e = f[(j + 1) * nx + i + 1];
    return (1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * c + fx * e);
}

/* velocity at a point (x, y) in domain units from the MAC fields */
static void vel_at(const or_smoke_t *sm, const double *u, const double *v, double x, double y, double *ux, double *vy)
{
    const int n = sm->n;
    const double inv_h = (double)n;
    *ux = sample(u, n + 1, n, x * inv_h, y * inv_h - 0.5);
    *vy = sample(v, n, n + 1, x * inv_h - 0.5, y * inv_h);
}

static void backtrace(const or_smoke_t *sm, const double *u, const double *v, double s, double x, double y,
                      double *xb, double *yb)
{
    double k1x, k1y, k2x, k2y, k3x, k3y;
    vel_at(sm, u, v, x, y, &k1x, &k1y);
    vel_at(sm, u, v, x - 0.5 * s * k1x, y - 0.5 * s * k1y, &k2x, &k2y);
    vel_at(sm, u, v, x - 0.75 * s * k2x, y - 0.75 * s * k2y, &k3x, &k3y);
    *xb = x - s * (2.0 * k1x + 3.0 * k2x + 4.0 * k3x) / 9.0;
    *yb = y - s * (2.0 * k1y + 3.0 * k2y + 4.0 * k3y) / 9.0;
}

/* A(f; w, s) for the three kinds of lattice: 0 = u faces, 1 = v faces, 2 = cells */
static void advect(const or_smoke_t *sm, int kind, const double *f, const double *wu, const double *wv, double s,
                   double *out)
{
    const int n = sm->n;
    const double h = 1.0 / n;
    const int nx = kind == 0 ? n + 1 : n, ny = kind == 1 ? n + 1 : n;
    const double ox = kind == 0 ? 0.0 : 0.5, oy = kind == 1 ? 0.0 : 0.5;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double xb, yb;
            backtrace(sm, wu, wv, s, (i + ox) * h, (j + oy) * h, &xb, &yb);
            out[j * nx + i] = sample(f, nx, ny, xb * n - ox, yb * n - oy);
        }
}

static void walls(int n, double *u, double *v)
{
    for (int j = 0; j < n; ++j) {
        u[j * (n + 1)] = 0.0;
        u[j * (n + 1) + n] = 0.0;
    }
    for (int i = 0; i < n; ++i) {
        v[i] = 0.0;
        v[n * n + i] = 0.0;
    }
}

/* One additive error injected at one store (field, sample index, store counter): the
 * derivative of z with respect to it is the sensitivity that Eq. 8 accumulates, which the
 * tests take by central differences. */
static struct {
    int active, field;
    uint32_t idx, counter;
    double delta;
} g_inject;

void or_smoke_inject(int active, int field, uint32_t idx, uint32_t counter, double delta)
{
    g_inject.active = active;
    g_inject.field = field;
    g_inject.idx = idx;
    g_inject.counter = counter;
    g_inject.delta = delta;
}

static double store_q(const or_smoke_t *sm, const or_smoke_scheme_t *sch, int field, double x, uint32_t idx,
                      uint32_t counter, int64_t *sat);

/* Noise at every store (sensitivity estimates by antithetic injection): sign * sigma_h * r
 * with r = +-1 the top bit of the 16-bit lane of the dither generator (Philox4x32-7; key = noise seed, counter
 * (i / 8, store counter, field, 0), lane i % 8), at every store of type h except the
 * reflected velocity and the wall faces (stores that make no rounding error). */
static struct {
    int active;
    double sigma[2], sign;
    uint64_t seed;
} g_noise;

void or_smoke_noise(int active, double sigma_v, double sigma_p, uint64_t seed, double sign)
{
    g_noise.active = active;
    g_noise.sigma[0] = sigma_v;
    g_noise.sigma[1] = sigma_p;
    g_noise.seed = seed;
    g_noise.sign = sign;
}

static int wall_face(int n, int field, uint32_t idx)
{
    if (field == 0) return idx % (uint32_t)(n + 1) == 0 || idx % (uint32_t)(n + 1) == (uint32_t)n;
    if (field == 1) return idx / (uint32_t)n == 0 || idx / (uint32_t)n == (uint32_t)n;
    return 0;
}

/* store of a value through the codec (quantized run) or as is, plus an injected error */
static double store(const or_smoke_t *sm, const or_smoke_scheme_t *sch, int field, double x, uint32_t idx,
                    uint32_t counter, int64_t *sat)
{
    double y = store_q(sm, sch, field, x, idx, counter, sat);
    if (g_inject.active && g_inject.field == field && g_inject.idx == idx && g_inject.counter == counter)
        y += g_inject.delta;
    const int type = field == 2 ? 1 : 0;
    if (g_noise.active && g_noise.sigma[type] != 0.0 && !wall_face(sm->n, field, idx) &&
        !(field < 2 && counter % 1024u == (uint32_t)sm->jacobi + 3u)) {
        const uint32_t q = or_dither_draw(g_noise.seed, idx >> 3, counter, 8 * field + (int)(idx & 7u)) >> 16;
        y += g_noise.sign * g_noise.sigma[type] * ((q & 0x8000u) ? 1.0 : -1.0);
    }
    return y;
}

static struct {
    uint32_t *buf;
    double *xs;   /* optional: the value each store was offered */
    int64_t n, pos;
} g_record;

void or_smoke_record(uint32_t *buf, int64_t n)
{
    g_record.buf = buf;
    g_record.xs = NULL;
    g_record.n = n;
    g_record.pos = 0;
}

void or_smoke_record_values(uint32_t *buf, double *xs, int64_t n)
{
    or_smoke_record(buf, n);
    g_record.xs = xs;
}

int64_t or_smoke_recorded(void) { return g_record.pos; }

static double store_q(const or_smoke_t *sm, const or_smoke_scheme_t *sch, int field, double x, uint32_t idx,
                      uint32_t counter, int64_t *sat)
{
    if (!sch) return x;
    const int bits = sch->bits[field == 2 ? 1 : 0], frac = sch->frac[field == 2 ? 1 : 0];
    const int64_t offset = sch->offset[field == 2 ? 1 : 0];
    const uint32_t r = sm->dither ? or_dither_draw(sm->seed, idx >> 3, counter, 8 * field + (int)(idx & 7u)) : 0u;
    int flags = 0;
    uint32_t q = or_encode(x, bits, frac, offset, sm->dither, r, &flags);
    if ((flags & OR_FLAG_SAT) && sat) *sat += 1;
    if (g_record.buf) {
        if (g_record.pos < g_record.n) {
            g_record.buf[g_record.pos] = q;
            if (g_record.xs) g_record.xs[g_record.pos] = x;
        }
        g_record.pos += 1;
    }
    return or_decode(q, frac, offset);
}

static void store_velocity(const or_smoke_t *sm, const or_smoke_scheme_t *sch, double *u, double *v,
                           uint32_t counter, int64_t *sat)
{
    const int n = sm->n;
    for (int k = 0; k < (n + 1) * n; ++k) u[k] = store(sm, sch, 0, u[k], (uint32_t)k, counter, sat);
    for (int k = 0; k < n * (n + 1); ++k) v[k] = store(sm, sch, 1, v[k], (uint32_t)k, counter, sat);
}

/* one Jacobi sweep of lap(q) = div from the iterate q into q2, each value stored */
static void jacobi_sweep(const or_smoke_t *sm, const or_smoke_scheme_t *sch, const double *q, double *q2,
                         const double *div, uint32_t counter, int64_t *sat)
{
    const int n = sm->n;
    const double h2 = 1.0 / ((double)n * n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            int cnt = 0;
            if (i > 0) { acc += q[j * n + i - 1]; ++cnt; }
            if (i < n - 1) { acc += q[j * n + i + 1]; ++cnt; }
            if (j > 0) { acc += q[(j - 1) * n + i]; ++cnt; }
            if (j < n - 1) { acc += q[(j + 1) * n + i]; ++cnt; }
            q2[j * n + i] = store(sm, sch, 2, (acc - h2 * div[j * n + i]) / cnt, (uint32_t)(j * n + i), counter, sat);
        }
}

/* w -= grad q on the interior faces, then the walls */
static void grad_subtract(const or_smoke_t *sm, double *u, double *v, const double *q)
{
    const int n = sm->n;
    const double inv_h = (double)n;
    for (int j = 0; j < n; ++j)
        for (int i = 1; i < n; ++i) u[j * (n + 1) + i] -= (q[j * n + i] - q[j * n + i - 1]) * inv_h;
    for (int j = 1; j < n; ++j)
        for (int i = 0; i < n; ++i) v[j * n + i] -= (q[j * n + i] - q[(j - 1) * n + i]) * inv_h;
    walls(n, u, v);
}

static void project(const or_smoke_t *sm, const or_smoke_scheme_t *sch, double *u, double *v, double *q,
                    double *q2, double *div, uint32_t *counter, int64_t *sat)
{
    const int n = sm->n;
    const double inv_h = (double)n;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            div[j * n + i] = (u[j * (n + 1) + i + 1] - u[j * (n + 1) + i] + v[(j + 1) * n + i] - v[j * n + i]) * inv_h;
    memset(q, 0, sizeof(double) * (size_t)n * n);
    for (int it = 0; it < sm->jacobi; ++it) {
        *counter += 1;
        jacobi_sweep(sm, sch, q, q2, div, *counter, sat);
        memcpy(q, q2, sizeof(double) * (size_t)n * n);
    }
    grad_subtract(sm, u, v, q);
}

int64_t or_smoke_step(const or_smoke_t *sm, const or_smoke_scheme_t *sch, uint32_t step, double *u, double *v,
                      double *d, double *q)
{
    const int n = sm->n;
    const size_t nu = (size_t)(n + 1) * n, nv = (size_t)n * (n + 1), nc = (size_t)n * n;
    double *ut = malloc(sizeof(double) * nu), *vt = malloc(sizeof(double) * nv);
    double *up = malloc(sizeof(double) * nu), *vp = malloc(sizeof(double) * nv);
    double *dt2 = malloc(sizeof(double) * nc), *q2 = malloc(sizeof(double) * nc), *div = malloc(sizeof(double) * nc);
    int64_t sat = 0;
    uint32_t counter = 1024u * step;
    const double h = 1.0 / n;
    /* 0. forces: source box and buoyancy */
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            const double x = (i + 0.5) * h, y = (j + 0.5) * h;
            if (x >= sm->src[0] && x <= sm->src[2] && y >= sm->src[1] && y <= sm->src[3]) d[j * n + i] = 1.0;
        }
    for (int j = 1; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            const double x = (i + 0.5) * h, y = j * h;
            v[j * n + i] += sm->dt * sm->buoyancy * 0.5 * (d[j * n + i] + d[(j - 1) * n + i]);
            if (x >= sm->src[0] && x <= sm->src[2] && y >= sm->src[1] && y <= sm->src[3]) v[j * n + i] = sm->v_in;
        }
    walls(n, u, v);
    /* 1. u~ = A(u; u, dt/2) */
    advect(sm, 0, u, u, v, 0.5 * sm->dt, ut);
    advect(sm, 1, v, u, v, 0.5 * sm->dt, vt);
    walls(n, ut, vt);
    store_velocity(sm, sch, ut, vt, ++counter, &sat);
    /* 2. u' = P(u~) */
    memcpy(up, ut, sizeof(double) * nu);
    memcpy(vp, vt, sizeof(double) * nv);
    project(sm, sch, up, vp, q, q2, div, &counter, &sat);
    store_velocity(sm, sch, up, vp, ++counter, &sat);
    /* 3. u^ = 2 u' - u~ (into ut, vt) */
    for (size_t k = 0; k < nu; ++k) ut[k] = 2.0 * up[k] - ut[k];
    for (size_t k = 0; k < nv; ++k) vt[k] = 2.0 * vp[k] - vt[k];
    store_velocity(sm, sch, ut, vt, ++counter, &sat);
    /* 4. u~2 = A(u^; u', dt/2) (into u, v) */
    advect(sm, 0, ut, up, vp, 0.5 * sm->dt, u);
    advect(sm, 1, vt, up, vp, 0.5 * sm->dt, v);
    walls(n, u, v);
    store_velocity(sm, sch, u, v, ++counter, &sat);
    /* 5. u'' = P(u~2) */
    project(sm, sch, u, v, q, q2, div, &counter, &sat);
    store_velocity(sm, sch, u, v, ++counter, &sat);
    /* 6. d = A(d; u', dt) */
    advect(sm, 2, d, up, vp, sm->dt, dt2);
    memcpy(d, dt2, sizeof(double) * nc);
    free(ut);
    free(vt);
    free(up);
    free(vp);
    free(dt2);
    free(q2);
    free(div);
    return sat;
}

double or_smoke_measure(const or_smoke_t *sm, const double *d)
{
    double acc = 0.0;
    for (int k = 0; k < sm->n * sm->n; ++k) acc += d[k] * d[k];
    return acc;
}

/* ------------------------------------------------------------------------------------
 * Single stages of the step, for a stage-by-stage comparison with kernels that compute
 * them from the same stored inputs (no value of the kernel enters here).  Step index
 * `step` (1-based: the store counter is 1024 step + k).  Velocity pairs in the MAC layout
 * of this file; arrays not used by a stage may be NULL.
 *   OR_SMOKE_ADVECT1  out = store_1(A(a; (a_u, a_v), dt/2)), a_v = v after the forces
 *   OR_SMOKE_JACOBI   out_q = store_(1 + it)(sweep it of the first projection from the
 *                     iterate q (zeros when it = 1) with the divergence div), it = arg
 *   OR_SMOKE_GRADSUB2 out = store_(J+2)(a - grad q), out2 = store_(J+3)(2 out - a)
 *   OR_SMOKE_ADVECT4  out = store_(J+4)(A(a; (b_u, b_v), dt/2))
 *   OR_SMOKE_GRADSUB5 out = store_(2J+5)(a - grad q)
 * ---------------------------------------------------------------------------------- */
int or_smoke_stage(const or_smoke_t *sm, const or_smoke_scheme_t *sch, int stage, int arg, uint32_t step,
                   const double *a_u, const double *a_v, const double *b_u, const double *b_v, const double *q,
                   const double *div, double *out_u, double *out_v, double *out2_u, double *out2_v, double *out_q)
{
    const int n = sm->n, J = sm->jacobi;
    const size_t nu = (size_t)(n + 1) * n, nv = (size_t)n * (n + 1), nc = (size_t)n * n;
    const uint32_t base = 1024u * step;
    int64_t sat = 0;
    switch (stage) {
    case OR_SMOKE_ADVECT1:
    case OR_SMOKE_ADVECT4: {
        const double *wu = stage == OR_SMOKE_ADVECT1 ? a_u : b_u, *wv = stage == OR_SMOKE_ADVECT1 ? a_v : b_v;
        advect(sm, 0, a_u, wu, wv, 0.5 * sm->dt, out_u);
        advect(sm, 1, a_v, wu, wv, 0.5 * sm->dt, out_v);
        walls(n, out_u, out_v);
        store_velocity(sm, sch, out_u, out_v, base + (stage == OR_SMOKE_ADVECT1 ? 1u : (uint32_t)J + 4u), &sat);
        return 0;
    }
    case OR_SMOKE_JACOBI: {
        if (arg < 1 || arg > J) return -1;
        double *zero = NULL;
        if (arg == 1) {
            zero = calloc(nc, sizeof(double));
            if (!zero) return -2;
        }
        jacobi_sweep(sm, sch, arg == 1 ? zero : q, out_q, div, base + 1u + (uint32_t)arg, &sat);
        free(zero);
        return 0;
    }
    case OR_SMOKE_GRADSUB2:
    case OR_SMOKE_GRADSUB5: {
        memcpy(out_u, a_u, sizeof(double) * nu);
        memcpy(out_v, a_v, sizeof(double) * nv);
        grad_subtract(sm, out_u, out_v, q);
        store_velocity(sm, sch, out_u, out_v, base + (stage == OR_SMOKE_GRADSUB2 ? (uint32_t)J + 2u : 2u * J + 5u),
                       &sat);
        if (stage == OR_SMOKE_GRADSUB2) {
            for (size_t k = 0; k < nu; ++k) out2_u[k] = 2.0 * out_u[k] - a_u[k];
            for (size_t k = 0; k < nv; ++k) out2_v[k] = 2.0 * out_v[k] - a_v[k];
            store_velocity(sm, sch, out2_u, out2_v, base + (uint32_t)J + 3u, &sat);
        }
        return 0;
    }
    default:
        return -1;
    }
}
