/*
 * or_mpm.c -- oracle: one MLS-MPM time step in FP64 (the simulator the paper quantizes,
 * MLS-MPM of Hu et al. 2018 cited in Sec. 8.1), its quantized form
 *   s~_t = F(s~_{t-1}) + e_t                                   (Sec. 3.1 Eq. 1)
 * i.e. decode -> FP64 step -> dithered encode, the particle ordering used by the dither
 * counter, and the position measurement.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The step (quadratic B-spline weights, APIC transfer, D^-1 = 4/dx^2):
 *   P2G   m_i  += w_ip m_p
 *         mv_i += w_ip (m_p v_p + A_p (x_i - x_p)),  A_p = -dt V_p D^-1 tau_p + m_p C_p
 *   grid  v_i = mv_i / m_i + dt g  (m_i > 0, else 0); v_i = 0 within `bound` nodes of a wall
 *   G2P   v_p = sum w_ip v_i,  C_p = D^-1 sum w_ip v_i (x_i - x_p)^T,  x_p += dt v_p,
 *         F_p = (I + dt C_p) F_p   or   J_p = (1 + dt tr C_p) J_p
 * Kirchhoff stress tau: neo-Hookean mu(FF^T - I) + lambda ln(J) I; fixed-corotated
 * 2mu(F - R)F^T + lambda (J - 1) J I; weakly compressible fluid K (J - 1) J I.
 *
 * A particle whose stencil base leaves [0, n-3] on some axis is "out of grid": its base
 * is clamped to the range (its weights then extrapolate) and it is counted.
 *
 * The OpenMP pragmas only matter in the separate threaded build used for long FP64
 * reference rollouts; there the P2G sums are atomic, so their order (and the last bits of
 * the grid) varies from run to run.  The default build ignores them and is sequential.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

void or_lame(double E, double nu, double *mu, double *lambda)
{
    *mu = E / (2.0 * (1.0 + nu));
    *lambda = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

/* 2D polar factor: the rotation maximising tr(R^T F). */
void or_polar2(const double F[4], double R[4])
{
    const double a = F[0] + F[3], b = F[2] - F[1];
    const double h = hypot(a, b);
    double c = 1.0, s = 0.0;
    if (h > 0.0) {
        c = a / h;
        s = b / h;
    }
    R[0] = c; R[1] = -s;
    R[2] = s; R[3] = c;
}

static void mat3_mul(const double *A, const double *B, double *Cm)
{
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += A[i * 3 + k] * B[k * 3 + j];
            T[i * 3 + j] = acc;
        }
    memcpy(Cm, T, sizeof(T));
}

static void mat3_transpose(const double *A, double *T)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[j * 3 + i] = A[i * 3 + j];
}

static double det_d(int d, const double *F);

/* 3D polar factor R = F S^-1 with S = (F^T F)^{1/2}; the symmetric square root comes
 * from a cyclic Jacobi eigen-decomposition of F^T F (Golub & Van Loan, Sec. 8.5).
 * For det F < 0 the factor has det R = -1.  A (nearly) singular F, |det F| < 1e-6, has
 * no unique factor (S^-1 does not exist): R = I there. */
void or_polar3(const double F[9], double R[9])
{
    if (!(fabs(det_d(3, F)) >= 1e-6)) {
        for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
        return;
    }
    double Ft[9], A[9], V[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    mat3_transpose(F, Ft);
    mat3_mul(Ft, F, A);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        double diag = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (off <= 1e-32 * diag) break;
        static const int PQ[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        for (int r = 0; r < 3; ++r) {
            const int p = PQ[r][0], q = PQ[r][1];
            const double apq = A[p * 3 + q];
            if (apq == 0.0) continue;
            const double theta = (A[q * 3 + q] - A[p * 3 + p]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
            double J[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, Jt[9];
            J[p * 3 + p] = c; J[q * 3 + q] = c;
            J[p * 3 + q] = s; J[q * 3 + p] = -s;
            mat3_transpose(J, Jt);
            mat3_mul(Jt, A, A);
            mat3_mul(A, J, A);
            mat3_mul(V, J, V);
        }
    }
    /* S^-1 = V diag(1/sqrt(lambda)) V^T */
    double Dinv[9] = {0}, Vt[9], Sinv[9];
    for (int i = 0; i < 3; ++i) Dinv[i * 4] = 1.0 / sqrt(A[i * 4]);
    mat3_transpose(V, Vt);
    mat3_mul(V, Dinv, Sinv);
    mat3_mul(Sinv, Vt, Sinv);
    mat3_mul(F, Sinv, R);
}

static double det_d(int d, const double *F)
{
    if (d == 2) return F[0] * F[3] - F[1] * F[2];
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
           F[2] * (F[3] * F[7] - F[4] * F[6]);
}

void or_kirchhoff(const or_phys_t *ph, const double *FJ, double *tau)
{
    const int d = ph->dim;
    memset(tau, 0, sizeof(double) * (size_t)(d * d));
    if (ph->material == OR_FLUID) {
        const double J = FJ[0];
        for (int a = 0; a < d; ++a) tau[a * d + a] = ph->bulk * (J - 1.0) * J;
        return;
    }
    double mu, la;
    or_lame(ph->E, ph->nu, &mu, &la);
    const double *F = FJ;
    const double J = det_d(d, F);
    if (ph->material == OR_NEOHOOKEAN) {
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                double ffT = 0.0;
                for (int k = 0; k < d; ++k) ffT += F[a * d + k] * F[b * d + k];
                tau[a * d + b] = mu * (ffT - (a == b ? 1.0 : 0.0));
            }
        for (int a = 0; a < d; ++a) tau[a * d + a] += la * log(J);
    } else {
        double R[9];
        if (d == 2) or_polar2(F, R); else or_polar3(F, R);
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                double acc = 0.0;
                for (int k = 0; k < d; ++k) acc += (F[a * d + k] - R[a * d + k]) * F[b * d + k];
                tau[a * d + b] = 2.0 * mu * acc;
            }
        for (int a = 0; a < d; ++a) tau[a * d + a] += la * (J - 1.0) * J;
    }
}

int or_n_nodes(const or_phys_t *ph)
{
    const int n = 1 << ph->grid_log2;
    return ph->dim == 2 ? n * n : n * n * n;
}

/* Stencil of one particle: base node, fractional offset f in [0.5, 1.5), weights. */
static int stencil(const or_phys_t *ph, const double *x, int *base, double *f, double w[3][3])
{
    const int n = 1 << ph->grid_log2;
    int out = 0;
    for (int a = 0; a < ph->dim; ++a) {
        const double fx = x[a] * (double)n;
        int b = (int)floor(fx - 0.5);
        if (b < 0) { b = 0; out = 1; }
        if (b > n - 3) { b = n - 3; out = 1; }
        base[a] = b;
        f[a] = fx - (double)b;
        w[a][0] = 0.5 * (1.5 - f[a]) * (1.5 - f[a]);
        w[a][1] = 0.75 - (f[a] - 1.0) * (f[a] - 1.0);
        w[a][2] = 0.5 * (f[a] - 0.5) * (f[a] - 0.5);
    }
    return out;
}

static int64_t node_index(int dim, int n, const int *idx)
{
    if (dim == 2) return (int64_t)idx[0] * n + idx[1];
    return ((int64_t)idx[0] * n + idx[1]) * n + idx[2];
}

int64_t or_p2g(const or_phys_t *ph, int64_t N, const double *s, double *grid)
{
    const int d = ph->dim, n = 1 << ph->grid_log2, nc = or_n_comp(d, ph->material);
    const int stride = 1 + d;
    const double dx = 1.0 / (double)n, Dinv = 4.0 * (double)n * (double)n;
    memset(grid, 0, sizeof(double) * (size_t)or_n_nodes(ph) * (size_t)stride);
    int64_t oog = 0;
    const int n_off = d == 2 ? 9 : 27;
#pragma omp parallel for schedule(static) reduction(+ : oog)
    for (int64_t p = 0; p < N; ++p) {
        const double *x = s + p * nc, *v = x + d, *C = x + 2 * d, *FJ = x + 2 * d + d * d;
        int base[3];
        double f[3], w[3][3];
        oog += stencil(ph, x, base, f, w);
        double tau[9], A[9];
        or_kirchhoff(ph, FJ, tau);
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b)
                A[a * d + b] = -ph->dt * ph->p_vol * Dinv * tau[a * d + b] + ph->p_mass * C[a * d + b];
        for (int o = 0; o < n_off; ++o) {
            int off[3] = {o / (d == 2 ? 3 : 9), (o / 3) % 3, o % 3};
            if (d == 2) { off[0] = o / 3; off[1] = o % 3; }
            double weight = 1.0, dpos[3];
            int idx[3];
            for (int a = 0; a < d; ++a) {
                weight *= w[a][off[a]];
                dpos[a] = ((double)off[a] - f[a]) * dx;
                idx[a] = base[a] + off[a];
            }
            double *g = grid + node_index(d, n, idx) * stride;
#pragma omp atomic
            g[0] += weight * ph->p_mass;
            for (int a = 0; a < d; ++a) {
                double Ad = 0.0;
                for (int b = 0; b < d; ++b) Ad += A[a * d + b] * dpos[b];
#pragma omp atomic
                g[1 + a] += weight * (ph->p_mass * v[a] + Ad);
            }
        }
    }
    return oog;
}

void or_grid_update(const or_phys_t *ph, double *grid)
{
    const int d = ph->dim, n = 1 << ph->grid_log2, stride = 1 + d;
    const int64_t nn = or_n_nodes(ph);
#pragma omp parallel for schedule(static)
    for (int64_t node = 0; node < nn; ++node) {
        int idx[3];
        if (d == 2) { idx[0] = (int)(node / n); idx[1] = (int)(node % n); }
        else { idx[0] = (int)(node / ((int64_t)n * n)); idx[1] = (int)((node / n) % n); idx[2] = (int)(node % n); }
        double *g = grid + node * stride;
        const double m = g[0];
        int wall = 0;
        for (int a = 0; a < d; ++a)
            if (idx[a] < ph->bound || idx[a] > n - 1 - ph->bound) wall = 1;
        for (int a = 0; a < d; ++a) {
            double vel = 0.0;
            if (m > 0.0) vel = g[1 + a] / m + ph->dt * ph->gravity[a];
            if (wall) vel = 0.0;
            g[1 + a] = vel;
        }
    }
}

int64_t or_g2p(const or_phys_t *ph, int64_t N, const double *grid, double *s)
{
    const int d = ph->dim, n = 1 << ph->grid_log2, nc = or_n_comp(d, ph->material);
    const int stride = 1 + d;
    const double dx = 1.0 / (double)n, Dinv = 4.0 * (double)n * (double)n;
    const int n_off = d == 2 ? 9 : 27;
    int64_t oog = 0;
#pragma omp parallel for schedule(static) reduction(+ : oog)
    for (int64_t p = 0; p < N; ++p) {
        double *x = s + p * nc, *v = x + d, *C = x + 2 * d, *FJ = x + 2 * d + d * d;
        int base[3];
        double f[3], w[3][3];
        oog += stencil(ph, x, base, f, w);
        double vn[3] = {0, 0, 0}, B[9] = {0};
        for (int o = 0; o < n_off; ++o) {
            int off[3] = {o / 9, (o / 3) % 3, o % 3};
            if (d == 2) { off[0] = o / 3; off[1] = o % 3; }
            double weight = 1.0, dpos[3];
            int idx[3];
            for (int a = 0; a < d; ++a) {
                weight *= w[a][off[a]];
                dpos[a] = ((double)off[a] - f[a]) * dx;
                idx[a] = base[a] + off[a];
            }
            const double *g = grid + node_index(d, n, idx) * stride;
            for (int a = 0; a < d; ++a) {
                vn[a] += weight * g[1 + a];
                for (int b = 0; b < d; ++b) B[a * d + b] += weight * g[1 + a] * dpos[b];
            }
        }
        for (int a = 0; a < d; ++a) {
            v[a] = vn[a];
            x[a] += ph->dt * vn[a];
            for (int b = 0; b < d; ++b) C[a * d + b] = Dinv * B[a * d + b];
        }
        if (ph->material == OR_FLUID) {
            double tr = 0.0;
            for (int a = 0; a < d; ++a) tr += C[a * d + a];
            FJ[0] = (1.0 + ph->dt * tr) * FJ[0];
        } else {
            double Fn[9];
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) {
                    double acc = 0.0;
                    for (int k = 0; k < d; ++k)
                        acc += ((a == k ? 1.0 : 0.0) + ph->dt * C[a * d + k]) * FJ[k * d + b];
                    Fn[a * d + b] = acc;
                }
            memcpy(FJ, Fn, sizeof(double) * (size_t)(d * d));
        }
    }
    return oog;
}

int64_t or_step_fp64(const or_phys_t *ph, int64_t N, double *s, double *grid_scratch)
{
    const int64_t oog = or_p2g(ph, N, s, grid_scratch);
    or_grid_update(ph, grid_scratch);
    or_g2p(ph, N, grid_scratch, s);
    return oog;
}

/* An explicit error at every store of step `step` (the second-order error model: Eq. 6
 * bounds the second moment of the error of z, Eq. 8 keeps its linear part): component c of
 * particle p gets sign * sigma[field(c)] * xi, xi uniform with unit variance.  The draw:
 * Philox4x32-10 block of counter (p, step, floor(c / 4), 0xA5) and key `seed` (low word
 * first); its word c mod 4, w, gives k = floor(w / 2^9) (23 bits), u = (k + 1/2) / 2^23 in
 * (0, 1) and xi = (2u - 1) sqrt(3), i.e. uniform on (-sqrt 3, sqrt 3). */
void or_add_noise(int dim, int material, int64_t N, double *s, uint32_t step, uint64_t seed,
                  const double sigma[4], double sign)
{
    or_add_noise_matched(dim, material, N, s, step, seed, sigma, sign, 0);
}

/* matched: sigma[h] is the resolution Delta_h and a store of value x gets the dithered
 * store's own variance, sigma = Delta_h sqrt(Y (1 - Y)), Y the fraction of x / Delta_h. */
void or_add_noise_matched(int dim, int material, int64_t N, double *s, uint32_t step, uint64_t seed,
                          const double sigma[4], double sign, int matched)
{
    const int nc = or_n_comp(dim, material);
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t p = 0; p < N; ++p) {
        uint32_t blk[4] = {0, 0, 0, 0};
        for (int c = 0; c < nc; ++c) {
            if (c % 4 == 0) {
                const uint32_t ctr[4] = {(uint32_t)p, step, (uint32_t)(c / 4), 0xA5u};
                or_philox4x32_10(ctr, key, blk);
            }
            const double k = (double)(blk[c % 4] >> 9);
            const double u = (k + 0.5) / 8388608.0;
            const double xi = (2.0 * u - 1.0) * sqrt(3.0);
            double sg = sigma[or_comp_field(dim, material, c)];
            if (matched && sg > 0.0) {
                const double t = s[p * nc + c] / sg;
                const double Y = t - floor(t);
                sg *= sqrt(Y * (1.0 - Y));
            }
            s[p * nc + c] += sign * sg * xi;
        }
    }
}

void or_step_quant(const or_phys_t *ph, const or_codec_t *cd, int64_t N, uint32_t *words,
                   uint32_t step, double *s_scratch, double *grid_scratch, int64_t *stats)
{
    or_decode_state(cd, N, words, s_scratch);
    const int64_t oog = or_step_fp64(ph, N, s_scratch, grid_scratch);
    if (stats) stats[OR_STAT_OOG] += oog;
    or_encode_state(cd, N, s_scratch, step, words, stats);
}

/* ------------------------------------------------------------------------------------
 * Particle ordering.  A particle with stencil base b (per axis) belongs to the tile whose
 * origin is block T = floor((b + 3) / 4) of a grid padded by one 4-node block on each
 * side; the tile of 2^d blocks T..T+1 then holds every stencil node of bases 4(T-1) ..
 * 4(T-1)+5, one node of slack on each side of the bases seen when the key was taken.
 * Within a tile, particles are ordered by their cell c = b - 4(T-1) - 1 in [0,4)^d:
 *   key = linear(T) * 4^d + linear(c).
 * ---------------------------------------------------------------------------------- */
int64_t or_n_keys(const or_phys_t *ph)
{
    const int64_t nb = ((int64_t)1 << ph->grid_log2) / 4 + 2;
    return ph->dim == 2 ? nb * nb * 16 : nb * nb * nb * 64;
}

void or_tile_keys(const or_phys_t *ph, int64_t N, const double *s, int64_t *keys)
{
    const int d = ph->dim, nc = or_n_comp(d, ph->material);
    const int64_t nb = ((int64_t)1 << ph->grid_log2) / 4 + 2;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int base[3];
        double f[3], w[3][3];
        stencil(ph, s + p * nc, base, f, w);
        int64_t tile = 0, cell = 0;
        for (int a = 0; a < d; ++a) {
            const int T = (base[a] + 3) / 4;
            tile = tile * nb + (int64_t)T;
            cell = cell * 4 + (int64_t)(base[a] - 4 * (T - 1) - 1);
        }
        keys[p] = tile * (d == 2 ? 16 : 64) + cell;
    }
}

void or_stable_sort(int64_t N, const int64_t *keys, int64_t n_keys, int64_t *perm)
{
    int64_t *start = (int64_t *)calloc((size_t)n_keys + 1, sizeof(int64_t));
    for (int64_t i = 0; i < N; ++i) start[keys[i] + 1] += 1;
    for (int64_t k = 0; k < n_keys; ++k) start[k + 1] += start[k];
    for (int64_t i = 0; i < N; ++i) perm[start[keys[i]]++] = i;
    free(start);
}

/* z = (1/N) sum_p |x_p|^2, the position measurement (a form of Eq. 2's Z). */
double or_mean_sq_pos(int dim, int n_comp, int64_t N, const double *s)
{
    double acc = 0.0;
    for (int64_t p = 0; p < N; ++p)
        for (int a = 0; a < dim; ++a) acc += s[p * n_comp + a] * s[p * n_comp + a];
    return N > 0 ? acc / (double)N : 0.0;
}
