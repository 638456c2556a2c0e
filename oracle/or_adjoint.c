/*
 * or_adjoint.c -- oracle: reverse-mode derivative of one FP64 MLS-MPM step (the adjoint
 * kernel G of Sec. 6 Eq. 13):  dz/ds_t = G(s_t, dz/ds_{t+1}).  TEST INFRASTRUCTURE ONLY.
 *
 * The forward step is the one of or_mpm.c.  Its reverse, written out from the chain rule:
 *   G2P   F' = (I + dt C') F      ->  Fb += (I + dt C')^T Fb',  Cb' += dt Fb' F^T
 *         (fluid J' = (1 + dt tr C') J -> Jb += (1 + dt tr C') Jb', Cb' += dt J Jb' I)
 *         x' = x + dt v'          ->  xb += xb',  vb' += dt xb'
 *         C' = D^-1 B,  B = sum_i w v_i dpos^T,  v' = sum_i w v_i
 *               -> vb_i += w vb' + w (D^-1 Cb') dpos,  wb += vb'.v_i + v_i^T (D^-1 Cb') dpos,
 *                  dposb = w (D^-1 Cb')^T v_i
 *   grid  v_i = mv_i / m_i + dt g  ->  mvb_i = vb_i / m_i,  mb_i = -vb_i . (v_i - dt g) / m_i
 *         (nothing flows through wall nodes or empty nodes)
 *   P2G   m_i += w m,  mv_i += w (m v + A dpos),  A = k tau(F) + m C,  k = -dt V D^-1
 *               -> vb += w m mvb_i,  Ab += w mvb_i dpos^T,  wb += m mb_i + mvb_i.(m v + A dpos),
 *                  dposb = w A^T mvb_i;  Cb += m Ab;  taub = k Ab -> Fb (stress adjoint)
 *   weights: dpos = x_i - x_p (so xb -= dposb) and w = prod_a N(x_a / dx - base_a - o_a)
 *            (xb_a += wb dw/dx_a); the stencil base is piecewise constant.
 * Stress adjoints (tau_b = upstream adjoint of tau):
 *   neo-Hookean:      Fb += mu (tau_b + tau_b^T) F + lambda tr(tau_b) F^-T
 *   fixed-corotated:  Fb += 2mu tau_b F + 2mu tau_b^T (F - R) - dR^T[2mu tau_b F]
 *                           + lambda (2J - 1) J tr(tau_b) F^-T
 *     with F = R S and dR = R W(w), w = (tr(S) I - S)^-1 axial(R^T dF - dF^T R) in 3D
 *     (dtheta = ((R^T dF)_10 - (R^T dF)_01) / tr S in 2D), so dR^T[G] = R W(u) with
 *     u = (tr(S) I - S)^-1 ax(R^T G), ax(X) = (X21 - X12, X02 - X20, X10 - X01)
 *     (2D: dR^T[G] = ((R^T G)_10 - (R^T G)_01) / tr(S) R J2, J2 = [[0,-1],[1,0]]).
 *   fluid:            Jb += K (2J - 1) tr(tau_b)
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int adj_stencil(const or_phys_t *ph, const double *x, int *base, double *f, double w[3][3],
                       double dw[3][3])
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
        /* derivatives with respect to x_a (df/dx = n) */
        dw[a][0] = -(1.5 - f[a]) * (double)n;
        dw[a][1] = -2.0 * (f[a] - 1.0) * (double)n;
        dw[a][2] = (f[a] - 0.5) * (double)n;
    }
    return out;
}

static int64_t adj_node(int dim, int n, const int *idx)
{
    if (dim == 2) return (int64_t)idx[0] * n + idx[1];
    return ((int64_t)idx[0] * n + idx[1]) * n + idx[2];
}

static void offsets(int d, int o, int *off)
{
    if (d == 2) { off[0] = o / 3; off[1] = o % 3; off[2] = 0; }
    else { off[0] = o / 9; off[1] = (o / 3) % 3; off[2] = o % 3; }
}

static double det_m(int d, const double *F)
{
    if (d == 2) return F[0] * F[3] - F[1] * F[2];
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
           F[2] * (F[3] * F[7] - F[4] * F[6]);
}

/* F^-T (row major) */
static void inv_transpose(int d, const double *F, double *FiT)
{
    const double J = det_m(d, F);
    if (d == 2) {
        FiT[0] = F[3] / J; FiT[1] = -F[2] / J;
        FiT[2] = -F[1] / J; FiT[3] = F[0] / J;
        return;
    }
    /* cofactor matrix / det */
    FiT[0] = (F[4] * F[8] - F[5] * F[7]) / J;
    FiT[1] = (F[5] * F[6] - F[3] * F[8]) / J;
    FiT[2] = (F[3] * F[7] - F[4] * F[6]) / J;
    FiT[3] = (F[7] * F[2] - F[8] * F[1]) / J;
    FiT[4] = (F[8] * F[0] - F[6] * F[2]) / J;
    FiT[5] = (F[6] * F[1] - F[7] * F[0]) / J;
    FiT[6] = (F[1] * F[5] - F[2] * F[4]) / J;
    FiT[7] = (F[2] * F[3] - F[0] * F[5]) / J;
    FiT[8] = (F[0] * F[4] - F[1] * F[3]) / J;
}

/* solve the symmetric 3x3 system K u = r by Cramer's rule */
static void solve3(const double *K, const double *r, double *u)
{
    const double D = det_m(3, K);
    for (int c = 0; c < 3; ++c) {
        double M[9];
        memcpy(M, K, sizeof(M));
        for (int i = 0; i < 3; ++i) M[i * 3 + c] = r[i];
        u[c] = det_m(3, M) / D;
    }
}

/* Fb += d tau / dF ^T [taub] */
static void stress_adjoint(const or_phys_t *ph, const double *FJ, const double *taub, double *Fb)
{
    const int d = ph->dim;
    double tr = 0.0;
    for (int a = 0; a < d; ++a) tr += taub[a * d + a];
    if (ph->material == OR_FLUID) {
        const double J = FJ[0];
        Fb[0] += ph->bulk * (2.0 * J - 1.0) * tr;
        return;
    }
    double mu, la;
    or_lame(ph->E, ph->nu, &mu, &la);
    const double *F = FJ;
    double FiT[9];
    inv_transpose(d, F, FiT);
    const double J = det_m(d, F);
    if (ph->material == OR_NEOHOOKEAN) {
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                double acc = 0.0;
                for (int k = 0; k < d; ++k) acc += (taub[a * d + k] + taub[k * d + a]) * F[k * d + b];
                Fb[a * d + b] += mu * acc + la * tr * FiT[a * d + b];
            }
        return;
    }
    /* fixed-corotated */
    double R[9];
    if (d == 2) or_polar2(F, R); else or_polar3(F, R);
    double G[9];  /* 2 mu taub F */
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double acc = 0.0;
            for (int k = 0; k < d; ++k) acc += taub[a * d + k] * F[k * d + b];
            G[a * d + b] = 2.0 * mu * acc;
        }
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double acc = 0.0;
            for (int k = 0; k < d; ++k) acc += taub[k * d + a] * (F[k * d + b] - R[k * d + b]);
            Fb[a * d + b] += G[a * d + b] + 2.0 * mu * acc + la * (2.0 * J - 1.0) * J * tr * FiT[a * d + b];
        }
    /* minus dR^T[G] */
    double RtG[9], S[9];
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double acc = 0.0, accS = 0.0;
            for (int k = 0; k < d; ++k) {
                acc += R[k * d + a] * G[k * d + b];
                accS += R[k * d + a] * F[k * d + b];
            }
            RtG[a * d + b] = acc;
            S[a * d + b] = accS;
        }
    if (d == 2) {
        const double trS = S[0] + S[3];
        const double c = (RtG[2] - RtG[1]) / trS;
        /* R J2, J2 = [[0,-1],[1,0]] */
        const double RJ[4] = {R[1], -R[0], R[3], -R[2]};
        for (int q = 0; q < 4; ++q) Fb[q] -= c * RJ[q];
        return;
    }
    const double trS = S[0] + S[4] + S[8];
    double K[9];
    for (int q = 0; q < 9; ++q) K[q] = -0.5 * (S[q] + S[(q % 3) * 3 + q / 3]);
    K[0] += trS; K[4] += trS; K[8] += trS;
    const double ax[3] = {RtG[7] - RtG[5], RtG[2] - RtG[6], RtG[3] - RtG[1]};
    double u[3];
    solve3(K, ax, u);
    const double W[9] = {0.0, -u[2], u[1], u[2], 0.0, -u[0], -u[1], u[0], 0.0};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += R[a * 3 + k] * W[k * 3 + b];
            Fb[a * 3 + b] -= acc;
        }
}

void or_adjoint_step(const or_phys_t *ph, int64_t N, const double *s, const double *sbn, double *sb)
{
    const int d = ph->dim, n = 1 << ph->grid_log2, nc = or_n_comp(d, ph->material);
    const int stride = 1 + d, n_off = d == 2 ? 9 : 27;
    const double dx = 1.0 / (double)n, Dinv = 4.0 * (double)n * (double)n;
    const double kcoef = -ph->dt * ph->p_vol * Dinv, m = ph->p_mass;
    const int64_t nn = or_n_nodes(ph);
    double *grid = (double *)calloc((size_t)nn * stride, sizeof(double));
    double *gb = (double *)calloc((size_t)nn * stride, sizeof(double));

    /* forward: P2G then the grid update (mass kept in slot 0, velocity in 1..d) */
    or_p2g(ph, N, s, grid);
    or_grid_update(ph, grid);

    memset(sb, 0, sizeof(double) * (size_t)N * nc);
    /* G2P reverse */
    for (int64_t p = 0; p < N; ++p) {
        const double *x = s + p * nc, *FJ = x + 2 * d + d * d;
        const double *xbn = sbn + p * nc, *vbn = xbn + d, *Cbn = xbn + 2 * d, *FJbn = xbn + 2 * d + d * d;
        double *xb = sb + p * nc, *Fb = xb + 2 * d + d * d;
        int base[3];
        double f[3], w[3][3], dw[3][3];
        adj_stencil(ph, x, base, f, w, dw);
        /* forward C' */
        double Cn[9] = {0};
        for (int o = 0; o < n_off; ++o) {
            int off[3], idx[3];
            offsets(d, o, off);
            double wt = 1.0, dpos[3];
            for (int a = 0; a < d; ++a) {
                wt *= w[a][off[a]];
                dpos[a] = ((double)off[a] - f[a]) * dx;
                idx[a] = base[a] + off[a];
            }
            const double *g = grid + adj_node(d, n, idx) * stride;
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) Cn[a * d + b] += Dinv * wt * g[1 + a] * dpos[b];
        }
        double Cb[9] = {0};
        for (int q = 0; q < d * d; ++q) Cb[q] = Cbn[q];
        if (ph->material == OR_FLUID) {
            double tr = 0.0;
            for (int a = 0; a < d; ++a) tr += Cn[a * d + a];
            Fb[0] += (1.0 + ph->dt * tr) * FJbn[0];
            for (int a = 0; a < d; ++a) Cb[a * d + a] += ph->dt * FJ[0] * FJbn[0];
        } else {
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) {
                    double accF = 0.0, accC = 0.0;
                    for (int k = 0; k < d; ++k) {
                        accF += ((k == a ? 1.0 : 0.0) + ph->dt * Cn[k * d + a]) * FJbn[k * d + b];
                        accC += FJbn[a * d + k] * FJ[b * d + k];
                    }
                    Fb[a * d + b] += accF;
                    Cb[a * d + b] += ph->dt * accC;
                }
        }
        double vbt[3], Bb[9];
        for (int a = 0; a < d; ++a) {
            xb[a] += xbn[a];
            vbt[a] = vbn[a] + ph->dt * xbn[a];
        }
        for (int q = 0; q < d * d; ++q) Bb[q] = Dinv * Cb[q];
        for (int o = 0; o < n_off; ++o) {
            int off[3], idx[3];
            offsets(d, o, off);
            double wt = 1.0, dpos[3], dwt[3];
            for (int a = 0; a < d; ++a) {
                wt *= w[a][off[a]];
                dpos[a] = ((double)off[a] - f[a]) * dx;
                idx[a] = base[a] + off[a];
            }
            for (int a = 0; a < d; ++a) {
                dwt[a] = dw[a][off[a]];
                for (int b = 0; b < d; ++b)
                    if (b != a) dwt[a] *= w[b][off[b]];
            }
            const int64_t node = adj_node(d, n, idx);
            const double *g = grid + node * stride;
            double *gbn = gb + node * stride;
            double wb = 0.0;
            for (int a = 0; a < d; ++a) {
                double Bd = 0.0;
                for (int b = 0; b < d; ++b) Bd += Bb[a * d + b] * dpos[b];
                gbn[1 + a] += wt * (vbt[a] + Bd);
                wb += vbt[a] * g[1 + a] + g[1 + a] * Bd;
            }
            for (int b = 0; b < d; ++b) {
                double dpb = 0.0;
                for (int a = 0; a < d; ++a) dpb += wt * Bb[a * d + b] * g[1 + a];
                xb[b] -= dpb;
            }
            for (int a = 0; a < d; ++a) xb[a] += wb * dwt[a];
        }
    }
    /* grid reverse */
    for (int64_t node = 0; node < nn; ++node) {
        int idx[3];
        if (d == 2) { idx[0] = (int)(node / n); idx[1] = (int)(node % n); }
        else { idx[0] = (int)(node / ((int64_t)n * n)); idx[1] = (int)((node / n) % n); idx[2] = (int)(node % n); }
        int wall = 0;
        for (int a = 0; a < d; ++a)
            if (idx[a] < ph->bound || idx[a] > n - 1 - ph->bound) wall = 1;
        double *g = grid + node * stride, *gbn = gb + node * stride;
        const double mi = g[0];
        if (wall || !(mi > 0.0)) {
            for (int a = 0; a <= d; ++a) gbn[a] = 0.0;
            continue;
        }
        double mb = 0.0;
        for (int a = 0; a < d; ++a) {
            mb -= gbn[1 + a] * (g[1 + a] - ph->dt * ph->gravity[a]) / mi;
            gbn[1 + a] /= mi;
        }
        gbn[0] = mb;
    }
    /* P2G reverse */
    for (int64_t p = 0; p < N; ++p) {
        const double *x = s + p * nc, *v = x + d, *C = x + 2 * d, *FJ = x + 2 * d + d * d;
        double *xb = sb + p * nc, *vb = xb + d, *Cb = xb + 2 * d, *Fb = xb + 2 * d + d * d;
        int base[3];
        double f[3], w[3][3], dw[3][3];
        adj_stencil(ph, x, base, f, w, dw);
        double tau[9], A[9], Ab[9] = {0};
        or_kirchhoff(ph, FJ, tau);
        for (int q = 0; q < d * d; ++q) A[q] = kcoef * tau[q] + m * C[q];
        for (int o = 0; o < n_off; ++o) {
            int off[3], idx[3];
            offsets(d, o, off);
            double wt = 1.0, dpos[3], dwt[3];
            for (int a = 0; a < d; ++a) {
                wt *= w[a][off[a]];
                dpos[a] = ((double)off[a] - f[a]) * dx;
                idx[a] = base[a] + off[a];
            }
            for (int a = 0; a < d; ++a) {
                dwt[a] = dw[a][off[a]];
                for (int b = 0; b < d; ++b)
                    if (b != a) dwt[a] *= w[b][off[b]];
            }
            const double *gbn = gb + adj_node(d, n, idx) * stride;
            double wb = m * gbn[0];
            for (int a = 0; a < d; ++a) {
                double Ad = 0.0;
                for (int b = 0; b < d; ++b) Ad += A[a * d + b] * dpos[b];
                vb[a] += wt * m * gbn[1 + a];
                wb += gbn[1 + a] * (m * v[a] + Ad);
                for (int b = 0; b < d; ++b) Ab[a * d + b] += wt * gbn[1 + a] * dpos[b];
            }
            for (int b = 0; b < d; ++b) {
                double dpb = 0.0;
                for (int a = 0; a < d; ++a) dpb += wt * A[a * d + b] * gbn[1 + a];
                xb[b] -= dpb;
            }
            for (int a = 0; a < d; ++a) xb[a] += wb * dwt[a];
        }
        double taub[9];
        for (int q = 0; q < d * d; ++q) {
            Cb[q] += m * Ab[q];
            taub[q] = kcoef * Ab[q];
        }
        stress_adjoint(ph, FJ, taub, Fb);
    }
    free(grid);
    free(gb);
}
