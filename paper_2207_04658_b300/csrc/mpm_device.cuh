// mpm_device.cuh -- MLS-MPM device math shared by the step and adjoint kernels: the
// polar decomposition, the Kirchhoff stress of the three materials and the quadratic
// B-spline stencil.
#pragma once

#include "device_common.cuh"

namespace qmpm {

// ------------------------------------------------------------------------------ materials
// 3D polar factor by the scaled Newton iteration X <- (g X + X^-T / g) / 2 with
// determinant scaling g = |det X|^(-1/3) (Higham 1986; Byers & Xu 2008).  X^-T is the
// cofactor matrix (rows: cross products of the other two rows) over det X.
// detF: det F, which the caller has already.  A (nearly) singular F has no unique polar
// factor and the iteration's scaling would overflow: R = I there (|det F| < 1e-6, or NaN).
__device__ __forceinline__ void polar3(const float *F, float detF, float *R)
{
    float X[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) X[i] = F[i];
    if (!(fabsf(detF) >= 1e-6f)) {
#pragma unroll
        for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0f : 0.0f;
        return;
    }
    for (int it = 0; it < 10; ++it) {
        const float c0 = X[4] * X[8] - X[5] * X[7], c1 = X[5] * X[6] - X[3] * X[8],
                    c2 = X[3] * X[7] - X[4] * X[6];
        const float c3 = X[7] * X[2] - X[8] * X[1], c4 = X[8] * X[0] - X[6] * X[2],
                    c5 = X[6] * X[1] - X[7] * X[0];
        const float c6 = X[1] * X[5] - X[2] * X[4], c7 = X[2] * X[3] - X[0] * X[5],
                    c8 = X[0] * X[4] - X[1] * X[3];
        const float det = X[0] * c0 + X[1] * c1 + X[2] * c2;
        // g = |det|^(-1/3); the scale only speeds convergence, so fast log2/exp2 suffice;
        // b to the hardware reciprocal's accuracy moves the fixed point by an ulp or two
        float g;
        asm("{\n\t.reg .f32 l;\n\tlg2.approx.ftz.f32 l, %1;\n\tmul.ftz.f32 l, l, 0fBEAAAAAB;\n\t"
            "ex2.approx.ftz.f32 %0, l;\n\t}"
            : "=f"(g)
            : "f"(fabsf(det)));
        const float a = 0.5f * g, b = __fdividef(0.5f, g * det);
        const float cof[9] = {c0, c1, c2, c3, c4, c5, c6, c7, c8};
        float diff = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float nx = a * X[i] + b * cof[i];
            diff += (nx - X[i]) * (nx - X[i]);
            X[i] = nx;
        }
        // quadratic convergence: after a step of size below 3e-4 (squared 1e-7) X is within
        // about half its square, ~5e-8, of the polar factor (FP32 resolution), so the
        // iteration stops without a confirming step
        if (diff < 1e-7f) break;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = X[i];
}

// Kirchhoff stress tau (row major DIM x DIM).
template <int DIM, int MAT>
__device__ __forceinline__ void kirchhoff(const float *FJ, const StepParams &P, float *tau)
{
    if (MAT == QMPM_FLUID) {
        const float J = FJ[0];
        const float p = P.bulk * (J - 1.0f) * J;
#pragma unroll
        for (int i = 0; i < DIM * DIM; ++i) tau[i] = (i % (DIM + 1) == 0) ? p : 0.0f;
        return;
    }
    const float *F = FJ;
    float J;
    if (DIM == 2)
        J = F[0] * F[3] - F[1] * F[2];
    else
        J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
            F[2] * (F[3] * F[7] - F[4] * F[6]);
    if (MAT == QMPM_NEOHOOKEAN) {
        const float vol = P.lambda * logf(J);
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
                float ff = 0.0f;
#pragma unroll
                for (int k = 0; k < DIM; ++k) ff += F[a * DIM + k] * F[b * DIM + k];
                tau[a * DIM + b] = P.mu * (ff - (a == b ? 1.0f : 0.0f)) + (a == b ? vol : 0.0f);
            }
    } else {
        float R[DIM * DIM];
        if (DIM == 2) {
            const float x = F[0] + F[3], y = F[2] - F[1];
            const float h = hypotf(x, y);
            const float c = h > 0.0f ? x / h : 1.0f, s = h > 0.0f ? y / h : 0.0f;
            R[0] = c;
            R[1] = -s;
            R[2] = s;
            R[3] = c;
        } else {
            polar3(F, J, R);
        }
        const float vol = P.lambda * (J - 1.0f) * J;
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k < DIM; ++k) acc += (F[a * DIM + k] - R[a * DIM + k]) * F[b * DIM + k];
                tau[a * DIM + b] = 2.0f * P.mu * acc + (a == b ? vol : 0.0f);
            }
    }
}

// stencil base per axis, clamped to [0, n-3]; returns true if clamped (out of grid)
template <int DIM>
__device__ __forceinline__ bool stencil(const float *x, const StepParams &P, int *base, float (*w)[3],
                                        float *f)
{
    bool out = false;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const float fx = x[a] * P.inv_dx;
        int b = __float2int_rd(fx - 0.5f);
        if (b < 0) {
            b = 0;
            out = true;
        }
        if (b > P.n - 3) {
            b = P.n - 3;
            out = true;
        }
        base[a] = b;
        f[a] = fx - (float)b;
        const float d0 = 1.5f - f[a], d1 = f[a] - 1.0f, d2 = f[a] - 0.5f;
        w[a][0] = 0.5f * d0 * d0;
        w[a][1] = 0.75f - d1 * d1;
        w[a][2] = 0.5f * d2 * d2;
    }
    return out;
}

}  // namespace qmpm
