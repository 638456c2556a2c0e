// adjoint.cu -- reverse mode of the FP32 MLS-MPM step (Sec. 6, Eq. 12-13) and the
// accumulation of squared sensitivities g_h of Eq. 8 that the bit-allocation solve needs.
//
// The adjoint runs its own FP32 forward from the handle's current state (decoded if the
// handle is quantized: the paper takes gradients in full precision), on an FP32
// array-of-structs state, particle-parallel with global atomics (no tiles, no re-sort, so
// slot order is fixed for the whole call).  Memory: uniform checkpoints every k steps
// (states t = 0, k, 2k, ...) and a tape of the k states of the segment being reversed,
// recomputed from its checkpoint.
//
// Reverse of one step, given the state s_t and the adjoint of s_{t+1}:
//   recompute the grid of s_t (P2G, grid update), then
//   G2P:  Fb += (I + dt C')^T Fb',  Cb' += dt Fb' F^T  (fluid: Jb += (1 + dt tr C') Jb',
//         Cb' += dt J Jb' I);  xb += xb',  vb' += dt xb';  with Bb = D^-1 Cb':
//         grid vb_i += w (vb' + Bb dpos),  wb = vb'.v_i + v_i^T Bb dpos,  dposb = w Bb^T v_i
//   grid: mvb_i = vb_i / m_i,  mb_i = -vb_i.(v_i - dt g) / m_i  (zero on walls / empty nodes)
//   P2G:  vb += w m mvb_i,  Ab += w mvb_i dpos^T,  wb += m mb_i + mvb_i.(m v + A dpos),
//         dposb = w A^T mvb_i;  Cb += m Ab;  Fb += stress adjoint of k Ab
//   weights and offsets: xb -= dposb,  xb_a += wb dw/dx_a.
// Stress adjoints: neo-Hookean  Fb += mu (T + T^T) F + lambda tr(T) F^-T;
// fixed-corotated  Fb += 2mu T F + 2mu T^T (F - R) + lambda (2J - 1) J tr(T) F^-T - dR^T[2mu T F]
// with dR^T[G] = R W(u), u = (tr(S) I - S)^-1 ax(R^T G), S = R^T F (3D) or
// ((R^T G)_10 - (R^T G)_01) / tr(S) R J2 (2D); fluid  Jb += K (2J - 1) tr(T).
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "mpm_device.cuh"

namespace qmpm {

namespace {

constexpr int kAdjThreads = 256;

template <int DIM>
__device__ __forceinline__ int64_t dense_node(int n, int i, int j, int k)
{
    return DIM == 2 ? (int64_t)i * n + j : ((int64_t)i * n + j) * n + k;
}

template <int DIM>
__device__ __forceinline__ void weight_grads(const float *f, const StepParams &P, float (*dw)[3])
{
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        dw[a][0] = -(1.5f - f[a]) * P.inv_dx;
        dw[a][1] = -2.0f * (f[a] - 1.0f) * P.inv_dx;
        dw[a][2] = (f[a] - 0.5f) * P.inv_dx;
    }
}

template <int DIM>
__device__ __forceinline__ void inv_transpose(const float *F, float *FiT, float &J)
{
    if (DIM == 2) {
        J = F[0] * F[3] - F[1] * F[2];
        const float r = 1.0f / J;
        FiT[0] = F[3] * r;
        FiT[1] = -F[2] * r;
        FiT[2] = -F[1] * r;
        FiT[3] = F[0] * r;
    } else {
        const float c[9] = {F[4] * F[8] - F[5] * F[7], F[5] * F[6] - F[3] * F[8], F[3] * F[7] - F[4] * F[6],
                            F[7] * F[2] - F[8] * F[1], F[8] * F[0] - F[6] * F[2], F[6] * F[1] - F[7] * F[0],
                            F[1] * F[5] - F[2] * F[4], F[2] * F[3] - F[0] * F[5], F[0] * F[4] - F[1] * F[3]};
        J = F[0] * c[0] + F[1] * c[1] + F[2] * c[2];
        const float r = 1.0f / J;
#pragma unroll
        for (int q = 0; q < 9; ++q) FiT[q] = c[q] * r;
    }
}

// Fb += (d tau / dF)^T [T]
template <int DIM, int MAT>
__device__ __forceinline__ void stress_adjoint(const float *FJ, const float *T, const StepParams &P, float *Fb)
{
    float tr = 0.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) tr += T[a * DIM + a];
    if (MAT == QMPM_FLUID) {
        Fb[0] += P.bulk * (2.0f * FJ[0] - 1.0f) * tr;
        return;
    }
    const float *F = FJ;
    float FiT[DIM * DIM], J;
    inv_transpose<DIM>(F, FiT, J);
    if (MAT == QMPM_NEOHOOKEAN) {
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k < DIM; ++k) acc += (T[a * DIM + k] + T[k * DIM + a]) * F[k * DIM + b];
                Fb[a * DIM + b] += P.mu * acc + P.lambda * tr * FiT[a * DIM + b];
            }
        return;
    }
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
    float G[DIM * DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < DIM; ++k) acc += T[a * DIM + k] * F[k * DIM + b];
            G[a * DIM + b] = 2.0f * P.mu * acc;
        }
    const float vol = P.lambda * (2.0f * J - 1.0f) * J * tr;
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < DIM; ++k) acc += T[k * DIM + a] * (F[k * DIM + b] - R[k * DIM + b]);
            Fb[a * DIM + b] += G[a * DIM + b] + 2.0f * P.mu * acc + vol * FiT[a * DIM + b];
        }
    float RtG[DIM * DIM], S[DIM * DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
            float g = 0.0f, sv = 0.0f;
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                g += R[k * DIM + a] * G[k * DIM + b];
                sv += R[k * DIM + a] * F[k * DIM + b];
            }
            RtG[a * DIM + b] = g;
            S[a * DIM + b] = sv;
        }
    if (DIM == 2) {
        const float c = (RtG[2] - RtG[1]) / (S[0] + S[3]);
        Fb[0] -= c * R[1];
        Fb[1] += c * R[0];
        Fb[2] -= c * R[3];
        Fb[3] += c * R[2];
        return;
    }
    const float trS = S[0] + S[4] + S[8];
    float K[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) K[q] = -0.5f * (S[q] + S[(q % 3) * 3 + q / 3]);
    K[0] += trS;
    K[4] += trS;
    K[8] += trS;
    const float ax[3] = {RtG[7] - RtG[5], RtG[2] - RtG[6], RtG[3] - RtG[1]};
    // u = K^-1 ax via the adjugate
    const float c0 = K[4] * K[8] - K[5] * K[7], c1 = K[5] * K[6] - K[3] * K[8], c2 = K[3] * K[7] - K[4] * K[6];
    const float c3 = K[7] * K[2] - K[8] * K[1], c4 = K[8] * K[0] - K[6] * K[2], c5 = K[6] * K[1] - K[7] * K[0];
    const float c6 = K[1] * K[5] - K[2] * K[4], c7 = K[2] * K[3] - K[0] * K[5], c8 = K[0] * K[4] - K[1] * K[3];
    const float rdet = 1.0f / (K[0] * c0 + K[1] * c1 + K[2] * c2);
    // inverse = adj / det, adj = cofactor^T
    const float u0 = (c0 * ax[0] + c3 * ax[1] + c6 * ax[2]) * rdet;
    const float u1 = (c1 * ax[0] + c4 * ax[1] + c7 * ax[2]) * rdet;
    const float u2 = (c2 * ax[0] + c5 * ax[1] + c8 * ax[2]) * rdet;
    const float W[9] = {0.0f, -u2, u1, u2, 0.0f, -u0, -u1, u0, 0.0f};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) acc += R[a * 3 + k] * W[k * 3 + b];
            Fb[a * 3 + b] -= acc;
        }
}

// ---------------------------------------------------------------------------- forward
template <int DIM, int MAT>
__global__ void adj_p2g_kernel(const __grid_constant__ StepParams P, const float *s, int64_t N, float *gm, float4 *gmv)
{
    constexpr int NC = 2 * DIM + DIM * DIM + (MAT == QMPM_FLUID ? 1 : DIM * DIM);
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    float val[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) val[c] = s[p * NC + c];
    const float *x = val, *v = val + DIM, *C = val + 2 * DIM, *FJ = val + 2 * DIM + DIM * DIM;
    int base[3] = {0, 0, 0};
    float w[3][3], f[3];
    stencil<DIM>(x, P, base, w, f);
    float tau[DIM * DIM], A[DIM * DIM];
    kirchhoff<DIM, MAT>(FJ, P, tau);
#pragma unroll
    for (int q = 0; q < DIM * DIM; ++q) A[q] = P.stress_coef * tau[q] + P.p_mass * C[q];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < (DIM == 3 ? 3 : 1); ++k) {
                const float wt = w[0][i] * w[1][j] * (DIM == 3 ? w[2][k] : 1.0f);
                const float dp[3] = {((float)i - f[0]) * P.dx, ((float)j - f[1]) * P.dx,
                                     DIM == 3 ? ((float)k - f[2]) * P.dx : 0.0f};
                float mom[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    float acc = P.p_mass * v[a];
#pragma unroll
                    for (int b = 0; b < DIM; ++b) acc += A[a * DIM + b] * dp[b];
                    mom[a] = wt * acc;
                }
                const int64_t node = dense_node<DIM>(P.n, base[0] + i, base[1] + j, DIM == 3 ? base[2] + k : 0);
                atomicAdd(gm + node, wt * P.p_mass);
                atomicAdd(gmv + node, make_float4(mom[0], mom[1], DIM == 3 ? mom[2] : 0.0f, 0.0f));
            }
}

// momentum -> velocity in place (gravity, sticky walls); empty and wall nodes get 0
template <int DIM>
__global__ void adj_grid_kernel(const __grid_constant__ StepParams P, const float *gm, float4 *gv, int64_t n_nodes)
{
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= n_nodes) return;
    const int n = P.n;
    const int i = DIM == 2 ? (int)(node / n) : (int)(node / ((int64_t)n * n));
    const int j = (int)((DIM == 2 ? node : node / n) % n);
    const int k = DIM == 2 ? 0 : (int)(node % n);
    const int hi = n - 1 - P.bound;
    bool wall = i < P.bound || i > hi || j < P.bound || j > hi;
    if (DIM == 3) wall = wall || k < P.bound || k > hi;
    const float m = gm[node];
    float4 mv = gv[node];
    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (m > 0.0f && !wall) {
        v.x = mv.x / m + P.dt * P.gravity[0];
        v.y = mv.y / m + P.dt * P.gravity[1];
        if (DIM == 3) v.z = mv.z / m + P.dt * P.gravity[2];
    }
    gv[node] = v;
}

template <int DIM, int MAT>
__global__ void adj_g2p_kernel(const __grid_constant__ StepParams P, const float *s, float *s_out, int64_t N,
                               const float4 *gv)
{
    constexpr int NC = 2 * DIM + DIM * DIM + (MAT == QMPM_FLUID ? 1 : DIM * DIM);
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    float val[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) val[c] = s[p * NC + c];
    float *x = val, *v = val + DIM, *C = val + 2 * DIM, *FJ = val + 2 * DIM + DIM * DIM;
    int base[3] = {0, 0, 0};
    float w[3][3], f[3];
    stencil<DIM>(x, P, base, w, f);
    float vn[3] = {0.0f, 0.0f, 0.0f}, B[DIM * DIM];
#pragma unroll
    for (int q = 0; q < DIM * DIM; ++q) B[q] = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < (DIM == 3 ? 3 : 1); ++k) {
                const float wt = w[0][i] * w[1][j] * (DIM == 3 ? w[2][k] : 1.0f);
                const float dp[3] = {((float)i - f[0]) * P.dx, ((float)j - f[1]) * P.dx,
                                     DIM == 3 ? ((float)k - f[2]) * P.dx : 0.0f};
                const float4 g = gv[dense_node<DIM>(P.n, base[0] + i, base[1] + j, DIM == 3 ? base[2] + k : 0)];
                const float ga[3] = {g.x, g.y, g.z};
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    vn[a] += wt * ga[a];
#pragma unroll
                    for (int b = 0; b < DIM; ++b) B[a * DIM + b] += wt * ga[a] * dp[b];
                }
            }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        v[a] = vn[a];
        x[a] += P.dt * vn[a];
#pragma unroll
        for (int b = 0; b < DIM; ++b) C[a * DIM + b] = P.Dinv * B[a * DIM + b];
    }
    if (MAT == QMPM_FLUID) {
        float tr = 0.0f;
#pragma unroll
        for (int a = 0; a < DIM; ++a) tr += C[a * DIM + a];
        FJ[0] = (1.0f + P.dt * tr) * FJ[0];
    } else {
        float Fn[DIM * DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
                float acc = FJ[a * DIM + b];
#pragma unroll
                for (int k = 0; k < DIM; ++k) acc += P.dt * C[a * DIM + k] * FJ[k * DIM + b];
                Fn[a * DIM + b] = acc;
            }
#pragma unroll
        for (int q = 0; q < DIM * DIM; ++q) FJ[q] = Fn[q];
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) s_out[p * NC + c] = val[c];
}

// ---------------------------------------------------------------------------- reverse
template <int DIM, int MAT>
__global__ void adj_g2p_rev_kernel(const __grid_constant__ StepParams P, const float *s, const float *sbn, float *sb,
                                   int64_t N, const float4 *gv, float4 *gb)
{
    constexpr int NC = 2 * DIM + DIM * DIM + (MAT == QMPM_FLUID ? 1 : DIM * DIM);
    constexpr int OF = 2 * DIM + DIM * DIM;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    float x[DIM], FJ[NC - OF];
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = s[p * NC + a];
#pragma unroll
    for (int q = 0; q < NC - OF; ++q) FJ[q] = s[p * NC + OF + q];
    int base[3] = {0, 0, 0};
    float w[3][3], f[3], dw[3][3];
    stencil<DIM>(x, P, base, w, f);
    weight_grads<DIM>(f, P, dw);
    // forward C'
    float Cn[DIM * DIM];
#pragma unroll
    for (int q = 0; q < DIM * DIM; ++q) Cn[q] = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < (DIM == 3 ? 3 : 1); ++k) {
                const float wt = w[0][i] * w[1][j] * (DIM == 3 ? w[2][k] : 1.0f);
                const float dp[3] = {((float)i - f[0]) * P.dx, ((float)j - f[1]) * P.dx,
                                     DIM == 3 ? ((float)k - f[2]) * P.dx : 0.0f};
                const float4 g = gv[dense_node<DIM>(P.n, base[0] + i, base[1] + j, DIM == 3 ? base[2] + k : 0)];
                const float ga[3] = {g.x, g.y, g.z};
#pragma unroll
                for (int a = 0; a < DIM; ++a)
#pragma unroll
                    for (int b = 0; b < DIM; ++b) Cn[a * DIM + b] += P.Dinv * wt * ga[a] * dp[b];
            }
    float xbn[DIM], vbt[DIM], Cb[DIM * DIM], FJbn[NC - OF], Fb[NC - OF];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        xbn[a] = sbn[p * NC + a];
        vbt[a] = sbn[p * NC + DIM + a] + P.dt * xbn[a];
    }
#pragma unroll
    for (int q = 0; q < DIM * DIM; ++q) Cb[q] = sbn[p * NC + 2 * DIM + q];
#pragma unroll
    for (int q = 0; q < NC - OF; ++q) {
        FJbn[q] = sbn[p * NC + OF + q];
        Fb[q] = 0.0f;
    }
    if (MAT == QMPM_FLUID) {
        float tr = 0.0f;
#pragma unroll
        for (int a = 0; a < DIM; ++a) tr += Cn[a * DIM + a];
        Fb[0] = (1.0f + P.dt * tr) * FJbn[0];
#pragma unroll
        for (int a = 0; a < DIM; ++a) Cb[a * DIM + a] += P.dt * FJ[0] * FJbn[0];
    } else {
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
                float accF = 0.0f, accC = 0.0f;
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    accF += ((k == a ? 1.0f : 0.0f) + P.dt * Cn[k * DIM + a]) * FJbn[k * DIM + b];
                    accC += FJbn[a * DIM + k] * FJ[b * DIM + k];
                }
                Fb[a * DIM + b] = accF;
                Cb[a * DIM + b] += P.dt * accC;
            }
    }
    float xb[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) xb[a] = xbn[a];
#pragma unroll
    for (int q = 0; q < DIM * DIM; ++q) Cb[q] *= P.Dinv;  // Bb
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < (DIM == 3 ? 3 : 1); ++k) {
                const int off[3] = {i, j, k};
                float wt = 1.0f, dwt[3];
#pragma unroll
                for (int a = 0; a < DIM; ++a) wt *= w[a][off[a]];
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    dwt[a] = dw[a][off[a]];
#pragma unroll
                    for (int b = 0; b < DIM; ++b)
                        if (b != a) dwt[a] *= w[b][off[b]];
                }
                const float dp[3] = {((float)i - f[0]) * P.dx, ((float)j - f[1]) * P.dx,
                                     DIM == 3 ? ((float)k - f[2]) * P.dx : 0.0f};
                const int64_t node = dense_node<DIM>(P.n, base[0] + i, base[1] + j, DIM == 3 ? base[2] + k : 0);
                const float4 g = gv[node];
                const float ga[3] = {g.x, g.y, g.z};
                float gbv[3] = {0.0f, 0.0f, 0.0f}, wb = 0.0f;
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    float Bd = 0.0f;
#pragma unroll
                    for (int b = 0; b < DIM; ++b) Bd += Cb[a * DIM + b] * dp[b];
                    gbv[a] = wt * (vbt[a] + Bd);
                    wb += vbt[a] * ga[a] + ga[a] * Bd;
                }
                atomicAdd(gb + node, make_float4(gbv[0], gbv[1], gbv[2], 0.0f));
#pragma unroll
                for (int b = 0; b < DIM; ++b) {
                    float dpb = 0.0f;
#pragma unroll
                    for (int a = 0; a < DIM; ++a) dpb += Cb[a * DIM + b] * ga[a];
                    xb[b] -= wt * dpb;
                }
#pragma unroll
                for (int a = 0; a < DIM; ++a) xb[a] += wb * dwt[a];
            }
    // write the G2P part of the adjoint of s_t (v and C receive theirs in P2G reverse)
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        sb[p * NC + a] = xb[a];
        sb[p * NC + DIM + a] = 0.0f;
    }
#pragma unroll
    for (int q = 0; q < DIM * DIM; ++q) sb[p * NC + 2 * DIM + q] = 0.0f;
#pragma unroll
    for (int q = 0; q < NC - OF; ++q) sb[p * NC + OF + q] = Fb[q];
}

template <int DIM>
__global__ void adj_grid_rev_kernel(const __grid_constant__ StepParams P, const float *gm, const float4 *gv,
                                    float4 *gb, int64_t n_nodes)
{
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= n_nodes) return;
    const int n = P.n;
    const int i = DIM == 2 ? (int)(node / n) : (int)(node / ((int64_t)n * n));
    const int j = (int)((DIM == 2 ? node : node / n) % n);
    const int k = DIM == 2 ? 0 : (int)(node % n);
    const int hi = n - 1 - P.bound;
    bool wall = i < P.bound || i > hi || j < P.bound || j > hi;
    if (DIM == 3) wall = wall || k < P.bound || k > hi;
    const float m = gm[node];
    float4 b = gb[node];
    if (wall || !(m > 0.0f)) {
        gb[node] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
    const float4 v = gv[node];
    const float rm = 1.0f / m;
    const float mb = -(b.x * (v.x - P.dt * P.gravity[0]) + b.y * (v.y - P.dt * P.gravity[1]) +
                       (DIM == 3 ? b.z * (v.z - P.dt * P.gravity[2]) : 0.0f)) * rm;
    gb[node] = make_float4(b.x * rm, b.y * rm, b.z * rm, mb);
}

template <int DIM, int MAT>
__global__ void adj_p2g_rev_kernel(const __grid_constant__ StepParams P, const float *s, float *sb, int64_t N,
                                   const float4 *gb)
{
    constexpr int NC = 2 * DIM + DIM * DIM + (MAT == QMPM_FLUID ? 1 : DIM * DIM);
    constexpr int OF = 2 * DIM + DIM * DIM;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    float val[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) val[c] = s[p * NC + c];
    const float *x = val, *v = val + DIM, *C = val + 2 * DIM, *FJ = val + OF;
    int base[3] = {0, 0, 0};
    float w[3][3], f[3], dw[3][3];
    stencil<DIM>(x, P, base, w, f);
    weight_grads<DIM>(f, P, dw);
    float tau[DIM * DIM], A[DIM * DIM], Ab[DIM * DIM];
    kirchhoff<DIM, MAT>(FJ, P, tau);
#pragma unroll
    for (int q = 0; q < DIM * DIM; ++q) {
        A[q] = P.stress_coef * tau[q] + P.p_mass * C[q];
        Ab[q] = 0.0f;
    }
    float xb[DIM], vb[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        xb[a] = 0.0f;
        vb[a] = 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < (DIM == 3 ? 3 : 1); ++k) {
                const int off[3] = {i, j, k};
                float wt = 1.0f, dwt[3];
#pragma unroll
                for (int a = 0; a < DIM; ++a) wt *= w[a][off[a]];
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    dwt[a] = dw[a][off[a]];
#pragma unroll
                    for (int b = 0; b < DIM; ++b)
                        if (b != a) dwt[a] *= w[b][off[b]];
                }
                const float dp[3] = {((float)i - f[0]) * P.dx, ((float)j - f[1]) * P.dx,
                                     DIM == 3 ? ((float)k - f[2]) * P.dx : 0.0f};
                const float4 g = gb[dense_node<DIM>(P.n, base[0] + i, base[1] + j, DIM == 3 ? base[2] + k : 0)];
                const float mvb[3] = {g.x, g.y, g.z};
                float wb = P.p_mass * g.w;
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    float Ad = 0.0f;
#pragma unroll
                    for (int b = 0; b < DIM; ++b) Ad += A[a * DIM + b] * dp[b];
                    vb[a] += wt * P.p_mass * mvb[a];
                    wb += mvb[a] * (P.p_mass * v[a] + Ad);
#pragma unroll
                    for (int b = 0; b < DIM; ++b) Ab[a * DIM + b] += wt * mvb[a] * dp[b];
                }
#pragma unroll
                for (int b = 0; b < DIM; ++b) {
                    float dpb = 0.0f;
#pragma unroll
                    for (int a = 0; a < DIM; ++a) dpb += A[a * DIM + b] * mvb[a];
                    xb[b] -= wt * dpb;
                }
#pragma unroll
                for (int a = 0; a < DIM; ++a) xb[a] += wb * dwt[a];
            }
    float T[DIM * DIM], Fb[NC - OF];
#pragma unroll
    for (int q = 0; q < DIM * DIM; ++q) T[q] = P.stress_coef * Ab[q];
#pragma unroll
    for (int q = 0; q < NC - OF; ++q) Fb[q] = 0.0f;
    stress_adjoint<DIM, MAT>(FJ, T, P, Fb);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        sb[p * NC + a] += xb[a];
        sb[p * NC + DIM + a] += vb[a];
    }
#pragma unroll
    for (int q = 0; q < DIM * DIM; ++q) sb[p * NC + 2 * DIM + q] += P.p_mass * Ab[q];
#pragma unroll
    for (int q = 0; q < NC - OF; ++q) sb[p * NC + OF + q] += Fb[q];
}

// ---------------------------------------------------------------------------- helpers
// word planes of the handle -> FP32 AoS state
__global__ void adj_load_kernel(const __grid_constant__ StepParams P, int quant, float *s, int64_t N)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    for (int c = 0; c < P.n_comp; ++c) {
        const CompCodec &cc = P.comp[c];
        float v;
        if (!quant) {
            v = __uint_as_float(P.words[c * P.ld + p]);
        } else {
            const uint32_t lo = P.words[cc.word * P.ld + p];
            const uint32_t hi = (cc.word + 1 < P.n_words) ? P.words[(cc.word + 1) * P.ld + p] : 0u;
            v = decode_u(__funnelshift_r(lo, hi, cc.shift) & cc.mask, cc);
        }
        s[p * P.n_comp + c] = v;
    }
}

// The quantized store of step `step` applied to an FP32 state in place: dithered encode
// (slot p = particle index of the adjoint's fixed order) and decode of the stored value.
// Used when the forward of the adjoint follows the quantized trajectory.
__global__ void adj_quantize_kernel(const __grid_constant__ StepParams P, float *s, int64_t N, uint32_t step)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    uint4 rnd = make_uint4(0, 0, 0, 0);
    for (int c = 0; c < P.n_comp; ++c) {
        if (P.dither && (c & 7) == 0)
            rnd = philox4x32(make_uint4((uint32_t)p, step, (uint32_t)(c >> 3), 0u), P.seed_lo, P.seed_hi);
        const CompCodec &cc = P.comp[c];
        int fl;
        const uint32_t u = encode_f32(s[p * P.n_comp + c], cc, P.dither != 0, dither_threshold(rnd, c), fl);
        s[p * P.n_comp + c] = decode_u(u, cc);
    }
}

// An explicit error added to every stored component of step `step`: component c of
// particle p gets sign * sigma[field(c)] * xi with xi uniform on [-sqrt 3, sqrt 3) (unit
// variance), drawn from Philox4x32-10 with counter (p, step, c / 4, 0xA5) and key `seed`:
// word c % 4 of the block gives u = (floor(w / 2^9) + 1/2) 2^-23 and xi = (2u - 1) sqrt 3.
// matched: sig holds the resolution Delta_h of each type, and the store of value x gets the
// dithered store's own variance there, sigma = Delta_h sqrt(Y (1 - Y)) with Y the fraction
// of x / Delta_h (a dithered store errs by -Y Delta or (1 - Y) Delta, zero mean).
__global__ void adj_noise_kernel(const __grid_constant__ StepParams P, float *s, int64_t N, uint32_t step,
                                 uint32_t seed_lo, uint32_t seed_hi, float4 sig, float sign, int matched)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    uint4 rnd = make_uint4(0, 0, 0, 0);
    for (int c = 0; c < P.n_comp; ++c) {
        if ((c & 3) == 0) rnd = philox4x32<10>(make_uint4((uint32_t)p, step, (uint32_t)(c >> 2), 0xA5u), seed_lo, seed_hi);
        const uint32_t w = uint4_at(rnd, c & 3);
        // 2u - 1 with u = (w / 2^9 + 1/2) 2^-23 in (0, 1): exact in FP32
        const float xi = ((float)(2u * (w >> 9) + 1u) * (1.0f / 8388608.0f) - 1.0f) * 1.7320508f;
        const int h = P.comp[c].field;
        float sg = h == 0 ? sig.x : h == 1 ? sig.y : h == 2 ? sig.z : sig.w;
        const float x = s[p * P.n_comp + c];
        if (matched && sg > 0.0f) {
            const float t = x / sg;  // sg a power of two: exact
            const float Y = t - floorf(t);
            sg *= sqrtf(Y * (1.0f - Y));
        }
        s[p * P.n_comp + c] = x + sign * sg * xi;
    }
}

// Order-preserving integer image of a float (signed comparison of the images orders the
// floats); the map is its own inverse on the bit patterns.
__host__ __device__ __forceinline__ int ordered_key(float f)
{
    int i;
    memcpy(&i, &f, sizeof(i));
    return i >= 0 ? i : (i ^ 0x7FFFFFFF);
}

__host__ __device__ __forceinline__ float ordered_value(int k)
{
    const int i = k >= 0 ? k : (k ^ 0x7FFFFFFF);
    float f;
    memcpy(&f, &i, sizeof(f));
    return f;
}

// per-field sum of squares (g_h, Eq. 8), per-field min / max, and z = mean |x|^2
// want_z: 1 = mean square position, 2 = kinetic energy (1/2) m sum |v|^2
__global__ void adj_reduce_kernel(const float *a, int64_t N, int nc, int dim, double *sq, float *lo, float *hi,
                                  double *z, int want_sq, int want_range, int want_z, float p_mass)
{
    double acc[4] = {0.0, 0.0, 0.0, 0.0}, zz = 0.0;
    float mn[4] = {INFINITY, INFINITY, INFINITY, INFINITY}, mx[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < nc; ++c) {
            const float v = a[p * nc + c];
            const int h = c < dim ? 0 : c < 2 * dim ? 1 : c < 2 * dim + dim * dim ? 2 : 3;
            acc[h] += (double)v * (double)v;
            mn[h] = fminf(mn[h], v);
            mx[h] = fmaxf(mx[h], v);
            if (want_z == 1 && c < dim) zz += (double)v * (double)v / (double)N;
            if (want_z == 2 && c >= dim && c < 2 * dim) zz += 0.5 * (double)p_mass * (double)v * (double)v;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        zz += __shfl_down_sync(0xFFFFFFFFu, zz, o);
        for (int h = 0; h < 4; ++h) {
            acc[h] += __shfl_down_sync(0xFFFFFFFFu, acc[h], o);
            mn[h] = fminf(mn[h], __shfl_down_sync(0xFFFFFFFFu, mn[h], o));
            mx[h] = fmaxf(mx[h], __shfl_down_sync(0xFFFFFFFFu, mx[h], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int h = 0; h < 4; ++h) {
            if (want_sq) atomicAdd(sq + h, acc[h]);
            if (want_range && mn[h] <= mx[h]) {
                atomicMin(reinterpret_cast<int *>(lo) + h, ordered_key(mn[h]));
                atomicMax(reinterpret_cast<int *>(hi) + h, ordered_key(mx[h]));
            }
        }
        if (want_z) atomicAdd(z, zz);
    }
}

// dz/ds_T of the built-in measurements: 2 x / N (mean square position) or m v (kinetic energy)
__global__ void adj_seed_kernel(const float *s, float *sb, int64_t N, int nc, int dim, int measure, float p_mass)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    for (int c = 0; c < nc; ++c) {
        float g = 0.0f;
        if (measure == QMPM_MEASURE_MEAN_SQ_POS && c < dim) g = 2.0f * s[p * nc + c] / (float)N;
        if (measure == QMPM_MEASURE_KINETIC_ENERGY && c >= dim && c < 2 * dim) g = p_mass * s[p * nc + c];
        sb[p * nc + c] = g;
    }
}

unsigned nblk(int64_t n) { return (unsigned)((n + kAdjThreads - 1) / kAdjThreads); }

template <int DIM, int MAT>
struct AdjRunner {
    static cudaError_t grid(const StepParams &P, const float *s, int64_t N, float *gm, float4 *gv, int64_t nn,
                            cudaStream_t st)
    {
        cudaError_t e = cudaMemsetAsync(gm, 0, sizeof(float) * (size_t)nn, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(gv, 0, sizeof(float4) * (size_t)nn, st);
        if (e != cudaSuccess) return e;
        if (N > 0) adj_p2g_kernel<DIM, MAT><<<nblk(N), kAdjThreads, 0, st>>>(P, s, N, gm, gv);
        adj_grid_kernel<DIM><<<nblk(nn), kAdjThreads, 0, st>>>(P, gm, gv, nn);
        return cudaGetLastError();
    }
    static cudaError_t forward(const StepParams &P, const float *s, float *s_out, int64_t N, float *gm, float4 *gv,
                               int64_t nn, cudaStream_t st)
    {
        cudaError_t e = grid(P, s, N, gm, gv, nn, st);
        if (e != cudaSuccess) return e;
        if (N > 0) adj_g2p_kernel<DIM, MAT><<<nblk(N), kAdjThreads, 0, st>>>(P, s, s_out, N, gv);
        return cudaGetLastError();
    }
    static cudaError_t reverse(const StepParams &P, const float *s, const float *sbn, float *sb, int64_t N, float *gm,
                               float4 *gv, float4 *gb, int64_t nn, cudaStream_t st)
    {
        cudaError_t e = grid(P, s, N, gm, gv, nn, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(gb, 0, sizeof(float4) * (size_t)nn, st);
        if (e != cudaSuccess) return e;
        if (N > 0) adj_g2p_rev_kernel<DIM, MAT><<<nblk(N), kAdjThreads, 0, st>>>(P, s, sbn, sb, N, gv, gb);
        adj_grid_rev_kernel<DIM><<<nblk(nn), kAdjThreads, 0, st>>>(P, gm, gv, gb, nn);
        if (N > 0) adj_p2g_rev_kernel<DIM, MAT><<<nblk(N), kAdjThreads, 0, st>>>(P, s, sb, N, gb);
        return cudaGetLastError();
    }
};

using ForwardFn = cudaError_t (*)(const StepParams &, const float *, float *, int64_t, float *, float4 *, int64_t,
                                  cudaStream_t);
using ReverseFn = cudaError_t (*)(const StepParams &, const float *, const float *, float *, int64_t, float *,
                                  float4 *, float4 *, int64_t, cudaStream_t);

void pick(int dim, int mat, ForwardFn &f, ReverseFn &r)
{
#define QMPM_ADJ(D, M)                                 \
    if (dim == D && mat == M) {                        \
        f = &AdjRunner<D, M>::forward;                 \
        r = &AdjRunner<D, M>::reverse;                 \
        return;                                        \
    }
    QMPM_ADJ(2, 0) QMPM_ADJ(2, 1) QMPM_ADJ(2, 2) QMPM_ADJ(3, 0) QMPM_ADJ(3, 1) QMPM_ADJ(3, 2)
#undef QMPM_ADJ
    f = nullptr;
    r = nullptr;
}

// The bisection schedule: slot d holds s_lo; reverse steps hi-1 .. lo.
void bisect(int32_t lo, int32_t hi, int32_t d, std::vector<qmpm_rev_op_t> &ops, int32_t &slots)
{
    slots = std::max(slots, d + 1);
    if (hi - lo == 1) {
        ops.push_back({QMPM_OP_REVERSE, d, d, lo, hi});
        return;
    }
    const int32_t mid = lo + (hi - lo + 1) / 2;  // the later half is the shorter one
    ops.push_back({QMPM_OP_ADVANCE, d, d + 1, lo, mid});
    bisect(mid, hi, d + 1, ops, slots);
    bisect(lo, mid, d, ops, slots);
}

}  // namespace

}  // namespace qmpm

extern "C" int qmpm_bisection_schedule(int32_t T, qmpm_rev_op_t *ops, int64_t max_ops, int64_t *n_ops,
                                       int32_t *n_slots)
{
    if (T < 0) {
        qmpm::set_last_error("qmpm_bisection_schedule: T < 0");
        return QMPM_ERR_INVALID_ARG;
    }
    std::vector<qmpm_rev_op_t> v;
    int32_t slots = 1;
    if (T > 0) qmpm::bisect(0, T, 0, v, slots);
    if (n_ops) *n_ops = (int64_t)v.size();
    if (n_slots) *n_slots = slots;
    if (ops) {
        if ((int64_t)v.size() > max_ops) {
            qmpm::set_last_error("qmpm_bisection_schedule: more ops than max_ops");
            return QMPM_ERR_INVALID_ARG;
        }
        std::copy(v.begin(), v.end(), ops);
    }
    return QMPM_OK;
}

extern "C" int qmpm_adjoint(qmpm_handle h, int32_t T, int32_t ckpt_every, int32_t measure, const float *d_seed,
                            float *d_grad0, qmpm_adjoint_out_t *out)
{
    using namespace qmpm;
    const bool qfwd = (measure & QMPM_ADJ_QUANTIZED_FORWARD) != 0;
    measure &= ~QMPM_ADJ_QUANTIZED_FORWARD;
    if (!h || T < 0 || ckpt_every < 0 || (qfwd && !h->quant) ||
        (measure != QMPM_MEASURE_MEAN_SQ_POS && measure != QMPM_MEASURE_USER &&
         measure != QMPM_MEASURE_KINETIC_ENERGY) ||
        (measure == QMPM_MEASURE_USER && !d_seed && h->N > 0)) {
        set_last_error("qmpm_adjoint: bad handle, T, ckpt_every, measure or seed");
        return QMPM_ERR_INVALID_ARG;
    }
    Ctx &c = *h;
    const int dim = c.scene.dim, nc = c.n_comp;
    const int64_t N = c.N;
    ForwardFn fwd;
    ReverseFn rev;
    pick(dim, c.scene.material, fwd, rev);
    StepParams P;
    fill_params(c, P);
    const int64_t nn = dim == 2 ? (int64_t)c.n * c.n : (int64_t)c.n * c.n * c.n;
    const bool bisection = ckpt_every == QMPM_CKPT_BISECTION;
    std::vector<qmpm_rev_op_t> sched;
    int32_t n_slots = 1;
    if (bisection && T > 0) bisect(0, T, 0, sched, n_slots);
    const int k = bisection ? 1 : std::min<int32_t>(ckpt_every, std::max<int32_t>(T, 1));
    // uniform: checkpoints every k steps plus a tape of one segment; bisection: one slot
    // per tree level plus a scratch state for the recomputation
    const int64_t n_ckpt = bisection ? n_slots : T / k + 1;
    const int64_t tape_states = bisection ? 2 : k + 1;
    int64_t fwd_steps = 0;
    const size_t state_bytes = sizeof(float) * (size_t)std::max<int64_t>(N, 1) * nc;
    cudaStream_t st = c.stream;

    std::vector<void *> allocs;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        allocs.push_back(p);
        return p;
    };
    auto cleanup = [&]() {
        for (void *p : allocs) cudaFree(p);
    };
    float *ckpt = static_cast<float *>(alloc(state_bytes * (size_t)n_ckpt));
    float *tape = static_cast<float *>(alloc(state_bytes * (size_t)tape_states));
    float *sbA = static_cast<float *>(alloc(state_bytes));
    float *sbB = static_cast<float *>(alloc(state_bytes));
    float *gm = static_cast<float *>(alloc(sizeof(float) * (size_t)nn));
    float4 *gv = static_cast<float4 *>(alloc(sizeof(float4) * (size_t)nn));
    float4 *gb = static_cast<float4 *>(alloc(sizeof(float4) * (size_t)nn));
    double *dsum = static_cast<double *>(alloc(sizeof(double) * 8));
    float *drange = static_cast<float *>(alloc(sizeof(float) * 8));
    if (!ckpt || !tape || !sbA || !sbB || !gm || !gv || !gb || !dsum || !drange) {
        cudaGetLastError();
        cleanup();
        set_last_error("qmpm_adjoint: device allocation failed");
        return QMPM_ERR_OOM;
    }
    cudaError_t e = cudaMemsetAsync(dsum, 0, sizeof(double) * 8, st);
    int range_init[8];
    for (int q = 0; q < 4; ++q) {
        range_init[q] = ordered_key(INFINITY);       // running minimum
        range_init[4 + q] = ordered_key(-INFINITY);  // running maximum
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(drange, range_init, sizeof(range_init), cudaMemcpyHostToDevice, st);
    // s_0 from the handle's state
    if (e == cudaSuccess && N > 0) {
        adj_load_kernel<<<nblk(N), kAdjThreads, 0, st>>>(P, c.quant ? 1 : 0, ckpt, N);
        e = cudaGetLastError();
    }
    const int64_t NE = N * nc;
    // one forward step s_t -> s_(t+1), through the quantized store of step t + 1 when the
    // adjoint follows the quantized trajectory
    auto step_fwd = [&](const float *a, float *b, int t) -> cudaError_t {
        cudaError_t r = fwd(P, a, b, N, gm, gv, nn, st);
        fwd_steps += 1;
        if (r == cudaSuccess && qfwd && N > 0) {
            adj_quantize_kernel<<<nblk(N), kAdjThreads, 0, st>>>(P, b, N, (uint32_t)(t + 1));
            r = cudaGetLastError();
        }
        return r;
    };
    auto reduce = [&](const float *a, int sq, int range, int z) {
        if (N == 0) return;
        unsigned b = std::min<unsigned>(nblk(N), (unsigned)c.n_sms * 8);
        adj_reduce_kernel<<<b, kAdjThreads, 0, st>>>(a, N, nc, dim, dsum, drange, drange + 4, dsum + 4, sq, range, z,
                                                     P.p_mass);
    };
    // forward with checkpoints; ranges over t = 0..T
    float *cur = tape, *nxt = tape + NE;
    if (e == cudaSuccess && N > 0) e = cudaMemcpyAsync(cur, ckpt, state_bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) reduce(cur, 0, 1, 0);
    for (int t = 0; t < T && e == cudaSuccess; ++t) {
        e = step_fwd(cur, nxt, t);
        std::swap(cur, nxt);
        if (e == cudaSuccess) reduce(cur, 0, 1, 0);
        if (e == cudaSuccess && !bisection && (t + 1) % k == 0 && (t + 1) / k < n_ckpt)
            e = cudaMemcpyAsync(ckpt + (size_t)((t + 1) / k) * NE, cur, state_bytes, cudaMemcpyDeviceToDevice, st);
    }
    // seed dz/ds_T
    if (e == cudaSuccess) {
        if (measure == QMPM_MEASURE_USER) {
            if (N > 0) e = cudaMemcpyAsync(sbA, d_seed, state_bytes, cudaMemcpyDeviceToDevice, st);
        } else if (N > 0) {
            adj_seed_kernel<<<nblk(N), kAdjThreads, 0, st>>>(cur, sbA, N, nc, dim, measure, P.p_mass);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) reduce(cur, 0, 0, measure == QMPM_MEASURE_KINETIC_ENERGY ? 2 : 1);  // z of s_T
    if (e == cudaSuccess) reduce(sbA, 1, 0, 0);  // t = T term of Eq. 8
    float *sbn = sbA, *sb = sbB;
    if (bisection) {
        // slot j of the schedule is checkpoint buffer j (slot 0 holds s_0); the recomputation
        // ping-pongs between its target slot and the scratch state `tape`
        for (size_t i = 0; i < sched.size() && e == cudaSuccess; ++i) {
            const qmpm_rev_op_t &op = sched[i];
            float *from = ckpt + (size_t)op.from * NE;
            if (op.kind == QMPM_OP_ADVANCE) {
                float *to = ckpt + (size_t)op.to * NE;
                const int n_adv = op.t1 - op.t0;
                // land on `to` after n_adv steps: start on the buffer of the right parity
                float *a = (n_adv % 2 == 1) ? to : tape, *b2 = (n_adv % 2 == 1) ? tape : to;
                const float *src = from;
                for (int j = 0; j < n_adv && e == cudaSuccess; ++j) {
                    float *dst = (j % 2 == 0) ? a : b2;
                    e = step_fwd(src, dst, op.t0 + j);
                    src = dst;
                }
            } else {
                e = rev(P, from, sbn, sb, N, gm, gv, gb, nn, st);
                if (e == cudaSuccess) reduce(sb, 1, 0, 0);
                std::swap(sbn, sb);
            }
        }
    }
    // backward over segments [t0, t1)
    for (int64_t seg = (!bisection && T > 0 ? (T - 1) / k : -1); seg >= 0 && e == cudaSuccess; --seg) {
        const int t0 = (int)(seg * k), t1 = std::min<int>(T, (int)(seg + 1) * k);
        if (N > 0) e = cudaMemcpyAsync(tape, ckpt + (size_t)seg * NE, state_bytes, cudaMemcpyDeviceToDevice, st);
        for (int t = t0; t < t1 - 1 && e == cudaSuccess; ++t)
            e = step_fwd(tape + (size_t)(t - t0) * NE, tape + (size_t)(t - t0 + 1) * NE, t);
        for (int t = t1 - 1; t >= t0 && e == cudaSuccess; --t) {
            e = rev(P, tape + (size_t)(t - t0) * NE, sbn, sb, N, gm, gv, gb, nn, st);
            if (e == cudaSuccess) reduce(sb, 1, 0, 0);
            std::swap(sbn, sb);
        }
    }
    if (e == cudaSuccess && d_grad0 && N > 0)
        e = cudaMemcpyAsync(d_grad0, sbn, state_bytes, cudaMemcpyDeviceToDevice, st);
    double hs[8];
    int hr[8];
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, dsum, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hr, drange, sizeof(hr), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) {
        set_last_error(std::string("qmpm_adjoint: ") + cudaGetErrorString(e));
        return QMPM_ERR_CUDA;
    }
    if (out) {
        std::memset(out, 0, sizeof(*out));
        out->z = hs[4];
        for (int q = 0; q < 4; ++q) {
            out->g[q] = hs[q];
            out->lo[q] = ordered_value(hr[q]);
            out->hi[q] = ordered_value(hr[4 + q]);
        }
        const int per[4] = {dim, dim, dim * dim, nc - 2 * dim - dim * dim};
        for (int q = 0; q < 4; ++q) out->P[q] = N * per[q];
        out->forward_steps = fwd_steps;
        out->state_buffers = (int32_t)(n_ckpt + tape_states);
    }
    return QMPM_OK;
}

namespace qmpm {
namespace {

// positions of the final state of a noise pair: m = (x+ + x-)/2 - x0 is added to acc, and
// sums[0] += |m|^2, sums[1] += |(x+ - x-)/2|^2 (FP64)
__global__ void noise_pair_kernel(const float *sp, const float *sm, const float *s0, int64_t N, int nc, int dim,
                                  float *acc, double *sums)
{
    double a = 0.0, b = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < dim; ++c) {
            const float xp = sp[p * nc + c], xm = sm[p * nc + c];
            const double m = 0.5 * ((double)xp + (double)xm) - (double)s0[p * nc + c];
            const double d = 0.5 * ((double)xp - (double)xm);
            acc[p * dim + c] += (float)m;
            a += m * m;
            b += d * d;
        }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xFFFFFFFFu, a, o);
        b += __shfl_down_sync(0xFFFFFFFFu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sums, a);
        atomicAdd(sums + 1, b);
    }
}

__global__ void sq_sum_kernel(const float *v, int64_t n, double scale, double *out)
{
    double a = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = (double)v[i] * scale;
        a += x * x;
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xFFFFFFFFu, a, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, a);
}

}  // namespace
}  // namespace qmpm

extern "C" int qmpm_noise_moments(qmpm_handle h, int32_t T, int32_t measure, const double *sigma, uint64_t seed0,
                                  int32_t n_pairs, qmpm_noise_out_t *out)
{
    using namespace qmpm;
    const int matched = (measure & QMPM_NOISE_MATCHED) ? 1 : 0;
    measure &= ~QMPM_NOISE_MATCHED;
    if (!h || T < 0 || n_pairs < 2 || !sigma || !out ||
        (measure != QMPM_MEASURE_MEAN_SQ_POS && measure != QMPM_MEASURE_KINETIC_ENERGY &&
         measure != QMPM_MEASURE_POSITIONS)) {
        set_last_error("qmpm_noise_moments: bad handle, T, measure, sigma, out or n_pairs (>= 2)");
        return QMPM_ERR_INVALID_ARG;
    }
    for (int q = 0; q < 4; ++q)
        if (!(sigma[q] >= 0.0) || (matched && sigma[q] > 0.0 && std::exp2(std::round(std::log2(sigma[q]))) != sigma[q])) {
            set_last_error("qmpm_noise_moments: sigma must be >= 0 (and powers of two, the resolutions, when matched)");
            return QMPM_ERR_INVALID_ARG;
        }
    Ctx &c = *h;
    const int dim = c.scene.dim, nc = c.n_comp;
    const int64_t N = c.N;
    const bool vec = measure == QMPM_MEASURE_POSITIONS;
    ForwardFn fwd;
    ReverseFn rev;
    pick(dim, c.scene.material, fwd, rev);
    StepParams P;
    fill_params(c, P);
    const int64_t nn = dim == 2 ? (int64_t)c.n * c.n : (int64_t)c.n * c.n * c.n;
    const size_t state_bytes = sizeof(float) * (size_t)std::max<int64_t>(N, 1) * nc;
    cudaStream_t st = c.stream;
    std::vector<void *> allocs;
    auto alloc = [&](size_t bytes) -> void * {
        void *ptr = nullptr;
        if (cudaMalloc(&ptr, bytes) != cudaSuccess) return nullptr;
        allocs.push_back(ptr);
        return ptr;
    };
    auto cleanup = [&]() {
        for (void *ptr : allocs) cudaFree(ptr);
    };
    // s0, two run buffers, the noise-free final state and the + run's final state (vector
    // measure), the accumulated shift vector, the grid
    float *s0 = static_cast<float *>(alloc(state_bytes));
    float *a = static_cast<float *>(alloc(state_bytes));
    float *b = static_cast<float *>(alloc(state_bytes));
    float *fin0 = vec ? static_cast<float *>(alloc(state_bytes)) : nullptr;
    float *finp = vec ? static_cast<float *>(alloc(state_bytes)) : nullptr;
    float *acc = vec ? static_cast<float *>(alloc(sizeof(float) * (size_t)std::max<int64_t>(N, 1) * dim)) : nullptr;
    float *gm = static_cast<float *>(alloc(sizeof(float) * (size_t)nn));
    float4 *gv = static_cast<float4 *>(alloc(sizeof(float4) * (size_t)nn));
    double *dz = static_cast<double *>(alloc(sizeof(double) * 8));
    if (!s0 || !a || !b || !gm || !gv || !dz || (vec && (!fin0 || !finp || !acc))) {
        cudaGetLastError();
        cleanup();
        set_last_error("qmpm_noise_moments: device allocation failed");
        return QMPM_ERR_OOM;
    }
    cudaError_t e = cudaSuccess;
    if (N > 0) {
        adj_load_kernel<<<nblk(N), kAdjThreads, 0, st>>>(P, c.quant ? 1 : 0, s0, N);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && vec) e = cudaMemsetAsync(acc, 0, sizeof(float) * (size_t)std::max<int64_t>(N, 1) * dim, st);
    const float4 sig = make_float4((float)sigma[0], (float)sigma[1], (float)sigma[2], (float)sigma[3]);
    const unsigned nbk = std::min<unsigned>(nblk(std::max<int64_t>(N, 1)), (unsigned)c.n_sms * 8);
    // a T-step run from s_0 with the noise of (seed, sign) or none (sign 0); the final state
    // is left in *final
    auto run = [&](uint64_t seed, float sign, float **final) -> cudaError_t {
        cudaError_t r = cudaMemcpyAsync(a, s0, state_bytes, cudaMemcpyDeviceToDevice, st);
        float *cur = a, *nxt = b;
        for (int t = 0; t < T && r == cudaSuccess; ++t) {
            r = fwd(P, cur, nxt, N, gm, gv, nn, st);
            if (r == cudaSuccess && sign != 0.0f && N > 0) {
                adj_noise_kernel<<<nblk(N), kAdjThreads, 0, st>>>(P, nxt, N, (uint32_t)(t + 1), (uint32_t)seed,
                                                                 (uint32_t)(seed >> 32), sig, sign, matched);
                r = cudaGetLastError();
            }
            std::swap(cur, nxt);
        }
        *final = cur;
        return r;
    };
    auto z_of = [&](const float *fin, double *zout) -> cudaError_t {
        cudaError_t r = cudaMemsetAsync(dz, 0, sizeof(double) * 8, st);
        if (r == cudaSuccess && N > 0) {
            adj_reduce_kernel<<<nbk, kAdjThreads, 0, st>>>(fin, N, nc, dim, dz, nullptr, nullptr, dz + 4, 0, 0,
                                                           measure == QMPM_MEASURE_KINETIC_ENERGY ? 2 : 1, P.p_mass);
            r = cudaGetLastError();
        }
        double hz[8];
        if (r == cudaSuccess) r = cudaMemcpyAsync(hz, dz, sizeof(hz), cudaMemcpyDeviceToHost, st);
        if (r == cudaSuccess) r = cudaStreamSynchronize(st);
        if (r == cudaSuccess) *zout = hz[4];
        return r;
    };
    double z0 = 0.0;
    std::vector<double> shift, spread;
    float *fin = nullptr;
    if (e == cudaSuccess) e = run(0, 0.0f, &fin);
    if (e == cudaSuccess) e = vec ? cudaMemcpyAsync(fin0, fin, state_bytes, cudaMemcpyDeviceToDevice, st) : z_of(fin, &z0);
    if (e == cudaSuccess && vec) e = z_of(fin0, &z0);
    for (int k = 0; k < n_pairs && e == cudaSuccess; ++k) {
        if (vec) {
            e = run(seed0 + (uint64_t)k, 1.0f, &fin);
            if (e == cudaSuccess) e = cudaMemcpyAsync(finp, fin, state_bytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = run(seed0 + (uint64_t)k, -1.0f, &fin);
            if (e == cudaSuccess) e = cudaMemsetAsync(dz, 0, sizeof(double) * 8, st);
            if (e == cudaSuccess && N > 0) {
                noise_pair_kernel<<<nbk, kAdjThreads, 0, st>>>(finp, fin, fin0, N, nc, dim, acc, dz);
                e = cudaGetLastError();
            }
            double hz[8];
            if (e == cudaSuccess) e = cudaMemcpyAsync(hz, dz, sizeof(hz), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            shift.push_back(hz[0]);   // |m_k|^2
            spread.push_back(hz[1]);  // sum |(x+ - x-)/2|^2
        } else {
            double zp = 0.0, zm = 0.0;
            e = run(seed0 + (uint64_t)k, 1.0f, &fin);
            if (e == cudaSuccess) e = z_of(fin, &zp);
            if (e == cudaSuccess) e = run(seed0 + (uint64_t)k, -1.0f, &fin);
            if (e == cudaSuccess) e = z_of(fin, &zm);
            shift.push_back(0.5 * (zp + zm) - z0);
            spread.push_back(0.25 * (zp - zm) * (zp - zm));
        }
    }
    double mean_sq = 0.0;  // |mean_k m_k|^2 (vector measure)
    if (e == cudaSuccess && vec) {
        e = cudaMemsetAsync(dz, 0, sizeof(double) * 8, st);
        if (e == cudaSuccess && N > 0) {
            sq_sum_kernel<<<nbk, kAdjThreads, 0, st>>>(acc, N * dim, 1.0 / n_pairs, dz);
            e = cudaGetLastError();
        }
        double hz[8];
        if (e == cudaSuccess) e = cudaMemcpyAsync(hz, dz, sizeof(hz), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        mean_sq = hz[0];
    }
    cleanup();
    if (e != cudaSuccess) {
        set_last_error(std::string("qmpm_noise_moments: ") + cudaGetErrorString(e));
        return QMPM_ERR_CUDA;
    }
    auto mean_se = [](const std::vector<double> &v, double &m, double &se) {
        m = 0.0;
        for (double x : v) m += x;
        m /= (double)v.size();
        double ss = 0.0;
        for (double x : v) ss += (x - m) * (x - m);
        se = std::sqrt(ss / (double)(v.size() - 1) / (double)v.size());
    };
    std::memset(out, 0, sizeof(*out));
    out->z0 = z0;
    mean_se(spread, out->spread, out->spread_se);
    if (vec) {
        // E|mean_k m_k|^2 = |b|^2 + E|m - b|^2 / K and E|m_k|^2 = |b|^2 + E|m - b|^2:
        // |b|^2 = (K |mean m|^2 - mean |m_k|^2) / (K - 1)
        double msq, msq_se;
        mean_se(shift, msq, msq_se);
        const double K = (double)n_pairs;
        out->shift = (K * mean_sq - msq) / (K - 1.0);
        out->shift_se = msq_se * K / (K - 1.0);  // scale of its noise: the per-pair spread of |m_k|^2
    } else {
        mean_se(shift, out->shift, out->shift_se);
    }
    out->pairs = n_pairs;
    return QMPM_OK;
}
