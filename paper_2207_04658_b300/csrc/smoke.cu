// smoke.cu -- the quantized 2D Eulerian smoke of the paper's second error-bounded
// experiment (Sec. 8.1): an advection-reflection solver (semi-Lagrangian advection along
// RK-3 paths, Jacobi pressure projection, reflection of the half-step velocity) whose
// velocity and pressure stores go through the dithered fixed-point codec (Sec. 3.1, Sec. 5)
// and live in HBM as bit streams, for a batch of independent scenes.
//
// Kernels (one CTA row of the grid per scene, blockIdx.y = scene):
//   forces      density source, buoyancy and inflow into an FP32 copy of v
//   advect_vel  u~ = A(u; u, dt/2) or u~2 = A(u^; u', dt/2), then the velocity store
//   divergence  FP32 div of a stored velocity
//   jacobi      one Jacobi sweep of the pressure Poisson equation, then the pressure store
//   gradsub     u - grad q on the interior faces, then the velocity store
//   reflect     u^ = 2 u' - u~, then the velocity store
//   advect_d    d = A(d; u', dt) (FP32)
//   advance     steps done += 1 (the kernels take the step index and the density buffer
//               parity from that device counter, so one captured step replays as is)
// A store is warp-cooperative: the 32 lanes of a warp hold 32 consecutive values of one
// field (rows padded to multiples of 32), encode them and assemble the `bits` words that
// hold them with warp OR-reductions, so each packed word is written whole by one lane.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "../../include/qmpm_smoke.h"

namespace qmpm {
namespace smoke {

constexpr int kT = 256;
constexpr int kSlots = 64;   // range-recording slots per scene and type (spreads the atomics)

struct Fld {
    uint32_t *p;   // scene 0's first word
    int64_t ss;    // words per scene
};

struct Params {
    int n, J, su;              // su: padded row length of u (n + 32)
    float dt, buoy, v_in, inv_h, h, h2;
    double hd, src[4];
    int quant, dither, ranges;
    CompCodec cc[2];           // 0 velocity, 1 pressure (word/shift unused)
    int bits[2];
    float sigma[2];
    Fld u, v, ut, vt, up, vp, q[2];
    float *vf, *div, *d[2];
    int64_t nvf_s, ncell_s;    // floats per scene of vf and of the cell arrays
    const uint2 *seed, *nseed;
    const float *sign;
    unsigned long long *sat;   // [S][2]
    unsigned int *lo, *hi;     // [S][2][kSlots], order-preserving keys of floats
    double *z;
    uint32_t *ctr;             // steps done
};

__device__ __forceinline__ unsigned int fkey(float x)
{
    const unsigned int u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// ---- packed bit streams --------------------------------------------------------------
__device__ __forceinline__ uint32_t get_code(const uint32_t *f, int64_t pidx, int bits, uint32_t mask)
{
    const int64_t b = pidx * bits;
    const uint32_t *w = f + (b >> 5);
    const int sh = (int)(b & 31);
    const uint64_t two = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    return (uint32_t)(two >> sh) & mask;
}

// All 32 lanes of the warp call this with pidx = 32 g + lane.
__device__ __forceinline__ void put_codes(uint32_t *f, int64_t pidx, uint32_t code, int bits)
{
    const int lane = threadIdx.x & 31;
    const int bo = lane * bits, w0 = bo >> 5, sh = bo & 31;
    const uint32_t lo = code << sh;
    const uint32_t hi = (sh + bits > 32) ? (code >> (32 - sh)) : 0u;
    uint32_t mine = 0u;
    for (int w = 0; w < bits; ++w) {
        const uint32_t part = (w == w0 ? lo : 0u) | (w == w0 + 1 ? hi : 0u);
        const uint32_t word = __reduce_or_sync(0xffffffffu, part);
        if (lane == w) mine = word;
    }
    if (lane < bits) f[(pidx >> 5) * bits + lane] = mine;
}

template <bool PK>
__device__ __forceinline__ float ld(const uint32_t *f, int64_t pidx, const CompCodec &c, int bits)
{
    if (PK) return decode_u(get_code(f, pidx, bits, c.mask), c);
    return __uint_as_float(f[pidx]);
}

// A lattice of nx x ny samples, row stride ld.
struct Lat {
    const uint32_t *f;
    int ld, nx, ny;
};

template <bool PK>
__device__ __forceinline__ float lat_at(const Lat &L, int i, int j, const CompCodec &c, int bits)
{
    return ld<PK>(L.f, (int64_t)j * L.ld + i, c, bits);
}

// Bilinear sample at lattice coordinates (gx, gy), clamped into the lattice.
template <bool PK>
__device__ __forceinline__ float sample(const Lat &L, float gx, float gy, const CompCodec &c, int bits)
{
    gx = fminf(fmaxf(gx, 0.0f), (float)(L.nx - 1));
    gy = fminf(fmaxf(gy, 0.0f), (float)(L.ny - 1));
    int i = (int)floorf(gx), j = (int)floorf(gy);
    i = min(max(i, 0), L.nx - 2);
    j = min(max(j, 0), L.ny - 2);
    const float fx = gx - (float)i, fy = gy - (float)j;
    const float a = lat_at<PK>(L, i, j, c, bits), b = lat_at<PK>(L, i + 1, j, c, bits);
    const float e = lat_at<PK>(L, i, j + 1, c, bits), g = lat_at<PK>(L, i + 1, j + 1, c, bits);
    return (1.0f - fy) * ((1.0f - fx) * a + fx * b) + fy * ((1.0f - fx) * e + fx * g);
}

// Velocity (u lattice PU, v lattice PV) at a point in domain units.
template <bool PU, bool PV>
__device__ __forceinline__ void vel_at(const Params &P, const Lat &U, const Lat &V, float x, float y, float &ux,
                                       float &vy)
{
    const float n = P.inv_h;
    ux = sample<PU>(U, x * n, y * n - 0.5f, P.cc[0], P.bits[0]);
    vy = sample<PV>(V, x * n - 0.5f, y * n, P.cc[0], P.bits[0]);
}

// Ralston's RK-3 backtrace over s.
template <bool PU, bool PV>
__device__ __forceinline__ void backtrace(const Params &P, const Lat &U, const Lat &V, float s, float x, float y,
                                          float &xb, float &yb)
{
    float k1x, k1y, k2x, k2y, k3x, k3y;
    vel_at<PU, PV>(P, U, V, x, y, k1x, k1y);
    vel_at<PU, PV>(P, U, V, x - 0.5f * s * k1x, y - 0.5f * s * k1y, k2x, k2y);
    vel_at<PU, PV>(P, U, V, x - 0.75f * s * k2x, y - 0.75f * s * k2y, k3x, k3y);
    xb = x - s * (2.0f * k1x + 3.0f * k2x + 4.0f * k3x) / 9.0f;
    yb = y - s * (2.0f * k1y + 3.0f * k2y + 4.0f * k3y) / 9.0f;
}

// Warp-reduced range keys into one of the scene's slots (whole warp calls).
__device__ __forceinline__ void record_range(const Params &P, int s, int type, unsigned kmin, unsigned kmax)
{
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    if ((threadIdx.x & 31) == 0) {
        const int64_t slot = ((int64_t)s * 2 + type) * kSlots + ((blockIdx.x * (kT / 32) + (threadIdx.x >> 5)) & (kSlots - 1));
        if (kmin != 0xffffffffu) atomicMin(P.lo + slot, kmin);
        if (kmax != 0u) atomicMax(P.hi + slot, kmax);
    }
}

// ---- the store ------------------------------------------------------------------------
// Called by every lane of a warp (valid = the lane holds a real sample).  Quantized: encode
// (dithered or nearest), count saturations, write the code to the packed stream and to the
// trace; returns the decoded value.  FP32: add the injected noise, write the float.  Both
// record the range of the values offered to the store.
template <bool Q>
__device__ __forceinline__ float store(const Params &P, int s, int type, int field, float x, uint32_t k,
                                       uint32_t counter, bool valid, bool wall, bool inject, uint32_t *out,
                                       int64_t pidx, uint32_t *trace)
{
    const unsigned full = 0xffffffffu;
    float y = x;
    if (Q) {
        const CompCodec &c = P.cc[type];
        uint32_t r = 0u;
        if (P.dither) {
            const uint2 key = P.seed[s];
            const uint4 blk = philox4x32_10(make_uint4(k >> 3, counter, (uint32_t)field, 0u), key.x, key.y);
            r = dither_threshold(blk, (int)(k & 7u));
        }
        int flags = 0;
        uint32_t code = encode_f32(x, c, P.dither != 0, r, flags);
        if (!valid) code = 0u;
        const unsigned satm = __ballot_sync(full, valid && (flags & 1));
        if (satm && (threadIdx.x & 31) == 0) atomicAdd(P.sat + 2 * s + type, (unsigned long long)__popc(satm));
        put_codes(out, pidx, code, P.bits[type]);
        if (trace && valid && s == 0) trace[k] = code;
        y = decode_u(code, c);
    } else {
        if (inject && !wall && P.sigma[type] != 0.0f) {
            const uint2 key = P.nseed[s];
            const uint4 blk = philox4x32_10(make_uint4(k >> 3, counter, (uint32_t)field, 0u), key.x, key.y);
            const uint32_t w = uint4_at(blk, (int)((k >> 1) & 3u));
            const uint32_t q16 = (k & 1u) ? (w >> 16) : (w & 0xFFFFu);
            y = x + P.sign[s] * P.sigma[type] * ((q16 & 0x8000u) ? 1.0f : -1.0f);
        }
        if (valid) out[pidx] = __float_as_uint(y);
    }
    if (P.ranges) record_range(P, s, type, valid ? fkey(x) : 0xffffffffu, valid ? fkey(x) : 0u);
    return y;
}

__device__ __forceinline__ bool in_box(const Params &P, double x, double y)
{
    return x >= P.src[0] && x <= P.src[2] && y >= P.src[1] && y <= P.src[3];
}

__device__ __forceinline__ uint32_t step_index(const Params &P) { return *P.ctr + 1u; }

// ---- kernels ---------------------------------------------------------------------------
template <bool Q>
__global__ void __launch_bounds__(kT) forces_kernel(Params P)
{
    const int s = blockIdx.y, n = P.n;
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    const uint32_t par = *P.ctr & 1u;
    float *d = P.d[par] + s * P.ncell_s;
    if (t < (int64_t)n * n) {
        const int i = (int)(t % n), j = (int)(t / n);
        if (in_box(P, (i + 0.5) * P.hd, (j + 0.5) * P.hd)) d[t] = 1.0f;
    }
    if (t < (int64_t)(n + 1) * n) {
        const int i = (int)(t % n), j = (int)(t / n);
        float vv = 0.0f;
        if (j > 0 && j < n) {
            vv = ld<Q>(P.v.p + s * P.v.ss, t, P.cc[0], P.bits[0]);
            const float d1 = in_box(P, (i + 0.5) * P.hd, (j + 0.5) * P.hd) ? 1.0f : d[(int64_t)j * n + i];
            const float d0 = in_box(P, (i + 0.5) * P.hd, (j - 0.5) * P.hd) ? 1.0f : d[(int64_t)(j - 1) * n + i];
            vv += P.dt * P.buoy * 0.5f * (d1 + d0);
            if (in_box(P, (i + 0.5) * P.hd, j * P.hd)) vv = P.v_in;
        }
        P.vf[s * P.nvf_s + t] = vv;
    }
}

// STAGE 1: f = w = (u, vf); out (ut, vt); store 1.   STAGE 4: f = (ut, vt), w = (up, vp);
// out (u, v); store J + 4.
template <bool Q, int STAGE>
__global__ void __launch_bounds__(kT) advect_vel_kernel(Params P, uint32_t *trace)
{
    constexpr bool PV = STAGE == 1 ? false : Q;
    const int s = blockIdx.y, n = P.n;
    const int64_t nu = (int64_t)n * P.su, nv = (int64_t)(n + 1) * n;
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t - (threadIdx.x & 31) >= nu + nv) return;  // whole warps only
    const uint32_t counter = 1024u * step_index(P) + (STAGE == 1 ? 1u : (uint32_t)P.J + 4u);
    const uint32_t *vsrc = STAGE == 1 ? reinterpret_cast<const uint32_t *>(P.vf + s * P.nvf_s) : P.vt.p + s * P.vt.ss;
    const Lat WU{STAGE == 1 ? P.u.p + s * P.u.ss : P.up.p + s * P.up.ss, P.su, n + 1, n};
    const Lat WV{STAGE == 1 ? vsrc : P.vp.p + s * P.vp.ss, n, n, n + 1};
    const Lat FU{STAGE == 1 ? P.u.p + s * P.u.ss : P.ut.p + s * P.ut.ss, P.su, n + 1, n};
    const Lat FV{vsrc, n, n, n + 1};
    const float half = 0.5f * P.dt;
    if (t < nu) {
        const int i = (int)(t % P.su), j = (int)(t / P.su);
        const bool valid = i <= n, wall = i == 0 || i == n;
        float x = 0.0f;
        if (valid && !wall) {
            float xb, yb;
            backtrace<Q, PV>(P, WU, WV, half, (float)i * P.h, ((float)j + 0.5f) * P.h, xb, yb);
            x = sample<Q>(FU, xb * P.inv_h, yb * P.inv_h - 0.5f, P.cc[0], P.bits[0]);
        }
        const uint32_t k = (uint32_t)(j * (n + 1) + i);
        Fld o = STAGE == 1 ? P.ut : P.u;
        store<Q>(P, s, 0, 0, x, k, counter, valid, wall, true, o.p + s * o.ss, t, trace);
    } else {
        const int64_t tv = t - nu;
        const int i = (int)(tv % n), j = (int)(tv / n);
        const bool wall = j == 0 || j == n;
        float x = 0.0f;
        if (!wall) {
            float xb, yb;
            backtrace<Q, PV>(P, WU, WV, half, ((float)i + 0.5f) * P.h, (float)j * P.h, xb, yb);
            x = sample<PV>(FV, xb * P.inv_h - 0.5f, yb * P.inv_h, P.cc[0], P.bits[0]);
        }
        const uint32_t k = (uint32_t)tv;
        Fld o = STAGE == 1 ? P.vt : P.v;
        store<Q>(P, s, 0, 1, x, k, counter, true, wall, true, o.p + s * o.ss, tv,
                 trace ? trace + (int64_t)(n + 1) * n : nullptr);
    }
}

template <bool Q>
__global__ void __launch_bounds__(kT) divergence_kernel(Params P, int which)  // 0: (ut, vt), 1: (u, v)
{
    const int s = blockIdx.y, n = P.n;
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t >= (int64_t)n * n) return;
    const int i = (int)(t % n), j = (int)(t / n);
    const Fld fu = which == 0 ? P.ut : P.u, fv = which == 0 ? P.vt : P.v;
    const uint32_t *u = fu.p + s * fu.ss, *v = fv.p + s * fv.ss;
    const CompCodec &c = P.cc[0];
    const int b = P.bits[0];
    const float ur = ld<Q>(u, (int64_t)j * P.su + i + 1, c, b), ul = ld<Q>(u, (int64_t)j * P.su + i, c, b);
    const float vt = ld<Q>(v, (int64_t)(j + 1) * n + i, c, b), vb = ld<Q>(v, (int64_t)j * n + i, c, b);
    P.div[s * P.ncell_s + t] = (ur - ul + vt - vb) * P.inv_h;
}

// Sweep it (1-based) of a projection: reads q[(it - 1) & 1] (zero for it = 1), writes
// q[it & 1]; store counter base + it.  A thread takes an octet, 8 consecutive cells of a
// row (n is a multiple of 32, so an octet never crosses a row), and draws one Philox block
// for all 8 (their dither counter is (cell / 8, counter, 2, 0), lanes cell % 8).  The warp's 256 codes are
// staged in shared memory and packed into its 8 * bits words by the lanes in turn.
template <bool Q>
__global__ void __launch_bounds__(kT) jacobi8_kernel(Params P, int it, uint32_t cbase, uint32_t *trace)
{
    __shared__ uint32_t stage[kT * 8];
    const int s = blockIdx.y, n = P.n, lane = threadIdx.x & 31;
    const int64_t nc = (int64_t)n * n;
    const int64_t o = (int64_t)blockIdx.x * kT + threadIdx.x;
    const int64_t t0 = o * 8;
    if (t0 - (int64_t)lane * 8 >= nc) return;  // whole warps (n^2 / 8 is a multiple of 32)
    const int i0 = (int)(t0 % n), j = (int)(t0 / n);
    const uint32_t *qi = P.q[(it - 1) & 1].p + s * P.q[0].ss;
    const CompCodec &c = P.cc[1];
    const int b = P.bits[1];
    const float4 *dv4 = reinterpret_cast<const float4 *>(P.div + s * P.ncell_s + t0);
    const float4 da = dv4[0], db = dv4[1];
    const float dv[8] = {da.x, da.y, da.z, da.w, db.x, db.y, db.z, db.w};
    float x[8];
    if (it > 1) {
        float row[10], dn[8], up[8];
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            const int ii = i0 - 1 + k;
            row[k] = (ii >= 0 && ii < n) ? ld<Q>(qi, (int64_t)j * n + ii, c, b) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            dn[k] = j > 0 ? ld<Q>(qi, (int64_t)(j - 1) * n + i0 + k, c, b) : 0.0f;
            up[k] = j < n - 1 ? ld<Q>(qi, (int64_t)(j + 1) * n + i0 + k, c, b) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = i0 + k;
            float acc = 0.0f;
            int cnt = 0;
            if (i > 0) { acc += row[k]; ++cnt; }
            if (i < n - 1) { acc += row[k + 2]; ++cnt; }
            if (j > 0) { acc += dn[k]; ++cnt; }
            if (j < n - 1) { acc += up[k]; ++cnt; }
            x[k] = (acc - P.h2 * dv[k]) / (float)cnt;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = i0 + k;
            const int cnt = (i > 0) + (i < n - 1) + (j > 0) + (j < n - 1);
            x[k] = (0.0f - P.h2 * dv[k]) / (float)cnt;
        }
    }
    const uint32_t counter = 1024u * step_index(P) + cbase + (uint32_t)it;
    uint32_t *qo = P.q[it & 1].p + s * P.q[0].ss;
    if (P.ranges) {
        unsigned kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            kmin = min(kmin, fkey(x[k]));
            kmax = max(kmax, fkey(x[k]));
        }
        record_range(P, s, 1, kmin, kmax);
    }
    if (Q) {
        uint4 blk = make_uint4(0u, 0u, 0u, 0u);
        if (P.dither) {
            const uint2 key = P.seed[s];
            blk = philox4x32_10(make_uint4((uint32_t)o, counter, 2u, 0u), key.x, key.y);
        }
        uint32_t code[8];
        int nsat = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            int flags = 0;
            code[k] = encode_f32(x[k], c, P.dither != 0, P.dither ? dither_threshold(blk, k) : 0u, flags);
            nsat += flags & 1;
        }
        nsat = __reduce_add_sync(0xffffffffu, nsat);
        if (nsat && lane == 0) atomicAdd(P.sat + 2 * s + 1, (unsigned long long)nsat);
        if (trace && s == 0) {
            uint4 *tw = reinterpret_cast<uint4 *>(trace + t0);
            tw[0] = make_uint4(code[0], code[1], code[2], code[3]);
            tw[1] = make_uint4(code[4], code[5], code[6], code[7]);
        }
        uint32_t *st = stage + (threadIdx.x >> 5) * 256;
#pragma unroll
        for (int k = 0; k < 8; ++k) st[lane * 8 + k] = code[k];
        __syncwarp();
        uint32_t *ow = qo + (t0 - (int64_t)lane * 8) / 32 * b;
        for (int w = lane; w < 8 * b; w += 32) {
            const int b0 = 32 * w, m1 = min((b0 + 31) / b, 255);
            uint32_t word = 0u;
            for (int m = b0 / b; m <= m1; ++m) {
                const int sh = m * b - b0;
                word |= sh >= 0 ? (st[m] << sh) : (st[m] >> -sh);
            }
            ow[w] = word;
        }
    } else {
        if (P.sigma[1] != 0.0f) {
            const uint2 key = P.nseed[s];
            const uint4 blk = philox4x32_10(make_uint4((uint32_t)o, counter, 2u, 0u), key.x, key.y);
            const float amp = P.sign[s] * P.sigma[1];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t w = uint4_at(blk, (k >> 1) & 3);
                const uint32_t q16 = (k & 1) ? (w >> 16) : (w & 0xFFFFu);
                x[k] += amp * ((q16 & 0x8000u) ? 1.0f : -1.0f);
            }
        }
        float4 *qw = reinterpret_cast<float4 *>(qo + t0);
        qw[0] = make_float4(x[0], x[1], x[2], x[3]);
        qw[1] = make_float4(x[4], x[5], x[6], x[7]);
    }
}

// out = in - grad q on interior faces (q = the last sweep's iterate; none when J = 0), then
// the velocity store.  STAGE 2: (ut, vt) -> (up, vp); STAGE 5: (u, v) in place.
template <bool Q, int STAGE>
__global__ void __launch_bounds__(kT) gradsub_kernel(Params P, uint32_t *trace)
{
    const int s = blockIdx.y, n = P.n;
    const int64_t nu = (int64_t)n * P.su, nv = (int64_t)(n + 1) * n;
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t - (threadIdx.x & 31) >= nu + nv) return;
    const uint32_t counter = 1024u * step_index(P) + (STAGE == 2 ? (uint32_t)P.J + 2u : 2u * (uint32_t)P.J + 5u);
    const uint32_t *q = P.q[P.J & 1].p + s * P.q[0].ss;
    const CompCodec &cq = P.cc[1];
    const int bq = P.bits[1];
    const Fld fin_u = STAGE == 2 ? P.ut : P.u, fin_v = STAGE == 2 ? P.vt : P.v;
    const Fld fo_u = STAGE == 2 ? P.up : P.u, fo_v = STAGE == 2 ? P.vp : P.v;
    if (t < nu) {
        const int i = (int)(t % P.su), j = (int)(t / P.su);
        const bool valid = i <= n, wall = i == 0 || i >= n;
        float x = 0.0f;
        if (valid && !wall) {
            x = ld<Q>(fin_u.p + s * fin_u.ss, t, P.cc[0], P.bits[0]);
            if (P.J > 0) x -= (ld<Q>(q, (int64_t)j * n + i, cq, bq) - ld<Q>(q, (int64_t)j * n + i - 1, cq, bq)) * P.inv_h;
        }
        store<Q>(P, s, 0, 0, x, (uint32_t)(j * (n + 1) + i), counter, valid, wall, true, fo_u.p + s * fo_u.ss, t,
                 trace);
    } else {
        const int64_t tv = t - nu;
        const int i = (int)(tv % n), j = (int)(tv / n);
        const bool wall = j == 0 || j == n;
        float x = 0.0f;
        if (!wall) {
            x = ld<Q>(fin_v.p + s * fin_v.ss, tv, P.cc[0], P.bits[0]);
            if (P.J > 0) x -= (ld<Q>(q, (int64_t)j * n + i, cq, bq) - ld<Q>(q, (int64_t)(j - 1) * n + i, cq, bq)) * P.inv_h;
        }
        store<Q>(P, s, 0, 1, x, (uint32_t)tv, counter, true, wall, true, fo_v.p + s * fo_v.ss, tv,
                 trace ? trace + (int64_t)(n + 1) * n : nullptr);
    }
}

// u^ = 2 u' - u~ into (ut, vt), store J + 3 (no noise: the value of two stored values of
// one lattice is itself on it).
template <bool Q>
__global__ void __launch_bounds__(kT) reflect_kernel(Params P, uint32_t *trace)
{
    const int s = blockIdx.y, n = P.n;
    const int64_t nu = (int64_t)n * P.su, nv = (int64_t)(n + 1) * n;
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t - (threadIdx.x & 31) >= nu + nv) return;
    const uint32_t counter = 1024u * step_index(P) + (uint32_t)P.J + 3u;
    const CompCodec &c = P.cc[0];
    const int b = P.bits[0];
    if (t < nu) {
        const int i = (int)(t % P.su), j = (int)(t / P.su);
        const bool valid = i <= n;
        float x = 0.0f;
        if (valid) x = 2.0f * ld<Q>(P.up.p + s * P.up.ss, t, c, b) - ld<Q>(P.ut.p + s * P.ut.ss, t, c, b);
        store<Q>(P, s, 0, 0, x, (uint32_t)(j * (n + 1) + i), counter, valid, i == 0 || i == n, false,
                 P.ut.p + s * P.ut.ss, t, trace);
    } else {
        const int64_t tv = t - nu;
        const int j = (int)(tv / n);
        const float x = 2.0f * ld<Q>(P.vp.p + s * P.vp.ss, tv, c, b) - ld<Q>(P.vt.p + s * P.vt.ss, tv, c, b);
        store<Q>(P, s, 0, 1, x, (uint32_t)tv, counter, true, j == 0 || j == n, false, P.vt.p + s * P.vt.ss, tv,
                 trace ? trace + (int64_t)(n + 1) * n : nullptr);
    }
}

template <bool Q>
__global__ void __launch_bounds__(kT) advect_d_kernel(Params P)
{
    const int s = blockIdx.y, n = P.n;
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t >= (int64_t)n * n) return;
    const int i = (int)(t % n), j = (int)(t / n);
    const uint32_t par = *P.ctr & 1u;
    const Lat WU{P.up.p + s * P.up.ss, P.su, n + 1, n};
    const Lat WV{P.vp.p + s * P.vp.ss, n, n, n + 1};
    const Lat D{reinterpret_cast<const uint32_t *>(P.d[par] + s * P.ncell_s), n, n, n};
    float xb, yb;
    backtrace<Q, Q>(P, WU, WV, P.dt, ((float)i + 0.5f) * P.h, ((float)j + 0.5f) * P.h, xb, yb);
    P.d[par ^ 1u][s * P.ncell_s + t] = sample<false>(D, xb * P.inv_h - 0.5f, yb * P.inv_h - 0.5f, P.cc[0], 0);
}

__global__ void advance_kernel(uint32_t *ctr) { *ctr += 1u; }

__global__ void __launch_bounds__(kT) measure_kernel(Params P)
{
    const int s = blockIdx.y, n = P.n;
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    const float *d = P.d[*P.ctr & 1u] + s * P.ncell_s;
    double acc = 0.0;
    for (int64_t c = t; c < (int64_t)n * n; c += (int64_t)gridDim.x * kT) acc += (double)d[c] * (double)d[c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double part[kT / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < kT / 32; ++w) a += part[w];
        atomicAdd(P.z + s, a);
    }
}

// Host FP32 state (oracle layout) -> stored fields; nearest rounding, walls zero.
template <bool Q>
__global__ void __launch_bounds__(kT) set_state_kernel(Params P, int s, const float *u, const float *v, const float *d)
{
    const int n = P.n;
    const int64_t nu = (int64_t)n * P.su, nv = (int64_t)(n + 1) * n;
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t - (threadIdx.x & 31) >= nu + nv) return;
    const uint32_t par = *P.ctr & 1u;
    if (t < (int64_t)n * n) P.d[par][s * P.ncell_s + t] = d ? d[t] : 0.0f;
    CompCodec c = P.cc[0];
    uint32_t *out;
    int64_t pidx;
    float x = 0.0f;
    bool valid = true;
    if (t < nu) {
        const int i = (int)(t % P.su), j = (int)(t / P.su);
        valid = i <= n;
        if (valid && i > 0 && i < n && u) x = u[(int64_t)j * (n + 1) + i];
        out = P.u.p + s * P.u.ss;
        pidx = t;
    } else {
        const int64_t tv = t - nu;
        const int j = (int)(tv / n);
        if (j > 0 && j < n && v) x = v[tv];
        out = P.v.p + s * P.v.ss;
        pidx = tv;
    }
    if (Q) {
        int flags = 0;
        uint32_t code = encode_f32(x, c, false, 0u, flags);
        if (!valid) code = 0u;
        put_codes(out, pidx, code, P.bits[0]);
    } else if (valid) {
        out[pidx] = __float_as_uint(x);
    }
}

// Stored fields of scene s -> FP32 arrays in the oracle layout (q: the final iterate).
template <bool Q>
__global__ void __launch_bounds__(kT) readback_kernel(Params P, int s, float *u, float *v, float *d, float *q)
{
    const int n = P.n;
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    const int64_t nu = (int64_t)n * (n + 1);
    if (t < nu) {
        const int i = (int)(t % (n + 1)), j = (int)(t / (n + 1));
        u[t] = ld<Q>(P.u.p + s * P.u.ss, (int64_t)j * P.su + i, P.cc[0], P.bits[0]);
        v[t] = ld<Q>(P.v.p + s * P.v.ss, t, P.cc[0], P.bits[0]);
    }
    if (t < (int64_t)n * n) {
        d[t] = P.d[*P.ctr & 1u][s * P.ncell_s + t];
        q[t] = P.J > 0 ? ld<Q>(P.q[P.J & 1].p + s * P.q[0].ss, t, P.cc[1], P.bits[1]) : 0.0f;
    }
}

}  // namespace smoke
}  // namespace qmpm

using namespace qmpm;
using namespace qmpm::smoke;

struct qmpm_smoke {
    Params p{};
    cudaStream_t st = nullptr;
    bool own_stream = false;       // created here: graphs cannot capture the legacy stream
    int S = 0;
    bool quant = false;
    std::vector<void *> allocs;
    uint32_t *stage = nullptr;     // device staging for set_state / readback (FP32)
    int64_t stage_floats = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t steps = 0, launches = 0, graph_launches = 0, device_bytes = 0;
};

namespace {

int fail(int code, const std::string &msg)
{
    qmpm::set_last_error(msg);
    return code;
}

int cuda_fail(const char *where, cudaError_t e)
{
    return fail(QMPM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int64_t round4(int64_t x) { return (x + 3) & ~(int64_t)3; }

int make_codec(int bits, int frac, int64_t offset, CompCodec &c)
{
    if (bits < 1 || bits > QMPM_MAX_FIELD_BITS || offset <= -(int64_t(1) << 24) || offset >= (int64_t(1) << 24) ||
        frac < -60 || frac > 60)
        return -1;
    c = CompCodec{};
    c.mask = (bits == 32) ? 0xFFFFFFFFu : ((1u << bits) - 1u);
    c.umax = c.mask;
    c.offset = (int32_t)offset;
    c.enc_scale = ldexpf(1.0f, frac);
    c.dec_scale = ldexpf(1.0f, -frac);
    c.dec_bias = (float)offset * c.dec_scale;
    return 0;
}

unsigned launches_per_step(int J) { return 11u + 2u * (unsigned)J; }

template <bool Q>
int enqueue_step(qmpm_smoke *h, uint32_t *trace)
{
    Params &P = h->p;
    const int n = P.n, J = P.J, S = h->S;
    const int64_t nfaces = (int64_t)n * P.su + (int64_t)(n + 1) * n;
    const dim3 gf((unsigned)((nfaces + kT - 1) / kT), S);
    const dim3 gc((unsigned)(((int64_t)n * n + kT - 1) / kT), S);
    const dim3 g8((unsigned)(((int64_t)n * n / 8 + kT - 1) / kT), S);
    const dim3 gv((unsigned)(((int64_t)(n + 1) * n + kT - 1) / kT), S);
    const int64_t V = 2 * (int64_t)n * (n + 1), Pq = (int64_t)n * n;
    auto tr = [&](int64_t off) { return trace ? trace + off : nullptr; };
    forces_kernel<Q><<<gv, kT, 0, h->st>>>(P);
    advect_vel_kernel<Q, 1><<<gf, kT, 0, h->st>>>(P, tr(0));
    divergence_kernel<Q><<<gc, kT, 0, h->st>>>(P, 0);
    for (int it = 1; it <= J; ++it) jacobi8_kernel<Q><<<g8, kT, 0, h->st>>>(P, it, 1u, tr(V + (it - 1) * Pq));
    gradsub_kernel<Q, 2><<<gf, kT, 0, h->st>>>(P, tr(V + J * Pq));
    reflect_kernel<Q><<<gf, kT, 0, h->st>>>(P, tr(2 * V + J * Pq));
    advect_vel_kernel<Q, 4><<<gf, kT, 0, h->st>>>(P, tr(3 * V + J * Pq));
    divergence_kernel<Q><<<gc, kT, 0, h->st>>>(P, 1);
    for (int it = 1; it <= J; ++it)
        jacobi8_kernel<Q><<<g8, kT, 0, h->st>>>(P, it, (uint32_t)J + 4u, tr(4 * V + (J + it - 1) * Pq));
    gradsub_kernel<Q, 5><<<gf, kT, 0, h->st>>>(P, tr(4 * V + 2 * J * Pq));
    advect_d_kernel<Q><<<gc, kT, 0, h->st>>>(P);
    advance_kernel<<<1, 1, 0, h->st>>>(P.ctr);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_step", e);
    h->launches += launches_per_step(J);
    return QMPM_OK;
}

int enqueue(qmpm_smoke *h, uint32_t *trace)
{
    return h->quant ? enqueue_step<true>(h, trace) : enqueue_step<false>(h, trace);
}

void drop_graph(qmpm_smoke *h)
{
    if (h->exec) cudaGraphExecDestroy(h->exec);
    h->exec = nullptr;
}

}  // namespace

extern "C" {

int qmpm_smoke_create(const qmpm_smoke_config_t *cfg, const qmpm_smoke_scheme_t *scheme, int32_t n_scenes,
                      const uint64_t *h_seeds, void *stream, qmpm_smoke_handle *out)
{
    if (!cfg || !out) return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_create: NULL argument");
    *out = nullptr;
    const int n = cfg->n;
    if (n < 32 || n > 4096 || n % 32 != 0 || cfg->jacobi < 0 || cfg->jacobi > 500 || n_scenes < 1 ||
        n_scenes > 4096 || !(cfg->dt > 0.0f))
        return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_create: n must be a multiple of 32 in 32..4096, jacobi "
                                          "0..500, n_scenes 1..4096, dt > 0");
    auto *h = new qmpm_smoke();
    h->st = (cudaStream_t)stream;
    if (!h->st) {
        if (cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return fail(QMPM_ERR_CUDA, "qmpm_smoke_create: stream creation failed");
        }
        h->own_stream = true;
    }
    h->S = n_scenes;
    h->quant = scheme != nullptr;
    Params &P = h->p;
    P.n = n;
    P.J = cfg->jacobi;
    P.su = n + 32;
    P.dt = cfg->dt;
    P.buoy = cfg->buoyancy;
    P.v_in = cfg->v_in;
    P.inv_h = (float)n;
    P.h = 1.0f / (float)n;
    P.h2 = 1.0f / ((float)n * (float)n);
    P.hd = 1.0 / n;
    for (int k = 0; k < 4; ++k) P.src[k] = cfg->src[k];
    P.quant = h->quant;
    P.dither = h->quant && cfg->dither;
    P.ranges = (cfg->flags & QMPM_SMOKE_RANGES) != 0;
    P.bits[0] = P.bits[1] = 32;
    if (h->quant) {
        for (int t = 0; t < 2; ++t) {
            if (make_codec(scheme->bits[t], scheme->frac[t], scheme->offset[t], P.cc[t])) {
                delete h;
                return fail(QMPM_ERR_SCHEME, "qmpm_smoke_create: bits outside 1..24 or |offset| >= 2^24");
            }
            P.bits[t] = scheme->bits[t];
        }
    }
    const int64_t nu = (int64_t)n * P.su, nv = (int64_t)(n + 1) * n, nc = (int64_t)n * n;
    auto words = [&](int64_t count, int t) {
        return round4(h->quant ? count / 32 * P.bits[t] + 2 : count + 2);
    };
    const int64_t wu = words(nu, 0), wv = words(nv, 0), wq = words(nc, 1);
    P.nvf_s = round4(nv);
    P.ncell_s = round4(nc);
    const int64_t S = n_scenes;
    bool ok = true;
    auto alloc = [&](size_t bytes) -> void * {
        void *ptr = nullptr;
        if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            ok = false;
            return nullptr;
        }
        h->allocs.push_back(ptr);
        h->device_bytes += (int64_t)bytes;
        return ptr;
    };
    auto fld = [&](int64_t w) { return Fld{(uint32_t *)alloc(sizeof(uint32_t) * w * S), w}; };
    P.u = fld(wu);
    P.v = fld(wv);
    P.ut = fld(wu);
    P.vt = fld(wv);
    P.up = fld(wu);
    P.vp = fld(wv);
    P.q[0] = fld(wq);
    P.q[1] = fld(wq);
    P.vf = (float *)alloc(sizeof(float) * P.nvf_s * S);
    P.div = (float *)alloc(sizeof(float) * P.ncell_s * S);
    P.d[0] = (float *)alloc(sizeof(float) * P.ncell_s * S);
    P.d[1] = (float *)alloc(sizeof(float) * P.ncell_s * S);
    uint2 *seeds = (uint2 *)alloc(sizeof(uint2) * S);
    uint2 *nseeds = (uint2 *)alloc(sizeof(uint2) * S);
    float *signs = (float *)alloc(sizeof(float) * S);
    P.sat = (unsigned long long *)alloc(sizeof(unsigned long long) * 2 * S);
    P.lo = (unsigned int *)alloc(sizeof(unsigned int) * 2 * kSlots * S);
    P.hi = (unsigned int *)alloc(sizeof(unsigned int) * 2 * kSlots * S);
    P.z = (double *)alloc(sizeof(double) * S);
    P.ctr = (uint32_t *)alloc(sizeof(uint32_t));
    h->stage_floats = 2 * nv + 2 * nc + 64;
    h->stage = (uint32_t *)alloc(sizeof(float) * h->stage_floats);
    if (!ok) {
        qmpm_smoke_destroy(h);
        return fail(QMPM_ERR_OOM, "qmpm_smoke_create: device allocation failed");
    }
    P.seed = seeds;
    P.nseed = nseeds;
    P.sign = signs;
    std::vector<uint2> hs(S);
    for (int64_t s = 0; s < S; ++s) {
        const uint64_t v = h_seeds ? h_seeds[s] : (uint64_t)s;
        hs[s] = make_uint2((uint32_t)v, (uint32_t)(v >> 32));
    }
    std::vector<unsigned int> lo(2 * kSlots * S, 0xffffffffu);
    cudaError_t e = cudaMemcpyAsync(seeds, hs.data(), sizeof(uint2) * S, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(nseeds, 0, sizeof(uint2) * S, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(signs, 0, sizeof(float) * S, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.sat, 0, sizeof(unsigned long long) * 2 * S, h->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.lo, lo.data(), sizeof(unsigned int) * 2 * kSlots * S, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.hi, 0, sizeof(unsigned int) * 2 * kSlots * S, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.ctr, 0, sizeof(uint32_t), h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        qmpm_smoke_destroy(h);
        return cuda_fail("qmpm_smoke_create", e);
    }
    // the temporaries start at zero; u, v and d are written by set_state below
    for (void *ptr : {(void *)P.ut.p, (void *)P.vt.p, (void *)P.up.p, (void *)P.vp.p, (void *)P.q[0].p,
                      (void *)P.q[1].p}) {
        const int64_t w = ptr == P.q[0].p || ptr == P.q[1].p ? wq : (ptr == P.ut.p || ptr == P.up.p ? wu : wv);
        if (e == cudaSuccess) e = cudaMemsetAsync(ptr, 0, sizeof(uint32_t) * w * S, h->st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(P.vf, 0, sizeof(float) * P.nvf_s * S, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.div, 0, sizeof(float) * P.ncell_s * S, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.d[1], 0, sizeof(float) * P.ncell_s * S, h->st);
    if (e != cudaSuccess) {
        qmpm_smoke_destroy(h);
        return cuda_fail("qmpm_smoke_create", e);
    }
    *out = h;
    const int r = qmpm_smoke_set_state(h, -1, nullptr, nullptr, nullptr);
    if (r != QMPM_OK) {
        qmpm_smoke_destroy(h);
        *out = nullptr;
        return r;
    }
    return QMPM_OK;
}

int qmpm_smoke_set_state(qmpm_smoke_handle h, int32_t scene, const float *h_u, const float *h_v, const float *h_d)
{
    if (!h || scene < -1 || scene >= h->S) return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_set_state: bad scene");
    const Params &P = h->p;
    const int n = P.n;
    const int64_t nu = (int64_t)n * (n + 1), nc = (int64_t)n * n;
    float *du = (float *)h->stage, *dv = du + nu, *dd = dv + nu;
    cudaError_t e = cudaSuccess;
    if (h_u) e = cudaMemcpyAsync(du, h_u, sizeof(float) * nu, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess && h_v) e = cudaMemcpyAsync(dv, h_v, sizeof(float) * nu, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess && h_d) e = cudaMemcpyAsync(dd, h_d, sizeof(float) * nc, cudaMemcpyHostToDevice, h->st);
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_set_state", e);
    const int64_t nfaces = (int64_t)n * P.su + (int64_t)(n + 1) * n;
    const dim3 g((unsigned)((nfaces + kT - 1) / kT));
    for (int s = (scene < 0 ? 0 : scene); s < (scene < 0 ? h->S : scene + 1); ++s) {
        if (h->quant)
            set_state_kernel<true><<<g, kT, 0, h->st>>>(P, s, h_u ? du : nullptr, h_v ? dv : nullptr, h_d ? dd : nullptr);
        else
            set_state_kernel<false><<<g, kT, 0, h->st>>>(P, s, h_u ? du : nullptr, h_v ? dv : nullptr, h_d ? dd : nullptr);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_set_state", e);
    return QMPM_OK;
}

int qmpm_smoke_set_noise(qmpm_smoke_handle h, const float sigma[2], const uint64_t *h_noise_seeds, const float *h_signs)
{
    if (!h || !sigma || h->quant || !h_noise_seeds || !h_signs)
        return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_set_noise: needs an FP32 handle, sigma, seeds and signs");
    std::vector<uint2> ns(h->S);
    for (int s = 0; s < h->S; ++s) ns[s] = make_uint2((uint32_t)h_noise_seeds[s], (uint32_t)(h_noise_seeds[s] >> 32));
    cudaError_t e = cudaMemcpyAsync((void *)h->p.nseed, ns.data(), sizeof(uint2) * h->S, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)h->p.sign, h_signs, sizeof(float) * h->S, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_set_noise", e);
    h->p.sigma[0] = sigma[0];
    h->p.sigma[1] = sigma[1];
    drop_graph(h);  // sigma is a kernel argument
    return QMPM_OK;
}

int qmpm_smoke_step(qmpm_smoke_handle h, int32_t steps, uint32_t *d_trace, int64_t trace_len)
{
    if (!h || steps < 0) return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_step: bad handle or steps");
    const int n = h->p.n, J = h->p.J;
    const int64_t per = 10 * (int64_t)n * (n + 1) + 2 * (int64_t)J * n * n;
    if (d_trace) {
        if (!h->quant || trace_len < per * steps)
            return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_step: trace needs a quantized handle and steps x "
                                              "(10 n (n+1) + 2 jacobi n^2) codes");
        for (int t = 0; t < steps; ++t) {
            const int r = enqueue(h, d_trace + per * t);
            if (r != QMPM_OK) return r;
            ++h->steps;
        }
        return QMPM_OK;
    }
    if (steps == 0) return QMPM_OK;
    if (!h->exec) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail("qmpm_smoke_step: capture", e);
        const int r = enqueue(h, nullptr);
        e = cudaStreamEndCapture(h->st, &g);
        if (r != QMPM_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->exec = nullptr;
            return cuda_fail("qmpm_smoke_step: graph", e);
        }
    }
    for (int t = 0; t < steps; ++t) {
        const cudaError_t e = cudaGraphLaunch(h->exec, h->st);
        if (e != cudaSuccess) return cuda_fail("qmpm_smoke_step: graph launch", e);
        ++h->graph_launches;
        ++h->steps;
    }
    return QMPM_OK;
}

int qmpm_smoke_measure(qmpm_smoke_handle h, double *h_z)
{
    if (!h || !h_z) return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_measure: NULL argument");
    cudaError_t e = cudaMemsetAsync(h->p.z, 0, sizeof(double) * h->S, h->st);
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_measure", e);
    const int n = h->p.n;
    const unsigned gx = (unsigned)std::min<int64_t>(((int64_t)n * n + kT - 1) / kT, 64);
    measure_kernel<<<dim3(gx, h->S), kT, 0, h->st>>>(h->p);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_z, h->p.z, sizeof(double) * h->S, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_measure", e);
    return QMPM_OK;
}

int qmpm_smoke_readback(qmpm_smoke_handle h, int32_t scene, float *h_u, float *h_v, float *h_d, float *h_q)
{
    if (!h || scene < 0 || scene >= h->S) return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_readback: bad scene");
    const int n = h->p.n;
    const int64_t nu = (int64_t)n * (n + 1), nc = (int64_t)n * n;
    float *du = (float *)h->stage, *dv = du + nu, *dd = dv + nu, *dq = dd + nc;
    const unsigned g = (unsigned)((nu + kT - 1) / kT);
    if (h->quant)
        readback_kernel<true><<<g, kT, 0, h->st>>>(h->p, scene, du, dv, dd, dq);
    else
        readback_kernel<false><<<g, kT, 0, h->st>>>(h->p, scene, du, dv, dd, dq);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && h_u) e = cudaMemcpyAsync(h_u, du, sizeof(float) * nu, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess && h_v) e = cudaMemcpyAsync(h_v, dv, sizeof(float) * nu, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess && h_d) e = cudaMemcpyAsync(h_d, dd, sizeof(float) * nc, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess && h_q) e = cudaMemcpyAsync(h_q, dq, sizeof(float) * nc, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_readback", e);
    return QMPM_OK;
}

int qmpm_smoke_ranges(qmpm_smoke_handle h, float *h_lo, float *h_hi, int64_t *h_sat)
{
    if (!h) return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_ranges: NULL handle");
    const int S = h->S;
    std::vector<unsigned int> lo(2 * kSlots * S), hi(2 * kSlots * S);
    std::vector<unsigned long long> sat(2 * S);
    cudaError_t e =
        cudaMemcpyAsync(lo.data(), h->p.lo, sizeof(unsigned) * 2 * kSlots * S, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hi.data(), h->p.hi, sizeof(unsigned) * 2 * kSlots * S, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sat.data(), h->p.sat, sizeof(unsigned long long) * 2 * S, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_ranges", e);
    auto unkey = [](unsigned k) {
        const unsigned u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
        float f;
        std::memcpy(&f, &u, 4);
        return f;
    };
    for (int i = 0; i < 2 * S; ++i) {
        unsigned kl = 0xffffffffu, kh = 0u;
        for (int k = 0; k < kSlots; ++k) {
            kl = std::min(kl, lo[(int64_t)i * kSlots + k]);
            kh = std::max(kh, hi[(int64_t)i * kSlots + k]);
        }
        if (h_lo) h_lo[i] = kl == 0xffffffffu ? 0.0f : unkey(kl);
        if (h_hi) h_hi[i] = kh == 0u ? 0.0f : unkey(kh);
        if (h_sat) h_sat[i] = (int64_t)sat[i];
    }
    return QMPM_OK;
}

int qmpm_smoke_info(qmpm_smoke_handle h, qmpm_smoke_info_t *out)
{
    if (!h || !out) return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_info: NULL argument");
    const int n = h->p.n;
    std::memset(out, 0, sizeof(*out));
    out->n = n;
    out->jacobi = h->p.J;
    out->n_scenes = h->S;
    out->quantized = h->quant;
    out->steps = h->steps;
    const int64_t nvel = 2 * (int64_t)n * (n + 1), nc = (int64_t)n * n;
    out->state_bytes_fp32 = 4 * (nvel + nc);
    out->state_bytes = h->quant ? (nvel * h->p.bits[0] + 7) / 8 + 4 * nc : out->state_bytes_fp32;
    out->device_bytes = h->device_bytes;
    out->kernel_launches = h->launches;
    out->graph_launches = h->graph_launches;
    out->launches_per_step = (int32_t)launches_per_step(h->p.J);
    return QMPM_OK;
}

int qmpm_smoke_destroy(qmpm_smoke_handle h)
{
    if (!h) return QMPM_OK;
    cudaStreamSynchronize(h->st);
    drop_graph(h);
    for (void *p : h->allocs) cudaFree(p);
    if (h->own_stream) cudaStreamDestroy(h->st);
    delete h;
    return QMPM_OK;
}

}  // extern "C"
