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
//   gradsub     u - grad q on the interior faces, then the velocity store (after the first
//               projection also the reflection u^ = 2 u' - u~ and its store)
//   advect_d    d = A(d; u', dt) (FP32)
//   advance     steps done += 1 (the kernels take the step index and the density buffer
//               parity from that device counter, so one captured step replays as is)
// A store is warp-cooperative: the 32 lanes of a warp hold 32 consecutive values of one
// field (rows padded to multiples of 32), encode them and assemble the `bits` words that
// hold them with warp OR-reductions, so each packed word is written whole by one lane.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "../../include/qmpm_smoke.h"

namespace qmpm {
namespace smoke {

constexpr int kT = 256;
constexpr int kSlots = 64;   // range-recording slots per scene and type (spreads the atomics)
constexpr int kMeasureBlocks = 64;  // blocks per scene of the z reduction

struct Fld {
    uint32_t *p;   // scene 0's first word
    int64_t ss;    // words per scene
};

struct Params {
    int n, J, su;              // su: padded row length of u (n + 32)
    int qfin;                  // buffer holding a projection's last iterate
    float dt, buoy, v_in, inv_h, h2;
    int box[6];                // source box as index ranges (inclusive): cell x, cell y, v-face y
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
    double *z;                 // [S][kMeasureBlocks] partial sums of d^2
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
    const uint32_t b = (uint32_t)pidx * (uint32_t)bits;  // a scene's stream holds < 2^32 bits
    const uint32_t *w = f + (b >> 5);
    const int sh = (int)(b & 31u);
    const uint64_t two = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    return (uint32_t)(two >> sh) & mask;
}

// All 32 lanes of the warp call this with pidx = 32 g + lane: the codes go through the
// warp's 32 shared slots, and lane w < bits assembles word w of the group from the (at most
// 32 / bits + 2) codes that overlap it.
__device__ __forceinline__ void put_codes(uint32_t *f, int64_t pidx, uint32_t code, int bits)
{
    __shared__ uint32_t slots[kT];
    const int lane = threadIdx.x & 31;
    uint32_t *sl = slots + (threadIdx.x & ~31);
    __syncwarp();  // the previous call's reads are done
    sl[lane] = code;
    __syncwarp();
    if (lane < bits) {
        const int b0 = 32 * lane, m1 = min((b0 + 31) / bits, 31);
        uint32_t word = 0u;
        for (int m = b0 / bits; m <= m1; ++m) {
            const int sh = m * bits - b0;
            word |= sh >= 0 ? (sl[m] << sh) : (sl[m] >> -sh);
        }
        f[(pidx >> 5) * bits + lane] = word;
    }
}

template <bool PK>
__device__ __forceinline__ float ld(const uint32_t *f, int64_t pidx, const CompCodec &c, int bits)
{
    if (PK) return decode_u(get_code(f, pidx, bits, c.mask), c);
    return __uint_as_float(f[pidx]);
}

// Eight consecutive values from index p0 (a multiple of 8): packed codes read once through a
// 64-bit shift register (every refill brings 32 bits, so a code of at most 24 bits is
// always whole), or two float4 loads.
template <bool PK>
__device__ __forceinline__ void ld_run8(const uint32_t *f, int64_t p0, const CompCodec &c, int bits, float *out)
{
    if (PK) {
        const int64_t b0 = p0 * bits;
        const uint32_t *w = f + (b0 >> 5);
        uint64_t acc = (uint64_t)(w[0] >> (b0 & 31));
        int have = 32 - (int)(b0 & 31), next = 1;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            if (have < bits) {
                acc |= (uint64_t)w[next++] << have;
                have += 32;
            }
            out[m] = decode_u((uint32_t)acc & c.mask, c);
            acc >>= bits;
            have -= bits;
        }
    } else {
        const float4 *f4 = reinterpret_cast<const float4 *>(f + p0);
        const float4 a = f4[0], e = f4[1];
        out[0] = a.x, out[1] = a.y, out[2] = a.z, out[3] = a.w;
        out[4] = e.x, out[5] = e.y, out[6] = e.z, out[7] = e.w;
    }
}

// 1 / (number of interior neighbours): exact for 4 and 2, within one rounding for 3.
__device__ __forceinline__ float inv_count(int cnt)
{
    return cnt == 4 ? 0.25f : cnt == 3 ? (1.0f / 3.0f) : cnt == 2 ? 0.5f : 1.0f;
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

// A point in cell units, (ci + fx, cj + fy): an integer part and a float offset that stays
// within a few cells of the sample point a backtrace starts from, so the position keeps
// its precision on any grid size (a single FP32 coordinate of a 4096-cell grid carries only
// 2^-11 cells).
struct Pt {
    int ci, cj;
    float fx, fy;
};

// One axis of a lattice coordinate gi + gf clamped into [0, n - 1]: the base index (at
// most n - 2) and the weight of the next sample.
__device__ __forceinline__ void lattice_axis(int gi, float gf, int n, int &i, float &f)
{
    const float fl = floorf(gf);
    i = gi + (int)fl;
    f = gf - fl;
    if (i < 0) {
        i = 0;
        f = 0.0f;
    } else if (i >= n - 1) {
        i = n - 2;
        f = 1.0f;
    }
}

// Bilinear sample at the point p of a lattice whose sample (0, 0) sits at cell coordinates
// (ox, oy), clamped into the lattice.
template <bool PK>
__device__ __forceinline__ float sample(const Lat &L, const Pt &p, float ox, float oy, const CompCodec &c, int bits)
{
    int i, j;
    float fx, fy;
    lattice_axis(p.ci, p.fx - ox, L.nx, i, fx);
    lattice_axis(p.cj, p.fy - oy, L.ny, j, fy);
    const float a = lat_at<PK>(L, i, j, c, bits), b = lat_at<PK>(L, i + 1, j, c, bits);
    const float e = lat_at<PK>(L, i, j + 1, c, bits), g = lat_at<PK>(L, i + 1, j + 1, c, bits);
    return (1.0f - fy) * ((1.0f - fx) * a + fx * b) + fy * ((1.0f - fx) * e + fx * g);
}

// Velocity (u lattice PU, v lattice PV) at p: u samples sit at (i, j + 1/2), v samples at
// (i + 1/2, j) in cell units.
template <bool PU, bool PV>
__device__ __forceinline__ void vel_at(const Params &P, const Lat &U, const Lat &V, const Pt &p, float &ux, float &vy)
{
    ux = sample<PU>(U, p, 0.0f, 0.5f, P.cc[0], P.bits[0]);
    vy = sample<PV>(V, p, 0.5f, 0.0f, P.cc[0], P.bits[0]);
}

// Ralston's RK-3 backtrace over s from p (velocities in domain units per second; one domain
// unit is n cells).
template <bool PU, bool PV>
__device__ __forceinline__ Pt backtrace(const Params &P, const Lat &U, const Lat &V, float s, const Pt &p)
{
    const float sn = s * P.inv_h;
    float k1x, k1y, k2x, k2y, k3x, k3y;
    vel_at<PU, PV>(P, U, V, p, k1x, k1y);
    vel_at<PU, PV>(P, U, V, Pt{p.ci, p.cj, p.fx - 0.5f * sn * k1x, p.fy - 0.5f * sn * k1y}, k2x, k2y);
    vel_at<PU, PV>(P, U, V, Pt{p.ci, p.cj, p.fx - 0.75f * sn * k2x, p.fy - 0.75f * sn * k2y}, k3x, k3y);
    return Pt{p.ci, p.cj, p.fx - sn * (2.0f * k1x + 3.0f * k2x + 4.0f * k3x) / 9.0f,
              p.fy - sn * (2.0f * k1y + 3.0f * k2y + 4.0f * k3y) / 9.0f};
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
            const uint4 blk = philox4x32(make_uint4(k >> 3, counter, (uint32_t)field, 0u), key.x, key.y);
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
            const uint4 blk = philox4x32(make_uint4(k >> 3, counter, (uint32_t)field, 0u), key.x, key.y);
            const uint32_t w = uint4_at(blk, (int)((k >> 1) & 3u));
            const uint32_t q16 = (k & 1u) ? (w >> 16) : (w & 0xFFFFu);
            y = x + P.sign[s] * P.sigma[type] * ((q16 & 0x8000u) ? 1.0f : -1.0f);
        }
        if (valid) out[pidx] = __float_as_uint(y);
    }
    if (P.ranges) record_range(P, s, type, valid ? fkey(x) : 0xffffffffu, valid ? fkey(x) : 0u);
    return y;
}

// Cell (i, j) inside the source box.
__device__ __forceinline__ bool cell_in_box(const Params &P, int i, int j)
{
    return i >= P.box[0] && i <= P.box[1] && j >= P.box[2] && j <= P.box[3];
}

// y-face (i, j) inside the source box.
__device__ __forceinline__ bool vface_in_box(const Params &P, int i, int j)
{
    return i >= P.box[0] && i <= P.box[1] && j >= P.box[4] && j <= P.box[5];
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
        const int i = (int)((uint32_t)t % (uint32_t)n), j = (int)((uint32_t)t / (uint32_t)n);
        if (cell_in_box(P, i, j)) d[t] = 1.0f;
    }
    if (t < (int64_t)(n + 1) * n) {
        const int i = (int)((uint32_t)t % (uint32_t)n), j = (int)((uint32_t)t / (uint32_t)n);
        float vv = 0.0f;
        if (j > 0 && j < n) {
            vv = ld<Q>(P.v.p + s * P.v.ss, t, P.cc[0], P.bits[0]);
            const float d1 = cell_in_box(P, i, j) ? 1.0f : d[(int64_t)j * n + i];
            const float d0 = cell_in_box(P, i, j - 1) ? 1.0f : d[(int64_t)(j - 1) * n + i];
            vv += P.dt * P.buoy * 0.5f * (d1 + d0);
            if (vface_in_box(P, i, j)) vv = P.v_in;
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
        const int i = (int)((uint32_t)t % (uint32_t)P.su), j = (int)((uint32_t)t / (uint32_t)P.su);
        const bool valid = i <= n, wall = i == 0 || i == n;
        float x = 0.0f;
        if (valid && !wall) {
            const Pt pb = backtrace<Q, PV>(P, WU, WV, half, Pt{i, j, 0.0f, 0.5f});
            x = sample<Q>(FU, pb, 0.0f, 0.5f, P.cc[0], P.bits[0]);
        }
        const uint32_t k = (uint32_t)(j * (n + 1) + i);
        Fld o = STAGE == 1 ? P.ut : P.u;
        store<Q>(P, s, 0, 0, x, k, counter, valid, wall, true, o.p + s * o.ss, t, trace);
    } else {
        const int64_t tv = t - nu;
        const int i = (int)((uint32_t)tv % (uint32_t)n), j = (int)((uint32_t)tv / (uint32_t)n);
        const bool wall = j == 0 || j == n;
        float x = 0.0f;
        if (!wall) {
            const Pt pb = backtrace<Q, PV>(P, WU, WV, half, Pt{i, j, 0.5f, 0.0f});
            x = sample<PV>(FV, pb, 0.5f, 0.0f, P.cc[0], P.bits[0]);
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
    const int i = (int)((uint32_t)t % (uint32_t)n), j = (int)((uint32_t)t / (uint32_t)n);
    const Fld fu = which == 0 ? P.ut : P.u, fv = which == 0 ? P.vt : P.v;
    const uint32_t *u = fu.p + s * fu.ss, *v = fv.p + s * fv.ss;
    const CompCodec &c = P.cc[0];
    const int b = P.bits[0];
    const float ur = ld<Q>(u, (int64_t)j * P.su + i + 1, c, b), ul = ld<Q>(u, (int64_t)j * P.su + i, c, b);
    const float vt = ld<Q>(v, (int64_t)(j + 1) * n + i, c, b), vb = ld<Q>(v, (int64_t)j * n + i, c, b);
    P.div[s * P.ncell_s + t] = (ur - ul + vt - vb) * P.inv_h;
}

// Jacobi sweeps it0 .. it0 + nsweep - 1 (1-based, nsweep <= kK) of a projection, blocked in
// time: a CTA loads a tile of kTY x kTX cells with a halo (kHX columns, kK rows) of the
// previous iterate (q[src]; zero when it0 = 1) into shared memory (div is read through the
// read-only cache as the sweeps need it), runs the
// sweeps there (every sweep's values stored through the codec: encode, then the decoded
// value is what the next sweep reads) and writes the tile's last iterate to q[src ^ 1].
// The halo's values go wrong by one cell per sweep from the region's edge inward, so
// after kK sweeps the tile itself is still exact (each sweep computes only the cells within
// the remaining sweeps' reach of the tile); halo cells are recomputed bit for bit as their
// own tile computes them (same inputs, same arithmetic, same dither draw).  A
// thread takes octets, 8 consecutive cells of a row aligned to 8 (one Philox block serves
// all 8: their dither counter is (cell / 8, counter, 2, 0), lanes cell % 8).  Only tile
// cells count saturations, record ranges and write the trace (sweep k of the launch to
// trace + k n^2).
constexpr int kTX = 128, kTY = 32, kK = 4, kHX = 8;
constexpr int kRW = kTX + 2 * kHX, kRH = kTY + 2 * kK, kRO = kRW / 8;
constexpr size_t kJacobiSmem = sizeof(float) * 2 * kRW * kRH;

template <bool Q>
__global__ void __launch_bounds__(kT, 4) jacobi_kernel(Params P, int it0, int nsweep, uint32_t cbase, int src,
                                                    uint32_t *trace)
{
    extern __shared__ float4 smem4[];
    float *qa = reinterpret_cast<float *>(smem4), *qb = qa + kRW * kRH;
    const int s = blockIdx.y, n = P.n;
    const int tiles_x = (n + kTX - 1) / kTX;
    const int x0 = (int)(blockIdx.x % tiles_x) * kTX, y0 = (int)(blockIdx.x / tiles_x) * kTY;
    const int w = min(kTX, n - x0);  // a multiple of 32
    const int gx0 = x0 - kHX, gy0 = y0 - kK;
    const CompCodec &c = P.cc[1];
    const int b = P.bits[1];
    const uint32_t *qin = P.q[src].p + s * P.q[0].ss;
    const uint32_t *div = reinterpret_cast<const uint32_t *>(P.div + s * P.ncell_s);
    for (int e = threadIdx.x; e < kRO * kRH; e += kT) {
        const int ry = e / kRO, ro = e % kRO;
        const int gy = gy0 + ry, gx = gx0 + ro * 8;
        float q8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (it0 > 1 && gy >= 0 && gy < n && gx >= 0 && gx < n)  // octets lie wholly inside or outside
            ld_run8<Q>(qin, (int64_t)gy * n + gx, c, b, q8);
        // both iterate buffers: the sweeps write only octets inside the domain, so the cells
        // outside it keep these zeros in either buffer for the whole launch
        float4 *qa4 = reinterpret_cast<float4 *>(qa + ry * kRW + ro * 8);
        float4 *qb4 = reinterpret_cast<float4 *>(qb + ry * kRW + ro * 8);
        qa4[0] = qb4[0] = make_float4(q8[0], q8[1], q8[2], q8[3]);
        qa4[1] = qb4[1] = make_float4(q8[4], q8[5], q8[6], q8[7]);
    }
    __syncthreads();
    float *cur = qa, *nxt = qb;
    unsigned nsat = 0;
    unsigned kmin = 0xffffffffu, kmax = 0u;
    const uint32_t step_base = 1024u * step_index(P) + cbase;
    // the scene's Philox keys, read once: inside the sweeps the compiler could not keep them
    // in registers across the trace stores
    const uint2 dkey = Q && P.dither ? P.seed[s] : make_uint2(0u, 0u);
    const bool noise = !Q && P.sigma[1] != 0.0f;
    const uint2 nkey = noise ? P.nseed[s] : make_uint2(0u, 0u);
    const float namp = noise ? P.sign[s] * P.sigma[1] : 0.0f;
    for (int k = 0; k < nsweep; ++k) {
        const int it = it0 + k;
        const uint32_t counter = step_base + (uint32_t)it;
        const bool last = k == nsweep - 1;
        // only what the tile's last sweep still depends on: r more rows and cells on each
        // side of the tile, r = the sweeps left after this one
        // (and inside the domain: the loop hands out no octet outside it)
        const int r = nsweep - 1 - k;
        const int ro_lo = max((kHX - r) / 8, -gx0 / 8), ro_hi = min((kHX + w - 1 + r) / 8, (n - 1 - gx0) / 8);
        const int ry_lo = max(kK - r, -gy0), ry_hi = min(kK + kTY - 1 + r, n - 1 - gy0);
        const int ncol = ro_hi - ro_lo + 1, nrow = ry_hi - ry_lo + 1;
        for (int e = threadIdx.x; e < nrow * ncol; e += kT) {
            const int ry = ry_lo + e / ncol, ro = ro_lo + e % ncol;
            const int gy = gy0 + ry, gx = gx0 + ro * 8;
            const float *rc = cur + ry * kRW + ro * 8;
            const float4 c0 = reinterpret_cast<const float4 *>(rc)[0], c1 = reinterpret_cast<const float4 *>(rc)[1];
            const float4 d0 = reinterpret_cast<const float4 *>(rc - kRW)[0], d1 = reinterpret_cast<const float4 *>(rc - kRW)[1];
            const float4 u0 = reinterpret_cast<const float4 *>(rc + kRW)[0], u1 = reinterpret_cast<const float4 *>(rc + kRW)[1];
            // the divergence through the read-only cache: kept out of shared memory, the
            // tile's two iterate buffers (46 KB) let four CTAs share an SM
            const float4 *dv4 = reinterpret_cast<const float4 *>(div + (int64_t)gy * n + gx);
            const float4 v0 = __ldg(dv4), v1 = __ldg(dv4 + 1);
            const float row[10] = {ro > 0 ? rc[-1] : 0.0f, c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w,
                                   ro < kRO - 1 ? rc[8] : 0.0f};
            const float dn[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
            const float up[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
            const float dv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            // neighbours outside the domain are the zeros of the tile's halo: the same sums, in
            // the same order, as adding only the interior ones, with no per-cell tests.  The
            // neighbour count differs only at the walls: rows 0 and n - 1 for the whole
            // octet, and the octet's first (last) cell when it starts (ends) at x = 0 (n - 1)
            // -- an octet lies wholly inside the domain
            float x[8];
            const int cnt_mid = 2 + (gy > 0) + (gy < n - 1);
            const float inv_mid = inv_count(cnt_mid);
            const float inv_first = inv_count(cnt_mid - (gx == 0)), inv_last = inv_count(cnt_mid - (gx + 8 == n));
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const float acc = it > 1 ? ((row[m] + row[m + 2]) + dn[m]) + up[m] : 0.0f;
                x[m] = (acc - P.h2 * dv[m]) * (m == 0 ? inv_first : m == 7 ? inv_last : inv_mid);
            }
            const bool inner = ry >= kK && ry < kK + kTY && ro >= 1 && (ro - 1) * 8 < w;
            const uint32_t oct = (uint32_t)(((int64_t)gy * n + gx) >> 3);
            if (inner && P.ranges) {
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    kmin = min(kmin, fkey(x[m]));
                    kmax = max(kmax, fkey(x[m]));
                }
            }
            if (Q) {
                uint4 blk = make_uint4(0u, 0u, 0u, 0u);
                if (P.dither) blk = philox4x32(make_uint4(oct, counter, 2u, 0u), dkey.x, dkey.y);
                uint32_t code[8];
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    int flags = 0;
                    code[m] = encode_f32(x[m], c, P.dither != 0, P.dither ? dither_threshold(blk, m) : 0u, flags);
                    if (inner) nsat += (unsigned)(flags & 1);
                    x[m] = decode_u(code[m], c);
                }
                if (inner) {
                    if (trace && s == 0) {
                        uint4 *tw = reinterpret_cast<uint4 *>(trace + (int64_t)k * n * n + (int64_t)gy * n + gx);
                        tw[0] = make_uint4(code[0], code[1], code[2], code[3]);
                        tw[1] = make_uint4(code[4], code[5], code[6], code[7]);
                    }
                }
                if (last) {  // nobody reads the last sweep's values here: keep its codes instead
#pragma unroll
                    for (int m = 0; m < 8; ++m) x[m] = __uint_as_float(code[m]);
                }
            } else if (noise) {
                const uint4 blk = philox4x32(make_uint4(oct, counter, 2u, 0u), nkey.x, nkey.y);
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const uint32_t wd = uint4_at(blk, (m >> 1) & 3);
                    const uint32_t q16 = (m & 1) ? (wd >> 16) : (wd & 0xFFFFu);
                    x[m] += namp * ((q16 & 0x8000u) ? 1.0f : -1.0f);
                }
            }
            float4 *nw = reinterpret_cast<float4 *>(nxt + ry * kRW + ro * 8);
            nw[0] = make_float4(x[0], x[1], x[2], x[3]);
            nw[1] = make_float4(x[4], x[5], x[6], x[7]);
            if (!Q && last && inner) {
                float4 *gw = reinterpret_cast<float4 *>(P.q[src ^ 1].p + s * P.q[0].ss + (int64_t)gy * n + gx);
                gw[0] = nw[0];
                gw[1] = nw[1];
            }
        }
        __syncthreads();
        float *t = cur;
        cur = nxt;
        nxt = t;
    }
    if (Q) {
        // the tile's last codes (in cur after the swap), row segments of w cells = w b / 32
        // whole words each
        const uint32_t *cs = reinterpret_cast<const uint32_t *>(cur) + kK * kRW + kHX;
        const int wpr = w / 32 * b;
        uint32_t *qout = P.q[src ^ 1].p + s * P.q[0].ss;
        for (int e = threadIdx.x; e < kTY * wpr; e += kT) {
            const int r = e / wpr, wr = e % wpr;
            const int b0 = 32 * wr, m1 = min((b0 + 31) / b, w - 1);
            uint32_t word = 0u;
            for (int m = b0 / b; m <= m1; ++m) {
                const int sh = m * b - b0;
                word |= sh >= 0 ? (cs[r * kRW + m] << sh) : (cs[r * kRW + m] >> -sh);
            }
            qout[((int64_t)(y0 + r) * n + x0) / 32 * b + wr] = word;
        }
        nsat = __reduce_add_sync(0xffffffffu, nsat);
        if (nsat && (threadIdx.x & 31) == 0) atomicAdd(P.sat + 2 * s + 1, (unsigned long long)nsat);
    }
    if (P.ranges) record_range(P, s, 1, kmin, kmax);
}

// out = in - grad q on interior faces (q = the last sweep's iterate; none when J = 0), then
// the velocity store.  STAGE 2: (ut, vt) -> (up, vp), followed by the reflection
// u^ = 2 u' - u~ stored over (ut, vt) (store J + 3, no noise: an integer combination of two
// stored values of one lattice is itself on it); STAGE 5: (u, v) in place.
template <bool Q, int STAGE>
__global__ void __launch_bounds__(kT) gradsub_kernel(Params P, uint32_t *trace, uint32_t *trace3)
{
    const int s = blockIdx.y, n = P.n;
    const int64_t nu = (int64_t)n * P.su, nv = (int64_t)(n + 1) * n;
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t - (threadIdx.x & 31) >= nu + nv) return;
    const uint32_t counter = 1024u * step_index(P) + (STAGE == 2 ? (uint32_t)P.J + 2u : 2u * (uint32_t)P.J + 5u);
    const uint32_t *q = P.q[P.qfin].p + s * P.q[0].ss;
    const CompCodec &cq = P.cc[1];
    const int bq = P.bits[1];
    const Fld fin_u = STAGE == 2 ? P.ut : P.u, fin_v = STAGE == 2 ? P.vt : P.v;
    const Fld fo_u = STAGE == 2 ? P.up : P.u, fo_v = STAGE == 2 ? P.vp : P.v;
    if (t < nu) {
        const int i = (int)((uint32_t)t % (uint32_t)P.su), j = (int)((uint32_t)t / (uint32_t)P.su);
        const bool valid = i <= n, wall = i == 0 || i >= n;
        const uint32_t k = (uint32_t)(j * (n + 1) + i);
        float xin = 0.0f, x = 0.0f;
        if (valid && !wall) {
            xin = ld<Q>(fin_u.p + s * fin_u.ss, t, P.cc[0], P.bits[0]);
            x = xin;
            if (P.J > 0) x -= (ld<Q>(q, (int64_t)j * n + i, cq, bq) - ld<Q>(q, (int64_t)j * n + i - 1, cq, bq)) * P.inv_h;
        }
        const float y = store<Q>(P, s, 0, 0, x, k, counter, valid, wall, true, fo_u.p + s * fo_u.ss, t, trace);
        if (STAGE == 2)  // u^ = 2 u' - u~ over u~ (store J + 3)
            store<Q>(P, s, 0, 0, 2.0f * y - xin, k, counter + 1u, valid, wall, false, P.ut.p + s * P.ut.ss, t, trace3);
    } else {
        const int64_t tv = t - nu;
        const int i = (int)((uint32_t)tv % (uint32_t)n), j = (int)((uint32_t)tv / (uint32_t)n);
        const bool wall = j == 0 || j == n;
        float xin = 0.0f, x = 0.0f;
        if (!wall) {
            xin = ld<Q>(fin_v.p + s * fin_v.ss, tv, P.cc[0], P.bits[0]);
            x = xin;
            if (P.J > 0) x -= (ld<Q>(q, (int64_t)j * n + i, cq, bq) - ld<Q>(q, (int64_t)(j - 1) * n + i, cq, bq)) * P.inv_h;
        }
        const int64_t tvo = (int64_t)(n + 1) * n;
        const float y = store<Q>(P, s, 0, 1, x, (uint32_t)tv, counter, true, wall, true, fo_v.p + s * fo_v.ss, tv,
                                 trace ? trace + tvo : nullptr);
        if (STAGE == 2)
            store<Q>(P, s, 0, 1, 2.0f * y - xin, (uint32_t)tv, counter + 1u, true, wall, false, P.vt.p + s * P.vt.ss, tv,
                     trace3 ? trace3 + tvo : nullptr);
    }
}

template <bool Q>
__global__ void __launch_bounds__(kT) advect_d_kernel(Params P)
{
    const int s = blockIdx.y, n = P.n;
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t >= (int64_t)n * n) return;
    const int i = (int)((uint32_t)t % (uint32_t)n), j = (int)((uint32_t)t / (uint32_t)n);
    const uint32_t par = *P.ctr & 1u;
    const Lat WU{P.up.p + s * P.up.ss, P.su, n + 1, n};
    const Lat WV{P.vp.p + s * P.vp.ss, n, n, n + 1};
    const Lat D{reinterpret_cast<const uint32_t *>(P.d[par] + s * P.ncell_s), n, n, n};
    const Pt pb = backtrace<Q, Q>(P, WU, WV, P.dt, Pt{i, j, 0.5f, 0.5f});
    P.d[par ^ 1u][s * P.ncell_s + t] = sample<false>(D, pb, 0.5f, 0.5f, P.cc[0], 0);
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
        P.z[(int64_t)s * kMeasureBlocks + blockIdx.x] = a;  // summed in order on the host
    }
}

// Host FP32 state (oracle layout) -> stored fields; nearest rounding, walls zero.
template <bool Q>
__global__ void __launch_bounds__(kT) set_state_kernel(Params P, int s0, const float *u, const float *v, const float *d,
                                                       int64_t stride_uv, int64_t stride_d)
{
    // scene s0 + blockIdx.y, its arrays blockIdx.y strides into the staged ones
    const int s = s0 + (int)blockIdx.y;
    if (u) u += blockIdx.y * stride_uv;
    if (v) v += blockIdx.y * stride_uv;
    if (d) d += blockIdx.y * stride_d;
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
        const int i = (int)((uint32_t)t % (uint32_t)P.su), j = (int)((uint32_t)t / (uint32_t)P.su);
        valid = i <= n;
        if (valid && i > 0 && i < n && u) x = u[(int64_t)j * (n + 1) + i];
        out = P.u.p + s * P.u.ss;
        pidx = t;
    } else {
        const int64_t tv = t - nu;
        const int j = (int)((uint32_t)tv / (uint32_t)n);
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
__global__ void __launch_bounds__(kT) readback_kernel(Params P, int s0, float *u, float *v, float *d, float *q,
                                                      int64_t stride_uv, int64_t stride_d)
{
    const int s = s0 + (int)blockIdx.y;
    u += blockIdx.y * stride_uv;
    v += blockIdx.y * stride_uv;
    d += blockIdx.y * stride_d;
    q += blockIdx.y * stride_d;
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
        q[t] = P.J > 0 ? ld<Q>(P.q[P.qfin].p + s * P.q[0].ss, t, P.cc[1], P.bits[1]) : 0.0f;
    }
}

// Stage inputs of scene 0 (qmpm_smoke_stage): a velocity pair in the oracle layout into
// the stored fields fu, fv (nearest rounding: values on the type's lattice are stored as
// they are), or n^2 cell values into the stored pressure field f.
__global__ void __launch_bounds__(kT) set_pair_kernel(Params P, Fld fu, Fld fv, const float *u, const float *v)
{
    const int n = P.n;
    const int64_t nu = (int64_t)n * P.su, nv = (int64_t)(n + 1) * n;
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t - (threadIdx.x & 31) >= nu + nv) return;
    uint32_t *out;
    int64_t pidx;
    float x = 0.0f;
    bool valid = true;
    if (t < nu) {
        const int i = (int)((uint32_t)t % (uint32_t)P.su), j = (int)((uint32_t)t / (uint32_t)P.su);
        valid = i <= n;
        if (valid) x = u[(int64_t)j * (n + 1) + i];
        out = fu.p;
        pidx = t;
    } else {
        pidx = t - nu;
        x = v[pidx];
        out = fv.p;
    }
    int flags = 0;
    uint32_t code = encode_f32(x, P.cc[0], false, 0u, flags);
    if (!valid) code = 0u;
    put_codes(out, pidx, code, P.bits[0]);
}

__global__ void __launch_bounds__(kT) set_cells_kernel(Params P, Fld f, const float *x)
{
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;  // n^2 is a multiple of 32
    if (t - (threadIdx.x & 31) >= (int64_t)P.n * P.n) return;
    int flags = 0;
    const uint32_t code = encode_f32(x[t], P.cc[1], false, 0u, flags);
    put_codes(f.p, t, code, P.bits[1]);
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
    float *stage_all = nullptr;    // every scene's u, v, d, q for the batch transfers (on first use)
    int64_t stage_floats = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t steps = 0, launches = 0, graph_launches = 0, device_bytes = 0;
    bool profile = false;
    std::vector<cudaEvent_t> ev;   // per profiled step: start, sweeps 1 begin/end, sweeps 2 begin/end, end
    int64_t prof_jacobi_launches = 0;
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

unsigned launches_per_step(int J) { return 10u + 2u * (unsigned)((J + kK - 1) / kK); }

template <bool Q>
int enqueue_step(qmpm_smoke *h, uint32_t *trace)
{
    Params &P = h->p;
    const int n = P.n, J = P.J, S = h->S;
    const int64_t nfaces = (int64_t)n * P.su + (int64_t)(n + 1) * n;
    const dim3 gf((unsigned)((nfaces + kT - 1) / kT), S);
    const dim3 gc((unsigned)(((int64_t)n * n + kT - 1) / kT), S);
    const dim3 gv((unsigned)(((int64_t)(n + 1) * n + kT - 1) / kT), S);
    const int64_t V = 2 * (int64_t)n * (n + 1), Pq = (int64_t)n * n;
    auto tr = [&](int64_t off) { return trace ? trace + off : nullptr; };
    cudaEvent_t ev[6] = {};
    if (h->profile) {
        for (auto &e : ev) {
            if (cudaEventCreate(&e) != cudaSuccess) return fail(QMPM_ERR_CUDA, "qmpm_smoke_step: event creation");
            h->ev.push_back(e);
        }
        h->prof_jacobi_launches += 2 * ((J + kK - 1) / kK);
    }
    auto mark = [&](int k) {
        if (h->profile) cudaEventRecord(ev[k], h->st);
    };
    mark(0);
    forces_kernel<Q><<<gv, kT, 0, h->st>>>(P);
    advect_vel_kernel<Q, 1><<<gf, kT, 0, h->st>>>(P, tr(0));
    divergence_kernel<Q><<<gc, kT, 0, h->st>>>(P, 0);
    const dim3 gj((unsigned)(((n + kTX - 1) / kTX) * (n / kTY)), S);
    auto sweeps = [&](uint32_t cbase, int64_t toff) {
        for (int l = 0; l * kK < J; ++l) {
            const int it0 = l * kK + 1, ns = std::min(kK, J - l * kK);
            jacobi_kernel<Q><<<gj, kT, kJacobiSmem, h->st>>>(P, it0, ns, cbase, l & 1, tr(toff + (int64_t)(it0 - 1) * Pq));
        }
    };
    mark(1);
    sweeps(1u, V);
    mark(2);
    gradsub_kernel<Q, 2><<<gf, kT, 0, h->st>>>(P, tr(V + J * Pq), tr(2 * V + J * Pq));
    advect_vel_kernel<Q, 4><<<gf, kT, 0, h->st>>>(P, tr(3 * V + J * Pq));
    divergence_kernel<Q><<<gc, kT, 0, h->st>>>(P, 1);
    mark(3);
    sweeps((uint32_t)J + 4u, 4 * V + J * Pq);
    mark(4);
    gradsub_kernel<Q, 5><<<gf, kT, 0, h->st>>>(P, tr(4 * V + 2 * J * Pq), nullptr);
    advect_d_kernel<Q><<<gc, kT, 0, h->st>>>(P);
    advance_kernel<<<1, 1, 0, h->st>>>(P.ctr);
    mark(5);
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
    auto *h = new (std::nothrow) qmpm_smoke();
    if (!h) return fail(QMPM_ERR_OOM, "qmpm_smoke_create: host allocation failed");
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
    P.h2 = 1.0f / ((float)n * (float)n);
    // the box as index ranges: the samples whose position (cell centre (i + 1/2) h, y-face
    // j h) lies in [src0, src2] x [src1, src3], decided in FP64 on the host
    {
        const double hd = 1.0 / n;
        auto range = [&](double lo, double hi, double off, int count, int &a, int &b) {
            a = 1;
            b = 0;
            bool any = false;
            for (int i = 0; i < count; ++i) {
                const double x = (i + off) * hd;
                if (x >= lo && x <= hi) {
                    if (!any) a = i;
                    b = i;
                    any = true;
                }
            }
        };
        range(cfg->src[0], cfg->src[2], 0.5, n, P.box[0], P.box[1]);  // the oracle's comparisons, in FP64
        range(cfg->src[1], cfg->src[3], 0.5, n, P.box[2], P.box[3]);
        range(cfg->src[1], cfg->src[3], 0.0, n + 1, P.box[4], P.box[5]);
    }
    P.quant = h->quant;
    P.dither = h->quant && cfg->dither;
    P.ranges = (cfg->flags & QMPM_SMOKE_RANGES) != 0;
    h->profile = (cfg->flags & QMPM_SMOKE_PROFILE) != 0;
    P.qfin = ((P.J + kK - 1) / kK) & 1;
    if (cudaFuncSetAttribute(jacobi_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kJacobiSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(jacobi_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kJacobiSmem) !=
            cudaSuccess) {
        qmpm_smoke_destroy(h);
        return fail(QMPM_ERR_CUDA, "qmpm_smoke_create: shared memory opt-in failed");
    }
    P.bits[0] = P.bits[1] = 32;
    if (h->quant) {
        for (int t = 0; t < 2; ++t) {
            if (make_codec(scheme->bits[t], scheme->frac[t], scheme->offset[t], P.cc[t])) {
                qmpm_smoke_destroy(h);  // nothing allocated yet but the stream
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
    P.z = (double *)alloc(sizeof(double) * kMeasureBlocks * S);
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
            set_state_kernel<true><<<g, kT, 0, h->st>>>(P, s, h_u ? du : nullptr, h_v ? dv : nullptr, h_d ? dd : nullptr,
                                                        0, 0);
        else
            set_state_kernel<false><<<g, kT, 0, h->st>>>(P, s, h_u ? du : nullptr, h_v ? dv : nullptr, h_d ? dd : nullptr,
                                                         0, 0);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_set_state", e);
    return QMPM_OK;
}

// Device staging of every scene's u, v, d (and q) for the batch transfers, made on first use.
static int ensure_stage_all(qmpm_smoke *h)
{
    if (h->stage_all) return QMPM_OK;
    const int64_t n = h->p.n, nu = n * (n + 1), nc = n * n;
    const size_t bytes = sizeof(float) * (size_t)h->S * (size_t)(2 * nu + 2 * nc);
    if (cudaMalloc(&h->stage_all, bytes) != cudaSuccess) {
        cudaGetLastError();
        h->stage_all = nullptr;
        return fail(QMPM_ERR_OOM, "smoke batch staging: device allocation failed");
    }
    h->allocs.push_back(h->stage_all);
    h->device_bytes += (int64_t)bytes;
    return QMPM_OK;
}

int qmpm_smoke_set_states(qmpm_smoke_handle h, const float *h_u, const float *h_v, const float *h_d)
{
    if (!h) return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_set_states: NULL handle");
    int r = ensure_stage_all(h);
    if (r != QMPM_OK) return r;
    const Params &P = h->p;
    const int n = P.n, S = h->S;
    const int64_t nu = (int64_t)n * (n + 1), nc = (int64_t)n * n;
    float *du = h->stage_all, *dv = du + S * nu, *dd = dv + S * nu;
    cudaError_t e = cudaSuccess;
    if (h_u) e = cudaMemcpyAsync(du, h_u, sizeof(float) * S * nu, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess && h_v) e = cudaMemcpyAsync(dv, h_v, sizeof(float) * S * nu, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess && h_d) e = cudaMemcpyAsync(dd, h_d, sizeof(float) * S * nc, cudaMemcpyHostToDevice, h->st);
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_set_states", e);
    const int64_t nfaces = (int64_t)n * P.su + (int64_t)(n + 1) * n;
    const dim3 g((unsigned)((nfaces + kT - 1) / kT), S);
    if (h->quant)
        set_state_kernel<true><<<g, kT, 0, h->st>>>(P, 0, h_u ? du : nullptr, h_v ? dv : nullptr, h_d ? dd : nullptr,
                                                    nu, nc);
    else
        set_state_kernel<false><<<g, kT, 0, h->st>>>(P, 0, h_u ? du : nullptr, h_v ? dv : nullptr, h_d ? dd : nullptr,
                                                     nu, nc);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_set_states", e);
    return QMPM_OK;
}

int qmpm_smoke_get_states(qmpm_smoke_handle h, float *h_u, float *h_v, float *h_d)
{
    if (!h) return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_get_states: NULL handle");
    int r = ensure_stage_all(h);
    if (r != QMPM_OK) return r;
    const int n = h->p.n, S = h->S;
    const int64_t nu = (int64_t)n * (n + 1), nc = (int64_t)n * n;
    float *du = h->stage_all, *dv = du + S * nu, *dd = dv + S * nu, *dq = dd + S * nc;
    const dim3 g((unsigned)((nu + kT - 1) / kT), S);
    if (h->quant)
        readback_kernel<true><<<g, kT, 0, h->st>>>(h->p, 0, du, dv, dd, dq, nu, nc);
    else
        readback_kernel<false><<<g, kT, 0, h->st>>>(h->p, 0, du, dv, dd, dq, nu, nc);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && h_u) e = cudaMemcpyAsync(h_u, du, sizeof(float) * S * nu, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess && h_v) e = cudaMemcpyAsync(h_v, dv, sizeof(float) * S * nu, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess && h_d) e = cudaMemcpyAsync(h_d, dd, sizeof(float) * S * nc, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_get_states", e);
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
    if (h->profile && !d_trace) {
        for (int t = 0; t < steps; ++t) {
            const int r = enqueue(h, nullptr);
            if (r != QMPM_OK) return r;
            ++h->steps;
        }
        return QMPM_OK;
    }
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
    measure_kernel<<<dim3(kMeasureBlocks, h->S), kT, 0, h->st>>>(h->p);
    std::vector<double> part((size_t)kMeasureBlocks * h->S);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(part.data(), h->p.z, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_measure", e);
    for (int s = 0; s < h->S; ++s) {  // a fixed order: the same z for the same state
        double a = 0.0;
        for (int b = 0; b < kMeasureBlocks; ++b) a += part[(size_t)s * kMeasureBlocks + b];
        h_z[s] = a;
    }
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
        readback_kernel<true><<<g, kT, 0, h->st>>>(h->p, scene, du, dv, dd, dq, 0, 0);
    else
        readback_kernel<false><<<g, kT, 0, h->st>>>(h->p, scene, du, dv, dd, dq, 0, 0);
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

int qmpm_smoke_profile(qmpm_smoke_handle h, double *h_step_ms, double *h_jacobi_ms, int64_t *h_jacobi_launches)
{
    if (!h || !h->profile) return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_profile: handle created without QMPM_SMOKE_PROFILE");
    cudaError_t e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_profile", e);
    double step = 0.0, jac = 0.0;
    for (size_t k = 0; k + 6 <= h->ev.size(); k += 6) {
        float a = 0.0f, b = 0.0f, c = 0.0f;
        cudaEventElapsedTime(&a, h->ev[k], h->ev[k + 5]);
        cudaEventElapsedTime(&b, h->ev[k + 1], h->ev[k + 2]);
        cudaEventElapsedTime(&c, h->ev[k + 3], h->ev[k + 4]);
        step += a;
        jac += (double)b + c;
    }
    for (cudaEvent_t ev : h->ev) cudaEventDestroy(ev);
    h->ev.clear();
    if (h_step_ms) *h_step_ms = step;
    if (h_jacobi_ms) *h_jacobi_ms = jac;
    if (h_jacobi_launches) *h_jacobi_launches = h->prof_jacobi_launches;
    h->prof_jacobi_launches = 0;
    return QMPM_OK;
}

int qmpm_smoke_destroy(qmpm_smoke_handle h)
{
    if (!h) return QMPM_OK;
    cudaStreamSynchronize(h->st);
    drop_graph(h);
    for (cudaEvent_t ev : h->ev) cudaEventDestroy(ev);
    for (void *p : h->allocs) cudaFree(p);
    if (h->own_stream) cudaStreamDestroy(h->st);
    delete h;
    return QMPM_OK;
}

}  // extern "C"

int qmpm_smoke_stage(qmpm_smoke_handle h, int32_t stage, int32_t arg, uint32_t step, const float *h_a_u,
                     const float *h_a_v, const float *h_b_u, const float *h_b_v, const float *h_q,
                     const float *h_div, uint32_t *h_codes)
{
    if (!h || !h->quant || stage < QMPM_SMOKE_ADVECT1 || stage > QMPM_SMOKE_GRADSUB5 || step < 1 || !h_codes)
        return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_stage: needs a quantized handle, a stage, step >= 1 and h_codes");
    Params P = h->p;
    const int n = P.n, J = P.J;
    const bool need_a = true, need_b = stage == QMPM_SMOKE_ADVECT4;
    const bool need_q = stage == QMPM_SMOKE_GRADSUB2 || stage == QMPM_SMOKE_GRADSUB5 ||
                        (stage == QMPM_SMOKE_JACOBI && arg > 1);
    const bool need_div = stage == QMPM_SMOKE_JACOBI;
    if (stage == QMPM_SMOKE_JACOBI && (arg < 1 || arg > J))
        return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_stage: the sweep index must be in 1..jacobi");
    if ((stage != QMPM_SMOKE_JACOBI && (!h_a_u || !h_a_v)) || (need_b && (!h_b_u || !h_b_v)) || (need_q && !h_q) ||
        (need_div && !h_div))
        return fail(QMPM_ERR_INVALID_ARG, "qmpm_smoke_stage: an input of the stage is NULL");
    const int64_t nu = (int64_t)n * (n + 1), nc = (int64_t)n * n;
    const int64_t V = 2 * nu;  // velocity codes of one store
    const int64_t n_codes = stage == QMPM_SMOKE_JACOBI ? nc : stage == QMPM_SMOKE_GRADSUB2 ? 2 * V : V;
    std::vector<void *> tmp;
    auto dal = [&](size_t bytes) -> void * {
        void *ptr = nullptr;
        if (cudaMalloc(&ptr, bytes) != cudaSuccess) return nullptr;
        tmp.push_back(ptr);
        return ptr;
    };
    auto cleanup = [&]() {
        for (void *ptr : tmp) cudaFree(ptr);
    };
    float *d_au = (float *)dal(sizeof(float) * nu), *d_av = (float *)dal(sizeof(float) * nu);
    float *d_bu = (float *)dal(sizeof(float) * nu), *d_bv = (float *)dal(sizeof(float) * nu);
    float *d_q = (float *)dal(sizeof(float) * nc);
    uint32_t *d_tr = (uint32_t *)dal(sizeof(uint32_t) * (size_t)n_codes);
    if (!d_au || !d_av || !d_bu || !d_bv || !d_q || !d_tr) {
        cudaGetLastError();
        cleanup();
        return fail(QMPM_ERR_OOM, "qmpm_smoke_stage: device allocation failed");
    }
    cudaStream_t st = h->st;
    cudaError_t e = cudaSuccess;
    auto up = [&](float *d, const float *hsrc, int64_t cnt) {
        if (e == cudaSuccess && hsrc) e = cudaMemcpyAsync(d, hsrc, sizeof(float) * cnt, cudaMemcpyHostToDevice, st);
    };
    up(d_au, h_a_u, nu);
    up(d_av, h_a_v, nu);
    up(d_bu, h_b_u, nu);
    up(d_bv, h_b_v, nu);
    up(d_q, h_q, nc);
    const uint32_t done = step - 1u;  // the kernels store with step index = steps done + 1
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.ctr, &done, sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_tr, 0, sizeof(uint32_t) * (size_t)n_codes, st);
    const int64_t nfaces = (int64_t)n * P.su + nu;
    const unsigned gf = (unsigned)((nfaces + kT - 1) / kT), gc = (unsigned)((nc + kT - 1) / kT);
    if (e == cudaSuccess) {
        switch (stage) {
        case QMPM_SMOKE_ADVECT1:
            // u stored; v after the forces is FP32 (vf)
            set_pair_kernel<<<gf, kT, 0, st>>>(P, P.u, P.v, d_au, d_av);
            e = cudaMemcpyAsync(P.vf, d_av, sizeof(float) * nu, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) advect_vel_kernel<true, 1><<<gf, kT, 0, st>>>(P, d_tr);
            break;
        case QMPM_SMOKE_JACOBI: {
            if (need_q) set_cells_kernel<<<gc, kT, 0, st>>>(P, P.q[0], d_q);
            e = cudaMemcpyAsync(P.div, h_div, sizeof(float) * nc, cudaMemcpyHostToDevice, st);
            const dim3 gj((unsigned)(((n + kTX - 1) / kTX) * (n / kTY)), 1);
            if (e == cudaSuccess) jacobi_kernel<true><<<gj, kT, kJacobiSmem, st>>>(P, arg, 1, 1u, 0, d_tr);
            break;
        }
        case QMPM_SMOKE_GRADSUB2:
        case QMPM_SMOKE_GRADSUB5:
            P.qfin = 0;
            set_cells_kernel<<<gc, kT, 0, st>>>(P, P.q[0], d_q);
            if (stage == QMPM_SMOKE_GRADSUB2) {
                set_pair_kernel<<<gf, kT, 0, st>>>(P, P.ut, P.vt, d_au, d_av);
                gradsub_kernel<true, 2><<<gf, kT, 0, st>>>(P, d_tr, d_tr + V);
            } else {
                set_pair_kernel<<<gf, kT, 0, st>>>(P, P.u, P.v, d_au, d_av);
                gradsub_kernel<true, 5><<<gf, kT, 0, st>>>(P, d_tr, nullptr);
            }
            break;
        case QMPM_SMOKE_ADVECT4:
            set_pair_kernel<<<gf, kT, 0, st>>>(P, P.ut, P.vt, d_au, d_av);
            set_pair_kernel<<<gf, kT, 0, st>>>(P, P.up, P.vp, d_bu, d_bv);
            advect_vel_kernel<true, 4><<<gf, kT, 0, st>>>(P, d_tr);
            break;
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_codes, d_tr, sizeof(uint32_t) * (size_t)n_codes, cudaMemcpyDeviceToHost, st);
    const uint32_t back = (uint32_t)h->steps;
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.ctr, &back, sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail("qmpm_smoke_stage", e);
    return QMPM_OK;
}
