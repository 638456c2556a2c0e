// device_common.cuh -- device helpers of libqmpm: the dither generator, the fixed-point
// codec and the padded block layout of the grid.
#pragma once

#ifndef __CUDACC_RTC__
#include <cstdint>
#include <cuda_runtime.h>
#endif

#include "qmpm_internal.h"

namespace qmpm {

// ------------------------------------------------------------------------------------
// Philox4x32-R (Salmon, Moraes, Dror, Shaw, SC 2011): R rounds of the 4x32 S-box, keys
// bumped by the Weyl constants between rounds.  The dither threshold of Sec. 5 takes
// R = kDitherRounds = 7 (the authors report 7 rounds already pass their Crush batteries;
// the published known answers are for 10): counter (slot, step, comp / 8, 0), key = scene
// seed; component comp takes the 16-bit half comp % 2 of word (comp / 2) % 4
// (dither_threshold).  The explicit store errors of qmpm_noise_moments take R = 10.
// ------------------------------------------------------------------------------------
constexpr int kDitherRounds = 7;

template <int R = kDitherRounds>
__device__ __forceinline__ uint4 philox4x32(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// The dither generator with its round keys given (round r: seed_lo + r 0x9E3779B9,
// seed_hi + r 0xBB67AE85, precomputed on the host): read from the kernel's parameters, each
// key is an operand of the round's XOR instead of two additions per round.
__device__ __forceinline__ uint4 philox4x32_rk(uint4 c, const uint32_t (&rk)[2][10])
{
#pragma unroll
    for (int r = 0; r < kDitherRounds; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ rk[0][r], lo1, hi0 ^ c.w ^ rk[1][r], lo0);
    }
    return c;
}

__device__ __forceinline__ uint32_t uint4_at(const uint4 &v, int i)
{
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Dither threshold of component c from the Philox block of its group of eight: a 16-bit
// draw q placed mid-bucket among the 32-bit fractions, r = q 2^16 + 2^15 (round up when the
// fraction f > r: probability f rounded to 16 bits).
__device__ __forceinline__ uint32_t dither_threshold(const uint4 &blk, int c)
{
    const uint32_t w = uint4_at(blk, (c >> 1) & 3);
    const uint32_t q = (c & 1) ? (w >> 16) : (w & 0xFFFFu);
    return (q << 16) | 0x8000u;
}

// ------------------------------------------------------------------------------------
// Fixed-point codec (Sec. 3.1 Eq. 3, Sec. 5 Eq. 11), FP32 side.
//   decode: (u + offset) * 2^-frac, one rounding to FP32 (exact for the |u + offset|
//           < 2^24 the scheme validation guarantees).
//   encode: t = v * 2^frac (exact), I = floor(t), Y = t - I (exact), f = floor(Y 2^32);
//           up = dithered ? f > r : f >= 2^31;  u = clamp(I - offset + up, 0, 2^bits - 1).
//           t is first clamped to +-2^26, far outside every valid window, so that the
//           conversions stay exact; NaN lands on the low clamp and saturates to 0.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ float decode_u(uint32_t u, const CompCodec &cc)
{
    return fmaf((float)u, cc.dec_scale, cc.dec_bias);
}

// flags: bit0 saturated, bit1 round-up, bit2 round-down
__device__ __forceinline__ uint32_t encode_f32(float v, const CompCodec &cc, bool dither, uint32_t r,
                                               int &flags)
{
    float t = v * cc.enc_scale;
    t = fminf(fmaxf(t, -67108864.0f), 67108864.0f);
    const float fl = floorf(t);
    const float Y = t - fl;
    const uint32_t f = __float2uint_rd(Y * 4294967296.0f);
    const int I = __float2int_rn(fl);
    const int up = dither ? (f > r ? 1 : 0) : (f >= 0x80000000u ? 1 : 0);
    int u = I - cc.offset + up;
    flags = 0;
    if (u < 0) {
        u = 0;
        flags = 1;
    } else if ((uint32_t)u > cc.umax) {
        u = (int)cc.umax;
        flags = 1;
    } else {
        flags = up ? 2 : (f != 0u ? 4 : 0);
    }
    return (uint32_t)u;
}

// Same rule in FP64 (initial state from the host): every step is exact in FP64.
__device__ __forceinline__ uint32_t encode_f64(double v, const CompCodec &cc, bool dither, uint32_t r,
                                               int &flags)
{
    const double t = v * (double)cc.enc_scale;
    flags = 0;
    if (isnan(t)) {
        flags = 1;
        return 0u;
    }
    if (t < (double)cc.offset - 1.0) {
        flags = 1;
        return 0u;
    }
    if (t >= (double)cc.offset + (double)cc.umax + 1.0) {
        flags = 1;
        return cc.umax;
    }
    const double I = floor(t);
    const double Y = t - I;
    const unsigned long long f = (unsigned long long)floor(Y * 4294967296.0);
    const int up = dither ? (f > (unsigned long long)r ? 1 : 0) : (f >= 0x80000000ull ? 1 : 0);
    long long u = (long long)I - cc.offset + up;
    if (u < 0) {
        flags = 1;
        return 0u;
    }
    if (u > (long long)cc.umax) {
        flags = 1;
        return cc.umax;
    }
    flags = up ? 2 : (f != 0ull ? 4 : 0);
    return (uint32_t)u;
}

__device__ __forceinline__ double decode_f64(uint32_t u, const CompCodec &cc)
{
    return ((double)u + (double)cc.offset) * (double)cc.dec_scale;
}

// Extract component c's integer from a record held as 32-bit words at w[j * stride].
__device__ __forceinline__ uint32_t extract(const uint32_t *w, int stride, const CompCodec &cc)
{
    uint32_t lo = w[cc.word * stride] >> cc.shift;
    if (cc.straddle) lo |= w[(cc.word + 1) * stride] << (32 - cc.shift);
    return lo & cc.mask;
}

__device__ __forceinline__ void insert(uint32_t *w, int stride, const CompCodec &cc, uint32_t u)
{
    w[cc.word * stride] |= u << cc.shift;
    if (cc.straddle) w[(cc.word + 1) * stride] |= u >> (32 - cc.shift);
}

// ------------------------------------------------------------------------------------
// Grid storage: blocks of 4^d nodes, float4 (m, mv) per node, on a block lattice padded
// by one block on each side (nb = n/4 + 2 blocks per axis).  Node g (per axis, may be
// -4 .. n+3) lives in block (g >> 2) + 1 at local index g & 3.
// ------------------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ int64_t node_addr(int nb, int gx, int gy, int gz)
{
    if (DIM == 2) {
        const int64_t blk = (int64_t)((gx >> 2) + 1) * nb + ((gy >> 2) + 1);
        return blk * 16 + ((gx & 3) * 4 + (gy & 3));
    } else {
        const int64_t blk = ((int64_t)((gx >> 2) + 1) * nb + ((gy >> 2) + 1)) * nb + ((gz >> 2) + 1);
        return blk * 64 + ((gx & 3) * 16 + (gy & 3) * 4 + (gz & 3));
    }
}

template <int DIM>
__device__ __forceinline__ int64_t block_of(int nb, int gx, int gy, int gz)
{
    if (DIM == 2) return (int64_t)((gx >> 2) + 1) * nb + ((gy >> 2) + 1);
    return ((int64_t)((gx >> 2) + 1) * nb + ((gy >> 2) + 1)) * nb + ((gz >> 2) + 1);
}

}  // namespace qmpm
