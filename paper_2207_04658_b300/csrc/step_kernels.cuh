// step_kernels.cuh -- the single-scene MLS-MPM step kernel of libqmpm and the pieces it is
// built from (grid update, G2P gather, the chunk of sorted particles, the tile queue).
// step.cu compiles it for every (dimension, material, state, statistics) class; the same
// source is compiled at run time for one scheme (QMPM_SPECIALIZED_CODEC defined, see
// jit.cpp), where the codec table is a set of compile-time constants.
#pragma once

#include "device_common.cuh"
#include "mpm_device.cuh"

namespace qmpm {

// ------------------------------------------------------------------------------ codec table
// The codec of component c.  The kernels compiled with the library read the scene's table
// from their parameters (P.comp, in the constant bank): a component's word index, shift
// and straddle are run-time values, so each component loads both of its words, computes
// their addresses and ORs itself into the record with a shared-memory atomic.  A kernel
// compiled at run time for one scene class (QMPM_SPECIALIZED_CODEC, jit.cpp) defines
// kSpecDim, kSpecMat, kSpecQuant, kSpecWords, kSpecDither and, for quantized state, the
// table kSpecCodec before including this header; there the decode reads fixed offsets
// (components that share a word share its load), the straddles are known, the encode
// assembles the record words in registers, and the loops over the record's words unroll.
#ifndef QMPM_SPECIALIZED_CODEC
constexpr int kSpecDim = 0, kSpecMat = -1, kSpecWords = 1;
constexpr bool kSpecQuant = false, kSpecDither = false;
__device__ constexpr CompCodec kSpecCodec[1] = {};
#endif

// this instantiation is the one the run-time compilation specialises
template <int DIM, int MAT, bool QUANT>
constexpr bool specialized() { return DIM == kSpecDim && MAT == kSpecMat && QUANT == kSpecQuant; }

// ... and its state is quantized: the codec table is a set of constants
template <int DIM, int MAT, bool QUANT>
constexpr bool specialized_codec() { return QUANT && specialized<DIM, MAT, QUANT>(); }

// The record's word count and whether the stores are dithered: compile-time constants in
// the specialised kernel (its loops over the words unroll), the parameters otherwise.
template <int DIM, int MAT, bool QUANT>
__device__ __forceinline__ int words_of(const StepParams &P)
{
    if constexpr (specialized<DIM, MAT, QUANT>())
        return kSpecWords;
    else
        return P.n_words;
}

template <int DIM, int MAT, bool QUANT>
__device__ __forceinline__ bool dithered(const StepParams &P)
{
    if constexpr (specialized<DIM, MAT, QUANT>())
        return kSpecDither;
    else
        return P.dither != 0;
}

template <int DIM, int MAT, bool QUANT>
__device__ __forceinline__ const CompCodec &codec_of(const StepParams &P, int c)
{
    if constexpr (specialized_codec<DIM, MAT, QUANT>())
        return kSpecCodec[c];
    else
        return P.comp[c];
}

template <int DIM, int MAT>
struct Traits {
    static constexpr int NC = 2 * DIM + DIM * DIM + (MAT == QMPM_FLUID ? 1 : DIM * DIM);
    static constexpr int TN = DIM == 2 ? 64 : 512;  // tile nodes (8^d)
    static constexpr int NOFF = DIM == 2 ? 9 : 27;  // stencil nodes (3^d)
};

// ------------------------------------------------------------------------------ grid update
// Node velocity for G2P: v = mv / m + dt g where m > 0 (else 0); zero within `bound`
// nodes of a wall (sticky).  Used both when staging a tile and on the slow path.
template <int DIM>
__device__ __forceinline__ float4 node_velocity(float4 mm, int gx, int gy, int gz, const StepParams &P)
{
    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const int hi = P.n - 1 - P.bound;
    bool wall = gx < P.bound || gx > hi || gy < P.bound || gy > hi;
    if (DIM == 3) wall = wall || gz < P.bound || gz > hi;
    if (mm.x > 0.0f && !wall) {
        const float inv_m = 1.0f / mm.x;  // one division for the d components
        v.x = mm.y * inv_m + P.dt * P.gravity[0];
        v.y = mm.z * inv_m + P.dt * P.gravity[1];
        if (DIM == 3) v.z = mm.w * inv_m + P.dt * P.gravity[2];
    }
    return v;
}

// Shared-memory tile of 8^d nodes, one float array per quantity (m, momentum or velocity
// components).  In 3D a node's slot is swizzled (z index XOR 4 on odd x rows) so that the
// 64 cells of a block spread over all 32 banks.
template <int DIM>
__device__ __forceinline__ int tile_index(int i, int j, int k)
{
    return DIM == 2 ? (i * 8 + j) : ((i * 8 + j) * 8 + (k ^ ((i & 1) << 2)));
}

__device__ __forceinline__ void stat_add(unsigned long long *stats, int idx, unsigned long long v)
{
    if (v) atomicAdd(stats + idx, v);
}

// G2P gather of one particle, as separable sums: for each (i, j) row, sum over k the
// weighted velocities (S) and the ones weighted by dpz (T); then over j, then over i:
//   v = sum_i wx S_i,  B[:,0] = sum_i wx dpx S_i,  B[:,1] = sum_i wx U_i,  B[:,2] = sum_i wx V_i,
//   with S_i = sum_j wy S_ij, U_i = sum_j wy dpy S_ij, V_i = sum_j wy T_ij.
// FAST reads the shared tile; otherwise the node velocities come from global memory.
template <int DIM, bool FAST>
__device__ __forceinline__ void g2p_gather(const StepParams &P, const float *tvx, const float *tvy,
                                           const float *tvz, int l0, int l1, int l2, const int *base,
                                           const float (*w)[3], const float *dpx, const float *dpy,
                                           const float *dpz, float *vn, float *B)
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float Si[3] = {0.0f, 0.0f, 0.0f}, Ui[3] = {0.0f, 0.0f, 0.0f}, Vi[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float Sij[3] = {0.0f, 0.0f, 0.0f}, Tij[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int k = 0; k < (DIM == 3 ? 3 : 1); ++k) {
                float g0, g1, g2 = 0.0f;
                if (FAST) {
                    const int q = tile_index<DIM>(l0 + i, l1 + j, l2 + k);
                    g0 = tvx[q];
                    g1 = tvy[q];
                    if (DIM == 3) g2 = tvz[q];
                } else {
                    const int gx = base[0] + i, gy = base[1] + j, gz = DIM == 3 ? base[2] + k : 0;
                    const float4 gv = node_velocity<DIM>(P.grid_in[node_addr<DIM>(P.nb, gx, gy, gz)], gx, gy, gz, P);
                    g0 = gv.x;
                    g1 = gv.y;
                    g2 = gv.z;
                }
                const float wz = DIM == 3 ? w[2][k] : 1.0f;
                const float wzd = DIM == 3 ? w[2][k] * dpz[k] : 0.0f;
                Sij[0] += wz * g0;
                Sij[1] += wz * g1;
                if (DIM == 3) {
                    Sij[2] += wz * g2;
                    Tij[0] += wzd * g0;
                    Tij[1] += wzd * g1;
                    Tij[2] += wzd * g2;
                }
            }
            const float wy = w[1][j], wyd = w[1][j] * dpy[j];
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                Si[a] += wy * Sij[a];
                Ui[a] += wyd * Sij[a];
                if (DIM == 3) Vi[a] += wy * Tij[a];
            }
        }
        const float wx = w[0][i], wxd = w[0][i] * dpx[i];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            vn[a] += wx * Si[a];
            B[a * DIM + 0] += wxd * Si[a];
            B[a * DIM + 1] += wx * Ui[a];
            if (DIM == 3) B[a * DIM + 2] += wx * Vi[a];
        }
    }
}


// The particle a thread works on in a chunk of `count` particles: the chunk takes
// nw = ceil(count / 32) warps, and lane l of warp w < nw the particle l * nw + w.  The chunk
// is sorted by cell, so a warp's lanes land on different cells and the shared-memory
// atomics of P2G rarely collide; a short chunk (the last of a tile: most tiles hold a few
// particles more than a multiple of the chunk size) occupies only the warps it needs, and
// the others skip the per-particle work.  Threads without a particle get kThreads.
__device__ __forceinline__ int chunk_particle(int t, int count)
{
    const int nw = min(kThreads / 32, (count + 31) >> 5), w = t >> 5;
    return w < nw ? (t & 31) * nw + w : kThreads;
}

// Shared column of particle p's record words: p's row of 32 rotated by p / 32, which keeps
// both the coalesced staging (lane l of warp w touches particle 32 w + l) and the compute
// mapping of a full chunk (lane l of warp w touches particle 8 l + w) free of bank
// conflicts.
__device__ __forceinline__ int column_of(int p) { return (p & ~31) | ((p + (p >> 5)) & 31); }

// ------------------------------------------------------------------------------ step kernel
// Per-thread event counters of QMPM_FLAG_STATS: saturations, round-ups and round-downs per
// field, out-of-grid and out-of-tile particles.
struct StepCounters {
    unsigned long long sat[4] = {0, 0, 0, 0}, up[4] = {0, 0, 0, 0}, dn[4] = {0, 0, 0, 0};
    unsigned long long oog = 0, oot = 0;
};

// Warp-aggregated flush of the counters into the scene's 16 statistics words.
__device__ __forceinline__ void flush_counters(StepCounters &cnt, unsigned long long *stats)
{
    const int tid = threadIdx.x;
    for (int h = 0; h < 4; ++h) {
        cnt.sat[h] = __reduce_add_sync(0xFFFFFFFFu, (unsigned)cnt.sat[h]);
        cnt.up[h] = __reduce_add_sync(0xFFFFFFFFu, (unsigned)cnt.up[h]);
        cnt.dn[h] = __reduce_add_sync(0xFFFFFFFFu, (unsigned)cnt.dn[h]);
    }
    cnt.oog = __reduce_add_sync(0xFFFFFFFFu, (unsigned)cnt.oog);
    cnt.oot = __reduce_add_sync(0xFFFFFFFFu, (unsigned)cnt.oot);
    if ((tid & 31) == 0 && stats) {
        for (int h = 0; h < 4; ++h) {
            stat_add(stats, h, cnt.sat[h]);
            stat_add(stats, 4 + h, cnt.up[h]);
            stat_add(stats, 8 + h, cnt.dn[h]);
        }
        stat_add(stats, 12, cnt.oog);
        stat_add(stats, 13, cnt.oot);
    }
    cnt = StepCounters();
}

// Four 256-thread CTAs per SM (64 registers a thread): 32 resident warps hide the
// shared-memory and L2 latencies of the chunk loop better than 24 at 80 registers (3D
// cubes, 8.2 M particles: 1.196 -> 1.127 ms quantized, 0.878 -> 0.812 ms FP32, then with
// the fallback P2G rolled 1.094 and 0.788 ms; 16 warps were 11 % slower than 24).  The 3D
// instantiations with saturation counters keep two, which they need to avoid spills.
template <int DIM, bool STATS>
constexpr int step_ctas_per_sm() { return DIM == 3 && STATS ? 2 : 4; }

// Shared memory of the step kernels: G2P velocity tile (3 x TN floats), P2G fixed-point
// tile (4 x TN ints), per-warp maxima, then the chunk's record words (W + 1 columns).
template <int DIM>
constexpr size_t step_smem_fixed() { return (size_t)7 * (DIM == 2 ? 64 : 512) * 4 + (kThreads / 32) * 4; }

// One work item: the chunk ch of the scene described by P.  Its dithered stores use step
// index P.step, or `step` in a multi-scene launch (MULTI).  All threads of the CTA call it
// together (it synchronises).
template <int DIM, int MAT, bool QUANT, bool STATS, bool DO_G2P, bool MULTI = false, bool ROUND_KEYS = !MULTI>
__device__ __forceinline__ void run_chunk(const StepParams &P, const uint32_t ci0, uint32_t step, StepCounters &cnt,
                                          const int tid)
{
    using Tr = Traits<DIM, MAT>;
    constexpr int NC = Tr::NC, TN = Tr::TN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tvx = reinterpret_cast<float *>(smem_raw);  // G2P velocities
    float *tvy = tvx + TN, *tvz = tvy + TN;
    int *tpm = reinterpret_cast<int *>(tvz + TN);       // P2G mass and momentum, fixed point
    int *tpx = tpm + TN, *tpy = tpx + TN, *tpz = tpy + TN;
    float *red = reinterpret_cast<float *>(tpz + TN);   // per-warp maxima (kThreads / 32)
    uint32_t *sw = reinterpret_cast<uint32_t *>(red + kThreads / 32);  // record words, column per particle

    const Chunk ch0 = P.chunks[ci0];
    const uint32_t key = ch0.key;
    int o0, o1, o2 = 0;  // tile origin node: 4 (T - 1) per axis, T the tile's origin block
    if (DIM == 2) {
        o1 = 4 * ((int)(key % P.nb) - 1);
        o0 = 4 * ((int)(key / P.nb) - 1);
    } else {
        o2 = 4 * ((int)(key % P.nb) - 1);
        o1 = 4 * ((int)((key / P.nb) % P.nb) - 1);
        o0 = 4 * ((int)(key / (P.nb * P.nb)) - 1);
    }
    // the tile's chunks: ch0 and the tile_chunks - 1 that follow it in the list; the block
    // fixed point must hold all their contributions to a node: total particles <= 2^b
    // gives each contribution at most 2^(31 - b) - 64 units
    const int n_tile_chunks = (int)ch0.tile_chunks;
    float kfix;
    {
        const Chunk chl = P.chunks[ci0 + n_tile_chunks - 1];
        const uint32_t tile_particles = chl.start + chl.count - ch0.start;
        const int tb = 32 - __clz((int)max(tile_particles, 2u) - 1);  // ceil(log2(particles))
        kfix = (float)((1u << (31 - tb)) - 64u);
    }


    // 1. stage the grid tile (velocities: the grid update) and clear the P2G tile
    for (int t = tid; t < TN; t += kThreads) {
        const int i = DIM == 2 ? (t >> 3) : (t >> 6), j = DIM == 2 ? (t & 7) : ((t >> 3) & 7);
        const int k = DIM == 2 ? 0 : (t & 7);
        const int q = tile_index<DIM>(i, j, k);
        if (DO_G2P) {
            const float4 mm = P.grid_in[node_addr<DIM>(P.nb, o0 + i, o1 + j, o2 + k)];
            const float4 v = node_velocity<DIM>(mm, o0 + i, o1 + j, o2 + k, P);
            tvx[q] = v.x;
            tvy[q] = v.y;
            if (DIM == 3) tvz[q] = v.z;
        }
        tpm[q] = 0;
        tpx[q] = 0;
        tpy[q] = 0;
        if (DIM == 3) tpz[q] = 0;
    }
    const int mycol = column_of(tid);
    // fixed-point units per (m/s) of the tile's momentum sums, a power of two; 0 while no
    // chunk of the tile has had a non-zero momentum contribution (the sums are all zero)
    float scale = 0.0f;
    for (int jc = 0; jc < n_tile_chunks; ++jc) {
    const Chunk ch = P.chunks[ci0 + jc];
    // 2. coalesced load of the chunk's records into shared memory (column per slot)
    if (tid < (int)ch.count)
        for (int j = 0; j < words_of<DIM, MAT, QUANT>(P); ++j)
            sw[j * kThreads + mycol] = P.words[j * P.ld + ch.start + tid];
    __syncthreads();

    const int pj = chunk_particle(tid, (int)ch.count);
    const bool active = pj < (int)ch.count;
    uint32_t *my = sw + column_of(min(pj, kThreads - 1));  // its column of record words, stride kThreads
    const int64_t slot = (int64_t)ch.start + pj;
    // P2G payload, kept across the barrier that fixes the chunk's fixed-point scale
    int pbase[3] = {0, 0, 0};
    float pw[3][3], pf[3] = {0.0f, 0.0f, 0.0f}, pA[DIM * DIM], pv[3] = {0.0f, 0.0f, 0.0f};
    bool p_in_tile = false;
    float bound = 0.0f;
    if (active) {
        float val[NC];
        if (QUANT) {
            // independent per-component extraction: words k and k+1 through a funnel shift
            // (the column carries one padding word after the record)
#pragma unroll
            for (int c = 0; c < (DO_G2P ? DIM : NC); ++c) {
                const CompCodec &cc = codec_of<DIM, MAT, QUANT>(P, c);
                const uint32_t lo = my[cc.word * kThreads], hi = my[(cc.word + 1) * kThreads];
                val[c] = decode_u(__funnelshift_r(lo, hi, cc.shift) & cc.mask, cc);
            }
        } else {
#pragma unroll
            for (int c = 0; c < (DO_G2P ? DIM : NC); ++c) val[c] = __uint_as_float(my[c * kThreads]);
        }
        float *x = val, *v = val + DIM, *C = val + 2 * DIM, *FJ = val + 2 * DIM + DIM * DIM;

        if (DO_G2P) {
            // 3. G2P and particle update
            int base[3] = {0, 0, 0};
            float w[3][3], f[3];
            stencil<DIM>(x, P, base, w, f);
            const int l0 = base[0] - o0, l1 = base[1] - o1, l2 = DIM == 3 ? base[2] - o2 : 0;
            const bool in_tile = l0 >= 0 && l0 <= 5 && l1 >= 0 && l1 <= 5 && l2 >= 0 && l2 <= 5;
            float vn[3] = {0.0f, 0.0f, 0.0f}, B[DIM * DIM];
#pragma unroll
            for (int q = 0; q < DIM * DIM; ++q) B[q] = 0.0f;
            float dpx[3], dpy[3], dpz[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                dpx[i] = ((float)i - f[0]) * P.dx;
                dpy[i] = ((float)i - f[1]) * P.dx;
                dpz[i] = DIM == 3 ? ((float)i - f[2]) * P.dx : 0.0f;
            }
            if (in_tile)
                g2p_gather<DIM, true>(P, tvx, tvy, tvz, l0, l1, l2, base, w, dpx, dpy, dpz, vn, B);
            else
                g2p_gather<DIM, false>(P, tvx, tvy, tvz, l0, l1, l2, base, w, dpx, dpy, dpz, vn, B);
            if (STATS && !in_tile) cnt.oot += 1;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                v[a] = vn[a];
                x[a] += P.dt * vn[a];
#pragma unroll
                for (int b = 0; b < DIM; ++b) C[a * DIM + b] = P.Dinv * B[a * DIM + b];
            }
            // the deformation gradient (or J) is read only now, after the gather
#pragma unroll
            for (int c = 2 * DIM + DIM * DIM; c < NC; ++c) {
                if (QUANT) {
                    const CompCodec &cc = codec_of<DIM, MAT, QUANT>(P, c);
                    const uint32_t lo = my[cc.word * kThreads], hi = my[(cc.word + 1) * kThreads];
                    val[c] = decode_u(__funnelshift_r(lo, hi, cc.shift) & cc.mask, cc);
                } else {
                    val[c] = __uint_as_float(my[c * kThreads]);
                }
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

            // 4. store: dithered encode (Sec. 5) into the particle's shared column
            if constexpr (specialized_codec<DIM, MAT, QUANT>()) {
                // the record words in registers: each component ORs itself into its
                // word(s) at offsets known when the kernel was compiled
                uint32_t ow[kSpecWords + 1];
#pragma unroll
                for (int j = 0; j <= kSpecWords; ++j) ow[j] = 0u;
                uint4 rnd = make_uint4(0, 0, 0, 0);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (dithered<DIM, MAT, QUANT>(P) && (c & 7) == 0) {
                        const uint4 ctr = make_uint4((uint32_t)slot, MULTI ? step : P.step, (uint32_t)(c >> 3), 0u);
                        if (ROUND_KEYS)
                            rnd = philox4x32_rk(ctr, P.round_key);
                        else
                            rnd = philox4x32(ctr, P.seed_lo, P.seed_hi);
                    }
                    int fl;
                    const CompCodec &cc = codec_of<DIM, MAT, QUANT>(P, c);
                    const uint32_t u = encode_f32(val[c], cc, dithered<DIM, MAT, QUANT>(P), dither_threshold(rnd, c), fl);
                    ow[cc.word] |= u << cc.shift;
                    if (cc.straddle) ow[cc.word + 1] |= __funnelshift_l(u, 0u, cc.shift);
                    val[c] = decode_u(u, cc);  // the stored (quantized) value
                    if (STATS) {
                        const int h = c < DIM ? 0 : c < 2 * DIM ? 1 : c < 2 * DIM + DIM * DIM ? 2 : 3;
                        cnt.sat[h] += (fl & 1);
                        cnt.up[h] += (fl >> 1) & 1;
                        cnt.dn[h] += (fl >> 2) & 1;
                    }
                }
#pragma unroll
                for (int j = 0; j < kSpecWords; ++j) my[j * kThreads] = ow[j];
            } else if (QUANT) {
                // every component ORs itself into its word(s) with a fire-and-forget shared
                // atomic, so the components do not wait on one another
                for (int j = 0; j < P.n_words; ++j) my[j * kThreads] = 0u;
                uint4 rnd = make_uint4(0, 0, 0, 0);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (P.dither && (c & 7) == 0) {
                        // the round keys are operands where P sits in the parameter space; the
                        // multi-scene kernel reads P from shared memory, and there the two
                        // additions per round are cheaper than loading the keys
                        const uint4 ctr = make_uint4((uint32_t)slot, MULTI ? step : P.step, (uint32_t)(c >> 3), 0u);
                        if (ROUND_KEYS)
                            rnd = philox4x32_rk(ctr, P.round_key);
                        else
                            rnd = philox4x32(ctr, P.seed_lo, P.seed_hi);
                    }
                    int fl;
                    const CompCodec &cc = codec_of<DIM, MAT, QUANT>(P, c);
                    const uint32_t u = encode_f32(val[c], cc, P.dither != 0, dither_threshold(rnd, c), fl);
                    atomicOr(my + cc.word * kThreads, u << cc.shift);
                    if (cc.straddle) atomicOr(my + (cc.word + 1) * kThreads, __funnelshift_l(u, 0u, cc.shift));
                    val[c] = decode_u(u, cc);  // the stored (quantized) value
                    if (STATS) {
                        // the field of component c (x, v, C, F/J), folded at compile time
                        const int h = c < DIM ? 0 : c < 2 * DIM ? 1 : c < 2 * DIM + DIM * DIM ? 2 : 3;
                        cnt.sat[h] += (fl & 1);
                        cnt.up[h] += (fl >> 1) & 1;
                        cnt.dn[h] += (fl >> 2) & 1;
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) my[c * kThreads] = __float_as_uint(val[c]);
            }
        }

        // 5a. P2G payload of the (stored) state: stencil, m v and the affine matrix A
        const bool oog = stencil<DIM>(x, P, pbase, pw, pf);
        if (STATS && oog) cnt.oog += 1;
        const int l0 = pbase[0] - o0, l1 = pbase[1] - o1, l2 = DIM == 3 ? pbase[2] - o2 : 0;
        // out-of-grid particles (clamped stencil, weights outside the B-spline range) and
        // particles that left their tile go through global memory in FP32
        p_in_tile = !oog && l0 >= 0 && l0 <= 5 && l1 >= 0 && l1 <= 5 && l2 >= 0 && l2 <= 5;
        if (STATS && !DO_G2P && !p_in_tile) cnt.oot += 1;
        float tau[DIM * DIM];
        kirchhoff<DIM, MAT>(FJ, P, tau);
#pragma unroll
        for (int q = 0; q < DIM * DIM; ++q) pA[q] = P.stress_coef * tau[q] + P.p_mass * C[q];
#pragma unroll
        for (int a = 0; a < DIM; ++a) pv[a] = v[a];
        if (p_in_tile) {
            // |v_a + (A dpos)_a / m| <= |v_a| + 1.5 dx sum_b |A_ab| / m on the whole stencil
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                float rowsum = 0.0f;
#pragma unroll
                for (int b = 0; b < DIM; ++b) rowsum += fabsf(pA[a * DIM + b]);
                bound = fmaxf(bound, fabsf(v[a]) + 1.5f * P.dx * rowsum * P.inv_p_mass);
            }
        }
    }
    // 5b. scale of the block fixed point: the largest in-tile contribution maps inside
    //     kfix, so no sum over the tile's particles can overflow 32 bits
    {
        float bm = __uint_as_float(__reduce_max_sync(0xFFFFFFFFu, __float_as_uint(bound)));
        if ((tid & 31) == 0) red[tid >> 5] = bm;
    }
    __syncthreads();
    float bmax = 0.0f;
#pragma unroll
    for (int w8 = 0; w8 < kThreads / 32; ++w8) bmax = fmaxf(bmax, red[w8]);
    // the largest power of two that maps this chunk's largest contribution inside kfix; a
    // chunk that needs a smaller one than the tile's sums so far shifts those sums down first
    // (kfix / bmax with its mantissa bits cleared, clamped so that a vanishing bmax cannot
    // make it infinite; the division's rounding stays inside the 64 units kfix keeps free)
    const float want =
        bmax > 0.0f ? __uint_as_float(__float_as_uint(fminf(kfix / bmax, 1.7e38f)) & 0xFF800000u) : 0.0f;
    if (want > 0.0f && scale == 0.0f) {
        scale = want;
    } else if (want > 0.0f && want < scale) {
        const int sh = (int)log2f(scale / want);
        for (int t = tid; t < TN; t += kThreads) {
            tpx[t] >>= sh;
            tpy[t] >>= sh;
            if (DIM == 3) tpz[t] >>= sh;
        }
        scale = want;
        __syncthreads();
    }
    if (active) {
        // 5c. scatter: momentum w (v + A dpos / m) * scale and mass w * kfix as integers
        float dpx[3], dpy[3], dpz[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            dpx[i] = ((float)i - pf[0]) * P.dx;
            dpy[i] = ((float)i - pf[1]) * P.dx;
            dpz[i] = DIM == 3 ? ((float)i - pf[2]) * P.dx : 0.0f;
        }
        if (p_in_tile) {
            const int l0 = pbase[0] - o0, l1 = pbase[1] - o1, l2 = DIM == 3 ? pbase[2] - o2 : 0;
            float As[DIM * DIM], vs[3];
            const float s_use = scale > 0.0f ? scale : 1.0f;  // no momentum yet: any scale
            const float am = s_use * P.inv_p_mass;
#pragma unroll
            for (int q = 0; q < DIM * DIM; ++q) As[q] = pA[q] * am;
#pragma unroll
            for (int a = 0; a < DIM; ++a) vs[a] = pv[a] * s_use;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float ui[3];
#pragma unroll
                for (int a = 0; a < DIM; ++a) ui[a] = vs[a] + As[a * DIM + 0] * dpx[i];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float uij[3];
#pragma unroll
                    for (int a = 0; a < DIM; ++a) uij[a] = ui[a] + As[a * DIM + 1] * dpy[j];
                    const float wij = pw[0][i] * pw[1][j];
#pragma unroll
                    for (int k = 0; k < (DIM == 3 ? 3 : 1); ++k) {
                        const float wt = DIM == 3 ? wij * pw[2][k] : wij;
                        const int q = tile_index<DIM>(l0 + i, l1 + j, l2 + k);
                        atomicAdd(tpm + q, __float2int_rn(wt * kfix));
                        if (DIM == 3) {
                            atomicAdd(tpx + q, __float2int_rn(wt * (uij[0] + As[2] * dpz[k])));
                            atomicAdd(tpy + q, __float2int_rn(wt * (uij[1] + As[5] * dpz[k])));
                            atomicAdd(tpz + q, __float2int_rn(wt * (uij[2] + As[8] * dpz[k])));
                        } else {
                            atomicAdd(tpx + q, __float2int_rn(wt * uij[0]));
                            atomicAdd(tpy + q, __float2int_rn(wt * uij[1]));
                        }
                    }
                }
            }
        } else {
            // slow path: FP32 global atomics straight into the grid (rolled loops over local
            // copies: rarely taken, and unrolled it would raise the hot path's register need)
            float spw[3][3], sdx[3], sdy[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                sdx[a] = dpx[a];
                sdy[a] = dpy[a];
#pragma unroll
                for (int b = 0; b < 3; ++b) spw[a][b] = pw[a][b];
            }
#pragma unroll 1
            for (int i = 0; i < 3; ++i)
#pragma unroll 1
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int k = 0; k < (DIM == 3 ? 3 : 1); ++k) {
                        const float wt = spw[0][i] * spw[1][j] * (DIM == 3 ? spw[2][k] : 1.0f);
                        const float dp[3] = {sdx[i], sdy[j], dpz[k]};
                        float mom[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                        for (int a = 0; a < DIM; ++a) {
                            float acc = P.p_mass * pv[a];
#pragma unroll
                            for (int b = 0; b < DIM; ++b) acc += pA[a * DIM + b] * dp[b];
                            mom[a] = wt * acc;
                        }
                        const int gx = pbase[0] + i, gy = pbase[1] + j, gz = DIM == 3 ? pbase[2] + k : 0;
                        atomicAdd(P.grid_out + node_addr<DIM>(P.nb, gx, gy, gz),
                                  make_float4(wt * P.p_mass, mom[0], mom[1], DIM == 3 ? mom[2] : 0.0f));
                        P.touched_out[block_of<DIM>(P.nb, gx, gy, gz)] = 1;
                    }
        }
    }
    __syncthreads();

    // 6. coalesced store of the new records
    if (DO_G2P && tid < (int)ch.count)
        for (int j = 0; j < words_of<DIM, MAT, QUANT>(P); ++j)
            __stcs(P.words + j * P.ld + ch.start + tid, sw[j * kThreads + mycol]);
    if (jc + 1 < n_tile_chunks) __syncthreads();  // the next chunk reuses the record columns
    }  // chunks of the tile

    // 7. the P2G tile flush: one vector atomic per node that received mass
    const float mm = P.p_mass / (scale > 0.0f ? scale : 1.0f);  // momentum units -> m v
    const float mmass = P.p_mass / kfix;                        // mass units -> m
    for (int t = tid; t < TN; t += kThreads) {
        const int i = DIM == 2 ? (t >> 3) : (t >> 6), j = DIM == 2 ? (t & 7) : ((t >> 3) & 7);
        const int k = DIM == 2 ? 0 : (t & 7);
        const int q = tile_index<DIM>(i, j, k);
        const int im = tpm[q];
        if (im != 0) {
            atomicAdd(P.grid_out + node_addr<DIM>(P.nb, o0 + i, o1 + j, o2 + k),
                      make_float4((float)im * mmass, (float)tpx[q] * mm, (float)tpy[q] * mm,
                                  DIM == 3 ? (float)tpz[q] * mm : 0.0f));
        }
    }
    if (tid < (1 << DIM)) {
        // the tile's 2^d blocks: origin block T = o / 4 + 1 per axis
        const int T0 = (o0 >> 2) + 1, T1 = (o1 >> 2) + 1, T2 = (o2 >> 2) + 1;
        const int i = tid & 1, j = (tid >> 1) & 1, k = (tid >> 2) & 1;
        const int64_t blk = DIM == 2 ? (int64_t)(T0 + i) * P.nb + (T1 + j)
                                     : ((int64_t)(T0 + i) * P.nb + (T1 + j)) * P.nb + (T2 + k);
        P.touched_out[blk] = 1;
    }
    __syncthreads();
}

// The CTAs of a launch take tiles from a shared counter (P.work[0]) instead of a fixed
// stride: tiles hold from one to sixteen chunks, and a fixed stride left the average SM
// idle for 6 % of the launch.  The last CTA to finish puts both words back to zero for the
// next launch (every CTA has taken its last ticket before it counts itself finished).
__device__ __forceinline__ uint32_t take_tile(uint32_t *work, uint32_t *slot)
{
    if (threadIdx.x == 0) *slot = atomicAdd(work, 1u);
    __syncthreads();
    return *slot;
}

__device__ __forceinline__ void finish_launch(uint32_t *work)
{
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(work + 1, 1u) == gridDim.x - 1) {
            work[0] = 0u;
            work[1] = 0u;
            __threadfence();
        }
    }
}

template <int DIM, int MAT, bool QUANT, bool STATS, bool DO_G2P>
__global__ void __launch_bounds__(kThreads, step_ctas_per_sm<DIM, STATS>()) step_kernel(const __grid_constant__ StepParams P)
{
    __shared__ uint32_t ticket;
    StepCounters cnt;
    const int tid = threadIdx.x;
    const uint32_t n_tiles = *P.n_tiles;
    for (;;) {
        // run_chunk ends with a barrier, so every thread has read the ticket before thread 0
        // takes the next one
        const uint32_t ti = take_tile(P.work, &ticket);
        if (ti >= n_tiles) break;
        run_chunk<DIM, MAT, QUANT, STATS, DO_G2P>(P, P.tile_first[ti], 0u, cnt, tid);
    }
    if (STATS) flush_counters(cnt, P.stats);
    finish_launch(P.work);
}

}  // namespace qmpm
