// step.cu -- the MLS-MPM step kernels of libqmpm (Sec. 8.1's simulator, quantized as in
// Sec. 3.1 Eq. 1 with the dithered store of Sec. 5 and the bit pack of Sec. 7).
//
// One launch advances the whole scene by one step, fused as G2P(t) -> store -> P2G(t+1):
//   1. stage the tile's 8^d grid nodes of the P2G result of step t into shared memory,
//      turning momentum into velocity with gravity and sticky walls on the way (the
//      grid update),
//   2. decode each particle's packed record (words staged in shared memory),
//   3. G2P: gather v, C; x += dt v; F = (I + dt C) F (or J = (1 + dt tr C) J),
//   4. dithered encode of the new state, whole-word stores back to HBM,
//   5. P2G of step t+1 from the decoded quantized values into a shared-memory tile,
//      flushed to the other grid buffer with one vector atomic per touched node.
// Work item: a chunk of up to 256 sorted particles that share one tile (2^d blocks of
// 4^d nodes); one thread per particle, records staged through shared memory so that
// global loads and stores stay coalesced; persistent CTAs stride over the chunk list.
// Particles that drifted out of their tile since the last re-sort take a slow path
// through global memory.
#include <cstdio>

#include "step_kernels.cuh"

namespace qmpm {

// One scene of a batch stepped by its own launch (parameters in the constant bank, as the
// step kernel), but with the dither step index from the member's device counter so that a
// captured graph can be replayed.
template <int DIM, int MAT, bool QUANT, bool STATS>
__global__ void __launch_bounds__(kThreads, step_ctas_per_sm<DIM, STATS>())
    step_kernel_ctr(const __grid_constant__ StepParams P)
{
    StepCounters cnt;
    const int tid = threadIdx.x;
    const uint32_t step = *P.step_ctr + 1u;
    const uint32_t n_tiles = *P.n_tiles;
    __shared__ uint32_t ticket;
    for (;;) {
        const uint32_t ti = take_tile(P.work, &ticket);
        if (ti >= n_tiles) break;
        run_chunk<DIM, MAT, QUANT, STATS, true, true, true>(P, P.tile_first[ti], step, cnt, tid);
    }
    if (STATS) flush_counters(cnt, P.stats);
    finish_launch(P.work);
}

// Multi-scene launch: the work queue is the concatenation of the members' tile lists
// (member-major); the CTAs take its items in turn, copying a member's parameters into
// shared memory when their items move on to the next member.  The members share the template
// class (dimension, material, quantized or not); everything else (grid size, scheme,
// physics, buffers, step index) is per member.
// CTAs per SM as for the single-scene kernel (a 32-scene batch of 3D serving scenes:
// 1.86 ms per step with two, 1.73 with three, 1.68 with four).
template <int DIM, int MAT, bool QUANT, bool STATS>
__global__ void __launch_bounds__(kThreads, step_ctas_per_sm<DIM, STATS>())
    step_kernel_multi(const StepParams *__restrict__ tab, int n_members)
{
    __shared__ uint32_t first[kMaxMembers + 1];  // prefix sums of the members' chunk counts
    __shared__ __align__(16) StepParams Ps;
    static_assert(sizeof(StepParams) % 4 == 0, "StepParams is copied as 32-bit words");
    const int tid = threadIdx.x;
    if (tid < n_members) first[tid + 1] = *tab[tid].n_tiles;
    if (tid == 0) first[0] = 0;
    __syncthreads();
    if (tid == 0)
        for (int m = 0; m < n_members; ++m) first[m + 1] += first[m];
    __syncthreads();
    const uint32_t total = first[n_members];
    StepCounters cnt;
    int cur = -1;
    uint32_t step = 0;
    // the launch's queue of items lives in the first member's queue words (a member is in
    // one launch at a time)
    uint32_t *queue = tab[0].work;
    __shared__ uint32_t ticket;
    for (;;) {
        const uint32_t item = take_tile(queue, &ticket);
        if (item >= total) break;
        int lo = 0, hi = n_members;  // first[lo] <= item < first[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (first[mid] <= item) lo = mid;
            else hi = mid;
        }
        if (lo != cur) {
            if (STATS && cur >= 0) flush_counters(cnt, Ps.stats);
            __syncthreads();  // nobody reads the previous member's parameters any more
            const uint32_t *src = reinterpret_cast<const uint32_t *>(tab + lo);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&Ps);
            for (int q = tid; q < (int)(sizeof(StepParams) / 4); q += kThreads) dst[q] = src[q];
            __syncthreads();
            cur = lo;
            step = *Ps.step_ctr + 1u;
        }
        run_chunk<DIM, MAT, QUANT, STATS, true, true>(Ps, Ps.tile_first[item - first[lo]], step, cnt, tid);
    }
    if (STATS && cur >= 0) flush_counters(cnt, Ps.stats);
    finish_launch(queue);
}

// ------------------------------------------------------------------------------ grid clear
// Zero the blocks of a grid buffer that were touched and reset their flags: a warp reads
// 32 flags and zeroes every flagged block with coalesced 16-byte stores.
template <int DIM>
__global__ void clear_kernel(float4 *grid, uint8_t *touched, int64_t n_blocks)
{
    constexpr int BN = DIM == 2 ? 16 : 64;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b0 = warp * 32; b0 < n_blocks; b0 += n_warps * 32) {
        const int64_t b = b0 + lane;
        const bool t = b < n_blocks && touched[b];
        unsigned mask = __ballot_sync(0xFFFFFFFFu, t);
        if (t) touched[b] = 0;
        while (mask) {
            const int l = __ffs(mask) - 1;
            mask &= mask - 1;
            float4 *blk = grid + (b0 + l) * BN;
            for (int q = lane; q < BN; q += 32) blk[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
}

// Clear of several members' consumed grid buffers in one launch: member m owns the
// virtual blocks [first, first + n_blocks) (ranges start on multiples of 32).
__global__ void clear_kernel_multi(const ClearItem *__restrict__ items, int n_items, int64_t virtual_blocks)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v0 = warp * 32; v0 < virtual_blocks; v0 += n_warps * 32) {
        int lo = 0, hi = n_items;  // items[lo].first <= v0 < items[hi].first
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (items[mid].first <= v0) lo = mid;
            else hi = mid;
        }
        const ClearItem it = items[lo];
        const int64_t b0 = v0 - it.first;
        const int64_t b = b0 + lane;
        const bool t = b < it.n_blocks && it.touched[b];
        unsigned mask = __ballot_sync(0xFFFFFFFFu, t);
        if (t) it.touched[b] = 0;
        while (mask) {
            const int l = __ffs(mask) - 1;
            mask &= mask - 1;
            float4 *blk = it.grid + (b0 + l) * it.block_nodes;
            for (int q = lane; q < it.block_nodes; q += 32) blk[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
}

__global__ void advance_kernel(uint32_t *ctr, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ctr[i] += 1u;
}

// ------------------------------------------------------------------------------ codec kernels
// Initial state (FP64 AoS from the host) -> word planes, dithered store of step 0.
template <bool QUANT>
__global__ void encode_init_kernel(const __grid_constant__ StepParams P, const double *s, int64_t N)
{
    extern __shared__ uint32_t sw_init[];
    const int tid = threadIdx.x;
    uint32_t *my = sw_init + tid;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + tid;
    if (p >= N) return;
    if (!QUANT) {
        for (int c = 0; c < P.n_comp; ++c) P.words[c * P.ld + p] = __float_as_uint((float)s[p * P.n_comp + c]);
        return;
    }
    for (int j = 0; j < P.n_words; ++j) my[j * blockDim.x] = 0u;
    uint4 rnd = make_uint4(0, 0, 0, 0);
    for (int c = 0; c < P.n_comp; ++c) {
        if (P.dither && (c & 7) == 0)
            rnd = philox4x32(make_uint4((uint32_t)p, 0u, (uint32_t)(c >> 3), 0u), P.seed_lo, P.seed_hi);
        int fl;
        const uint32_t u = encode_f64(s[p * P.n_comp + c], P.comp[c], P.dither != 0, dither_threshold(rnd, c), fl);
        if (P.stats && fl) {
            const int h = P.comp[c].field;
            atomicAdd(P.stats + ((fl & 1) ? h : (fl & 2) ? 4 + h : 8 + h), 1ull);
        }
        uint32_t *w = my;
        const CompCodec &cc = P.comp[c];
        w[cc.word * blockDim.x] |= u << cc.shift;
        if (cc.straddle) w[(cc.word + 1) * blockDim.x] |= u >> (32 - cc.shift);
    }
    for (int j = 0; j < P.n_words; ++j) P.words[j * P.ld + p] = my[j * blockDim.x];
}

// Word planes -> FP64 AoS (exact decode), for readback.
template <bool QUANT>
__global__ void decode_f64_kernel(const __grid_constant__ StepParams P, double *s, int64_t N)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    for (int c = 0; c < P.n_comp; ++c) {
        const CompCodec &cc = P.comp[c];
        if (!QUANT) {
            s[p * P.n_comp + c] = (double)__uint_as_float(P.words[c * P.ld + p]);
            continue;
        }
        uint32_t lo = P.words[cc.word * P.ld + p] >> cc.shift;
        if (cc.straddle) lo |= P.words[(cc.word + 1) * P.ld + p] << (32 - cc.shift);
        s[p * P.n_comp + c] = decode_f64(lo & cc.mask, cc);
    }
}

// z = (1/N) sum |x|^2 accumulated in FP64 (position measurement).
template <int DIM, bool QUANT>
__global__ void measure_kernel(const __grid_constant__ StepParams P, int64_t N, double *z)
{
    __shared__ double red[kThreads / 32];
    double acc = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const CompCodec &cc = P.comp[a];
            double xa;
            if (!QUANT) {
                xa = (double)__uint_as_float(P.words[a * P.ld + p]);
            } else {
                uint32_t lo = P.words[cc.word * P.ld + p] >> cc.shift;
                if (cc.straddle) lo |= P.words[(cc.word + 1) * P.ld + p] << (32 - cc.shift);
                xa = decode_f64(lo & cc.mask, cc);
            }
            acc += xa * xa;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) t += red[i];
        atomicAdd(z, t / (double)N);
    }
}

__global__ void count_flags_kernel(const uint8_t *flags, int64_t n, unsigned long long *out)
{
    unsigned long long acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += flags[i] ? 1ull : 0ull;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

cudaError_t launch_count_flags(Ctx &c, const uint8_t *flags, int64_t n, unsigned long long *d_out)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)c.n_sms * 8) blocks = (int64_t)c.n_sms * 8;
    if (blocks < 1) blocks = 1;
    count_flags_kernel<<<(unsigned)blocks, 256, 0, c.stream>>>(flags, n, d_out);
    return cudaGetLastError();
}

// FP32 values [N][nc] -> word planes with the dithered store of `step` (codec tests).
__global__ void pack_f32_kernel(const __grid_constant__ StepParams P, const float *vals, int64_t N)
{
    extern __shared__ uint32_t sw_pack[];
    const int tid = threadIdx.x;
    uint32_t *my = sw_pack + tid;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + tid;
    if (p >= N) return;
    for (int j = 0; j < P.n_words; ++j) my[j * blockDim.x] = 0u;
    uint4 rnd = make_uint4(0, 0, 0, 0);
    for (int c = 0; c < P.n_comp; ++c) {
        if (P.dither && (c & 7) == 0)
            rnd = philox4x32(make_uint4((uint32_t)p, P.step, (uint32_t)(c >> 3), 0u), P.seed_lo, P.seed_hi);
        int fl;
        const uint32_t u = encode_f32(vals[p * P.n_comp + c], P.comp[c], P.dither != 0, dither_threshold(rnd, c), fl);
        if (P.stats && fl) {
            const int h = P.comp[c].field;
            atomicAdd(P.stats + ((fl & 1) ? h : (fl & 2) ? 4 + h : 8 + h), 1ull);
        }
        const CompCodec &cc = P.comp[c];
        my[cc.word * blockDim.x] |= u << cc.shift;
        if (cc.straddle) my[(cc.word + 1) * blockDim.x] |= u >> (32 - cc.shift);
    }
    for (int j = 0; j < P.n_words; ++j) P.words[j * P.ld + p] = my[j * blockDim.x];
}

__global__ void unpack_f32_kernel(const __grid_constant__ StepParams P, float *vals, int64_t N)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    for (int c = 0; c < P.n_comp; ++c) {
        const CompCodec &cc = P.comp[c];
        uint32_t lo = P.words[cc.word * P.ld + p] >> cc.shift;
        if (cc.straddle) lo |= P.words[(cc.word + 1) * P.ld + p] << (32 - cc.shift);
        vals[p * P.n_comp + c] = decode_u(lo & cc.mask, cc);
    }
}

// ------------------------------------------------------------------------------ launchers
void fill_params(const Ctx &c, StepParams &p)
{
    memset(&p, 0, sizeof(p));
    const qmpm_scene_t &s = c.scene;
    p.n = c.n;
    p.nb = c.nb;
    p.bound = s.bound;
    p.n_comp = c.n_comp;
    p.dt = (float)s.dt;
    p.inv_dx = (float)c.n;
    p.dx = 1.0f / (float)c.n;
    p.Dinv = 4.0f * (float)c.n * (float)c.n;
    p.p_mass = (float)s.p_mass;
    p.inv_p_mass = (float)(1.0 / s.p_mass);
    p.stress_coef = (float)(-s.dt * s.p_vol * 4.0 * (double)c.n * (double)c.n);
    const double mu = s.E / (2.0 * (1.0 + s.nu));
    const double la = s.E * s.nu / ((1.0 + s.nu) * (1.0 - 2.0 * s.nu));
    p.mu = (float)mu;
    p.lambda = (float)la;
    p.bulk = (float)s.bulk;
    for (int a = 0; a < 3; ++a) p.gravity[a] = (float)s.gravity[a];
    p.n_words = c.W;
    p.dither = s.dither;
    p.seed_lo = (uint32_t)s.seed;
    p.seed_hi = (uint32_t)(s.seed >> 32);
    for (int r = 0; r < 10; ++r) {
        p.round_key[0][r] = p.seed_lo + (uint32_t)r * 0x9E3779B9u;
        p.round_key[1][r] = p.seed_hi + (uint32_t)r * 0xBB67AE85u;
    }
    for (int q = 0; q < c.n_comp; ++q) p.comp[q] = c.cc[q];
    p.words = c.words[c.cur];
    p.ld = c.ld;
    p.chunks = c.chunks;
    p.n_chunks = c.n_chunks;
    p.tile_first = c.tile_first;
    p.n_tiles = c.n_tiles;
    p.stats = (s.flags & QMPM_FLAG_STATS) ? c.d_stats : nullptr;
    p.work = reinterpret_cast<uint32_t *>(c.d_stats + 16);  // the word after the 16 statistics
}

size_t step_smem_bytes(int dim, int W)
{
    const int TN = dim == 2 ? 64 : 512;
    return (size_t)7 * TN * sizeof(float) + (kThreads / 32) * sizeof(float) +
           (size_t)(W + 1) * kThreads * sizeof(uint32_t);
}

static size_t step_smem(const Ctx &c) { return step_smem_bytes(c.scene.dim, c.W); }

template <int DIM, int MAT, bool QUANT, bool STATS, bool DO_G2P>
static cudaError_t launch_step_t(Ctx &c, const StepParams &p)
{
    auto kern = step_kernel<DIM, MAT, QUANT, STATS, DO_G2P>;
    const size_t smem = step_smem(c);
    // persistent grid: as many CTAs as fit on every SM at once (queried once per shared
    // memory size of this instantiation)
    static size_t cached_smem = 0;
    static int cached_per_sm = 0;
    if (cached_smem != smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
        if (e != cudaSuccess) return e;
        cached_per_sm = per_sm > 0 ? per_sm : 1;
        cached_smem = smem;
    }
    kern<<<c.n_sms * cached_per_sm, kThreads, smem, c.stream>>>(p);
    return cudaGetLastError();
}

template <bool DO_G2P>
static cudaError_t dispatch_step(Ctx &c, const StepParams &p)
{
    const bool st = (c.scene.flags & QMPM_FLAG_STATS) != 0;
    const int key = (c.scene.dim == 3 ? 100 : 0) + c.scene.material * 10 + (c.quant ? 2 : 0) + (st ? 1 : 0);
#define QMPM_CASE(D, M, Q, S)                                                                      \
    case (D == 3 ? 100 : 0) + M * 10 + (Q ? 2 : 0) + (S ? 1 : 0):                                    \
        return launch_step_t<D, M, Q, S, DO_G2P>(c, p);
#define QMPM_CASES_DM(D, M) QMPM_CASE(D, M, false, false) QMPM_CASE(D, M, true, false) QMPM_CASE(D, M, true, true) \
    QMPM_CASE(D, M, false, true)
    switch (key) {
        QMPM_CASES_DM(2, 0)
        QMPM_CASES_DM(2, 1)
        QMPM_CASES_DM(2, 2)
        QMPM_CASES_DM(3, 0)
        QMPM_CASES_DM(3, 1)
        QMPM_CASES_DM(3, 2)
    default:
        return cudaErrorInvalidValue;
    }
#undef QMPM_CASES_DM
#undef QMPM_CASE
}

cudaError_t launch_p2g(Ctx &c)
{
    StepParams p;
    fill_params(c, p);
    p.grid_in = nullptr;
    p.grid_out = c.grid[c.gcur];
    p.touched_out = c.touched[c.gcur];
    p.step = 0;
    return dispatch_step<false>(c, p);
}

void step_params(const Ctx &c, StepParams &p, uint32_t step)
{
    fill_params(c, p);
    p.grid_in = c.grid[c.gcur];
    p.grid_out = c.grid[1 - c.gcur];
    p.touched_out = c.touched[1 - c.gcur];
    p.step = step;
}

cudaError_t launch_g2p2g(Ctx &c, uint32_t step)
{
    StepParams p;
    step_params(c, p, step);
    if (c.spec_kernel) return launch_specialized(c, p);
    return dispatch_step<true>(c, p);
}

template <int DIM, int MAT, bool QUANT, bool STATS>
static cudaError_t launch_multi_t(const StepParams *d_tab, int n, size_t smem, int n_sms, cudaStream_t s)
{
    auto kern = step_kernel_multi<DIM, MAT, QUANT, STATS>;
    static size_t cached_smem = 0;
    static int cached_per_sm = 0;
    if (cached_smem != smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
        if (e != cudaSuccess) return e;
        cached_per_sm = per_sm > 0 ? per_sm : 1;
        cached_smem = smem;
    }
    if (!d_tab || n <= 0) return cudaSuccess;  // attributes only (before a stream capture)
    kern<<<n_sms * cached_per_sm, kThreads, smem, s>>>(d_tab, n);
    return cudaGetLastError();
}

cudaError_t launch_step_multi(int dim, int material, bool quant, bool stats, const StepParams *d_tab, int n,
                              size_t smem, int n_sms, cudaStream_t s)
{
    if (n < 0 || n > kMaxMembers) return cudaErrorInvalidValue;
    const int key = (dim == 3 ? 100 : 0) + material * 10 + (quant ? 2 : 0) + (stats ? 1 : 0);
#define QMPM_CASE(D, M, Q, S)                                                                      \
    case (D == 3 ? 100 : 0) + M * 10 + (Q ? 2 : 0) + (S ? 1 : 0):                                    \
        return launch_multi_t<D, M, Q, S>(d_tab, n, smem, n_sms, s);
#define QMPM_CASES_DM(D, M) QMPM_CASE(D, M, false, false) QMPM_CASE(D, M, true, false) QMPM_CASE(D, M, true, true) \
    QMPM_CASE(D, M, false, true)
    switch (key) {
        QMPM_CASES_DM(2, 0)
        QMPM_CASES_DM(2, 1)
        QMPM_CASES_DM(2, 2)
        QMPM_CASES_DM(3, 0)
        QMPM_CASES_DM(3, 1)
        QMPM_CASES_DM(3, 2)
    default:
        return cudaErrorInvalidValue;
    }
#undef QMPM_CASES_DM
#undef QMPM_CASE
}

template <int DIM, int MAT, bool QUANT, bool STATS>
static cudaError_t launch_ctr_t(const StepParams *p, size_t smem, int n_sms, cudaStream_t s)
{
    auto kern = step_kernel_ctr<DIM, MAT, QUANT, STATS>;
    static size_t cached_smem = 0;
    static int cached_per_sm = 0;
    if (cached_smem != smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
        if (e != cudaSuccess) return e;
        cached_per_sm = per_sm > 0 ? per_sm : 1;
        cached_smem = smem;
    }
    if (!p) return cudaSuccess;  // attributes only (before a stream capture)
    kern<<<n_sms * cached_per_sm, kThreads, smem, s>>>(*p);
    return cudaGetLastError();
}

cudaError_t launch_step_ctr(int dim, int material, bool quant, bool stats, const StepParams *p, size_t smem,
                            int n_sms, cudaStream_t s)
{
    const int key = (dim == 3 ? 100 : 0) + material * 10 + (quant ? 2 : 0) + (stats ? 1 : 0);
#define QMPM_CASE(D, M, Q, S)                                                                      \
    case (D == 3 ? 100 : 0) + M * 10 + (Q ? 2 : 0) + (S ? 1 : 0):                                    \
        return launch_ctr_t<D, M, Q, S>(p, smem, n_sms, s);
#define QMPM_CASES_DM(D, M) QMPM_CASE(D, M, false, false) QMPM_CASE(D, M, true, false) QMPM_CASE(D, M, true, true) \
    QMPM_CASE(D, M, false, true)
    switch (key) {
        QMPM_CASES_DM(2, 0)
        QMPM_CASES_DM(2, 1)
        QMPM_CASES_DM(2, 2)
        QMPM_CASES_DM(3, 0)
        QMPM_CASES_DM(3, 1)
        QMPM_CASES_DM(3, 2)
    default:
        return cudaErrorInvalidValue;
    }
#undef QMPM_CASES_DM
#undef QMPM_CASE
}

cudaError_t launch_clear_multi(const ClearItem *d_items, int n, int64_t virtual_blocks, int n_sms, cudaStream_t s)
{
    if (n <= 0 || virtual_blocks <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t ctas = (virtual_blocks / 32 + threads / 32 - 1) / (threads / 32);
    if (ctas > (int64_t)n_sms * 8) ctas = (int64_t)n_sms * 8;
    if (ctas < 1) ctas = 1;
    clear_kernel_multi<<<(unsigned)ctas, threads, 0, s>>>(d_items, n, virtual_blocks);
    return cudaGetLastError();
}

cudaError_t launch_advance(uint32_t *d_ctr, int n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    advance_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_ctr, n);
    return cudaGetLastError();
}

cudaError_t launch_clear(Ctx &c, int buf)
{
    const int threads = 256;
    const int64_t warps_needed = (c.n_blocks + 31) / 32;
    int64_t ctas = (warps_needed + threads / 32 - 1) / (threads / 32);
    if (ctas > (int64_t)c.n_sms * 8) ctas = (int64_t)c.n_sms * 8;
    if (ctas < 1) ctas = 1;
    if (c.scene.dim == 2)
        clear_kernel<2><<<(unsigned)ctas, threads, 0, c.stream>>>(c.grid[buf], c.touched[buf], c.n_blocks);
    else
        clear_kernel<3><<<(unsigned)ctas, threads, 0, c.stream>>>(c.grid[buf], c.touched[buf], c.n_blocks);
    return cudaGetLastError();
}

cudaError_t launch_encode_init(Ctx &c, const double *d_state)
{
    StepParams p;
    fill_params(c, p);
    const int threads = 128;
    const unsigned blocks = (unsigned)((c.N + threads - 1) / threads);
    const size_t smem = (size_t)c.W * threads * sizeof(uint32_t);
    if (c.quant)
        encode_init_kernel<true><<<blocks, threads, smem, c.stream>>>(p, d_state, c.N);
    else
        encode_init_kernel<false><<<blocks, threads, 0, c.stream>>>(p, d_state, c.N);
    return cudaGetLastError();
}

cudaError_t launch_decode_f64(Ctx &c, double *d_state)
{
    StepParams p;
    fill_params(c, p);
    const int threads = 256;
    const unsigned blocks = (unsigned)((c.N + threads - 1) / threads);
    if (c.quant)
        decode_f64_kernel<true><<<blocks, threads, 0, c.stream>>>(p, d_state, c.N);
    else
        decode_f64_kernel<false><<<blocks, threads, 0, c.stream>>>(p, d_state, c.N);
    return cudaGetLastError();
}

cudaError_t launch_measure(Ctx &c)
{
    StepParams p;
    fill_params(c, p);
    cudaError_t e = cudaMemsetAsync(c.d_z, 0, sizeof(double), c.stream);
    if (e != cudaSuccess) return e;
    int64_t blocks = (c.N + kThreads - 1) / kThreads;
    if (blocks > (int64_t)c.n_sms * 8) blocks = (int64_t)c.n_sms * 8;
    if (blocks < 1) blocks = 1;
    const unsigned b = (unsigned)blocks;
    if (c.scene.dim == 2) {
        if (c.quant) measure_kernel<2, true><<<b, kThreads, 0, c.stream>>>(p, c.N, c.d_z);
        else measure_kernel<2, false><<<b, kThreads, 0, c.stream>>>(p, c.N, c.d_z);
    } else {
        if (c.quant) measure_kernel<3, true><<<b, kThreads, 0, c.stream>>>(p, c.N, c.d_z);
        else measure_kernel<3, false><<<b, kThreads, 0, c.stream>>>(p, c.N, c.d_z);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_f32(int dim, int material, const CompCodec *cc, int nc, int W, uint64_t seed, int dither,
                            uint32_t step, const float *d_vals, int64_t N, uint32_t *d_words, int64_t ld,
                            unsigned long long *d_stats, cudaStream_t s)
{
    (void)dim;
    (void)material;
    StepParams p;
    memset(&p, 0, sizeof(p));
    p.n_comp = nc;
    p.n_words = W;
    p.dither = dither;
    p.seed_lo = (uint32_t)seed;
    p.seed_hi = (uint32_t)(seed >> 32);
    p.step = step;
    for (int q = 0; q < nc; ++q) p.comp[q] = cc[q];
    p.words = d_words;
    p.ld = ld;
    p.stats = d_stats;
    const int threads = 128;
    const unsigned blocks = (unsigned)((N + threads - 1) / threads);
    if (N > 0) pack_f32_kernel<<<blocks, threads, (size_t)W * threads * sizeof(uint32_t), s>>>(p, d_vals, N);
    return cudaGetLastError();
}

cudaError_t launch_unpack_f32(int dim, int material, const CompCodec *cc, int nc, const uint32_t *d_words,
                              int64_t N, int64_t ld, float *d_vals, cudaStream_t s)
{
    (void)dim;
    (void)material;
    StepParams p;
    memset(&p, 0, sizeof(p));
    p.n_comp = nc;
    for (int q = 0; q < nc; ++q) p.comp[q] = cc[q];
    p.words = const_cast<uint32_t *>(d_words);
    p.ld = ld;
    const int threads = 256;
    const unsigned blocks = (unsigned)((N + threads - 1) / threads);
    if (N > 0) unpack_f32_kernel<<<blocks, threads, 0, s>>>(p, d_vals, N);
    return cudaGetLastError();
}

}  // namespace qmpm
