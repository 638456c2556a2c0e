// sort.cu -- particle ordering of libqmpm.
//
// The dither counter of a store is the particle's slot (its position in the array), so
// the device and the CPU oracle must agree on the order: particles are kept sorted,
// stably, by the key of the 2^d-block tile that holds their stencil.  A re-sort:
//   1. key of every slot from its decoded position (integer tile coordinates),
//   2. stable LSD radix sort of (key, slot) with 8-bit digits: per-tile digit counts,
//      one exclusive scan over (digit, tile), a scatter that ranks equal digits in
//      input order with warp match masks,
//   3. gather of the packed records (all word planes) and ids into the other buffer,
//   4. segment bounds per key and the chunk list (runs of <= chunk particles that share
//      a tile) consumed by the step kernels.
#include "device_common.cuh"

namespace qmpm {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per tile

int64_t sort_scratch_tiles(int64_t N) { return (N + kSortTile - 1) / kSortTile; }

// ------------------------------------------------------------------------------ scan
__global__ void scan_reduce_kernel(const uint32_t *data, int64_t n, uint32_t *partials)
{
    __shared__ uint32_t red[kSortThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    uint32_t acc = 0;
    for (int i = 0; i < kSortItems; ++i) {
        const int64_t idx = base + (int64_t)i * kSortThreads + threadIdx.x;
        if (idx < n) acc += data[idx];
    }
    acc = __reduce_add_sync(0xFFFFFFFFu, acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kSortThreads / 32; ++w) t += red[w];
        partials[blockIdx.x] = t;
    }
}

// exclusive scan of n partials in place by one CTA of 1024 threads
__global__ void scan_partials_kernel(uint32_t *partials, int64_t n)
{
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < n; b0 += blockDim.x) {
        const int64_t idx = b0 + threadIdx.x;
        const uint32_t v = idx < n ? partials[idx] : 0u;
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t ws = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, ws, o);
                if (lane >= o) ws += t;
            }
            warp_sums[lane] = ws;  // inclusive over warps
        }
        __syncthreads();
        const uint32_t warp_excl = warp > 0 ? warp_sums[warp - 1] : 0u;
        const uint32_t total = warp_sums[(blockDim.x >> 5) - 1];
        if (idx < n) partials[idx] = carry + warp_excl + incl - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
}

__global__ void scan_down_kernel(uint32_t *data, int64_t n, const uint32_t *partials)
{
    __shared__ uint32_t warp_sums[kSortThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)threadIdx.x * kSortItems;
    uint32_t v[kSortItems];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        v[i] = (base + i < n) ? data[base + i] : 0u;
        sum += v[i];
    }
    uint32_t incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    uint32_t warp_excl = 0;
    for (int w = 0; w < warp; ++w) warp_excl += warp_sums[w];
    uint32_t run = partials[blockIdx.x] + warp_excl + incl - sum;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        if (base + i < n) data[base + i] = run;
        run += v[i];
    }
}

cudaError_t exclusive_scan_u32(uint32_t *data, int64_t n, uint32_t *partials, int64_t max_partials, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t nblk = (n + kSortTile - 1) / kSortTile;
    if (nblk > max_partials) return cudaErrorInvalidValue;
    scan_reduce_kernel<<<(unsigned)nblk, kSortThreads, 0, s>>>(data, n, partials);
    scan_partials_kernel<<<1, 1024, 0, s>>>(partials, nblk);
    scan_down_kernel<<<(unsigned)nblk, kSortThreads, 0, s>>>(data, n, partials);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ keys
template <int DIM, bool QUANT>
__global__ void tile_key_kernel(const __grid_constant__ StepParams P, int64_t N, uint32_t *keys, uint32_t *vals)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    uint32_t key = 0, cell = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const CompCodec &cc = P.comp[a];
        float x;
        if (QUANT) {
            uint32_t lo = P.words[cc.word * P.ld + p] >> cc.shift;
            if (cc.straddle) lo |= P.words[(cc.word + 1) * P.ld + p] << (32 - cc.shift);
            x = decode_u(lo & cc.mask, cc);
        } else {
            x = __uint_as_float(P.words[a * P.ld + p]);
        }
        int b = __float2int_rd(x * P.inv_dx - 0.5f);
        b = b < 0 ? 0 : (b > P.n - 3 ? P.n - 3 : b);
        const int T = (b + 3) >> 2;
        key = key * (uint32_t)P.nb + (uint32_t)T;
        cell = cell * 4u + (uint32_t)(b - 4 * (T - 1) - 1);
    }
    keys[p] = key * (DIM == 2 ? 16u : 64u) + cell;  // tile, then cell inside the tile
    vals[p] = (uint32_t)p;
}

// ------------------------------------------------------------------------------ radix sort
__global__ void radix_hist_kernel(const uint32_t *keys, int64_t N, int shift, uint32_t *counts, int64_t n_tiles)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = 0; i < kSortItems; ++i) {
        const int64_t idx = base + (int64_t)i * kSortThreads + threadIdx.x;
        if (idx < N) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Scatter of one pass.  A CTA ranks its 4096 keys stably by digit (warp match masks, then
// a prefix over warps), places them in shared memory in digit order, and writes each
// digit's run out with consecutive threads on consecutive addresses: the destinations are
// those of a direct scatter, but the stores coalesce instead of landing one 4-byte word
// per digit run and warp.
__global__ void radix_scatter_kernel(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *keys_out,
                                     uint32_t *vals_out, int64_t N, int shift, const uint32_t *offsets,
                                     int64_t n_tiles)
{
    constexpr int kWarps = kSortThreads / 32;
    static_assert(kSortThreads == 256, "one thread per digit in the digit prefix");
    __shared__ uint32_t wcount[kWarps][257];
    __shared__ uint32_t dstart[256];       // first local position of each digit
    __shared__ uint32_t dglobal[256];      // its global destination minus dstart
    __shared__ uint32_t wsum[kWarps];
    __shared__ uint32_t skey[kSortTile], sval[kSortTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * 257; i += kSortThreads) (&wcount[0][0])[i] = 0;
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t base = tile0 + (int64_t)warp * (kSortItems * 32);
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t k[kSortItems], v[kSortItems], rank[kSortItems];
    int dg[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t idx = base + r * 32 + lane;
        const bool valid = idx < N;
        k[r] = valid ? keys_in[idx] : 0u;
        v[r] = valid ? vals_in[idx] : 0u;
        const int d = valid ? (int)((k[r] >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const int before = __popc(peers & lt_mask);
        rank[r] = wcount[warp][d] + before;
        __syncwarp();
        if (before == 0) wcount[warp][d] += __popc(peers);
        __syncwarp();
        dg[r] = d;
    }
    __syncthreads();
    // digit d = threadIdx.x: prefix over warps, then the exclusive prefix over digits
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t t = wcount[w][d];
            wcount[w][d] = run;
            run += t;
        }
        uint32_t incl = run;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t before_warp = 0;
        for (int w = 0; w < warp; ++w) before_warp += wsum[w];
        const uint32_t start = before_warp + incl - run;
        dstart[d] = start;
        dglobal[d] = offsets[(int64_t)d * n_tiles + blockIdx.x] - start;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (dg[r] < 256) {
            const uint32_t lp = dstart[dg[r]] + wcount[warp][dg[r]] + rank[r];
            skey[lp] = k[r];
            sval[lp] = v[r];
        }
    }
    __syncthreads();
    const int n_here = (int)min((int64_t)kSortTile, N - tile0);
    for (int i = threadIdx.x; i < n_here; i += kSortThreads) {
        const uint32_t key = skey[i];
        const uint32_t dst = dglobal[(key >> shift) & 255u] + (uint32_t)i;
        keys_out[dst] = key;
        vals_out[dst] = sval[i];
    }
}

// ------------------------------------------------------------------------------ gather + chunks
__global__ void gather_kernel(const uint32_t *words_in, uint32_t *words_out, const int64_t *ids_in, int64_t *ids_out,
                              const uint32_t *perm, int64_t N, int64_t ld, int W)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t src = perm[i];
    for (int j = 0; j < W; ++j) words_out[j * ld + i] = words_in[j * ld + src];
    ids_out[i] = ids_in[src];
}

// segment bounds per tile (the key without its cell bits)
__global__ void segment_kernel(const uint32_t *sorted_keys, int64_t N, int cell_bits, uint32_t *seg_begin,
                               uint32_t *seg_end)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t k = sorted_keys[i] >> cell_bits;
    if (i == 0 || (sorted_keys[i - 1] >> cell_bits) != k) seg_begin[k] = (uint32_t)i;
    if (i == N - 1 || (sorted_keys[i + 1] >> cell_bits) != k) seg_end[k] = (uint32_t)(i + 1);
}

__global__ void chunk_count_kernel(const uint32_t *seg_begin, const uint32_t *seg_end, uint32_t *key_chunks,
                                   int64_t n_keys, int chunk)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n_keys) return;
    if (k == n_keys) {
        key_chunks[k] = 0;
        return;
    }
    const uint32_t cnt = seg_end[k] - seg_begin[k];
    key_chunks[k] = (cnt + chunk - 1) / chunk;
}

__global__ void chunk_emit_kernel(const uint32_t *seg_begin, const uint32_t *seg_end, const uint32_t *chunk_base,
                                  Chunk *chunks, int64_t n_keys, int chunk)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_keys) return;
    const uint32_t b = seg_begin[k], cnt = seg_end[k] - b;
    uint32_t out = chunk_base[k];
    const uint32_t n = (cnt + chunk - 1) / chunk;
    for (uint32_t s = 0; s < cnt; s += chunk, ++out) {
        Chunk c;
        c.start = b + s;
        c.count = (cnt - s) < (uint32_t)chunk ? (cnt - s) : (uint32_t)chunk;
        c.key = (uint32_t)k;
        c.tile_chunks = s == 0 ? n : 0u;
        chunks[out] = c;
    }
}

// Non-empty tiles: flag per key (1 if the key has particles; entry n_keys is 0), scanned
// into tile_idx, then each non-empty key writes the index of its first chunk at its rank.
__global__ void tile_flag_kernel(const uint32_t *seg_begin, const uint32_t *seg_end, uint32_t *tile_idx,
                                 int64_t n_keys)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n_keys) return;
    tile_idx[k] = (k < n_keys && seg_end[k] > seg_begin[k]) ? 1u : 0u;
}

__global__ void tile_emit_kernel(const uint32_t *seg_begin, const uint32_t *seg_end, const uint32_t *tile_idx,
                                 const uint32_t *chunk_base, uint32_t *tile_first, int64_t n_keys)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_keys || seg_end[k] <= seg_begin[k]) return;
    tile_first[tile_idx[k]] = chunk_base[k];
}

static unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

cudaError_t sort_tile_order(const StepParams &p, int dim, bool quant, int64_t N, int key_bits, uint32_t *keys[2],
                            uint32_t *vals[2], uint32_t *counts, uint32_t *partials, int64_t max_partials,
                            cudaStream_t s, int *result)
{
    *result = 0;
    if (N <= 0) return cudaSuccess;
    if (dim == 2)
        quant ? tile_key_kernel<2, true><<<blocks_for(N, 256), 256, 0, s>>>(p, N, keys[0], vals[0])
              : tile_key_kernel<2, false><<<blocks_for(N, 256), 256, 0, s>>>(p, N, keys[0], vals[0]);
    else
        quant ? tile_key_kernel<3, true><<<blocks_for(N, 256), 256, 0, s>>>(p, N, keys[0], vals[0])
              : tile_key_kernel<3, false><<<blocks_for(N, 256), 256, 0, s>>>(p, N, keys[0], vals[0]);
    const int64_t n_tiles = sort_scratch_tiles(N);
    int src = 0;
    for (int shift = 0; shift < key_bits; shift += 8) {
        radix_hist_kernel<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(keys[src], N, shift, counts, n_tiles);
        const cudaError_t e = exclusive_scan_u32(counts, 256 * n_tiles, partials, max_partials, s);
        if (e != cudaSuccess) return e;
        radix_scatter_kernel<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(keys[src], vals[src], keys[1 - src],
                                                                       vals[1 - src], N, shift, counts, n_tiles);
        src = 1 - src;
    }
    *result = src;
    return cudaGetLastError();
}

int resort(Ctx &c, std::string &err)
{
    cudaStream_t s = c.stream;
    const int64_t N = c.N;
    StepParams p;
    fill_params(c, p);
    cudaError_t e = cudaSuccess;
    if (N > 0) {
        if (c.scene.dim == 2)
            c.quant ? tile_key_kernel<2, true><<<blocks_for(N, 256), 256, 0, s>>>(p, N, c.keys[0], c.vals[0])
                    : tile_key_kernel<2, false><<<blocks_for(N, 256), 256, 0, s>>>(p, N, c.keys[0], c.vals[0]);
        else
            c.quant ? tile_key_kernel<3, true><<<blocks_for(N, 256), 256, 0, s>>>(p, N, c.keys[0], c.vals[0])
                    : tile_key_kernel<3, false><<<blocks_for(N, 256), 256, 0, s>>>(p, N, c.keys[0], c.vals[0]);
        const int64_t n_tiles = sort_scratch_tiles(N);
        int src = 0;
        for (int shift = 0; shift < c.key_bits; shift += 8) {
            radix_hist_kernel<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(c.keys[src], N, shift, c.digit_counts, n_tiles);
            e = exclusive_scan_u32(c.digit_counts, 256 * n_tiles, c.scan_partials, c.max_scan_partials, s);
            if (e != cudaSuccess) break;
            radix_scatter_kernel<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(c.keys[src], c.vals[src], c.keys[1 - src],
                                                                           c.vals[1 - src], N, shift, c.digit_counts,
                                                                           n_tiles);
            src = 1 - src;
        }
        if (e == cudaSuccess) {
            gather_kernel<<<blocks_for(N, 256), 256, 0, s>>>(c.words[c.cur], c.words[1 - c.cur], c.ids[c.cur],
                                                             c.ids[1 - c.cur], c.vals[src], N, c.ld, c.W);
            c.cur = 1 - c.cur;
            e = cudaMemsetAsync(c.seg_begin, 0, sizeof(uint32_t) * c.n_blocks, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(c.seg_end, 0, sizeof(uint32_t) * c.n_blocks, s);
            if (e == cudaSuccess) {
                segment_kernel<<<blocks_for(N, 256), 256, 0, s>>>(c.keys[src], N, c.scene.dim == 2 ? 4 : 6,
                                                                  c.seg_begin, c.seg_end);
                chunk_count_kernel<<<blocks_for(c.n_blocks + 1, 256), 256, 0, s>>>(c.seg_begin, c.seg_end,
                                                                                   c.key_chunks, c.n_blocks, c.chunk);
                e = exclusive_scan_u32(c.key_chunks, c.n_blocks + 1, c.scan_partials, c.max_scan_partials, s);
            }
            if (e == cudaSuccess) {
                chunk_emit_kernel<<<blocks_for(c.n_blocks, 256), 256, 0, s>>>(c.seg_begin, c.seg_end, c.key_chunks,
                                                                              c.chunks, c.n_blocks, c.chunk);
                tile_flag_kernel<<<blocks_for(c.n_blocks + 1, 256), 256, 0, s>>>(c.seg_begin, c.seg_end, c.tile_idx,
                                                                                 c.n_blocks);
                e = exclusive_scan_u32(c.tile_idx, c.n_blocks + 1, c.scan_partials, c.max_scan_partials, s);
            }
            if (e == cudaSuccess)
                tile_emit_kernel<<<blocks_for(c.n_blocks, 256), 256, 0, s>>>(c.seg_begin, c.seg_end, c.tile_idx,
                                                                             c.key_chunks, c.tile_first, c.n_blocks);
        }
    } else {
        e = cudaMemsetAsync(c.key_chunks + c.n_blocks, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(c.tile_idx + c.n_blocks, 0, sizeof(uint32_t), s);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("re-sort: ") + cudaGetErrorString(e);
        return QMPM_ERR_CUDA;
    }
    return QMPM_OK;
}

}  // namespace qmpm
