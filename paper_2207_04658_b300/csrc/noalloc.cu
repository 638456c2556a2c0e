// noalloc.cu -- qmpm_tile_order_static: the particle ordering of qmpm_init computed without
// any device allocation, for callers that cannot call cudaMalloc (for example code running
// inside another runtime's memory pool, or a host thread that must not synchronise the
// device the way an allocation can).  Its scratch lives in one file-scope device array.
#include <cstring>
#include <mutex>
#include <string>

#include "qmpm_internal.h"

namespace {

// Scratch of the sort: two key and two value buffers of QMPM_STATIC_SORT_MAX entries, the
// per-tile digit counts (256 per 4096 keys) and the scan partials.
constexpr int64_t kMaxN = QMPM_STATIC_SORT_MAX;
constexpr int64_t kTiles = (kMaxN + 4095) / 4096;
constexpr int64_t kCounts = 256 * kTiles;
constexpr int64_t kPartials = (kCounts + 4095) / 4096 + 1;
constexpr int64_t kScratchWords = 4 * kMaxN + kCounts + kPartials;

__device__ __align__(256) uint32_t g_static_sort_scratch[kScratchWords];

// The host-side name of the array is not a device address; each device's address comes
// from cudaGetSymbolAddress, looked up once per device with that device current and kept
// for the life of the process (a cudaDeviceReset, after which the module may be reloaded
// elsewhere, is not supported).
std::mutex g_mutex;
uint32_t *g_scratch_addr[256] = {nullptr};

int fail(int code, const std::string &msg)
{
    qmpm::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int qmpm_tile_order_static(int32_t dim, int32_t material, int32_t grid_log2, const qmpm_scheme_t *scheme,
                                      const uint32_t *d_words, int64_t N, int64_t ld, uint32_t *d_order,
                                      void *stream)
{
    if (dim != 2 && dim != 3) return fail(QMPM_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (material < 0 || material > 2) return fail(QMPM_ERR_INVALID_ARG, "unknown material");
    if (grid_log2 < 4 || grid_log2 > (dim == 2 ? 11 : 10))
        return fail(QMPM_ERR_INVALID_ARG, "grid_log2 must be in 4..11 (2D) or 4..10 (3D)");
    if (N < 0 || N > kMaxN)
        return fail(QMPM_ERR_INVALID_ARG, "N = " + std::to_string(N) + " exceeds the static scratch limit of " +
                                              std::to_string(kMaxN) + " particles (QMPM_STATIC_SORT_MAX)");
    if (ld < N || (N > 0 && (!d_words || !d_order))) return fail(QMPM_ERR_INVALID_ARG, "bad buffers or ld");
    qmpm_scheme_t s;
    if (scheme && scheme->quantized)
        s = *scheme;
    else
        std::memset(&s, 0, sizeof(s));
    std::string err;
    int rc = qmpm::layout(dim, material, &s, err);
    if (rc != QMPM_OK) return fail(rc, err);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(QMPM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return fail(QMPM_ERR_INVALID_ARG, "device ordinal out of range");
    uint32_t *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_sort_scratch);
            if (e != cudaSuccess || !p)
                return fail(QMPM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_addr[dev] = static_cast<uint32_t *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    if (N == 0) return QMPM_OK;

    qmpm::StepParams p;
    std::memset(&p, 0, sizeof(p));
    const int n = 1 << grid_log2;
    p.n = n;
    p.nb = n / 4 + 2;
    p.inv_dx = (float)n;
    p.n_comp = qmpm::n_comp(dim, material);
    p.n_words = s.n_words;
    qmpm::build_codec(s, dim, material, p.comp);
    p.words = const_cast<uint32_t *>(d_words);
    p.ld = ld;
    const int64_t n_blocks = dim == 2 ? (int64_t)p.nb * p.nb : (int64_t)p.nb * p.nb * p.nb;
    int key_bits = 1;
    while ((int64_t(1) << key_bits) < n_blocks) ++key_bits;
    key_bits += dim == 2 ? 4 : 6;
    key_bits = (key_bits + 7) / 8 * 8;

    uint32_t *keys[2] = {scratch, scratch + kMaxN};
    uint32_t *vals[2] = {scratch + 2 * kMaxN, scratch + 3 * kMaxN};
    uint32_t *counts = scratch + 4 * kMaxN;
    uint32_t *partials = counts + kCounts;
    // every scratch word the sort reads is written earlier in the same call, so nothing
    // needs clearing between calls
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int result = 0;
    e = qmpm::sort_tile_order(p, dim, s.quantized != 0, N, key_bits, keys, vals, counts, partials, kPartials, st,
                              &result);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_order, vals[result], sizeof(uint32_t) * (size_t)N, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(QMPM_ERR_CUDA, std::string("static sort: ") + cudaGetErrorString(e));
    return QMPM_OK;
}
