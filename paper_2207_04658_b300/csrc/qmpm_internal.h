// qmpm_internal.h -- internal types of libqmpm shared by its translation units.
#pragma once

#ifndef __CUDACC_RTC__
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#endif

#include "../../include/qmpm.h"

struct qmpm_batch;

namespace qmpm {

constexpr int kMaxComp = QMPM_MAX_COMP;
constexpr int kThreads = 256;       // threads per CTA of the step kernels
constexpr int kMaxChunk = 256;      // particles per work item (one per thread)

// Per-component codec constants, precomputed on the host from the scheme.
struct CompCodec {
    int32_t word;       // word holding the component's first bit
    int32_t shift;      // bit offset inside that word
    int32_t straddle;   // 1 if the component continues in word + 1
    uint32_t mask;      // (1 << bits) - 1
    int32_t offset;     // L: value = (u + L) * 2^-frac
    uint32_t umax;      // 2^bits - 1
    float enc_scale;    // 2^frac
    float dec_scale;    // 2^-frac
    float dec_bias;     // L * 2^-frac
    int32_t field;      // 0..3
};

// A run of sorted particles that share one tile.  The step kernels take a tile's chunks
// together (one grid staging and one flush per tile): the first chunk of a tile carries
// the tile's chunk count, the others 0.
struct Chunk {
    uint32_t start;        // first slot
    uint32_t count;        // <= chunk size
    uint32_t key;          // tile key: linear index of the tile's origin block
    uint32_t tile_chunks;  // chunks of the tile if this is its first, else 0
};

struct StepParams {
    // physics
    int32_t n, nb, bound, n_comp;
    float dt, inv_dx, dx, Dinv;
    float p_mass, inv_p_mass, stress_coef;  // stress_coef = -dt * p_vol * Dinv
    float mu, lambda, bulk;
    float gravity[3];
    // codec
    int32_t n_words;
    int32_t dither;
    uint32_t seed_lo, seed_hi;
    uint32_t round_key[2][10];  // Philox round keys: seed + r x Weyl constant (host-filled)
    uint32_t step;              // dither step index of this step's store
    CompCodec comp[kMaxComp];
    // data
    uint32_t *words;            // word planes
    int64_t ld;                 // plane stride
    const Chunk *chunks;
    const uint32_t *n_chunks;   // device scalar
    const uint32_t *tile_first; // index of each non-empty tile's first chunk
    const uint32_t *n_tiles;    // device scalar
    const float4 *grid_in;      // P2G result of the current state (G2P source)
    float4 *grid_out;           // zeroed target of the next P2G
    uint8_t *touched_out;       // blocks of grid_out that received mass
    unsigned long long *stats;  // QMPM_FLAG_STATS counters (13) or null
    const uint32_t *step_ctr;   // multi-scene launches: steps done so far (the store uses + 1)
    uint32_t *work;             // [0] next tile to take, [1] CTAs finished; both 0 between launches
};

}  // namespace qmpm

// Everything below is host-side (or host-visible) only; a step kernel compiled at run time
// for one scheme sees the types above.
#ifndef __CUDACC_RTC__
namespace qmpm {

// Grid buffer of one member of a multi-scene clear.
struct ClearItem {
    float4 *grid;
    uint8_t *touched;
    int64_t n_blocks;
    int64_t first;              // first virtual block: sum of the previous members' counts,
                                // each rounded up to a multiple of 32
    int32_t block_nodes;
    int32_t pad;
};

constexpr int kMaxMembers = 256;   // scenes of one multi-scene launch

// Event records of QMPM_FLAG_PROFILE: (start, end, kind) per launch group.
struct Profile {
    struct Rec {
        cudaEvent_t a, b;
        int kind;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    double ms[4] = {0.0, 0.0, 0.0, 0.0};
    int64_t n[4] = {0, 0, 0, 0};
};

// particle ranges of qmpm_step_host_stream's pipelined copies
constexpr int kMaxCopyChunks = 64;

struct Ctx {
    qmpm_scene_t scene;
    qmpm_scheme_t scheme;
    bool quant;
    int n_comp;
    int W;                      // words per particle
    int64_t N, ld;
    int n, nb;
    int64_t n_blocks;           // nb^d
    int64_t block_nodes;        // 4^d
    int chunk;
    cudaStream_t stream;
    bool own_stream;
    int n_sms;

    uint32_t *words[2];         // word planes (ping-pong for the re-sort gather)
    int64_t *ids[2];
    int cur;                    // which words/ids buffer is live
    float4 *grid[2];            // the two grid buffers
    uint8_t *touched[2];
    int gcur;                   // grid buffer holding the P2G of the live state
    bool primed;                // grid[gcur] holds the P2G of the live state

    // sort and chunk scratch
    uint32_t *keys[2], *vals[2];
    uint32_t *digit_counts;     // 256 * n_tiles
    uint32_t *scan_partials;
    int64_t max_scan_partials;
    uint32_t *seg_begin, *seg_end, *key_chunks; // per key
    Chunk *chunks;
    uint32_t *n_chunks;
    uint32_t *tile_idx;         // per key: non-empty keys before it (exclusive scan); [n_blocks] = count
    uint32_t *tile_first;       // per non-empty tile: its first chunk
    uint32_t *n_tiles;          // = tile_idx + n_blocks
    int64_t max_chunks;
    int key_bits;

    struct Profile *prof;       // event records (QMPM_FLAG_PROFILE), owned
    int64_t launches;           // kernel launches since the last profile reset

    qmpm_batch *batch;          // the batch the scene steps in, or null

    // QMPM_FLAG_SPECIALIZE: the step kernel compiled for this scheme (a cudaKernel_t), its
    // NVRTC compile time, and the launch shape cached for its shared-memory size
    void *spec_kernel;
    double spec_seconds;
    size_t spec_smem;
    int spec_per_sm;

    // qmpm_step_host_stream: the download stream and its events, created on first use
    cudaStream_t copy_stream;
    cudaEvent_t copy_ev[kMaxCopyChunks];
    cudaEvent_t step_ev;

    unsigned long long *d_stats; // 16 counters, then the step kernels' tile queue (2 x u32)
    double *d_z;
    int64_t steps;
    CompCodec cc[kMaxComp];
};

// kernels launched by one re-sort: keys, radix passes (hist, 3 scan, scatter), gather,
// segments, chunk counts, 3 scan, chunk emit, tile flags, 3 scan, tile emit
inline int64_t resort_launches(int key_bits) { return 14 + 5 * (int64_t)(key_bits / 8); }

// api.cu: message returned by qmpm_last_error() on this thread
void set_last_error(const std::string &msg);
// True if an armed fault of this kind (QMPM_FAULT_*) fires now (qmpm_fault_inject).
bool fault_hit(int kind);
// The scene checks of qmpm_init (sets the last error on failure).
int validate_scene(const qmpm_scene_t *s);

// scheme.cpp
int layout(int dim, int material, qmpm_scheme_t *scheme, std::string &err);
int n_comp(int dim, int material);
int comp_field(int dim, int comp);
void build_codec(const qmpm_scheme_t &s, int dim, int material, CompCodec *cc);

// sort.cu
int resort(Ctx &c, std::string &err);
// keys of N packed records (codec and grid in p) and a stable radix sort of (key, slot)
// in the given buffers; on return vals[*result] holds the sorted slots
cudaError_t sort_tile_order(const StepParams &p, int dim, bool quant, int64_t N, int key_bits, uint32_t *keys[2],
                            uint32_t *vals[2], uint32_t *counts, uint32_t *partials, int64_t max_partials,
                            cudaStream_t s, int *result);
int64_t sort_scratch_tiles(int64_t N);
cudaError_t exclusive_scan_u32(uint32_t *data, int64_t n, uint32_t *partials, int64_t max_partials,
                               cudaStream_t s);

// step.cu
cudaError_t launch_encode_init(Ctx &c, const double *d_state);
cudaError_t launch_p2g(Ctx &c);
cudaError_t launch_g2p2g(Ctx &c, uint32_t step);
cudaError_t launch_clear(Ctx &c, int buf);
cudaError_t launch_decode_f64(Ctx &c, double *d_state);
cudaError_t launch_measure(Ctx &c);
cudaError_t launch_count_flags(Ctx &c, const uint8_t *flags, int64_t n, unsigned long long *d_out);
cudaError_t launch_pack_f32(int dim, int material, const CompCodec *cc, int n_comp, int W, uint64_t seed,
                            int dither, uint32_t step, const float *d_vals, int64_t N, uint32_t *d_words,
                            int64_t ld, unsigned long long *d_stats, cudaStream_t s);
cudaError_t launch_unpack_f32(int dim, int material, const CompCodec *cc, int n_comp,
                              const uint32_t *d_words, int64_t N, int64_t ld, float *d_vals,
                              cudaStream_t s);
void fill_params(const Ctx &c, StepParams &p);
// parameters of the G2P -> store -> P2G launch of the live state (grid buffers by gcur)
void step_params(const Ctx &c, StepParams &p, uint32_t step);
size_t step_smem_bytes(int dim, int W);

// multi-scene launches (batch.cu drives them): one persistent step kernel over the chunks
// of n members of one (dim, material, quantized, stats) class; one clear over n grids;
// the members' step counters advanced by one
cudaError_t launch_step_multi(int dim, int material, bool quant, bool stats, const StepParams *d_tab, int n,
                              size_t smem, int n_sms, cudaStream_t s);
cudaError_t launch_clear_multi(const ClearItem *d_items, int n, int64_t virtual_blocks, int n_sms, cudaStream_t s);
// one batch member in a launch of its own (p NULL: set the kernel's attributes only)
cudaError_t launch_step_ctr(int dim, int material, bool quant, bool stats, const StepParams *p, size_t smem,
                            int n_sms, cudaStream_t s);
cudaError_t launch_advance(uint32_t *d_ctr, int n, cudaStream_t s);

// jit.cpp: the step kernel specialised to the handle's scheme (sets spec_kernel; compiled on
// first use and kept for the process), the compile alone (no device), and its launch
int specialize_step_kernel(Ctx &c, std::string &err);
int specialize_compile_only(int dim, int material, bool stats, bool dither, int W, const CompCodec *cc, int nc,
                            double *seconds, int64_t *cubin_bytes, std::string &err);
cudaError_t launch_specialized(Ctx &c, const StepParams &p);

// batch.cu: a member's host-side state changed outside the batch (its tables are stale)
void batch_invalidate(qmpm_batch *b);

}  // namespace qmpm
struct qmpm_ctx;
namespace qmpm {
// api.cu: free a handle with stream-ordered frees on its stream, without synchronising
void destroy_nosync(qmpm_ctx *c);

}  // namespace qmpm

// The opaque handle type of the C ABI is the context itself.
struct qmpm_ctx : public qmpm::Ctx {
};

#endif  // __CUDACC_RTC__
