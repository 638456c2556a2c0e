// api.cu -- the C ABI of libqmpm (declared in include/qmpm.h): scene lifetime, stepping,
// readback, the measurement and the device codec entry points.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "qmpm_internal.h"

extern "C" int qmpm_scheme_solve_impl(const qmpm_solve_in_t *in, qmpm_solve_out_t *out, std::string &err);
extern "C" int qmpm_scheme_shift_impl(qmpm_scheme_t *s, int32_t h, int32_t k, std::string &err);
extern "C" int qmpm_scheme_widen_impl(qmpm_scheme_t *s, int32_t h, std::string &err);
extern "C" int qmpm_scheme_window_impl(qmpm_scheme_t *s, int32_t h, double lo, double hi, double kappa,
                                       int32_t src, double gain, int32_t grow, std::string &err);
extern "C" int qmpm_scheme_fill_words_impl(int32_t dim, int32_t material, qmpm_scheme_t *s, int32_t type_mask,
                                           int32_t *widened, std::string &err);

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(QMPM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Device buffers come from the stream-ordered pool on the handle's stream: neither the
// allocation nor the free synchronises the device, so scenes can come and go while other
// scenes' work is in flight.
template <class T>
cudaError_t dalloc(T **p, size_t count, cudaStream_t s)
{
    *p = nullptr;
    if (count == 0) count = 1;
    if (qmpm::fault_hit(QMPM_FAULT_DEVICE_ALLOC)) return cudaErrorMemoryAllocation;
    return cudaMallocAsync(reinterpret_cast<void **>(p), count * sizeof(T), s);
}

void release(qmpm_ctx *c)
{
    if (!c) return;
    const cudaStream_t s = c->stream;
    auto fr = [s](void *p) {
        if (p) cudaFreeAsync(p, s);
    };
    for (int i = 0; i < 2; ++i) {
        fr(c->words[i]);
        fr(c->ids[i]);
        fr(c->grid[i]);
        fr(c->touched[i]);
        fr(c->keys[i]);
        fr(c->vals[i]);
    }
    fr(c->digit_counts);
    fr(c->scan_partials);
    fr(c->seg_begin);
    fr(c->seg_end);
    fr(c->key_chunks);
    fr(c->tile_idx);
    fr(c->tile_first);
    fr(c->chunks);
    fr(c->d_stats);
    fr(c->d_z);
    if (c->prof) {
        for (auto &r : c->prof->recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : c->prof->pool) cudaEventDestroy(e);
        delete c->prof;
    }
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    for (int j = 0; j < qmpm::kMaxCopyChunks; ++j)
        if (c->copy_ev[j]) cudaEventDestroy(c->copy_ev[j]);
    if (c->step_ev) cudaEventDestroy(c->step_ev);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

enum { PROF_STEP = 0, PROF_CLEAR = 1, PROF_SORT = 2, PROF_P2G = 3 };

cudaEvent_t prof_event(qmpm::Profile *p)
{
    if (!p->pool.empty()) {
        cudaEvent_t e = p->pool.back();
        p->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

cudaEvent_t prof_begin(qmpm::Ctx &c)
{
    if (!(c.scene.flags & QMPM_FLAG_PROFILE) || !c.prof) return nullptr;
    cudaEvent_t a = prof_event(c.prof);
    if (a) cudaEventRecord(a, c.stream);
    return a;
}

void prof_end(qmpm::Ctx &c, cudaEvent_t a, int kind)
{
    if (!a) return;
    cudaEvent_t b = prof_event(c.prof);
    if (!b) return;
    cudaEventRecord(b, c.stream);
    c.prof->recs.push_back({a, b, kind});
}

__global__ void iota_kernel(int64_t *ids, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ids[i] = i;
}

int prime(qmpm::Ctx &c)
{
    cudaEvent_t ev = prof_begin(c);
    cudaError_t e = qmpm::launch_p2g(c);
    prof_end(c, ev, PROF_P2G);
    c.launches += 1;
    if (e != cudaSuccess) return cuda_fail(e, "P2G");
    c.primed = true;
    return QMPM_OK;
}

int do_resort(qmpm::Ctx &c)
{
    std::string err;
    cudaEvent_t ev = prof_begin(c);
    const int rc = qmpm::resort(c, err);
    prof_end(c, ev, PROF_SORT);
    c.launches += qmpm::resort_launches(c.key_bits);
    if (rc != QMPM_OK) return fail(rc, err);
    return QMPM_OK;
}

int do_clear(qmpm::Ctx &c, int buf)
{
    cudaEvent_t ev = prof_begin(c);
    cudaError_t e = qmpm::launch_clear(c, buf);
    prof_end(c, ev, PROF_CLEAR);
    c.launches += 1;
    if (e != cudaSuccess) return cuda_fail(e, "grid clear");
    return QMPM_OK;
}

int check_scene(const qmpm_scene_t *s)
{
    if (!s) return fail(QMPM_ERR_INVALID_ARG, "scene is NULL");
    if (s->dim != 2 && s->dim != 3) return fail(QMPM_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (s->material < 0 || s->material > 2) return fail(QMPM_ERR_INVALID_ARG, "unknown material");
    if (s->grid_log2 < 4 || s->grid_log2 > (s->dim == 2 ? 11 : 10))
        return fail(QMPM_ERR_INVALID_ARG, "grid_log2 must be in 4..11 (2D) or 4..10 (3D)");
    if (s->bound < 2) return fail(QMPM_ERR_INVALID_ARG, "bound must be >= 2 (stencils must stay inside)");
    if (s->n_particles < 0 || s->n_particles > 0x7FFFFFFFLL)
        return fail(QMPM_ERR_INVALID_ARG, "n_particles must be in [0, 2^31)");
    if (!(s->dt > 0.0) || !(s->p_vol > 0.0) || !(s->p_mass > 0.0))
        return fail(QMPM_ERR_INVALID_ARG, "dt, p_vol and p_mass must be positive");
    if (s->chunk < 0 || s->chunk > qmpm::kMaxChunk) return fail(QMPM_ERR_INVALID_ARG, "chunk must be in 0..256");
    if (s->resort_every < 0) return fail(QMPM_ERR_INVALID_ARG, "resort_every must be >= 0");
    return QMPM_OK;
}

}  // namespace

namespace qmpm {
void set_last_error(const std::string &msg) { g_err = msg; }
int validate_scene(const qmpm_scene_t *s) { return check_scene(s); }

// Free a handle's device memory in order on its stream, without waiting for the stream.
void destroy_nosync(qmpm_ctx *c)
{
    if (!c) return;
    if (c->batch) qmpm_batch_remove(c->batch, c);
    release(c);
}
}  // namespace qmpm

namespace {

// Scene, scheme and the derived sizes of a handle (no device work).
int setup(qmpm_ctx *c, const qmpm_scene_t *scene, const qmpm_scheme_t *scheme)
{
    c->scene = *scene;
    if (scheme && scheme->quantized) {
        c->scheme = *scheme;
    } else {
        std::memset(&c->scheme, 0, sizeof(c->scheme));
    }
    std::string err;
    const int rc = qmpm::layout(scene->dim, scene->material, &c->scheme, err);
    if (rc != QMPM_OK) return fail(rc, err);
    c->quant = c->scheme.quantized != 0;
    c->n_comp = qmpm::n_comp(scene->dim, scene->material);
    c->W = c->scheme.n_words;
    qmpm::build_codec(c->scheme, scene->dim, scene->material, c->cc);
    c->N = scene->n_particles;
    c->ld = std::max<int64_t>(32, (c->N + 31) / 32 * 32);
    c->n = 1 << scene->grid_log2;
    c->nb = c->n / 4 + 2;
    c->n_blocks = scene->dim == 2 ? (int64_t)c->nb * c->nb : (int64_t)c->nb * c->nb * c->nb;
    c->block_nodes = scene->dim == 2 ? 16 : 64;
    c->chunk = scene->chunk > 0 ? scene->chunk : qmpm::kMaxChunk;
    c->key_bits = 1;
    while ((int64_t(1) << c->key_bits) < c->n_blocks) ++c->key_bits;
    c->key_bits += scene->dim == 2 ? 4 : 6;  // cell inside the tile
    c->key_bits = (c->key_bits + 7) / 8 * 8;
    const int64_t N1 = std::max<int64_t>(c->N, 1);
    const int64_t n_tiles = qmpm::sort_scratch_tiles(N1);
    const int64_t scan_len = std::max<int64_t>(256 * n_tiles, c->n_blocks + 1);
    c->max_scan_partials = (scan_len + 4095) / 4096 + 1;
    c->max_chunks = (c->N + c->chunk - 1) / c->chunk + std::min<int64_t>(c->N, c->n_blocks) + 1;
    return QMPM_OK;
}

// Element counts of the handle's device buffers (qmpm_init allocates exactly these).
struct Sizes {
    size_t words, ids, grid, touched, keys, digit_counts, scan_partials, seg, key_chunks, chunks;
    size_t bytes() const
    {
        return 2 * (words * 4 + ids * 8 + grid * 16 + touched + keys * 4 * 2) + digit_counts * 4 +
               scan_partials * 4 + 3 * seg * 4 + 2 * key_chunks * 4 + chunks * sizeof(qmpm::Chunk) + 17 * 8 + 8;
    }
};

Sizes sizes_of(const qmpm::Ctx &c)
{
    const int64_t N1 = std::max<int64_t>(c.N, 1);
    Sizes z;
    z.words = (size_t)c.W * c.ld;
    z.ids = (size_t)c.ld;
    z.grid = (size_t)(c.n_blocks * c.block_nodes);
    z.touched = (size_t)c.n_blocks;
    z.keys = (size_t)N1;
    z.digit_counts = (size_t)(256 * qmpm::sort_scratch_tiles(N1));
    z.scan_partials = (size_t)c.max_scan_partials;
    z.seg = (size_t)c.n_blocks;
    z.key_chunks = (size_t)c.n_blocks + 1;
    z.chunks = (size_t)c.max_chunks;
    return z;
}

}  // namespace

using qmpm::Ctx;

extern "C" {

const char *qmpm_last_error(void) { return g_err.c_str(); }

int qmpm_scheme_layout(int32_t dim, int32_t material, qmpm_scheme_t *scheme)
{
    if (!scheme) return fail(QMPM_ERR_INVALID_ARG, "scheme is NULL");
    std::string err;
    const int rc = qmpm::layout(dim, material, scheme, err);
    if (rc != QMPM_OK) return fail(rc, err);
    return QMPM_OK;
}

int qmpm_scheme_solve(const qmpm_solve_in_t *in, qmpm_solve_out_t *out)
{
    std::string err;
    const int rc = qmpm_scheme_solve_impl(in, out, err);
    if (rc != QMPM_OK) return fail(rc, err);
    return QMPM_OK;
}

int qmpm_scheme_shift(qmpm_scheme_t *scheme, int32_t h, int32_t k)
{
    std::string err;
    const int rc = qmpm_scheme_shift_impl(scheme, h, k, err);
    return rc == QMPM_OK ? QMPM_OK : fail(rc, err);
}

int qmpm_scheme_widen(qmpm_scheme_t *scheme, int32_t h)
{
    std::string err;
    const int rc = qmpm_scheme_widen_impl(scheme, h, err);
    return rc == QMPM_OK ? QMPM_OK : fail(rc, err);
}

int qmpm_scheme_window(qmpm_scheme_t *scheme, int32_t h, double lo, double hi, double kappa, int32_t src,
                       double gain, int32_t grow)
{
    std::string err;
    const int rc = qmpm_scheme_window_impl(scheme, h, lo, hi, kappa, src, gain, grow, err);
    return rc == QMPM_OK ? QMPM_OK : fail(rc, err);
}

int qmpm_scheme_fill_words(int32_t dim, int32_t material, qmpm_scheme_t *scheme, int32_t type_mask,
                           int32_t *widened)
{
    std::string err;
    const int rc = qmpm_scheme_fill_words_impl(dim, material, scheme, type_mask, widened, err);
    return rc == QMPM_OK ? QMPM_OK : fail(rc, err);
}

int qmpm_init(const qmpm_scene_t *scene, const qmpm_scheme_t *scheme, const double *h_state, void *stream,
              qmpm_handle *out)
{
    if (!out) return fail(QMPM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_scene(scene);
    if (rc != QMPM_OK) return rc;
    if (scene->n_particles > 0 && !h_state) return fail(QMPM_ERR_INVALID_ARG, "h_state is NULL");
    qmpm_ctx *c = new (std::nothrow) qmpm_ctx();
    if (!c) return fail(QMPM_ERR_OOM, "host allocation failed");
    std::memset(static_cast<void *>(c), 0, sizeof(qmpm_ctx));
    c->stream = stream ? static_cast<cudaStream_t>(stream) : 0;
    rc = setup(c, scene, scheme);
    if (rc != QMPM_OK) {
        release(c);
        return rc;
    }
    cudaError_t e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, dev);
    if (c->n_sms <= 0) c->n_sms = 1;

    const Sizes z = sizes_of(*c);
    const cudaStream_t st = c->stream;
    bool ok = true;
    cudaError_t ae = cudaSuccess;  // the first failed allocation's error
    auto okd = [&ae](cudaError_t r) {
        if (r != cudaSuccess && ae == cudaSuccess) ae = r;
        return r == cudaSuccess;
    };
    for (int i = 0; i < 2 && ok; ++i) {
        ok = ok && okd(dalloc(&c->words[i], z.words, st));
        ok = ok && okd(dalloc(&c->ids[i], z.ids, st));
        ok = ok && okd(dalloc(&c->grid[i], z.grid, st));
        ok = ok && okd(dalloc(&c->touched[i], z.touched, st));
        ok = ok && okd(dalloc(&c->keys[i], z.keys, st));
        ok = ok && okd(dalloc(&c->vals[i], z.keys, st));
    }
    ok = ok && okd(dalloc(&c->digit_counts, z.digit_counts, st));
    ok = ok && okd(dalloc(&c->scan_partials, z.scan_partials, st));
    ok = ok && okd(dalloc(&c->seg_begin, z.seg, st));
    ok = ok && okd(dalloc(&c->seg_end, z.seg, st));
    ok = ok && okd(dalloc(&c->key_chunks, z.key_chunks, st));
    ok = ok && okd(dalloc(&c->chunks, z.chunks, st));
    ok = ok && okd(dalloc(&c->tile_idx, z.key_chunks, st));
    ok = ok && okd(dalloc(&c->tile_first, z.seg, st));
    ok = ok && okd(dalloc(&c->d_stats, 17, st));  // 16 statistics + the step kernels' tile queue
    ok = ok && okd(dalloc(&c->d_z, 1, st));
    if (!ok) {
        cudaGetLastError();
        release(c);
        if (ae == cudaErrorMemoryAllocation) return fail(QMPM_ERR_OOM, "device allocation failed");
        return cuda_fail(ae, "device allocation");
    }
    if (scene->flags & QMPM_FLAG_SPECIALIZE) {
        std::string err;
        rc = qmpm::specialize_step_kernel(*c, err);
        if (rc != QMPM_OK) {
            release(c);
            return fail(rc, err);
        }
    }
    c->n_chunks = c->key_chunks + c->n_blocks;
    c->n_tiles = c->tile_idx + c->n_blocks;
    c->prof = new (std::nothrow) qmpm::Profile();
    if (!c->prof) {
        release(c);
        return fail(QMPM_ERR_OOM, "host allocation failed");
    }
    for (int i = 0; i < 2; ++i) {
        e = cudaMemsetAsync(c->grid[i], 0, sizeof(float4) * (size_t)(c->n_blocks * c->block_nodes), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->touched[i], 0, (size_t)c->n_blocks, c->stream);
        if (e != cudaSuccess) {
            release(c);
            return cuda_fail(e, "grid clear");
        }
    }
    e = cudaMemsetAsync(c->d_stats, 0, 17 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) {
        release(c);
        return cuda_fail(e, "stats clear");
    }
    if (c->N > 0) {
        double *d_state = nullptr;
        e = cudaMallocAsync(reinterpret_cast<void **>(&d_state), sizeof(double) * (size_t)c->N * c->n_comp, c->stream);
        if (e != cudaSuccess) {
            release(c);
            return fail(QMPM_ERR_OOM, "device allocation of the initial state failed");
        }
        e = cudaMemcpyAsync(d_state, h_state, sizeof(double) * (size_t)c->N * c->n_comp, cudaMemcpyHostToDevice,
                            c->stream);
        if (e == cudaSuccess) e = qmpm::launch_encode_init(*c, d_state);
        if (e == cudaSuccess) {
            iota_kernel<<<(unsigned)((c->N + 255) / 256), 256, 0, c->stream>>>(c->ids[0], c->N);
            e = cudaGetLastError();
        }
        cudaFreeAsync(d_state, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            release(c);
            return cuda_fail(e, "initial encode");
        }
    }
    c->cur = 0;
    c->gcur = 0;
    rc = do_resort(*c);
    if (rc != QMPM_OK) {
        release(c);
        return rc;
    }
    rc = prime(*c);
    if (rc != QMPM_OK) {
        release(c);
        return rc;
    }
    *out = c;
    return QMPM_OK;
}

int qmpm_footprint(const qmpm_scene_t *scene, const qmpm_scheme_t *scheme, int64_t *resident_bytes,
                   int64_t *init_peak_bytes)
{
    int rc = check_scene(scene);
    if (rc != QMPM_OK) return rc;
    qmpm_ctx *c = new (std::nothrow) qmpm_ctx();
    if (!c) return fail(QMPM_ERR_OOM, "host allocation failed");
    std::memset(static_cast<void *>(c), 0, sizeof(qmpm_ctx));
    rc = setup(c, scene, scheme);
    if (rc == QMPM_OK) {
        const int64_t resident = (int64_t)sizes_of(*c).bytes();
        if (resident_bytes) *resident_bytes = resident;
        if (init_peak_bytes) *init_peak_bytes = resident + (int64_t)sizeof(double) * c->N * c->n_comp;
    }
    delete c;
    return rc;
}

int qmpm_step(qmpm_handle h, int32_t nsteps)
{
    if (!h || nsteps < 0) return fail(QMPM_ERR_INVALID_ARG, "bad handle or nsteps");
    Ctx &c = *h;
    std::string err;
    if (nsteps > 0) qmpm::batch_invalidate(c.batch);
    if (!c.primed) {
        const int rc = prime(c);
        if (rc != QMPM_OK) return rc;
    }
    for (int i = 0; i < nsteps; ++i) {
        const uint32_t t = (uint32_t)(c.steps + 1);
        cudaEvent_t ev = prof_begin(c);
        cudaError_t e = qmpm::launch_g2p2g(c, t);
        prof_end(c, ev, PROF_STEP);
        c.launches += 1;
        if (e != cudaSuccess) return cuda_fail(e, "G2P2G");
        int rc = do_clear(c, c.gcur);
        if (rc != QMPM_OK) return rc;
        c.gcur = 1 - c.gcur;
        c.steps += 1;
        if (c.scene.resort_every > 0 && c.steps % c.scene.resort_every == 0) {
            rc = do_resort(c);
            if (rc != QMPM_OK) return rc;
        }
    }
    return QMPM_OK;
}

int qmpm_readback(qmpm_handle h, double *h_state, uint32_t *h_words, int64_t *h_ids, qmpm_stats_t *stats)
{
    if (!h) return fail(QMPM_ERR_INVALID_ARG, "bad handle");
    Ctx &c = *h;
    cudaError_t e = cudaSuccess;
    if (h_state && c.N > 0) {
        double *d_state = nullptr;
        e = cudaMallocAsync(reinterpret_cast<void **>(&d_state), sizeof(double) * (size_t)c.N * c.n_comp, c.stream);
        if (e != cudaSuccess) return fail(QMPM_ERR_OOM, "device allocation for readback failed");
        e = qmpm::launch_decode_f64(c, d_state);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_state, d_state, sizeof(double) * (size_t)c.N * c.n_comp, cudaMemcpyDeviceToHost,
                                c.stream);
        cudaFreeAsync(d_state, c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        if (e != cudaSuccess) return cuda_fail(e, "readback");
    }
    if (h_words && c.N > 0) {
        e = cudaMemcpy2DAsync(h_words, sizeof(uint32_t) * (size_t)c.N, c.words[c.cur], sizeof(uint32_t) * (size_t)c.ld,
                              sizeof(uint32_t) * (size_t)c.N, (size_t)c.W, cudaMemcpyDeviceToHost, c.stream);
        if (e != cudaSuccess) return cuda_fail(e, "readback words");
    }
    if (h_ids && c.N > 0) {
        e = cudaMemcpyAsync(h_ids, c.ids[c.cur], sizeof(int64_t) * (size_t)c.N, cudaMemcpyDeviceToHost, c.stream);
        if (e != cudaSuccess) return cuda_fail(e, "readback ids");
    }
    unsigned long long st[16];
    e = cudaMemsetAsync(c.d_stats + 15, 0, sizeof(unsigned long long), c.stream);
    if (e == cudaSuccess) e = qmpm::launch_count_flags(c, c.touched[c.gcur], c.n_blocks, c.d_stats + 15);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st, c.d_stats, sizeof(st), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_fail(e, "readback stats");
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        for (int k = 0; k < 4; ++k) {
            stats->saturations[k] = (int64_t)st[k];
            stats->round_ups[k] = (int64_t)st[4 + k];
            stats->round_downs[k] = (int64_t)st[8 + k];
        }
        stats->out_of_grid = (int64_t)st[12];
        stats->out_of_tile = (int64_t)st[13];
        stats->error_word = (int32_t)st[14];
        stats->steps = c.steps;
        stats->active_blocks = (int64_t)st[15];
        stats->n_words = c.W;
    }
    if ((c.scene.flags & QMPM_FLAG_STRICT) && (st[0] + st[1] + st[2] + st[3]) > 0)
        return fail(QMPM_ERR_OVERFLOW, "a quantized store saturated (strict mode)");
    if (st[14] != 0) return fail((int)(int32_t)st[14], "device error word set");
    return QMPM_OK;
}

int qmpm_measure(qmpm_handle h, double *z)
{
    if (!h || !z) return fail(QMPM_ERR_INVALID_ARG, "bad handle or z");
    Ctx &c = *h;
    if (c.N == 0) {
        *z = 0.0;
        return QMPM_OK;
    }
    cudaError_t e = qmpm::launch_measure(c);
    if (e == cudaSuccess) e = cudaMemcpyAsync(z, c.d_z, sizeof(double), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_fail(e, "measure");
    return QMPM_OK;
}

int qmpm_step_host(qmpm_handle h, int32_t nsteps, const uint32_t *h_words_in, uint32_t *h_words_out)
{
    if (!h || nsteps < 0) return fail(QMPM_ERR_INVALID_ARG, "bad handle or nsteps");
    Ctx &c = *h;
    cudaError_t e;
    if (h_words_in && c.N > 0) {
        e = cudaMemcpy2DAsync(c.words[c.cur], sizeof(uint32_t) * (size_t)c.ld, h_words_in,
                              sizeof(uint32_t) * (size_t)c.N, sizeof(uint32_t) * (size_t)c.N, (size_t)c.W,
                              cudaMemcpyHostToDevice, c.stream);
        if (e != cudaSuccess) return cuda_fail(e, "upload words");
        // the grid of the previous state is stale: clear it and redo the P2G
        qmpm::batch_invalidate(c.batch);
        const int rc = do_clear(c, c.gcur);
        if (rc != QMPM_OK) return rc;
        c.primed = false;
    }
    int rc = qmpm_step(h, nsteps);
    if (rc != QMPM_OK) return rc;
    if (h_words_out && c.N > 0) {
        e = cudaMemcpy2DAsync(h_words_out, sizeof(uint32_t) * (size_t)c.N, c.words[c.cur],
                              sizeof(uint32_t) * (size_t)c.ld, sizeof(uint32_t) * (size_t)c.N, (size_t)c.W,
                              cudaMemcpyDeviceToHost, c.stream);
        if (e != cudaSuccess) return cuda_fail(e, "download words");
    }
    e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_fail(e, "step_host");
    return QMPM_OK;
}

int qmpm_step_host_stream(qmpm_handle h, int32_t nsteps, uint32_t *h_words, int32_t chunks)
{
    if (!h || nsteps < 0 || chunks < 0 || chunks > qmpm::kMaxCopyChunks)
        return fail(QMPM_ERR_INVALID_ARG, "qmpm_step_host_stream: bad handle, nsteps or chunks");
    Ctx &c = *h;
    if (c.N == 0 || nsteps == 0) return QMPM_OK;
    if (!h_words) return fail(QMPM_ERR_INVALID_ARG, "qmpm_step_host_stream: no host buffer");
    if (chunks == 0) {
        // ranges of at least 16 MiB (a small state goes in one copy each way), at most 8
        const int64_t bytes = (int64_t)sizeof(uint32_t) * c.N * c.W;
        chunks = (int)std::max<int64_t>(1, std::min<int64_t>(8, bytes >> 24));
    }
    cudaError_t e = cudaSuccess;
    if (!c.copy_stream) e = cudaStreamCreateWithFlags(&c.copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !c.step_ev) e = cudaEventCreateWithFlags(&c.step_ev, cudaEventDisableTiming);
    for (int j = 0; j < chunks && e == cudaSuccess; ++j)
        if (!c.copy_ev[j]) e = cudaEventCreateWithFlags(&c.copy_ev[j], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "qmpm_step_host_stream: copy stream");
    const int64_t per = (c.N + chunks - 1) / chunks;
    const size_t hp = sizeof(uint32_t) * (size_t)c.N, dp = sizeof(uint32_t) * (size_t)c.ld;
    for (int s = 0; s < nsteps; ++s) {
        // the input: range j after the previous step's download of range j (the same host
        // words), so that it overlaps the download of the ranges after it
        for (int j = 0; j < chunks; ++j) {
            const int64_t p0 = (int64_t)j * per, n = std::min<int64_t>(per, c.N - p0);
            if (n <= 0) break;
            if (s > 0) e = cudaStreamWaitEvent(c.stream, c.copy_ev[j], 0);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(c.words[c.cur] + p0, dp, h_words + p0, hp, sizeof(uint32_t) * (size_t)n,
                                      (size_t)c.W, cudaMemcpyHostToDevice, c.stream);
            if (e != cudaSuccess) return cuda_fail(e, "qmpm_step_host_stream: upload");
        }
        // the grid of the device's previous state is stale: clear it and redo the P2G
        qmpm::batch_invalidate(c.batch);
        int rc = do_clear(c, c.gcur);
        if (rc != QMPM_OK) return rc;
        c.primed = false;
        rc = qmpm_step(h, 1);
        if (rc != QMPM_OK) return rc;
        // the result, range by range on the copy stream
        e = cudaEventRecord(c.step_ev, c.stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c.copy_stream, c.step_ev, 0);
        for (int j = 0; j < chunks && e == cudaSuccess; ++j) {
            const int64_t p0 = (int64_t)j * per, n = std::min<int64_t>(per, c.N - p0);
            if (n <= 0) break;
            e = cudaMemcpy2DAsync(h_words + p0, hp, c.words[c.cur] + p0, dp, sizeof(uint32_t) * (size_t)n,
                                  (size_t)c.W, cudaMemcpyDeviceToHost, c.copy_stream);
            if (e == cudaSuccess) e = cudaEventRecord(c.copy_ev[j], c.copy_stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "qmpm_step_host_stream: download");
    }
    e = cudaStreamSynchronize(c.copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_fail(e, "qmpm_step_host_stream");
    return QMPM_OK;
}

int qmpm_specialize_compile(int32_t dim, int32_t material, const qmpm_scheme_t *scheme, int32_t stats,
                            int32_t dither, double *seconds, int64_t *cubin_bytes)
{
    if ((dim != 2 && dim != 3) || material < 0 || material > 2)
        return fail(QMPM_ERR_INVALID_ARG, "qmpm_specialize_compile: bad dim or material");
    qmpm_scheme_t s;
    if (scheme && scheme->quantized) {
        s = *scheme;
    } else {
        std::memset(&s, 0, sizeof(s));  // FP32 state
    }
    std::string err;
    int rc = qmpm::layout(dim, material, &s, err);
    if (rc != QMPM_OK) return fail(rc, err);
    qmpm::CompCodec cc[qmpm::kMaxComp];
    qmpm::build_codec(s, dim, material, cc);
    rc = qmpm::specialize_compile_only(dim, material, stats != 0, dither != 0, s.n_words, s.quantized ? cc : nullptr,
                                       qmpm::n_comp(dim, material), seconds, cubin_bytes, err);
    if (rc != QMPM_OK) return fail(rc, err);
    return QMPM_OK;
}

int qmpm_step_kernel_info(qmpm_handle h, int32_t *specialized, double *compile_seconds)
{
    if (!h) return fail(QMPM_ERR_INVALID_ARG, "bad handle");
    if (specialized) *specialized = h->spec_kernel ? 1 : 0;
    if (compile_seconds) *compile_seconds = h->spec_kernel ? h->spec_seconds : 0.0;
    return QMPM_OK;
}

int qmpm_profile(qmpm_handle h, qmpm_profile_t *out, int32_t reset)
{
    if (!h) return fail(QMPM_ERR_INVALID_ARG, "bad handle");
    Ctx &c = *h;
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_fail(e, "profile");
    qmpm::Profile &p = *c.prof;
    for (auto &r : p.recs) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            p.ms[r.kind] += ms;
            p.n[r.kind] += 1;
        }
        p.pool.push_back(r.a);
        p.pool.push_back(r.b);
    }
    p.recs.clear();
    if (out) {
        out->step_ms = p.ms[PROF_STEP];
        out->step_launches = p.n[PROF_STEP];
        out->clear_ms = p.ms[PROF_CLEAR];
        out->clear_launches = p.n[PROF_CLEAR];
        out->sort_ms = p.ms[PROF_SORT];
        out->sort_calls = p.n[PROF_SORT];
        out->p2g_ms = p.ms[PROF_P2G];
        out->p2g_launches = p.n[PROF_P2G];
        out->kernel_launches = c.launches;
    }
    if (reset) {
        for (int k = 0; k < 4; ++k) {
            p.ms[k] = 0.0;
            p.n[k] = 0;
        }
        c.launches = 0;
    }
    return QMPM_OK;
}

int qmpm_state_device(qmpm_handle h, uint32_t **d_words, int64_t *ld, int64_t **d_ids)
{
    if (!h) return fail(QMPM_ERR_INVALID_ARG, "bad handle");
    if (d_words) *d_words = h->words[h->cur];
    if (ld) *ld = h->ld;
    if (d_ids) *d_ids = h->ids[h->cur];
    return QMPM_OK;
}

int qmpm_destroy(qmpm_handle h)
{
    if (!h) return QMPM_OK;
    if (h->batch) qmpm_batch_remove(h->batch, h);
    cudaStreamSynchronize(h->stream);
    release(h);
    return QMPM_OK;
}

int qmpm_pack_f32(int32_t dim, int32_t material, const qmpm_scheme_t *scheme, uint64_t seed, int32_t dither,
                  uint32_t step, const float *d_vals, int64_t N, uint32_t *d_words, int64_t ld, qmpm_stats_t *stats,
                  void *stream)
{
    if (!scheme || N < 0 || ld < N || (N > 0 && (!d_vals || !d_words)))
        return fail(QMPM_ERR_INVALID_ARG, "qmpm_pack_f32: bad arguments");
    if (!scheme->quantized) return fail(QMPM_ERR_SCHEME, "qmpm_pack_f32 needs a quantized scheme");
    qmpm_scheme_t s = *scheme;
    std::string err;
    int rc = qmpm::layout(dim, material, &s, err);
    if (rc != QMPM_OK) return fail(rc, err);
    qmpm::CompCodec cc[qmpm::kMaxComp];
    qmpm::build_codec(s, dim, material, cc);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long *d_stats = nullptr;
    cudaError_t e;
    if (stats) {
        e = cudaMalloc(&d_stats, 16 * sizeof(unsigned long long));
        if (e != cudaSuccess) return fail(QMPM_ERR_OOM, "stats allocation failed");
        e = cudaMemsetAsync(d_stats, 0, 16 * sizeof(unsigned long long), st);
        if (e != cudaSuccess) {
            cudaFree(d_stats);
            return cuda_fail(e, "stats clear");
        }
    }
    e = qmpm::launch_pack_f32(dim, material, cc, qmpm::n_comp(dim, material), s.n_words, seed, dither, step, d_vals, N,
                              d_words, ld, d_stats, st);
    if (e != cudaSuccess) {
        if (d_stats) cudaFree(d_stats);
        return cuda_fail(e, "pack");
    }
    if (stats) {
        unsigned long long h[16];
        e = cudaMemcpyAsync(h, d_stats, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(d_stats);
        if (e != cudaSuccess) return cuda_fail(e, "pack stats");
        std::memset(stats, 0, sizeof(*stats));
        for (int k = 0; k < 4; ++k) {
            stats->saturations[k] = (int64_t)h[k];
            stats->round_ups[k] = (int64_t)h[4 + k];
            stats->round_downs[k] = (int64_t)h[8 + k];
        }
        stats->n_words = s.n_words;
    }
    return QMPM_OK;
}

int qmpm_unpack_f32(int32_t dim, int32_t material, const qmpm_scheme_t *scheme, const uint32_t *d_words, int64_t N,
                    int64_t ld, float *d_vals, void *stream)
{
    if (!scheme || N < 0 || ld < N || (N > 0 && (!d_vals || !d_words)))
        return fail(QMPM_ERR_INVALID_ARG, "qmpm_unpack_f32: bad arguments");
    if (!scheme->quantized) return fail(QMPM_ERR_SCHEME, "qmpm_unpack_f32 needs a quantized scheme");
    qmpm_scheme_t s = *scheme;
    std::string err;
    int rc = qmpm::layout(dim, material, &s, err);
    if (rc != QMPM_OK) return fail(rc, err);
    qmpm::CompCodec cc[qmpm::kMaxComp];
    qmpm::build_codec(s, dim, material, cc);
    cudaError_t e = qmpm::launch_unpack_f32(dim, material, cc, qmpm::n_comp(dim, material), d_words, N, ld, d_vals,
                                            static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "unpack");
    return QMPM_OK;
}

}  // extern "C"
