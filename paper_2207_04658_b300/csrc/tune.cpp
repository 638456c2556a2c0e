// tune.cpp -- the autotuner of libqmpm (qmpm_autotune): times the step of a scene for every
// candidate (particles per work item, re-sort interval) on scratch copies of the scene and
// returns the fastest, remembering the answer per scene class for the rest of the process.
//
// The work item size trades the per-chunk cost (grid tile staging, flush atomics, barriers)
// against load balance over the persistent CTAs; the re-sort interval trades the sort's
// cost against particles drifting out of their tile (the slow path) between sorts.  The
// grid block is fixed at 4^d nodes (the tile, shared-memory layout and sort key are built
// around it) and the CTAs per SM are fixed per kernel by its register budget.
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "qmpm_internal.h"

namespace {

using Key = std::tuple<int, int, int, int, int, int>;  // dim, material, quantized, words, grid, log2 N

std::mutex g_mu;
std::map<Key, qmpm_tune_t> g_cache;

const int kChunks[] = {64, 128, 192, 256};
const int kResorts[] = {4, 8, 16, 32};

int tfail(int code, const std::string &msg)
{
    qmpm::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" {

int qmpm_autotune(const qmpm_scene_t *scene, const qmpm_scheme_t *scheme, const double *h_state,
                  int32_t trial_steps, int32_t use_cache, qmpm_tune_t *out)
{
    if (!scene || !out || (scene->n_particles > 0 && !h_state) || trial_steps < 1)
        return tfail(QMPM_ERR_INVALID_ARG, "bad autotune arguments");
    qmpm_scheme_t sch;
    std::memset(&sch, 0, sizeof(sch));
    const bool quant = scheme && scheme->quantized;
    if (quant) sch = *scheme;
    int rc = qmpm_scheme_layout(scene->dim, scene->material, &sch);
    if (rc != QMPM_OK) return rc;
    const int log2n = scene->n_particles > 0 ? (int)std::lround(std::log2((double)scene->n_particles)) : 0;
    const Key key(scene->dim, scene->material, quant ? 1 : 0, sch.n_words, scene->grid_log2, log2n);
    if (use_cache) {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            *out = it->second;
            out->from_cache = 1;
            return QMPM_OK;
        }
    }
    std::memset(out, 0, sizeof(*out));
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        if (s) cudaStreamDestroy(s);
        return tfail(QMPM_ERR_CUDA, std::string("autotune setup: ") + cudaGetErrorString(e));
    }
    double best = 1e300;
    int idx = 0;
    for (int ci = 0; ci < 4; ++ci)
        for (int ri = 0; ri < 4; ++ri, ++idx) {
            qmpm_scene_t sc = *scene;
            sc.chunk = kChunks[ci];
            sc.resort_every = kResorts[ri];
            sc.flags &= ~(QMPM_FLAG_PROFILE | QMPM_FLAG_STATS | QMPM_FLAG_STRICT);
            qmpm_handle h = nullptr;
            rc = qmpm_init(&sc, quant ? &sch : nullptr, h_state, s, &h);
            if (rc != QMPM_OK) break;
            rc = qmpm_step(h, 2);  // warm-up
            // time a whole number of re-sort periods
            const int T = ((trial_steps + sc.resort_every - 1) / sc.resort_every) * sc.resort_every;
            if (rc == QMPM_OK) e = cudaEventRecord(a, s);
            if (rc == QMPM_OK && e == cudaSuccess) rc = qmpm_step(h, T);
            if (rc == QMPM_OK && e == cudaSuccess) e = cudaEventRecord(b, s);
            if (rc == QMPM_OK && e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0.0f;
            if (rc == QMPM_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            qmpm_destroy(h);
            if (rc != QMPM_OK) break;
            if (e != cudaSuccess) {
                rc = tfail(QMPM_ERR_CUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
                break;
            }
            const double per_step = ms / T;
            out->chunk_cand[idx] = sc.chunk;
            out->resort_cand[idx] = sc.resort_every;
            out->ms_per_step[idx] = per_step;
            if (per_step < best) {
                best = per_step;
                out->chunk = sc.chunk;
                out->resort_every = sc.resort_every;
                out->best_ms_per_step = per_step;
            }
        }
    out->n_candidates = idx;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(s);
    if (rc != QMPM_OK) return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = *out;
    return QMPM_OK;
}

}  // extern "C"
