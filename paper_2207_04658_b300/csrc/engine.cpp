// engine.cpp -- the serving loop of libqmpm (qmpm_engine_*): scenes arrive as requests
// (scene, scheme, initial state, step count), wait in a FIFO queue, are admitted while their
// device footprint fits the memory budget and a batch slot is free, step together in one
// multi-scene batch (continuous batching: members join and leave between iterations while
// the others keep running), and leave with their measurement and, on request, their final
// state.  The loop runs on a background thread (qmpm_engine_start) or in the caller's thread
// (qmpm_engine_run).
//
// Threads and streams: admitted scenes are created (upload, encode, sort, P2G) by an init
// thread, each on a stream of its own, while the loop thread keeps the batch stream busy;
// they join the batch at the loop's next iteration.  Finished scenes are measured on their
// own stream and freed by the stream-ordered allocator without synchronising the device.
// At most two iterations are in flight on the batch stream.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "qmpm_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    qmpm_scene_t scene;
    qmpm_scheme_t scheme;
    bool has_scheme = false;
    bool keep_state = false;
    std::vector<double> state;  // initial state until admission, final state if kept
    const double *borrowed = nullptr;  // the caller's initial state (QMPM_SUBMIT_BORROW)
    std::vector<int64_t> ids;
    int32_t steps = 0;
    int32_t done_steps = 0;
    int64_t resident = 0, peak = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int32_t status = QMPM_REQ_QUEUED;
    int32_t error = 0;
    double z = 0;
    qmpm_handle h = nullptr;
    cudaStream_t stream = nullptr;  // the scene's own stream (init, measurement, frees)
    cudaEvent_t done_ev = nullptr;
    double *h_z = nullptr;  // pinned
};

}  // namespace

struct qmpm_engine {
    qmpm_engine_config_t cfg;
    int dev = 0;
    bool device_ready = false;  // streams, events, pinned slots and batch made (first iteration)
    cudaStream_t step_stream = nullptr;
    qmpm_batch_handle batch = nullptr;
    double *pinned = nullptr;  // one z slot per request id modulo kSlots
    static constexpr int kSlots = 4096;

    std::mutex mu;  // guards queue, to_init, ready, done, kept, next_id, reserved, counters
    std::condition_variable cv, init_cv;
    std::deque<Request *> queue;
    std::deque<Request *> to_init;   // admitted, waiting for the init thread
    std::vector<Request *> ready;    // created, waiting to join the batch
    int64_t reserved = 0;            // bytes of admitted scenes (peak until created, then resident)
    int in_init = 0;                 // requests between admission and joining
    std::thread init_worker;
    bool init_stop = false;
    std::vector<Request *> done;
    std::map<int64_t, Request *> kept;
    int64_t next_id = 1;
    int64_t pending = 0;             // submitted requests not yet finished (idle when 0)
    int64_t snap_active = 0, snap_bytes = 0, snap_particle_steps = 0, snap_iterations = 0;  // for stats
    int64_t snap_launches = 0, snap_graph_launches = 0;

    // loop-thread state
    std::vector<Request *> active, finishing;
    int64_t particle_steps = 0, iterations = 0, n_done = 0;
    cudaEvent_t iter_ev[2] = {nullptr, nullptr};
    bool iter_pending[2] = {false, false};
    int iter_idx = 0;

    std::thread worker;
    std::atomic<bool> running{false}, stop_req{false}, drain{false};
    Clock::time_point t0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

int efail(int code, const std::string &msg)
{
    qmpm::set_last_error(msg);
    return code;
}

void finish(qmpm_engine &e, Request *r, int32_t status)
{
    r->status = status;
    r->t_done = e.now();
    if (r->h) {
        qmpm::destroy_nosync(r->h);  // frees ordered on the scene's stream, no wait
        r->h = nullptr;
        std::lock_guard<std::mutex> lk(e.mu);
        e.reserved -= r->resident;
    }
    if (r->stream) {
        cudaStreamDestroy(r->stream);  // released once its work is done
        r->stream = nullptr;
    }
    if (r->done_ev) {
        cudaEventDestroy(r->done_ev);
        r->done_ev = nullptr;
    }
    if (!r->keep_state) {
        std::vector<double>().swap(r->state);
        std::vector<int64_t>().swap(r->ids);
    }
    std::lock_guard<std::mutex> lk(e.mu);
    e.done.push_back(r);
    e.n_done += 1;
    e.pending -= 1;
}

// Requests whose measurement has reached the host.
void collect(qmpm_engine &e)
{
    for (size_t i = 0; i < e.finishing.size();) {
        Request *r = e.finishing[i];
        const cudaError_t q = cudaEventQuery(r->done_ev);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        e.finishing.erase(e.finishing.begin() + i);
        if (q != cudaSuccess) {
            r->error = QMPM_ERR_CUDA;
            finish(e, r, QMPM_REQ_FAILED);
            continue;
        }
        r->z = *r->h_z;
        if (r->keep_state) {
            const qmpm::Ctx &c = *r->h;
            r->state.resize((size_t)c.N * c.n_comp);
            r->ids.resize((size_t)c.N);
            const int rc = qmpm_readback(r->h, r->state.data(), nullptr, r->ids.data(), nullptr);
            if (rc != QMPM_OK) {
                r->error = rc;
                finish(e, r, QMPM_REQ_FAILED);
                continue;
            }
        }
        finish(e, r, QMPM_REQ_DONE);
    }
}

// FIFO admission while the next request's peak footprint fits and a batch slot is free:
// the request's bytes are reserved and it goes to the init thread.
void admit(qmpm_engine &e)
{
    std::vector<Request *> too_big;
    {
        std::lock_guard<std::mutex> lk(e.mu);
        while (!e.queue.empty()) {
            Request *f = e.queue.front();
            if (f->peak > e.cfg.budget_bytes) {  // can never fit
                e.queue.pop_front();
                f->error = QMPM_ERR_OOM;
                too_big.push_back(f);
                continue;
            }
            if ((int)e.active.size() + e.in_init >= e.cfg.max_active) break;
            if (e.reserved + f->peak > e.cfg.budget_bytes) break;
            e.queue.pop_front();
            e.reserved += f->peak;
            e.in_init += 1;
            f->t_admit = e.now();
            e.to_init.push_back(f);
        }
    }
    e.init_cv.notify_one();
    for (Request *r : too_big) finish(e, r, QMPM_REQ_FAILED);
}

// The init thread: create admitted scenes; the reservation drops from the peak footprint to
// the resident one once the initial state is gone.
void init_loop(qmpm_engine *e)
{
    cudaSetDevice(e->dev);
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(e->mu);
            e->init_cv.wait(lk, [e] { return e->init_stop || !e->to_init.empty(); });
            if (e->to_init.empty()) return;
            r = e->to_init.front();
            e->to_init.pop_front();
        }
        int rc = cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) == cudaSuccess ? QMPM_OK
                                                                                           : QMPM_ERR_CUDA;
        if (rc == QMPM_OK)
            rc = qmpm_init(&r->scene, r->has_scheme ? &r->scheme : nullptr,
                           r->borrowed ? r->borrowed : r->state.data(), r->stream, &r->h);
        r->borrowed = nullptr;  // the caller's buffer is no longer needed
        std::vector<double>().swap(r->state);
        std::lock_guard<std::mutex> lk(e->mu);
        e->reserved -= r->peak - (rc == QMPM_OK ? r->resident : 0);
        if (rc != QMPM_OK) {
            r->h = nullptr;
            r->error = rc;
        }
        e->ready.push_back(r);
        e->cv.notify_all();
    }
}

// Created scenes join the batch (or, with nothing to step, go straight to measurement).
void join_ready(qmpm_engine &e)
{
    std::vector<Request *> rd;
    {
        std::lock_guard<std::mutex> lk(e.mu);
        rd.swap(e.ready);
        e.in_init -= (int)rd.size();
    }
    for (Request *r : rd) {
        r->h_z = e.pinned + (r->id % qmpm_engine::kSlots);
        int rc = r->error ? r->error : QMPM_OK;
        if (rc == QMPM_OK && r->steps > 0) rc = qmpm_batch_add(e.batch, r->h);
        if (rc != QMPM_OK) {
            r->error = rc;
            finish(e, r, QMPM_REQ_FAILED);
            continue;
        }
        r->status = QMPM_REQ_RUNNING;
        if (r->steps == 0) {
            qmpm::launch_measure(*r->h);
            cudaMemcpyAsync(r->h_z, r->h->d_z, sizeof(double), cudaMemcpyDeviceToHost, r->h->stream);
            cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
            cudaEventRecord(r->done_ev, r->h->stream);
            e.finishing.push_back(r);
        } else {
            e.active.push_back(r);
        }
    }
}

// The engine's device resources, made on the first iteration (creation stays host only).
int setup_device(qmpm_engine &e)
{
    cudaSetDevice(e.dev);
    // keep freed scene memory in the pool between requests instead of returning it to the
    // driver at every synchronisation (a setting of this process's pool only)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, e.dev) == cudaSuccess) {
        uint64_t keep = ~uint64_t(0);
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaError_t ce = cudaSuccess;
    if (!e.step_stream) ce = cudaStreamCreateWithFlags(&e.step_stream, cudaStreamNonBlocking);
    if (ce == cudaSuccess && !e.iter_ev[0]) ce = cudaEventCreateWithFlags(&e.iter_ev[0], cudaEventDisableTiming);
    if (ce == cudaSuccess && !e.iter_ev[1]) ce = cudaEventCreateWithFlags(&e.iter_ev[1], cudaEventDisableTiming);
    if (ce == cudaSuccess && !e.pinned)
        ce = cudaMallocHost(reinterpret_cast<void **>(&e.pinned), sizeof(double) * qmpm_engine::kSlots);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return efail(QMPM_ERR_CUDA, std::string("engine device setup: ") + cudaGetErrorString(ce));
    }
    if (!e.batch) {
        const int rc = qmpm_batch_create(e.step_stream, e.cfg.resort_every, e.cfg.flags, &e.batch);
        if (rc != QMPM_OK) return rc;
    }
    e.device_ready = true;
    return QMPM_OK;
}

// One iteration: completions, admissions, then up to resort_every steps of every member.
// Returns the number of members stepped.
int iterate(qmpm_engine &e, int *rc_out = nullptr)
{
    collect(e);
    admit(e);
    if (!e.device_ready) {
        const int rc = setup_device(e);
        if (rc != QMPM_OK) {
            if (rc_out) *rc_out = rc;
            return 0;
        }
    }
    join_ready(e);
    if (e.active.empty()) return 0;
    int32_t L = e.cfg.resort_every > 0 ? e.cfg.resort_every : 8;
    for (Request *r : e.active) L = std::min(L, r->steps - r->done_steps);
    // at most two iterations in flight
    if (e.iter_pending[e.iter_idx]) {
        cudaEventSynchronize(e.iter_ev[e.iter_idx]);
        e.iter_pending[e.iter_idx] = false;
    }
    int rc = qmpm_batch_step(e.batch, L);
    if (rc == QMPM_OK) {
        cudaEventRecord(e.iter_ev[e.iter_idx], e.step_stream);
        e.iter_pending[e.iter_idx] = true;
        e.iter_idx ^= 1;
    }
    const int stepped = (int)e.active.size();
    for (size_t i = 0; i < e.active.size();) {
        Request *r = e.active[i];
        if (rc != QMPM_OK) {
            qmpm_batch_remove(e.batch, r->h);
            r->error = rc;
            e.active.erase(e.active.begin() + i);
            finish(e, r, QMPM_REQ_FAILED);
            continue;
        }
        r->done_steps += L;
        e.particle_steps += (int64_t)L * r->scene.n_particles;
        if (r->done_steps >= r->steps) {
            // leave the batch; measure on the scene's own stream after the batch's work
            qmpm_batch_remove(e.batch, r->h);
            qmpm::launch_measure(*r->h);
            cudaMemcpyAsync(r->h_z, r->h->d_z, sizeof(double), cudaMemcpyDeviceToHost, r->h->stream);
            cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
            cudaEventRecord(r->done_ev, r->h->stream);
            e.active.erase(e.active.begin() + i);
            e.finishing.push_back(r);
            continue;
        }
        ++i;
    }
    e.iterations += 1;
    std::lock_guard<std::mutex> lk(e.mu);
    e.snap_active = (int64_t)e.active.size();
    e.snap_bytes = e.reserved;
    e.snap_particle_steps = e.particle_steps;
    e.snap_iterations = e.iterations;
    qmpm_batch_info_t bi;
    if (qmpm_batch_info(e.batch, &bi) == QMPM_OK) {
        e.snap_launches = bi.kernel_launches;
        e.snap_graph_launches = bi.graph_launches;
    }
    return stepped;
}

// (called from the loop's thread, which alone changes active and finishing)
bool idle(qmpm_engine &e)
{
    std::lock_guard<std::mutex> lk(e.mu);
    return e.queue.empty() && e.in_init == 0 && e.active.empty() && e.finishing.empty();
}

void loop(qmpm_engine *e)
{
    cudaSetDevice(e->dev);
    while (true) {
        if (e->stop_req.load() && (!e->drain.load() || idle(*e))) break;
        int rc = QMPM_OK;
        const int stepped = iterate(*e, &rc);
        if (rc != QMPM_OK) break;  // no device: nothing can run
        if (stepped == 0) {
            std::unique_lock<std::mutex> lk(e->mu);
            e->cv.wait_for(lk, std::chrono::microseconds(e->finishing.empty() ? 1000 : 50),
                           [e] { return !e->queue.empty() || !e->ready.empty() || e->stop_req.load(); });
        }
    }
    collect(*e);
}

}  // namespace

extern "C" {

int qmpm_engine_create(const qmpm_engine_config_t *cfg, qmpm_engine_handle *out)
{
    if (!cfg || !out) return efail(QMPM_ERR_INVALID_ARG, "cfg or out is NULL");
    if (cfg->budget_bytes <= 0 || cfg->max_active <= 0 || cfg->max_active > 256 || cfg->resort_every < 0 ||
        cfg->max_queued < 0)
        return efail(QMPM_ERR_INVALID_ARG, "bad engine configuration");
    *out = nullptr;
    qmpm_engine *e = new (std::nothrow) qmpm_engine();
    if (!e) return efail(QMPM_ERR_OOM, "host allocation failed");
    e->cfg = *cfg;
    e->t0 = Clock::now();
    if (cudaGetDevice(&e->dev) != cudaSuccess) {
        cudaGetLastError();
        e->dev = 0;
    }
    e->init_worker = std::thread(init_loop, e);
    *out = e;
    return QMPM_OK;
}

int qmpm_engine_submit(qmpm_engine_handle e, const qmpm_scene_t *scene, const qmpm_scheme_t *scheme,
                       const double *h_state, int32_t steps, int32_t flags, int64_t *id)
{
    if (!e || !scene || steps < 0 || (scene->n_particles > 0 && !h_state))
        return efail(QMPM_ERR_INVALID_ARG, "bad request");
    int vrc = qmpm::validate_scene(scene);
    if (vrc != QMPM_OK) return vrc;
    if (scheme && scheme->quantized) {
        qmpm_scheme_t chk = *scheme;
        vrc = qmpm_scheme_layout(scene->dim, scene->material, &chk);
        if (vrc != QMPM_OK) return vrc;
    }
    {
        // a corrupted initial state (NaN or infinite values) is refused before it is queued
        const int nc0 = 2 * scene->dim + scene->dim * scene->dim +
                        (scene->material == QMPM_FLUID ? 1 : scene->dim * scene->dim);
        const size_t nv = (size_t)scene->n_particles * (size_t)nc0;
        for (size_t i = 0; i < nv; ++i)
            if (!std::isfinite(h_state[i]))
                return efail(QMPM_ERR_INVALID_ARG, "request state holds a non-finite value at index " +
                                                       std::to_string(i));
    }
    Request *r = qmpm::fault_hit(QMPM_FAULT_HOST_ALLOC) ? nullptr : new (std::nothrow) Request();
    if (!r) return efail(QMPM_ERR_OOM, "host allocation failed");
    r->scene = *scene;
    r->has_scheme = scheme && scheme->quantized;
    if (r->has_scheme) r->scheme = *scheme;
    int rc = qmpm_footprint(scene, r->has_scheme ? scheme : nullptr, &r->resident, &r->peak);
    if (rc != QMPM_OK) {
        delete r;
        return rc;
    }
    const int nc = 2 * scene->dim + scene->dim * scene->dim +
                   (scene->material == QMPM_FLUID ? 1 : scene->dim * scene->dim);
    if (flags & QMPM_SUBMIT_BORROW)
        r->borrowed = h_state;
    else
        r->state.assign(h_state, h_state + (size_t)scene->n_particles * nc);
    r->steps = steps;
    r->keep_state = (flags & QMPM_SUBMIT_KEEP_STATE) != 0;
    r->t_submit = e->now();
    {
        std::lock_guard<std::mutex> lk(e->mu);
        if (e->cfg.max_queued > 0 && (int64_t)e->queue.size() >= e->cfg.max_queued) {
            delete r;
            return efail(QMPM_ERR_QUEUE_FULL, "the request queue is full (max_queued)");
        }
        r->id = e->next_id++;
        e->pending += 1;
        e->queue.push_back(r);
    }
    e->cv.notify_one();
    if (id) *id = r->id;
    return QMPM_OK;
}

int qmpm_engine_run(qmpm_engine_handle e, int32_t iterations, int32_t *busy)
{
    if (!e || iterations < 0) return efail(QMPM_ERR_INVALID_ARG, "bad engine or iterations");
    if (e->running.load()) return efail(QMPM_ERR_INVALID_ARG, "the engine's thread is running");
    int rc = QMPM_OK;
    for (int i = 0; i < iterations && rc == QMPM_OK; ++i) iterate(*e, &rc);
    if (busy) *busy = idle(*e) ? 0 : 1;
    return rc;
}

int qmpm_engine_wait(qmpm_engine_handle e, double timeout_s, int32_t *busy)
{
    if (!e || !(timeout_s >= 0.0)) return efail(QMPM_ERR_INVALID_ARG, "bad engine or timeout");
    if (qmpm::fault_hit(QMPM_FAULT_WAIT)) {
        if (busy) *busy = 1;
        return efail(QMPM_ERR_TIMEOUT, "qmpm_engine_wait: deadline passed (injected)");
    }
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(e->mu);
            if (e->pending == 0) {  // every submitted request has finished
                if (busy) *busy = 0;
                return QMPM_OK;
            }
        }
        if (Clock::now() >= deadline) {
            if (busy) *busy = 1;
            return efail(QMPM_ERR_TIMEOUT, "qmpm_engine_wait: deadline passed with work remaining");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(500));
    }
}

int qmpm_engine_start(qmpm_engine_handle e)
{
    if (!e) return efail(QMPM_ERR_INVALID_ARG, "bad engine");
    if (e->running.exchange(true)) return QMPM_OK;
    e->stop_req = false;
    e->worker = std::thread(loop, e);
    return QMPM_OK;
}

int qmpm_engine_stop(qmpm_engine_handle e, int32_t drain)
{
    if (!e) return efail(QMPM_ERR_INVALID_ARG, "bad engine");
    if (!e->running.load()) return QMPM_OK;
    e->drain = drain != 0;
    e->stop_req = true;
    e->cv.notify_all();
    e->worker.join();
    e->running = false;
    return QMPM_OK;
}

int qmpm_engine_poll(qmpm_engine_handle e, qmpm_request_t *out, int32_t max, int32_t *n_out)
{
    if (!e || (max > 0 && !out) || !n_out) return efail(QMPM_ERR_INVALID_ARG, "bad poll arguments");
    std::lock_guard<std::mutex> lk(e->mu);
    int32_t n = 0;
    while (n < max && !e->done.empty()) {
        Request *r = e->done.front();
        e->done.erase(e->done.begin());
        qmpm_request_t &o = out[n++];
        std::memset(&o, 0, sizeof(o));
        o.id = r->id;
        o.status = r->status;
        o.error = r->error;
        o.steps = r->steps;
        o.particles = r->scene.n_particles;
        o.resident_bytes = r->resident;
        o.t_submit = r->t_submit;
        o.t_admit = r->t_admit;
        o.t_done = r->t_done;
        o.z = r->z;
        if (r->keep_state && r->status == QMPM_REQ_DONE) e->kept[r->id] = r;
        else delete r;
    }
    *n_out = n;
    return QMPM_OK;
}

int qmpm_engine_result(qmpm_engine_handle e, int64_t id, double *h_state, int64_t *h_ids)
{
    if (!e) return efail(QMPM_ERR_INVALID_ARG, "bad engine");
    std::lock_guard<std::mutex> lk(e->mu);
    auto it = e->kept.find(id);
    if (it == e->kept.end()) return efail(QMPM_ERR_INVALID_ARG, "no kept result for this id (poll it first)");
    Request *r = it->second;
    if (h_state) std::memcpy(h_state, r->state.data(), r->state.size() * sizeof(double));
    if (h_ids) std::memcpy(h_ids, r->ids.data(), r->ids.size() * sizeof(int64_t));
    return QMPM_OK;
}

int qmpm_engine_release(qmpm_engine_handle e, int64_t id)
{
    if (!e) return efail(QMPM_ERR_INVALID_ARG, "bad engine");
    std::lock_guard<std::mutex> lk(e->mu);
    auto it = e->kept.find(id);
    if (it != e->kept.end()) {
        delete it->second;
        e->kept.erase(it);
    }
    return QMPM_OK;
}

int qmpm_engine_stats(qmpm_engine_handle e, qmpm_engine_stats_t *out)
{
    if (!e || !out) return efail(QMPM_ERR_INVALID_ARG, "bad engine or out");
    std::memset(out, 0, sizeof(*out));
    std::lock_guard<std::mutex> lk(e->mu);
    out->queued = (int64_t)e->queue.size();
    out->active = e->snap_active;
    out->finished = e->n_done;
    out->bytes_in_use = e->snap_bytes;
    out->particle_steps = e->snap_particle_steps;
    out->iterations = e->snap_iterations;
    out->elapsed = e->now();
    out->kernel_launches = e->snap_launches;
    out->graph_launches = e->snap_graph_launches;
    return QMPM_OK;
}

int qmpm_engine_destroy(qmpm_engine_handle e)
{
    if (!e) return QMPM_OK;
    qmpm_engine_stop(e, 0);
    if (e->init_worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(e->mu);
            e->init_stop = true;
            for (Request *r : e->to_init) delete r;
            e->to_init.clear();
        }
        e->init_cv.notify_all();
        e->init_worker.join();
    }
    for (Request *r : e->ready) {
        if (r->h) qmpm_destroy(r->h);
        if (r->stream) cudaStreamDestroy(r->stream);
        delete r;
    }
    e->ready.clear();
    if (e->step_stream) cudaStreamSynchronize(e->step_stream);
    for (Request *r : e->active) {
        if (r->h) qmpm_destroy(r->h);
        if (r->stream) cudaStreamDestroy(r->stream);
        delete r;
    }
    for (Request *r : e->finishing) {
        if (r->h) qmpm_destroy(r->h);
        if (r->done_ev) cudaEventDestroy(r->done_ev);
        if (r->stream) cudaStreamDestroy(r->stream);
        delete r;
    }
    for (Request *r : e->queue) delete r;
    for (Request *r : e->done) delete r;
    for (auto &kv : e->kept) delete kv.second;
    if (e->batch) qmpm_batch_destroy(e->batch);
    for (auto ev : e->iter_ev)
        if (ev) cudaEventDestroy(ev);
    if (e->pinned) cudaFreeHost(e->pinned);
    if (e->step_stream) cudaStreamDestroy(e->step_stream);
    delete e;
    return QMPM_OK;
}

}  // extern "C"
