// batch.cu -- multi-scene stepping (qmpm_batch_*): scenes of uneven sizes advance together,
// one persistent step launch per (dimension, material, quantized) class, driven by a
// table of per-scene parameters and the concatenated chunk lists as the work queue; one
// clear launch for all consumed grid buffers; the scenes' re-sorts where they fall due.
//
// Each member's host-side state (grid buffer parity, word buffer, step count) evolves with
// period 2S (S = the re-sort interval): the grid buffers swap every step and the word
// buffers at every re-sort.  The parameter tables of one period are therefore fixed, so a
// half period (S steps) is captured once as a CUDA graph and replayed; the dither step index
// comes from a per-member device counter that the graph advances.
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "qmpm_internal.h"

namespace {

struct Group {
    int dim, material;
    bool quant, stats;
    size_t smem;
    int64_t tab_off;  // first StepParams of the group in the batch's table
    int n;
};

// A member large enough to fill the GPU on its own steps in its own launch (parameters in
// the constant bank run faster than the multi-scene kernel's shared-memory copy).
struct Solo {
    int dim, material;
    bool quant, stats;
    size_t smem;
    qmpm::StepParams p;
};

constexpr int64_t kSoloChunks = 1024;  // about 260,000 particles

struct Phase {
    std::vector<Group> groups;
    std::vector<Solo> solos;
    int64_t clear_off;
    int n_clear;
    int64_t virtual_blocks;
    std::vector<int> resort;  // members re-sorted after this step
};

struct Saved {
    cudaStream_t stream;
    int32_t resort_every;
};

}  // namespace

struct qmpm_batch {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int S = 8;
    int flags = 0;
    int n_sms = 1;
    std::vector<qmpm_ctx *> members;
    std::vector<Saved> saved;
    bool planned = false;
    std::vector<Phase> phases;  // one period
    int phase = 0;              // next phase to run
    qmpm::StepParams *d_tab = nullptr;
    size_t tab_cap = 0;
    qmpm::ClearItem *d_clear = nullptr;
    size_t clear_cap = 0;
    uint32_t *d_ctr = nullptr;
    size_t ctr_cap = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_kernels[2] = {0, 0};  // kernels each graph launches
    bool fresh = false;                 // tables rebuilt during the current qmpm_batch_step
    // pinned staging of the tables, two sets used in turn: a set is rewritten only after its
    // previous upload (two plans back) has completed
    struct Staging {
        qmpm::StepParams *tab = nullptr;
        qmpm::ClearItem *clr = nullptr;
        uint32_t *ctr = nullptr;
        size_t tab_cap = 0, clr_cap = 0, ctr_cap = 0;
        cudaEvent_t uploaded = nullptr;
        bool pending = false;
    } staging[2];
    int next_staging = 0;
    int64_t launches = 0;
    int64_t graph_launches = 0;
    int64_t steps = 0;
};

namespace {

int bfail(int code, const std::string &msg)
{
    qmpm::set_last_error(msg);
    return code;
}

int bcuda(cudaError_t e, const char *what)
{
    return bfail(QMPM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int period(const qmpm_batch &b) { return b.S > 0 ? 2 * b.S : 2; }

void drop_graphs(qmpm_batch &b)
{
    for (auto &g : b.graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

template <class T>
cudaError_t grow(T **p, size_t *cap, size_t need)
{
    if (need <= *cap) return cudaSuccess;
    const size_t n = std::max<size_t>(need, 2 * *cap);
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), n * sizeof(T));
    if (e == cudaSuccess) *cap = n;
    return e;
}

template <class T>
cudaError_t pinned_grow(T **p, size_t *cap, size_t need)
{
    if (need <= *cap) return cudaSuccess;
    const size_t n = std::max<size_t>(need, 2 * *cap);
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMallocHost(reinterpret_cast<void **>(p), n * sizeof(T));
    if (e == cudaSuccess) *cap = n;
    return e;
}

struct HostState {
    int gcur, cur;
    int64_t steps;
};

// Build the parameter and clear tables of one period from the members' current state.
int plan(qmpm_batch &b)
{
    const int P = period(b);
    const int n = (int)b.members.size();
    std::vector<qmpm::StepParams> tab;
    std::vector<qmpm::ClearItem> clr;
    b.phases.assign(P, Phase());
    std::vector<HostState> st(n);
    for (int m = 0; m < n; ++m) st[m] = {b.members[m]->gcur, b.members[m]->cur, b.members[m]->steps};
    // members of one launch class are contiguous in the table
    std::map<std::tuple<int, int, int, int>, std::vector<int>> cls;
    for (int m = 0; m < n; ++m) {
        const qmpm::Ctx &c = *b.members[m];
        if (c.N == 0) continue;
        if ((c.N + c.chunk - 1) / c.chunk >= kSoloChunks) continue;  // a solo member
        cls[std::make_tuple(c.scene.dim, c.scene.material, c.quant ? 1 : 0,
                            (c.scene.flags & QMPM_FLAG_STATS) ? 1 : 0)]
            .push_back(m);
    }
    for (int k = 0; k < P; ++k) {
        Phase &ph = b.phases[k];
        for (auto &kv : cls) {
            Group g;
            g.dim = std::get<0>(kv.first);
            g.material = std::get<1>(kv.first);
            g.quant = std::get<2>(kv.first) != 0;
            g.stats = std::get<3>(kv.first) != 0;
            g.smem = 0;
            g.tab_off = (int64_t)tab.size();
            g.n = (int)kv.second.size();
            for (int m : kv.second) {
                qmpm::Ctx c = *b.members[m];  // a copy with the simulated buffer state
                c.gcur = st[m].gcur;
                c.cur = st[m].cur;
                qmpm::StepParams p;
                qmpm::step_params(c, p, 0u);
                p.step_ctr = b.d_ctr + m;
                tab.push_back(p);
                g.smem = std::max(g.smem, qmpm::step_smem_bytes(c.scene.dim, c.W));
            }
            ph.groups.push_back(g);
        }
        for (int m = 0; m < n; ++m) {
            const qmpm::Ctx &c0 = *b.members[m];
            if (c0.N == 0 || (c0.N + c0.chunk - 1) / c0.chunk < kSoloChunks) continue;
            qmpm::Ctx c = c0;
            c.gcur = st[m].gcur;
            c.cur = st[m].cur;
            Solo so;
            so.dim = c.scene.dim;
            so.material = c.scene.material;
            so.quant = c.quant;
            so.stats = (c.scene.flags & QMPM_FLAG_STATS) != 0;
            so.smem = qmpm::step_smem_bytes(c.scene.dim, c.W);
            qmpm::step_params(c, so.p, 0u);
            so.p.step_ctr = b.d_ctr + m;
            ph.solos.push_back(so);
        }
        ph.clear_off = (int64_t)clr.size();
        int64_t first = 0;
        for (int m = 0; m < n; ++m) {
            const qmpm::Ctx &c = *b.members[m];
            qmpm::ClearItem it;
            it.grid = c.grid[st[m].gcur];
            it.touched = c.touched[st[m].gcur];
            it.n_blocks = c.n_blocks;
            it.first = first;
            it.block_nodes = (int32_t)c.block_nodes;
            it.pad = 0;
            first += (c.n_blocks + 31) / 32 * 32;
            clr.push_back(it);
        }
        ph.n_clear = n;
        ph.virtual_blocks = first;
        for (int m = 0; m < n; ++m) {
            st[m].gcur = 1 - st[m].gcur;
            st[m].steps += 1;
            if (b.S > 0 && st[m].steps % b.S == 0) {
                ph.resort.push_back(m);
                st[m].cur = 1 - st[m].cur;
            }
        }
    }
    // device tables grow rarely (a free synchronises the device); the uploads are ordered
    // on the batch stream after the work that still reads the previous tables
    cudaError_t e = grow(&b.d_tab, &b.tab_cap, std::max<size_t>(tab.size(), 64 * (size_t)P));
    if (e == cudaSuccess) e = grow(&b.d_clear, &b.clear_cap, std::max<size_t>(clr.size(), 64 * (size_t)P));
    if (e != cudaSuccess) return bfail(QMPM_ERR_OOM, "batch tables: device allocation failed");
    auto &st_ = b.staging[b.next_staging];
    b.next_staging ^= 1;
    if (st_.pending) {
        e = cudaEventSynchronize(st_.uploaded);  // this set's previous upload is done
        st_.pending = false;
        if (e != cudaSuccess) return bcuda(e, "batch tables");
    }
    e = pinned_grow(&st_.tab, &st_.tab_cap, std::max<size_t>(tab.size(), 1));
    if (e == cudaSuccess) e = pinned_grow(&st_.clr, &st_.clr_cap, std::max<size_t>(clr.size(), 1));
    if (e == cudaSuccess) e = pinned_grow(&st_.ctr, &st_.ctr_cap, (size_t)std::max(n, 1));
    if (e != cudaSuccess) return bfail(QMPM_ERR_OOM, "batch tables: pinned allocation failed");
    if (!tab.empty()) std::memcpy(st_.tab, tab.data(), tab.size() * sizeof(qmpm::StepParams));
    if (!clr.empty()) std::memcpy(st_.clr, clr.data(), clr.size() * sizeof(qmpm::ClearItem));
    for (int m = 0; m < n; ++m) st_.ctr[m] = (uint32_t)b.members[m]->steps;  // steps done so far
    if (!tab.empty())
        e = cudaMemcpyAsync(b.d_tab, st_.tab, tab.size() * sizeof(qmpm::StepParams), cudaMemcpyHostToDevice,
                            b.stream);
    if (e == cudaSuccess && !clr.empty())
        e = cudaMemcpyAsync(b.d_clear, st_.clr, clr.size() * sizeof(qmpm::ClearItem), cudaMemcpyHostToDevice,
                            b.stream);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(b.d_ctr, st_.ctr, n * sizeof(uint32_t), cudaMemcpyHostToDevice, b.stream);
    if (e == cudaSuccess && !st_.uploaded) e = cudaEventCreateWithFlags(&st_.uploaded, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(st_.uploaded, b.stream);
    if (e != cudaSuccess) return bcuda(e, "batch tables");
    st_.pending = true;
    b.phase = 0;
    b.planned = true;
    b.fresh = true;
    return QMPM_OK;
}

// Advance every member's host-side state by one step of phase k, launching the work
// unless `dry` (a graph replay does the launches).
int run_phase(qmpm_batch &b, int k, bool dry)
{
    const Phase &ph = b.phases[k];
    if (!dry) {
        for (const Solo &so : ph.solos) {
            cudaError_t e = qmpm::launch_step_ctr(so.dim, so.material, so.quant, so.stats, &so.p, so.smem, b.n_sms,
                                                  b.stream);
            if (e != cudaSuccess) return bcuda(e, "batch member step");
            b.launches += 1;
        }
        for (const Group &g : ph.groups) {
            cudaError_t e = qmpm::launch_step_multi(g.dim, g.material, g.quant, g.stats, b.d_tab + g.tab_off, g.n,
                                                    g.smem, b.n_sms, b.stream);
            if (e != cudaSuccess) return bcuda(e, "multi-scene step");
            b.launches += 1;
        }
        cudaError_t e = qmpm::launch_clear_multi(b.d_clear + ph.clear_off, ph.n_clear, ph.virtual_blocks, b.n_sms,
                                                 b.stream);
        if (e == cudaSuccess && ph.virtual_blocks > 0) b.launches += 1;
        if (e == cudaSuccess) e = qmpm::launch_advance(b.d_ctr, (int)b.members.size(), b.stream);
        if (e != cudaSuccess) return bcuda(e, "multi-scene clear");
        b.launches += 1;
    }
    for (qmpm_ctx *c : b.members) {
        c->gcur = 1 - c->gcur;
        c->steps += 1;
    }
    for (int m : ph.resort) {
        qmpm::Ctx &c = *b.members[m];
        if (dry) {
            c.cur = 1 - c.cur;
            continue;
        }
        std::string err;
        const int rc = qmpm::resort(c, err);
        if (rc != QMPM_OK) return bfail(rc, err);
        b.launches += qmpm::resort_launches(c.key_bits);
    }
    b.phase = (k + 1) % period(b);
    b.steps += 1;
    return QMPM_OK;
}

// Capture both half periods as graphs, leaving the members' host state unchanged.  The
// capture starts from the current phase (a half-period boundary): its half first, then
// the other one from the state after it.
int capture(qmpm_batch &b)
{
    drop_graphs(b);
    const int half = period(b) / 2;
    std::vector<HostState> keep;
    for (qmpm_ctx *c : b.members) keep.push_back({c->gcur, c->cur, c->steps});
    const int64_t keep_launches = b.launches, keep_steps = b.steps;
    const int keep_phase = b.phase;
    int rc = QMPM_OK;
    for (int i = 0; i < 2 && rc == QMPM_OK; ++i) {
        const int h = (keep_phase / half + i) % 2;
        cudaError_t e = cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            rc = bcuda(e, "graph capture");
            break;
        }
        const int64_t before = b.launches;
        for (int k = h * half; k < (h + 1) * half && rc == QMPM_OK; ++k) rc = run_phase(b, k, false);
        b.graph_kernels[h] = b.launches - before;
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(b.stream, &g);
        if (rc == QMPM_OK && e != cudaSuccess) rc = bcuda(e, "graph capture");
        if (rc == QMPM_OK) {
            e = cudaGraphInstantiate(&b.graph[h], g, 0);
            if (e != cudaSuccess) rc = bcuda(e, "graph instantiate");
        }
        if (g) cudaGraphDestroy(g);
    }
    for (size_t m = 0; m < b.members.size(); ++m) {
        b.members[m]->gcur = keep[m].gcur;
        b.members[m]->cur = keep[m].cur;
        b.members[m]->steps = keep[m].steps;
    }
    b.launches = keep_launches;
    b.steps = keep_steps;
    b.phase = keep_phase;
    if (rc != QMPM_OK) drop_graphs(b);
    return rc;
}

// Kernels' one-time attributes must be set before a capture (they are not stream work).
int prepare_kernels(qmpm_batch &b)
{
    for (const Phase &ph : b.phases) {
        for (const Solo &so : ph.solos) {
            cudaError_t e = qmpm::launch_step_ctr(so.dim, so.material, so.quant, so.stats, nullptr, so.smem, b.n_sms,
                                                  b.stream);
            if (e != cudaSuccess) return bcuda(e, "batch member kernel setup");
        }
        for (const Group &g : ph.groups) {
            cudaError_t e = qmpm::launch_step_multi(g.dim, g.material, g.quant, g.stats, nullptr, 0, g.smem, b.n_sms,
                                                    b.stream);
            if (e != cudaSuccess) return bcuda(e, "multi-scene kernel setup");
        }
    }
    return QMPM_OK;
}

int ensure_plan(qmpm_batch &b)
{
    if (b.planned) return QMPM_OK;
    drop_graphs(b);
    cudaError_t e = grow(&b.d_ctr, &b.ctr_cap, std::max<size_t>(b.members.size(), 64));
    if (e != cudaSuccess) return bfail(QMPM_ERR_OOM, "batch counters: device allocation failed");
    int rc = plan(b);
    if (rc != QMPM_OK) return rc;
    return prepare_kernels(b);
}

}  // namespace

namespace qmpm {
void batch_invalidate(qmpm_batch *b)
{
    if (b) b->planned = false;
}
}  // namespace qmpm

extern "C" {

int qmpm_batch_create(void *stream, int32_t resort_every, int32_t flags, qmpm_batch_handle *out)
{
    if (!out || resort_every < 0 || resort_every > 1024) return bfail(QMPM_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    qmpm_batch *b = new (std::nothrow) qmpm_batch();
    if (!b) return bfail(QMPM_ERR_OOM, "host allocation failed");
    b->S = resort_every;
    b->flags = flags;
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return bcuda(e, "batch stream");
        }
        b->own_stream = true;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->n_sms, cudaDevAttrMultiProcessorCount, dev);
    if (b->n_sms <= 0) b->n_sms = 1;
    *out = b;
    return QMPM_OK;
}

int qmpm_batch_add(qmpm_batch_handle b, qmpm_handle h)
{
    if (!b || !h) return bfail(QMPM_ERR_INVALID_ARG, "bad batch or handle");
    if (h->batch) return bfail(QMPM_ERR_INVALID_ARG, "the scene already belongs to a batch");
    if ((int)b->members.size() >= qmpm::kMaxMembers) return bfail(QMPM_ERR_INVALID_ARG, "batch is full");
    if (!h->primed) return bfail(QMPM_ERR_INVALID_ARG, "the scene has no grid of its current state");
    // the batch stream starts after the scene's pending work
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, ev, 0);
    if (ev) cudaEventDestroy(ev);
    if (e != cudaSuccess) return bcuda(e, "batch join");
    b->saved.push_back({h->stream, h->scene.resort_every});
    h->stream = b->stream;
    h->scene.resort_every = b->S;
    h->batch = b;
    b->members.push_back(h);
    b->planned = false;
    return QMPM_OK;
}

int qmpm_batch_remove(qmpm_batch_handle b, qmpm_handle h)
{
    if (!b || !h || h->batch != b) return bfail(QMPM_ERR_INVALID_ARG, "the scene is not in this batch");
    auto it = std::find(b->members.begin(), b->members.end(), h);
    const size_t m = (size_t)(it - b->members.begin());
    const Saved sv = b->saved[m];
    // the scene's own stream continues after the batch's work
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sv.stream, ev, 0);
    if (ev) cudaEventDestroy(ev);
    h->stream = sv.stream;
    h->scene.resort_every = sv.resort_every;
    h->batch = nullptr;
    b->members.erase(it);
    b->saved.erase(b->saved.begin() + m);
    b->planned = false;
    if (e != cudaSuccess) return bcuda(e, "batch leave");
    return QMPM_OK;
}

int qmpm_batch_step(qmpm_batch_handle b, int32_t nsteps)
{
    if (!b || nsteps < 0) return bfail(QMPM_ERR_INVALID_ARG, "bad batch or nsteps");
    if (b->members.empty() || nsteps == 0) return QMPM_OK;
    for (qmpm_ctx *c : b->members)
        if (!c->primed) {
            const int r = qmpm_step(c, 0);  // P2G of a state uploaded since
            if (r != QMPM_OK) return r;
        }
    b->fresh = false;
    int rc = ensure_plan(*b);
    if (rc != QMPM_OK) return rc;
    const int half = period(*b) / 2;
    // graphs pay off once replayed: a membership that just changed steps with direct
    // launches, and is captured on a later call if it stays the same
    const bool graphs = (b->flags & QMPM_BATCH_GRAPHS) != 0 && !b->fresh;
    while (nsteps > 0) {
        if (graphs && b->phase % half == 0 && nsteps >= half) {
            if (!b->graph[0]) {
                rc = capture(*b);
                if (rc != QMPM_OK) return rc;
            }
            const int h = b->phase / half;
            cudaError_t e = cudaGraphLaunch(b->graph[h], b->stream);
            if (e != cudaSuccess) return bcuda(e, "graph launch");
            b->graph_launches += 1;
            b->launches += b->graph_kernels[h];
            for (int k = h * half; k < (h + 1) * half; ++k) {
                rc = run_phase(*b, k, true);
                if (rc != QMPM_OK) return rc;
            }
            nsteps -= half;
        } else {
            rc = run_phase(*b, b->phase, false);
            if (rc != QMPM_OK) return rc;
            nsteps -= 1;
        }
    }
    return QMPM_OK;
}

int qmpm_batch_info(qmpm_batch_handle b, qmpm_batch_info_t *out)
{
    if (!b || !out) return bfail(QMPM_ERR_INVALID_ARG, "bad batch or out");
    std::memset(out, 0, sizeof(*out));
    out->n_members = (int32_t)b->members.size();
    out->n_classes = b->planned && !b->phases.empty() ? (int32_t)b->phases[0].groups.size() : 0;
    out->n_solo = b->planned && !b->phases.empty() ? (int32_t)b->phases[0].solos.size() : 0;
    out->resort_every = b->S;
    out->steps = b->steps;
    out->kernel_launches = b->launches;
    out->graph_launches = b->graph_launches;
    for (qmpm_ctx *c : b->members) out->particles += c->N;
    return QMPM_OK;
}

int qmpm_batch_destroy(qmpm_batch_handle b)
{
    if (!b) return QMPM_OK;
    while (!b->members.empty()) qmpm_batch_remove(b, b->members.back());
    cudaStreamSynchronize(b->stream);
    drop_graphs(*b);
    for (auto &st : b->staging) {
        if (st.uploaded) cudaEventDestroy(st.uploaded);
        if (st.tab) cudaFreeHost(st.tab);
        if (st.clr) cudaFreeHost(st.clr);
        if (st.ctr) cudaFreeHost(st.ctr);
    }
    if (b->d_tab) cudaFree(b->d_tab);
    if (b->d_clear) cudaFree(b->d_clear);
    if (b->d_ctr) cudaFree(b->d_ctr);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return QMPM_OK;
}

}  // extern "C"
