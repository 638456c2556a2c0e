// fault.cpp -- host-side fault injection of libqmpm (qmpm_fault_*): makes the library's
// error paths (a failed device or host allocation, an expired bounded wait) reachable in
// tests without faulting a GPU.  Each kind keeps a count of occurrences to let pass and a
// count to fail; the check on the hot paths is one relaxed atomic load while nothing is armed.
#include <atomic>
#include <mutex>

#include "qmpm_internal.h"

namespace {

struct Slot {
    int64_t skip = 0, fail = 0, hits = 0;
};

std::mutex g_mu;
Slot g_slot[QMPM_FAULT_KINDS];
std::atomic<int> g_armed{0};  // kinds with fail > 0

}  // namespace

namespace qmpm {

bool fault_hit(int kind)
{
    if (kind < 0 || kind >= QMPM_FAULT_KINDS || g_armed.load(std::memory_order_relaxed) == 0) return false;
    std::lock_guard<std::mutex> lk(g_mu);
    Slot &s = g_slot[kind];
    if (s.fail <= 0) return false;
    if (s.skip > 0) {
        --s.skip;
        return false;
    }
    --s.fail;
    ++s.hits;
    if (s.fail == 0) g_armed.fetch_sub(1, std::memory_order_relaxed);
    return true;
}

}  // namespace qmpm

extern "C" {

int qmpm_fault_inject(int32_t kind, int64_t after, int64_t count)
{
    if (kind < 0 || kind >= QMPM_FAULT_KINDS || after < 0 || count < 0) {
        qmpm::set_last_error("qmpm_fault_inject: unknown kind or negative count");
        return QMPM_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    Slot &s = g_slot[kind];
    const bool was = s.fail > 0, now = count > 0;
    s.skip = after;
    s.fail = count;
    if (now && !was) g_armed.fetch_add(1, std::memory_order_relaxed);
    if (!now && was) g_armed.fetch_sub(1, std::memory_order_relaxed);
    return QMPM_OK;
}

int qmpm_fault_hits(int32_t kind, int64_t *hits)
{
    if (kind < 0 || kind >= QMPM_FAULT_KINDS || !hits) {
        qmpm::set_last_error("qmpm_fault_hits: unknown kind or NULL out");
        return QMPM_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    *hits = g_slot[kind].hits;
    return QMPM_OK;
}

int qmpm_fault_clear(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (Slot &s : g_slot) s = Slot();
    g_armed.store(0, std::memory_order_relaxed);
    return QMPM_OK;
}

}  // extern "C"
