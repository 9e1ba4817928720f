// Launch counting and optional per-kernel CUDA-event timing.
//
// Every kernel launch of the library goes through note_launch(), so a caller can
// ask how many of this library's kernels ran (cheb_launch_count). When timing is
// enabled (cheb_profile_enable), the step kernels are bracketed by CUDA events on
// their own stream; cheb_profile_read synchronises those events and reports the
// count and total device time per kernel kind.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/cheb_expmv.h"
#include "cheb_internal.h"

namespace cheb {

static std::atomic<long long> g_launches{0};
static std::atomic<bool> g_prof_on{false};
static std::mutex g_prof_mu;

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};
static std::vector<ProfRec> g_recs;
static std::vector<cudaEvent_t> g_pool;

void note_launch(int) { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long count) { g_launches.fetch_add(count, std::memory_order_relaxed); }
bool prof_enabled() { return g_prof_on.load(std::memory_order_relaxed); }

static cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

static std::atomic<bool> g_pdl_on{true};
bool pdl_enabled() { return g_pdl_on.load(std::memory_order_relaxed) && !g_prof_on.load(std::memory_order_relaxed); }
void pdl_set(bool on) { g_pdl_on.store(on, std::memory_order_relaxed); }

int prof_begin(int kind, cudaStream_t s) {
    if (!g_prof_on.load(std::memory_order_relaxed)) return -1;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfRec r{kind, take_event(), take_event()};
    if (!r.a || !r.b) return -1;
    cudaEventRecord(r.a, s);
    g_recs.push_back(r);
    return (int)g_recs.size() - 1;
}

void prof_end(int idx, cudaStream_t s) {
    if (idx < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (idx < (int)g_recs.size()) cudaEventRecord(g_recs[idx].b, s);
}

}  // namespace cheb

using namespace cheb;

extern "C" {

long long cheb_launch_count(void) { return g_launches.load(); }

cheb_status_t cheb_profile_enable(int on) {
    g_prof_on.store(on != 0);
    return CHEB_OK;
}

cheb_status_t cheb_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g_recs) {
        cudaEventSynchronize(r.b);
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    return CHEB_OK;
}

cheb_status_t cheb_profile_read(int kind, long long* count, double* total_ms) {
    if (!count || !total_ms) return CHEB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    long long c = 0;
    double ms = 0.0;
    for (auto& r : g_recs) {
        if (r.kind != kind) continue;
        if (cudaEventSynchronize(r.b) != cudaSuccess) return CHEB_ERR_CUDA;
        float x = 0.f;
        if (cudaEventElapsedTime(&x, r.a, r.b) != cudaSuccess) return CHEB_ERR_CUDA;
        ms += x;
        ++c;
    }
    *count = c;
    *total_ms = ms;
    return CHEB_OK;
}

}  // extern "C"

extern "C" cheb_status_t cheb_set_programmatic_launch(int on) {
    if (on != 0 && on != 1) return CHEB_ERR_INVALID_ARG;
    cheb::pdl_set(on != 0);
    return CHEB_OK;
}
