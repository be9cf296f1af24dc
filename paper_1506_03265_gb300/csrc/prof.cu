// Launch counters and CUDA-event timing per kernel class (see prof.cuh).
#include <atomic>
#include <mutex>
#include <vector>

#include "prof.cuh"

namespace cld {

namespace {

struct Pending {
    int cls;
    cudaEvent_t a, b;
};

std::mutex g_mu;
std::atomic<uint64_t> g_launches[K_NCLASS];
double g_ms[K_NCLASS];
double g_bytes[K_NCLASS];
std::atomic<uint32_t> g_timing_mask{0};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
thread_local cudaEvent_t t_open[K_NCLASS];

const char* kNames[K_NCLASS] = {"relax",     "snapshot",     "rebuild", "select", "finalize", "growable",
                                "radix_hist", "radix_scatter", "scan",    "csr",    "components", "quotient",
                                "floyd_warshall", "delta_stepping", "reduce", "misc",
                                "relax_pull"};

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void flush_locked(bool wait) {
    size_t keep = 0;
    for (size_t i = 0; i < g_pending.size(); ++i) {
        Pending& p = g_pending[i];
        if (wait) cudaEventSynchronize(p.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_ms[p.cls] += ms;
            g_pool.push_back(p.a);
            g_pool.push_back(p.b);
        } else {
            cudaGetLastError();
            g_pending[keep++] = p;
        }
    }
    g_pending.resize(keep);
}

}  // namespace

const char* kclass_name(int c) { return (c >= 0 && c < K_NCLASS) ? kNames[c] : "?"; }

void prof_begin(int cls, cudaStream_t s) {
    g_launches[cls].fetch_add(1, std::memory_order_relaxed);
    if (g_timing_mask.load(std::memory_order_relaxed) & (1u << cls)) {
        std::lock_guard<std::mutex> lk(g_mu);
        cudaEvent_t e = take_event();
        cudaEventRecord(e, s);
        t_open[cls] = e;
    } else {
        t_open[cls] = nullptr;
    }
}

void prof_end(int cls, cudaStream_t s) {
    if (!t_open[cls]) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t e = take_event();
    cudaEventRecord(e, s);
    g_pending.push_back({cls, t_open[cls], e});
    t_open[cls] = nullptr;
    if (g_pending.size() > 4096) flush_locked(true);
}

void prof_add_bytes(int cls, double bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_bytes[cls] += bytes;
}

void prof_flush() {
    std::lock_guard<std::mutex> lk(g_mu);
    flush_locked(false);
}

}  // namespace cld

using namespace cld;

extern "C" {

cldiam_status cldiam_profile_set_timing(uint32_t class_mask) {
    g_timing_mask.store(class_mask);
    return CLDIAM_OK;
}

cldiam_status cldiam_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    flush_locked(true);
    for (int i = 0; i < K_NCLASS; ++i) {
        g_launches[i].store(0);
        g_ms[i] = 0.0;
        g_bytes[i] = 0.0;
    }
    return CLDIAM_OK;
}

uint32_t cldiam_profile_num_classes(void) { return (uint32_t)K_NCLASS; }

cldiam_status cldiam_profile_get(uint32_t cls, const char** name, uint64_t* launches, double* ms, double* bytes) {
    if (cls >= (uint32_t)K_NCLASS) return fail(CLDIAM_ERR_INVALID_ARG, "kernel class out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    flush_locked(true);
    if (name) *name = kNames[cls];
    if (launches) *launches = g_launches[cls].load();
    if (ms) *ms = g_ms[cls];
    if (bytes) *bytes = g_bytes[cls];
    return CLDIAM_OK;
}

}  // extern "C"
