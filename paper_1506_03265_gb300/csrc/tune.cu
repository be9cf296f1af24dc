// Tuning knobs and the autotuner.  No counterpart in the paper: the knobs are
// launch shapes and cut-overs between forms of one step that compute the same
// integers (the pushed or the dense pull form of a growing step, dense matrix
// or radix-sort de-duplication of the quotient, Floyd-Warshall or batched
// SSSP for its diameter, sources per CTA, Delta-stepping's bucket width, the
// many-graph kernel's shared-memory Floyd-Warshall cut-over), so a choice only
// changes the time.
//
// Effective value of a knob for one call: the process-wide setting if it is
// non-zero, else the autotuner's cached choice for this device and the call's
// size class (floor(log2) of its adjacency entries), else the library default.
//
// The autotuner times the caller's own work (CUDA events on the work's
// stream, median of `reps` runs) for each candidate value of one knob at a
// time (coordinate descent over fixed candidate lists), keeps a change only
// when it is at least 2 % faster, and checks that every candidate gives the
// same result as the starting point (a candidate that does not is a library
// fault: the search stops with DIVERGED).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace cld {

namespace {

std::mutex g_tmu;
cldiam_tuning g_tuning{};                                  // zero = not set
std::map<std::pair<int, uint32_t>, cldiam_tuning> g_cache;  // (device, size class) -> tuned knobs
bool g_measuring = false;  // the autotuner is timing a candidate: the process-wide knobs are the whole setting

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return dev;
}

// take every knob of `from` that is unset (0) in `into`
void merge_unset(cldiam_tuning& into, const cldiam_tuning& from) {
    if (into.pull_ratio == 0.f) into.pull_ratio = from.pull_ratio;
    if (into.relax_ctas_per_sm == 0) into.relax_ctas_per_sm = from.relax_ctas_per_sm;
    if (into.dense_quotient_k == 0) into.dense_quotient_k = from.dense_quotient_k;
    if (into.apsp_sources_per_cta == 0) into.apsp_sources_per_cta = from.apsp_sources_per_cta;
    if (into.apsp_fw_density == 0) into.apsp_fw_density = from.apsp_fw_density;
    if (into.batch_fw_k == 0) into.batch_fw_k = from.batch_fw_k;
    if (into.sssp_delta_scale == 0.f) into.sssp_delta_scale = from.sssp_delta_scale;
    if (into.batch_split == 0) into.batch_split = from.batch_split;
}

// Candidate values of each knob (bit i of a knob mask = knob i).
struct Knob {
    const char* name;
    std::vector<double> values;
};
const std::vector<Knob>& knob_table() {
    static const std::vector<Knob> t = {
        {"pull_ratio", {-1.0, 0.15, 0.3, 0.5, 0.8}},
        {"relax_ctas_per_sm", {0, 2, 4}},
        {"dense_quotient_k", {1024, 4096, 8192}},
        {"apsp_sources_per_cta", {0, 1, 4, 8}},
        {"apsp_fw_density", {4, 8, 16}},
        {"batch_fw_k", {64, 128, 200}},
        {"sssp_delta_scale", {1, 2, 4, 8}},
        {"batch_split", {1, 2}},
    };
    return t;
}

double knob_get(const cldiam_tuning& t, size_t i) {
    switch (i) {
        case 0: return t.pull_ratio;
        case 1: return t.relax_ctas_per_sm;
        case 2: return t.dense_quotient_k;
        case 3: return t.apsp_sources_per_cta;
        case 4: return t.apsp_fw_density;
        case 5: return t.batch_fw_k;
        case 6: return t.sssp_delta_scale;
        default: return t.batch_split;
    }
}
void knob_set(cldiam_tuning& t, size_t i, double v) {
    switch (i) {
        case 0: t.pull_ratio = (float)v; break;
        case 1: t.relax_ctas_per_sm = (uint32_t)v; break;
        case 2: t.dense_quotient_k = (uint32_t)v; break;
        case 3: t.apsp_sources_per_cta = (uint32_t)v; break;
        case 4: t.apsp_fw_density = (uint32_t)v; break;
        case 5: t.batch_fw_k = (uint32_t)v; break;
        case 6: t.sssp_delta_scale = (float)v; break;
        default: t.batch_split = (uint32_t)v; break;
    }
}

uint64_t fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

}  // namespace

cldiam_tuning tuning_defaults_filled(const cldiam_tuning& t) {
    cldiam_tuning r = t;
    if (r.pull_ratio == 0.f) r.pull_ratio = 0.3f;  // < 0 stays: never
    if (r.dense_quotient_k == 0) r.dense_quotient_k = 4096;
    if (r.apsp_fw_density == 0) r.apsp_fw_density = 8;
    if (r.batch_fw_k == 0) r.batch_fw_k = 200;
    if (r.sssp_delta_scale == 0.f) r.sssp_delta_scale = 1.f;
    if (r.batch_split == 0) r.batch_split = 2;
    return r;
}

cldiam_status tuning_check(const cldiam_tuning& t) {
    if (!(t.pull_ratio == t.pull_ratio)) return fail(CLDIAM_ERR_INVALID_ARG, "pull_ratio is NaN");
    if (t.relax_ctas_per_sm > 64) return fail(CLDIAM_ERR_INVALID_ARG, "relax_ctas_per_sm > 64");
    if (t.dense_quotient_k > 65535) return fail(CLDIAM_ERR_INVALID_ARG, "dense_quotient_k > 65535");
    if (t.apsp_sources_per_cta != 0 && t.apsp_sources_per_cta != 1 && t.apsp_sources_per_cta != 4 &&
        t.apsp_sources_per_cta != 8)
        return fail(CLDIAM_ERR_INVALID_ARG, "apsp_sources_per_cta must be 0, 1, 4 or 8");
    if (t.apsp_fw_density > 1024) return fail(CLDIAM_ERR_INVALID_ARG, "apsp_fw_density > 1024");
    if (t.batch_fw_k > 200) return fail(CLDIAM_ERR_INVALID_ARG, "batch_fw_k > 200");
    if (!(t.sssp_delta_scale == 0.f || t.sssp_delta_scale >= 1.f) || !(t.sssp_delta_scale < 1e9f))
        return fail(CLDIAM_ERR_INVALID_ARG, "sssp_delta_scale must be 0 or in [1, 1e9)");
    if (t.batch_split > 2) return fail(CLDIAM_ERR_INVALID_ARG, "batch_split must be 0, 1 or 2");
    for (uint32_t r : t.reserved)
        if (r) return fail(CLDIAM_ERR_INVALID_ARG, "reserved tuning fields must be 0");
    return CLDIAM_OK;
}

uint32_t size_class(uint64_t entries) {
    uint32_t c = 0;
    while (c < 63 && (entries >> (c + 1)) != 0) ++c;
    return c;
}

cldiam_tuning tuning_effective(int device, uint32_t cls) {
    std::lock_guard<std::mutex> lk(g_tmu);
    cldiam_tuning t = g_tuning;
    const auto it = g_measuring ? g_cache.end() : g_cache.find({device, cls});
    if (it != g_cache.end()) merge_unset(t, it->second);
    return tuning_defaults_filled(t);
}

cldiam_tuning tuning_for(uint64_t entries) { return tuning_effective(current_device(), size_class(entries)); }

cldiam_tuning tuning_for_batch(uint64_t entries) {
    return tuning_effective(current_device(), 64u + size_class(entries));
}

cldiam_tuning tuning_current() {
    std::lock_guard<std::mutex> lk(g_tmu);
    return tuning_defaults_filled(g_tuning);
}

namespace {

// Coordinate descent over the knobs in `mask`, from `start` (unset knobs take their defaults).
cldiam_status search(const cldiam_tuning& start, uint32_t mask, cldiam_tune_measure_fn fn, void* user,
                     cldiam_tuning* best, double* best_seconds) {
    if (!fn || !best) return fail(CLDIAM_ERR_INVALID_ARG, "NULL measure function or best");
    const auto& table = knob_table();
    if (mask == 0 || (mask >> table.size()) != 0) return fail(CLDIAM_ERR_INVALID_ARG, "knob mask out of range");
    CLD_TRY(tuning_check(start));
    cldiam_tuning cur = tuning_defaults_filled(start);
    double cur_t = 0.0;
    uint64_t ref = 0;
    CLD_TRY(fn(&cur, user, &cur_t, &ref));
    static const size_t order[] = {0, 1, 2, 3, 4, 5, 6, 7};
    static_assert(sizeof(order) / sizeof(order[0]) == 8, "one entry per knob");
    for (size_t i : order) {
        if (!(mask & (1u << i))) continue;
        const float at_start = (float)knob_get(cur, i);  // measured already (as part of cur)
        for (double v : table[i].values) {
            if ((float)v == at_start || (float)v == (float)knob_get(cur, i)) continue;  // floats or integers
            cldiam_tuning cand = cur;
            knob_set(cand, i, v);
            double t = 0.0;
            uint64_t h = 0;
            const cldiam_status st = fn(&cand, user, &t, &h);
            if (st != CLDIAM_OK) continue;  // a candidate the work cannot use (e.g. out of memory)
            if (h != ref) {
                char buf[160];
                snprintf(buf, sizeof buf, "tuning knob %s = %g changed the result (a library fault)", table[i].name, v);
                return fail(CLDIAM_ERR_DIVERGED, buf);
            }
            if (t < cur_t * 0.98) {
                cur = cand;
                cur_t = t;
            }
        }
    }
    *best = cur;
    if (best_seconds) *best_seconds = cur_t;
    return CLDIAM_OK;
}

// Set the process-wide knobs for the duration of one measurement, restoring them afterwards.
struct TuningScope {
    cldiam_tuning saved;
    explicit TuningScope(const cldiam_tuning& t) {
        std::lock_guard<std::mutex> lk(g_tmu);
        saved = g_tuning;
        g_tuning = t;
        g_measuring = true;
    }
    ~TuningScope() {
        std::lock_guard<std::mutex> lk(g_tmu);
        g_tuning = saved;
        g_measuring = false;
    }
};

template <class F>
cldiam_status time_median(cudaStream_t s, uint32_t reps, F&& work, double* seconds) {
    std::vector<float> ms;
    cudaEvent_t a = nullptr, b = nullptr;
    CLD_CUDA(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return cuda_fail(cudaGetLastError(), "cudaEventCreate", __FILE__, __LINE__);
    }
    cldiam_status st = CLDIAM_OK;
    for (uint32_t r = 0; r < reps && st == CLDIAM_OK; ++r) {
        cudaEventRecord(a, s);
        st = work();
        cudaEventRecord(b, s);
        if (st == CLDIAM_OK && cudaEventSynchronize(b) == cudaSuccess) {
            float x = 0.f;
            cudaEventElapsedTime(&x, a, b);
            ms.push_back(x);
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != CLDIAM_OK) return st;
    if (ms.empty()) return cuda_fail(cudaGetLastError(), "timing", __FILE__, __LINE__);
    std::sort(ms.begin(), ms.end());
    *seconds = ms[ms.size() / 2] * 1e-3;
    return CLDIAM_OK;
}

uint64_t result_hash(const cldiam_result* r, size_t count, uint64_t h = 1469598103934665603ull) {
    return fnv1a(r, sizeof(cldiam_result) * count, h);
}

struct GraphWork {
    cldiam_graph* g;
    double tau;
    uint64_t seed;
    cldiam_opts opts;
    uint32_t reps;
};

cldiam_status measure_graph(const cldiam_tuning* t, void* user, double* seconds, uint64_t* hash) {
    GraphWork* w = static_cast<GraphWork*>(user);
    TuningScope scope(*t);
    cldiam_result res{};
    auto work = [&]() -> cldiam_status {
        cldiam_clustering* c = nullptr;
        CLD_TRY(cluster(w->g, w->tau, w->seed, &w->opts, &c));
        cldiam_quotient* q = nullptr;
        cldiam_status st = quotient(c, &q);
        if (st == CLDIAM_OK) st = cldiam_estimate(q, &res);
        free_quotient(q);
        free_clustering(c);
        return st;
    };
    CLD_TRY(work());  // warm-up
    CLD_TRY(time_median(w->g->stream, w->reps, work, seconds));
    *hash = result_hash(&res, 1);
    return CLDIAM_OK;
}

struct BatchWork {
    cldiam_arena* a;
    const uint32_t* ids;
    const double* tau;
    const uint64_t* seed;
    uint32_t count;
    cldiam_opts opts;
    uint32_t reps;
    cudaStream_t s;
};

cldiam_status measure_batch(const cldiam_tuning* t, void* user, double* seconds, uint64_t* hash) {
    BatchWork* w = static_cast<BatchWork*>(user);
    TuningScope scope(*t);
    std::vector<cldiam_result> out(w->count);
    std::vector<cldiam_status> sts(w->count);
    auto work = [&]() -> cldiam_status {
        return batch_run(w->a, w->ids, w->tau, w->seed, w->count, &w->opts, out.data(), sts.data());
    };
    CLD_TRY(work());
    CLD_TRY(time_median(w->s, w->reps, work, seconds));
    *hash = fnv1a(sts.data(), sts.size() * sizeof(cldiam_status), result_hash(out.data(), out.size()));
    return CLDIAM_OK;
}

struct SsspWork {
    cldiam_graph* g;
    uint32_t source;
    uint32_t reps;
};

cldiam_status measure_sssp(const cldiam_tuning* t, void* user, double* seconds, uint64_t* hash) {
    SsspWork* w = static_cast<SsspWork*>(user);
    TuningScope scope(*t);
    std::vector<uint32_t> dist(w->g->n);
    uint64_t ecc = 0;
    auto work = [&]() -> cldiam_status { return sssp_delta(w->g, w->source, 0, nullptr, &ecc, nullptr, nullptr); };
    CLD_TRY(work());
    CLD_TRY(time_median(w->g->stream, w->reps, work, seconds));
    CLD_TRY(sssp_delta(w->g, w->source, 0, dist.data(), &ecc, nullptr, nullptr));
    *hash = fnv1a(dist.data(), dist.size() * 4, ecc);
    return CLDIAM_OK;
}

void cache_put(int device, uint32_t cls, const cldiam_tuning& t, uint32_t mask) {
    // only the searched knobs are cached; the others stay unset (0) so they keep their own source
    cldiam_tuning c{};
    for (size_t i = 0; i < knob_table().size(); ++i)
        if (mask & (1u << i)) knob_set(c, i, knob_get(t, i));
    std::lock_guard<std::mutex> lk(g_tmu);
    auto& slot = g_cache[{device, cls}];
    cldiam_tuning merged = c;
    merge_unset(merged, slot);
    slot = merged;
}

constexpr uint32_t kGraphKnobs = (1u << 0) | (1u << 1) | (1u << 2) | (1u << 3) | (1u << 4);
constexpr uint32_t kBatchKnobs = (1u << 7) | (1u << 5);
constexpr uint32_t kSsspKnobs = 1u << 6;

cldiam_tuning start_point() {
    std::lock_guard<std::mutex> lk(g_tmu);
    return g_tuning;
}

}  // namespace

}  // namespace cld

using namespace cld;

extern "C" {

cldiam_status cldiam_tuning_get(cldiam_tuning* out) {
    if (!out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL out");
    *out = tuning_current();
    return CLDIAM_OK;
}

cldiam_status cldiam_tuning_set(const cldiam_tuning* t) {
    cldiam_tuning v{};
    if (t) {
        CLD_TRY(tuning_check(*t));
        v = *t;
    }
    std::lock_guard<std::mutex> lk(g_tmu);
    g_tuning = v;
    return CLDIAM_OK;
}

uint32_t cldiam_size_class(uint64_t entries) { return size_class(entries); }

cldiam_status cldiam_tuning_effective(int32_t device, uint32_t size_class, cldiam_tuning* out) {
    if (!out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL out");
    *out = tuning_effective(device, size_class);
    return CLDIAM_OK;
}

cldiam_status cldiam_tuning_cache_put(int32_t device, uint32_t size_class, const cldiam_tuning* t) {
    if (!t) return fail(CLDIAM_ERR_INVALID_ARG, "NULL tuning");
    CLD_TRY(tuning_check(*t));
    std::lock_guard<std::mutex> lk(g_tmu);
    g_cache[{device, size_class}] = *t;
    return CLDIAM_OK;
}

cldiam_status cldiam_tuning_cache_get(int32_t device, uint32_t size_class, cldiam_tuning* out) {
    if (!out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL out");
    std::lock_guard<std::mutex> lk(g_tmu);
    const auto it = g_cache.find({device, size_class});
    if (it == g_cache.end()) return fail(CLDIAM_ERR_INVALID_ARG, "no cached tuning for this device and size class");
    *out = it->second;
    return CLDIAM_OK;
}

void cldiam_tuning_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_cache.clear();
}

cldiam_status cldiam_tuning_cache_save(const char* path) {
    if (!path) return fail(CLDIAM_ERR_INVALID_ARG, "NULL path");
    FILE* f = fopen(path, "w");
    if (!f) return fail(CLDIAM_ERR_INVALID_ARG, std::string("cannot write ") + path);
    std::lock_guard<std::mutex> lk(g_tmu);
    fprintf(f, "# cldiam tuning cache: device size_class");
    for (const auto& k : knob_table()) fprintf(f, " %s", k.name);
    fprintf(f, "\n");
    for (const auto& e : g_cache) {
        fprintf(f, "%d %u", e.first.first, e.first.second);
        for (size_t i = 0; i < knob_table().size(); ++i) fprintf(f, " %.9g", knob_get(e.second, i));
        fprintf(f, "\n");
    }
    const bool ok = fclose(f) == 0;
    return ok ? CLDIAM_OK : fail(CLDIAM_ERR_INVALID_ARG, std::string("cannot write ") + path);
}

cldiam_status cldiam_tuning_cache_load(const char* path) {
    if (!path) return fail(CLDIAM_ERR_INVALID_ARG, "NULL path");
    FILE* f = fopen(path, "r");
    if (!f) return fail(CLDIAM_ERR_INVALID_ARG, std::string("cannot read ") + path);
    std::vector<std::pair<std::pair<int, uint32_t>, cldiam_tuning>> rows;
    char line[512];
    cldiam_status st = CLDIAM_OK;
    while (st == CLDIAM_OK && fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        int dev = 0;
        unsigned cls = 0;
        double v[8];
        if (sscanf(line, "%d %u %lf %lf %lf %lf %lf %lf %lf %lf", &dev, &cls, &v[0], &v[1], &v[2], &v[3], &v[4], &v[5],
                   &v[6], &v[7]) != 10) {
            st = fail(CLDIAM_ERR_INVALID_ARG, "malformed tuning cache line");
            break;
        }
        cldiam_tuning t{};
        static_assert(sizeof(v) / sizeof(v[0]) == 8, "one column per knob");
        for (size_t i = 0; i < 8; ++i) knob_set(t, i, v[i]);
        st = tuning_check(t);
        if (st == CLDIAM_OK) rows.push_back({{dev, cls}, t});
    }
    fclose(f);
    if (st != CLDIAM_OK) return st;
    std::lock_guard<std::mutex> lk(g_tmu);
    for (const auto& r : rows) g_cache[r.first] = r.second;
    return CLDIAM_OK;
}

cldiam_status cldiam_autotune_search(const cldiam_tuning* start, uint32_t knob_mask, cldiam_tune_measure_fn measure,
                                     void* user, cldiam_tuning* best, double* best_seconds) {
    cldiam_tuning s0{};
    if (start) s0 = *start;
    return search(s0, knob_mask, measure, user, best, best_seconds);
}

cldiam_status cldiam_autotune_graph(cldiam_graph* g, double tau, uint64_t seed, const cldiam_opts* opts,
                                    uint32_t reps, cldiam_tuning* out) {
    if (!g || !out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL graph or out");
    GraphWork w{g, tau, seed, opts ? *opts : cldiam_opts{}, reps ? reps : 3u};
    cldiam_tuning best{};
    CLD_TRY(search(start_point(), kGraphKnobs, measure_graph, &w, &best, nullptr));
    cache_put(current_device(), size_class(g->nnz), best, kGraphKnobs);
    *out = best;
    return CLDIAM_OK;
}

cldiam_status cldiam_autotune_batch(cldiam_arena* a, const uint32_t* ids, const double* tau, const uint64_t* seed,
                                    uint32_t count, const cldiam_opts* opts, uint32_t reps, cldiam_tuning* out) {
    if (!a || !out || !count || !ids || !tau || !seed) return fail(CLDIAM_ERR_INVALID_ARG, "NULL argument");
    uint64_t entries = 0;
    for (uint32_t i = 0; i < count; ++i) {
        cldiam_graph* view = nullptr;
        CLD_TRY(arena_graph(a, ids[i], &view));
        entries += view->nnz;
        free_graph(view);
    }
    BatchWork w{a, ids, tau, seed, count, opts ? *opts : cldiam_opts{}, reps ? reps : 3u, arena_stream(a)};
    cldiam_tuning best{};
    CLD_TRY(search(start_point(), kBatchKnobs, measure_batch, &w, &best, nullptr));
    cache_put(current_device(), 64u + size_class(entries), best, kBatchKnobs);
    *out = best;
    return CLDIAM_OK;
}

cldiam_status cldiam_autotune_sssp(cldiam_graph* g, uint32_t source, uint32_t reps, cldiam_tuning* out) {
    if (!g || !out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL graph or out");
    if (source >= g->n) return fail(CLDIAM_ERR_INVALID_ARG, "source >= n");
    SsspWork w{g, source, reps ? reps : 3u};
    cldiam_tuning best{};
    CLD_TRY(search(start_point(), kSsspKnobs, measure_sssp, &w, &best, nullptr));
    cache_put(current_device(), size_class(g->nnz), best, kSsspKnobs);
    *out = best;
    return CLDIAM_OK;
}

}  // extern "C"
