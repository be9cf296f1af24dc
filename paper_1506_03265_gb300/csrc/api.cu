// extern "C" entry points of include/cldiam.h: argument checks, stream and
// pointer plumbing, and translation of internal failures into status codes.
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>

#include "internal.cuh"

namespace cld {

const char* last_error_cstr();

cudaStream_t resolve_stream(void* user_stream) {
    if (user_stream) return static_cast<cudaStream_t>(user_stream);
    static std::mutex mu;
    static cudaStream_t streams[64];
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!streams[dev]) cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    return streams[dev];
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cldiam_status to_device(const void* src, size_t bytes, cudaStream_t s, void** dev, bool* owned) {
    *owned = false;
    *dev = nullptr;
    if (bytes == 0 || !src) return CLDIAM_OK;
    if (is_device_ptr(src)) {
        *dev = const_cast<void*>(src);
        return CLDIAM_OK;
    }
    CLD_TRY(dmalloc(dev, bytes, s));
    *owned = true;
    cudaError_t e = cudaMemcpyAsync(*dev, src, bytes, cudaMemcpyDefault, s);
    if (e != cudaSuccess) {
        dfree(*dev, s);
        *dev = nullptr;
        *owned = false;
        return cuda_fail(e, "cudaMemcpyAsync(input)", __FILE__, __LINE__);
    }
    return CLDIAM_OK;
}

static cldiam_status copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (!dst || bytes == 0) return CLDIAM_OK;
    CLD_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
    return CLDIAM_OK;
}

// Run f() and turn a stray C++ exception into a status (none may cross the ABI).
template <class F>
static cldiam_status guarded(F&& f) {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return fail(CLDIAM_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(CLDIAM_ERR_CUDA, "internal error");
    }
}

}  // namespace cld

using namespace cld;

extern "C" {

const char* cldiam_status_string(cldiam_status s) {
    switch (s) {
        case CLDIAM_OK: return "ok";
        case CLDIAM_ERR_INVALID_ARG: return "invalid argument";
        case CLDIAM_ERR_OOM: return "out of memory";
        case CLDIAM_ERR_OVERFLOW: return "distance overflow";
        case CLDIAM_ERR_TIMEOUT: return "device wait timed out";
        case CLDIAM_ERR_CUDA: return "CUDA error";
        case CLDIAM_ERR_BUSY: return "busy";
        case CLDIAM_ERR_CANCELLED: return "cancelled";
        case CLDIAM_ERR_DIVERGED: return "stage limit exceeded";
        case CLDIAM_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

const char* cldiam_last_error(void) { return last_error_cstr(); }


cldiam_status cldiam_version(int32_t* major, int32_t* minor) {
    if (major) *major = 1;
    if (minor) *minor = 0;
    return CLDIAM_OK;
}

cldiam_status cldiam_build_csr(const uint32_t* src, const uint32_t* dst, const uint32_t* w, uint64_t m, uint32_t n,
                               uint32_t flags, void* stream, cldiam_graph** out) {
    return guarded([&] { return build_csr(src, dst, w, m, n, flags, resolve_stream(stream), out); });
}

cldiam_status cldiam_graph_info(const cldiam_graph* g, uint32_t* n, uint64_t* nnz) {
    if (!g) return fail(CLDIAM_ERR_INVALID_ARG, "NULL graph");
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    return CLDIAM_OK;
}

cldiam_status cldiam_graph_copy(const cldiam_graph* g, uint64_t* off, uint32_t* col, uint32_t* w, uint32_t* orig) {
    if (!g) return fail(CLDIAM_ERR_INVALID_ARG, "NULL graph");
    return guarded([&]() -> cldiam_status {
        cudaStream_t s = g->stream;
        CLD_TRY(copy_out(off, g->off, ((size_t)g->n + 1) * 8, s));
        CLD_TRY(copy_out(orig, g->orig, (size_t)g->n * 4, s));
        if ((col || w) && g->nnz) {
            // adjacency is interleaved (col, w); split it with 2D copies
            if (col) CLD_CUDA(cudaMemcpy2DAsync(col, 4, g->adj, 8, 4, g->nnz, cudaMemcpyDefault, s));
            if (w) CLD_CUDA(cudaMemcpy2DAsync(w, 4, reinterpret_cast<const char*>(g->adj) + 4, 8, 4, g->nnz,
                                              cudaMemcpyDefault, s));
        }
        CLD_CUDA(cudaStreamSynchronize(s));
        return CLDIAM_OK;
    });
}

void cldiam_graph_free(cldiam_graph* g) { free_graph(g); }

cldiam_status cldiam_delta0(const cldiam_graph* g, int32_t mode, uint32_t* out) {
    if (!g || !out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL graph or out");
    if (mode != CLDIAM_DELTA0_AVG && mode != CLDIAM_DELTA0_MIN) return fail(CLDIAM_ERR_INVALID_ARG, "mode");
    return delta0(g, mode, 0, out);
}

cldiam_status cldiam_cluster(cldiam_graph* g, double tau, uint64_t seed, const cldiam_opts* opts,
                             cldiam_clustering** out) {
    return guarded([&] { return cluster(g, tau, seed, opts, out); });
}

cldiam_status cldiam_cluster2(cldiam_graph* g, double tau, uint64_t seed, const cldiam_opts* opts,
                              cldiam_clustering** out) {
    return guarded([&] { return cluster2(g, tau, seed, opts, out); });
}

cldiam_status cldiam_clustering_info(const cldiam_clustering* c, cldiam_result* out) {
    if (!c || !out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL clustering or out");
    *out = c->stats;
    return CLDIAM_OK;
}

cldiam_status cldiam_clustering_copy(const cldiam_clustering* c, uint32_t* center, uint32_t* D, uint32_t* cid) {
    if (!c) return fail(CLDIAM_ERR_INVALID_ARG, "NULL clustering");
    return guarded([&]() -> cldiam_status {
        cudaStream_t s = c->g->stream;
        size_t b = (size_t)c->g->n * 4;
        CLD_TRY(copy_out(center, c->center, b, s));
        CLD_TRY(copy_out(D, c->D, b, s));
        CLD_TRY(copy_out(cid, c->cid, b, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        return CLDIAM_OK;
    });
}

void cldiam_clustering_free(cldiam_clustering* c) { free_clustering(c); }

cldiam_status cldiam_quotient_build(const cldiam_clustering* c, cldiam_quotient** out) {
    return guarded([&] { return quotient(c, out); });
}

cldiam_status cldiam_quotient_info(const cldiam_quotient* q, uint32_t* k, uint64_t* nnz) {
    if (!q) return fail(CLDIAM_ERR_INVALID_ARG, "NULL quotient");
    if (k) *k = q->k;
    if (nnz) *nnz = q->nnz;
    return CLDIAM_OK;
}

cldiam_status cldiam_quotient_copy(const cldiam_quotient* q, uint64_t* off, uint32_t* col, uint32_t* w) {
    if (!q) return fail(CLDIAM_ERR_INVALID_ARG, "NULL quotient");
    return guarded([&]() -> cldiam_status {
        cudaStream_t s = q->stream;
        CLD_TRY(copy_out(off, q->off, ((size_t)q->k + 1) * 8, s));
        CLD_TRY(copy_out(col, q->col, q->nnz * 4, s));
        CLD_TRY(copy_out(w, q->w, q->nnz * 4, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        return CLDIAM_OK;
    });
}

void cldiam_quotient_free(cldiam_quotient* q) { free_quotient(q); }

cldiam_status cldiam_estimate(const cldiam_quotient* q, cldiam_result* out) {
    if (!q || !out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL quotient or out");
    return guarded([&]() -> cldiam_status {
        const cldiam_clustering* c = q->c;
        cldiam_result r = c->stats;
        uint64_t phi = 0;
        CLD_TRY(apsp_max_device(q->k, q->off, q->col, q->w, q->nnz, q->stream, &phi, false, q->max_fw_k,
                                tuning_for(q->c->g->nnz)));
        DBuf<uint32_t> rmax;
        CLD_TRY(rmax.alloc(1, q->stream));
        CLD_TRY(reduce_max_u32(c->D, c->g->n, rmax.get(), q->stream));
        uint32_t R = 0;
        CLD_CUDA(cudaMemcpyAsync(&R, rmax.get(), 4, cudaMemcpyDeviceToHost, q->stream));
        CLD_CUDA(cudaStreamSynchronize(q->stream));
        r.phi_gc = phi;
        r.radius = R;
        r.phi_approx = phi + 2ull * R;
        r.quotient_edges = q->nnz;
        *out = r;
        return CLDIAM_OK;
    });
}

cldiam_status cldiam_apsp_max(uint32_t k, const uint64_t* off, const uint32_t* col, const uint32_t* w, void* stream,
                              uint64_t* phi) {
    if (!phi || (k > 0 && !off)) return fail(CLDIAM_ERR_INVALID_ARG, "NULL argument");
    return guarded([&]() -> cldiam_status {
        cudaStream_t s = resolve_stream(stream);
        if (k == 0) {
            *phi = 0;
            return CLDIAM_OK;
        }
        uint64_t nnz = 0;
        CLD_CUDA(cudaMemcpyAsync(&nnz, off + k, 8, cudaMemcpyDefault, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        void *doff, *dcol = nullptr, *dw = nullptr;
        bool o1, o2 = false, o3 = false;
        CLD_TRY(to_device(off, ((size_t)k + 1) * 8, s, &doff, &o1));
        cldiam_status st = CLDIAM_OK;
        if (nnz) {
            st = to_device(col, nnz * 4, s, &dcol, &o2);
            if (st == CLDIAM_OK) st = to_device(w, nnz * 4, s, &dw, &o3);
        }
        if (st == CLDIAM_OK)
            st = apsp_max_device(k, (const uint64_t*)doff, (const uint32_t*)dcol, (const uint32_t*)dw, nnz, s, phi, true,
                                 8192u, tuning_for(nnz));
        if (o1) dfree(doff, s);
        if (o2) dfree(dcol, s);
        if (o3) dfree(dw, s);
        cudaStreamSynchronize(s);
        return st;
    });
}

cldiam_status cldiam_apsp_max_noalloc(uint32_t k, const uint64_t* off, const uint32_t* col, const uint32_t* w,
                                      void* stream, uint64_t* phi) {
    if (!phi || (k > 0 && (!off || !col || !w))) return fail(CLDIAM_ERR_INVALID_ARG, "NULL argument");
    return guarded([&] { return apsp_max_noalloc(k, off, col, w, resolve_stream(stream), phi); });
}

cldiam_status cldiam_sssp_source(const cldiam_graph* g, uint64_t seed, uint32_t* source) {
    if (!g || !source) return fail(CLDIAM_ERR_INVALID_ARG, "NULL graph or source");
    U4 r = philox4x32_10(seed, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u);
    *source = r.x % g->n;
    return CLDIAM_OK;
}

cldiam_status cldiam_sssp_delta(cldiam_graph* g, uint32_t source, uint32_t delta, uint32_t* dist, uint64_t* ecc,
                                uint64_t* rounds, uint64_t* edges_scanned) {
    return guarded([&] { return sssp_delta(g, source, delta, dist, ecc, rounds, edges_scanned); });
}

cldiam_status cldiam_arena_job_times(const cldiam_arena* a, uint32_t count, double* start_s, double* end_s) {
    return guarded([&] { return arena_job_times(a, count, start_s, end_s); });
}

cldiam_status cldiam_arena_create(uint64_t hbm_budget_bytes, void* stream, cldiam_arena** out) {
    return guarded([&] { return arena_create(hbm_budget_bytes, resolve_stream(stream), out); });
}

cldiam_status cldiam_arena_add(cldiam_arena* a, const uint32_t* src, const uint32_t* dst, const uint32_t* w,
                               uint64_t m, uint32_t n, uint32_t flags, uint32_t* graph_id) {
    return guarded([&] { return arena_add(a, src, dst, w, m, n, flags, graph_id); });
}

cldiam_status cldiam_arena_info(const cldiam_arena* a, uint32_t* graphs, uint64_t* device_bytes) {
    if (!a) return fail(CLDIAM_ERR_INVALID_ARG, "NULL arena");
    if (graphs) *graphs = arena_count(a);
    if (device_bytes) *device_bytes = arena_device_bytes(a);
    return CLDIAM_OK;
}

cldiam_status cldiam_arena_graph(cldiam_arena* a, uint32_t graph_id, cldiam_graph** out) {
    return guarded([&] { return arena_graph(a, graph_id, out); });
}

cldiam_status cldiam_batch_run(cldiam_arena* a, const uint32_t* graph_ids, const double* tau, const uint64_t* seed,
                               uint32_t count, const cldiam_opts* opts, cldiam_result* out, cldiam_status* status) {
    return guarded([&] { return batch_run(a, graph_ids, tau, seed, count, opts, out, status); });
}

void cldiam_arena_free(cldiam_arena* a) { arena_free(a); }

cldiam_status cldiam_server_create(cldiam_arena* a, const cldiam_server_opts* opts, cldiam_server** out) {
    if (opts && opts->reserved) return fail(CLDIAM_ERR_INVALID_ARG, "reserved must be 0");
    return guarded([&] { return server_create(a, opts, out); });
}

cldiam_status cldiam_server_submit(cldiam_server* s, uint32_t graph_id, double tau, uint64_t seed, uint64_t* ticket) {
    return guarded([&] { return server_submit(s, graph_id, tau, seed, ticket); });
}

cldiam_status cldiam_server_poll(cldiam_server* s, uint64_t ticket, cldiam_result* out) {
    return guarded([&] { return server_poll(s, ticket, out); });
}

cldiam_status cldiam_server_replay(cldiam_server* s, const uint32_t* graph_ids, const double* tau,
                                   const uint64_t* seed, const double* arrival_s, uint32_t count, int32_t plain,
                                   cldiam_result* out, double* latency_s, double* elapsed_s) {
    return guarded([&] {
        return server_replay(s, graph_ids, tau, seed, arrival_s, count, plain, out, latency_s, elapsed_s);
    });
}

void cldiam_server_free(cldiam_server* s) { server_free(s); }

cldiam_status cldiam_run(const uint32_t* src, const uint32_t* dst, const uint32_t* w, uint64_t m, uint32_t n,
                         uint32_t flags, double tau, uint64_t seed, const cldiam_opts* opts, void* stream,
                         cldiam_result* out) {
    if (!out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL out");
    return guarded([&]() -> cldiam_status {
        cldiam_graph* g = nullptr;
        CLD_TRY(build_csr(src, dst, w, m, n, flags, resolve_stream(stream), &g));
        cldiam_clustering* c = nullptr;
        cldiam_quotient* q = nullptr;
        cldiam_status st = cluster(g, tau, seed, opts, &c);
        if (st == CLDIAM_OK) st = quotient(c, &q);
        if (st == CLDIAM_OK) st = cldiam_estimate(q, out);
        free_quotient(q);
        free_clustering(c);
        free_graph(g);
        return st;
    });
}

}  // extern "C"
