// Library handles and cross-file entry points of the CL-DIAM CUDA library.
#pragma once

#include "common.cuh"

// Device-resident symmetric CSR (Section 2 graph model).
struct cldiam_graph {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint32_t n = 0;
    uint64_t nnz = 0;            // directed entries = 2 x undirected edges
    uint64_t* off = nullptr;     // [n+1]
    uint2* adj = nullptr;        // [nnz] (col, w), rows sorted by col
    uint32_t* row = nullptr;     // [nnz] row of each entry (COO view), or null: a CSR assembled from the
                                 // sorted edge lists has none (fill_rows builds it from off when needed)
    uint32_t* orig = nullptr;    // [n] original id
    uint64_t wsum_upper = 0;     // sum of weights over u < v entries
    uint32_t wmin = 0;
    uint32_t max_deg = 0;
    bool connected = false;      // built with the LCC flag: one connected component
    bool borrowed = false;       // a view into arena memory: the arrays are not ours to free
    cld::Pinned host;            // small pinned block for counter read-back
};

struct cldiam_clustering {
    cldiam_graph* g = nullptr;
    cudaStream_t stream = nullptr;  // the graph's stream, kept so that freeing needs no live graph
    uint32_t* center = nullptr;  // [n] center node id
    uint32_t* D = nullptr;       // [n] upper bound on dist_G(center, v)
    uint32_t* cid = nullptr;     // [n] cluster id (rank of the center id)
    uint32_t k = 0;
    uint32_t max_fw_k = 8192;
    uint32_t quotient_mode = 0;  // CLDIAM_QUOTIENT_*
    cldiam_result stats{};
};

struct cldiam_quotient {
    const cldiam_clustering* c = nullptr;
    cudaStream_t stream = nullptr;
    uint32_t k = 0;
    uint64_t nnz = 0;
    uint64_t* off = nullptr;  // [k+1]
    uint32_t* col = nullptr;  // [nnz]
    uint32_t* w = nullptr;    // [nnz]
    uint32_t max_fw_k = 8192;
};

namespace cld {

cudaStream_t resolve_stream(void* user_stream);
// Device copy of a caller array: device pointers are used as they are (*dev = src, *owned = false); host
// memory is copied into a new device buffer by cudaMemcpyAsync on `s` (*owned = true): from pinned memory
// that is the copy engine, which leaves the SMs to other work while the data crosses the host link.
cldiam_status to_device(const void* src, size_t bytes, cudaStream_t s, void** dev, bool* owned);
bool is_device_ptr(const void* p);

cldiam_status build_csr(const uint32_t* src, const uint32_t* dst, const uint32_t* w, uint64_t m, uint32_t n,
                        uint32_t flags, cudaStream_t s, cldiam_graph** out);
void free_graph(cldiam_graph* g);

cldiam_status delta0(const cldiam_graph* g, int mode, uint32_t explicit_value, uint32_t* out);
cldiam_status cluster(cldiam_graph* g, double tau, uint64_t seed, const cldiam_opts* o, cldiam_clustering** out);
cldiam_status cluster2(cldiam_graph* g, double tau, uint64_t seed, const cldiam_opts* o, cldiam_clustering** out);
// cid[v] = rank of center[v] among the centers; *k = their number (synchronises the graph's stream)
cldiam_status relabel_clusters(cldiam_graph* g, const uint32_t* center, uint32_t* cid, uint32_t* k);
void free_clustering(cldiam_clustering* c);

cldiam_status quotient(const cldiam_clustering* c, cldiam_quotient** out);
void free_quotient(cldiam_quotient* q);

// Largest finite APSP distance of a k-node CSR already on the device.
// `tun` holds the cut-over knobs (Floyd-Warshall density, sources per CTA).
cldiam_status apsp_max_device(uint32_t k, const uint64_t* off, const uint32_t* col, const uint32_t* w,
                              uint64_t nnz, cudaStream_t s, uint64_t* phi, bool validate, uint32_t max_fw_k,
                              const cldiam_tuning& tun);

// Same result as apsp_max_device on device-resident inputs, with all scratch in a fixed
// device array instead of allocations.
cldiam_status apsp_max_noalloc(uint32_t k, const uint64_t* off, const uint32_t* col, const uint32_t* w,
                               cudaStream_t s, uint64_t* phi);

// many-graph form (batch.cu)
cldiam_status arena_create(uint64_t budget, cudaStream_t s, cldiam_arena** out);
void arena_free(cldiam_arena* a);
cldiam_status arena_add(cldiam_arena* a, const uint32_t* src, const uint32_t* dst, const uint32_t* w, uint64_t m,
                        uint32_t n, uint32_t flags, uint32_t* id);
cldiam_status arena_graph(cldiam_arena* a, uint32_t id, cldiam_graph** out);
cldiam_status batch_run(cldiam_arena* a, const uint32_t* ids, const double* tau, const uint64_t* seed, uint32_t count,
                        const cldiam_opts* o, cldiam_result* out, cldiam_status* status);
uint32_t arena_count(const cldiam_arena* a);
cldiam_status server_create(cldiam_arena* a, const cldiam_server_opts* o, cldiam_server** out);
cldiam_status server_submit(cldiam_server* sv, uint32_t graph_id, double tau, uint64_t seed, uint64_t* ticket);
cldiam_status server_poll(cldiam_server* sv, uint64_t ticket, cldiam_result* out);
cldiam_status server_free(cldiam_server* sv);
cldiam_status server_replay(cldiam_server* sv, const uint32_t* ids, const double* tau, const uint64_t* seed,
                            const double* arrival, uint32_t count, int plain, cldiam_result* out, double* latency,
                            double* elapsed);
uint64_t arena_device_bytes(const cldiam_arena* a);
cudaStream_t arena_stream(const cldiam_arena* a);

cldiam_status arena_job_times(const cldiam_arena* a, uint32_t count, double* start_s, double* end_s);
// adjacency entries of the listed graphs (ids out of range count 0)
uint64_t arena_entries(const cldiam_arena* a, const uint32_t* ids, uint32_t count);

// row[p] = v for every CSR position p of row v (a graph assembled from the sorted lists keeps no row array)
cldiam_status fill_rows(const uint64_t* off, uint32_t n, uint32_t* row, cudaStream_t s);

cldiam_status sssp_delta(cldiam_graph* g, uint32_t source, uint32_t delta, uint32_t* dist_out, uint64_t* ecc,
                         uint64_t* rounds, uint64_t* scanned);

// tuning knobs in effect (defaults filled in) and their validation (tune.cu): the process-wide
// settings alone, or for a call on `entries` adjacency entries of one graph (or of one batch), where the
// autotuner's cached choice for this device and size class fills the knobs not set process-wide
cldiam_tuning tuning_current();
cldiam_tuning tuning_for(uint64_t entries);
cldiam_tuning tuning_for_batch(uint64_t entries);
uint32_t size_class(uint64_t entries);
cldiam_tuning tuning_defaults_filled(const cldiam_tuning& t);
cldiam_status tuning_check(const cldiam_tuning& t);

}  // namespace cld
