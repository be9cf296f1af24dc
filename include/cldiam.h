/*
 * cldiam.h — C ABI of the GB300 (sm_103a) CL-DIAM library.
 *
 * CL-DIAM estimates the weighted diameter of a large undirected graph
 * (Ceccarello, Pietracaprina, Pucci, Upfal, arXiv 1506.03265):
 *   1. CLUSTER(tau) grows clusters from batches of randomly drawn centers by
 *      Delta-bounded relaxation rounds, doubling Delta until half of the
 *      uncovered nodes are reached (Section 3, Algorithm 1);
 *   2. the clustering is contracted into the weighted quotient graph G_C
 *      (Section 4): one node per cluster, edge weight w(u,v) + d_u + d_v,
 *      minimum per cluster pair;
 *   3. Phi_approx = Phi(G_C) + 2 R, R the largest center distance (Section 4).
 * A Delta-stepping SSSP (Meyer and Sanders) gives the competitor's
 * 2-approximation 2 * ecc(s) (Section 5).
 *
 * Conventions for every entry point:
 *  - Status: 0 = CLDIAM_OK, negative = error (below).  No C++ exception ever
 *    crosses this boundary.  cldiam_last_error() describes the last failure of
 *    the calling thread.
 *  - Pointers: arrays passed in or out may live in host memory (pageable or
 *    pinned) or in device memory of the current device; the library copies
 *    with unified addressing and never keeps a borrowed pointer after the
 *    call returns.
 *  - Ownership: every handle (cldiam_graph, cldiam_clustering,
 *    cldiam_quotient, ...) is created and owned by the library and released by
 *    its matching *_free function, which accepts NULL.  A clustering or
 *    quotient refers to (does not copy) the graph it came from; free it first.
 *  - Streams: `stream` is a cudaStream_t or NULL (the library's own stream).
 *    All work for a graph runs on the stream it was built with.  Calls return
 *    after their results are complete (they synchronise that stream), except
 *    where noted.
 *  - Integers: node ids and weights are uint32; weights must be >= 1 (the
 *    paper's positive integral weights, Section 2).  Distances inside the
 *    library are exact uint32; a distance or quotient weight that would
 *    reach 2^32 - 1 yields CLDIAM_ERR_OVERFLOW instead of a wrong answer.
 *    The quotient diameter is exact whenever every quotient distance is
 *    below 2^31 - 1; beyond that, a candidate path sum that reaches 2^32 - 1
 *    is reported as CLDIAM_ERR_OVERFLOW even if the shortest distances fit.
 *  - Threads: one handle must not be used by two threads at once.  Calls on
 *    different handles (and cldiam_run) may run at once from several threads,
 *    each on its own stream; they give the results they give alone.
 */
#ifndef CLDIAM_H
#define CLDIAM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t cldiam_status;

#define CLDIAM_OK 0
#define CLDIAM_ERR_INVALID_ARG (-1) /* a size, pointer, id or weight is out of range */
#define CLDIAM_ERR_OOM (-2)         /* device (or host) allocation failed            */
#define CLDIAM_ERR_OVERFLOW (-3)    /* an exact distance would not fit in uint32     */
#define CLDIAM_ERR_TIMEOUT (-4)     /* a bounded device-side wait expired            */
#define CLDIAM_ERR_CUDA (-5)        /* a CUDA runtime call failed                    */
#define CLDIAM_ERR_BUSY (-6)        /* result not ready yet (serving poll)           */
#define CLDIAM_ERR_CANCELLED (-7)   /* request cancelled or server stopped           */
#define CLDIAM_ERR_DIVERGED (-8)    /* CLUSTER / CLUSTER2 growth exceeded its limits */
#define CLDIAM_ERR_UNSUPPORTED (-9) /* valid request this build does not handle      */

/* cldiam_build_csr flags */
#define CLDIAM_CSR_LCC 1u /* keep only the largest connected component */

/* cldiam_opts.delta0_mode: initial Delta of CLUSTER */
#define CLDIAM_DELTA0_AVG 0      /* floor(mean edge weight), the choice of Section 5 (default) */
#define CLDIAM_DELTA0_MIN 1      /* minimum edge weight, as in Algorithm 1                     */
#define CLDIAM_DELTA0_EXPLICIT 2 /* cldiam_opts.delta0                                         */

typedef struct cldiam_graph cldiam_graph;           /* device-resident symmetric CSR          */
typedef struct cldiam_clustering cldiam_clustering; /* device-resident centers, D, cluster ids */
typedef struct cldiam_quotient cldiam_quotient;     /* device-resident quotient CSR            */
typedef struct cldiam_arena cldiam_arena;           /* many graphs packed in one device CSR arena */
typedef struct cldiam_server cldiam_server;         /* request server over an arena              */

/* Options of cldiam_cluster.  Zero-initialised = the defaults. */
typedef struct {
    int32_t delta0_mode;   /* CLDIAM_DELTA0_*                                              */
    uint32_t delta0;       /* used with CLDIAM_DELTA0_EXPLICIT; must be >= 1                */
    int32_t contract_mode; /* CLDIAM_CONTRACT_*                                             */
    uint32_t step_cap;     /* growing steps per PartialGrowth execution; 0 = no cap         */
    uint32_t max_fw_k;     /* largest dense quotient solved by Floyd-Warshall; 0 = 8192     */
    uint32_t quotient_mode; /* CLDIAM_QUOTIENT_*: how cldiam_quotient_build deduplicates     */
    uint32_t reserved[2];  /* must be 0                                                     */
} cldiam_opts;

/* cldiam_opts.contract_mode */
#define CLDIAM_CONTRACT_RESET 0      /* clusters of earlier stages relax from distance 0 through every
                                        member (Procedure Contract); D_v = d_v + R[c_v] (default) */
#define CLDIAM_CONTRACT_CUMULATIVE 1 /* a member u of an earlier cluster relaxes with its own bound
                                        D_u (while D_u < Delta); D_v = d_v <= final Delta         */

/* cldiam_opts.quotient_mode (same result either way) */
#define CLDIAM_QUOTIENT_AUTO 0  /* dense while k <= 4096, else radix sort (default) */
#define CLDIAM_QUOTIENT_SORT 1  /* radix sort of (cid_u, cid_v) keys + segmented min */
#define CLDIAM_QUOTIENT_DENSE 2 /* atomicMin into a k x k matrix (k <= 65535)        */

/* Result of the whole method plus the paper-style counters (Table 2: rounds and work). */
typedef struct {
    uint64_t phi_gc;      /* Phi(G_C): largest finite distance in the quotient graph      */
    uint64_t radius;      /* R = max over nodes of D_v (upper bound on dist(c_v, v))      */
    uint64_t phi_approx;  /* Phi(G_C) + 2 R  (>= Phi(G), Section 4)                       */
    uint32_t k;           /* number of clusters = quotient nodes                          */
    uint32_t stages;      /* iterations of Algorithm 1's outer loop                       */
    uint32_t steps;       /* Delta-growing steps executed (the paper's rounds of growth)  */
    uint32_t doublings;   /* times Delta was doubled                                      */
    uint32_t delta_end;   /* Delta at the end                                             */
    uint32_t guard_exits; /* stages ended at a fixed point with coverage under half      */
    uint64_t node_updates;   /* node state decreases over all steps (the paper's work)   */
    uint64_t edges_scanned;  /* adjacency entries read by the relaxation kernels         */
    uint64_t quotient_edges; /* directed entries of the quotient CSR                     */
    uint64_t centers_drawn;  /* centers drawn over all stages (singletons not included)  */
} cldiam_result;

/* ------------------------------------------------------------------------ */
const char* cldiam_status_string(cldiam_status s);
/* Message for the calling thread's last failure ("" if none).  Valid until the next call. */
const char* cldiam_last_error(void);
/* Library version (major, minor); either pointer may be NULL. */
cldiam_status cldiam_version(int32_t* major, int32_t* minor);

/*
 * Build the device CSR of an undirected weighted graph (Section 2 graph model).
 *  src, dst, w : m edges (host or device arrays); node ids < n, weights >= 1.
 *               Host arrays are copied to the device first, on the call's
 *               stream (from pinned memory by the copy engine, which leaves
 *               the SMs to work queued on other streams meanwhile).
 *  Self-loops are dropped; parallel edges merge to their minimum weight; the
 *  result is symmetric with rows sorted by column.  With CLDIAM_CSR_LCC only
 *  the largest connected component is kept (ties: the component holding the
 *  smallest id) and its nodes are renumbered by increasing original id.
 *  Errors: INVALID_ARG (n == 0, id >= n, weight 0), OOM, CUDA.
 */
cldiam_status cldiam_build_csr(const uint32_t* src, const uint32_t* dst, const uint32_t* w, uint64_t m,
                               uint32_t n, uint32_t flags, void* stream, cldiam_graph** out);
/* Node count and directed entry count (2 x undirected edges) of a built graph. */
cldiam_status cldiam_graph_info(const cldiam_graph* g, uint32_t* n, uint64_t* nnz);
/* Copy the CSR out: off[n+1], col[nnz], w[nnz], orig[n] (original id of each node).
 * Any pointer may be NULL to skip that array. */
cldiam_status cldiam_graph_copy(const cldiam_graph* g, uint64_t* off, uint32_t* col, uint32_t* w,
                                uint32_t* orig);
void cldiam_graph_free(cldiam_graph* g);

/* Initial Delta by mode (CLDIAM_DELTA0_AVG or _MIN), Algorithm 1 / Section 5. */
cldiam_status cldiam_delta0(const cldiam_graph* g, int32_t mode, uint32_t* out);

/*
 * CLUSTER(G, tau) of Algorithm 1, on the device.
 *  tau  : > 0.  Stages run while |U| >= 8 tau log2 n (U = uncovered nodes);
 *         each draws node v of U as a center iff Philox4x32-10(key = seed,
 *         counter = (v, stage, 0, 0)) word 0 < floor(p 2^32),
 *         p = 4 ln2 tau log2 n / |U|.
 *  Growth: synchronous Delta-growing steps (Section 3) with the
 *         (distance, center id) tie-break; PartialGrowth stops when no state
 *         changes, 2 covered >= |U|, or (opts->step_cap > 0) after step_cap
 *         steps -- the O(n / tau) limit of Section 3's closing remark; Delta
 *         doubles (capped at 2^31) while coverage is under half and some
 *         uncovered node is still reachable.
 *  Contract: clusters of earlier stages relax from distance 0 through every
 *         member; D_v = d_v + R[c_v] bounds dist_G(c_v, v).  With
 *         CLDIAM_CONTRACT_CUMULATIVE a member u relaxes with its own D_u
 *         instead and D_v = d_v, so every D_v is within the final Delta.
 *  Leftover nodes become singleton clusters.  Results are a deterministic
 *  function of (graph, tau, seed, opts).
 *  Errors: INVALID_ARG, OVERFLOW (a D_v >= 2^32 - 1), DIVERGED, OOM, CUDA.
 */
cldiam_status cldiam_cluster(cldiam_graph* g, double tau, uint64_t seed, const cldiam_opts* opts,
                             cldiam_clustering** out);
/*
 * CLUSTER2(G, tau) of Algorithm 2 (Section 4), on the device: the clustering
 * behind the O(log^3 n) approximation bound of Section 4 (CL-DIAM itself, as
 * Section 5 describes it, uses cldiam_cluster).
 *  First cldiam_cluster(g, tau, seed, opts); R_CL = the largest D_v of that
 *  clustering.  Then iterations i = 1..L, L = the least i >= 1 with 2^i >= n:
 *   - a node not yet covered is drawn as a new center iff
 *     Philox4x32-10(key = seed, counter = (v, i, 1, 0)) word 0 < floor(2^i 2^32 / n)
 *     (every such node when 2^i >= n);
 *   - PartialGrowth2: growth with Delta = 2 R_CL until no state changes,
 *     (distance, center id) tie-break, only edges of weight <= 2 R_CL;
 *   - Contract2: the covered nodes merge into their clusters, an edge leaving a
 *     cluster gets weight d_u + w - 2 R_CL.
 *  D_v = d_v + (i_v - i_c) 2 R_CL for v reached in iteration i_v (distance d_v
 *  in that iteration's contracted graph) by a center drawn in iteration i_c:
 *  the length of the path the growth followed, >= dist_G(c_v, v).
 *  The result feeds cldiam_quotient_build / cldiam_estimate like a
 *  cldiam_cluster result (Phi_approx = Phi(G_C) + 2 max D_v).  Counters:
 *  stages = L, steps = device growth rounds (asynchronous relaxation to the
 *  same fixed point as the paper's synchronous steps), delta_end = 2 R_CL,
 *  centers_drawn = centers drawn by the iterations.  Deterministic in
 *  (graph, tau, seed, opts).
 *  Errors: those of cldiam_cluster; UNSUPPORTED when L x 2 R_CL >= 2^32 - 1.
 */
cldiam_status cldiam_cluster2(cldiam_graph* g, double tau, uint64_t seed, const cldiam_opts* opts,
                              cldiam_clustering** out);
/* Counters of the clustering (k, stages, steps, ... ; phi fields are 0). */
cldiam_status cldiam_clustering_info(const cldiam_clustering* c, cldiam_result* out);
/* center[n] (center node id), D[n], cid[n] (cluster id = rank of the center id); any may be NULL. */
cldiam_status cldiam_clustering_copy(const cldiam_clustering* c, uint32_t* center, uint32_t* D, uint32_t* cid);
void cldiam_clustering_free(cldiam_clustering* c);

/*
 * Weighted quotient graph G_C (Section 4): node i = cluster i; for every edge
 * (u,v) with different clusters an edge of weight w(u,v) + D_u + D_v, minimum
 * per pair, stored as a symmetric CSR sorted by (row, col).  Pairs are
 * deduplicated by a radix sort of (cid_u, cid_v) keys with a segmented min, or
 * in a dense k x k matrix (opts.quotient_mode of the clustering).
 * Errors: OVERFLOW (a weight >= 2^32 - 1), OOM, CUDA.
 */
cldiam_status cldiam_quotient_build(const cldiam_clustering* c, cldiam_quotient** out);
cldiam_status cldiam_quotient_info(const cldiam_quotient* q, uint32_t* k, uint64_t* nnz);
/* off[k+1], col[nnz], w[nnz]; any may be NULL. */
cldiam_status cldiam_quotient_copy(const cldiam_quotient* q, uint64_t* off, uint32_t* col, uint32_t* w);
void cldiam_quotient_free(cldiam_quotient* q);

/*
 * Estimate (Section 4): out->phi_gc = Phi(G_C) by exact all-pairs shortest
 * paths on the quotient -- batched SSSP (multi-source Bellman-Ford, k <= 51,200)
 * when it has fewer than k^2/8 entries, else blocked Floyd-Warshall (k <=
 * max_fw_k) -- out->radius = max D, out->phi_approx = phi_gc + 2 radius; the
 * clustering counters are filled in too.  out is a host pointer.
 * Errors: OVERFLOW, UNSUPPORTED (no path applies to this k), OOM, CUDA.
 */
cldiam_status cldiam_estimate(const cldiam_quotient* q, cldiam_result* out);

/*
 * Largest finite shortest-path distance of a small weighted graph given as a
 * symmetric CSR (k nodes, off[k+1], col/w[nnz]; host or device), exact, on the
 * device: batched SSSP for sparse graphs, blocked Floyd-Warshall (k <= 8192,
 * with a k x k scratch matrix) for dense ones; used for Phi(G_C).  The CSR is
 * validated on the device first.  *phi is a host pointer.  Exact when every
 * distance is below 2^31 - 1; above, OVERFLOW if a candidate path sum reaches
 * 2^32 - 1 (see the integer rules at the top).
 * Errors: INVALID_ARG (malformed CSR), OVERFLOW, UNSUPPORTED, OOM, CUDA.
 */
cldiam_status cldiam_apsp_max(uint32_t k, const uint64_t* off, const uint32_t* col, const uint32_t* w,
                              void* stream, uint64_t* phi);

/*
 * cldiam_apsp_max without any device allocation.  The paper has no
 * counterpart; this exists for callers that are not allowed to allocate GPU
 * memory themselves or through us -- for example a host application that
 * owns the whole device memory budget through its own allocator, or code
 * that must not risk an allocation failure or the latency of a first
 * allocation in the middle of its work.
 *  - Same result as cldiam_apsp_max.  off, col and w must already be in device
 *    memory (nothing is copied); *phi is a host pointer.
 *  - Scratch is one fixed array inside the library (about 4 MB per GPU that
 *    loads it, resident until the process exits).  Limits: k <= 1024 when the
 *    graph has at least k^2/8 entries (Floyd-Warshall in that array), k <=
 *    51,200 otherwise (batched SSSP with the same kernels cldiam_apsp_max
 *    takes by default, its distances in shared memory); larger k returns
 *    CLDIAM_ERR_UNSUPPORTED.  No cudaMalloc, cudaFree or allocating library call.
 *  - The first call on each device looks up the array's device address (with
 *    that device current); make that first call before any stream capture.
 *  - Each call waits for `stream` to finish its work before it returns.
 *  - Every call reuses the same array, so two calls whose work overlaps on the
 *    GPU (different streams or threads) race on it: serialise them.
 * Errors: INVALID_ARG (NULL, host pointers, malformed CSR), UNSUPPORTED, OVERFLOW,
 * DIVERGED (the SSSP exceeded its round limit), CUDA.
 */
cldiam_status cldiam_apsp_max_noalloc(uint32_t k, const uint64_t* off, const uint32_t* col, const uint32_t* w,
                                      void* stream, uint64_t* phi);

/* Source node of the SSSP baseline: Philox4x32-10(seed; (2^32-1, 2^32-1, 0, 0)) word 0 mod n. */
cldiam_status cldiam_sssp_source(const cldiam_graph* g, uint64_t seed, uint32_t* source);
/*
 * Delta-stepping SSSP (Meyer and Sanders) from `source` with bucket width
 * `delta` (>= 1; 0 = average edge weight times cldiam_tuning.sssp_delta_scale):
 * exact distances, so any delta gives the same result.  dist[n] (may be NULL;
 * 0xFFFFFFFF = unreachable) and *ecc = largest finite distance (host pointer);
 * 2 * ecc is the SSSP 2-approximation of Section 5.  *rounds (may be NULL) =
 * light/heavy phases run; *edges_scanned (may be NULL) = adjacency entries the
 * phases read (0 on graphs with 2^32 or more entries, which are not counted).
 * Errors: INVALID_ARG, OVERFLOW, OOM, CUDA.
 */
cldiam_status cldiam_sssp_delta(cldiam_graph* g, uint32_t source, uint32_t delta, uint32_t* dist,
                                uint64_t* ecc, uint64_t* rounds, uint64_t* edges_scanned);

/*
 * Whole method from an edge list: build CSR (with `flags`), CLUSTER, quotient,
 * estimate.  Inputs may be host or device arrays; out is a host pointer.
 */
cldiam_status cldiam_run(const uint32_t* src, const uint32_t* dst, const uint32_t* w, uint64_t m, uint32_t n,
                         uint32_t flags, double tau, uint64_t seed, const cldiam_opts* opts, void* stream,
                         cldiam_result* out);

/* ------------------------------------------------------------------------
 * Many-graph form (no counterpart in the paper, which runs one graph on a
 * cluster): graphs are packed into one device-resident CSR arena and a batch
 * of (graph, tau, seed) jobs runs the whole method -- CLUSTER (Algorithm 1),
 * the weighted quotient graph and Phi_approx (Section 4) -- in one persistent
 * launch, one graph per CTA at a time, largest graphs first.  The launch
 * ends with its largest graph on one CTA or with the even split of all work,
 * whichever is later; the largest graphs may therefore run first on the
 * one-graph path with the whole device (cldiam_tuning.batch_split).  Every result is
 * identical to cldiam_cluster + cldiam_quotient_build + cldiam_estimate on the
 * same graph, tau and seed with the same options.
 */
/* Empty arena on `stream`; hbm_budget_bytes (0 = unlimited) caps the device memory it may hold
 * (graphs plus the batch workspace); an add that would exceed it fails with OOM. */
cldiam_status cldiam_arena_create(uint64_t hbm_budget_bytes, void* stream, cldiam_arena** out);
/* Build one graph's CSR (as cldiam_build_csr with `flags`) and append it; *graph_id is its index. */
cldiam_status cldiam_arena_add(cldiam_arena* a, const uint32_t* src, const uint32_t* dst, const uint32_t* w,
                               uint64_t m, uint32_t n, uint32_t flags, uint32_t* graph_id);
/* Number of graphs and device bytes held (either pointer may be NULL). */
cldiam_status cldiam_arena_info(const cldiam_arena* a, uint32_t* graphs, uint64_t* device_bytes);
/* A graph handle viewing one arena graph, for the one-graph entry points; free it with
 * cldiam_graph_free (the arena's memory is not released) before freeing the arena. */
cldiam_status cldiam_arena_graph(cldiam_arena* a, uint32_t graph_id, cldiam_graph** out);
/* Run `count` jobs: graph_ids[i], tau[i] (> 0), seed[i]; opts applies to all (NULL = defaults).
 * out[i] (host) receives job i's result; status[i] (host, may be NULL) its status.  Returns the
 * first failing status (OVERFLOW, DIVERGED, TIMEOUT) if any job failed, else OK. */
cldiam_status cldiam_batch_run(cldiam_arena* a, const uint32_t* graph_ids, const double* tau, const uint64_t* seed,
                               uint32_t count, const cldiam_opts* opts, cldiam_result* out, cldiam_status* status);
/* Device time of each job of the last cldiam_batch_run on this arena, in the caller's job order:
 * start_s[i] / end_s[i] (host arrays of `count`) = when job i started / ended, in seconds from the start
 * of the batch: the graphs run first on the one-graph path back to back (CUDA events), then the
 * persistent launch's jobs (device global timer, offset by the one-graph runs); a job finished on the
 * one-graph path after the launch keeps its in-kernel times.  INVALID_ARG if count exceeds the last
 * batch. */
cldiam_status cldiam_arena_job_times(const cldiam_arena* a, uint32_t count, double* start_s, double* end_s);
void cldiam_arena_free(cldiam_arena* a);

/* ------------------------------------------------------------------------
 * Served form (no counterpart in the paper): diameter queries on arena graphs
 * with continuous batching.  A persistent kernel keeps running; each of its
 * CTAs takes the next submitted request as soon as it finishes the previous
 * one, so requests that arrive while others run join at once and their work
 * overlaps on the device.  Graphs above opts.big_nodes nodes run on the
 * one-graph path on a second stream, on the SMs the kernel leaves free, one
 * at a time, admitted when their device memory fits the budget.  Results are
 * identical to the one-graph path (CLDIAM_DELTA0_AVG, default options).
 */
typedef struct {
    uint32_t ctas;             /* CTAs of the serving kernel; 0 = SMs - 24 (the rest serve large graphs) */
    uint32_t capacity;         /* requests over the server's lifetime; 0 = 2^20                         */
    uint32_t big_nodes;        /* graphs with more nodes take the one-graph path; 0 = 2^19              */
    uint32_t reserved;         /* must be 0                                                              */
    uint64_t hbm_budget_bytes; /* device memory cap for arena + workspaces + large requests; 0 = none   */
    double idle_seconds;       /* CTAs leave after this long without requests (relaunched on demand); 0 = 10 */
} cldiam_server_opts;
/* Start serving the graphs of `a` (which must outlive the server; add no graphs meanwhile). */
cldiam_status cldiam_server_create(cldiam_arena* a, const cldiam_server_opts* opts, cldiam_server** out);
/* Queue one query; *ticket identifies it.  BUSY when the lifetime capacity is used up. */
cldiam_status cldiam_server_submit(cldiam_server* s, uint32_t graph_id, double tau, uint64_t seed, uint64_t* ticket);
/* CLDIAM_ERR_BUSY until the query has finished; then its status, and *out (host) its result. */
cldiam_status cldiam_server_poll(cldiam_server* s, uint64_t ticket, cldiam_result* out);
/* Replay an arrival trace natively: query i is submitted arrival_s[i] seconds after the start;
 * latency_s[i] = completion - arrival.  plain != 0 serves the same trace one query at a time in
 * arrival order on the one-graph path instead (the baseline).  out/latency_s are host arrays of
 * `count`; *elapsed_s (may be NULL) = wall time of the whole replay. */
cldiam_status cldiam_server_replay(cldiam_server* s, const uint32_t* graph_ids, const double* tau,
                                   const uint64_t* seed, const double* arrival_s, uint32_t count, int32_t plain,
                                   cldiam_result* out, double* latency_s, double* elapsed_s);
/* Finish the queries already submitted, stop the kernel and release everything the server holds. */
void cldiam_server_free(cldiam_server* s);

/* ------------------------------------------------------------------------
 * Tuning.  No counterpart in the paper: launch shapes of the kernels and the
 * cut-overs between equivalent forms of one step.  Every knob is
 * result-invariant -- each form computes the same integers -- so a choice only
 * changes the time.  A field left 0 takes the library default.
 */
typedef struct {
    float pull_ratio;              /* a growing step takes the dense pull form (every node reads its
                                      own adjacency) when its relaxers' adjacency is at least this share
                                      of all adjacency entries; < 0 = never; 0 = 0.3                */
    uint32_t relax_ctas_per_sm;    /* CTAs per SM of the growing-step kernels; 0 = all that fit     */
    uint32_t dense_quotient_k;     /* CLDIAM_QUOTIENT_AUTO: dense k x k de-duplication up to this k
                                      (<= 65535), radix sort above; 0 = 4096                       */
    uint32_t apsp_sources_per_cta; /* quotient diameter by batched SSSP: sources per CTA, 1, 4 or 8;
                                      0 = by k (8 below 2,048 nodes, else 4)                       */
    uint32_t apsp_fw_density;      /* quotient diameter by Floyd-Warshall when nnz >= k^2 / this,
                                      batched SSSP otherwise; 0 = 8                                 */
    uint32_t batch_fw_k;           /* many-graph form: quotients up to this k (<= 200) are closed by
                                      Floyd-Warshall in shared memory; 0 = 200                     */
    float sssp_delta_scale;        /* Delta-stepping with delta = 0: Delta = this x the average
                                      weight (>= 1); 0 = 1                                          */
    uint32_t batch_split;          /* many-graph form: 2 = the k largest graphs (each with at least
                                      2^16 entries) run first on the one-graph path with the whole
                                      device, k chosen by a makespan model (one CTA's rate in the
                                      launch against a fixed cost per graph on the one-graph path);
                                      1 = every graph in the persistent launch; 0 = 2              */
    uint32_t reserved[8];          /* must be 0                                                     */
} cldiam_tuning;

/* The process-wide knobs (defaults filled in). */
cldiam_status cldiam_tuning_get(cldiam_tuning* out);
/* Replace the process-wide knobs; NULL restores the defaults.  INVALID_ARG on a value out of range.
 * Takes effect for calls that start afterwards; not meant to race with calls in flight. */
cldiam_status cldiam_tuning_set(const cldiam_tuning* t);

/*
 * Autotuner (no counterpart in the paper).  The knob that a call uses is, per
 * field: the process-wide value if set (non-zero), else the autotuner's cached
 * choice for this device and the call's size class, else the default.  The
 * size class of a one-graph call is floor(log2(adjacency entries of the
 * graph)); a many-graph call uses 64 + floor(log2(entries of the batch)) (the
 * served form: of the whole arena).
 *
 * The tuners time the caller's own work -- CUDA events on its stream, the
 * median of `reps` runs (0 = 3) after one warm-up -- for each candidate value
 * of one knob at a time (coordinate descent over fixed candidate lists,
 * starting from the process-wide setting), keep a change only when it is at
 * least 2 % faster, check that every candidate returns the same result (a
 * change is a library fault: DIVERGED), store the chosen knobs in the cache
 * and return them in *out.  They replace the process-wide knobs while they
 * run, so no other call may run meanwhile.
 *  graph: pull_ratio, relax_ctas_per_sm, dense_quotient_k, apsp_sources_per_cta,
 *         apsp_fw_density on cldiam_cluster + cldiam_quotient_build + cldiam_estimate;
 *  batch: batch_split, batch_fw_k on cldiam_batch_run of the listed jobs;
 *  sssp:  sssp_delta_scale on cldiam_sssp_delta(delta = 0) from `source`.
 */
cldiam_status cldiam_autotune_graph(cldiam_graph* g, double tau, uint64_t seed, const cldiam_opts* opts,
                                    uint32_t reps, cldiam_tuning* out);
cldiam_status cldiam_autotune_batch(cldiam_arena* a, const uint32_t* graph_ids, const double* tau,
                                    const uint64_t* seed, uint32_t count, const cldiam_opts* opts, uint32_t reps,
                                    cldiam_tuning* out);
cldiam_status cldiam_autotune_sssp(cldiam_graph* g, uint32_t source, uint32_t reps, cldiam_tuning* out);
/*
 * The search itself, for work the caller measures: `measure` runs the work
 * with the candidate knobs and returns its time in *seconds and a digest of
 * its result in *result_hash (any non-OK status skips the candidate).
 * knob_mask bit i = the i-th field of cldiam_tuning (0 pull_ratio ..
 * 7 batch_split).  Host code only: needs no GPU.
 */
typedef cldiam_status (*cldiam_tune_measure_fn)(const cldiam_tuning* candidate, void* user, double* seconds,
                                                 uint64_t* result_hash);
cldiam_status cldiam_autotune_search(const cldiam_tuning* start, uint32_t knob_mask,
                                     cldiam_tune_measure_fn measure, void* user, cldiam_tuning* best,
                                     double* best_seconds);
/* Size class of a call on `entries` adjacency entries: floor(log2(entries)) (0 for 0 or 1). */
uint32_t cldiam_size_class(uint64_t entries);
/* The knobs a call on `device` in `size_class` would use (process-wide, cache, defaults). */
cldiam_status cldiam_tuning_effective(int32_t device, uint32_t size_class, cldiam_tuning* out);
/* The tuning cache: set or read one entry (fields 0 = not cached), clear all, save to or load from a
 * text file (one line per entry: device, size class, the eight knobs).  INVALID_ARG when an entry is
 * missing, a value is out of range or the file cannot be read or written. */
cldiam_status cldiam_tuning_cache_put(int32_t device, uint32_t size_class, const cldiam_tuning* t);
cldiam_status cldiam_tuning_cache_get(int32_t device, uint32_t size_class, cldiam_tuning* out);
void cldiam_tuning_cache_clear(void);
cldiam_status cldiam_tuning_cache_save(const char* path);
cldiam_status cldiam_tuning_cache_load(const char* path);

/* ------------------------------------------------------------------------
 * Instrumentation.  No counterpart in the method itself; it exposes what the
 * paper measures (rounds and work, Table 2) plus per-kernel device time.
 * Kernel classes: 0 relax, 1 snapshot, 2 rebuild, 3 select, 4 finalize,
 * 5 growable, 6 radix_hist, 7 radix_scatter, 8 scan, 9 csr, 10 components,
 * 11 quotient, 12 floyd_warshall, 13 delta_stepping, 14 reduce, 15 misc,
 * 16 relax_pull (the dense form of a growing step).
 * Process-wide; not meant for concurrent use from several threads.
 */
/* Bit i set: bracket every launch of class i with CUDA events on its stream. 0 = off (default). */
cldiam_status cldiam_profile_set_timing(uint32_t class_mask);
/* Zero all counters (waits for pending timing events). */
cldiam_status cldiam_profile_reset(void);
uint32_t cldiam_profile_num_classes(void);
/* Launch count, summed event time (ms, timed classes only) and algorithmic bytes of one class since
 * the last reset; *name is a static string.  Any output pointer may be NULL. */
cldiam_status cldiam_profile_get(uint32_t cls, const char** name, uint64_t* launches, double* ms, double* bytes);

#ifdef __cplusplus
}
#endif

#endif /* CLDIAM_H */
