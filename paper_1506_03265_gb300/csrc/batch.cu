// Many-graph form: graphs packed into one device CSR arena and processed by
// one persistent launch.  Each CTA (1024 threads, one per SM) takes whole
// graphs from a work queue (largest first) and runs CLUSTER(tau) (the phase
// bodies of cluster_dev.cuh, rank 0 of 1, block barriers between phases),
// the weighted quotient graph (Section 4) and the exact Phi(G_C) for it.
// Results are identical to the one-graph-per-launch path: the same phase
// bodies run in the same order on the same data, and the stage control uses
// the same host-computed log2 n.
//
// The quotient is deduplicated in a dense k x k matrix (atomicMin per
// inter-cluster edge) instead of a sort; its row order equals the sorted
// quotient CSR of the other path.  Graphs whose quotient exceeds the dense
// capacity are finished with the one-graph path after the launch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "cluster_dev.cuh"
#include "internal.cuh"
#include "prof.cuh"

namespace cld {

namespace {

// many-graph CTAs resident per SM.  One 1,024-thread CTA per SM: two 512-thread CTAs per SM (shared-memory
// carveout at its maximum, Floyd-Warshall cut-over 128) gave 16 % more aggregate work per second on the
// 2,000-graph mixture but 1.6x the time per large graph on one CTA, and its 111 R-MAT 16 graphs set the
// tail (17.4k against 25.4k graphs/s)
constexpr int kBatchCtasPerSm = 1;
constexpr int BT = 1024 / kBatchCtasPerSm;  // threads per CTA
constexpr int kRelaxU = 1024 / BT;          // positions per thread of a growing-step chunk (1,024 per chunk)
constexpr uint32_t kDenseCap = 1024;  // largest quotient deduplicated in the dense matrix
constexpr uint64_t kSplitMinEntries = 1u << 16;  // graphs below this many entries always stay in the launch
// makespan model of the many-graph split (GB300): seconds per unit of work (entry or node) on one 1,024-thread
// CTA of the launch, and a graph's cost on the one-graph path (a fixed part for its launches and counter
// reads, and a per-unit part with the whole device)
constexpr double kCtaSecPerUnit = kBatchCtasPerSm == 1 ? 37e-9 : 63e-9;
constexpr double kPlainSecPerGraph = 1.5e-3;
constexpr double kPlainSecPerUnit = 0.05e-9;
// quotients up to this size are closed by Floyd-Warshall in shared memory (the k x k matrix, next to the
// static shared memory, must fit kBatchCtasPerSm times per SM)
constexpr uint32_t kSmemFwK = kBatchCtasPerSm == 1 ? 200 : 128;
constexpr uint32_t kJobOk = 0, kJobNeedsPlain = 1, kJobOverflow = 2, kJobDiverged = 3, kJobTimeout = 4;

struct ArenaDesc {  // one graph of the arena (device copy)
    uint64_t off_base;  // into the arena's offset array (n + 1 entries, local values)
    uint64_t adj_base;  // into the arena's adjacency / row arrays
    uint64_t nnz;
    uint32_t n;
    uint32_t connected;
};

struct Job {
    double tau;
    double L;  // log2 n, computed on the host
    uint64_t seed;
    uint32_t graph;
    uint32_t delta0;
    uint32_t out;         // index in the caller's result array
    uint32_t step_cap;    // growing steps per PartialGrowth, 0 = no cap
    uint32_t cumulative;  // cumulative contract mode
    uint32_t fw_k;        // quotients up to this size (<= kSmemFwK) are closed by Floyd-Warshall in shared memory
    uint32_t pad;
};

struct Workspace {  // one slice per CTA
    unsigned long long* key;
    unsigned long long* fkey[2];
    uint32_t* center;
    uint32_t* D;
    uint32_t* R;
    uint32_t* stamp;
    uint32_t* fbase[2];
    uint32_t* fpre[2];
    uint32_t* next;
    uint32_t* cid;
    uint32_t* M;      // dense quotient, kDenseCap^2
    uint32_t* qoff;   // quotient CSR extracted from M
    uint32_t* qcol;
    uint32_t* qw;
    Counters* ctr;
};

struct JobOut {
    cldiam_result r;
    uint32_t status;
    uint32_t pad;
    uint64_t t_start, t_end;  // device global timer (ns) when the job started and ended
};


__device__ __forceinline__ uint32_t relax_min_u32(uint32_t c, uint32_t a, uint32_t b, bool& ovf) {
    const uint32_t s = a + b;
    const bool carry = s < a;
    const bool finite = (a != kNone) & (b != kNone);
    ovf |= finite & (carry | (s == kNone));
    return (carry | !finite) ? c : (s < c ? s : c);
}

// every thread gets op over the block's values; ident is op's identity (it fills the lanes past the
// block's warp count)
template <class T, class Op>
__device__ __forceinline__ T block_all_reduce(T v, Op op, T ident, T* red) {
    v = op(v, __shfl_xor_sync(0xffffffffu, v, 16));
    v = op(v, __shfl_xor_sync(0xffffffffu, v, 8));
    v = op(v, __shfl_xor_sync(0xffffffffu, v, 4));
    v = op(v, __shfl_xor_sync(0xffffffffu, v, 2));
    v = op(v, __shfl_xor_sync(0xffffffffu, v, 1));
    const unsigned w = threadIdx.x >> 5, l = lane_id(), nw = blockDim.x >> 5;
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        T x = l < nw ? red[l] : ident;
        x = op(x, __shfl_xor_sync(0xffffffffu, x, 16));
        x = op(x, __shfl_xor_sync(0xffffffffu, x, 8));
        x = op(x, __shfl_xor_sync(0xffffffffu, x, 4));
        x = op(x, __shfl_xor_sync(0xffffffffu, x, 2));
        x = op(x, __shfl_xor_sync(0xffffffffu, x, 1));
        if (l == 0) red[32] = x;
    }
    __syncthreads();
    const T r = red[32];
    __syncthreads();
    return r;
}

struct BatchSmem {
    RelaxSmem relax;
    uint32_t relax_next[relax_nbuf_words<kRelaxU>(BT / 32)];
    unsigned long long scratch[33];
    unsigned long long red64[33];
    uint32_t red32[33];
    uint32_t woff[33];
    uint32_t job;
    uint32_t changed[3];
};

// cid[v] = rank of v's center among all centers (block-wide scan); returns k
__device__ uint32_t block_relabel(uint32_t n, const uint32_t* __restrict__ center, uint32_t* __restrict__ rank,
                                  uint32_t* __restrict__ cid, BatchSmem& sm) {
    const unsigned w = threadIdx.x >> 5, l = lane_id(), nw = blockDim.x >> 5;
    uint32_t running = 0;
    for (uint32_t base = 0; base < n; base += blockDim.x) {
        const uint32_t v = base + threadIdx.x;
        const bool f = v < n && __ldcg(&center[v]) == v;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (l == 0) sm.woff[w] = (uint32_t)__popc(bal);
        __syncthreads();
        if (w == 0) {
            const uint32_t c = l < nw ? sm.woff[l] : 0u;  // lanes past the warp count add nothing
            const uint32_t incl = warp_incl_scan(c);
            sm.woff[l] = incl - c;
            if (l == 31) sm.woff[32] = incl;
        }
        __syncthreads();
        if (f) rank[v] = running + sm.woff[w] + (uint32_t)__popc(bal & lanemask_lt());
        running += sm.woff[32];
        __syncthreads();
    }
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) cid[v] = __ldcg(&rank[__ldcg(&center[v])]);
    __syncthreads();
    return running;
}

// exact max finite distance of the k-node quotient held densely in M (row stride k)
__device__ uint32_t block_quotient_diameter(uint32_t k, uint32_t* __restrict__ M, const Workspace& ws,
                                            uint32_t* dyn, BatchSmem& sm, bool& ovf, uint32_t fw_k) {
    if (k <= 1) return 0;
    uint32_t best = 0;
    if (k <= min(fw_k, kSmemFwK)) {
        // Floyd-Warshall in shared memory; row p and column p are fixed during iteration p
        for (uint32_t i = threadIdx.x; i < k * k; i += blockDim.x) dyn[i] = __ldcg(&M[i]);
        __syncthreads();
        for (uint32_t p = 0; p < k; ++p) {
            for (uint32_t idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
                const uint32_t i = idx / k, j = idx - i * k;
                dyn[idx] = relax_min_u32(dyn[idx], dyn[i * k + p], dyn[p * k + j], ovf);
            }
            __syncthreads();
        }
        for (uint32_t i = threadIdx.x; i < k * k; i += blockDim.x)
            if (dyn[i] != kNone && dyn[i] > best) best = dyn[i];
    } else {
        // quotient CSR from M (warp per row, ballot compaction keeps columns sorted), then
        // batched exact SSSP on it
        const unsigned w = threadIdx.x >> 5, l = lane_id(), nw = blockDim.x >> 5;
        for (uint32_t a = w; a < k; a += nw) {
            uint32_t c = 0;
            for (uint32_t b0 = 0; b0 < k; b0 += 32) {
                const uint32_t b = b0 + l;
                c += __popc(__ballot_sync(0xffffffffu, b < k && b != a && __ldcg(&M[a * k + b]) != kNone));
            }
            if (l == 0) ws.qoff[a + 1] = c;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            ws.qoff[0] = 0;
            for (uint32_t a = 0; a < k; ++a) ws.qoff[a + 1] += ws.qoff[a];
        }
        __syncthreads();
        for (uint32_t a = w; a < k; a += nw) {
            uint32_t pos = __ldcg(&ws.qoff[a]);
            for (uint32_t b0 = 0; b0 < k; b0 += 32) {
                const uint32_t b = b0 + l;
                const uint32_t x = (b < k && b != a) ? __ldcg(&M[a * k + b]) : kNone;
                const unsigned bal = __ballot_sync(0xffffffffu, x != kNone);
                if (x != kNone) {
                    const uint32_t at = pos + (uint32_t)__popc(bal & lanemask_lt());
                    ws.qcol[at] = b;
                    ws.qw[at] = x;
                }
                pos += (uint32_t)__popc(bal);
            }
        }
        __syncthreads();
        // worklist multi-source Bellman-Ford, 8 sources at a time: dist[v][s] and one word of change
        // bits per node (two rounds) in shared memory; a changed node pushes to its neighbours
        constexpr uint32_t S = 8;
        uint32_t* dist = dyn;  // k x S
        uint32_t* chg0 = dyn + (size_t)k * S;
        uint32_t* chg1 = chg0 + k;
        for (uint32_t s0 = 0; s0 < k; s0 += S) {
            for (uint32_t i = threadIdx.x; i < k * S; i += blockDim.x) dist[i] = (s0 + i % S == i / S) ? 0u : kNone;
            for (uint32_t v = threadIdx.x; v < k; v += blockDim.x) {
                chg0[v] = (v >= s0 && v < s0 + S) ? 1u << (v - s0) : 0u;
                chg1[v] = 0;
            }
            __syncthreads();
            for (uint32_t round = 0;; ++round) {
                uint32_t* cur = (round & 1) ? chg1 : chg0;
                uint32_t* nxt = (round & 1) ? chg0 : chg1;
                for (uint32_t v = w; v < k; v += nw) {
                    const uint32_t bits = cur[v];
                    if (!bits) continue;
                    const uint32_t beg = __ldcg(&ws.qoff[v]), end = __ldcg(&ws.qoff[v + 1]);
                    for (uint32_t j = beg + l; j < end; j += 32) {
                        const uint32_t u = __ldcg(&ws.qcol[j]), wj = __ldcg(&ws.qw[j]);
                        for (uint32_t b = bits; b; b &= b - 1) {
                            const uint32_t si = (uint32_t)__ffs(b) - 1;
                            const uint32_t dv = dist[v * S + si];
                            if (dv == kNone) continue;
                            const uint64_t nd = (uint64_t)dv + wj;
                            if (nd >= kNone) {
                                ovf = true;
                                continue;
                            }
                            uint32_t* du = &dist[u * S + si];
                            if ((uint32_t)nd < *du && (uint32_t)nd < atomicMin(du, (uint32_t)nd))
                                atomicOr(&nxt[u], 1u << si);
                        }
                    }
                }
                __syncthreads();
                bool any = false;
                for (uint32_t v = threadIdx.x; v < k; v += blockDim.x) {
                    cur[v] = 0;
                    any |= nxt[v] != 0;
                }
                if (!__syncthreads_or(any)) break;
                if (round > k * S + 64) {  // distances only decrease: far above any real count, reported
                    ovf = true;
                    break;
                }
            }
            for (uint32_t i = threadIdx.x; i < k * S; i += blockDim.x)
                if (s0 + i % S < k && dist[i] != kNone && dist[i] > best) best = dist[i];
            __syncthreads();
        }
    }
    __syncthreads();
    return block_all_reduce(best, [](uint32_t a, uint32_t b) { return a > b ? a : b; }, 0u, sm.red32);
}

// One job: CLUSTER + quotient + Phi(G_C) of one arena graph by this CTA; thread 0 stores the result.
// The end of a job on one CTA: singletons, relabel, the dense quotient and Phi(G_C); thread 0 stores
// the result.  `res` holds the CLUSTER counters so far.
__device__ void finish_job(const Job& job, const ArenaDesc& d, const uint64_t* __restrict__ off,
                           const uint2* __restrict__ adj, const uint32_t* __restrict__ row, const Workspace& ws,
                           BatchSmem& sm, uint32_t* dyn, JobOut* out, cldiam_result res, uint32_t status,
                           uint32_t delta) {
    const unsigned tid = threadIdx.x;
    const uint32_t n = d.n;
    if (status == kJobOk) {
        dev_singletons(n, ws.center, ws.D, 0, 1);
        __syncthreads();
        res.delta_end = delta;
        const uint32_t k = block_relabel(n, ws.center, ws.stamp, ws.cid, sm);  // stamp reused as rank
        res.k = k;
        const uint32_t rmax =
            block_all_reduce([&] {
                uint32_t m = 0;
                for (uint32_t v = tid; v < n; v += BT) m = max(m, __ldcg(&ws.D[v]));
                return m;
            }(), [](uint32_t a, uint32_t b) { return a > b ? a : b; }, 0u, sm.red32);
        res.radius = rmax;
        if (k > kDenseCap) {
            status = kJobNeedsPlain;
        } else {
            // weighted quotient graph, deduplicated densely
            uint32_t* M = ws.M;
            for (uint32_t i = tid; i < k * k; i += BT) M[i] = (i / k == i % k) ? 0u : kNone;
            __syncthreads();
            bool ovf = false;
            for (uint64_t i = tid; i < d.nnz; i += BT) {
                const uint32_t u = row[i];
                const uint2 e = adj[i];
                const uint32_t a = __ldcg(&ws.cid[u]), b = __ldcg(&ws.cid[e.x]);
                if (a != b) {
                    uint64_t s = (uint64_t)__ldcg(&ws.D[u]) + e.y + __ldcg(&ws.D[e.x]);
                    if (s >= 0xFFFFFFFFull) {
                        ovf = true;
                        s = 0xFFFFFFFEull;
                    }
                    atomicMin(&M[(size_t)a * k + b], (uint32_t)s);
                }
            }
            __syncthreads();
            const unsigned long long qe = block_all_reduce(
                [&] {
                    unsigned long long c = 0;
                    for (uint32_t i = tid; i < k * k; i += BT) c += (i / k != i % k && __ldcg(&M[i]) != kNone);
                    return c;
                }(),
                [](unsigned long long a, unsigned long long b) { return a + b; }, 0ull, sm.red64);
            res.quotient_edges = qe;
            bool ovf2 = false;
            const uint32_t phi = block_quotient_diameter(k, M, ws, dyn, sm, ovf2, job.fw_k);
            const uint32_t any_ovf = block_all_reduce((uint32_t)(ovf || ovf2),
                                                      [](uint32_t a, uint32_t b) { return a | b; }, 0u, sm.red32);
            if (any_ovf) status = kJobOverflow;
            res.phi_gc = phi;
            res.phi_approx = (uint64_t)phi + 2ull * rmax;
        }
    }
    if (tid == 0) {
        out->r = res;
        out->status = status;
    }
    __syncthreads();
}

__device__ void run_job(const Job& job, const ArenaDesc& d, const uint64_t* __restrict__ arena_off,
                        const uint2* __restrict__ arena_adj, const uint32_t* __restrict__ arena_row,
                        const Workspace& ws, BatchSmem& sm, uint32_t* dyn, JobOut* out) {
    Counters* ctr = ws.ctr;
    volatile Counters* vc = ctr;
    const unsigned tid = threadIdx.x;
    const uint32_t n = d.n;
    const uint64_t* off = arena_off + d.off_base;
    const uint2* adj = arena_adj + d.adj_base;
    const uint32_t* row = arena_row + d.adj_base;
    cldiam_result res;
    memset(&res, 0, sizeof res);
    uint32_t status = kJobOk;

    for (uint32_t v = tid; v < n; v += BT) {
        ws.center[v] = kNone;
        ws.D[v] = 0;
        ws.R[v] = 0;
        ws.stamp[v] = 0;
        ws.key[v] = kInfKey;
    }
    if (tid == 0) memset(ctr, 0, sizeof(Counters));
    __syncthreads();

    uint64_t U = n, frozen_deg = 0, covered = 0;
    uint32_t stage = 1, stepid = 0, delta = job.delta0, cur = 0;
    const bool pull_ok = d.nnz < 0x80000000ull;
    uint32_t nf = 0, E = 0;
    for (;;) {
        uint64_t thr = 0;
        if (!stage_threshold(U, job.tau, job.L, &thr)) break;
        if (stage > kMaxStages) {
            status = kJobDiverged;
            break;
        }
        if (tid == 0) {
            ctr->selected = 0;
            ctr->front = 0;
        }
        __syncthreads();
        dev_select(n, ws.center, ws.key, job.seed, stage, thr, ctr, 0, 1);
        __syncthreads();
        {
            const bool pull = pull_ok && (d.nnz - frozen_deg) < frozen_deg;
            dev_rebuild(n, ws.key, ws.center, job.cumulative ? ws.D : nullptr, off, delta, pull, ws.fbase[cur],
                        ws.fkey[cur], ws.fpre[cur], nullptr,
                        ctr, sm.scratch, 0, 1);
        }
        __syncthreads();
        covered = vc->selected;
        res.centers_drawn += vc->selected;
        nf = (uint32_t)(vc->front >> 32);
        E = (uint32_t)vc->front;
        __syncthreads();
        for (;;) {
            uint32_t updated, growth_steps = 0;
            do {
                ++growth_steps;
                ++stepid;
                updated = 0;
                if (nf > 0) {
                    if (tid == 0) {
                        ctr->newly_covered = 0;
                        ctr->front = 0;
                        ctr->nnext = 0;
                    }
                    __syncthreads();
                    dev_relax<kRelaxU>(ws.fbase[cur], ws.fkey[cur], ws.fpre[cur], nf, E, adj, ws.center,
                                 job.cumulative ? ws.D : nullptr, ws.key,
                                 delta, ws.stamp, stepid, ws.next, ctr, sm.relax, sm.relax_next, 0, 1);
                    __syncthreads();
                    const uint32_t nn = vc->nnext;
                    dev_snapshot(ws.next, nn, ws.key, off, delta, ws.fbase[cur ^ 1], ws.fkey[cur ^ 1],
                                 ws.fpre[cur ^ 1], nullptr, ctr, sm.scratch, 0, 1);
                    __syncthreads();
                    updated = nn;
                    covered += vc->newly_covered;
                    res.edges_scanned += E;
                    nf = (uint32_t)(vc->front >> 32);
                    E = (uint32_t)vc->front;
                    cur ^= 1;
                    __syncthreads();
                }
                res.steps++;
                res.node_updates += updated;
            } while (updated != 0 && 2 * covered < U && (job.step_cap == 0 || growth_steps < job.step_cap));
            if (2 * covered >= U) break;
            bool growable = false;
            if (delta < kDeltaMax && d.connected) {
                growable = covered > 0 || U < n;
            } else if (delta < kDeltaMax && d.nnz) {
                if (tid == 0) ctr->growable = 0;
                __syncthreads();
                dev_growable(row, adj, d.nnz, ws.key, ctr, 0, 1);
                __syncthreads();
                growable = vc->growable != 0;
                __syncthreads();
            }
            if (!growable) {
                res.guard_exits++;
                break;
            }
            delta = (delta > kDeltaMax / 2) ? kDeltaMax : 2 * delta;
            res.doublings++;
            if (tid == 0) ctr->front = 0;
            __syncthreads();
            {
                const bool pull = pull_ok && (d.nnz - frozen_deg) < frozen_deg;
                dev_rebuild(n, ws.key, ws.center, job.cumulative ? ws.D : nullptr, off, delta, pull, ws.fbase[cur],
                        ws.fkey[cur], ws.fpre[cur], nullptr,
                            ctr, sm.scratch, 0, 1);
            }
            __syncthreads();
            nf = (uint32_t)(vc->front >> 32);
            E = (uint32_t)vc->front;
            __syncthreads();
        }
        if (tid == 0) {
            ctr->frozen = 0;
            ctr->frozen_deg = 0;
        }
        __syncthreads();
        dev_finalize_d(n, ws.key, ws.center, job.cumulative ? nullptr : ws.R, ws.D, ctr, 0, 1);
        __syncthreads();
        dev_finalize_freeze(n, ws.key, ws.center, ws.R, ws.D, off, ctr, 0, 1);
        __syncthreads();
        if (vc->overflow) status = kJobOverflow;
        U -= vc->frozen;
        frozen_deg += vc->frozen_deg;
        res.stages++;
        ++stage;
        __syncthreads();
        if (status != kJobOk) break;
    }
    finish_job(job, d, off, adj, row, ws, sm, dyn, out, res, status, delta);
}

__global__ void __launch_bounds__(BT, kBatchCtasPerSm)
    k_batch(const ArenaDesc* __restrict__ descs, const Job* __restrict__ jobs, uint32_t count,
            const uint64_t* __restrict__ arena_off, const uint2* __restrict__ arena_adj,
            const uint32_t* __restrict__ arena_row, Workspace* __restrict__ wss, uint32_t* __restrict__ queue,
            JobOut* __restrict__ outs) {
    extern __shared__ __align__(16) uint32_t dyn[];
    __shared__ BatchSmem sm;
    const Workspace ws = wss[blockIdx.x];
    for (;;) {
        if (threadIdx.x == 0) sm.job = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t j = sm.job;
        __syncthreads();
        if (j >= count) break;
        const Job job = jobs[j];
        const uint64_t t0 = global_ns();
        run_job(job, descs[job.graph], arena_off, arena_adj, arena_row, ws, sm, dyn, &outs[job.out]);
        if (threadIdx.x == 0) {
            outs[job.out].t_start = t0;
            outs[job.out].t_end = global_ns();
        }
    }
}

// ---------------------------------------------------------------------------- serving
// Host-mapped control block of the serving kernel.
struct ServeCtl {
    uint32_t tail;   // requests published by the host (store-release)
    uint32_t stop;   // host asks the CTAs to leave
    uint32_t idle;   // a CTA left after the idle limit with no request
    uint32_t pad;
};

__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(uint32_t* p, uint32_t v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Continuous batching: every CTA takes the next published request as soon as
// it finishes its previous one, so requests that arrive while others run join
// immediately.  Waiting for work is bounded by idle_cycles; the host
// relaunches the kernel when a request arrives after the CTAs left.
__global__ void __launch_bounds__(BT, kBatchCtasPerSm)
    k_serve(const ArenaDesc* __restrict__ descs, const uint64_t* __restrict__ arena_off,
            const uint2* __restrict__ arena_adj, const uint32_t* __restrict__ arena_row,
            Workspace* __restrict__ wss, const Job* ring, ServeCtl* ctl, uint32_t* head, JobOut* outs,
            uint32_t* done, long long idle_cycles) {
    extern __shared__ __align__(16) uint32_t dyn[];
    __shared__ BatchSmem sm;
    __shared__ Job s_job;
    const Workspace ws = wss[blockIdx.x];
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t claimed = kNone;
            const long long t0 = clock64();
            for (;;) {
                const uint32_t t = ld_acquire_sys(&ctl->tail);
                const uint32_t h = atomicAdd(head, 0u);
                if (h < t) {
                    if (atomicCAS(head, h, h + 1) == h) {
                        claimed = h;
                        break;
                    }
                    continue;
                }
                if (ld_acquire_sys(&ctl->stop)) break;
                if (clock64() - t0 > idle_cycles) {
                    atomicExch(&ctl->idle, 1u);
                    break;
                }
                __nanosleep(2000);
            }
            sm.job = claimed;
            if (claimed != kNone) {
                const volatile Job* vj = ring + claimed;
                s_job.tau = vj->tau;
                s_job.L = vj->L;
                s_job.seed = vj->seed;
                s_job.graph = vj->graph;
                s_job.delta0 = vj->delta0;
                s_job.out = vj->out;
                s_job.step_cap = vj->step_cap;
                s_job.cumulative = vj->cumulative;
                s_job.fw_k = vj->fw_k;
            }
        }
        __syncthreads();
        const uint32_t slot = sm.job;
        if (slot == kNone) break;
        const Job job = s_job;
        __syncthreads();
        run_job(job, descs[job.graph], arena_off, arena_adj, arena_row, ws, sm, dyn, &outs[job.out]);
        if (threadIdx.x == 0) {
            __threadfence_system();
            st_release_sys(&done[job.out], 1u);
        }
        __syncthreads();
    }
}

}  // namespace

}  // namespace cld

// ---------------------------------------------------------------------------- arena
struct cldiam_arena {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint64_t budget = 0;
    std::vector<cld::ArenaDesc> graphs;
    std::vector<uint64_t> wsum_upper;
    std::vector<uint32_t> wmin;
    uint64_t* off = nullptr;
    uint2* adj = nullptr;
    uint32_t* row = nullptr;
    uint64_t off_cap = 0, adj_cap = 0, off_used = 0, adj_used = 0;
    void* ws = nullptr;  // cached per-CTA workspaces
    size_t ws_bytes = 0;
    std::vector<double> last_start, last_end;  // per-job device times of the last batch (seconds)
};

namespace cld {

static uint64_t arena_bytes(const cldiam_arena* a) { return a->off_cap * 8 + a->adj_cap * 12 + a->ws_bytes; }

// grow a device array to hold `need` elements (doubling), keeping the first `used`
template <class T>
static cldiam_status grow(T** p, uint64_t* cap, uint64_t used, uint64_t need, cudaStream_t s) {
    if (need <= *cap) return CLDIAM_OK;
    uint64_t nc = std::max<uint64_t>(need, *cap * 2 + 1024);
    T* q = nullptr;
    CLD_TRY(dmalloc(reinterpret_cast<void**>(&q), nc * sizeof(T), s));
    if (used) CLD_CUDA(cudaMemcpyAsync(q, *p, used * sizeof(T), cudaMemcpyDeviceToDevice, s));
    dfree(*p, s);
    *p = q;
    *cap = nc;
    return CLDIAM_OK;
}

cldiam_status arena_create(uint64_t budget, cudaStream_t s, cldiam_arena** out) {
    if (!out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL out");
    cldiam_arena* a = new cldiam_arena();
    cudaGetDevice(&a->device);
    a->stream = s;
    a->budget = budget;
    *out = a;
    return CLDIAM_OK;
}

void arena_free(cldiam_arena* a) {
    if (!a) return;
    dfree(a->off, a->stream);
    dfree(a->adj, a->stream);
    dfree(a->row, a->stream);
    dfree(a->ws, a->stream);
    cudaStreamSynchronize(a->stream);
    delete a;
}

cldiam_status arena_add(cldiam_arena* a, const uint32_t* src, const uint32_t* dst, const uint32_t* w, uint64_t m,
                        uint32_t n, uint32_t flags, uint32_t* id) {
    if (!a || !id) return fail(CLDIAM_ERR_INVALID_ARG, "NULL arena or id");
    cldiam_graph* g = nullptr;
    CLD_TRY(build_csr(src, dst, w, m, n, flags, a->stream, &g));
    struct Free {
        cldiam_graph* g;
        ~Free() { free_graph(g); }
    } fg{g};
    const uint64_t need_off = a->off_used + g->n + 1, need_adj = a->adj_used + g->nnz;
    const uint64_t extra = (need_off > a->off_cap ? (need_off - a->off_cap) * 8 : 0) +
                           (need_adj > a->adj_cap ? (need_adj - a->adj_cap) * 12 : 0);
    if (a->budget && arena_bytes(a) + extra > a->budget)
        return fail(CLDIAM_ERR_OOM, "graph does not fit the arena's device memory budget");
    CLD_TRY(grow(&a->off, &a->off_cap, a->off_used, need_off, a->stream));
    {
        uint64_t cap = a->adj_cap;
        CLD_TRY(grow(&a->adj, &cap, a->adj_used, need_adj, a->stream));
        uint64_t cap2 = a->adj_cap;
        CLD_TRY(grow(&a->row, &cap2, a->adj_used, need_adj, a->stream));
        a->adj_cap = std::max(cap, cap2);
    }
    CLD_CUDA(cudaMemcpyAsync(a->off + a->off_used, g->off, (g->n + 1) * 8, cudaMemcpyDeviceToDevice, a->stream));
    if (g->nnz) {
        CLD_CUDA(cudaMemcpyAsync(a->adj + a->adj_used, g->adj, g->nnz * 8, cudaMemcpyDeviceToDevice, a->stream));
        if (g->row) {
            CLD_CUDA(cudaMemcpyAsync(a->row + a->adj_used, g->row, g->nnz * 4, cudaMemcpyDeviceToDevice, a->stream));
        } else {
            CLD_TRY(fill_rows(g->off, g->n, a->row + a->adj_used, a->stream));
        }
    }
    ArenaDesc dsc{};
    dsc.off_base = a->off_used;
    dsc.adj_base = a->adj_used;
    dsc.nnz = g->nnz;
    dsc.n = g->n;
    dsc.connected = g->connected ? 1u : 0u;
    a->graphs.push_back(dsc);
    a->wsum_upper.push_back(g->wsum_upper);
    a->wmin.push_back(g->wmin);
    a->off_used = need_off;
    a->adj_used = need_adj;
    *id = (uint32_t)(a->graphs.size() - 1);
    CLD_CUDA(cudaStreamSynchronize(a->stream));
    return CLDIAM_OK;
}

// a non-owning graph handle over one arena graph (for the one-graph path)
static void arena_view(const cldiam_arena* a, uint32_t id, cldiam_graph* g) {
    const ArenaDesc& d = a->graphs[id];
    g->device = a->device;
    g->stream = a->stream;
    g->n = d.n;
    g->nnz = d.nnz;
    g->off = a->off + d.off_base;
    g->adj = a->adj + d.adj_base;
    g->row = a->row + d.adj_base;
    g->orig = nullptr;
    g->wsum_upper = a->wsum_upper[id];
    g->wmin = a->wmin[id];
    g->connected = d.connected != 0;
    g->borrowed = true;
}

cldiam_status arena_graph(cldiam_arena* a, uint32_t id, cldiam_graph** out) {
    if (!a || !out || id >= a->graphs.size()) return fail(CLDIAM_ERR_INVALID_ARG, "bad arena or graph id");
    cldiam_graph* g = new cldiam_graph();
    arena_view(a, id, g);
    CLD_TRY(g->host.alloc(256));
    *out = g;
    return CLDIAM_OK;
}

uint32_t arena_count(const cldiam_arena* a) { return (uint32_t)a->graphs.size(); }
cudaStream_t arena_stream(const cldiam_arena* a) { return a->stream; }
cldiam_status arena_job_times(const cldiam_arena* a, uint32_t count, double* start_s, double* end_s) {
    if (!a || (count && (!start_s || !end_s))) return fail(CLDIAM_ERR_INVALID_ARG, "NULL argument");
    if (count > a->last_start.size()) return fail(CLDIAM_ERR_INVALID_ARG, "count exceeds the last batch");
    for (uint32_t i = 0; i < count; ++i) {
        start_s[i] = a->last_start[i];
        end_s[i] = a->last_end[i];
    }
    return CLDIAM_OK;
}
uint64_t arena_entries(const cldiam_arena* a, const uint32_t* ids, uint32_t count) {
    uint64_t e = 0;
    for (uint32_t i = 0; i < count; ++i)
        if (ids[i] < a->graphs.size()) e += a->graphs[ids[i]].nnz;
    return e;
}
uint64_t arena_device_bytes(const cldiam_arena* a) { return arena_bytes(a); }

// Per-CTA workspaces for graphs of up to nmax nodes, carved from one (cached) device buffer.
static cldiam_status make_workspaces(uint32_t nmax, int ctas, cudaStream_t s, void** buf, size_t* buf_bytes,
                                     std::vector<Workspace>* out) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t n8 = al((size_t)nmax * 8), n4 = al((size_t)nmax * 4), f8 = al((size_t)nmax * 16),
                 f4 = al((size_t)nmax * 8), mm = al((size_t)kDenseCap * kDenseCap * 4),
                 qo = al(((size_t)kDenseCap + 1) * 4), ctrb = al(sizeof(Counters));
    const size_t slice = n8 + 2 * f8 + 6 * n4 + 4 * f4 + mm + qo + 2 * mm + ctrb;
    const size_t need = slice * ctas;
    if (need > *buf_bytes) {
        dfree(*buf, s);
        *buf = nullptr;
        *buf_bytes = 0;
        CLD_TRY(dmalloc(buf, need, s));
        *buf_bytes = need;
    }
    out->assign(ctas, Workspace{});
    for (int b = 0; b < ctas; ++b) {
        char* p = static_cast<char*>(*buf) + (size_t)b * slice;
        Workspace& w = (*out)[b];
        w.key = reinterpret_cast<unsigned long long*>(p); p += n8;
        w.fkey[0] = reinterpret_cast<unsigned long long*>(p); p += f8;
        w.fkey[1] = reinterpret_cast<unsigned long long*>(p); p += f8;
        w.center = reinterpret_cast<uint32_t*>(p); p += n4;
        w.D = reinterpret_cast<uint32_t*>(p); p += n4;
        w.R = reinterpret_cast<uint32_t*>(p); p += n4;
        w.stamp = reinterpret_cast<uint32_t*>(p); p += n4;
        w.next = reinterpret_cast<uint32_t*>(p); p += n4;
        w.cid = reinterpret_cast<uint32_t*>(p); p += n4;
        w.fbase[0] = reinterpret_cast<uint32_t*>(p); p += f4;
        w.fbase[1] = reinterpret_cast<uint32_t*>(p); p += f4;
        w.fpre[0] = reinterpret_cast<uint32_t*>(p); p += f4;
        w.fpre[1] = reinterpret_cast<uint32_t*>(p); p += f4;
        w.M = reinterpret_cast<uint32_t*>(p); p += mm;
        w.qoff = reinterpret_cast<uint32_t*>(p); p += qo;
        w.qcol = reinterpret_cast<uint32_t*>(p); p += mm;
        w.qw = reinterpret_cast<uint32_t*>(p); p += mm;
        w.ctr = reinterpret_cast<Counters*>(p);
    }
    return CLDIAM_OK;
}

struct CudaEvent {
    cudaEvent_t e = nullptr;
    cldiam_status create() {
        CLD_CUDA(cudaEventCreate(&e));
        return CLDIAM_OK;
    }
    ~CudaEvent() {
        if (e) cudaEventDestroy(e);
    }
};

static size_t batch_dyn_smem() {
    // shared Floyd-Warshall matrix, or the quotient SSSP's k x 8 distances and two words of change bits per node
    return std::max<size_t>((size_t)kSmemFwK * kSmemFwK * 4, (size_t)kDenseCap * (8 * 4 + 8));
}

template <class Kern>
static cldiam_status set_dyn_smem(Kern k, std::atomic<bool>* done_flags) {
    int dev = 0;
    CLD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !done_flags[dev]) {
        CLD_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_dyn_smem()));
        if (kBatchCtasPerSm > 1)  // room for several CTAs' shared memory on one SM
            CLD_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared));
        if (dev >= 0 && dev < 64) done_flags[dev] = true;
    }
    return CLDIAM_OK;
}

// CTAs of a persistent many-graph kernel resident on one SM: kBatchCtasPerSm when they fit, else what does
template <class Kern>
static cldiam_status resident_per_sm(Kern k, std::atomic<bool>* done_flags, int* out) {
    CLD_TRY(set_dyn_smem(k, done_flags));
    int nb = 0;
    CLD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, BT, batch_dyn_smem()));
    *out = std::max(1, std::min(nb, kBatchCtasPerSm));
    return CLDIAM_OK;
}

cldiam_status batch_run(cldiam_arena* a, const uint32_t* ids, const double* tau, const uint64_t* seed, uint32_t count,
                        const cldiam_opts* o, cldiam_result* out, cldiam_status* status) {
    if (!a || (count && (!ids || !tau || !seed || !out))) return fail(CLDIAM_ERR_INVALID_ARG, "NULL argument");
    if (count == 0) return CLDIAM_OK;
    cldiam_opts opts{};
    if (o) opts = *o;
    if (opts.contract_mode != CLDIAM_CONTRACT_RESET && opts.contract_mode != CLDIAM_CONTRACT_CUMULATIVE)
        return fail(CLDIAM_ERR_INVALID_ARG, "unknown contract_mode");
    if (opts.reserved[0] || opts.reserved[1]) return fail(CLDIAM_ERR_INVALID_ARG, "reserved options must be 0");
    const cudaStream_t s = a->stream;
    const uint32_t fw_k = tuning_for_batch(arena_entries(a, ids, count)).batch_fw_k;
    std::vector<Job> jobs(count);
    for (uint32_t i = 0; i < count; ++i) {
        if (ids[i] >= a->graphs.size()) return fail(CLDIAM_ERR_INVALID_ARG, "graph id out of range");
        if (!(tau[i] > 0.0) || !std::isfinite(tau[i])) return fail(CLDIAM_ERR_INVALID_ARG, "tau must be positive");
        cldiam_graph view;
        arena_view(a, ids[i], &view);
        uint32_t d0 = 0;
        CLD_TRY(delta0(&view, opts.delta0_mode, opts.delta0, &d0));
        jobs[i].tau = tau[i];
        jobs[i].L = std::log2((double)view.n);
        jobs[i].seed = seed[i];
        jobs[i].graph = ids[i];
        jobs[i].delta0 = d0;
        jobs[i].out = i;
        jobs[i].step_cap = opts.step_cap;
        jobs[i].cumulative = opts.contract_mode == CLDIAM_CONTRACT_CUMULATIVE ? 1u : 0u;
        jobs[i].fw_k = fw_k;
    }
    // largest graphs first: the work queue then balances the tail
    std::stable_sort(jobs.begin(), jobs.end(), [&](const Job& x, const Job& y) {
        return a->graphs[x.graph].nnz + a->graphs[x.graph].n > a->graphs[y.graph].nnz + a->graphs[y.graph].n;
    });
    static std::atomic<bool> attr[64];
    int cps = 1;
    CLD_TRY(resident_per_sm(k_batch, attr, &cps));
    const int nsm = num_sms() * cps;  // CTAs of the launch
    // The launch ends with its largest graph on one CTA, or with the even split of all work over the CTAs,
    // whichever is later.  The k largest graphs can instead run first on the one-graph path, each with the
    // whole device at a fixed cost per graph; k is chosen to minimise the estimated makespan
    // (batch_split = 2; 1 keeps every graph in the launch).  Work = adjacency entries + nodes.
    const uint32_t split = tuning_for_batch(arena_entries(a, ids, count)).batch_split;
    std::vector<double> cost(count);
    double rest = 0.0;
    for (uint32_t j = 0; j < count; ++j) {
        cost[j] = (double)(a->graphs[jobs[j].graph].nnz + a->graphs[jobs[j].graph].n);
        rest += cost[j];
    }
    uint32_t nbig = 0;  // jobs[0 .. nbig) take the one-graph path (largest first, so a prefix)
    if (split == 2) {
        const auto launch_s = [&](uint32_t k, double rest_work) {
            return k < count ? std::max(cost[k] * kCtaSecPerUnit, rest_work * kCtaSecPerUnit / nsm) : 0.0;
        };
        double plain_s = 0.0, best = launch_s(0, rest);
        for (uint32_t k = 1; k <= count && a->graphs[jobs[k - 1].graph].nnz >= kSplitMinEntries; ++k) {
            plain_s += kPlainSecPerGraph + cost[k - 1] * kPlainSecPerUnit;
            rest -= cost[k - 1];
            const double t = plain_s + launch_s(k, rest);
            if (t < best) {
                best = t;
                nbig = k;
            }
        }
    }
    a->last_start.assign(count, 0.0);
    a->last_end.assign(count, 0.0);
    std::vector<JobOut> ho(count);
    for (auto& h : ho) h.status = kJobOk;
    double big_s = 0.0;  // device time of the one-graph runs, the offset of the launch's job times
    std::vector<cldiam_status> big_st(count, CLDIAM_OK);
    if (nbig > 0) {
        CudaEvent e0, e1;
        CLD_TRY(e0.create());
        CLD_TRY(e1.create());
        for (uint32_t j = 0; j < nbig; ++j) {
            const uint32_t i = jobs[j].out;
            cldiam_graph view;
            arena_view(a, ids[i], &view);
            CLD_TRY(view.host.alloc(256));
            CLD_CUDA(cudaEventRecord(e0.e, s));
            cldiam_clustering* c = nullptr;
            cldiam_quotient* q = nullptr;
            cldiam_status st = cluster(&view, tau[i], seed[i], &opts, &c);
            if (st == CLDIAM_OK) st = quotient(c, &q);
            if (st == CLDIAM_OK) st = cldiam_estimate(q, &ho[i].r);
            free_quotient(q);
            free_clustering(c);
            CLD_CUDA(cudaEventRecord(e1.e, s));
            CLD_CUDA(cudaEventSynchronize(e1.e));
            float ms = 0.f;
            CLD_CUDA(cudaEventElapsedTime(&ms, e0.e, e1.e));
            a->last_start[i] = big_s;
            big_s += ms * 1e-3;
            a->last_end[i] = big_s;
            big_st[i] = st;
        }
    }
    const uint32_t nrest = count - nbig;
    if (nrest > 0) {
        uint32_t nmax_rest = 1;
        for (uint32_t j = nbig; j < count; ++j) nmax_rest = std::max(nmax_rest, a->graphs[jobs[j].graph].n);
        std::vector<Workspace> wsh;
        CLD_TRY(make_workspaces(nmax_rest, nsm, s, &a->ws, &a->ws_bytes, &wsh));
        DBuf<ArenaDesc> ddesc;
        DBuf<Job> djobs;
        DBuf<Workspace> dws;
        DBuf<uint32_t> queue;
        DBuf<JobOut> douts;
        CLD_TRY(ddesc.alloc(a->graphs.size(), s));
        CLD_TRY(djobs.alloc(nrest, s));
        CLD_TRY(dws.alloc(nsm, s));
        CLD_TRY(queue.alloc(1, s));
        CLD_TRY(douts.alloc(count, s));
        CLD_CUDA(cudaMemcpyAsync(ddesc.get(), a->graphs.data(), a->graphs.size() * sizeof(ArenaDesc),
                                 cudaMemcpyHostToDevice, s));
        CLD_CUDA(cudaMemcpyAsync(djobs.get(), jobs.data() + nbig, nrest * sizeof(Job), cudaMemcpyHostToDevice, s));
        CLD_CUDA(cudaMemcpyAsync(dws.get(), wsh.data(), nsm * sizeof(Workspace), cudaMemcpyHostToDevice, s));
        CLD_CUDA(cudaMemsetAsync(queue.get(), 0, 4, s));
        const size_t dyn = batch_dyn_smem();
        CLD_K(K_MISC, s, k_batch<<<nsm, BT, dyn, s>>>(ddesc.get(), djobs.get(), nrest, a->off, a->adj, a->row, dws.get(),
                                                       queue.get(), douts.get()));
        CLD_LAUNCH_CHECK();
        std::vector<JobOut> hl(count);
        CLD_CUDA(cudaMemcpyAsync(hl.data(), douts.get(), count * sizeof(JobOut), cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        // per-job device times of the launch, relative to its first job's start, after the one-graph runs
        uint64_t t0 = ~0ull;
        for (uint32_t j = nbig; j < count; ++j) t0 = std::min(t0, hl[jobs[j].out].t_start);
        for (uint32_t j = nbig; j < count; ++j) {
            const uint32_t i = jobs[j].out;
            ho[i] = hl[i];
            a->last_start[i] = big_s + (double)(hl[i].t_start - t0) * 1e-9;
            a->last_end[i] = big_s + (double)(hl[i].t_end - t0) * 1e-9;
        }
    }
    cldiam_status first_err = CLDIAM_OK;
    for (uint32_t i = 0; i < count; ++i) {
        cldiam_status st = big_st[i];
        if (ho[i].status == kJobNeedsPlain) {
            // quotient larger than the dense capacity: finish this graph with the one-graph path
            cldiam_graph view;
            arena_view(a, ids[i], &view);
            CLD_TRY(view.host.alloc(256));
            cldiam_clustering* c = nullptr;
            cldiam_quotient* q = nullptr;
            st = cluster(&view, tau[i], seed[i], &opts, &c);
            if (st == CLDIAM_OK) st = quotient(c, &q);
            if (st == CLDIAM_OK) st = cldiam_estimate(q, &ho[i].r);
            free_quotient(q);
            free_clustering(c);
        } else if (ho[i].status == kJobOverflow) {
            st = CLDIAM_ERR_OVERFLOW;
        } else if (ho[i].status == kJobDiverged) {
            st = CLDIAM_ERR_DIVERGED;
        } else if (ho[i].status != kJobOk) {
            st = CLDIAM_ERR_TIMEOUT;
        }
        out[i] = ho[i].r;
        if (status) status[i] = st;
        if (st != CLDIAM_OK && first_err == CLDIAM_OK) first_err = st;
    }
    if (first_err != CLDIAM_OK) return fail(first_err, "one or more graphs of the batch failed (see status[])");
    return CLDIAM_OK;
}

// ---------------------------------------------------------------------------- server
namespace {
inline void host_store_release(uint32_t* p, uint32_t v) { __atomic_store_n(p, v, __ATOMIC_RELEASE); }
inline uint32_t host_load_acquire(const uint32_t* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
}  // namespace

}  // namespace cld

struct cldiam_server {
    cldiam_arena* arena = nullptr;
    int device = 0;
    cudaStream_t kstream = nullptr, bstream = nullptr;
    uint32_t ctas = 0, cap = 0, big_nodes = 0;
    uint64_t budget = 0;
    long long idle_cycles = 0;
    // host-mapped (pinned) memory, shared with the serving kernel
    cld::ServeCtl* ctl = nullptr;
    cld::Job* ring = nullptr;
    cld::JobOut* outs = nullptr;
    uint32_t* done = nullptr;
    // device memory
    uint32_t* head = nullptr;
    cld::Workspace* wss = nullptr;
    cld::ArenaDesc* descs = nullptr;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // host state
    std::mutex mu;
    uint32_t next_ticket = 0, next_ring = 0;
    bool kernel_live = false;
    std::vector<uint32_t> big_graph;
    std::vector<double> big_tau;
    std::vector<uint64_t> big_seed;
    std::thread big;
    std::mutex bmu;
    std::condition_variable bcv;
    std::deque<uint32_t> bq;
    bool bstop = false;
    cld::Pinned bhost;  // counter block of the big lane's one-graph runs
};

namespace cld {

static std::atomic<bool> g_serve_attr[64];

static cldiam_status server_launch(cldiam_server* sv) {
    CLD_TRY(set_dyn_smem(k_serve, g_serve_attr));
    sv->ctl->idle = 0;
    CLD_K(K_MISC, sv->kstream,
          k_serve<<<sv->ctas, BT, batch_dyn_smem(), sv->kstream>>>(sv->descs, sv->arena->off, sv->arena->adj,
                                                                   sv->arena->row, sv->wss, sv->ring, sv->ctl,
                                                                   sv->head, sv->outs, sv->done, sv->idle_cycles));
    CLD_LAUNCH_CHECK();
    sv->kernel_live = true;
    return CLDIAM_OK;
}

// relaunch the serving kernel if its CTAs left after the idle limit (caller holds sv->mu)
static cldiam_status server_ensure_live(cldiam_server* sv) {
    if (sv->kernel_live) {
        cudaError_t q = cudaStreamQuery(sv->kstream);
        if (q == cudaErrorNotReady) return CLDIAM_OK;
        if (q != cudaSuccess) return cuda_fail(q, "serving kernel", __FILE__, __LINE__);
        sv->kernel_live = false;
    }
    return server_launch(sv);
}

static void big_lane(cldiam_server* sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        uint32_t t;
        {
            std::unique_lock<std::mutex> lk(sv->bmu);
            sv->bcv.wait(lk, [&] { return sv->bstop || !sv->bq.empty(); });
            if (sv->bq.empty()) return;
            t = sv->bq.front();
            sv->bq.pop_front();
        }
        cldiam_graph view;
        arena_view(sv->arena, sv->big_graph[t], &view);
        view.stream = sv->bstream;
        view.host.h = sv->bhost.h;  // borrowed pinned block; released with the server
        cldiam_result r{};
        cldiam_status st = CLDIAM_OK;
        // admission by device memory: the one-graph path needs ~100 B per node plus ~40 B per entry
        const uint64_t need = (uint64_t)view.n * 100 + view.nnz * 40;
        if (sv->budget && arena_bytes(sv->arena) + sv->ws_bytes + need > sv->budget) {
            st = fail(CLDIAM_ERR_OOM, "request does not fit the server's device memory budget");
        } else {
            cldiam_clustering* c = nullptr;
            cldiam_quotient* q = nullptr;
            cldiam_opts o{};
            st = cluster(&view, sv->big_tau[t], sv->big_seed[t], &o, &c);
            if (st == CLDIAM_OK) st = quotient(c, &q);
            if (st == CLDIAM_OK) st = cldiam_estimate(q, &r);
            free_quotient(q);
            free_clustering(c);
        }
        view.host.h = nullptr;
        sv->outs[t].r = r;
        sv->outs[t].status = st == CLDIAM_OK ? kJobOk
                             : st == CLDIAM_ERR_OVERFLOW ? kJobOverflow
                             : st == CLDIAM_ERR_DIVERGED ? kJobDiverged : kJobTimeout;
        host_store_release(&sv->done[t], 1u);
    }
}

cldiam_status server_free(cldiam_server* sv);

// Servers alive in this process: while one is, its persistent kernel may hold SMs, so CLUSTER keeps its
// host-driven stage loop (a cooperative launch would wait for every SM).

cldiam_status server_create(cldiam_arena* a, const cldiam_server_opts* o, cldiam_server** out) {
    if (!a || !out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL arena or out");
    *out = nullptr;
    cldiam_server_opts opts{};
    if (o) opts = *o;
    cldiam_server* sv = new cldiam_server();
    sv->arena = a;
    CLD_CUDA(cudaGetDevice(&sv->device));
    const int nsm = num_sms();
    int cps = 1;
    if (cldiam_status st = resident_per_sm(k_serve, g_serve_attr, &cps); st != CLDIAM_OK) {
        delete sv;
        return st;
    }
    sv->ctas = opts.ctas ? std::min<uint32_t>(opts.ctas, (uint32_t)(nsm * cps)) : (uint32_t)(std::max(1, nsm - 24) * cps);
    sv->cap = opts.capacity ? opts.capacity : (1u << 20);
    sv->big_nodes = opts.big_nodes ? opts.big_nodes : (1u << 19);
    sv->budget = opts.hbm_budget_bytes;
    int khz = 0;
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, sv->device);
    const double idle_s = opts.idle_seconds > 0 ? opts.idle_seconds : 10.0;
    sv->idle_cycles = (long long)(idle_s * (khz > 0 ? khz : 2000000) * 1e3);
    auto cleanup = [&](cldiam_status st) {
        server_free(sv);
        return st;
    };
    if (cudaStreamCreateWithFlags(&sv->kstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sv->bstream, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup(fail(CLDIAM_ERR_CUDA, "stream creation failed"));
    void* p = nullptr;
    const size_t host_bytes = sizeof(ServeCtl) + (size_t)sv->cap * (sizeof(Job) + sizeof(JobOut) + sizeof(uint32_t));
    if (cudaHostAlloc(&p, host_bytes, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(CLDIAM_ERR_OOM, "pinned host memory for the request ring"));
    }
    memset(p, 0, host_bytes);
    char* c = static_cast<char*>(p);
    sv->ctl = reinterpret_cast<ServeCtl*>(c); c += sizeof(ServeCtl);
    sv->ring = reinterpret_cast<Job*>(c); c += (size_t)sv->cap * sizeof(Job);
    sv->outs = reinterpret_cast<JobOut*>(c); c += (size_t)sv->cap * sizeof(JobOut);
    sv->done = reinterpret_cast<uint32_t*>(c);
    cldiam_status st = sv->bhost.alloc(256);
    if (st != CLDIAM_OK) return cleanup(st);
    // device state: descriptors, head counter, workspaces for the graphs the kernel serves
    uint32_t nmax = 1;
    for (const ArenaDesc& d : a->graphs)
        if (d.n <= sv->big_nodes) nmax = std::max(nmax, d.n);
    std::vector<Workspace> wsh;
    if ((st = make_workspaces(nmax, (int)sv->ctas, sv->kstream, &sv->ws, &sv->ws_bytes, &wsh)) != CLDIAM_OK)
        return cleanup(st);
    if (sv->budget && arena_bytes(a) + sv->ws_bytes > sv->budget)
        return cleanup(fail(CLDIAM_ERR_OOM, "arena plus serving workspace exceed the budget"));
    if ((st = dmalloc((void**)&sv->head, 4, sv->kstream)) != CLDIAM_OK ||
        (st = dmalloc((void**)&sv->wss, wsh.size() * sizeof(Workspace), sv->kstream)) != CLDIAM_OK ||
        (st = dmalloc((void**)&sv->descs, std::max<size_t>(1, a->graphs.size()) * sizeof(ArenaDesc), sv->kstream)) !=
            CLDIAM_OK)
        return cleanup(st);
    cudaMemsetAsync(sv->head, 0, 4, sv->kstream);
    cudaMemcpyAsync(sv->wss, wsh.data(), wsh.size() * sizeof(Workspace), cudaMemcpyHostToDevice, sv->kstream);
    if (!a->graphs.empty())
        cudaMemcpyAsync(sv->descs, a->graphs.data(), a->graphs.size() * sizeof(ArenaDesc), cudaMemcpyHostToDevice,
                        sv->kstream);
    if (cudaStreamSynchronize(sv->kstream) != cudaSuccess) return cleanup(fail(CLDIAM_ERR_CUDA, "server set-up"));
    sv->big_graph.resize(sv->cap);
    sv->big_tau.resize(sv->cap);
    sv->big_seed.resize(sv->cap);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if ((st = server_launch(sv)) != CLDIAM_OK) return cleanup(st);
    }
    sv->big = std::thread(big_lane, sv);
    *out = sv;
    return CLDIAM_OK;
}

cldiam_status server_submit(cldiam_server* sv, uint32_t graph_id, double tau, uint64_t seed, uint64_t* ticket) {
    if (!sv || !ticket) return fail(CLDIAM_ERR_INVALID_ARG, "NULL server or ticket");
    if (graph_id >= sv->arena->graphs.size()) return fail(CLDIAM_ERR_INVALID_ARG, "graph id out of range");
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(CLDIAM_ERR_INVALID_ARG, "tau must be positive");
    cldiam_graph view;
    arena_view(sv->arena, graph_id, &view);
    uint32_t d0 = 0;
    CLD_TRY(delta0(&view, CLDIAM_DELTA0_AVG, 0, &d0));
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->next_ticket >= sv->cap) return fail(CLDIAM_ERR_BUSY, "server request capacity exhausted");
    const uint32_t t = sv->next_ticket++;
    if (view.n > sv->big_nodes) {
        // large graph: the one-graph path on the big-lane stream, using the SMs the kernel leaves free
        sv->big_graph[t] = graph_id;
        sv->big_tau[t] = tau;
        sv->big_seed[t] = seed;
        {
            std::lock_guard<std::mutex> bl(sv->bmu);
            sv->bq.push_back(t);
        }
        sv->bcv.notify_one();
    } else {
        Job j{};
        j.tau = tau;
        j.L = std::log2((double)view.n);
        j.seed = seed;
        j.graph = graph_id;
        j.delta0 = d0;
        j.out = t;
        j.fw_k = tuning_for_batch(sv->arena->adj_used).batch_fw_k;
        sv->ring[sv->next_ring] = j;
        host_store_release(&sv->ctl->tail, ++sv->next_ring);  // publish after the entry is written
        CLD_TRY(server_ensure_live(sv));
    }
    *ticket = t;
    return CLDIAM_OK;
}

cldiam_status server_poll(cldiam_server* sv, uint64_t ticket, cldiam_result* out) {
    if (!sv || !out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL server or out");
    if (ticket >= sv->next_ticket) return fail(CLDIAM_ERR_INVALID_ARG, "unknown ticket");
    if (!host_load_acquire(&sv->done[ticket])) {
        std::lock_guard<std::mutex> lk(sv->mu);
        CLD_TRY(server_ensure_live(sv));
        return CLDIAM_ERR_BUSY;
    }
    *out = sv->outs[ticket].r;
    switch (sv->outs[ticket].status) {
        case kJobOk: return CLDIAM_OK;
        case kJobOverflow: return fail(CLDIAM_ERR_OVERFLOW, "distance overflow");
        case kJobDiverged: return fail(CLDIAM_ERR_DIVERGED, "stage limit exceeded");
        case kJobNeedsPlain: return fail(CLDIAM_ERR_UNSUPPORTED, "quotient above the serving kernel's capacity");
        default: return fail(CLDIAM_ERR_TIMEOUT, "request failed");
    }
}

cldiam_status server_free(cldiam_server* sv) {
    if (!sv) return CLDIAM_OK;
    if (sv->ctl) host_store_release(&sv->ctl->stop, 1u);
    if (sv->big.joinable()) {
        {
            std::lock_guard<std::mutex> bl(sv->bmu);
            sv->bstop = true;
        }
        sv->bcv.notify_all();
        sv->big.join();
    }
    if (sv->kstream) cudaStreamSynchronize(sv->kstream);
    if (sv->bstream) cudaStreamSynchronize(sv->bstream);
    dfree(sv->head, sv->kstream);
    dfree(sv->wss, sv->kstream);
    dfree(sv->descs, sv->kstream);
    dfree(sv->ws, sv->kstream);
    if (sv->kstream) cudaStreamSynchronize(sv->kstream);
    if (sv->ctl) cudaFreeHost(sv->ctl);
    if (sv->kstream) cudaStreamDestroy(sv->kstream);
    if (sv->bstream) cudaStreamDestroy(sv->bstream);
    delete sv;
    return CLDIAM_OK;
}

// Replay an arrival trace: request i is submitted at arrival[i] seconds after the start and its
// latency is completion minus arrival.  plain != 0 serves the same trace one request at a time
// in arrival order on the one-graph path instead (the one-query-per-call baseline).
cldiam_status server_replay(cldiam_server* sv, const uint32_t* ids, const double* tau, const uint64_t* seed,
                            const double* arrival, uint32_t count, int plain, cldiam_result* out, double* latency,
                            double* elapsed) {
    using clk = std::chrono::steady_clock;
    if (!sv || (count && (!ids || !tau || !seed || !arrival || !out || !latency)))
        return fail(CLDIAM_ERR_INVALID_ARG, "NULL argument");
    const auto t0 = clk::now();
    auto since = [&](clk::time_point t) { return std::chrono::duration<double>(t - t0).count(); };
    auto wait_until = [&](double at) {
        for (;;) {
            const double now = since(clk::now());
            if (now >= at) return;
            if (at - now > 200e-6) std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
    };
    cldiam_status first = CLDIAM_OK;
    if (plain) {
        cldiam_graph view;
        for (uint32_t i = 0; i < count; ++i) {
            wait_until(arrival[i]);
            arena_view(sv->arena, ids[i], &view);
            view.stream = sv->bstream;
            view.host.h = sv->bhost.h;
            cldiam_clustering* c = nullptr;
            cldiam_quotient* q = nullptr;
            cldiam_opts o{};
            cldiam_status st = cluster(&view, tau[i], seed[i], &o, &c);
            if (st == CLDIAM_OK) st = quotient(c, &q);
            if (st == CLDIAM_OK) st = cldiam_estimate(q, &out[i]);
            free_quotient(q);
            free_clustering(c);
            view.host.h = nullptr;
            latency[i] = since(clk::now()) - arrival[i];
            if (st != CLDIAM_OK && first == CLDIAM_OK) first = st;
        }
    } else {
        std::vector<uint64_t> tickets(count, ~0ull);
        std::atomic<uint32_t> submitted{0};
        cldiam_status sub_err = CLDIAM_OK;
        std::thread submitter([&] {
            cudaSetDevice(sv->device);
            for (uint32_t i = 0; i < count; ++i) {
                wait_until(arrival[i]);
                uint64_t t = 0;
                cldiam_status st = server_submit(sv, ids[i], tau[i], seed[i], &t);
                if (st != CLDIAM_OK) {
                    sub_err = st;
                    break;
                }
                tickets[i] = t;
                submitted.store(i + 1, std::memory_order_release);
            }
        });
        std::vector<uint32_t> pending;
        uint32_t seen = 0, finished = 0;
        while (finished < count) {
            const uint32_t s = submitted.load(std::memory_order_acquire);
            while (seen < s) pending.push_back(seen++);
            if (sub_err != CLDIAM_OK && pending.empty()) break;
            size_t keep = 0;
            for (uint32_t i : pending) {
                if (host_load_acquire(&sv->done[tickets[i]])) {
                    latency[i] = since(clk::now()) - arrival[i];
                    cldiam_status st = server_poll(sv, tickets[i], &out[i]);
                    if (st != CLDIAM_OK && first == CLDIAM_OK) first = st;
                    ++finished;
                } else {
                    pending[keep++] = i;
                }
            }
            const bool progressed = keep < pending.size();
            pending.resize(keep);
            static thread_local auto last_check = clk::now();
            if (!pending.empty() && !progressed && clk::now() - last_check > std::chrono::milliseconds(1)) {
                last_check = clk::now();
                std::lock_guard<std::mutex> lk(sv->mu);
                CLD_TRY(server_ensure_live(sv));
            }
        }
        submitter.join();
        if (sub_err != CLDIAM_OK) return sub_err;
    }
    if (elapsed) *elapsed = since(clk::now());
    if (first != CLDIAM_OK) return first;
    return CLDIAM_OK;
}

}  // namespace cld
