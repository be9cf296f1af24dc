// CLUSTER(G, tau) of Algorithm 1 on the GPU, one graph per launch: each
// phase body of cluster_dev.cuh runs as its own grid kernel and the host
// drives the stage / step / doubling control flow from small counter reads.

#include <atomic>
#include <cmath>
#include <vector>


#include "cluster_dev.cuh"
#include "internal.cuh"
#include "prof.cuh"

namespace cld {

namespace {

__global__ void k_select(uint32_t n, const uint32_t* __restrict__ center, unsigned long long* __restrict__ key,
                         uint64_t seed, uint32_t stage, uint64_t thr, Counters* ctr,
                         unsigned long long* __restrict__ keyS) {
    dev_select(n, center, key, seed, stage, thr, ctr, blockIdx.x, gridDim.x, keyS);
}

__global__ void k_rebuild(uint32_t n, const unsigned long long* __restrict__ key, const uint32_t* __restrict__ center,
                          const uint32_t* __restrict__ Dcum, const uint64_t* __restrict__ off, uint32_t delta,
                          bool pull, uint32_t* __restrict__ fbase, unsigned long long* __restrict__ fkey,
                          uint32_t* __restrict__ fpre, uint32_t* __restrict__ cfirst, Counters* ctr) {
    __shared__ unsigned long long scratch[33];
    dev_rebuild(n, key, center, Dcum, off, delta, pull, fbase, fkey, fpre, cfirst, ctr, scratch, blockIdx.x,
                gridDim.x);
}

__global__ void k_snapshot(const uint32_t* __restrict__ next, const unsigned long long* __restrict__ key,
                           const uint64_t* __restrict__ off, uint32_t delta, uint32_t* __restrict__ fbase,
                           unsigned long long* __restrict__ fkey, uint32_t* __restrict__ fpre,
                           uint32_t* __restrict__ cfirst, Counters* ctr, unsigned long long* __restrict__ keyS) {
    __shared__ unsigned long long scratch[33];
    const uint32_t nn = __ldcg(&ctr->nnext);
    dev_snapshot(next, nn, key, off, delta, fbase, fkey, fpre, cfirst, ctr, scratch, blockIdx.x, gridDim.x, keyS);
}

__global__ void k_growable(const uint32_t* __restrict__ row, const uint2* __restrict__ adj, uint64_t nnz,
                           const unsigned long long* __restrict__ key, Counters* ctr) {
    dev_growable(row, adj, nnz, key, ctr, blockIdx.x, gridDim.x);
}

__global__ void k_finalize_d(uint32_t n, const unsigned long long* __restrict__ key, const uint32_t* __restrict__ center,
                             const uint32_t* __restrict__ R, uint32_t* __restrict__ D, Counters* ctr) {
    dev_finalize_d(n, key, center, R, D, ctr, blockIdx.x, gridDim.x);
}

__global__ void k_finalize_freeze(uint32_t n, unsigned long long* __restrict__ key, uint32_t* __restrict__ center,
                                  uint32_t* __restrict__ R, const uint32_t* __restrict__ D, const uint64_t* __restrict__ off,
                                  Counters* ctr, unsigned long long* __restrict__ keyS, bool cumulative) {
    dev_finalize_freeze(n, key, center, R, D, off, ctr, blockIdx.x, gridDim.x, keyS, cumulative);
}

__global__ void k_singletons(uint32_t n, uint32_t* __restrict__ center, uint32_t* __restrict__ D) {
    dev_singletons(n, center, D, blockIdx.x, gridDim.x);
}

// a9: cluster id = rank of the center's node id among all centers.
__global__ void k_center_flags(uint32_t n, const uint32_t* __restrict__ center, uint32_t* __restrict__ flag) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        flag[v] = center[v] == v ? 1u : 0u;
}
__global__ void k_assign_cid(uint32_t n, const uint32_t* __restrict__ center, const uint32_t* __restrict__ rank,
                             uint32_t* __restrict__ cid) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) cid[v] = rank[center[v]];
}

// ---------------------------------------------------------------- dense (pull) form of the growing step
// When the step's relaxers hold a large share of the adjacency, every node v
// instead reads its own adjacency and takes the smallest candidate
// (d_u + w, c_u) over its neighbours u, each read from a snapshot of the
// start-of-step keys (keyS), and lowers its key once.  keyS holds, for a
// contracted node, the key it relaxes with: (0, c_u), or (D_u, c_u) in the
// cumulative mode.  A neighbour is a relaxer iff d_u < Delta (a node without a
// key has d = 2^32 - 1 >= Delta), and its candidate counts iff
// d_u + w <= Delta: the same candidate set as the pushed form (a relaxer whose
// key did not change since its last push only repeats candidates that are
// already applied, and min is idempotent), so the step gives the same keys.
// A contracted row is never lowered: in the reset mode its snapshot key
// (0, c) is below every candidate, in the cumulative mode its center is read.
//
// Work unit: one warp takes PW consecutive CSR positions (4 groups of 32:
// coalesced evict-first adjacency loads, then snapshot gathers), maps each
// position to its row from the row starts of the chunk (held in a per-warp
// shared array), reduces every row's candidates over its lanes with shuffles
// (a row that continues into the next group carries its partial minimum
// there), and the lane heading each row segment lowers the row's key with an
// atomic minimum when it undercuts the snapshot; the per-step stamp decides
// "first change" (next list) and "newly covered" as in the pushed form.  No
// block barrier: warps run independently, so many gathers stay in flight.

// a5, pushed form: the frontier's adjacency lists are one flattened range of E
// positions; each warp takes QC consecutive positions (4 groups of 32), finds
// the entries they span from the chunk table (cfirst, written by the frontier
// producers) and maps positions to entries with the start words.  A pushing
// entry (start-of-step key of its node) sends (d_u + w, c_u) to each
// neighbour: a key read (evict-last) filters candidates that cannot win, the
// rest lower the neighbour's key with a no-return atomic minimum.  A pulling
// entry (an unfrozen node that reads the candidates of its contracted
// neighbours, kPullTag | v) reduces its candidates over its lanes first, so
// it lowers its own key once per group segment.  No block barrier.
struct PushSmem {
    uint32_t spre[PT / 32][QC + 1];  // first positions of the entries after the chunk's first
    uint32_t sbase[PT / 32][QC + 2];
    unsigned long long skey[PT / 32][QC + 2];
    uint32_t sbuf[PT / 32][PNB];
};

__device__ __forceinline__ void dev_push(const uint32_t* __restrict__ fbase, const unsigned long long* __restrict__ fkey,
                                         const uint32_t* __restrict__ fpre, const uint32_t* __restrict__ cfirst,
                                         uint32_t nf, uint32_t E, const uint2* __restrict__ adj,
                                         const uint32_t* __restrict__ center, const uint32_t* __restrict__ Dcum,
                                         unsigned long long* __restrict__ key, uint32_t delta,
                                         uint32_t* __restrict__ stamp, uint32_t stepid,
                                         uint32_t* __restrict__ next, Counters* ctr, PushSmem& smp, uint32_t br,
                                         uint32_t nb) {
    auto& spre = smp.spre;
    auto& sbase = smp.sbase;
    auto& skey = smp.skey;
    auto& sbuf = smp.sbuf;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint64_t pol_stream = l2_evict_first_policy(), pol_keep = l2_evict_last_policy();
    const unsigned le_mask = 0xffffffffu >> (31u - lane);
    WarpNext wn{sbuf[warp], 0};
    unsigned long long newly = 0;
    const uint32_t nq = (uint32_t)(((uint64_t)E + QC - 1) / QC);
    const uint32_t nwarps = nb * (PT / 32);
    for (uint32_t q = br * (PT / 32) + warp; q < nq; q += nwarps) {
        const uint32_t p0 = q * QC, e1 = min(E, p0 + QC);
        // entry i0 holds p0; entries i0 + 1 .. il start inside (p0, p0 + QC] (at most QC of them)
        const uint32_t i0 = __ldcg(&cfirst[q]);
        const uint32_t il = q + 1 < nq ? __ldcg(&cfirst[q + 1]) : nf - 1;
        const uint32_t ne = min(il - i0 + 1, (uint32_t)QC + 1);
        for (uint32_t j = lane; j < ne; j += 32) {
            if (j) spre[warp][j - 1] = __ldcg(&fpre[i0 + j]);
            sbase[warp][j] = __ldcg(&fbase[i0 + j]);
            skey[warp][j] = __ldcg(&fkey[i0 + j]);
        }
        __syncwarp();
        uint32_t word[4], own[4];
        {
            uint32_t B = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                word[u] = group_starts(spre[warp] + B, ne - 1 - B, p0 + 32u * u, B, lane, le_mask, &own[u]);
                B += (uint32_t)__popc(word[u]);
            }
        }
        uint2 ed[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t p = p0 + 32u * u + lane;
            ed[u] = p < e1 ? ld_stream_u2(adj + (sbase[warp][own[u]] + p), pol_stream) : make_uint2(0u, 0xFFFFFFFFu);
        }
        unsigned long long carry = kInfKey;  // pull entry still open at the previous group's end
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const unsigned long long ku = skey[warp][own[u]];
            const bool is_pull = (ku & kPullTag) == kPullTag;
            const bool live = p0 + 32u * u + lane < e1;
            unsigned long long nk = kInfKey;
            uint32_t target = 0;
            if (live && !is_pull) {
                const uint64_t cand = (ku >> 32) + ed[u].y;
                if (cand <= delta) {
                    target = ed[u].x;
                    nk = (cand << 32) | (ku & 0xFFFFFFFFull);
                }
            } else if (live && ed[u].y <= delta) {  // pull: candidate of a contracted neighbour
                const uint32_t cu = __ldg(&center[ed[u].x]);
                if (cu != kNone) {
                    const uint64_t cand = (uint64_t)(Dcum ? __ldg(&Dcum[ed[u].x]) : 0u) + ed[u].y;
                    if (cand <= delta) nk = (cand << 32) | cu;
                }
            }
            // pulling entries: one candidate per segment (all lanes of an entry share its kind)
            if (__any_sync(0xffffffffu, is_pull)) {
                unsigned long long pv = is_pull ? nk : kInfKey;
                if (lane == 0 && !(word[u] & 1u)) pv = carry < pv ? carry : pv;
                pv = segment_min(pv, word[u], lane);
                const uint32_t last_head = word[u] ? 31u - (uint32_t)__clz(word[u]) : 0u;
                const bool cont = u < 3 && !(word[(u + 1) & 3] & 1u);
                carry = __shfl_sync(0xffffffffu, pv, last_head);
                const unsigned le = word[u] & le_mask;
                const uint32_t head = le ? 31u - (uint32_t)__clz(le) : 0u;
                if (is_pull) {
                    const bool flush = lane == head && !(cont && head == last_head);
                    nk = flush ? pv : kInfKey;
                    target = (uint32_t)ku;
                }
            } else {
                carry = kInfKey;
            }
            bool first = false;
            if (nk != kInfKey) {
                // the target's key and stamp in one round trip, through L1 (a stale line only lets an
                // extra candidate through: keys only fall within a launch, and the atomics decide); most
                // candidates lose to the current key
                const unsigned long long cur = ld_keep_u64(&key[target], pol_keep);
                const uint32_t stp = ld_keep_u32(&stamp[target], pol_keep);
                if (nk < cur) {
                    red_min_keep_u64(&key[target], nk, pol_keep);
                    if (stp != stepid) {  // hubs see many lowerings: only the first ones exchange
                        const uint32_t old = atomicExch(&stamp[target], stepid);
                        first = old != stepid;
                        newly += old == 0u ? 1 : 0;
                    }
                }
            }
            wn.put(first, target, lane);
        }
        if (wn.cnt >= (uint32_t)PW) wn.flush(next, &ctr->nnext, lane);
    }
    if (wn.cnt) wn.flush(next, &ctr->nnext, lane);
    warp_add_u64(&ctr->newly_covered, newly);
}

__global__ void __launch_bounds__(PT, 6) k_push(const uint32_t* __restrict__ fbase,
                                                const unsigned long long* __restrict__ fkey,
                                                const uint32_t* __restrict__ fpre, const uint32_t* __restrict__ cfirst,
                                                uint32_t nf, uint32_t E, const uint2* __restrict__ adj,
                                                const uint32_t* __restrict__ center, const uint32_t* __restrict__ Dcum,
                                                unsigned long long* __restrict__ key, uint32_t delta,
                                                uint32_t* __restrict__ stamp, uint32_t stepid,
                                                uint32_t* __restrict__ next, Counters* ctr) {
    __shared__ PushSmem smp;
    dev_push(fbase, fkey, fpre, cfirst, nf, E, adj, center, Dcum, key, delta, stamp, stepid, next, ctr, smp,
                    blockIdx.x, gridDim.x);
}

// crow[q] = the row that holds CSR position q * PW (every row has >= 1 entry)
__global__ void k_pull_rows(uint32_t n, const uint64_t* __restrict__ off, uint32_t* __restrict__ crow) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint64_t o0 = off[v], o1 = off[v + 1];
        for (uint64_t q = (o0 + PW - 1) / PW; q * PW < o1; ++q) crow[q] = v;
    }
}

struct PullSmem {
    uint32_t sst[PT / 32][PW + 1];            // starts of the rows after the chunk's first row
    unsigned long long sks[PT / 32][PW + 2];  // snapshot keys of the chunk's rows
    uint32_t sbuf[PT / 32][PNB];              // changed rows waiting for the next list
};

__device__ __forceinline__ void dev_pull(uint32_t n, uint32_t nnz, uint32_t nq, const uint32_t* __restrict__ crow,
                                         const uint64_t* __restrict__ off, const uint2* __restrict__ adj,
                                         const uint32_t* __restrict__ center_cum,
                                         const unsigned long long* __restrict__ keyS,
                                         unsigned long long* __restrict__ key, uint32_t delta,
                                         uint32_t* __restrict__ stamp, uint32_t stepid,
                                         uint32_t* __restrict__ next, Counters* ctr, PullSmem& smq, uint32_t br,
                                         uint32_t nb) {
    auto& sst = smq.sst;
    auto& sks = smq.sks;
    auto& sbuf = smq.sbuf;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint64_t pol_stream = l2_evict_first_policy(), pol_keep = l2_evict_last_policy();
    uint32_t* st = sst[warp];
    WarpNext wn{sbuf[warp], 0};
    unsigned long long newly = 0;
    const uint32_t nwarps = nb * (PT / 32);
    const unsigned le_mask = 0xffffffffu >> (31u - lane);  // lanes <= this one
    // lower row r to v if v undercuts its start-of-step key ks; true for the one lowering that is r's first
    const auto lower_row = [&](uint32_t r, unsigned long long v, unsigned long long ks) -> bool {
        if (!(v < ks)) return false;
        if (center_cum && __ldg(&center_cum[r]) != kNone) return false;  // contracted: keeps its key
        // exactly one lowering of r finds its start-of-step key: that one is the first change
        if (atom_min_keep_u64(&key[r], v, pol_keep) != ks) return false;
        stamp[r] = stepid;  // r has been lowered (a later pushed step reads it)
        newly += ks == kInfKey ? 1 : 0;
        return true;
    };
    for (uint32_t q = br * (PT / 32) + warp; q < nq; q += nwarps) {
        const uint32_t p0 = q * PW;
        uint2 ed[PWG];
#pragma unroll
        for (int u = 0; u < PWG; ++u) {
            const uint32_t p = p0 + 32u * u + lane;
            ed[u] = p < nnz ? ld_stream_u2(adj + p, pol_stream) : make_uint2(0u, 0u);
        }
        // row B0 holds p0; rows B0 + 1 .. B1 start inside (p0, p0 + PW] (at most PW of them)
        const uint32_t B0 = __ldg(&crow[q]);
        const uint32_t B1 = q + 1 < nq ? __ldg(&crow[q + 1]) : n - 1;
        const uint32_t nr = min(B1 - B0, (uint32_t)PW);
        for (uint32_t j = lane; j <= nr; j += 32) {
            if (j < nr) st[j] = (uint32_t)__ldg(&off[B0 + 1 + j]);
            sks[warp][j] = ld_nc_keep_u64(&keyS[B0 + j], pol_keep);
        }
        unsigned long long cv[PWG];  // each position's candidate (d_u + w, c_u), or none
#pragma unroll
        for (int u = 0; u < PWG; ++u) {
            const unsigned long long ku =
                p0 + 32u * u + lane < nnz ? ld_nc_keep_u64(&keyS[ed[u].x], pol_keep) : kInfKey;
            const uint32_t du = (uint32_t)(ku >> 32);
            const uint64_t cand = (uint64_t)du + ed[u].y;
            cv[u] = (du < delta && cand <= delta) ? (cand << 32) | (ku & 0xFFFFFFFFull) : kInfKey;
        }
        __syncwarp();
        if (B1 == B0) {
            // the chunk lies inside one row (a hub): one minimum over the warp, two 32-bit reductions
            unsigned long long v = cv[0];
#pragma unroll
            for (int u = 1; u < PWG; ++u) v = cv[u] < v ? cv[u] : v;
            const uint32_t hi = __reduce_min_sync(0xffffffffu, (uint32_t)(v >> 32));
            const uint32_t lo = __reduce_min_sync(0xffffffffu, (uint32_t)(v >> 32) == hi ? (uint32_t)v : 0xFFFFFFFFu);
            v = ((unsigned long long)hi << 32) | lo;
            const bool first = lane == 0 && lower_row(B0, v, sks[warp][0]);
            wn.put(first, B0, lane);
        } else {
            // row starts inside each group: bit d of word[u] = a row starts at position p0 + 32u + d
            uint32_t word[PWG], own[PWG];
            {
                uint32_t B = 0;  // row B0 + B holds the current group's first position
#pragma unroll
                for (int u = 0; u < PWG; ++u) {
                    word[u] = group_starts(st + B, nr - B, p0 + 32u * u, B, lane, le_mask, &own[u]);
                    B += (uint32_t)__popc(word[u]);
                }
            }
            unsigned long long carry = kInfKey;  // minimum of the row still open at the previous group's end
#pragma unroll
            for (int u = 0; u < PWG; ++u) {
                unsigned long long v = cv[u];
                if (lane == 0 && !(word[u] & 1u)) v = carry < v ? carry : v;
                v = segment_min(v, word[u], lane);
                const unsigned le = word[u] & le_mask;
                const uint32_t head = le ? 31u - (uint32_t)__clz(le) : 0u;
                const uint32_t last_head = word[u] ? 31u - (uint32_t)__clz(word[u]) : 0u;
                const bool cont = u + 1 < PWG && !(word[(u + 1) % PWG] & 1u);  // the last row goes on
                carry = __shfl_sync(0xffffffffu, v, last_head);
                bool first = false;
                const uint32_t r = B0 + own[u];
                if (lane == head && v != kInfKey && !(cont && head == last_head))
                    first = lower_row(r, v, sks[warp][own[u]]);
                wn.put(first, r, lane);
            }
        }
        if (wn.cnt >= (uint32_t)PW) wn.flush(next, &ctr->nnext, lane);
    }
    if (wn.cnt) wn.flush(next, &ctr->nnext, lane);
    warp_add_u64(&ctr->newly_covered, newly);
}

__global__ void __launch_bounds__(PT, 6) k_pull(uint32_t n, uint32_t nnz, uint32_t nq, const uint32_t* __restrict__ crow,
                                             const uint64_t* __restrict__ off, const uint2* __restrict__ adj,
                                             const uint32_t* __restrict__ center_cum,
                                             const unsigned long long* __restrict__ keyS,
                                             unsigned long long* __restrict__ key, uint32_t delta,
                                             uint32_t* __restrict__ stamp, uint32_t stepid,
                                             uint32_t* __restrict__ next, Counters* ctr) {
    __shared__ PullSmem smq;
    dev_pull(n, nnz, nq, crow, off, adj, center_cum, keyS, key, delta, stamp, stepid, next, ctr, smq,
                    blockIdx.x, gridDim.x);
}

// node state before the first stage: no center, D = R = 0, no stamp, no key
__global__ void k_cluster_init(uint32_t n, uint32_t* __restrict__ center, uint32_t* __restrict__ D,
                               uint32_t* __restrict__ R, uint32_t* __restrict__ stamp,
                               unsigned long long* __restrict__ key, unsigned long long* __restrict__ keyS) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        center[i] = kNone;
        D[i] = 0;
        R[i] = 0;
        stamp[i] = 0;
        key[i] = kInfKey;
        if (keyS) keyS[i] = kInfKey;
    }
}


struct ClusterOwner {
    cldiam_clustering* c;
    explicit ClusterOwner(cldiam_clustering* x) : c(x) {}
    ~ClusterOwner() {
        if (c) free_clustering(c);
    }
};

}  // namespace

// a9: cluster id = rank of the center's node id among all centers; *k = number of clusters (synchronises)
cldiam_status relabel_clusters(cldiam_graph* g, const uint32_t* center, uint32_t* cid, uint32_t* k) {
    const cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    const unsigned gb = grid_for(n, 256);
    DBuf<uint32_t> flag, rank, kdev;
    CLD_TRY(flag.alloc(n, s));
    CLD_TRY(rank.alloc(n, s));
    CLD_TRY(kdev.alloc(1, s));
    CLD_K(K_MISC, s, k_center_flags<<<gb, 256, 0, s>>>(n, center, flag.get()));
    CLD_LAUNCH_CHECK();
    CLD_TRY(scan_exclusive_u32(flag.get(), rank.get(), n, kdev.get(), s));
    CLD_K(K_MISC, s, k_assign_cid<<<gb, 256, 0, s>>>(n, center, rank.get(), cid));
    CLD_LAUNCH_CHECK();
    uint32_t* hk = reinterpret_cast<uint32_t*>(static_cast<char*>(g->host.h) + 128);
    CLD_CUDA(cudaMemcpyAsync(hk, kdev.get(), 4, cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    *k = *hk;
    return CLDIAM_OK;
}

void free_clustering(cldiam_clustering* c) {
    if (!c) return;
    cudaStream_t s = c->stream;
    dfree(c->center, s);
    dfree(c->D, s);
    dfree(c->cid, s);
    if (s) cudaStreamSynchronize(s);
    delete c;
}

cldiam_status cluster(cldiam_graph* g, double tau, uint64_t seed, const cldiam_opts* o, cldiam_clustering** out) {
    if (!g || !out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL graph or out");
    *out = nullptr;
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(CLDIAM_ERR_INVALID_ARG, "tau must be a positive number");
    cldiam_opts opts{};
    if (o) opts = *o;
    if (opts.contract_mode != CLDIAM_CONTRACT_RESET && opts.contract_mode != CLDIAM_CONTRACT_CUMULATIVE)
        return fail(CLDIAM_ERR_INVALID_ARG, "unknown contract_mode");
    if (opts.reserved[0] || opts.reserved[1]) return fail(CLDIAM_ERR_INVALID_ARG, "reserved options must be 0");
    const bool cumulative = opts.contract_mode == CLDIAM_CONTRACT_CUMULATIVE;
    const uint32_t step_cap = opts.step_cap;  // growing steps per PartialGrowth, 0 = no cap
    if (opts.quotient_mode > CLDIAM_QUOTIENT_DENSE) return fail(CLDIAM_ERR_INVALID_ARG, "unknown quotient_mode");
    uint32_t delta = 0;
    CLD_TRY(delta0(g, opts.delta0_mode, opts.delta0, &delta));

    const cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    ClusterOwner owner(new cldiam_clustering());
    cldiam_clustering* cl = owner.c;
    cl->g = g;
    cl->stream = g->stream;
    cl->max_fw_k = opts.max_fw_k ? opts.max_fw_k : 8192u;
    cl->quotient_mode = opts.quotient_mode;

    // a frontier lists each node at most twice (push + pull entry)
    const size_t fcap = 2 * (size_t)n;
    DBuf<uint32_t> center, D, cid;
    DBuf<unsigned long long> key, fkeyA, fkeyB;
    DBuf<uint32_t> R, stamp, fvA, fvB, fpA, fpB, cfA, cfB, next;
    DBuf<Counters> ctr;
    // dense (pull) steps: every row has an entry (connected graph, n >= 2) and positions index below 2^32
    const cldiam_tuning tun = tuning_for(g->nnz);
    const bool pull_dense = tun.pull_ratio > 0.f && g->connected && n >= 2 && g->nnz < 0xFFFFFFFFull;
    const uint32_t pull_chunks = pull_dense ? (uint32_t)((g->nnz + PW - 1) / PW) : 0u;
    DBuf<unsigned long long> keyS;
    DBuf<uint32_t> crow;
    if (pull_dense) {
        CLD_TRY(keyS.alloc(n, s));
        CLD_TRY(crow.alloc(pull_chunks, s));
    }
    CLD_TRY(center.alloc(n, s));
    CLD_TRY(D.alloc(n, s));
    CLD_TRY(cid.alloc(n, s));
    CLD_TRY(key.alloc(n, s));
    CLD_TRY(R.alloc(n, s));
    CLD_TRY(stamp.alloc(n, s));
    CLD_TRY(fvA.alloc(fcap, s));
    CLD_TRY(fvB.alloc(fcap, s));
    CLD_TRY(fpA.alloc(fcap, s));
    CLD_TRY(fpB.alloc(fcap, s));
    CLD_TRY(fkeyA.alloc(fcap, s));
    CLD_TRY(fkeyB.alloc(fcap, s));
    // chunk tables: a frontier has at most 2 * nnz adjacency entries (push + pull)
    const size_t ccap = (2 * (size_t)g->nnz) / QC + 2;
    CLD_TRY(cfA.alloc(ccap, s));
    CLD_TRY(cfB.alloc(ccap, s));
    CLD_TRY(next.alloc(n, s));
    CLD_TRY(ctr.alloc(1, s));
    Counters* hc = static_cast<Counters*>(g->host.h);
    static_assert(sizeof(Counters) <= 128, "counter block must fit the pinned area");

    const unsigned gb = grid_for(n, 256);
    CLD_K(K_MISC, s, k_cluster_init<<<gb, 256, 0, s>>>(n, center.get(), D.get(), R.get(), stamp.get(), key.get(),
                                                        keyS.get()));
    CLD_LAUNCH_CHECK();
    if (pull_dense) {
        CLD_K(K_MISC, s, k_pull_rows<<<gb, 256, 0, s>>>(n, g->off, crow.get()));
        CLD_LAUNCH_CHECK();
    }
    CLD_CUDA(cudaMemsetAsync(ctr.get(), 0, sizeof(Counters), s));

    auto sync_counters = [&]() -> cldiam_status {
        CLD_CUDA(cudaMemcpyAsync(hc, ctr.get(), sizeof(Counters), cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        prof_flush();
        return CLDIAM_OK;
    };
    auto zero_field = [&](size_t offset, size_t bytes) -> cldiam_status {
        CLD_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(ctr.get()) + offset, 0, bytes, s));
        return CLDIAM_OK;
    };

    cldiam_result st{};
    const double L = std::log2((double)n);
    uint64_t U = n;               // unfrozen nodes
    uint64_t frozen_deg = 0;      // adjacency entries of frozen nodes
    const bool pull_ok = g->nnz < 0x80000000ull;  // push + pull entries must index below 2^32
    uint32_t stage = 1, stepid = 0;
    uint32_t* fv = fvA.get();
    uint32_t* fp = fpA.get();
    unsigned long long* fk = fkeyA.get();
    uint32_t* fv2 = fvB.get();
    uint32_t* fp2 = fpB.get();
    unsigned long long* fk2 = fkeyB.get();
    uint32_t* cf = cfA.get();
    uint32_t* cf2 = cfB.get();
    const unsigned max_relax_grid = (unsigned)num_sms() * 8;
    // the growing-step kernels loop over warp chunks: launch at most the resident CTAs (no partial second
    // wave after the first has finished its chunks)
    static std::atomic<int> push_per_sm[64], pull_per_sm[64];  // concurrent first calls store the same values
    int dev = 0;
    CLD_CUDA(cudaGetDevice(&dev));
    const int di = (dev >= 0 && dev < 64) ? dev : 0;
    if (push_per_sm[di].load() == 0) {
        int a = 0, b = 0;
        CLD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_push, PT, 0));
        CLD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pull, PT, 0));
        pull_per_sm[di] = std::max(1, b);
        push_per_sm[di] = std::max(1, a);
    }
    unsigned push_ctas = (unsigned)push_per_sm[di].load(), pull_ctas = (unsigned)pull_per_sm[di].load();
    if (tun.relax_ctas_per_sm) {
        push_ctas = std::min(push_ctas, tun.relax_ctas_per_sm);
        pull_ctas = std::min(pull_ctas, tun.relax_ctas_per_sm);
    }
    const unsigned push_grid = (unsigned)num_sms() * push_ctas;
    const unsigned pull_grid =
        (unsigned)std::min<uint64_t>((uint64_t)num_sms() * pull_ctas, (pull_chunks + PT / 32 - 1) / (PT / 32));
    uint32_t nf = 0, E = 0;
    DBuf<uint32_t> rows_built;  // COO rows for the guard's edge scan when the graph keeps none

    // list every relaxer (stage start, or after Delta doubled)
    auto rebuild = [&]() -> cldiam_status {
        const bool pull = pull_ok && (g->nnz - frozen_deg) < frozen_deg;
        CLD_TRY(zero_field(offsetof(Counters, front), 8));
        CLD_K(K_REBUILD, s, k_rebuild<<<gb, 256, 0, s>>>(n, key.get(), center.get(), cumulative ? D.get() : nullptr,
                                                          g->off, delta, pull, fv, fk, fp, cf, ctr.get()));
        CLD_LAUNCH_CHECK();
        return CLDIAM_OK;
    };

    {
        for (;;) {
            uint64_t thr = 0;
            if (!stage_threshold(U, tau, L, &thr)) break;  // outer while test of Algorithm 1, center draw threshold
            if (stage > kMaxStages) return fail(CLDIAM_ERR_DIVERGED, "CLUSTER exceeded its stage limit");

            // selection + reset, then the stage's first frontier
            CLD_TRY(zero_field(offsetof(Counters, selected), 8));
            CLD_TRY(zero_field(offsetof(Counters, unfrozen), 8));
            CLD_K(K_SELECT, s, k_select<<<gb, 256, 0, s>>>(n, center.get(), key.get(), seed, stage, thr, ctr.get(),
                                                            keyS.get()));
            CLD_LAUNCH_CHECK();
            CLD_TRY(rebuild());
            CLD_TRY(sync_counters());
            if (hc->unfrozen != U) {
                char buf[200];
                snprintf(buf, sizeof buf, "the draw of stage %u saw %llu unfrozen nodes, the loop tracked %llu",
                         stage, (unsigned long long)hc->unfrozen, (unsigned long long)U);
                return fail(CLDIAM_ERR_DIVERGED, buf);
            }
            uint64_t covered = hc->selected;
            nf = (uint32_t)(hc->front >> 32);
            E = (uint32_t)hc->front;
            st.centers_drawn += hc->selected;

            for (;;) {
                uint32_t updated, growth_steps = 0;
                do {
                    ++growth_steps;
                    ++stepid;
                    updated = 0;
                    if (nf > 0) {
                        CLD_TRY(zero_field(offsetof(Counters, newly_covered), 24));  // newly_covered, front, nnext
                        // the dense form reads the whole adjacency: worth it when the relaxers hold a large share
                        const bool dense = pull_dense && (double)E >= (double)tun.pull_ratio * (double)g->nnz;
                        if (dense) {
                            CLD_K(K_PULL, s, k_pull<<<pull_grid, PT, 0, s>>>(n, (uint32_t)g->nnz, pull_chunks, crow.get(),
                                                                              g->off, g->adj,
                                                                              cumulative ? center.get() : nullptr, keyS.get(),
                                                                              key.get(), delta, stamp.get(), stepid,
                                                                              next.get(), ctr.get()));
                        } else {
                            const uint64_t warps = ((uint64_t)E + QC - 1) / QC;
                            const unsigned rg = (unsigned)std::min<uint64_t>((warps + PT / 32 - 1) / (PT / 32), push_grid);
                            CLD_K(K_RELAX, s, k_push<<<rg, PT, 0, s>>>(fv, fk, fp, cf, nf, E, g->adj, center.get(),
                                                                        cumulative ? D.get() : nullptr, key.get(), delta,
                                                                        stamp.get(), stepid, next.get(), ctr.get()));
                        }
                        CLD_LAUNCH_CHECK();
                        CLD_K(K_SNAPSHOT, s, k_snapshot<<<max_relax_grid, 256, 0, s>>>(next.get(), key.get(), g->off, delta,
                                                                                     fv2, fk2, fp2, cf2, ctr.get(),
                                                                                     keyS.get()));
                        CLD_LAUNCH_CHECK();
                        CLD_TRY(sync_counters());
                        updated = hc->nnext;
                        covered += hc->newly_covered;
                        st.edges_scanned += E;
                        if (dense) {
                            // algorithmic bytes of a dense step: per adjacency entry the (col, w) pair (8 B) and
                            // the neighbour's snapshot key (8 B); per row its start and snapshot key (16 B); per
                            // changed node its key, stamp and list slot (16 B)
                            prof_add_bytes(K_PULL, 16.0 * (double)g->nnz + 16.0 * n + 16.0 * updated);
                        } else {
                            // algorithmic bytes of a pushed step: per frontier entry its slot (4 + 8 + 4 B)
                            // and row start (8 B); per adjacency entry the (col, w) pair (8 B) and the target's
                            // key (8 B); per changed node its key, stamp and list slot (16 B)
                            prof_add_bytes(K_RELAX, 24.0 * nf + 16.0 * (double)E + 16.0 * updated);
                        }
                        prof_add_bytes(K_SNAPSHOT, 4.0 * updated + 16.0 * updated + 16.0 * updated + 16.0 * (hc->front >> 32));
                        std::swap(fv, fv2);
                        std::swap(fp, fp2);
                        std::swap(fk, fk2);
                        std::swap(cf, cf2);
                        nf = (uint32_t)(hc->front >> 32);
                        E = (uint32_t)hc->front;
                    }
                    st.steps++;
                    st.node_updates += updated;
                } while (updated != 0 && 2 * covered < U && (step_cap == 0 || growth_steps < step_cap));
                if (2 * covered >= U) break;
                bool growable = false;
                if (delta < kDeltaMax && g->connected) {
                    // connected graph: some covered or frozen node touches an uncovered one iff any exists
                    growable = covered > 0 || U < n;
                } else if (delta < kDeltaMax && g->nnz) {
                    CLD_TRY(zero_field(offsetof(Counters, growable), 4));
                    if (!g->row && !rows_built.get()) {  // (graphs without a row array are connected LCCs)
                        CLD_TRY(rows_built.alloc(g->nnz, s));
                        CLD_TRY(fill_rows(g->off, n, rows_built.get(), s));
                    }
                    const uint32_t* rows = g->row ? g->row : rows_built.get();
                    CLD_K(K_GROWABLE, s, k_growable<<<grid_for(g->nnz, 256), 256, 0, s>>>(rows, g->adj, g->nnz,
                                                                                             key.get(), ctr.get()));
                    CLD_LAUNCH_CHECK();
                    CLD_TRY(sync_counters());
                    growable = hc->growable != 0;
                }
                if (!growable) {
                    st.guard_exits++;
                    break;
                }
                delta = (delta > kDeltaMax / 2) ? kDeltaMax : 2 * delta;
                st.doublings++;
                CLD_TRY(rebuild());
                CLD_TRY(sync_counters());
                nf = (uint32_t)(hc->front >> 32);
                E = (uint32_t)hc->front;
            }

            // assign and contract
            CLD_TRY(zero_field(offsetof(Counters, frozen), 16));  // frozen + frozen_deg
            CLD_K(K_FINALIZE, s, k_finalize_d<<<gb, 256, 0, s>>>(n, key.get(), center.get(), cumulative ? nullptr : R.get(),
                                                                 D.get(), ctr.get()));
            CLD_K(K_FINALIZE, s, k_finalize_freeze<<<gb, 256, 0, s>>>(n, key.get(), center.get(), R.get(), D.get(), g->off,
                                                                      ctr.get(), keyS.get(), cumulative));
            CLD_LAUNCH_CHECK();
            CLD_TRY(sync_counters());
            if (hc->overflow) return fail(CLDIAM_ERR_OVERFLOW, "a cluster distance bound reached 2^32 - 1");
            U -= hc->frozen;
            frozen_deg += hc->frozen_deg;
            st.stages++;
            ++stage;
        }
        CLD_K(K_FINALIZE, s, k_singletons<<<gb, 256, 0, s>>>(n, center.get(), D.get()));
        CLD_LAUNCH_CHECK();
    }

    CLD_TRY(relabel_clusters(g, center.get(), cid.get(), &st.k));
    prof_flush();
    st.delta_end = delta;

    cl->center = center.detach();
    cl->D = D.detach();
    cl->cid = cid.detach();
    cl->k = st.k;
    cl->stats = st;
    *out = cl;
    owner.c = nullptr;
    return CLDIAM_OK;
}

}  // namespace cld
