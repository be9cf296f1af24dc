// Device bodies of the CLUSTER(tau) phases (Algorithm 1), shared by the
// one-graph-per-launch path (each body runs as its own grid kernel, rank =
// blockIdx.x) and the many-graph persistent kernel (one CTA runs every body
// for its graph, rank 0 of 1, with block barriers between phases).
//
// Node state (Section 3) is one 64-bit word per node, key = d << 32 | c, so
// the paper's tie-break (smallest distance, then smallest center index) is
// the integer minimum and a Delta-growing step is an atomicMin per light
// edge.  Frozen nodes (clustered in an earlier stage; Procedure Contract)
// hold key 0, which no candidate can undercut, so the relaxation needs no
// frozen test; they are relaxers with the virtual key (0, c_u).
//
// Steps are synchronous: each frontier entry carries the key its node had
// at the start of the step, so in-place atomicMin gives exactly the
// start-of-step (Jacobi) semantics of the paper's "in parallel" step.  The
// next frontier is the set of nodes whose key decreased (deduplicated with a
// per-node step stamp); nodes whose key did not change would only repeat
// candidates that are already applied.  After a stage start or a Delta
// doubling every relaxer is listed again.
//
// Mutable node state is read with L2 loads (__ldcg): inside one persistent
// CTA there is no kernel boundary to drop stale L1 lines between phases.
#pragma once

#include "common.cuh"

namespace cld {

struct Counters {
    unsigned long long selected;       // centers drawn in this stage
    unsigned long long newly_covered;  // nodes that got their first key this step
    unsigned long long edges_scanned;  // adjacency entries read by relax
    unsigned long long frozen;         // nodes frozen by finalize
    unsigned long long frozen_deg;     // their degree sum
    unsigned long long front;          // next frontier: (entries << 32) | adjacency entries
    uint32_t nnext;                    // changed nodes this step
    uint32_t growable;                 // some covered/frozen node touches an uncovered one
    uint32_t overflow;                 // a D_v reached 2^32 - 1
    uint32_t pad;
};

constexpr unsigned long long kPull = kInfKey;  // frontier key marking a pull entry
constexpr int RT = 256;                        // relax threads per CTA in the grid form
constexpr int RC = 1024;                       // adjacency entries per relax chunk

__device__ __forceinline__ void warp_add_u64(unsigned long long* p, unsigned long long v) {
    v = warp_sum(v);
    if (lane_id() == 0 && v) atomicAdd(p, v);
}

// Append to the frontier: one packed atomicAdd per CTA hands out both the
// entry slots (high word) and the entries' first positions in the flattened
// edge list (low word), so positions increase with slots and the frontier's
// degree prefix needs no separate scan.  All threads of the block must call
// it (it synchronises the block); `scratch` holds 33 words.
__device__ __forceinline__ void front_append(unsigned long long* ctr, bool pred, uint32_t deg, uint32_t& slot,
                                             uint32_t& pre, unsigned long long* scratch) {
    const unsigned mask = __ballot_sync(0xffffffffu, pred);
    const unsigned w = threadIdx.x >> 5, l = lane_id(), nw = blockDim.x >> 5;
    const uint32_t d = pred ? deg : 0u;
    const uint32_t incl = warp_incl_scan(d);
    if (l == 31) scratch[w] = ((unsigned long long)__popc(mask) << 32) | incl;
    __syncthreads();
    if (w == 0) {
        const unsigned long long v = l < nw ? scratch[l] : 0ull;
        const unsigned long long iv = warp_incl_scan(v);  // packed (count, entries): no carry, block sums < 2^32
        if (l < nw) scratch[l] = iv - v;
        if (l == 31) scratch[32] = iv ? atomicAdd(ctr, iv) : 0ull;
    }
    __syncthreads();
    const unsigned long long base = scratch[32] + scratch[w];
    slot = (uint32_t)(base >> 32) + (uint32_t)__popc(mask & lanemask_lt());
    pre = (uint32_t)base + (incl - d);
    __syncthreads();
}

// a3: draw the new centers of this stage among unfrozen nodes, reset the others.
__device__ __forceinline__ void dev_select(uint32_t n, const uint32_t* __restrict__ center,
                                           unsigned long long* __restrict__ key, uint64_t seed, uint32_t stage,
                                           uint64_t thr, Counters* ctr, uint32_t br, uint32_t nb) {
    unsigned long long cnt = 0;
    for (uint32_t base = br * blockDim.x; base < n; base += nb * blockDim.x) {
        const uint32_t v = base + threadIdx.x;
        if (v < n && __ldcg(&center[v]) == kNone) {
            const U4 r = philox4x32_10(seed, v, stage, 0u, 0u);
            const bool sel = (uint64_t)r.x < thr;
            key[v] = sel ? (unsigned long long)v : kInfKey;
            cnt += sel ? 1 : 0;
        }
    }
    warp_add_u64(&ctr->selected, cnt);
}

// a4: list every relaxer with its current key: unfrozen nodes with d < Delta
// push their key; the contracted clusters either push (0, c_u) from every
// frozen u, or (pull mode) every unfrozen node lists itself to pull
// (w, c_u) from its frozen neighbours -- the same candidates, read from the
// side with fewer adjacency entries.
__device__ __forceinline__ void dev_rebuild(uint32_t n, const unsigned long long* __restrict__ key,
                                            const uint32_t* __restrict__ center, const uint64_t* __restrict__ off,
                                            uint32_t delta, bool pull, uint32_t* __restrict__ fv,
                                            unsigned long long* __restrict__ fkey, uint32_t* __restrict__ fpre,
                                            Counters* ctr, unsigned long long* scratch, uint32_t br, uint32_t nb) {
    for (uint32_t base = br * blockDim.x; base < n; base += nb * blockDim.x) {
        const uint32_t v = base + threadIdx.x;
        bool push = false, pl = false;
        unsigned long long k = 0;
        uint32_t deg = 0;
        if (v < n) {
            deg = (uint32_t)(off[v + 1] - off[v]);
            const uint32_t c = __ldcg(&center[v]);
            if (deg > 0) {
                if (c != kNone) {
                    push = !pull;
                    k = c;  // (0, c_u)
                } else {
                    k = __ldcg(&key[v]);
                    push = k != kInfKey && (uint32_t)(k >> 32) < delta;
                    pl = pull;
                }
            }
        }
        uint32_t slot = 0, pre = 0;
        front_append(&ctr->front, push, deg, slot, pre, scratch);
        if (push) {
            fv[slot] = v;
            fkey[slot] = k;
            fpre[slot] = pre;
        }
        front_append(&ctr->front, pl, deg, slot, pre, scratch);
        if (pl) {
            fv[slot] = v;
            fkey[slot] = kPull;
            fpre[slot] = pre;
        }
    }
}

// Shared memory of one relax chunk.
struct RelaxSmem {
    uint32_t pre[RC];
    uint32_t beg[RC];
    uint32_t v[RC];
    unsigned long long key[RC];
    uint32_t next[RC];  // nodes first changed by this chunk (at most one per entry)
    uint32_t i0, cnt, nn, nbase;
};

// a5: one synchronous Delta-growing step over the frontier, edge-balanced:
// the frontier's adjacency lists are viewed as one flattened range of E
// entries cut into chunks of RC; each CTA takes chunks, loads the frontier
// entries the chunk spans into shared memory and maps every entry position to
// its frontier entry by binary search, so hubs spread over many CTAs.
__device__ __forceinline__ void dev_relax(const uint32_t* __restrict__ fv, const unsigned long long* __restrict__ fkey,
                                          const uint32_t* __restrict__ fpre, uint32_t nf, uint32_t E,
                                          const uint64_t* __restrict__ off, const uint2* __restrict__ adj,
                                          const uint32_t* __restrict__ center, unsigned long long* __restrict__ key,
                                          uint32_t delta, uint32_t* __restrict__ stamp, uint32_t stepid,
                                          uint32_t* __restrict__ next, Counters* ctr, RelaxSmem& sm, uint32_t br,
                                          uint32_t nb) {
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    unsigned long long newly = 0;
    for (uint32_t chunk = br; (uint64_t)chunk * RC < E; chunk += nb) {
        const uint32_t e0 = chunk * RC;
        const uint32_t e1 = min(E, e0 + RC);
        if (tid == 0) {
            uint32_t lo = 0, hi = nf - 1;  // last entry starting at or before e0
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (fpre[mid] <= e0) lo = mid; else hi = mid - 1;
            }
            const uint32_t i0 = lo;
            hi = nf - 1;  // last entry starting at or before e1 - 1
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (fpre[mid] <= e1 - 1) lo = mid; else hi = mid - 1;
            }
            sm.i0 = i0;
            sm.cnt = lo - i0 + 1;
            sm.nn = 0;
        }
        __syncthreads();
        const uint32_t i0 = sm.i0, cnt = sm.cnt;  // cnt <= RC: every entry has >= 1 adjacency entry
        for (uint32_t j = tid; j < cnt; j += nt) {
            const uint32_t v = fv[i0 + j];
            sm.pre[j] = fpre[i0 + j];
            sm.v[j] = v;
            sm.key[j] = fkey[i0 + j];
            sm.beg[j] = (uint32_t)off[v];
        }
        __syncthreads();
        uint32_t jlo = 0;
        for (uint32_t base = e0; base < e1; base += nt) {
            const uint32_t e = base + tid;
            bool changed_first = false;
            uint32_t target = 0;
            if (e < e1) {
                uint32_t lo = jlo, hi = cnt - 1;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (sm.pre[mid] <= e) lo = mid; else hi = mid - 1;
                }
                jlo = lo;
                const uint2 ed = adj[sm.beg[lo] + (e - sm.pre[lo])];
                const unsigned long long ku = sm.key[lo];
                unsigned long long nk = kInfKey;
                if (ku != kPull) {
                    const uint64_t cand = (ku >> 32) + ed.y;
                    if (cand <= delta) {
                        target = ed.x;
                        nk = (cand << 32) | (ku & 0xFFFFFFFFull);
                    }
                } else if (ed.y <= delta) {
                    const uint32_t cu = __ldcg(&center[ed.x]);
                    if (cu != kNone) {
                        target = sm.v[lo];
                        nk = ((unsigned long long)ed.y << 32) | cu;
                    }
                }
                if (nk != kInfKey && nk < __ldcg(&key[target])) {
                    const unsigned long long old = atomicMin(&key[target], nk);
                    if (nk < old) {
                        newly += (old == kInfKey) ? 1 : 0;
                        changed_first = atomicExch(&stamp[target], stepid) != stepid;
                    }
                }
            }
            if (changed_first) sm.next[atomicAdd(&sm.nn, 1u)] = target;
        }
        __syncthreads();
        if (tid == 0) sm.nbase = sm.nn ? atomicAdd(&ctr->nnext, sm.nn) : 0u;  // one global atomic per chunk
        __syncthreads();
        for (uint32_t j = tid; j < sm.nn; j += nt) next[sm.nbase + j] = sm.next[j];
        __syncthreads();  // the next chunk reuses the shared arrays
    }
    warp_add_u64(&ctr->newly_covered, newly);
}

// the changed nodes become the next frontier, with their end-of-step keys
// (read after the step has finished, so they are the next step's
// start-of-step values); nodes that reached d = Delta do not relax.
__device__ __forceinline__ void dev_snapshot(const uint32_t* __restrict__ next, uint32_t nn,
                                             const unsigned long long* __restrict__ key,
                                             const uint64_t* __restrict__ off, uint32_t delta,
                                             uint32_t* __restrict__ fv, unsigned long long* __restrict__ fkey,
                                             uint32_t* __restrict__ fpre, Counters* ctr, unsigned long long* scratch,
                                             uint32_t br, uint32_t nb) {
    for (uint32_t base = br * blockDim.x; base < nn; base += nb * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        bool take = false;
        uint32_t v = 0, deg = 0;
        unsigned long long k = 0;
        if (i < nn) {
            v = __ldcg(&next[i]);
            k = __ldcg(&key[v]);
            deg = (uint32_t)(off[v + 1] - off[v]);
            take = (uint32_t)(k >> 32) < delta && deg > 0;
        }
        uint32_t slot = 0, pre = 0;
        front_append(&ctr->front, take, deg, slot, pre, scratch);
        if (take) {
            fv[slot] = v;
            fkey[slot] = k;
            fpre[slot] = pre;
        }
    }
}

// guard of the doubling loop: does any covered or frozen node have an uncovered neighbour?
__device__ __forceinline__ void dev_growable(const uint32_t* __restrict__ row, const uint2* __restrict__ adj,
                                             uint64_t nnz, const unsigned long long* __restrict__ key, Counters* ctr,
                                             uint32_t br, uint32_t nb) {
    bool any = false;
    for (uint64_t i = (uint64_t)br * blockDim.x + threadIdx.x; i < nnz; i += (uint64_t)nb * blockDim.x) {
        if (__ldcg(&key[adj[i].x]) == kInfKey && __ldcg(&key[row[i]]) != kInfKey) any = true;
    }
    if (__any_sync(0xffffffffu, any) && lane_id() == 0) atomicExch(&ctr->growable, 1u);
}

// a7 (part 1): D_v = d_v + R[c_v] for the nodes covered in this stage (R as before the stage).
__device__ __forceinline__ void dev_finalize_d(uint32_t n, const unsigned long long* __restrict__ key,
                                               const uint32_t* __restrict__ center, const uint32_t* __restrict__ R,
                                               uint32_t* __restrict__ D, Counters* ctr, uint32_t br, uint32_t nb) {
    for (uint32_t v = br * blockDim.x + threadIdx.x; v < n; v += nb * blockDim.x) {
        if (__ldcg(&center[v]) != kNone) continue;
        const unsigned long long k = __ldcg(&key[v]);
        if (k == kInfKey) continue;
        uint64_t dv = (k >> 32) + (uint64_t)__ldcg(&R[(uint32_t)k]);
        if (dv >= 0xFFFFFFFFull) {
            atomicExch(&ctr->overflow, 1u);
            dv = 0xFFFFFFFEull;
        }
        D[v] = (uint32_t)dv;
    }
}

// a7 (part 2): freeze them (key 0), record the center, grow R[c].
__device__ __forceinline__ void dev_finalize_freeze(uint32_t n, unsigned long long* __restrict__ key,
                                                    uint32_t* __restrict__ center, uint32_t* __restrict__ R,
                                                    const uint32_t* __restrict__ D, const uint64_t* __restrict__ off,
                                                    Counters* ctr, uint32_t br, uint32_t nb) {
    unsigned long long cnt = 0, degs = 0;
    for (uint32_t base = br * blockDim.x; base < n; base += nb * blockDim.x) {
        const uint32_t v = base + threadIdx.x;
        bool take = false;
        uint32_t c = kNone, dv = 0;
        if (v < n && __ldcg(&center[v]) == kNone) {
            const unsigned long long k = __ldcg(&key[v]);
            if (k != kInfKey) {
                take = true;
                c = (uint32_t)k;
                dv = __ldcg(&D[v]);
                center[v] = c;
                key[v] = 0;
                ++cnt;
                degs += off[v + 1] - off[v];
            }
        }
        // nodes of one cluster often share a warp: one atomicMax per distinct center
        const unsigned peers = __match_any_sync(0xffffffffu, take ? c : kNone);
        const uint32_t m = __reduce_max_sync(peers, dv);
        if (take && lane_id() == (unsigned)(__ffs(peers) - 1)) atomicMax(&R[c], m);
    }
    warp_add_u64(&ctr->frozen, cnt);
    warp_add_u64(&ctr->frozen_deg, degs);
}

// a8: leftover nodes become singleton clusters.
__device__ __forceinline__ void dev_singletons(uint32_t n, uint32_t* __restrict__ center, uint32_t* __restrict__ D,
                                               uint32_t br, uint32_t nb) {
    for (uint32_t v = br * blockDim.x + threadIdx.x; v < n; v += nb * blockDim.x)
        if (__ldcg(&center[v]) == kNone) {
            center[v] = v;
            D[v] = 0;
        }
}

// Stage control shared by both forms: the outer-loop test of Algorithm 1 and
// the center-draw threshold floor(p 2^32), p = gamma tau log2 n / |U|; log2 n
// comes from the host so both forms (and the oracle) use the same double.
__host__ __device__ inline bool stage_threshold(uint64_t U, double tau, double L, uint64_t* thr) {
    if (U == 0) return false;
    if ((double)U < 8.0 * tau * L) return false;
    const double p = kGamma * tau * L / (double)U;
    *thr = (p >= 1.0) ? 4294967296ull : (uint64_t)floor(p * 4294967296.0);
    return *thr != 0;
}

}  // namespace cld
