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
// In the cumulative contract mode (Dcum != nullptr) a frozen node relaxes
// with its own bound (D_u, c_u) instead, and only while D_u < Delta.
//
// Steps are synchronous: each frontier entry carries the key its node had
// at the start of the step, so in-place atomicMin gives exactly the
// start-of-step (Jacobi) semantics of the paper's "in parallel" step.  The
// next frontier is the set of nodes whose key decreased (deduplicated with a
// per-node step stamp); nodes whose key did not change would only repeat
// candidates that are already applied.  After a stage start or a Delta
// doubling every relaxer is listed again.
//
// A frontier entry is three parallel words: key (the start-of-step key of a
// pushing node, or kPullTag | v for a node that pulls), pre (its first
// position in the frontier's flattened adjacency) and base = off[v] - pre
// (mod 2^32), so that adjacency index = base + position.
//
// Mutable node state is read with L2 loads (__ldcg): inside one persistent
// CTA there is no kernel boundary to drop stale L1 lines between phases.
#pragma once

#include <cstddef>

#include "common.cuh"

namespace cld {

struct Counters {
    unsigned long long selected;       // centers drawn in this stage
    unsigned long long edges_scanned;  // adjacency entries read by relax
    unsigned long long frozen;         // nodes frozen by finalize
    unsigned long long frozen_deg;     // their degree sum
    // reset before every growing step (one contiguous block)
    unsigned long long newly_covered;  // nodes that got their first key this step
    unsigned long long front;          // next frontier: (entries << 32) | adjacency entries
    uint32_t nnext;                    // changed nodes this step
    uint32_t pad;
    // others
    uint32_t growable;                 // some covered/frozen node touches an uncovered one
    uint32_t overflow;                 // a D_v reached 2^32 - 1
    unsigned long long unfrozen;       // unfrozen nodes the stage's draw saw (checks the tracked |U|)
};
static_assert(offsetof(Counters, pad) + 4 - offsetof(Counters, newly_covered) == 24,
              "the per-step counters form one block");

constexpr int RC = 1024;  // adjacency entries per relax chunk of one CTA (the many-graph form)
constexpr int QC = 128;   // frontier positions per chunk-table slot (one warp chunk of the one-graph form)
// In shared memory a pull entry's key is kPullTag | v: a pushed key has
// d < Delta <= 2^31, so its high word is never all ones.
constexpr unsigned long long kPullTag = 0xFFFFFFFF00000000ull;

// Chunk table of a frontier: cfirst[c] = the entry whose adjacency range
// holds flattened position c * QC.  The producer of each entry writes the
// chunk starts that fall inside its range, so relax finds a chunk's entries
// with two loads instead of a search over the frontier.
__device__ __forceinline__ void chunk_table_put(uint32_t* __restrict__ cfirst, uint32_t slot, uint32_t pre,
                                                uint32_t deg) {
    const uint64_t end = (uint64_t)pre + deg;
    for (uint64_t c = ((uint64_t)pre + QC - 1) / QC; c * QC < end; ++c) cfirst[c] = slot;
}

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

// ---------------------------------------------------------------- warp-chunk sweeps
// The one-graph kernels that sweep a flattened range of positions (a
// frontier's adjacency, or the whole CSR) give each warp PW consecutive
// positions (PWG groups of 32 lanes) and run without block barriers.
constexpr int PT = 256;          // threads per CTA of the warp-chunk kernels
constexpr int PW = 128;          // positions per warp chunk (== QC, the chunk-table granularity)
constexpr int PWG = PW / 32;     // groups of 32 positions per chunk
constexpr int PNB = 2 * PW + 8;  // per-warp buffer of changed nodes (flushed once >= PW)
static_assert(PW == QC, "one chunk-table slot per warp chunk");

// Row (or frontier entry) segments of a warp's 32-position group.  Entries
// start at strictly increasing positions and each holds at least one; B is
// the index of the entry that holds position g0 (the group's first), and
// starts[j] the first position of entry B + 1 + j for j < n_after.  Returns
// the group's start word (bit d = an entry starts at g0 + d); *own = the
// entry index of this lane's position.
__device__ __forceinline__ uint32_t group_starts(const uint32_t* starts, uint32_t n_after, uint32_t g0,
                                                 uint32_t B, uint32_t lane, unsigned le_mask, uint32_t* own) {
    const uint32_t d = (lane < n_after ? starts[lane] : 0xFFFFFFFFu) - g0;  // entries after B start after g0
    const uint32_t word = __reduce_or_sync(0xffffffffu, d < 32u ? 1u << d : 0u);
    *own = B + (uint32_t)__popc(word & le_mask);
    return word;
}

// Minimum of v over this lane's segment [head, tail] of a group (segments are
// runs of consecutive lanes bounded by the start word); valid at every lane,
// so the head lane holds the segment's minimum.
__device__ __forceinline__ unsigned long long segment_min(unsigned long long v, uint32_t word, uint32_t lane) {
    const unsigned above = lane == 31 ? 0u : word & (0xfffffffeu << lane);
    const uint32_t tail = above ? (uint32_t)__ffs(above) - 2u : 31u;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_down_sync(0xffffffffu, v, o);
        if (lane + o <= tail) v = t < v ? t : v;
    }
    return v;
}

// Per-warp list of changed nodes, appended to the next list with one atomic per >= PW of them.
struct WarpNext {
    uint32_t* buf;
    uint32_t cnt;
    __device__ __forceinline__ void put(bool first, uint32_t r, uint32_t lane) {
        const unsigned m = __ballot_sync(0xffffffffu, first);
        if (first) buf[cnt + (uint32_t)__popc(m & lanemask_lt())] = r;
        cnt += (uint32_t)__popc(m);
    }
    __device__ __forceinline__ void flush(uint32_t* __restrict__ next, uint32_t* counter, uint32_t lane) {
        __syncwarp();
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(counter, cnt);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (uint32_t j = lane; j < cnt; j += 32) next[base + j] = buf[j];
        cnt = 0;
        __syncwarp();
    }
};

// a3: draw the new centers of this stage among unfrozen nodes, reset the others.
__device__ __forceinline__ void dev_select(uint32_t n, const uint32_t* __restrict__ center,
                                           unsigned long long* __restrict__ key, uint64_t seed, uint32_t stage,
                                           uint64_t thr, Counters* ctr, uint32_t br, uint32_t nb,
                                           unsigned long long* __restrict__ keyS = nullptr) {
    unsigned long long cnt = 0, unfrozen = 0;
    for (uint32_t base = br * blockDim.x; base < n; base += nb * blockDim.x) {
        const uint32_t v = base + threadIdx.x;
        if (v < n && __ldcg(&center[v]) == kNone) {
            const U4 r = philox4x32_10(seed, v, stage, 0u, 0u);
            const bool sel = (uint64_t)r.x < thr;
            key[v] = sel ? (unsigned long long)v : kInfKey;
            if (keyS) keyS[v] = sel ? (unsigned long long)v : kInfKey;
            cnt += sel ? 1 : 0;
            ++unfrozen;
        }
    }
    warp_add_u64(&ctr->selected, cnt);
    warp_add_u64(&ctr->unfrozen, unfrozen);
}

// a4: list every relaxer with its current key: unfrozen nodes with d < Delta
// push their key; the contracted clusters either push (0, c_u) from every
// frozen u, or (pull mode) every unfrozen node lists itself to pull
// (w, c_u) from its frozen neighbours -- the same candidates, read from the
// side with fewer adjacency entries.
__device__ __forceinline__ void dev_rebuild(uint32_t n, const unsigned long long* __restrict__ key,
                                            const uint32_t* __restrict__ center, const uint32_t* __restrict__ Dcum,
                                            const uint64_t* __restrict__ off, uint32_t delta, bool pull,
                                            uint32_t* __restrict__ fbase,
                                            unsigned long long* __restrict__ fkey, uint32_t* __restrict__ fpre,
                                            uint32_t* __restrict__ cfirst, Counters* ctr, unsigned long long* scratch,
                                            uint32_t br, uint32_t nb) {
    for (uint32_t base = br * blockDim.x; base < n; base += nb * blockDim.x) {
        const uint32_t v = base + threadIdx.x;
        bool push = false, pl = false;
        unsigned long long k = 0;
        uint32_t deg = 0, b0 = 0;
        if (v < n) {
            const uint64_t o = off[v];
            b0 = (uint32_t)o;
            deg = (uint32_t)(off[v + 1] - o);
            const uint32_t c = __ldcg(&center[v]);
            if (deg > 0) {
                if (c != kNone) {
                    const uint32_t dd = Dcum ? __ldcg(&Dcum[v]) : 0u;  // (0, c_u), or (D_u, c_u) cumulative
                    push = !pull && dd < delta;
                    k = ((unsigned long long)dd << 32) | c;
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
            fbase[slot] = b0 - pre;
            fkey[slot] = k;
            fpre[slot] = pre;
            if (cfirst) chunk_table_put(cfirst, slot, pre, deg);
        }
        front_append(&ctr->front, pl, deg, slot, pre, scratch);
        if (pl) {
            fbase[slot] = b0 - pre;
            fkey[slot] = kPullTag | v;
            fpre[slot] = pre;
            if (cfirst) chunk_table_put(cfirst, slot, pre, deg);
        }
    }
}

// Shared memory of the relax chunks: the frontier entries a chunk spans,
// double-buffered so that one block barrier per chunk separates staging from
// use (a buffer is restaged only after every thread has passed the barrier
// that follows its last use).
struct RelaxSmem {
    uint32_t pre[2][RC + 1];              // entry's first position in the flattened list
    uint32_t base[2][RC + 1];             // off[v] - pre (mod 2^32): adjacency index = base + position
    unsigned long long key[2][RC + 1];    // start-of-step key, or kPullTag | v for a pull entry
};
// Changed nodes waiting to be appended to the next list: 2 x U x 32 words per
// warp, flushed once half full.
template <int U>
constexpr int relax_nbuf_words(int warps) { return warps * 2 * U * 32; }

// largest i < n with a[i] <= x, for nondecreasing a with a[lo] <= x: a
// blockDim-ary search, one probe per thread and one barrier per round.
__device__ __forceinline__ uint32_t block_last_le(const uint32_t* __restrict__ a, uint32_t lo, uint32_t n, uint32_t x) {
    uint32_t len = n - lo;
    while (len > 1) {
        const uint32_t step = (len + blockDim.x - 1) / blockDim.x;
        const uint64_t idx = (uint64_t)lo + (uint64_t)threadIdx.x * step;
        const bool pred = threadIdx.x > 0 && idx < (uint64_t)lo + len && __ldcg(&a[idx]) <= x;
        const uint32_t c = (uint32_t)__syncthreads_count(pred);  // probes 1..c hold, the rest do not
        const uint32_t nlo = lo + c * step;
        len = min(step, lo + len - nlo);
        lo = nlo;
    }
    return lo;
}

__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// a5: one synchronous Delta-growing step over the frontier, edge-balanced:
// the frontier's adjacency lists are viewed as one flattened range of E
// entries cut into chunks of U x blockDim.x; each CTA takes chunks, each warp
// U x 32 consecutive positions of it, and maps every position to its
// frontier entry from the entries the chunk spans, held in shared memory, so
// hubs spread over many CTAs.  A block-wide search finds a chunk's entries.  The entries of the
// next chunk are copied into the other shared buffer (cp.async) while the
// current one is processed, so one barrier per chunk remains.  Every thread
// handles U positions per chunk with their loads issued together; a key is
// lowered with a plain atomicMin whose result is not needed, and the
// per-step stamp decides both "first change this step" (the node joins the
// next list) and "newly covered" (a node that was never lowered before had
// no key: centers and frozen nodes cannot be lowered).  Changed nodes gather
// in a per-warp shared buffer that is appended to the next list with one
// atomic per U x 32 or more nodes.  L2STAGE: the frontier entries are staged
// with L2 loads instead of cp.async through L1 (several CTAs of one job write
// the frontier, and none of them ends its kernel between steps).
template <int U, bool L2STAGE = false>
__device__ __forceinline__ void dev_relax(const uint32_t* __restrict__ fbase, const unsigned long long* __restrict__ fkey,
                                          const uint32_t* __restrict__ fpre,
                                          uint32_t nf, uint32_t E, const uint2* __restrict__ adj,
                                          const uint32_t* __restrict__ center, const uint32_t* __restrict__ Dcum,
                                          unsigned long long* __restrict__ key, uint32_t delta,
                                          uint32_t* __restrict__ stamp, uint32_t stepid,
                                          uint32_t* __restrict__ next, Counters* ctr, RelaxSmem& sm,
                                          uint32_t* nbuf, uint32_t br, uint32_t nb) {
    constexpr uint32_t kNB = 2 * U * 32;  // a chunk adds at most U x 32 nodes per warp
    const uint32_t tid = threadIdx.x, nt = blockDim.x, CL = U * nt;  // CL <= RC
    const uint64_t pol_stream = l2_evict_first_policy(), pol_keep = l2_evict_last_policy();
    unsigned long long newly = 0;
    uint32_t* wbuf = nbuf + (tid >> 5) * kNB;
    uint32_t wcnt = 0;  // entries in this warp's buffer (warp-uniform)
    const auto flush = [&]() {  // one atomic per kNB / 2 or more changed nodes
        uint32_t wb = 0;
        if (lane_id() == 0) wb = atomicAdd(&ctr->nnext, wcnt);
        wb = __shfl_sync(0xffffffffu, wb, 0);
        for (uint32_t j = lane_id(); j < wcnt; j += 32) next[wb + j] = wbuf[j];
        wcnt = 0;
        __syncwarp();
    };
    // entries [i0, i0 + cnt) that chunk c spans (cnt <= CL + 1: every entry has >= 1 adjacency entry)
    const auto range_of = [&](uint32_t c, uint32_t& i0, uint32_t& cnt) {
        const uint32_t e0 = c * CL;
        const uint32_t e1 = (uint32_t)min((uint64_t)E, (uint64_t)e0 + CL);
        i0 = block_last_le(fpre, 0, nf, e0);
        const uint32_t il = block_last_le(fpre, i0, nf, e1 - 1);
        cnt = il - i0 + 1;
    };
    const auto stage = [&](uint32_t b, uint32_t i0, uint32_t cnt) {
        for (uint32_t j = tid; j < cnt; j += nt) {
            if constexpr (L2STAGE) {
                sm.pre[b][j] = __ldcg(&fpre[i0 + j]);
                sm.base[b][j] = __ldcg(&fbase[i0 + j]);
                sm.key[b][j] = __ldcg(&fkey[i0 + j]);
            } else {
                cp_async_4(&sm.pre[b][j], &fpre[i0 + j]);
                cp_async_4(&sm.base[b][j], &fbase[i0 + j]);
                cp_async_8(&sm.key[b][j], &fkey[i0 + j]);
            }
        }
    };
    uint32_t chunk = br;  // chunks br, br + nb, ...
    if ((uint64_t)chunk * CL >= E) return;
    uint32_t i0, cnt;
    range_of(chunk, i0, cnt);
    stage(0, i0, cnt);
    cp_async_commit_wait_all();
    __syncthreads();
    for (uint32_t b = 0;; b ^= 1) {
        const uint32_t e0 = chunk * CL;
        const uint32_t e1 = (uint32_t)min((uint64_t)E, (uint64_t)e0 + CL);
        const uint32_t nchunk = chunk + nb;
        const bool has_next = (uint64_t)nchunk * CL < E;
        uint32_t ni0 = 0, ncnt = 0;
        if (has_next) {
            range_of(nchunk, ni0, ncnt);
            stage(b ^ 1, ni0, ncnt);  // buffer b ^ 1 was last read before the previous barrier
        }
        // owners of this warp's U x 32 consecutive positions: one binary search for the first, then
        // per group of 32 the entries starting inside it are found with one OR-reduction (at most 32
        // entries start in 32 positions, and they follow the previous group's last owner)
        uint32_t pos[U], own[U];
        {
            const uint32_t lane = lane_id();
            const uint32_t wp0 = e0 + (tid >> 5) * 32u * U;
            uint32_t B = 0;
            if (wp0 < e1) {
                // entry j >= 1 starts at or after e0 + j, so the owner of position r is <= r
                uint32_t lo = 0, hi = min(cnt - 1, wp0 - e0);
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (sm.pre[b][mid] <= wp0) lo = mid; else hi = mid - 1;
                }
                B = lo;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t p0 = wp0 + 32u * u;
                pos[u] = p0 + lane;
                const uint32_t jj = B + 1 + lane;
                const uint32_t pj = jj < cnt ? sm.pre[b][jj] : 0xFFFFFFFFu;
                const uint32_t d = pj - p0;  // entries after B start at or after p0
                const unsigned word = __reduce_or_sync(0xffffffffu, d < 32u ? 1u << d : 0u);
                own[u] = B + (uint32_t)__popc(word & (0xffffffffu >> (31u - lane)));
                B += (uint32_t)__popc(word);
            }
        }
        uint2 ed[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            ed[u] = pos[u] < e1 ? ld_stream_u2(adj + (sm.base[b][own[u]] + pos[u]), pol_stream)
                                : make_uint2(0u, 0xFFFFFFFFu);
        uint32_t target[U];
        unsigned long long nk[U], cur[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned long long ku = sm.key[b][own[u]];
            nk[u] = kInfKey;
            target[u] = 0;
            if (pos[u] < e1) {
                if ((ku & kPullTag) != kPullTag) {
                    const uint64_t cand = (ku >> 32) + ed[u].y;
                    if (cand <= delta) {
                        target[u] = ed[u].x;
                        nk[u] = (cand << 32) | (ku & 0xFFFFFFFFull);
                    }
                } else if (ed[u].y <= delta) {
                    const uint32_t cu = __ldcg(&center[ed[u].x]);
                    if (cu != kNone) {
                        const uint64_t cand = (uint64_t)(Dcum ? __ldcg(&Dcum[ed[u].x]) : 0u) + ed[u].y;
                        if (cand <= delta) {
                            target[u] = (uint32_t)ku;
                            nk[u] = (cand << 32) | cu;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) cur[u] = nk[u] != kInfKey ? ld_cg_keep_u64(&key[target[u]], pol_keep) : 0ull;
        bool first[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            first[u] = false;
            if (nk[u] < cur[u]) {
                // the key is below its start-of-step value after this, whoever wins the minimum
                red_min_keep_u64(&key[target[u]], nk[u], pol_keep);
                // only the first changers of a node this step need the exchange (hubs see many)
                if (__ldcg(&stamp[target[u]]) != stepid) {
                    const uint32_t old = atomicExch(&stamp[target[u]], stepid);
                    first[u] = old != stepid;
                    newly += old == 0u ? 1 : 0;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned m = __ballot_sync(0xffffffffu, first[u]);
            if (first[u]) wbuf[wcnt + (uint32_t)__popc(m & lanemask_lt())] = target[u];
            wcnt += (uint32_t)__popc(m);
        }
        __syncwarp();
        if (wcnt >= kNB / 2) flush();
        cp_async_commit_wait_all();
        __syncthreads();
        if (!has_next) break;
        chunk = nchunk;
        i0 = ni0;
        cnt = ncnt;
    }
    if (wcnt) flush();
    warp_add_u64(&ctr->newly_covered, newly);
}

// the changed nodes become the next frontier, with their end-of-step keys
// (read after the step has finished, so they are the next step's
// start-of-step values); nodes that reached d = Delta do not relax.
__device__ __forceinline__ void dev_snapshot(const uint32_t* __restrict__ next, uint32_t nn,
                                             const unsigned long long* __restrict__ key,
                                             const uint64_t* __restrict__ off, uint32_t delta,
                                             uint32_t* __restrict__ fbase, unsigned long long* __restrict__ fkey,
                                             uint32_t* __restrict__ fpre, uint32_t* __restrict__ cfirst, Counters* ctr,
                                             unsigned long long* scratch, uint32_t br, uint32_t nb,
                                             unsigned long long* __restrict__ keyS = nullptr) {
    for (uint32_t base = br * blockDim.x; base < nn; base += nb * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        bool take = false;
        uint32_t v = 0, deg = 0, b0 = 0;
        unsigned long long k = 0;
        if (i < nn) {
            v = __ldcg(&next[i]);
            k = __ldcg(&key[v]);
            if (keyS) keyS[v] = k;  // the next step's start-of-step key
            const uint64_t o = off[v];
            b0 = (uint32_t)o;
            deg = (uint32_t)(off[v + 1] - o);
            take = (uint32_t)(k >> 32) < delta && deg > 0;
        }
        uint32_t slot = 0, pre = 0;
        front_append(&ctr->front, take, deg, slot, pre, scratch);
        if (take) {
            fbase[slot] = b0 - pre;
            fkey[slot] = k;
            fpre[slot] = pre;
            if (cfirst) chunk_table_put(cfirst, slot, pre, deg);
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

// a7 (part 1): D_v = d_v + R[c_v] for the nodes covered in this stage (R as before the stage);
// D_v = d_v in the cumulative contract mode (R null), whose d_v already bounds dist_G(c_v, v).
__device__ __forceinline__ void dev_finalize_d(uint32_t n, const unsigned long long* __restrict__ key,
                                               const uint32_t* __restrict__ center, const uint32_t* __restrict__ R,
                                               uint32_t* __restrict__ D, Counters* ctr, uint32_t br, uint32_t nb) {
    for (uint32_t v = br * blockDim.x + threadIdx.x; v < n; v += nb * blockDim.x) {
        if (__ldcg(&center[v]) != kNone) continue;
        const unsigned long long k = __ldcg(&key[v]);
        if (k == kInfKey) continue;
        uint64_t dv = (k >> 32) + (R ? (uint64_t)__ldcg(&R[(uint32_t)k]) : 0ull);  // cumulative mode: R null
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
                                                    Counters* ctr, uint32_t br, uint32_t nb,
                                                    unsigned long long* __restrict__ keyS = nullptr,
                                                    bool cumulative = false) {
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
                // as a relaxer a contracted node holds (0, c_v), or (D_v, c_v) in the cumulative mode
                if (keyS) keyS[v] = ((cumulative ? (unsigned long long)dv : 0ull) << 32) | c;
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
