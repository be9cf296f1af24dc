// CLUSTER(G, tau) of Algorithm 1 on the GPU.
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
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "prof.cuh"

namespace cld {

namespace {

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
__global__ void k_select(uint32_t n, const uint32_t* __restrict__ center, unsigned long long* __restrict__ key,
                         uint64_t seed, uint32_t stage, uint64_t thr, Counters* ctr) {
    unsigned long long cnt = 0;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        uint32_t v = base + threadIdx.x;
        if (v < n && center[v] == kNone) {
            U4 r = philox4x32_10(seed, v, stage, 0u, 0u);
            bool sel = (uint64_t)r.x < thr;
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
__global__ void k_rebuild(uint32_t n, const unsigned long long* __restrict__ key, const uint32_t* __restrict__ center,
                          const uint64_t* __restrict__ off, uint32_t delta, bool pull, uint32_t* __restrict__ fv,
                          unsigned long long* __restrict__ fkey, uint32_t* __restrict__ fpre, Counters* ctr) {
    __shared__ unsigned long long scratch[33];
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        uint32_t v = base + threadIdx.x;
        bool push = false, pl = false;
        unsigned long long k = 0;
        uint32_t deg = 0;
        if (v < n) {
            deg = (uint32_t)(off[v + 1] - off[v]);
            uint32_t c = center[v];
            if (deg > 0) {
                if (c != kNone) {
                    push = !pull;
                    k = c;  // (0, c_u)
                } else {
                    k = key[v];
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

constexpr int RT = 256;   // relax threads per CTA
constexpr int RC = 1024;  // adjacency entries per chunk

// a5: one synchronous Delta-growing step over the frontier, edge-balanced:
// the frontier's adjacency lists are viewed as one flattened range of E
// entries cut into chunks of RC; each CTA takes chunks, loads the frontier
// entries the chunk spans into shared memory and maps every entry position to
// its frontier entry by binary search, so hubs spread over many CTAs.
__global__ void __launch_bounds__(RT) k_relax(const uint32_t* __restrict__ fv, const unsigned long long* __restrict__ fkey,
                                              const uint32_t* __restrict__ fpre, uint32_t nf, uint32_t E,
                                              const uint64_t* __restrict__ off, const uint2* __restrict__ adj,
                                              const uint32_t* __restrict__ center, unsigned long long* __restrict__ key,
                                              uint32_t delta, uint32_t* __restrict__ stamp, uint32_t stepid,
                                              uint32_t* __restrict__ next, Counters* ctr) {
    __shared__ uint32_t s_pre[RC];
    __shared__ uint32_t s_beg[RC];
    __shared__ uint32_t s_v[RC];
    __shared__ unsigned long long s_key[RC];
    __shared__ uint32_t s_next[RC];  // nodes first changed by this chunk (at most one per entry)
    __shared__ uint32_t s_i0, s_cnt, s_nn, s_nbase;
    const uint32_t tid = threadIdx.x;
    unsigned long long newly = 0;
    for (uint32_t chunk = blockIdx.x; (uint64_t)chunk * RC < E; chunk += gridDim.x) {
        const uint32_t e0 = chunk * RC;
        const uint32_t e1 = min(E, e0 + RC);
        if (tid == 0) {
            uint32_t lo = 0, hi = nf - 1;  // last entry starting at or before e0
            while (lo < hi) {
                uint32_t mid = (lo + hi + 1) >> 1;
                if (fpre[mid] <= e0) lo = mid; else hi = mid - 1;
            }
            uint32_t i0 = lo;
            hi = nf - 1;                    // last entry starting at or before e1 - 1
            while (lo < hi) {
                uint32_t mid = (lo + hi + 1) >> 1;
                if (fpre[mid] <= e1 - 1) lo = mid; else hi = mid - 1;
            }
            s_i0 = i0;
            s_cnt = lo - i0 + 1;
            s_nn = 0;
        }
        __syncthreads();
        const uint32_t i0 = s_i0, cnt = s_cnt;  // cnt <= RC: every entry has >= 1 adjacency entry
        for (uint32_t j = tid; j < cnt; j += RT) {
            uint32_t v = fv[i0 + j];
            s_pre[j] = fpre[i0 + j];
            s_v[j] = v;
            s_key[j] = fkey[i0 + j];
            s_beg[j] = (uint32_t)off[v];
        }
        __syncthreads();
        uint32_t jlo = 0;
        for (uint32_t base = e0; base < e1; base += RT) {
            const uint32_t e = base + tid;
            bool changed_first = false;
            uint32_t target = 0;
            if (e < e1) {
                uint32_t lo = jlo, hi = cnt - 1;
                while (lo < hi) {
                    uint32_t mid = (lo + hi + 1) >> 1;
                    if (s_pre[mid] <= e) lo = mid; else hi = mid - 1;
                }
                jlo = lo;
                const uint2 ed = adj[s_beg[lo] + (e - s_pre[lo])];
                const unsigned long long ku = s_key[lo];
                unsigned long long nk = kInfKey;
                if (ku != kPull) {
                    const uint64_t cand = (ku >> 32) + ed.y;
                    if (cand <= delta) {
                        target = ed.x;
                        nk = (cand << 32) | (ku & 0xFFFFFFFFull);
                    }
                } else if (ed.y <= delta) {
                    const uint32_t cu = center[ed.x];
                    if (cu != kNone) {
                        target = s_v[lo];
                        nk = ((unsigned long long)ed.y << 32) | cu;
                    }
                }
                if (nk != kInfKey && nk < key[target]) {
                    const unsigned long long old = atomicMin(&key[target], nk);
                    if (nk < old) {
                        newly += (old == kInfKey) ? 1 : 0;
                        changed_first = atomicExch(&stamp[target], stepid) != stepid;
                    }
                }
            }
            if (changed_first) s_next[atomicAdd(&s_nn, 1u)] = target;
        }
        __syncthreads();
        if (tid == 0) s_nbase = s_nn ? atomicAdd(&ctr->nnext, s_nn) : 0u;  // one global atomic per chunk
        __syncthreads();
        for (uint32_t j = tid; j < s_nn; j += RT) next[s_nbase + j] = s_next[j];
        __syncthreads();  // the next chunk reuses the shared arrays
    }
    warp_add_u64(&ctr->newly_covered, newly);
}

// the changed nodes become the next frontier, with their end-of-step keys
// (read after the step kernel has finished, so they are the next step's
// start-of-step values); nodes that reached d = Delta do not relax.
__global__ void k_snapshot(const uint32_t* __restrict__ next, const unsigned long long* __restrict__ key,
                           const uint64_t* __restrict__ off, uint32_t delta, uint32_t* __restrict__ fv,
                           unsigned long long* __restrict__ fkey, uint32_t* __restrict__ fpre, Counters* ctr) {
    __shared__ unsigned long long scratch[33];
    const uint32_t nn = ctr->nnext;
    for (uint32_t base = blockIdx.x * blockDim.x; base < nn; base += gridDim.x * blockDim.x) {
        uint32_t i = base + threadIdx.x;
        bool take = false;
        uint32_t v = 0, deg = 0;
        unsigned long long k = 0;
        if (i < nn) {
            v = next[i];
            k = key[v];
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
__global__ void k_growable(const uint32_t* __restrict__ row, const uint2* __restrict__ adj, uint64_t nnz,
                           const unsigned long long* __restrict__ key, Counters* ctr) {
    bool any = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (uint64_t)gridDim.x * blockDim.x) {
        if (key[adj[i].x] == kInfKey && key[row[i]] != kInfKey) any = true;
    }
    if (__any_sync(0xffffffffu, any) && lane_id() == 0) atomicExch(&ctr->growable, 1u);
}

// a7 (part 1): D_v = d_v + R[c_v] for the nodes covered in this stage (R as before the stage).
__global__ void k_finalize_d(uint32_t n, const unsigned long long* __restrict__ key, const uint32_t* __restrict__ center,
                             const uint32_t* __restrict__ R, uint32_t* __restrict__ D, Counters* ctr) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (center[v] != kNone) continue;
        unsigned long long k = key[v];
        if (k == kInfKey) continue;
        uint64_t dv = (k >> 32) + (uint64_t)R[(uint32_t)k];
        if (dv >= 0xFFFFFFFFull) {
            atomicExch(&ctr->overflow, 1u);
            dv = 0xFFFFFFFEull;
        }
        D[v] = (uint32_t)dv;
    }
}

// a7 (part 2): freeze them (key 0), record the center, grow R[c].
__global__ void k_finalize_freeze(uint32_t n, unsigned long long* __restrict__ key, uint32_t* __restrict__ center,
                                  uint32_t* __restrict__ R, const uint32_t* __restrict__ D, const uint64_t* __restrict__ off,
                                  Counters* ctr) {
    unsigned long long cnt = 0, degs = 0;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t v = base + threadIdx.x;
        bool take = false;
        uint32_t c = kNone, dv = 0;
        if (v < n && center[v] == kNone) {
            const unsigned long long k = key[v];
            if (k != kInfKey) {
                take = true;
                c = (uint32_t)k;
                dv = D[v];
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
__global__ void k_singletons(uint32_t n, uint32_t* __restrict__ center, uint32_t* __restrict__ D) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (center[v] == kNone) {
            center[v] = v;
            D[v] = 0;
        }
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

__global__ void k_fill_u32(uint32_t* __restrict__ a, uint32_t n, uint32_t x) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = x;
}
__global__ void k_fill_u64(unsigned long long* __restrict__ a, uint32_t n, unsigned long long x) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = x;
}

struct ClusterOwner {
    cldiam_clustering* c;
    explicit ClusterOwner(cldiam_clustering* x) : c(x) {}
    ~ClusterOwner() {
        if (c) free_clustering(c);
    }
};

}  // namespace

void free_clustering(cldiam_clustering* c) {
    if (!c) return;
    cudaStream_t s = c->g ? c->g->stream : nullptr;
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
    if (opts.contract_mode != 0 || opts.step_cap != 0 || opts.reserved[0] || opts.reserved[1] || opts.reserved[2])
        return fail(CLDIAM_ERR_UNSUPPORTED, "only contract_mode 0 without a step cap is implemented");
    uint32_t delta = 0;
    CLD_TRY(delta0(g, opts.delta0_mode, opts.delta0, &delta));

    const cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    ClusterOwner owner(new cldiam_clustering());
    cldiam_clustering* cl = owner.c;
    cl->g = g;
    cl->max_fw_k = opts.max_fw_k ? opts.max_fw_k : 8192u;

    // a frontier lists each node at most twice (push + pull entry)
    const size_t fcap = 2 * (size_t)n;
    DBuf<uint32_t> center, D, cid;
    DBuf<unsigned long long> key, fkeyA, fkeyB;
    DBuf<uint32_t> R, stamp, fvA, fvB, fpA, fpB, next;
    DBuf<Counters> ctr;
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
    CLD_TRY(next.alloc(n, s));
    CLD_TRY(ctr.alloc(1, s));
    Counters* hc = static_cast<Counters*>(g->host.h);
    static_assert(sizeof(Counters) <= 128, "counter block must fit the pinned area");

    const unsigned gb = grid_for(n, 256);
    CLD_K(K_MISC, s, k_fill_u32<<<gb, 256, 0, s>>>(center.get(), n, kNone));
    CLD_K(K_MISC, s, k_fill_u32<<<gb, 256, 0, s>>>(D.get(), n, 0u));
    CLD_K(K_MISC, s, k_fill_u32<<<gb, 256, 0, s>>>(R.get(), n, 0u));
    CLD_K(K_MISC, s, k_fill_u32<<<gb, 256, 0, s>>>(stamp.get(), n, 0u));
    CLD_K(K_MISC, s, k_fill_u64<<<gb, 256, 0, s>>>(key.get(), n, kInfKey));
    CLD_LAUNCH_CHECK();
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
    const unsigned max_relax_grid = (unsigned)num_sms() * 8;
    uint32_t nf = 0, E = 0;

    // list every relaxer (stage start, or after Delta doubled)
    auto rebuild = [&]() -> cldiam_status {
        const bool pull = pull_ok && (g->nnz - frozen_deg) < frozen_deg;
        CLD_TRY(zero_field(offsetof(Counters, front), 8));
        CLD_K(K_REBUILD, s, k_rebuild<<<gb, 256, 0, s>>>(n, key.get(), center.get(), g->off, delta, pull, fv, fk, fp,
                                                          ctr.get()));
        CLD_LAUNCH_CHECK();
        return CLDIAM_OK;
    };

    for (;;) {
        if (U == 0) break;
        if ((double)U < 8.0 * tau * L) break;  // outer while test of Algorithm 1
        const double p = kGamma * tau * L / (double)U;
        const uint64_t thr = (p >= 1.0) ? 4294967296ull : (uint64_t)std::floor(p * 4294967296.0);
        if (thr == 0) break;
        if (stage > kMaxStages) return fail(CLDIAM_ERR_DIVERGED, "CLUSTER exceeded its stage limit");

        // selection + reset, then the stage's first frontier
        CLD_TRY(zero_field(offsetof(Counters, selected), 8));
        CLD_K(K_SELECT, s, k_select<<<gb, 256, 0, s>>>(n, center.get(), key.get(), seed, stage, thr, ctr.get()));
        CLD_LAUNCH_CHECK();
        CLD_TRY(rebuild());
        CLD_TRY(sync_counters());
        uint64_t covered = hc->selected;
        nf = (uint32_t)(hc->front >> 32);
        E = (uint32_t)hc->front;
        st.centers_drawn += hc->selected;

        for (;;) {
            uint32_t updated;
            do {
                ++stepid;
                updated = 0;
                if (nf > 0) {
                    CLD_TRY(zero_field(offsetof(Counters, newly_covered), 8));
                    CLD_TRY(zero_field(offsetof(Counters, front), 8));
                    CLD_TRY(zero_field(offsetof(Counters, nnext), 4));
                    const unsigned rg = (unsigned)std::min<uint64_t>((E + RC - 1) / RC, max_relax_grid);
                    CLD_K(K_RELAX, s, k_relax<<<rg, RT, 0, s>>>(fv, fk, fp, nf, E, g->off, g->adj, center.get(),
                                                                 key.get(), delta, stamp.get(), stepid, next.get(),
                                                                 ctr.get()));
                    CLD_LAUNCH_CHECK();
                    CLD_K(K_SNAPSHOT, s, k_snapshot<<<max_relax_grid, 256, 0, s>>>(next.get(), key.get(), g->off, delta,
                                                                                 fv2, fk2, fp2, ctr.get()));
                    CLD_LAUNCH_CHECK();
                    CLD_TRY(sync_counters());
                    updated = hc->nnext;
                    covered += hc->newly_covered;
                    st.edges_scanned += E;
                    // algorithmic bytes of this relax launch: per frontier entry its slot (4 + 8 + 4 B)
                    // and row start (8 B); per adjacency entry the (col, w) pair (8 B) and the target's
                    // key (8 B); per changed node its key, stamp and list slot (16 B)
                    prof_add_bytes(K_RELAX, 24.0 * nf + 16.0 * (double)E + 16.0 * updated);
                    prof_add_bytes(K_SNAPSHOT, 4.0 * updated + 8.0 * updated + 16.0 * updated + 16.0 * (hc->front >> 32));
                    std::swap(fv, fv2);
                    std::swap(fp, fp2);
                    std::swap(fk, fk2);
                    nf = (uint32_t)(hc->front >> 32);
                    E = (uint32_t)hc->front;
                }
                st.steps++;
                st.node_updates += updated;
            } while (updated != 0 && 2 * covered < U);
            if (2 * covered >= U) break;
            bool growable = false;
            if (delta < kDeltaMax && g->connected) {
                // connected graph: some covered or frozen node touches an uncovered one iff any exists
                growable = covered > 0 || U < n;
            } else if (delta < kDeltaMax && g->nnz) {
                CLD_TRY(zero_field(offsetof(Counters, growable), 4));
                CLD_K(K_GROWABLE, s, k_growable<<<grid_for(g->nnz, 256), 256, 0, s>>>(g->row, g->adj, g->nnz,
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
        CLD_K(K_FINALIZE, s, k_finalize_d<<<gb, 256, 0, s>>>(n, key.get(), center.get(), R.get(), D.get(), ctr.get()));
        CLD_K(K_FINALIZE, s, k_finalize_freeze<<<gb, 256, 0, s>>>(n, key.get(), center.get(), R.get(), D.get(), g->off,
                                                                  ctr.get()));
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

    // relabel
    DBuf<uint32_t> flag, rank, kdev;
    CLD_TRY(flag.alloc(n, s));
    CLD_TRY(rank.alloc(n, s));
    CLD_TRY(kdev.alloc(1, s));
    CLD_K(K_MISC, s, k_center_flags<<<gb, 256, 0, s>>>(n, center.get(), flag.get()));
    CLD_LAUNCH_CHECK();
    CLD_TRY(scan_exclusive_u32(flag.get(), rank.get(), n, kdev.get(), s));
    CLD_K(K_MISC, s, k_assign_cid<<<gb, 256, 0, s>>>(n, center.get(), rank.get(), cid.get()));
    CLD_LAUNCH_CHECK();
    uint32_t* hk = reinterpret_cast<uint32_t*>(static_cast<char*>(g->host.h) + 128);
    CLD_CUDA(cudaMemcpyAsync(hk, kdev.get(), 4, cudaMemcpyDeviceToHost, s));
    CLD_TRY(sync_counters());
    st.k = *hk;
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
