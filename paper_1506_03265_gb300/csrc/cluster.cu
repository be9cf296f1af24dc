// CLUSTER(G, tau) of Algorithm 1 on the GPU, one graph per launch: each
// phase body of cluster_dev.cuh runs as its own grid kernel and the host
// drives the stage / step / doubling control flow from small counter reads.
#include <cmath>
#include <vector>

#include "cluster_dev.cuh"
#include "internal.cuh"
#include "prof.cuh"

namespace cld {

namespace {

__global__ void k_select(uint32_t n, const uint32_t* __restrict__ center, unsigned long long* __restrict__ key,
                         uint64_t seed, uint32_t stage, uint64_t thr, Counters* ctr) {
    dev_select(n, center, key, seed, stage, thr, ctr, blockIdx.x, gridDim.x);
}

__global__ void k_rebuild(uint32_t n, const unsigned long long* __restrict__ key, const uint32_t* __restrict__ center,
                          const uint32_t* __restrict__ Dcum, const uint64_t* __restrict__ off, uint32_t delta,
                          bool pull, uint32_t* __restrict__ fbase, unsigned long long* __restrict__ fkey,
                          uint32_t* __restrict__ fpre, uint32_t* __restrict__ cfirst, Counters* ctr) {
    __shared__ unsigned long long scratch[33];
    dev_rebuild(n, key, center, Dcum, off, delta, pull, fbase, fkey, fpre, cfirst, ctr, scratch, blockIdx.x,
                gridDim.x);
}

__global__ void __launch_bounds__(RT) k_relax(const uint32_t* __restrict__ fbase,
                                              const unsigned long long* __restrict__ fkey,
                                              const uint32_t* __restrict__ fpre, const uint32_t* __restrict__ cfirst,
                                              uint32_t nf, uint32_t E, const uint2* __restrict__ adj,
                                              const uint32_t* __restrict__ center, const uint32_t* __restrict__ Dcum,
                                              unsigned long long* __restrict__ key, uint32_t delta,
                                              uint32_t* __restrict__ stamp, uint32_t stepid,
                                              uint32_t* __restrict__ next, Counters* ctr) {
    __shared__ RelaxSmem sm;
    __shared__ uint32_t nbuf[relax_nbuf_words<RU>(RT / 32)];
    dev_relax<RU>(fbase, fkey, fpre, cfirst, nf, E, adj, center, Dcum, key, delta, stamp, stepid, next, ctr, sm, nbuf,
                  blockIdx.x, gridDim.x);
}

__global__ void k_snapshot(const uint32_t* __restrict__ next, const unsigned long long* __restrict__ key,
                           const uint64_t* __restrict__ off, uint32_t delta, uint32_t* __restrict__ fbase,
                           unsigned long long* __restrict__ fkey, uint32_t* __restrict__ fpre,
                           uint32_t* __restrict__ cfirst, Counters* ctr) {
    __shared__ unsigned long long scratch[33];
    const uint32_t nn = __ldcg(&ctr->nnext);
    dev_snapshot(next, nn, key, off, delta, fbase, fkey, fpre, cfirst, ctr, scratch, blockIdx.x, gridDim.x);
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
                                  Counters* ctr) {
    dev_finalize_freeze(n, key, center, R, D, off, ctr, blockIdx.x, gridDim.x);
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

// node state before the first stage: no center, D = R = 0, no stamp, no key
__global__ void k_cluster_init(uint32_t n, uint32_t* __restrict__ center, uint32_t* __restrict__ D,
                               uint32_t* __restrict__ R, uint32_t* __restrict__ stamp,
                               unsigned long long* __restrict__ key) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        center[i] = kNone;
        D[i] = 0;
        R[i] = 0;
        stamp[i] = 0;
        key[i] = kInfKey;
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
    cl->max_fw_k = opts.max_fw_k ? opts.max_fw_k : 8192u;
    cl->quotient_mode = opts.quotient_mode;

    // a frontier lists each node at most twice (push + pull entry)
    const size_t fcap = 2 * (size_t)n;
    DBuf<uint32_t> center, D, cid;
    DBuf<unsigned long long> key, fkeyA, fkeyB;
    DBuf<uint32_t> R, stamp, fvA, fvB, fpA, fpB, cfA, cfB, next;
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
    // chunk tables: a frontier has at most 2 * nnz adjacency entries (push + pull)
    const size_t ccap = (2 * (size_t)g->nnz) / RC + 2;
    CLD_TRY(cfA.alloc(ccap, s));
    CLD_TRY(cfB.alloc(ccap, s));
    CLD_TRY(next.alloc(n, s));
    CLD_TRY(ctr.alloc(1, s));
    Counters* hc = static_cast<Counters*>(g->host.h);
    static_assert(sizeof(Counters) <= 128, "counter block must fit the pinned area");

    const unsigned gb = grid_for(n, 256);
    CLD_K(K_MISC, s, k_cluster_init<<<gb, 256, 0, s>>>(n, center.get(), D.get(), R.get(), stamp.get(), key.get()));
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
    uint32_t* cf = cfA.get();
    uint32_t* cf2 = cfB.get();
    const unsigned max_relax_grid = (unsigned)num_sms() * 8;
    // relax CTAs loop over chunks: launch exactly the resident ones (shared memory limits them to a few per
    // SM), so that no second, partial wave of CTAs runs after the first has finished its chunks
    static int relax_per_sm[64];
    int dev = 0;
    CLD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || relax_per_sm[dev] == 0) {
        int per_sm = 0;
        CLD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_relax, RT, 0));
        if (dev >= 0 && dev < 64) relax_per_sm[dev] = std::max(1, per_sm);
        else relax_per_sm[0] = std::max(1, per_sm);
    }
    const unsigned relax_grid = (unsigned)num_sms() * (unsigned)relax_per_sm[(dev >= 0 && dev < 64) ? dev : 0];
    uint32_t nf = 0, E = 0;

    // list every relaxer (stage start, or after Delta doubled)
    auto rebuild = [&]() -> cldiam_status {
        const bool pull = pull_ok && (g->nnz - frozen_deg) < frozen_deg;
        CLD_TRY(zero_field(offsetof(Counters, front), 8));
        CLD_K(K_REBUILD, s, k_rebuild<<<gb, 256, 0, s>>>(n, key.get(), center.get(), cumulative ? D.get() : nullptr,
                                                          g->off, delta, pull, fv, fk, fp, cf, ctr.get()));
        CLD_LAUNCH_CHECK();
        return CLDIAM_OK;
    };

    for (;;) {
        uint64_t thr = 0;
        if (!stage_threshold(U, tau, L, &thr)) break;  // outer while test of Algorithm 1, center draw threshold
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
            uint32_t updated, growth_steps = 0;
            do {
                ++growth_steps;
                ++stepid;
                updated = 0;
                if (nf > 0) {
                    CLD_TRY(zero_field(offsetof(Counters, newly_covered), 24));  // newly_covered, front, nnext
                    const unsigned rg = (unsigned)std::min<uint64_t>((E + RC - 1) / RC, relax_grid);
                    CLD_K(K_RELAX, s, k_relax<<<rg, RT, 0, s>>>(fv, fk, fp, cf, nf, E, g->adj, center.get(),
                                                                 cumulative ? D.get() : nullptr, key.get(), delta,
                                                                 stamp.get(), stepid, next.get(), ctr.get()));
                    CLD_LAUNCH_CHECK();
                    CLD_K(K_SNAPSHOT, s, k_snapshot<<<max_relax_grid, 256, 0, s>>>(next.get(), key.get(), g->off, delta,
                                                                                 fv2, fk2, fp2, cf2, ctr.get()));
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
        CLD_K(K_FINALIZE, s, k_finalize_d<<<gb, 256, 0, s>>>(n, key.get(), center.get(), cumulative ? nullptr : R.get(),
                                                             D.get(), ctr.get()));
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
