// Delta-stepping SSSP (Meyer and Sanders, J. Algorithms 2003), the parallel
// SSSP the paper compares against (Sections 1 and 5): bucket i holds the
// nodes with tentative distance in [i Delta, (i+1) Delta).  The current
// bucket is settled by repeated rounds over its light edges (w <= Delta);
// then the heavy edges (w > Delta) of every node settled in it are relaxed
// once; the next non-empty bucket is then taken from the far pile.  Twice
// the source's eccentricity is the SSSP 2-approximation of the diameter.
//
// Dedup: a node enters a light round's frontier at most once per round
// (round stamp), the bucket's settled list once per bucket and the far pile
// once per bucket epoch (epoch stamps); stale far entries are dropped when
// the next bucket is chosen.
#include "internal.cuh"
#include "prof.cuh"

namespace cld {

namespace {

struct SCounters {
    uint32_t nnext;      // next light-round frontier
    uint32_t nsettled;   // nodes settled in the current bucket
    uint32_t nfar;       // far pile entries appended
    uint32_t nfar2;      // far pile after compaction
    uint32_t overflow;
    uint32_t minbucket;  // smallest bucket index in the far pile
    uint32_t pad[2];
};

// one light round (heavy = false) over `list`, or the heavy phase (heavy = true); one warp per node
__global__ void __launch_bounds__(256) k_ds_relax(const uint32_t* __restrict__ list, uint32_t nl, bool heavy,
                                                  const uint64_t* __restrict__ off, const uint2* __restrict__ adj,
                                                  uint32_t* __restrict__ dist, uint32_t delta, uint64_t hi,
                                                  uint32_t* __restrict__ rstamp, uint32_t round_id,
                                                  uint32_t* __restrict__ sstamp, uint32_t* __restrict__ fstamp,
                                                  uint32_t epoch, uint32_t* __restrict__ next,
                                                  uint32_t* __restrict__ settled, uint32_t* __restrict__ far,
                                                  SCounters* ctr) {
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t lane = lane_id();
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nl; i += warps) {
        const uint32_t u = list[i];
        if (!heavy && lane == 0 && atomicExch(&sstamp[u], epoch) != epoch) settled[atomicAdd(&ctr->nsettled, 1u)] = u;
        const uint64_t du = dist[u];
        const uint64_t beg = off[u], end = off[u + 1];
        for (uint64_t b = beg; b < end; b += 32) {
            const uint64_t j = b + lane;
            bool to_next = false, to_far = false;
            uint32_t v = 0;
            if (j < end) {
                const uint2 e = adj[j];
                v = e.x;
                const bool light = e.y <= delta;
                if (light != heavy) {
                    const uint64_t nd = du + e.y;
                    if (nd >= 0xFFFFFFFFull) {
                        atomicExch(&ctr->overflow, 1u);
                    } else if ((uint32_t)nd < dist[v]) {
                        const uint32_t old = atomicMin(&dist[v], (uint32_t)nd);
                        if ((uint32_t)nd < old) {
                            if (nd < hi) to_next = atomicExch(&rstamp[v], round_id) != round_id;
                            else to_far = atomicExch(&fstamp[v], epoch) != epoch;
                        }
                    }
                }
            }
            uint32_t s1 = warp_append(&ctr->nnext, to_next);
            if (to_next) next[s1] = v;
            uint32_t s2 = warp_append(&ctr->nfar, to_far);
            if (to_far) far[s2] = v;
        }
    }
}

// smallest bucket among far entries still beyond the settled range
__global__ void k_ds_minbucket(const uint32_t* __restrict__ far, uint32_t nfar, const uint32_t* __restrict__ dist,
                               uint64_t hi, uint32_t delta, SCounters* ctr) {
    uint32_t m = 0xFFFFFFFFu;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nfar; i += gridDim.x * blockDim.x) {
        uint32_t d = dist[far[i]];
        if ((uint64_t)d >= hi) m = min(m, d / delta);
    }
    m = block_reduce(m, [](uint32_t a, uint32_t b) { return a < b ? a : b; }, 0xFFFFFFFFu);
    if (threadIdx.x == 0) atomicMin(&ctr->minbucket, m);
}

// split the far pile: entries of the new bucket become the frontier, later ones stay (re-stamped)
__global__ void k_ds_split(const uint32_t* __restrict__ far, uint32_t nfar, const uint32_t* __restrict__ dist,
                           uint64_t old_hi, uint64_t new_hi, uint32_t* __restrict__ fstamp, uint32_t new_epoch,
                           uint32_t* __restrict__ cur, uint32_t* __restrict__ far2, SCounters* ctr) {
    for (uint32_t base = blockIdx.x * blockDim.x; base < nfar; base += gridDim.x * blockDim.x) {
        uint32_t i = base + threadIdx.x;
        bool to_cur = false, keep = false;
        uint32_t v = 0;
        if (i < nfar) {
            v = far[i];
            uint64_t d = dist[v];
            if (d >= old_hi) {
                if (d < new_hi) to_cur = true;
                else keep = atomicExch(&fstamp[v], new_epoch) != new_epoch;
            }
        }
        uint32_t s1 = warp_append(&ctr->nnext, to_cur);
        if (to_cur) cur[s1] = v;
        uint32_t s2 = warp_append(&ctr->nfar2, keep);
        if (keep) far2[s2] = v;
    }
}

__global__ void k_ds_init(uint32_t* __restrict__ dist, uint32_t* __restrict__ a, uint32_t* __restrict__ b,
                          uint32_t* __restrict__ c, uint32_t n, uint32_t source) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        dist[v] = v == source ? 0u : 0xFFFFFFFFu;
        a[v] = 0;
        b[v] = 0;
        c[v] = 0;
    }
}

__global__ void k_ds_ecc(const uint32_t* __restrict__ dist, uint32_t n, uint32_t* __restrict__ out) {
    uint32_t m = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (dist[v] != 0xFFFFFFFFu) m = max(m, dist[v]);
    m = block_reduce(m, [](uint32_t a, uint32_t b) { return a > b ? a : b; }, 0u);
    if (threadIdx.x == 0) atomicMax(out, m);
}

}  // namespace

cldiam_status sssp_delta(cldiam_graph* g, uint32_t source, uint32_t delta, uint32_t* dist_out, uint64_t* ecc,
                         uint64_t* rounds_out) {
    if (!g || !ecc) return fail(CLDIAM_ERR_INVALID_ARG, "NULL graph or ecc");
    if (source >= g->n) return fail(CLDIAM_ERR_INVALID_ARG, "source >= n");
    const uint32_t n = g->n;
    const cudaStream_t s = g->stream;
    if (delta == 0) {
        uint32_t d0 = 1;
        CLD_TRY(cld::delta0(g, CLDIAM_DELTA0_AVG, 0, &d0));
        delta = d0;
    }
    DBuf<uint32_t> dist, rstamp, sstamp, fstamp, cur, next, settled, far, far2, ecc_d;
    DBuf<SCounters> ctr;
    CLD_TRY(dist.alloc(n, s));
    CLD_TRY(rstamp.alloc(n, s));
    CLD_TRY(sstamp.alloc(n, s));
    CLD_TRY(fstamp.alloc(n, s));
    CLD_TRY(cur.alloc(n, s));
    CLD_TRY(next.alloc(n, s));
    CLD_TRY(settled.alloc(n, s));
    CLD_TRY(far.alloc(n, s));
    CLD_TRY(far2.alloc(n, s));
    CLD_TRY(ecc_d.alloc(1, s));
    CLD_TRY(ctr.alloc(1, s));
    SCounters* hc = reinterpret_cast<SCounters*>(static_cast<char*>(g->host.h) + 192);
    static_assert(sizeof(SCounters) <= 64, "counter block must fit the pinned area");
    const unsigned gb = grid_for(n, 256);
    CLD_K(K_SSSP, s, k_ds_init<<<gb, 256, 0, s>>>(dist.get(), rstamp.get(), sstamp.get(), fstamp.get(), n, source));
    CLD_LAUNCH_CHECK();
    CLD_CUDA(cudaMemcpyAsync(cur.get(), &source, 4, cudaMemcpyHostToDevice, s));
    CLD_CUDA(cudaMemsetAsync(ctr.get(), 0, sizeof(SCounters), s));

    auto sync = [&]() -> cldiam_status {
        CLD_CUDA(cudaMemcpyAsync(hc, ctr.get(), sizeof(SCounters), cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        if (hc->overflow) return fail(CLDIAM_ERR_OVERFLOW, "a distance reached 2^32 - 1");
        return CLDIAM_OK;
    };
    const unsigned relax_grid = (unsigned)num_sms() * 8;
    uint32_t ncur = 1, round_id = 0, epoch = 1, nfar = 0;
    uint64_t lo = 0, hi = delta, rounds = 0;
    uint32_t* pcur = cur.get();
    uint32_t* pnext = next.get();
    uint32_t* pfar = far.get();
    uint32_t* pfar2 = far2.get();
    for (;;) {
        // light rounds of the current bucket
        CLD_CUDA(cudaMemsetAsync(&ctr.get()->nsettled, 0, 4, s));
        while (ncur > 0) {
            ++round_id;
            CLD_CUDA(cudaMemsetAsync(&ctr.get()->nnext, 0, 4, s));
            CLD_CUDA(cudaMemcpyAsync(&ctr.get()->nfar, &nfar, 4, cudaMemcpyHostToDevice, s));
            unsigned rg = (unsigned)std::min<uint64_t>((ncur + 7) / 8, relax_grid);
            CLD_K(K_SSSP, s, k_ds_relax<<<rg, 256, 0, s>>>(pcur, ncur, false, g->off, g->adj, dist.get(), delta, hi, rstamp.get(),
                                          round_id, sstamp.get(), fstamp.get(), epoch, pnext, settled.get(), pfar,
                                          ctr.get()));
            CLD_LAUNCH_CHECK();
            CLD_TRY(sync());
            ++rounds;
            ncur = hc->nnext;
            nfar = hc->nfar;
            std::swap(pcur, pnext);
        }
        // heavy phase of the bucket
        uint32_t ns = hc->nsettled;
        if (ns > 0) {
            CLD_CUDA(cudaMemcpyAsync(&ctr.get()->nfar, &nfar, 4, cudaMemcpyHostToDevice, s));
            unsigned rg = (unsigned)std::min<uint64_t>((ns + 7) / 8, relax_grid);
            CLD_K(K_SSSP, s, k_ds_relax<<<rg, 256, 0, s>>>(settled.get(), ns, true, g->off, g->adj, dist.get(), delta, hi, rstamp.get(),
                                          round_id, sstamp.get(), fstamp.get(), epoch, pnext, settled.get(), pfar,
                                          ctr.get()));
            CLD_LAUNCH_CHECK();
            CLD_TRY(sync());
            ++rounds;
            nfar = hc->nfar;
        }
        if (nfar == 0) break;
        // next bucket
        CLD_CUDA(cudaMemsetAsync(&ctr.get()->minbucket, 0xFF, 4, s));
        CLD_K(K_SSSP, s, k_ds_minbucket<<<grid_for(nfar, 256), 256, 0, s>>>(pfar, nfar, dist.get(), hi, delta, ctr.get()));
        CLD_LAUNCH_CHECK();
        CLD_TRY(sync());
        if (hc->minbucket == 0xFFFFFFFFu) break;
        const uint64_t old_hi = hi;
        lo = (uint64_t)hc->minbucket * delta;
        hi = lo + delta;
        ++epoch;
        CLD_CUDA(cudaMemsetAsync(&ctr.get()->nnext, 0, 4, s));
        CLD_CUDA(cudaMemsetAsync(&ctr.get()->nfar2, 0, 4, s));
        CLD_K(K_SSSP, s, k_ds_split<<<grid_for(nfar, 256), 256, 0, s>>>(pfar, nfar, dist.get(), old_hi, hi, fstamp.get(), epoch, pcur,
                                                      pfar2, ctr.get()));
        CLD_LAUNCH_CHECK();
        CLD_TRY(sync());
        ncur = hc->nnext;
        nfar = hc->nfar2;
        std::swap(pfar, pfar2);
    }
    CLD_CUDA(cudaMemsetAsync(ecc_d.get(), 0, 4, s));
    CLD_K(K_SSSP, s, k_ds_ecc<<<gb, 256, 0, s>>>(dist.get(), n, ecc_d.get()));
    CLD_LAUNCH_CHECK();
    uint32_t* he = reinterpret_cast<uint32_t*>(static_cast<char*>(g->host.h) + 240);
    CLD_CUDA(cudaMemcpyAsync(he, ecc_d.get(), 4, cudaMemcpyDeviceToHost, s));
    if (dist_out) CLD_CUDA(cudaMemcpyAsync(dist_out, dist.get(), (size_t)n * 4, cudaMemcpyDefault, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    *ecc = *he;
    if (rounds_out) *rounds_out = rounds;
    return CLDIAM_OK;
}

}  // namespace cld
