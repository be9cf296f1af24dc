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
//
// Work distribution: each round's node list becomes a frontier with the
// first position of every node's adjacency in one flattened range (one packed
// atomic per CTA hands out slots and positions) and a chunk table; the relax
// kernel gives each warp PW consecutive positions, so a hub's adjacency is
// spread over many warps instead of one (edge-balanced, as the growing step of
// CLUSTER).  Graphs with 2^32 or more adjacency entries keep one warp per node.
#include <algorithm>
#include <atomic>

#include "cluster_dev.cuh"
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
    unsigned long long front;  // listed frontier: (entries << 32) | adjacency positions
};

// A round's node list as a frontier: slot, first position and adjacency base of every node with
// entries, its distance when listed, and the chunk table; light rounds also record the bucket's
// settled nodes (once per bucket epoch).
__global__ void k_ds_list(const uint32_t* __restrict__ list, uint32_t nl, const uint32_t* __restrict__ dist,
                          const uint64_t* __restrict__ off, bool settle, uint32_t* __restrict__ sstamp, uint32_t epoch,
                          uint32_t* __restrict__ settled, uint32_t* __restrict__ fbase, uint32_t* __restrict__ fdist,
                          uint32_t* __restrict__ fpre, uint32_t* __restrict__ cfirst, SCounters* ctr) {
    __shared__ unsigned long long scratch[33];
    for (uint32_t base = blockIdx.x * blockDim.x; base < nl; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        bool take = false, settle_now = false;
        uint32_t u = 0, deg = 0, b0 = 0, du = 0;
        if (i < nl) {
            u = list[i];
            du = __ldcg(&dist[u]);
            const uint64_t o = off[u];
            b0 = (uint32_t)o;
            deg = (uint32_t)(off[u + 1] - o);
            take = deg > 0;
            settle_now = settle && atomicExch(&sstamp[u], epoch) != epoch;
        }
        const uint32_t s1 = warp_append(&ctr->nsettled, settle_now);
        if (settle_now) settled[s1] = u;
        uint32_t slot = 0, pre = 0;
        front_append(&ctr->front, take, deg, slot, pre, scratch);
        if (take) {
            fbase[slot] = b0 - pre;
            fdist[slot] = du;
            fpre[slot] = pre;
            chunk_table_put(cfirst, slot, pre, deg);
        }
    }
}

// One light round (heavy = false) or the heavy phase over a listed frontier: each warp takes PW
// consecutive positions of the flattened adjacency; a candidate that undercuts the target's distance
// lowers it with an atomic minimum, and an improved target goes to the next round (below hi) or to
// the far pile, each deduplicated by its stamp.
__global__ void __launch_bounds__(PT, 6) k_ds_push(const uint32_t* __restrict__ fbase,
                                                   const uint32_t* __restrict__ fdist,
                                                   const uint32_t* __restrict__ fpre,
                                                   const uint32_t* __restrict__ cfirst,
                                                   const uint2* __restrict__ adj, bool heavy,
                                                   uint32_t* __restrict__ dist, uint32_t delta, uint64_t hi,
                                                   uint32_t* __restrict__ rstamp, uint32_t round_id,
                                                   uint32_t* __restrict__ fstamp, uint32_t epoch,
                                                   uint32_t* __restrict__ next, uint32_t* __restrict__ far,
                                                   SCounters* ctr) {
    __shared__ uint32_t spre[PT / 32][PW + 1];
    __shared__ uint32_t sbase[PT / 32][PW + 2];
    __shared__ uint32_t sdist[PT / 32][PW + 2];
    __shared__ uint32_t snext[PT / 32][PNB];
    __shared__ uint32_t sfar[PT / 32][PNB];
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint64_t pol_stream = l2_evict_first_policy(), pol_keep = l2_evict_last_policy();
    const unsigned le_mask = 0xffffffffu >> (31u - lane);
    const unsigned long long fr = __ldcg(&ctr->front);
    const uint32_t nf = (uint32_t)(fr >> 32), E = (uint32_t)fr;
    WarpNext wn{snext[warp], 0}, wf{sfar[warp], 0};
    bool ovf = false;
    const uint32_t nq = (uint32_t)(((uint64_t)E + PW - 1) / PW);
    const uint32_t nwarps = gridDim.x * (PT / 32);
    for (uint32_t q = blockIdx.x * (PT / 32) + warp; q < nq; q += nwarps) {
        const uint32_t p0 = q * PW, e1 = min(E, p0 + PW);
        const uint32_t i0 = __ldcg(&cfirst[q]);
        const uint32_t il = q + 1 < nq ? __ldcg(&cfirst[q + 1]) : nf - 1;
        const uint32_t ne = min(il - i0 + 1, (uint32_t)PW + 1);
        for (uint32_t j = lane; j < ne; j += 32) {
            if (j) spre[warp][j - 1] = __ldcg(&fpre[i0 + j]);
            sbase[warp][j] = __ldcg(&fbase[i0 + j]);
            sdist[warp][j] = __ldcg(&fdist[i0 + j]);
        }
        __syncwarp();
        uint32_t own[PWG];
        {
            uint32_t B = 0;
#pragma unroll
            for (int u = 0; u < PWG; ++u) {
                const uint32_t word = group_starts(spre[warp] + B, ne - 1 - B, p0 + 32u * u, B, lane, le_mask, &own[u]);
                B += (uint32_t)__popc(word);
            }
        }
        uint2 ed[PWG];
#pragma unroll
        for (int u = 0; u < PWG; ++u) {
            const uint32_t p = p0 + 32u * u + lane;
            ed[u] = p < e1 ? ld_stream_u2(adj + (sbase[warp][own[u]] + p), pol_stream) : make_uint2(0u, 0u);
        }
        uint64_t nd[PWG];
        uint32_t cur[PWG];
#pragma unroll
        for (int u = 0; u < PWG; ++u) {
            const bool live = p0 + 32u * u + lane < e1 && ((ed[u].y <= delta) != heavy);
            nd[u] = live ? (uint64_t)sdist[warp][own[u]] + ed[u].y : ~0ull;
            cur[u] = nd[u] != ~0ull ? ld_keep_u32(&dist[ed[u].x], pol_keep) : 0u;  // filter through L1
        }
#pragma unroll
        for (int u = 0; u < PWG; ++u) {
            bool to_next = false, to_far = false;
            if (nd[u] != ~0ull && nd[u] >= 0xFFFFFFFFull) {
                ovf = true;
            } else if (nd[u] < cur[u]) {
                const uint32_t v = ed[u].x;
                if ((uint32_t)nd[u] < atomicMin(&dist[v], (uint32_t)nd[u])) {
                    if (nd[u] < hi) to_next = atomicExch(&rstamp[v], round_id) != round_id;
                    else to_far = atomicExch(&fstamp[v], epoch) != epoch;
                }
            }
            wn.put(to_next, ed[u].x, lane);
            wf.put(to_far, ed[u].x, lane);
        }
        if (wn.cnt >= (uint32_t)PW) wn.flush(next, &ctr->nnext, lane);
        if (wf.cnt >= (uint32_t)PW) wf.flush(far, &ctr->nfar, lane);
    }
    if (wn.cnt) wn.flush(next, &ctr->nnext, lane);
    if (wf.cnt) wf.flush(far, &ctr->nfar, lane);
    if (__any_sync(0xffffffffu, ovf) && lane == 0) atomicExch(&ctr->overflow, 1u);
}

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
                         uint64_t* rounds_out, uint64_t* scanned_out) {
    if (!g || !ecc) return fail(CLDIAM_ERR_INVALID_ARG, "NULL graph or ecc");
    if (source >= g->n) return fail(CLDIAM_ERR_INVALID_ARG, "source >= n");
    const uint32_t n = g->n;
    const cudaStream_t s = g->stream;
    if (delta == 0) {
        uint32_t d0 = 1;
        CLD_TRY(cld::delta0(g, CLDIAM_DELTA0_AVG, 0, &d0));
        const double scaled = (double)d0 * (double)tuning_for(g->nnz).sssp_delta_scale;
        delta = (uint32_t)std::min(std::max(scaled, 1.0), 2147483648.0);
    }
    // edge-balanced rounds index positions with 32 bits
    const bool chunked = g->nnz < 0xFFFFFFFFull;
    DBuf<uint32_t> dist, rstamp, sstamp, fstamp, cur, next, settled, far, far2, ecc_d;
    DBuf<uint32_t> fbase, fdist, fpre, cfirst;
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
    if (chunked) {
        CLD_TRY(fbase.alloc(n, s));
        CLD_TRY(fdist.alloc(n, s));
        CLD_TRY(fpre.alloc(n, s));
        CLD_TRY(cfirst.alloc(g->nnz / PW + 2, s));
    }
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
    static std::atomic<int> push_per_sm[64];  // concurrent first calls store the same value
    int dev = 0;
    CLD_CUDA(cudaGetDevice(&dev));
    const int di = (dev >= 0 && dev < 64) ? dev : 0;
    if (chunked && push_per_sm[di].load() == 0) {
        int a = 0;
        CLD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_ds_push, PT, 0));
        push_per_sm[di] = std::max(1, a);
    }
    const unsigned push_grid = (unsigned)num_sms() * (unsigned)std::max(1, push_per_sm[di].load());
    const unsigned relax_grid = (unsigned)num_sms() * 8;
    uint32_t ncur = 1, round_id = 0, epoch = 1, nfar = 0;
    uint64_t lo = 0, hi = delta, rounds = 0, scanned = 0;
    uint32_t* pcur = cur.get();
    uint32_t* pnext = next.get();
    uint32_t* pfar = far.get();
    uint32_t* pfar2 = far2.get();
    // one light round or the heavy phase over `list`
    auto relax = [&](const uint32_t* list, uint32_t nl, bool heavy) -> cldiam_status {
        if (chunked) {
            CLD_CUDA(cudaMemsetAsync(&ctr.get()->front, 0, 8, s));
            CLD_K(K_SSSP, s, k_ds_list<<<grid_for(nl, 256), 256, 0, s>>>(list, nl, dist.get(), g->off, !heavy,
                                                                         sstamp.get(), epoch, settled.get(),
                                                                         fbase.get(), fdist.get(), fpre.get(),
                                                                         cfirst.get(), ctr.get()));
            CLD_LAUNCH_CHECK();
            CLD_K(K_SSSP, s, k_ds_push<<<push_grid, PT, 0, s>>>(fbase.get(), fdist.get(), fpre.get(), cfirst.get(),
                                                                g->adj, heavy, dist.get(), delta, hi, rstamp.get(),
                                                                round_id, fstamp.get(), epoch, pnext, pfar,
                                                                ctr.get()));
        } else {
            const unsigned rg = (unsigned)std::min<uint64_t>((nl + 7) / 8, relax_grid);
            CLD_K(K_SSSP, s, k_ds_relax<<<rg, 256, 0, s>>>(list, nl, heavy, g->off, g->adj, dist.get(), delta, hi,
                                                           rstamp.get(), round_id, sstamp.get(), fstamp.get(), epoch,
                                                           pnext, settled.get(), pfar, ctr.get()));
        }
        CLD_LAUNCH_CHECK();
        return CLDIAM_OK;
    };
    for (;;) {
        // light rounds of the current bucket
        CLD_CUDA(cudaMemsetAsync(&ctr.get()->nsettled, 0, 4, s));
        while (ncur > 0) {
            ++round_id;
            CLD_CUDA(cudaMemsetAsync(&ctr.get()->nnext, 0, 4, s));
            CLD_CUDA(cudaMemcpyAsync(&ctr.get()->nfar, &nfar, 4, cudaMemcpyHostToDevice, s));
            CLD_TRY(relax(pcur, ncur, false));
            CLD_TRY(sync());
            ++rounds;
            ncur = hc->nnext;
            nfar = hc->nfar;
            scanned += (uint32_t)hc->front;
            // list: 16 B per node (+ its chunk-table share); relax: 8 B (col, w) + 4 B target distance per
            // position (+ 8 B per improved target: distance, stamp, list slot)
            prof_add_bytes(K_SSSP, 24.0 * (double)(uint32_t)(hc->front >> 32) + 12.0 * (double)(uint32_t)hc->front +
                                       8.0 * ncur);
            std::swap(pcur, pnext);
        }
        // heavy phase of the bucket
        uint32_t ns = hc->nsettled;
        if (ns > 0) {
            CLD_CUDA(cudaMemcpyAsync(&ctr.get()->nfar, &nfar, 4, cudaMemcpyHostToDevice, s));
            CLD_TRY(relax(settled.get(), ns, true));
            CLD_TRY(sync());
            ++rounds;
            nfar = hc->nfar;
            scanned += (uint32_t)hc->front;
            prof_add_bytes(K_SSSP, 24.0 * (double)(uint32_t)(hc->front >> 32) + 12.0 * (double)(uint32_t)hc->front);
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
    if (scanned_out) *scanned_out = scanned;
    return CLDIAM_OK;
}

}  // namespace cld
