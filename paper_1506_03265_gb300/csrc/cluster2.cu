// CLUSTER2(G, tau) of Algorithm 2 (Section 4) on the GPU.
//
// Algorithm 2 contracts the clusters after every iteration and rescales an
// edge leaving a cluster to d_u + w - 2 R_CL (Contract2).  Rescaling by 2 R_CL
// per contraction is the same as giving every node a global offset instead:
// a center drawn in iteration i starts at g = (i - 1) 2 R_CL, a node reached
// from u over an edge of weight w gets g_u + w, and iteration i keeps exactly
// the nodes with g <= i 2 R_CL (distance <= 2 R_CL in the contracted graph
// G_i).  So the device keeps the original CSR and one offset per node: no
// edge list is rebuilt.  PartialGrowth2 runs growth to its fixed point
// (unique: the (distance, center id) minimum over the allowed paths), here by
// frontier rounds of asynchronous relaxations, which reach the same fixed
// point as the paper's synchronous steps.  D_v = g_v - g_{c_v} is the length
// of the path the growth followed.
#include <cmath>

#include "internal.cuh"
#include "prof.cuh"

namespace cld {

namespace {

constexpr uint32_t kC2Stream = 1;  // third Philox counter word of CLUSTER2's center draws

struct C2Counters {
    unsigned long long drawn;     // centers drawn
    unsigned long long updates;   // successful state decreases
    unsigned long long scanned;   // adjacency entries read
    unsigned long long joined;    // nodes that joined a cluster by growth
    uint32_t nfront;              // entries of the frontier being built
    uint32_t uncovered;           // nodes left without a center at the end
    uint32_t nhub;                // high-degree frontier nodes listed this round
    uint32_t pad;
};

// iteration i: an uncovered v is drawn iff Philox(seed; (v, i, 1, 0)) word 0 < thr; it starts at g = base
__global__ void k_c2_select(uint32_t n, uint32_t* __restrict__ center, uint32_t* __restrict__ g, uint64_t seed,
                            uint32_t it, uint64_t thr, uint32_t base, C2Counters* ctr) {
    unsigned long long cnt = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (center[v] != kNone) continue;
        const U4 r = philox4x32_10(seed, v, it, kC2Stream, 0u);
        if ((uint64_t)r.x < thr) {
            center[v] = v;
            g[v] = base;
            ++cnt;
        }
    }
    cnt = warp_sum(cnt);
    if (lane_id() == 0 && cnt) atomicAdd(&ctr->drawn, cnt);
}

// first frontier of an iteration: every covered node whose cluster may still reach an uncovered
// neighbour (done[v]: a scan of v found no uncovered neighbour over an edge of weight <= 2 R_CL, which
// stays true since coverage only grows)
__global__ void k_c2_front_init(uint32_t n, const uint32_t* __restrict__ center, const uint8_t* __restrict__ done,
                                uint32_t* __restrict__ front, C2Counters* ctr) {
    for (uint32_t b = blockIdx.x * blockDim.x; b < n; b += gridDim.x * blockDim.x) {
        const uint32_t v = b + threadIdx.x;
        const bool p = v < n && center[v] != kNone && !done[v];
        const uint32_t slot = warp_append(&ctr->nfront, p);
        if (p) front[slot] = v;
    }
}

constexpr uint32_t kC2Hub = 256;  // frontier nodes above this degree are relaxed by a whole CTA

// relaxation of adjacency entries [b0, b1) of u by the calling threads (stride `step` from `first`);
// returns whether some entry leads to an uncovered node over an edge of weight <= delta
__device__ __forceinline__ bool c2_relax_range(uint32_t u, uint64_t b0, uint64_t b1, uint64_t first, uint32_t step,
                                               const uint2* __restrict__ adj, const uint32_t* __restrict__ center,
                                               const uint32_t* __restrict__ g, unsigned long long* __restrict__ key,
                                               uint32_t base, uint32_t delta, uint32_t* __restrict__ stamp,
                                               uint32_t round, uint32_t* __restrict__ next, C2Counters* ctr,
                                               unsigned long long& upd) {
    // u's value: g_u when covered, else base + (its current distance); a candidate is kept when
    // g_u + w <= base + delta, as the key (g_u + w - base, c_u)
    uint64_t gu;
    uint32_t cu;
    const uint32_t cc = center[u];
    if (cc != kNone) {
        gu = g[u];
        cu = cc;
    } else {
        const unsigned long long k = __ldcg(&key[u]);
        gu = (uint64_t)base + (k >> 32);
        cu = (uint32_t)k;
    }
    bool open = false;
    for (uint64_t j = b0 + first; j < b1; j += step) {
        const uint2 e = adj[j];
        if (e.y > delta || center[e.x] != kNone) continue;
        open = true;
        const uint64_t cg = gu + e.y;
        if (cg > (uint64_t)base + delta) continue;
        const unsigned long long ck = ((unsigned long long)(cg - base) << 32) | cu;
        if (ck < atomicMin(&key[e.x], ck)) {
            ++upd;
            if (atomicExch(&stamp[e.x], round) != round) next[atomicAdd(&ctr->nfront, 1u)] = e.x;
        }
    }
    return open;
}

// One round, nodes of degree <= kC2Hub: a group of GW lanes per frontier node (GW = 32, or 4 on graphs of
// low average degree); improved nodes enter the next frontier once per round (stamp); a node with no
// uncovered neighbour over a usable edge is marked done.  Larger nodes are listed in hubs[] for
// k_c2_relax_hubs.
template <int GW>
__global__ void __launch_bounds__(256) k_c2_relax(const uint32_t* __restrict__ front, uint32_t nf,
                                                  const uint64_t* __restrict__ off, const uint2* __restrict__ adj,
                                                  const uint32_t* __restrict__ center, const uint32_t* __restrict__ g,
                                                  unsigned long long* __restrict__ key, uint32_t base, uint32_t delta,
                                                  uint32_t* __restrict__ stamp, uint32_t round,
                                                  uint32_t* __restrict__ next, uint8_t* __restrict__ done,
                                                  uint32_t* __restrict__ hubs, C2Counters* ctr) {
    const uint32_t groups = (gridDim.x * blockDim.x) / GW;
    const unsigned l = lane_id(), gl = l % GW;
    unsigned long long upd = 0, scanned = 0;
    // warp-uniform trip count (the group vote below needs every lane)
    const uint32_t first = (blockIdx.x * blockDim.x + threadIdx.x) / GW;
    const uint32_t wfirst = (blockIdx.x * blockDim.x + (threadIdx.x & ~31u)) / GW;
    for (uint32_t f0 = wfirst; f0 < nf; f0 += groups) {
        const uint32_t f = f0 + (first - wfirst);
        bool open = false, mine = false;
        if (f < nf) {
            const uint32_t u = front[f];
            const uint64_t b0 = off[u], b1 = off[u + 1];
            if (b1 - b0 > kC2Hub) {
                if (gl == 0) hubs[atomicAdd(&ctr->nhub, 1u)] = u;
            } else {
                mine = true;
                if (gl == 0) scanned += b1 - b0;
                open = c2_relax_range(u, b0, b1, gl, GW, adj, center, g, key, base, delta, stamp, round, next, ctr,
                                      upd);
            }
        }
        const unsigned vote = __ballot_sync(0xffffffffu, open);
        const unsigned gmask = (GW == 32) ? 0xffffffffu : (((1u << GW) - 1u) << (l - gl));
        if (mine && gl == 0 && !(vote & gmask)) done[front[f]] = 1;
    }
    upd = warp_sum(upd);
    scanned = warp_sum(scanned);
    if (l == 0 && (upd || scanned)) {
        atomicAdd(&ctr->updates, upd);
        atomicAdd(&ctr->scanned, scanned);
    }
}

// the same round for the listed high-degree nodes: a CTA per node (never marked done)
__global__ void __launch_bounds__(256) k_c2_relax_hubs(const uint32_t* __restrict__ hubs,
                                                       const uint64_t* __restrict__ off, const uint2* __restrict__ adj,
                                                       const uint32_t* __restrict__ center,
                                                       const uint32_t* __restrict__ g,
                                                       unsigned long long* __restrict__ key, uint32_t base,
                                                       uint32_t delta, uint32_t* __restrict__ stamp, uint32_t round,
                                                       uint32_t* __restrict__ next, C2Counters* ctr) {
    const uint32_t nh = __ldcg(&ctr->nhub);
    unsigned long long upd = 0, scanned = 0;
    for (uint32_t h = blockIdx.x; h < nh; h += gridDim.x) {
        const uint32_t u = hubs[h];
        const uint64_t b0 = off[u], b1 = off[u + 1];
        if (threadIdx.x == 0) scanned += b1 - b0;
        c2_relax_range(u, b0, b1, threadIdx.x, blockDim.x, adj, center, g, key, base, delta, stamp, round, next, ctr,
                       upd);
    }
    upd = warp_sum(upd);
    scanned = warp_sum(scanned);
    if (lane_id() == 0 && (upd || scanned)) {
        atomicAdd(&ctr->updates, upd);
        atomicAdd(&ctr->scanned, scanned);
    }
}

// reached nodes join their clusters at g = base + distance; keys reset for the next iteration
__global__ void k_c2_finalize(uint32_t n, uint32_t* __restrict__ center, uint32_t* __restrict__ g,
                              unsigned long long* __restrict__ key, uint32_t base, C2Counters* ctr) {
    unsigned long long cnt = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const unsigned long long k = key[v];
        if (k == kInfKey) continue;
        center[v] = (uint32_t)k;
        g[v] = base + (uint32_t)(k >> 32);
        key[v] = kInfKey;
        ++cnt;
    }
    cnt = warp_sum(cnt);
    if (lane_id() == 0 && cnt) atomicAdd(&ctr->joined, cnt);
}

// D_v = g_v - g_{c_v}; counts nodes left uncovered (none after the last iteration)
__global__ void k_c2_distances(uint32_t n, const uint32_t* __restrict__ center, const uint32_t* __restrict__ g,
                               uint32_t* __restrict__ D, C2Counters* ctr) {
    uint32_t bad = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint32_t c = center[v];
        if (c == kNone) {
            ++bad;
            D[v] = 0;
        } else {
            D[v] = g[v] - g[c];
        }
    }
    bad = warp_sum(bad);
    if (lane_id() == 0 && bad) atomicAdd(&ctr->uncovered, bad);
}

__global__ void k_c2_fill(uint32_t n, uint32_t* __restrict__ center, uint32_t* __restrict__ g,
                          unsigned long long* __restrict__ key, uint32_t* __restrict__ stamp,
                          uint8_t* __restrict__ done) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        center[v] = kNone;
        g[v] = 0;
        key[v] = kInfKey;
        stamp[v] = 0;
        done[v] = 0;
    }
}

struct Owner {
    cldiam_clustering* c;
    explicit Owner(cldiam_clustering* x) : c(x) {}
    ~Owner() {
        if (c) free_clustering(c);
    }
};

}  // namespace

cldiam_status cluster2(cldiam_graph* g, double tau, uint64_t seed, const cldiam_opts* o, cldiam_clustering** out) {
    if (!g || !out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL graph or out");
    *out = nullptr;
    // R_CL: the radius of CLUSTER(G, tau) under the same options
    cldiam_clustering* first = nullptr;
    CLD_TRY(cluster(g, tau, seed, o, &first));
    Owner own_first(first);
    const cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    C2Counters* hc = static_cast<C2Counters*>(g->host.h);
    static_assert(sizeof(C2Counters) <= 128, "counter block must fit the pinned area");
    DBuf<C2Counters> ctr;
    CLD_TRY(ctr.alloc(1, s));
    uint32_t R = 0;
    {
        DBuf<uint32_t> rmax;
        CLD_TRY(rmax.alloc(1, s));
        CLD_TRY(reduce_max_u32(first->D, n, rmax.get(), s));
        CLD_CUDA(cudaMemcpyAsync(&hc->nfront, rmax.get(), 4, cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        R = hc->nfront;
    }
    uint32_t L = 1;
    while ((1ull << L) < (uint64_t)n) ++L;
    const uint64_t delta64 = 2ull * R;
    if (delta64 * L >= 0xFFFFFFFFull)
        return fail(CLDIAM_ERR_UNSUPPORTED, "CLUSTER2 offsets (log2 n x 2 R_CL) need more than 32 bits");
    const uint32_t delta = (uint32_t)delta64;

    Owner owner(new cldiam_clustering());
    cldiam_clustering* cl = owner.c;
    cl->g = g;
    cl->stream = g->stream;
    cl->max_fw_k = first->max_fw_k;
    cl->quotient_mode = first->quotient_mode;
    DBuf<uint32_t> center, D, cid, gv, stamp, frA, frB;
    DBuf<unsigned long long> key;
    DBuf<uint8_t> done;
    DBuf<uint32_t> hubs;
    CLD_TRY(done.alloc(n, s));
    CLD_TRY(hubs.alloc(n, s));
    CLD_TRY(center.alloc(n, s));
    CLD_TRY(D.alloc(n, s));
    CLD_TRY(cid.alloc(n, s));
    CLD_TRY(gv.alloc(n, s));
    CLD_TRY(stamp.alloc(n, s));
    CLD_TRY(frA.alloc(n, s));
    CLD_TRY(frB.alloc(n, s));
    CLD_TRY(key.alloc(n, s));
    const unsigned gb = grid_for(n, 256);
    CLD_K(K_MISC, s, k_c2_fill<<<gb, 256, 0, s>>>(n, center.get(), gv.get(), key.get(), stamp.get(), done.get()));
    CLD_LAUNCH_CHECK();
    CLD_CUDA(cudaMemsetAsync(ctr.get(), 0, sizeof(C2Counters), s));
    auto read_nfront = [&](uint32_t* nf) -> cldiam_status {
        CLD_CUDA(cudaMemcpyAsync(&hc->nfront, &ctr.get()->nfront, 4, cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        *nf = hc->nfront;
        CLD_CUDA(cudaMemsetAsync(&ctr.get()->nfront, 0, 4, s));
        return CLDIAM_OK;
    };

    cldiam_result st{};
    uint32_t round = 0;
    const bool narrow = g->nnz < 8ull * n;  // average degree below 8: four lanes per frontier node
    const uint64_t max_rounds = (uint64_t)L * ((uint64_t)n + 2);  // each round settles some node for good
    for (uint32_t i = 1; i <= L; ++i) {
        const uint64_t thr = ((1ull << i) >= (uint64_t)n) ? (1ull << 32) : ((1ull << (32 + i)) / n);
        const uint32_t base = (uint32_t)((uint64_t)(i - 1) * delta);
        CLD_K(K_SELECT, s, k_c2_select<<<gb, 256, 0, s>>>(n, center.get(), gv.get(), seed, i, thr, base, ctr.get()));
        CLD_K(K_REBUILD, s, k_c2_front_init<<<gb, 256, 0, s>>>(n, center.get(), done.get(), frA.get(), ctr.get()));
        CLD_LAUNCH_CHECK();
        uint32_t nf = 0;
        CLD_TRY(read_nfront(&nf));
        uint32_t* fr = frA.get();
        uint32_t* fr2 = frB.get();
        // PartialGrowth2: rounds until no state decreases
        while (nf > 0) {
            if (++round > max_rounds) return fail(CLDIAM_ERR_DIVERGED, "CLUSTER2 growth did not settle");
            CLD_CUDA(cudaMemsetAsync(&ctr.get()->nhub, 0, 4, s));
            const uint64_t lanes = (uint64_t)nf * (narrow ? 4 : 32);
            const unsigned rg = (unsigned)std::min<uint64_t>((lanes + 255) / 256, (uint64_t)num_sms() * 8);
            if (narrow)
                CLD_K(K_RELAX, s, k_c2_relax<4><<<rg, 256, 0, s>>>(fr, nf, g->off, g->adj, center.get(), gv.get(),
                                                                   key.get(), base, delta, stamp.get(), round, fr2,
                                                                   done.get(), hubs.get(), ctr.get()));
            else
                CLD_K(K_RELAX, s, k_c2_relax<32><<<rg, 256, 0, s>>>(fr, nf, g->off, g->adj, center.get(), gv.get(),
                                                                    key.get(), base, delta, stamp.get(), round, fr2,
                                                                    done.get(), hubs.get(), ctr.get()));
            CLD_K(K_RELAX, s, k_c2_relax_hubs<<<num_sms() * 2, 256, 0, s>>>(hubs.get(), g->off, g->adj, center.get(),
                                                                          gv.get(), key.get(), base, delta,
                                                                          stamp.get(), round, fr2, ctr.get()));
            CLD_LAUNCH_CHECK();
            CLD_TRY(read_nfront(&nf));
            std::swap(fr, fr2);
        }
        CLD_K(K_FINALIZE, s, k_c2_finalize<<<gb, 256, 0, s>>>(n, center.get(), gv.get(), key.get(), base, ctr.get()));
        CLD_LAUNCH_CHECK();
        // every node covered: the remaining iterations can neither draw nor grow anything
        CLD_CUDA(cudaMemcpyAsync(hc, ctr.get(), sizeof(C2Counters), cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        if (hc->drawn + hc->joined >= n) break;
    }
    CLD_K(K_FINALIZE, s, k_c2_distances<<<gb, 256, 0, s>>>(n, center.get(), gv.get(), D.get(), ctr.get()));
    CLD_LAUNCH_CHECK();
    CLD_CUDA(cudaMemcpyAsync(hc, ctr.get(), sizeof(C2Counters), cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    if (hc->uncovered) return fail(CLDIAM_ERR_DIVERGED, "CLUSTER2 left nodes uncovered");
    st.centers_drawn = hc->drawn;
    st.node_updates = hc->updates;
    st.edges_scanned = hc->scanned;
    CLD_TRY(relabel_clusters(g, center.get(), cid.get(), &st.k));
    prof_flush();
    st.stages = L;
    st.steps = round;
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
