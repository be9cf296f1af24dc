// CSR construction on the device (Section 2 graph model): drop self-loops,
// merge parallel edges to their minimum weight, symmetrise, sort rows by
// column, optionally keep the largest connected component.
//
// Pipeline: when 2 * bits(n - 1) + bits(max w) <= 64 every undirected edge is
// one packed word (min << b | max) << wb | w, sorted on its (min, max) bits;
// run heads give the distinct edges and the minimum over a run the lightest
// parallel edge.  The distinct edges sorted again on max alone (stable, so
// by (max, min)) give each row's entries below the diagonal; row x of the
// CSR is those, then its entries above the diagonal from the first order.
// Otherwise every edge becomes two directed (row * n + col, weight) pairs,
// sorted and de-duplicated the same way.  Components come from min-label
// hooking with pointer jumping: every tree points to a smaller id of its
// component, so roots are component minima and the labelling is
// deterministic.
#include <algorithm>
#include <atomic>
#include <vector>

#include "internal.cuh"
#include "prof.cuh"

namespace cld {

namespace {

__global__ void k_emit_directed(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                                const uint32_t* __restrict__ w, uint64_t m, uint32_t n, uint64_t sentinel,
                                uint64_t* __restrict__ keys, uint32_t* __restrict__ vals, uint32_t* __restrict__ bad) {
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = src[e], v = dst[e], ww = w[e];
        bool ok = u < n && v < n && ww != 0;
        if (!ok) atomicExch(bad, 1u);
        uint64_t k0 = sentinel, k1 = sentinel;
        if (ok && u != v) {
            k0 = (uint64_t)u * n + v;
            k1 = (uint64_t)v * n + u;
        }
        keys[2 * e] = k0;
        keys[2 * e + 1] = k1;
        vals[2 * e] = ww;
        vals[2 * e + 1] = ww;
    }
}

// one item per edge, (min(u,v) << vb | max(u,v)) << wb | w, a self-loop as ~0 (dropped, sorts last); also
// the input check (ids < n, weights >= 1 -> *bad) and whether a weight needs more than wb bits (*wide: the
// caller falls back to (key, weight) pairs)
// The same pass counts the digits of every pass of the sort that follows (8-bit digits of the item's
// 2 vb (a, b) bits, the last one masked to the bits left) into per-warp shared histograms
// (warps x npass x 256 words of dynamic shared memory), flushed into hist (npass x 256) at the end: the
// sort then needs no read of its own to count them.
__global__ void k_emit_canon(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                             const uint32_t* __restrict__ w, uint64_t m, uint32_t n, int vb, int wb,
                             uint64_t* __restrict__ items, uint32_t* __restrict__ bad, uint32_t* __restrict__ wide,
                             uint32_t* __restrict__ hist) {
    extern __shared__ uint32_t eh[];
    const int npass = (2 * vb + 7) / 8;
    for (int i = threadIdx.x; i < (int)(blockDim.x >> 5) * npass * 256; i += blockDim.x) eh[i] = 0;
    __syncthreads();
    uint32_t* h = eh + (threadIdx.x >> 5) * npass * 256;
    bool b = false, wd = false;
    const uint64_t wlim = wb >= 32 ? ~0ull : (1ull << wb);
    // EU edges per thread and iteration, their loads issued before the counting (which would otherwise
    // hold back the next loads: fewer CTAs fit per SM with the histograms)
    constexpr int EU = 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; base < m; base += stride * EU) {
        uint32_t su[EU], sv[EU], sw[EU];
#pragma unroll
        for (int k = 0; k < EU; ++k) {
            const uint64_t e = base + k * stride;
            su[k] = e < m ? src[e] : 0u;
            sv[k] = e < m ? dst[e] : 0u;
            sw[k] = e < m ? w[e] : 1u;
        }
#pragma unroll
        for (int k = 0; k < EU; ++k) {
            const uint64_t e = base + k * stride;
            if (e >= m) break;
            const uint64_t u = su[k], v = sv[k], ww = sw[k];
            b |= u >= n || v >= n || ww == 0;
            wd |= ww >= wlim;
            const uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
            const uint64_t it = u != v ? (((lo << vb) | hi) << wb) | ww : ~0ull;
            items[e] = it;
            for (int p = 0; p < npass; ++p) {
                const int left = 2 * vb - 8 * p;
                const uint32_t dm = left >= 8 ? 0xFFu : ((1u << left) - 1u);
                atomicAdd(&h[p * 256 + ((uint32_t)(it >> (wb + 8 * p)) & dm)], 1u);
            }
        }
    }
    if (__any_sync(0xffffffffu, b) && lane_id() == 0) atomicExch(bad, 1u);
    if (__any_sync(0xffffffffu, wd) && lane_id() == 0) atomicExch(wide, 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < npass * 256; i += blockDim.x) {
        uint32_t c = 0;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) c += eh[ww * npass * 256 + i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// Distinct edges in two orders: U by (a, b) and T by (b, a) (a < b).  Row x of the symmetric CSR is its
// lower entries (the a of T's run b = x, ascending) followed by its upper entries (the b of U's run
// a = x, ascending).  Run boundaries give each row's two counts: U's are written by the de-duplication
// that produces U, T's here.
// (also the directed entry count 2 mu into *nnz)
__global__ void k_canon_runs(const uint64_t* __restrict__ T, uint32_t mu, int vb, int wb,
                             uint32_t* __restrict__ tstart, uint32_t* __restrict__ tend, uint32_t* __restrict__ nnz) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *nnz = 2 * mu;
    const uint32_t cmask = vb >= 32 ? 0xFFFFFFFFu : ((1u << vb) - 1u);
    constexpr uint32_t kNo = 0xFFFFFFFFu;  // no neighbour (ids are below n <= 2^32 - 1)
    constexpr int CU = 4;                  // 32-entry chunks per warp and iteration, loaded together
    const unsigned l = lane_id();
    const uint64_t wstride = (uint64_t)gridDim.x * blockDim.x * CU;
    // warp-uniform trip count; a warp takes CU * 32 consecutive entries, neighbours' row ids come by
    // shuffle (across chunks through lanes 31 and 0), the two ends of the span are loaded
    for (uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u)) * CU; i0 < mu; i0 += wstride) {
        uint32_t b[CU];
#pragma unroll
        for (int k = 0; k < CU; ++k) {
            const uint64_t i = i0 + 32 * k + l;
            b[k] = i < mu ? (uint32_t)(T[i] >> wb) & cmask : kNo;
        }
        uint32_t before = kNo, after = kNo;
        if (l == 0 && i0 > 0) before = (uint32_t)(T[i0 - 1] >> wb) & cmask;
        if (l == 31 && i0 + 32 * CU < mu) after = (uint32_t)(T[i0 + 32 * CU] >> wb) & cmask;
#pragma unroll
        for (int k = 0; k < CU; ++k) {
            const uint64_t i = i0 + 32 * k + l;
            uint32_t bp = __shfl_up_sync(0xffffffffu, b[k], 1), bn = __shfl_down_sync(0xffffffffu, b[k], 1);
            const uint32_t prev_last = __shfl_sync(0xffffffffu, k > 0 ? b[k > 0 ? k - 1 : 0] : before, k > 0 ? 31 : 0);
            const uint32_t next_first = __shfl_sync(0xffffffffu, k < CU - 1 ? b[k < CU - 1 ? k + 1 : k] : after,
                                                    k < CU - 1 ? 0 : 31);
            if (l == 0) bp = prev_last;
            if (l == 31) bn = next_first;
            if (i >= mu) continue;
            if (bp != b[k]) tstart[b[k]] = (uint32_t)i;
            if (bn != b[k]) tend[b[k]] = (uint32_t)i + 1;
        }
    }
}

// row degrees
__global__ void k_canon_deg(uint32_t n, const uint32_t* __restrict__ ustart, const uint32_t* __restrict__ uend,
                            const uint32_t* __restrict__ tstart, const uint32_t* __restrict__ tend,
                            uint64_t* __restrict__ deg) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        deg[x] = (uint64_t)(uend[x] - ustart[x]) + (tend[x] - tstart[x]);
}

// (a position outside its row's part means inconsistent runs: recorded in *err, the write skipped)
__global__ void k_canon_scatter(const uint64_t* __restrict__ U, const uint64_t* __restrict__ T, uint32_t mu, int vb,
                                int wb, const uint32_t* __restrict__ ustart, const uint32_t* __restrict__ tstart,
                                const uint32_t* __restrict__ tend, const uint64_t* __restrict__ off,
                                uint32_t* __restrict__ row, uint2* __restrict__ adj, uint32_t* __restrict__ err) {
    const int ash = 64 - vb;
    const uint32_t cmask = vb >= 32 ? 0xFFFFFFFFu : ((1u << vb) - 1u);
    const uint32_t wmask = wb >= 32 ? 0xFFFFFFFFu : ((1u << wb) - 1u);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < mu; i += gridDim.x * blockDim.x) {
        const uint64_t u = U[i], t = T[i];
        const uint32_t a = (uint32_t)(u >> ash), b = (uint32_t)(u >> wb) & cmask;
        const uint64_t pu = off[a] + (tend[a] - tstart[a]) + (i - ustart[a]);  // after row a's lower entries
        if (i >= ustart[a] && pu < off[a + 1]) {
            adj[pu] = make_uint2(b, (uint32_t)u & wmask);
            row[pu] = a;
        } else {
            atomicExch(err, 1u);
        }
        const uint32_t ta = (uint32_t)(t >> ash), tb = (uint32_t)(t >> wb) & cmask;
        const uint64_t pt = off[tb] + (i - tstart[tb]);
        if (i >= tstart[tb] && i < tend[tb]) {
            adj[pt] = make_uint2(ta, (uint32_t)t & wmask);
            row[pt] = tb;
        } else {
            atomicExch(err, 1u);
        }
    }
}

__global__ void k_iota(uint32_t* __restrict__ a, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
}

// Union of the trees of u and v: the larger root is hooked under the smaller
// one with a compare-and-swap, so every tree root stays the minimum id of its
// tree.  Each retry strictly lowers the larger of the two candidate roots,
// so the loop ends.
__device__ __forceinline__ void cc_link(uint32_t u, uint32_t v, uint32_t* parent) {
    uint32_t p1 = parent[u], p2 = parent[v];
    while (p1 != p2) {
        const uint32_t high = p1 > p2 ? p1 : p2, low = p1 > p2 ? p2 : p1;
        const uint32_t ph = parent[high];
        if (ph == low) break;
        if (ph == high && atomicCAS(&parent[high], high, low) == high) break;
        p1 = parent[parent[high]];
        p2 = parent[low];
    }
}

// A node's neighbours in CSR order, from the CSR ...
struct CsrAdj {
    const uint64_t* off;
    const uint2* adj;
    __device__ uint32_t deg(uint32_t v) const { return (uint32_t)(off[v + 1] - off[v]); }
    __device__ uint32_t nbr(uint32_t v, uint32_t r) const { return adj[off[v] + r].x; }
};
// ... or from the two orders of the distinct edges (a, b), a < b: first the lower neighbours (the a of
// v's run in T, sorted by (b, a)), then the upper ones (the b of v's run in U, sorted by (a, b))
struct ListAdj {
    const uint64_t* U;
    const uint64_t* T;
    const uint32_t *ustart, *uend, *tstart, *tend;
    int ash, wb;
    uint32_t cmask;
    __device__ uint32_t lo(uint32_t v) const { return tend[v] - tstart[v]; }
    __device__ uint32_t deg(uint32_t v) const { return lo(v) + (uend[v] - ustart[v]); }
    __device__ uint32_t nbr(uint32_t v, uint32_t r) const {
        const uint32_t l = lo(v);
        return r < l ? (uint32_t)(T[tstart[v] + r] >> ash) : (uint32_t)(U[ustart[v] + (r - l)] >> wb) & cmask;
    }
};

// first passes: link every node with its r-th neighbour (ids >= n, which a consistent graph never holds,
// are skipped rather than followed).  One launch per r with pointer jumping in between: linking several
// neighbours in one pass builds long parent chains on meshes, which every later link then walks.
template <class A>
__global__ void k_cc_link_nth(A g, uint32_t n, uint32_t r, uint32_t* __restrict__ parent) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (r >= g.deg(v)) continue;
        const uint32_t c = g.nbr(v, r);
        if (c < n) cc_link(v, c, parent);
    }
}

// final pass: nodes outside the dominant tree link all their remaining
// neighbours (an edge with both ends in the dominant tree adds nothing; an
// edge with one end outside is linked from that end)
template <class A>
__global__ void k_cc_link_rest(A g, uint32_t n, uint32_t skip, uint32_t giant, uint32_t* __restrict__ parent) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t r = parent[v];
        while (parent[r] != r) r = parent[r];
        if (r == giant) continue;
        const uint32_t d = g.deg(v);
        for (uint32_t j = skip; j < d; ++j) {
            const uint32_t c = g.nbr(v, j);
            if (c < n) cc_link(v, c, parent);
        }
    }
}

__global__ void k_cc_sample(const uint32_t* __restrict__ parent, uint32_t n, uint32_t count, uint32_t* __restrict__ out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        uint32_t v = (uint32_t)(((uint64_t)i * 2654435761ull) % n);
        uint32_t r = parent[v];
        while (parent[r] != r) r = parent[r];
        out[i] = r;
    }
}

// pointer jumping to the root (parents only ever decrease within a component)
__global__ void k_cc_compress(uint32_t* __restrict__ parent, uint32_t n) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t p = parent[v];
        uint32_t pp = parent[p];
        while (p != pp) {
            p = pp;
            pp = parent[p];
        }
        parent[v] = p;
    }
}

// size of the sampled dominant tree; when it holds more than half of the nodes it is the largest
// component and the per-root counts below are skipped
__global__ void k_cc_size_of(const uint32_t* __restrict__ parent, uint32_t n, uint32_t giant,
                             uint32_t* __restrict__ count) {
    uint32_t c = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) c += parent[v] == giant;
    c = block_reduce(c, [](uint32_t a, uint32_t b) { return a + b; }, 0u);
    if (threadIdx.x == 0 && c) atomicAdd(count, c);
}
__device__ __forceinline__ bool giant_is_largest(const uint32_t* count, uint32_t n) {
    return count && 2ull * *count > n;
}
__global__ void k_cc_giant_best(const uint32_t* __restrict__ count, uint32_t n, uint32_t giant,
                                unsigned long long* __restrict__ best) {
    if (giant_is_largest(count, n)) *best = ((unsigned long long)*count << 32) | (unsigned long long)(0xFFFFFFFFu - giant);
}

__global__ void k_cc_count(const uint32_t* __restrict__ parent, uint32_t n, uint32_t* __restrict__ size,
                           const uint32_t* __restrict__ gcount) {
    if (giant_is_largest(gcount, n)) return;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t v = base + threadIdx.x;
        const uint32_t r = v < n ? parent[v] : 0xFFFFFFFFu;
        // most nodes share one root: one atomic per distinct root per warp
        const unsigned peers = __match_any_sync(0xffffffffu, r);
        if (v < n && lane_id() == (unsigned)(__ffs(peers) - 1)) atomicAdd(&size[r], (uint32_t)__popc(peers));
    }
}

// best component: largest size, then smallest root id
__global__ void k_cc_best(const uint32_t* __restrict__ parent, const uint32_t* __restrict__ size, uint32_t n,
                          unsigned long long* __restrict__ best, const uint32_t* __restrict__ gcount) {
    if (giant_is_largest(gcount, n)) return;
    unsigned long long b = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (parent[v] == v) {
            unsigned long long key = ((unsigned long long)size[v] << 32) | (unsigned long long)(0xFFFFFFFFu - v);
            b = key > b ? key : b;
        }
    b = block_reduce(b, [](unsigned long long x, unsigned long long y) { return x > y ? x : y; }, 0ull);
    if (threadIdx.x == 0) atomicMax(best, b);
}

__global__ void k_cc_keep(const uint32_t* __restrict__ parent, uint32_t n, const unsigned long long* __restrict__ best,
                          uint32_t* __restrict__ keep) {
    uint32_t root = 0xFFFFFFFFu - (uint32_t)(*best & 0xFFFFFFFFull);
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        keep[v] = parent[v] == root ? 1u : 0u;
}

template <class A>
__global__ void k_lcc_degrees(const uint32_t* __restrict__ keep, const uint32_t* __restrict__ newid, A g, uint32_t n,
                              uint32_t* __restrict__ ndeg, uint32_t* __restrict__ orig) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (keep[v]) {
            ndeg[newid[v]] = g.deg(v);
            orig[newid[v]] = v;
        }
}

// new offsets (widened from the 32-bit scan of the kept degrees) and, for each kept node orig[i], its
// new id and the shift from its old adjacency positions to its new ones (positions are < 2^32, so
// the shift is taken modulo 2^32); map of a dropped node keeps its 0xFFFFFFFF pre-fill
__global__ void k_lcc_offsets(const uint32_t* __restrict__ excl, uint32_t n, const uint32_t* __restrict__ n_out_dev,
                              const uint32_t* __restrict__ total_dev, const uint32_t* __restrict__ orig,
                              const uint64_t* __restrict__ off, uint64_t* __restrict__ noff, uint2* __restrict__ map) {
    const uint32_t n_out = *n_out_dev, total = *total_dev;  // n_out <= n
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= n_out; i += gridDim.x * blockDim.x) {
        noff[i] = (i == n_out) ? (uint64_t)total : (uint64_t)excl[i];
        if (map && i < n_out) {
            const uint32_t u = orig[i];
            map[u] = make_uint2(i, excl[i] - (uint32_t)off[u]);
        }
    }
}

// copy of the kept rows with new ids (monotone, so rows stay sorted), and the
// weight statistics of the copy: sum over u < v and minimum.  Each thread
// handles LU entries a grid stride apart with all their loads issued first.
__global__ void __launch_bounds__(256) k_lcc_copy(const uint2* __restrict__ map, const uint32_t* __restrict__ newid,
                                                  const uint32_t* __restrict__ row, const uint2* __restrict__ adj,
                                                  uint64_t nnz, uint32_t* __restrict__ nrow, uint2* __restrict__ nadj,
                                                  unsigned long long* __restrict__ wsum, uint32_t* __restrict__ wmin) {
    constexpr int LU = 4;
    unsigned long long sum = 0;
    uint32_t mn = 0xFFFFFFFFu;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nnz; b += stride * LU) {
        uint32_t u[LU];
        uint2 e[LU], mp[LU];
        uint32_t nv[LU];
#pragma unroll
        for (int k = 0; k < LU; ++k) {
            const uint64_t i = b + (uint64_t)k * stride;
            u[k] = i < nnz ? row[i] : 0u;
            e[k] = i < nnz ? adj[i] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int k = 0; k < LU; ++k) {
            const uint64_t i = b + (uint64_t)k * stride;
            mp[k] = i < nnz ? map[u[k]] : make_uint2(0xFFFFFFFFu, 0u);
            nv[k] = i < nnz ? newid[e[k].x] : 0u;
        }
#pragma unroll
        for (int k = 0; k < LU; ++k) {
            if (mp[k].x == 0xFFFFFFFFu) continue;  // dropped row, or past the end
            const uint64_t i = b + (uint64_t)k * stride;
            const uint32_t pos = (uint32_t)i + mp[k].y;
            nadj[pos] = make_uint2(nv[k], e[k].y);
            nrow[pos] = mp[k].x;
            if (u[k] < e[k].x) sum += e[k].y;
            mn = e[k].y < mn ? e[k].y : mn;
        }
    }
    sum = block_reduce(sum, [](unsigned long long a, unsigned long long b) { return a + b; }, 0ull);
    if (threadIdx.x == 0 && sum) atomicAdd(wsum, sum);
    mn = block_reduce(mn, [](uint32_t a, uint32_t b) { return a < b ? a : b; }, 0xFFFFFFFFu);
    if (threadIdx.x == 0 && mn != 0xFFFFFFFFu) atomicMin(wmin, mn);
}

// New offsets of the LCC from the scan of its degrees, and per kept node u = orig[i] one word of four:
// (i, the position shift of u's upper entries from their index in U, the shift of its lower entries from
// their index in T, 0), positions and shifts taken modulo 2^32 (positions are < 2^32); dropped nodes keep
// the all-ones pre-fill
__global__ void k_lcc_offsets_lists(const uint32_t* __restrict__ excl, const uint32_t* __restrict__ n_out_dev,
                                    const uint32_t* __restrict__ total_dev, const uint32_t* __restrict__ orig, ListAdj g,
                                    uint64_t* __restrict__ noff, uint4* __restrict__ info) {
    const uint32_t n_out = *n_out_dev, total = *total_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= n_out; i += gridDim.x * blockDim.x) {
        noff[i] = (i == n_out) ? (uint64_t)total : (uint64_t)excl[i];
        if (i < n_out) {
            const uint32_t u = orig[i];
            info[u] = make_uint4(i, excl[i] + g.lo(u) - g.ustart[u], excl[i] - g.tstart[u], 0u);
        }
    }
}

// The LCC's CSR straight from the two orders of the distinct edges: an edge (a, b) of the kept component
// goes to row newid[a] after its lower entries (from U) and to row newid[b] (from T); new ids are
// monotone, so rows stay sorted.  Weight statistics as k_lcc_copy (each undirected edge once: from U).
// A position past the output (inconsistent input) is recorded in *err and the write skipped.  The row's
// own record (info, 16 B) is read in runs (U is sorted on a, T on b); the far end's new id comes from
// the 4-byte newid array (evict-last: it stays in L2 while the two edge lists stream through, evict-first).
__global__ void __launch_bounds__(256, 4) k_lcc_assemble(ListAdj g, uint32_t mu, const uint4* __restrict__ info,
                                                         const uint32_t* __restrict__ newid, uint64_t cap,
                                                         uint2* __restrict__ nadj, unsigned long long* __restrict__ wsum,
                                                         uint32_t* __restrict__ wmin, uint32_t* __restrict__ err) {
    const uint32_t wmask = g.wb >= 32 ? 0xFFFFFFFFu : ((1u << g.wb) - 1u);
    const uint64_t pol_stream = l2_evict_first_policy(), pol_keep = l2_evict_last_policy();
    unsigned long long sum = 0;
    uint32_t mn = 0xFFFFFFFFu;
    // AU entries per thread and iteration: the loads of each level (edge words, row records, far-end ids)
    // are issued for all of them before the next level, so the dependent gathers overlap
    constexpr int AU = 4;
    constexpr uint32_t kDrop = 0xFFFFFFFFu;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; base < mu; base += stride * AU) {
        uint64_t u[AU], t[AU];
#pragma unroll
        for (int k = 0; k < AU; ++k) {
            const uint64_t i = base + k * stride;
            u[k] = i < mu ? ld_stream_u64(g.U + i, pol_stream) : 0ull;
            t[k] = i < mu ? ld_stream_u64(g.T + i, pol_stream) : 0ull;
        }
        // position shifts of the kept rows' entries, and which rows are kept (bit k: the edge's row in U,
        // bit AU + k: its row in T)
        uint32_t iy[AU], jz[AU], kept = 0;
#pragma unroll
        for (int k = 0; k < AU; ++k) {
            iy[k] = jz[k] = 0;
            if (base + k * stride < mu) {
                const uint4 ia = info[(uint32_t)(u[k] >> g.ash)], ib = info[(uint32_t)(t[k] >> g.wb) & g.cmask];
                iy[k] = ia.y;
                jz[k] = ib.z;
                kept |= (ia.x != kDrop ? 1u : 0u) << k;
                kept |= (ib.x != kDrop ? 1u : 0u) << (AU + k);
            }
        }
        // far ends (a kept row's neighbours are kept: their new ids are valid)
        uint32_t nb[AU], na[AU];
#pragma unroll
        for (int k = 0; k < AU; ++k) {
            nb[k] = (kept >> k) & 1u ? ld_nc_keep_u32(newid + ((uint32_t)(u[k] >> g.wb) & g.cmask), pol_keep) : 0u;
            na[k] = (kept >> (AU + k)) & 1u ? ld_nc_keep_u32(newid + (uint32_t)(t[k] >> g.ash), pol_keep) : 0u;
        }
#pragma unroll
        for (int k = 0; k < AU; ++k) {
            const uint32_t i = (uint32_t)(base + k * stride);  // < mu when the row is kept
            if ((kept >> k) & 1u) {  // kept (then b is kept too)
                const uint32_t w = (uint32_t)u[k] & wmask;
                const uint32_t pos = iy[k] + i;
                if (pos < cap) {
                    nadj[pos] = make_uint2(nb[k], w);
                } else {
                    atomicExch(err, 1u);
                }
                sum += w;
                mn = w < mn ? w : mn;
            }
            if ((kept >> (AU + k)) & 1u) {
                const uint32_t pos = jz[k] + i;
                if (pos < cap) {
                    nadj[pos] = make_uint2(na[k], (uint32_t)t[k] & wmask);
                } else {
                    atomicExch(err, 1u);
                }
            }
        }
    }
    sum = block_reduce(sum, [](unsigned long long x, unsigned long long y) { return x + y; }, 0ull);
    if (threadIdx.x == 0 && sum) atomicAdd(wsum, sum);
    mn = block_reduce(mn, [](uint32_t x, uint32_t y) { return x < y ? x : y; }, 0xFFFFFFFFu);
    if (threadIdx.x == 0 && mn != 0xFFFFFFFFu) atomicMin(wmin, mn);
}

__global__ void k_graph_stats(const uint32_t* __restrict__ row, const uint2* __restrict__ adj, uint64_t nnz,
                              unsigned long long* __restrict__ wsum, uint32_t* __restrict__ wmin) {
    unsigned long long s = 0;
    uint32_t mn = 0xFFFFFFFFu;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (uint64_t)gridDim.x * blockDim.x) {
        uint2 e = adj[i];
        if (row[i] < e.x) s += e.y;
        mn = e.y < mn ? e.y : mn;
    }
    s = block_reduce(s, [](unsigned long long a, unsigned long long b) { return a + b; }, 0ull);
    if (threadIdx.x == 0 && s) atomicAdd(wsum, s);
    mn = block_reduce(mn, [](uint32_t a, uint32_t b) { return a < b ? a : b; }, 0xFFFFFFFFu);
    if (threadIdx.x == 0) atomicMin(wmin, mn);
}

// largest degree of rows 0..n-1 (n = *n_dev when given: a count still on the device, <= the bound n)
__global__ void k_degree_max(const uint64_t* __restrict__ off, uint32_t n, const uint32_t* __restrict__ n_dev,
                             uint32_t* __restrict__ out) {
    if (n_dev) n = min(n, *n_dev);
    uint32_t m = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        m = max(m, (uint32_t)(off[v + 1] - off[v]));
    m = block_reduce(m, [](uint32_t a, uint32_t b) { return a > b ? a : b; }, 0u);
    if (threadIdx.x == 0) atomicMax(out, m);
}

struct GraphOwner {
    cldiam_graph* g;
    explicit GraphOwner(cldiam_graph* x) : g(x) {}
    ~GraphOwner() {
        if (g) free_graph(g);
    }
    cldiam_graph* release() {
        cldiam_graph* x = g;
        g = nullptr;
        return x;
    }
};

}  // namespace

void free_graph(cldiam_graph* g) {
    if (!g) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g->device);
    if (!g->borrowed) {
        dfree(g->off, g->stream);
        dfree(g->adj, g->stream);
        dfree(g->row, g->stream);
        dfree(g->orig, g->stream);
    }
    cudaStreamSynchronize(g->stream);
    cudaSetDevice(cur);
    delete g;
}

cldiam_status build_csr(const uint32_t* src, const uint32_t* dst, const uint32_t* w, uint64_t m, uint32_t n,
                        uint32_t flags, cudaStream_t s, cldiam_graph** out) {
    if (!out) return fail(CLDIAM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n == 0) return fail(CLDIAM_ERR_INVALID_ARG, "n must be >= 1");
    if (m > 0 && (!src || !dst || !w)) return fail(CLDIAM_ERR_INVALID_ARG, "edge arrays are NULL");
    if (2 * m > 0xFFFFFFFFull) return fail(CLDIAM_ERR_UNSUPPORTED, "more than 2^31 - 1 edges");
    if (flags & ~CLDIAM_CSR_LCC) return fail(CLDIAM_ERR_INVALID_ARG, "unknown flags");

    GraphOwner owner(new cldiam_graph());
    cldiam_graph* g = owner.g;
    CLD_CUDA(cudaGetDevice(&g->device));
    g->stream = s;
    CLD_TRY(g->host.alloc(256));
    uint32_t* hbad = static_cast<uint32_t*>(g->host.h);

    // inputs on the device
    void *dsrc = nullptr, *ddst = nullptr, *dw = nullptr;
    bool osrc = false, odst = false, ow = false;
    struct InFree {
        void** p; bool* o; cudaStream_t s;
        ~InFree() { if (*o) dfree(*p, s); }
    };
    // host edge arrays are copied to the device by the copy engine (cudaMemcpyAsync on the call's stream),
    // not read in place by the emission kernel: the copy then occupies no SM, so another call's kernels can
    // run on the whole device while this call's edge list crosses the host link
    CLD_TRY(to_device(src, m * 4, s, &dsrc, &osrc));
    InFree f1{&dsrc, &osrc, s};
    CLD_TRY(to_device(dst, m * 4, s, &ddst, &odst));
    InFree f2{&ddst, &odst, s};
    CLD_TRY(to_device(w, m * 4, s, &dw, &ow));
    InFree f3{&dw, &ow, s};

    // items: packed words when the weight fits in the bits the two ids leave, else (key, weight) pairs
    const uint64_t cnt = 2 * m;
    // device words read back by the host: [0] bad input, [1] unique entries, [2] wide weight, [3] sampled
    // giant size, [4] LCC nodes, [5] LCC entries, [6] min weight, [7] max degree, [8] sort look-back error
    DBuf<uint32_t> scal;
    CLD_TRY(scal.alloc(9, s));
    CLD_CUDA(cudaMemsetAsync(scal.get(), 0, 9 * sizeof(uint32_t), s));
    const int vb = std::max(1, bits_for((uint64_t)n - 1));
    const int wb = 64 - 2 * vb;  // weight bits of a packed item

    DBuf<uint32_t> row, deg, degx;
    DBuf<uint64_t> off;
    DBuf<uint2> adj;
    // the whole graph's row / adj arrays are allocated only where they are built (the packed path with the
    // LCC goes from the edge lists straight to the LCC's CSR)
    const auto alloc_full = [&]() -> cldiam_status {
        CLD_TRY(row.alloc(cnt ? cnt : 1, s));
        CLD_TRY(adj.alloc(cnt ? cnt : 1, s));
        return CLDIAM_OK;
    };
    CLD_TRY(deg.alloc((size_t)n + 1, s));
    CLD_TRY(degx.alloc((size_t)n + 1, s));
    CLD_TRY(off.alloc((size_t)n + 1, s));
    const bool lcc = (flags & CLDIAM_CSR_LCC) != 0;
    bool packed = wb >= 1;
    // packed path: the distinct edges in two orders and their run bounds (the adjacency in list form)
    DBuf<uint64_t> items, items2, uniq;
    DBuf<uint32_t> hist1;  // digit counts of the first sort, accumulated by the emission
    DBuf<uint32_t> hist2;  // digit counts of the second sort, accumulated by the de-duplication
    DBuf<uint32_t> runs;
    ListAdj la{};
    uint32_t mu = 0;
    if (packed) {
        // one item per edge, sorted on (a, b) and de-duplicated (U); the same distinct edges sorted on b alone
        // (stable, so by (b, a): T) give every row's entries below the diagonal
        CLD_TRY(items.alloc(m ? m : 1, s));
        const int npass1 = (2 * vb + 7) / 8;
        CLD_TRY(hist1.alloc((size_t)npass1 * 256, s));
        CLD_CUDA(cudaMemsetAsync(hist1.get(), 0, (size_t)npass1 * 256 * 4, s));
        if (m > 0) {
            const size_t esm = (size_t)8 * npass1 * 256 * 4;  // 8 warps; <= 64 KB
            static std::atomic<bool> emit_attr[64];
            int dev = 0;
            CLD_CUDA(cudaGetDevice(&dev));
            if (dev < 0 || dev >= 64 || !emit_attr[dev]) {
                CLD_CUDA(cudaFuncSetAttribute(k_emit_canon, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
                if (dev >= 0 && dev < 64) emit_attr[dev] = true;
            }
            CLD_K(K_CSR, s, k_emit_canon<<<grid_for(m, 256, 4), 256, esm, s>>>(
                                (const uint32_t*)dsrc, (const uint32_t*)ddst, (const uint32_t*)dw, m, n, vb, wb, items.get(),
                                scal.get(), scal.get() + 2, hist1.get()));
            CLD_LAUNCH_CHECK();
        }
        CLD_CUDA(cudaMemcpyAsync(hbad, scal.get(), 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        if (hbad[0]) return fail(CLDIAM_ERR_INVALID_ARG, "edge with node id >= n or weight 0");
        packed = hbad[2] == 0;
        if (packed) {
            CLD_TRY(items2.alloc(m ? m : 1, s));
            CLD_TRY(uniq.alloc(m ? m : 1, s));
            bool alt = false;
            CLD_TRY(radix_sort_keys_u64(items.get(), items2.get(), m, wb, 2 * vb, &alt, s, scal.get() + 8, nullptr,
                                        hist1.get()));
            const int npass2 = (vb + 7) / 8;
            CLD_TRY(hist2.alloc((size_t)npass2 * 256, s));
            CLD_CUDA(cudaMemsetAsync(hist2.get(), 0, (size_t)npass2 * 256 * 4, s));
            // every row's run bounds in both orders; the de-duplication writes the first order's
            CLD_TRY(runs.alloc(4 * (size_t)n, s));
            CLD_CUDA(cudaMemsetAsync(runs.get(), 0, 4 * (size_t)n * 4, s));
            CLD_TRY(unique_items_u64(alt ? items2.get() : items.get(), m, vb, uniq.get(), scal.get() + 1, s, hist2.get(),
                                     runs.get(), runs.get() + n));
            CLD_CUDA(cudaMemcpyAsync(hbad + 1, scal.get() + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            CLD_CUDA(cudaStreamSynchronize(s));
            mu = hbad[1];  // distinct undirected edges
            bool alt2 = false;
            CLD_TRY(radix_sort_keys_u64(items.get(), items2.get(), mu, wb, vb, &alt2, s, scal.get() + 8, uniq.get(),
                                        hist2.get()));
            la.U = uniq.get();
            la.T = alt2 ? items2.get() : items.get();
            la.ustart = runs.get();
            la.uend = runs.get() + n;
            la.tstart = runs.get() + 2 * (size_t)n;
            la.tend = runs.get() + 3 * (size_t)n;
            la.ash = 64 - vb;
            la.wb = wb;
            la.cmask = vb >= 32 ? 0xFFFFFFFFu : ((1u << vb) - 1u);
            uint32_t* r0 = runs.get();
            if (mu > 0) {
                CLD_K(K_CSR, s, k_canon_runs<<<grid_for(mu, 256), 256, 0, s>>>(la.T, mu, vb, wb, r0 + 2 * (size_t)n,
                                                                              r0 + 3 * (size_t)n, scal.get() + 1));
                CLD_LAUNCH_CHECK();
            }
            if (!lcc) {
                // the whole graph's CSR: row x = its lower entries, then its upper entries
                CLD_TRY(alloc_full());
                DBuf<uint64_t> degs;
                CLD_TRY(degs.alloc(n, s));
                CLD_K(K_CSR, s, k_canon_deg<<<grid_for(n, 256), 256, 0, s>>>(n, la.ustart, la.uend, la.tstart, la.tend,
                                                                            degs.get()));
                CLD_LAUNCH_CHECK();
                CLD_TRY(scan_exclusive_u64(degs.get(), off.get(), n, off.get() + n, s));
                if (mu > 0) {
                    CLD_K(K_CSR, s, k_canon_scatter<<<grid_for(mu, 256), 256, 0, s>>>(la.U, la.T, mu, vb, wb, la.ustart,
                                                                                     la.tstart, la.tend, off.get(),
                                                                                     row.get(), adj.get(),
                                                                                     scal.get() + 8));
                    CLD_LAUNCH_CHECK();
                }
            }
        }
    }
    if (!packed) {
        // keys u*n + v (u != v) are at most n^2 - 2; n^2 - 1 marks a dropped self-loop
        CLD_TRY(alloc_full());
        CLD_CUDA(cudaMemsetAsync(adj.get(), 0xFF, (size_t)(cnt ? cnt : 1) * 8, s));  // run minima fold in
        const uint64_t sentinel = (uint64_t)n * (uint64_t)n - 1;
        DBuf<uint64_t> keys, keys2;
        DBuf<uint32_t> vals, vals2;
        CLD_TRY(keys.alloc(cnt ? cnt : 1, s));
        CLD_TRY(keys2.alloc(cnt ? cnt : 1, s));
        CLD_TRY(vals.alloc(cnt ? cnt : 1, s));
        CLD_TRY(vals2.alloc(cnt ? cnt : 1, s));
        if (m > 0) {
            CLD_K(K_CSR, s, k_emit_directed<<<grid_for(m, 256), 256, 0, s>>>((const uint32_t*)dsrc,
                                                                            (const uint32_t*)ddst, (const uint32_t*)dw,
                                                                            m, n, sentinel, keys.get(), vals.get(),
                                                                            scal.get()));
            CLD_LAUNCH_CHECK();
        }
        CLD_CUDA(cudaMemcpyAsync(hbad, scal.get(), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        if (hbad[0]) return fail(CLDIAM_ERR_INVALID_ARG, "edge with node id >= n or weight 0");
        bool alt = false;
        CLD_TRY(radix_sort_pairs_u64(keys.get(), vals.get(), keys2.get(), vals2.get(), cnt, bits_for(sentinel), &alt,
                                     s));
        CLD_TRY(unique_min_sorted_u64(alt ? keys2.get() : keys.get(), alt ? vals2.get() : vals.get(), cnt, sentinel, n,
                                      row.get(), &adj.get()->x, &adj.get()->y, 2, off.get(), n, scal.get() + 1, s));
    }
    // (the entry count stays on the device until the host needs it, read together with the next result)
    uint32_t nnz = 0;
    DBuf<uint32_t> orig;
    // weight statistics for the initial Delta (Algorithm 1 / Section 5): sum over u < v, minimum
    DBuf<unsigned long long> wsum;
    CLD_TRY(wsum.alloc(1, s));
    CLD_CUDA(cudaMemsetAsync(wsum.get(), 0, 8, s));
    CLD_CUDA(cudaMemsetAsync(scal.get() + 6, 0xFF, 4, s));
    CLD_CUDA(cudaMemsetAsync(scal.get() + 7, 0, 4, s));
    if (lcc) {
        DBuf<uint32_t> parent, size, keep, newid;
        DBuf<unsigned long long> best;
        CLD_TRY(parent.alloc(n, s));
        CLD_TRY(best.alloc(1, s));
        CLD_K(K_MISC, s, k_iota<<<grid_for(n, 256), 256, 0, s>>>(parent.get(), n));
        CLD_LAUNCH_CHECK();
        const CsrAdj ca{off.get(), adj.get()};
        // Afforest-style: link two neighbours per node, find the dominant tree by sampling,
        // then link the remaining edges of the nodes outside it (all no-ops on a graph without edges)
        constexpr uint32_t kNeighbourRounds = 2;
        for (uint32_t r = 0; r < kNeighbourRounds; ++r) {
            if (packed) CLD_K(K_CC, s, k_cc_link_nth<<<grid_for(n, 256), 256, 0, s>>>(la, n, r, parent.get()));
            else CLD_K(K_CC, s, k_cc_link_nth<<<grid_for(n, 256), 256, 0, s>>>(ca, n, r, parent.get()));
            CLD_K(K_CC, s, k_cc_compress<<<grid_for(n, 256), 256, 0, s>>>(parent.get(), n));
        }
        CLD_LAUNCH_CHECK();
        constexpr uint32_t kSamples = 1024;
        DBuf<uint32_t> samp;
        CLD_TRY(samp.alloc(kSamples, s));
        CLD_K(K_CC, s, k_cc_sample<<<4, 256, 0, s>>>(parent.get(), n, kSamples, samp.get()));
        CLD_LAUNCH_CHECK();
        std::vector<uint32_t> hs(kSamples);
        CLD_CUDA(cudaMemcpyAsync(hs.data(), samp.get(), kSamples * 4, cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaMemcpyAsync(hbad + 1, scal.get() + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaMemcpyAsync(hbad + 8, scal.get() + 8, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        // a failed sort leaves the graph unusable: stop before anything indexes by its entries
        if (hbad[8]) return fail(CLDIAM_ERR_TIMEOUT, "radix sort look-back wait expired or CSR assembly inconsistent");
        nnz = hbad[1];
        if (nnz > 0) {
            std::sort(hs.begin(), hs.end());
            uint32_t giant = hs[0], best_run = 0;
            for (size_t i = 0; i < hs.size();) {
                size_t j = i;
                while (j < hs.size() && hs[j] == hs[i]) ++j;
                if (j - i > best_run) { best_run = (uint32_t)(j - i); giant = hs[i]; }
                i = j;
            }
            if (packed)
                CLD_K(K_CC, s, k_cc_link_rest<<<grid_for(n, 256), 256, 0, s>>>(la, n, kNeighbourRounds, giant,
                                                                                parent.get()));
            else
                CLD_K(K_CC, s, k_cc_link_rest<<<grid_for(n, 256), 256, 0, s>>>(ca, n, kNeighbourRounds, giant,
                                                                                parent.get()));
            CLD_K(K_CC, s, k_cc_compress<<<grid_for(n, 256), 256, 0, s>>>(parent.get(), n));
            CLD_LAUNCH_CHECK();
            CLD_CUDA(cudaMemsetAsync(scal.get() + 3, 0, 4, s));
            CLD_K(K_CC, s, k_cc_size_of<<<grid_for(n, 256), 256, 0, s>>>(parent.get(), n, giant, scal.get() + 3));
            CLD_CUDA(cudaMemsetAsync(best.get(), 0, 8, s));
            CLD_K(K_CC, s, k_cc_giant_best<<<1, 1, 0, s>>>(scal.get() + 3, n, giant, best.get()));
            CLD_LAUNCH_CHECK();
        } else {
            CLD_CUDA(cudaMemsetAsync(best.get(), 0, 8, s));
        }
        CLD_TRY(size.alloc(n, s));
        CLD_CUDA(cudaMemsetAsync(size.get(), 0, (size_t)n * 4, s));
        const uint32_t* gcount = nnz > 0 ? scal.get() + 3 : nullptr;
        CLD_K(K_CC, s, k_cc_count<<<grid_for(n, 256), 256, 0, s>>>(parent.get(), n, size.get(), gcount));
        CLD_LAUNCH_CHECK();
        CLD_K(K_CC, s, k_cc_best<<<grid_for(n, 256), 256, 0, s>>>(parent.get(), size.get(), n, best.get(), gcount));
        CLD_LAUNCH_CHECK();
        CLD_TRY(keep.alloc(n, s));
        CLD_TRY(newid.alloc(n, s));
        CLD_K(K_CC, s, k_cc_keep<<<grid_for(n, 256), 256, 0, s>>>(parent.get(), n, best.get(), keep.get()));
        CLD_LAUNCH_CHECK();
        CLD_TRY(scan_exclusive_u32(keep.get(), newid.get(), n, scal.get() + 4, s));
        // the LCC's node and entry counts stay on the device: its arrays are sized by the bounds n and
        // nnz, and the kernels read the counts from scal[4] / scal[5]
        CLD_TRY(orig.alloc(n, s));
        CLD_CUDA(cudaMemsetAsync(deg.get(), 0, ((size_t)n + 1) * 4, s));
        if (packed)
            CLD_K(K_CSR, s, k_lcc_degrees<<<grid_for(n, 256), 256, 0, s>>>(keep.get(), newid.get(), la, n, deg.get(),
                                                                          orig.get()));
        else
            CLD_K(K_CSR, s, k_lcc_degrees<<<grid_for(n, 256), 256, 0, s>>>(keep.get(), newid.get(), ca, n, deg.get(),
                                                                          orig.get()));
        CLD_LAUNCH_CHECK();
        CLD_TRY(scan_exclusive_u32(deg.get(), degx.get(), n, scal.get() + 5, s));  // zeros past the kept nodes
        DBuf<uint64_t> noff;
        DBuf<uint2> nadj;
        DBuf<uint32_t> nrow;
        CLD_TRY(noff.alloc((size_t)n + 1, s));
        CLD_TRY(nadj.alloc(nnz ? nnz : 1, s));
        // the row of every entry (COO form) is written only by the (key, weight) copy; a CSR assembled from the
        // lists leaves it out (its users build it from the offsets when they need it: fill_rows)
        if (!packed) CLD_TRY(nrow.alloc(nnz ? nnz : 1, s));
        if (packed) {
            // the LCC's CSR straight from the lists: the whole graph's CSR is never built
            DBuf<uint4> info;
            CLD_TRY(info.alloc(n, s));
            CLD_CUDA(cudaMemsetAsync(info.get(), 0xFF, (size_t)n * 16, s));
            CLD_K(K_CSR, s, k_lcc_offsets_lists<<<grid_for((size_t)n + 1, 256), 256, 0, s>>>(
                                degx.get(), scal.get() + 4, scal.get() + 5, orig.get(), la, noff.get(), info.get()));
            CLD_LAUNCH_CHECK();
            if (mu > 0) {
                CLD_K(K_CSR, s, k_lcc_assemble<<<grid_for(mu, 256, 4), 256, 0, s>>>(la, mu, info.get(), newid.get(),
                                                                                nnz ? nnz : 1, nadj.get(),
                                                                                wsum.get(), scal.get() + 6,
                                                                                scal.get() + 8));
                CLD_LAUNCH_CHECK();
            }
        } else {
            DBuf<uint2> map;
            CLD_TRY(map.alloc(n, s));
            CLD_CUDA(cudaMemsetAsync(map.get(), 0xFF, (size_t)n * 8, s));
            CLD_K(K_CSR, s, k_lcc_offsets<<<grid_for((size_t)n + 1, 256), 256, 0, s>>>(degx.get(), n, scal.get() + 4,
                                                                                    scal.get() + 5, orig.get(),
                                                                                    off.get(), noff.get(), map.get()));
            CLD_LAUNCH_CHECK();
            if (nnz) {
                CLD_K(K_CSR, s, k_lcc_copy<<<grid_for(nnz, 256), 256, 0, s>>>(map.get(), newid.get(), row.get(),
                                                                             adj.get(), nnz, nrow.get(), nadj.get(),
                                                                             wsum.get(), scal.get() + 6));
                CLD_LAUNCH_CHECK();
            }
        }
        g->off = noff.detach();
        g->adj = nadj.detach();
        g->row = nrow.detach();
        CLD_K(K_CSR, s, k_degree_max<<<grid_for(n, 256), 256, 0, s>>>(g->off, n, scal.get() + 4, scal.get() + 7));
        CLD_LAUNCH_CHECK();
    } else {
        CLD_CUDA(cudaMemcpyAsync(hbad + 1, scal.get() + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        nnz = hbad[1];
        CLD_TRY(orig.alloc(n, s));
        CLD_K(K_MISC, s, k_iota<<<grid_for(n, 256), 256, 0, s>>>(orig.get(), n));
        CLD_LAUNCH_CHECK();
        g->off = off.detach();
        g->adj = adj.detach();
        g->row = row.detach();
        if (nnz) {
            CLD_K(K_CSR, s, k_graph_stats<<<grid_for(nnz, 256), 256, 0, s>>>(g->row, g->adj, nnz, wsum.get(),
                                                                             scal.get() + 6));
            CLD_LAUNCH_CHECK();
        }
        CLD_K(K_CSR, s, k_degree_max<<<grid_for(n, 256), 256, 0, s>>>(g->off, n, nullptr, scal.get() + 7));
        CLD_LAUNCH_CHECK();
    }
    g->orig = orig.detach();
    g->connected = lcc;
    uint64_t* hsum = reinterpret_cast<uint64_t*>(static_cast<char*>(g->host.h) + 64);
    CLD_CUDA(cudaMemcpyAsync(hsum, wsum.get(), 8, cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaMemcpyAsync(hbad + 1, scal.get() + 1, 8 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    if (hbad[8]) return fail(CLDIAM_ERR_TIMEOUT, "radix sort look-back wait expired or CSR assembly inconsistent");
    if (lcc) {
        g->n = hbad[4];
        g->nnz = hbad[5];
    } else {
        g->n = n;
        g->nnz = nnz;
    }
    g->wsum_upper = *hsum;
    g->wmin = hbad[6];
    g->max_deg = hbad[7];
    *out = owner.release();
    return CLDIAM_OK;
}

// row[p] = v for every position p of row v (an empty row writes nothing): a lane per row writes a short row
// itself; the rows of more than 32 entries in a warp are written by the whole warp, one after another
__global__ void k_fill_rows(const uint64_t* __restrict__ off, uint32_t n, uint32_t* __restrict__ row) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
        const uint32_t v = base + lane;
        const uint64_t o0 = v < n ? off[v] : 0, o1 = v < n ? off[v + 1] : 0;
        const bool big = o1 - o0 > 32;
        if (!big)
            for (uint64_t p = o0; p < o1; ++p) row[p] = v;
        unsigned bigs = __ballot_sync(0xffffffffu, big);
        while (bigs) {
            const uint32_t src = (uint32_t)__ffs(bigs) - 1;
            const uint64_t b0 = __shfl_sync(0xffffffffu, o0, src), b1 = __shfl_sync(0xffffffffu, o1, src);
            for (uint64_t p = b0 + lane; p < b1; p += 32) row[p] = base + src;
            bigs &= bigs - 1;
        }
    }
}

cldiam_status fill_rows(const uint64_t* off, uint32_t n, uint32_t* row, cudaStream_t s) {
    if (n == 0) return CLDIAM_OK;
    CLD_K(K_CSR, s, k_fill_rows<<<grid_for(n, 256), 256, 0, s>>>(off, n, row));
    CLD_LAUNCH_CHECK();
    return CLDIAM_OK;
}

cldiam_status delta0(const cldiam_graph* g, int mode, uint32_t explicit_value, uint32_t* out) {
    if (mode == CLDIAM_DELTA0_EXPLICIT) {
        if (explicit_value == 0) return fail(CLDIAM_ERR_INVALID_ARG, "explicit delta0 must be >= 1");
        *out = explicit_value > kDeltaMax ? kDeltaMax : explicit_value;
        return CLDIAM_OK;
    }
    if (g->nnz == 0) {
        *out = 1;
        return CLDIAM_OK;
    }
    if (mode == CLDIAM_DELTA0_MIN) {
        *out = g->wmin;
        return CLDIAM_OK;
    }
    if (mode != CLDIAM_DELTA0_AVG) return fail(CLDIAM_ERR_INVALID_ARG, "unknown delta0 mode");
    uint64_t avg = g->wsum_upper / (g->nnz / 2);
    if (avg < 1) avg = 1;
    if (avg > kDeltaMax) avg = kDeltaMax;
    *out = (uint32_t)avg;
    return CLDIAM_OK;
}

}  // namespace cld
