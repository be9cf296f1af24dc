// Weighted quotient graph G_C (Section 4): for every edge (u,v) of G whose
// endpoints lie in different clusters, an edge between the clusters of weight
// w(u,v) + D_u + D_v; only the lightest edge per cluster pair is kept.
//
// Every directed CSR entry emits (cid_u * k + cid_v, weight); a stable radix
// sort on the 2 log2 k significant key bits groups equal pairs, whose run
// heads become the quotient entries and an atomicMin over each run keeps the
// minimum.  Because the CSR is symmetric the result is symmetric, sorted by
// (row, col).
#include "internal.cuh"
#include "prof.cuh"

namespace cld {

namespace {

template <class K>
__global__ void k_q_emit(const uint32_t* __restrict__ row, const uint2* __restrict__ adj, uint64_t nnz,
                         const uint32_t* __restrict__ cid, const uint32_t* __restrict__ D, uint32_t k,
                         K* __restrict__ keys, uint32_t* __restrict__ vals, uint32_t* __restrict__ count,
                         uint32_t* __restrict__ overflow) {
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < nnz; base += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t i = base + threadIdx.x;
        bool take = false;
        K key = 0;
        uint32_t wq = 0;
        if (i < nnz) {
            uint32_t u = row[i];
            uint2 e = adj[i];
            uint32_t a = cid[u], b = cid[e.x];
            if (a != b) {
                uint64_t s = (uint64_t)D[u] + e.y + D[e.x];
                if (s >= 0xFFFFFFFFull) {
                    atomicExch(overflow, 1u);
                    s = 0xFFFFFFFEull;
                }
                take = true;
                key = (K)a * (K)k + (K)b;
                wq = (uint32_t)s;
            }
        }
        uint32_t slot = warp_append(count, take);
        if (take) {
            keys[slot] = key;
            vals[slot] = wq;
        }
    }
}

template <class K>
__global__ void k_q_heads(const K* __restrict__ keys, uint32_t cnt, uint32_t* __restrict__ flags) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
        flags[i] = (i == 0 || keys[i - 1] != keys[i]) ? 1u : 0u;
}

template <class K>
__global__ void k_q_unique(const K* __restrict__ keys, const uint32_t* __restrict__ vals,
                           const uint32_t* __restrict__ flags, const uint32_t* __restrict__ excl, uint32_t cnt,
                           uint32_t k, uint32_t* __restrict__ col, uint32_t* __restrict__ w, uint32_t* __restrict__ deg) {
    for (uint32_t base = blockIdx.x * blockDim.x; base < cnt; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const bool valid = i < cnt;
        const K key = valid ? keys[i] : (K)0;
        uint32_t v = valid ? vals[i] : 0xFFFFFFFFu;
        // one atomicMin per run segment of this warp instead of one per item
        v = warp_seg_min(key, valid, v);
        const bool tail = warp_run_tail(key, valid);  // all lanes take part in the shuffles
        if (!valid) continue;
        const uint32_t r = excl[i] + flags[i] - 1u;
        if (tail) atomicMin(&w[r], v);
        if (flags[i]) {
            uint32_t a = (uint32_t)(key / k);
            col[r] = (uint32_t)(key - (K)a * k);
            atomicAdd(&deg[a], 1u);
        }
    }
}

__global__ void k_q_offsets(const uint32_t* __restrict__ excl, uint32_t k, uint32_t total, uint64_t* __restrict__ off) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= k; i += gridDim.x * blockDim.x)
        off[i] = (i == k) ? (uint64_t)total : (uint64_t)excl[i];
}

template <class K>
cldiam_status build_quotient(const cldiam_clustering* c, cldiam_quotient* q) {
    const cldiam_graph* g = c->g;
    const cudaStream_t s = g->stream;
    const uint32_t k = c->k;
    uint32_t* hh = reinterpret_cast<uint32_t*>(static_cast<char*>(const_cast<cldiam_graph*>(g)->host.h) + 160);
    DBuf<K> keys, keys2;
    DBuf<uint32_t> vals, vals2, scal;
    const uint64_t cap = g->nnz ? g->nnz : 1;
    CLD_TRY(keys.alloc(cap, s));
    CLD_TRY(vals.alloc(cap, s));
    CLD_TRY(scal.alloc(4, s));
    CLD_CUDA(cudaMemsetAsync(scal.get(), 0, 16, s));
    if (g->nnz) {
        CLD_K(K_QUOTIENT, s, k_q_emit<K><<<grid_for(g->nnz, 256), 256, 0, s>>>(g->row, g->adj, g->nnz, c->cid, c->D, k, keys.get(),
                                                          vals.get(), scal.get(), scal.get() + 1));
        CLD_LAUNCH_CHECK();
    }
    CLD_CUDA(cudaMemcpyAsync(hh, scal.get(), 8, cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    const uint32_t cnt = hh[0];
    if (hh[1]) return fail(CLDIAM_ERR_OVERFLOW, "a quotient edge weight reached 2^32 - 1");

    CLD_TRY(keys2.alloc(cnt ? cnt : 1, s));
    CLD_TRY(vals2.alloc(cnt ? cnt : 1, s));
    bool alt = false;
    const int bits = bits_for((uint64_t)k * k - 1);
    if (sizeof(K) == 8)
        CLD_TRY(radix_sort_pairs_u64((uint64_t*)keys.get(), vals.get(), (uint64_t*)keys2.get(), vals2.get(), cnt,
                                     bits, &alt, s));
    else
        CLD_TRY(radix_sort_pairs_u32((uint32_t*)keys.get(), vals.get(), (uint32_t*)keys2.get(), vals2.get(), cnt,
                                     bits, &alt, s));
    K* sk = alt ? keys2.get() : keys.get();
    uint32_t* sv = alt ? vals2.get() : vals.get();

    DBuf<uint32_t> flags, excl, deg, degx;
    CLD_TRY(flags.alloc(cnt ? cnt : 1, s));
    CLD_TRY(excl.alloc(cnt ? cnt : 1, s));
    if (cnt) {
        CLD_K(K_QUOTIENT, s, k_q_heads<K><<<grid_for(cnt, 256), 256, 0, s>>>(sk, cnt, flags.get()));
        CLD_LAUNCH_CHECK();
    }
    CLD_TRY(scan_exclusive_u32(flags.get(), excl.get(), cnt, scal.get() + 2, s));
    CLD_CUDA(cudaMemcpyAsync(hh + 2, scal.get() + 2, 4, cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    const uint32_t nq = hh[2];

    DBuf<uint32_t> col, w;
    DBuf<uint64_t> off;
    CLD_TRY(col.alloc(nq ? nq : 1, s));
    CLD_TRY(w.alloc(nq ? nq : 1, s));
    CLD_TRY(deg.alloc((size_t)k + 1, s));
    CLD_TRY(degx.alloc((size_t)k + 1, s));
    CLD_TRY(off.alloc((size_t)k + 1, s));
    CLD_CUDA(cudaMemsetAsync(w.get(), 0xFF, (size_t)(nq ? nq : 1) * 4, s));
    CLD_CUDA(cudaMemsetAsync(deg.get(), 0, ((size_t)k + 1) * 4, s));
    if (cnt) {
        CLD_K(K_QUOTIENT, s, k_q_unique<K><<<grid_for(cnt, 256), 256, 0, s>>>(sk, sv, flags.get(), excl.get(), cnt, k, col.get(), w.get(),
                                                         deg.get()));
        CLD_LAUNCH_CHECK();
    }
    CLD_TRY(scan_exclusive_u32(deg.get(), degx.get(), k, nullptr, s));
    CLD_K(K_QUOTIENT, s, k_q_offsets<<<grid_for((size_t)k + 1, 256), 256, 0, s>>>(degx.get(), k, nq, off.get()));
    CLD_LAUNCH_CHECK();
    CLD_CUDA(cudaStreamSynchronize(s));
    q->k = k;
    q->nnz = nq;
    q->off = off.detach();
    q->col = col.detach();
    q->w = w.detach();
    return CLDIAM_OK;
}

}  // namespace

void free_quotient(cldiam_quotient* q) {
    if (!q) return;
    dfree(q->off, q->stream);
    dfree(q->col, q->stream);
    dfree(q->w, q->stream);
    if (q->stream) cudaStreamSynchronize(q->stream);
    delete q;
}

cldiam_status quotient(const cldiam_clustering* c, cldiam_quotient** out) {
    if (!c || !out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL clustering or out");
    *out = nullptr;
    cldiam_quotient* q = new cldiam_quotient();
    q->c = c;
    q->stream = c->g->stream;
    q->max_fw_k = c->max_fw_k;
    cldiam_status st = ((uint64_t)c->k * c->k <= 0x100000000ull) ? build_quotient<uint32_t>(c, q)
                                                                  : build_quotient<uint64_t>(c, q);
    if (st != CLDIAM_OK) {
        free_quotient(q);
        return st;
    }
    *out = q;
    return CLDIAM_OK;
}

}  // namespace cld
