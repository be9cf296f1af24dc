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
    __shared__ uint32_t scratch[33];
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
        uint32_t slot = block_append(count, take, scratch);  // one global atomic per CTA
        if (take) {
            keys[slot] = key;
            vals[slot] = wq;
        }
    }
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

    // unique cluster pairs with their lightest weight, in one look-back pass
    DBuf<uint32_t> qrow, col, w;
    DBuf<uint64_t> off;
    CLD_TRY(qrow.alloc(cnt ? cnt : 1, s));
    CLD_TRY(col.alloc(cnt ? cnt : 1, s));
    CLD_TRY(w.alloc(cnt ? cnt : 1, s));
    CLD_TRY(off.alloc((size_t)k + 1, s));
    CLD_CUDA(cudaMemsetAsync(w.get(), 0xFF, (size_t)(cnt ? cnt : 1) * 4, s));
    if (sizeof(K) == 8)
        CLD_TRY(unique_min_sorted_u64((const uint64_t*)sk, sv, cnt, ~0ull, k, qrow.get(), col.get(), w.get(), 1,
                                      scal.get() + 2, s));
    else
        CLD_TRY(unique_min_sorted_u32((const uint32_t*)sk, sv, cnt, 0xFFFFFFFFu, k, qrow.get(), col.get(), w.get(), 1,
                                      scal.get() + 2, s));
    CLD_CUDA(cudaMemcpyAsync(hh + 2, scal.get() + 2, 4, cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    const uint32_t nq = hh[2];
    CLD_TRY(offsets_from_rows(qrow.get(), nq, k, off.get(), s));
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
    cldiam_status st = ((uint64_t)c->k * c->k <= 0xFFFFFFFFull) ? build_quotient<uint32_t>(c, q)
                                                                  : build_quotient<uint64_t>(c, q);
    if (st != CLDIAM_OK) {
        free_quotient(q);
        return st;
    }
    *out = q;
    return CLDIAM_OK;
}

}  // namespace cld
