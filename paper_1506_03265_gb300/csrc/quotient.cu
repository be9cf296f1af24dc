// Weighted quotient graph G_C (Section 4): for every edge (u,v) of G whose
// endpoints lie in different clusters, an edge between the clusters of weight
// w(u,v) + D_u + D_v; only the lightest edge per cluster pair is kept.
//
// Every directed CSR entry emits (cid_u * k + cid_v, weight); a stable radix
// sort on the 2 log2 k significant key bits groups equal pairs, whose run
// heads become the quotient entries and an atomicMin over each run keeps the
// minimum.  Because the CSR is symmetric the result is symmetric, sorted by
// (row, col).  While k is small enough for a dense k x k matrix to stay in
// L2, the pairs are instead folded into that matrix with atomicMin and read
// out row by row, which gives the same sorted CSR.
#include "cluster_dev.cuh"
#include "internal.cuh"
#include "prof.cuh"

namespace cld {

namespace {


// (cid, D) of every node in one word, so an edge's far end costs one gather
__global__ void k_q_pack_cd(uint32_t n, const uint32_t* __restrict__ cid, const uint32_t* __restrict__ D,
                            uint2* __restrict__ cd) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        cd[v] = make_uint2(cid[v], D[v]);
}

template <class K>
__global__ void k_q_emit(const uint32_t* __restrict__ row, const uint2* __restrict__ adj, uint64_t nnz,
                         const uint2* __restrict__ cd, uint32_t k, K* __restrict__ keys, uint32_t* __restrict__ vals,
                         uint32_t* __restrict__ count, uint32_t* __restrict__ overflow) {
    __shared__ uint32_t scratch[33];
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < nnz; base += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t i = base + threadIdx.x;
        bool take = false;
        K key = 0;
        uint32_t wq = 0;
        if (i < nnz) {
            uint32_t u = row[i];
            uint2 e = adj[i];
            const uint2 pu = cd[u], pv = cd[e.x];
            uint32_t a = pu.x, b = pv.x;
            if (a != b) {
                uint64_t s = (uint64_t)pu.y + e.y + pv.y;
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

// Dense alternative for small k: fold every inter-cluster edge into the k x k matrix M with
// atomicMin (it stays in L2), then read the rows out in column order.  The quotient is symmetric
// (an edge's weight D_u + w + D_v does not depend on its direction), so each undirected edge is
// folded once, from its u < v entry, into the upper triangle, which is then mirrored.
constexpr int QE_U = 4;  // entries per thread per sweep, loads issued together
__global__ void __launch_bounds__(256) k_q_dense_emit(const uint32_t* __restrict__ row, const uint2* __restrict__ adj,
                                                      uint64_t nnz, const uint2* __restrict__ cd, uint32_t k,
                                                      uint32_t* __restrict__ M, uint32_t* __restrict__ overflow) {
    // the CSR streams through once (evict-first, no L1); (cid, D) and the matrix are reused (evict-last)
    const uint64_t pol_stream = l2_evict_first_policy(), pol_keep = l2_evict_last_policy();
    bool ovf = false;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * QE_U;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x * QE_U + threadIdx.x; base < nnz; base += stride) {
        uint32_t u[QE_U];
        uint2 e[QE_U];
#pragma unroll
        for (int j = 0; j < QE_U; ++j) {
            const uint64_t i = base + (uint64_t)j * blockDim.x;
            u[j] = i < nnz ? ld_stream_u32(row + i, pol_stream) : 0u;
            e[j] = i < nnz ? ld_stream_u2(adj + i, pol_stream) : make_uint2(0u, 0u);
        }
        unsigned long long pu[QE_U], pv[QE_U];
#pragma unroll
        for (int j = 0; j < QE_U; ++j) {
            const bool take = u[j] < e[j].x;  // each undirected edge once (padding has u = e.x = 0)
            pu[j] = take ? ld_nc_keep_u64(reinterpret_cast<const unsigned long long*>(cd) + u[j], pol_keep) : 0ull;
            pv[j] = take ? ld_nc_keep_u64(reinterpret_cast<const unsigned long long*>(cd) + e[j].x, pol_keep) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < QE_U; ++j) {
            const uint32_t a = (uint32_t)pu[j], b = (uint32_t)pv[j];
            if (!(u[j] < e[j].x) || a == b) continue;
            uint64_t s = (pu[j] >> 32) + e[j].y + (pv[j] >> 32);
            if (s >= 0xFFFFFFFFull) {
                ovf = true;
                s = 0xFFFFFFFEull;
            }
            uint32_t* m = &M[(size_t)min(a, b) * k + max(a, b)];
            // entries only decrease, so a stale copy in this SM's L1 is never below the current value: reading
            // through L1 can let a useless atomicMin through but never hold back one that lowers the entry
            if ((uint32_t)s < __ldca(m)) atomicMin(m, (uint32_t)s);
        }
    }
    if (__any_sync(0xffffffffu, ovf) && lane_id() == 0) atomicExch(overflow, 1u);
}

// The same folds for a CSR without a row array (every row has an entry: the LCC): each warp takes QW
// consecutive positions, finds the row holding its first from the chunk table (qrow: the row holding
// position QW * q) and the rows that start inside from the offsets, and gives every position its row with
// one OR-reduction of start bits per 32 positions.  The adjacency loads of a chunk are issued first.
constexpr int QW = 128;  // positions per warp chunk
__global__ void k_q_rows(uint32_t n, const uint64_t* __restrict__ off, uint32_t* __restrict__ qrow) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint64_t o0 = off[v], o1 = off[v + 1];
        for (uint64_t q = (o0 + QW - 1) / QW; q * QW < o1; ++q) qrow[q] = v;
    }
}

__global__ void __launch_bounds__(256) k_q_dense_emit_chunks(uint32_t n, uint32_t nnz, uint32_t nq,
                                                             const uint32_t* __restrict__ qrow,
                                                             const uint64_t* __restrict__ off,
                                                             const uint2* __restrict__ adj, const uint2* __restrict__ cd,
                                                             uint32_t k, uint32_t* __restrict__ M,
                                                             uint32_t* __restrict__ overflow) {
    __shared__ uint32_t sst[8][QW + 1];
    const uint64_t pol_stream = l2_evict_first_policy(), pol_keep = l2_evict_last_policy();
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned le_mask = 0xffffffffu >> (31u - lane);  // lanes <= this one
    const uint32_t nwarps = gridDim.x * 8;
    bool ovf = false;
    for (uint32_t q = blockIdx.x * 8 + warp; q < nq; q += nwarps) {
        const uint32_t p0 = q * QW;
        uint2 e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t p = p0 + 32u * u + lane;
            e[u] = p < nnz ? ld_stream_u2(adj + p, pol_stream) : make_uint2(0u, 0u);
        }
        // row B0 holds p0; rows B0 + 1 .. B1 start inside (p0, p0 + QW] (at most QW of them)
        const uint32_t B0 = __ldg(&qrow[q]);
        const uint32_t B1 = q + 1 < nq ? __ldg(&qrow[q + 1]) : n - 1;
        const uint32_t nr = min(B1 - B0, (uint32_t)QW);
        __syncwarp();  // the previous chunk's starts have been read
        for (uint32_t j = lane; j < nr; j += 32) sst[warp][j] = (uint32_t)__ldg(&off[B0 + 1 + j]);
        __syncwarp();
        uint32_t own[4];
        {
            uint32_t B = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) B += (uint32_t)__popc(group_starts(sst[warp] + B, nr - B, p0 + 32u * u, B, lane,
                                                                         le_mask, &own[u]));
        }
        unsigned long long pu[4], pv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t r = B0 + own[u];
            const bool take = p0 + 32u * u + lane < nnz && r < e[u].x;  // each undirected edge once
            pu[u] = take ? ld_nc_keep_u64(reinterpret_cast<const unsigned long long*>(cd) + r, pol_keep) : 0ull;
            pv[u] = take ? ld_nc_keep_u64(reinterpret_cast<const unsigned long long*>(cd) + e[u].x, pol_keep) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t r = B0 + own[u];
            const uint32_t a = (uint32_t)pu[u], b = (uint32_t)pv[u];
            if (!(p0 + 32u * u + lane < nnz && r < e[u].x) || a == b) continue;
            uint64_t sw = (pu[u] >> 32) + e[u].y + (pv[u] >> 32);
            if (sw >= 0xFFFFFFFFull) {
                ovf = true;
                sw = 0xFFFFFFFEull;
            }
            uint32_t* m = &M[(size_t)min(a, b) * k + max(a, b)];
            if ((uint32_t)sw < __ldca(m)) atomicMin(m, (uint32_t)sw);
        }
    }
    if (__any_sync(0xffffffffu, ovf) && lane == 0) atomicExch(overflow, 1u);
}

// lower triangle := transpose of the upper one, through 32 x 32 shared-memory tiles
__global__ void k_q_dense_mirror(uint32_t* __restrict__ M, uint32_t k) {
    __shared__ uint32_t t[32][33];
    const uint32_t r = blockIdx.y, c = blockIdx.x;  // source tile (r, c) with c >= r
    if (c < r) return;
    for (uint32_t y = threadIdx.y; y < 32; y += blockDim.y) {
        const uint32_t a = r * 32 + y, b = c * 32 + threadIdx.x;
        t[y][threadIdx.x] = (a < k && b < k) ? M[(size_t)a * k + b] : 0xFFFFFFFFu;
    }
    __syncthreads();
    for (uint32_t y = threadIdx.y; y < 32; y += blockDim.y) {
        const uint32_t a = c * 32 + y, b = r * 32 + threadIdx.x;  // destination (a, b) = source (b, a)
        if (a < k && b < k && a > b) M[(size_t)a * k + b] = t[threadIdx.x][y];
    }
}

// row a's entry count (warp per row)
__global__ void k_q_dense_count(const uint32_t* __restrict__ M, uint32_t k, uint32_t* __restrict__ deg) {
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < k; a += warps) {
        uint32_t c = 0;
        for (uint32_t b0 = 0; b0 < k; b0 += 32) {
            const uint32_t b = b0 + lane_id();
            c += __popc(__ballot_sync(0xffffffffu, b < k && M[(size_t)a * k + b] != 0xFFFFFFFFu));
        }
        if (lane_id() == 0) deg[a] = c;
    }
}

__global__ void k_q_dense_fill(const uint32_t* __restrict__ M, uint32_t k, const uint32_t* __restrict__ start,
                               uint32_t* __restrict__ col, uint32_t* __restrict__ w) {
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < k; a += warps) {
        uint32_t pos = start[a];
        for (uint32_t b0 = 0; b0 < k; b0 += 32) {
            const uint32_t b = b0 + lane_id();
            const uint32_t x = b < k ? M[(size_t)a * k + b] : 0xFFFFFFFFu;
            const unsigned bal = __ballot_sync(0xffffffffu, x != 0xFFFFFFFFu);
            if (x != 0xFFFFFFFFu) {
                const uint32_t at = pos + (uint32_t)__popc(bal & lanemask_lt());
                col[at] = b;
                w[at] = x;
            }
            pos += (uint32_t)__popc(bal);
        }
    }
}

__global__ void k_q_widen(const uint32_t* __restrict__ start, uint32_t k, uint32_t total, uint64_t* __restrict__ off) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= k; i += gridDim.x * blockDim.x)
        off[i] = (i == k) ? (uint64_t)total : (uint64_t)start[i];
}

cldiam_status build_quotient_dense(const cldiam_clustering* c, cldiam_quotient* q) {
    const cldiam_graph* g = c->g;
    const cudaStream_t s = g->stream;
    const uint32_t k = c->k;
    uint32_t* hh = reinterpret_cast<uint32_t*>(static_cast<char*>(const_cast<cldiam_graph*>(g)->host.h) + 160);
    DBuf<uint32_t> M, scal, deg, start;
    CLD_TRY(M.alloc((size_t)k * k, s));
    CLD_TRY(scal.alloc(2, s));
    CLD_TRY(deg.alloc((size_t)k + 1, s));
    CLD_TRY(start.alloc((size_t)k + 1, s));
    CLD_CUDA(cudaMemsetAsync(M.get(), 0xFF, (size_t)k * k * 4, s));
    CLD_CUDA(cudaMemsetAsync(scal.get(), 0, 8, s));
    if (g->nnz) {
        DBuf<uint2> cd;
        CLD_TRY(cd.alloc(g->n, s));
        CLD_K(K_QUOTIENT, s, k_q_pack_cd<<<grid_for(g->n, 256), 256, 0, s>>>(g->n, c->cid, c->D, cd.get()));
        if (g->row) {
            CLD_K(K_QUOTIENT, s, k_q_dense_emit<<<grid_for((g->nnz + QE_U - 1) / QE_U, 256), 256, 0, s>>>(
                                     g->row, g->adj, g->nnz, cd.get(), k, M.get(), scal.get()));
        } else {
            // no row array: an assembled LCC, where every row has an entry (positions fit 32 bits)
            if (g->nnz >= 0xFFFFFFFFull) return fail(CLDIAM_ERR_UNSUPPORTED, "2^32 or more CSR entries");
            const uint32_t nqc = (uint32_t)((g->nnz + QW - 1) / QW);
            DBuf<uint32_t> qrow;
            CLD_TRY(qrow.alloc(nqc, s));
            CLD_K(K_QUOTIENT, s, k_q_rows<<<grid_for(g->n, 256), 256, 0, s>>>(g->n, g->off, qrow.get()));
            CLD_K(K_QUOTIENT, s, k_q_dense_emit_chunks<<<grid_for((size_t)nqc * 32, 256), 256, 0, s>>>(
                                     g->n, (uint32_t)g->nnz, nqc, qrow.get(), g->off, g->adj, cd.get(), k, M.get(),
                                     scal.get()));
        }
        CLD_LAUNCH_CHECK();
    }
    {
        const uint32_t nt = (k + 31) / 32;
        CLD_K(K_QUOTIENT, s, k_q_dense_mirror<<<dim3(nt, nt), dim3(32, 8), 0, s>>>(M.get(), k));
        CLD_LAUNCH_CHECK();
    }
    CLD_K(K_QUOTIENT, s, k_q_dense_count<<<grid_for((size_t)k * 32, 256), 256, 0, s>>>(M.get(), k, deg.get()));
    CLD_LAUNCH_CHECK();
    CLD_TRY(scan_exclusive_u32(deg.get(), start.get(), k, scal.get() + 1, s));
    CLD_CUDA(cudaMemcpyAsync(hh, scal.get(), 8, cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    if (hh[0]) return fail(CLDIAM_ERR_OVERFLOW, "a quotient edge weight reached 2^32 - 1");
    const uint32_t nq = hh[1];
    DBuf<uint32_t> col, w;
    DBuf<uint64_t> off;
    CLD_TRY(col.alloc(nq ? nq : 1, s));
    CLD_TRY(w.alloc(nq ? nq : 1, s));
    CLD_TRY(off.alloc((size_t)k + 1, s));
    CLD_K(K_QUOTIENT, s, k_q_dense_fill<<<grid_for((size_t)k * 32, 256), 256, 0, s>>>(M.get(), k, start.get(), col.get(),
                                                                                    w.get()));
    CLD_K(K_QUOTIENT, s, k_q_widen<<<grid_for((size_t)k + 1, 256), 256, 0, s>>>(start.get(), k, nq, off.get()));
    CLD_LAUNCH_CHECK();
    // algorithmic bytes: each CSR entry's (col, w) and, with a row array, its row (else the offsets of the
    // chunks' rows); for half of the entries two cluster ids and two D values; the matrix mirrored and read twice
    prof_add_bytes(K_QUOTIENT, (double)g->nnz * (g->row ? 20.0 : 16.0) + (g->row ? 0.0 : 8.0 * g->n) +
                                   (double)k * k * 12.0);
    CLD_CUDA(cudaStreamSynchronize(s));
    q->k = k;
    q->nnz = nq;
    q->off = off.detach();
    q->col = col.detach();
    q->w = w.detach();
    return CLDIAM_OK;
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
        DBuf<uint2> cd;
        CLD_TRY(cd.alloc(g->n, s));
        CLD_K(K_QUOTIENT, s, k_q_pack_cd<<<grid_for(g->n, 256), 256, 0, s>>>(g->n, c->cid, c->D, cd.get()));
        DBuf<uint32_t> rows;  // the COO rows, built from the offsets when the graph keeps none
        const uint32_t* row = g->row;
        if (!row) {
            CLD_TRY(rows.alloc(g->nnz, s));
            CLD_TRY(fill_rows(g->off, g->n, rows.get(), s));
            row = rows.get();
        }
        CLD_K(K_QUOTIENT, s, k_q_emit<K><<<grid_for(g->nnz, 256), 256, 0, s>>>(row, g->adj, g->nnz, cd.get(), k,
                                                                              keys.get(), vals.get(), scal.get(),
                                                                              scal.get() + 1));
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

    // unique cluster pairs with their lightest weight (run heads, scan, write)
    DBuf<uint32_t> col, w;
    DBuf<uint64_t> off;
    CLD_TRY(col.alloc(cnt ? cnt : 1, s));
    CLD_TRY(w.alloc(cnt ? cnt : 1, s));
    CLD_TRY(off.alloc((size_t)k + 1, s));
    CLD_CUDA(cudaMemsetAsync(w.get(), 0xFF, (size_t)(cnt ? cnt : 1) * 4, s));
    if (sizeof(K) == 8)
        CLD_TRY(unique_min_sorted_u64((const uint64_t*)sk, sv, cnt, ~0ull, k, nullptr, col.get(), w.get(), 1,
                                      off.get(), k, scal.get() + 2, s));
    else
        CLD_TRY(unique_min_sorted_u32((const uint32_t*)sk, sv, cnt, 0xFFFFFFFFu, k, nullptr, col.get(), w.get(), 1,
                                      off.get(), k, scal.get() + 2, s));
    CLD_CUDA(cudaMemcpyAsync(hh + 2, scal.get() + 2, 4, cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    const uint32_t nq = hh[2];
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
    // dense deduplication while the k x k matrix fits in L2 (auto) or when asked; radix sort otherwise
    const bool dense = c->quotient_mode == CLDIAM_QUOTIENT_DENSE ||
                       (c->quotient_mode == CLDIAM_QUOTIENT_AUTO && c->k <= tuning_for(c->g->nnz).dense_quotient_k);
    if (dense && c->k > 65535u) {
        free_quotient(q);
        return fail(CLDIAM_ERR_UNSUPPORTED, "dense quotient deduplication needs k <= 65535");
    }
    cldiam_status st = dense ? build_quotient_dense(c, q)
                       : ((uint64_t)c->k * c->k <= 0xFFFFFFFFull) ? build_quotient<uint32_t>(c, q)
                                                                  : build_quotient<uint64_t>(c, q);
    if (st != CLDIAM_OK) {
        free_quotient(q);
        return st;
    }
    *out = q;
    return CLDIAM_OK;
}

}  // namespace cld
