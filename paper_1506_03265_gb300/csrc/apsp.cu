// Phi(G_C) (Section 4): the largest finite shortest-path distance of the
// quotient graph, by exact blocked Floyd-Warshall over the dense k x k
// distance matrix in (min, +) arithmetic on the integer ALUs (min-plus is not
// a tensor-core contraction).
//
// Blocked FW with 64 x 64 tiles (Venkataraman, Sahni, Mukhopadhyaya): for
// each pivot tile r, (1) close the diagonal tile, (2) update the tiles of
// row r and column r through it, (3) update every other tile from its row-r
// and column-r tiles.  Two arithmetic forms share the kernels: the checked
// form keeps uint32 entries with 0xFFFFFFFF = no path, and a sum of two
// finite entries that reaches 2^32 - 1 raises the overflow flag instead of
// wrapping; the fast form uses 0x7FFFFFFF = no path, so a sum never wraps and
// one fused add-min per relaxation suffices (a path that would reach
// 0x7FFFFFFF stays "no path").  The fast form runs first; its result is
// exact when every pair ends up connected, otherwise the checked form
// recomputes the matrix.
#include <algorithm>
#include <atomic>
#include <mutex>

#include "internal.cuh"
#include "prof.cuh"

namespace cld {

namespace {

constexpr uint32_t INF = 0xFFFFFFFFu;
constexpr uint32_t INFF = 0x7FFFFFFFu;  // "no path" of the fast form

__device__ __forceinline__ uint32_t relax_min(uint32_t c, uint32_t a, uint32_t b, bool& ovf) {
    uint32_t s = a + b;
    bool carry = s < a;
    bool finite = (a != INF) & (b != INF);
    ovf |= finite & (carry | (s == INF));
    return (carry | !finite) ? c : (s < c ? s : c);
}

// one relaxation c = min(c, a + b) in the form's arithmetic
template <bool FAST>
__device__ __forceinline__ uint32_t fw_relax(uint32_t c, uint32_t a, uint32_t b, bool& ovf) {
    if constexpr (FAST) return __viaddmin_u32(a, b, c);
    else return relax_min(c, a, b, ovf);
}

__global__ void k_fw_init(uint32_t* __restrict__ M, uint32_t kp, uint32_t k, uint32_t none) {
    size_t total = (size_t)kp * kp;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t r = (uint32_t)(i / kp), c = (uint32_t)(i % kp);
        M[i] = (r == c) ? 0u : none;
    }
}

// caller-supplied CSR: offsets must start at 0, never decrease, end at nnz; columns < k
__global__ void k_fw_validate(const uint64_t* __restrict__ off, const uint32_t* __restrict__ col, uint32_t k,
                              uint64_t nnz, uint32_t* __restrict__ bad) {
    bool b = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= (uint64_t)k + nnz;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if (i <= k) {
            uint64_t o = off[i];
            if (o > nnz || (i == 0 && o != 0) || (i == k && o != nnz) || (i > 0 && off[i - 1] > o)) b = true;
        } else if (col[i - k - 1] >= k) {
            b = true;
        }
    }
    if (b) atomicExch(bad, 1u);
}

// edge weights into the matrix; a weight of 0x7FFFFFFF or more sets *wide (the fast form cannot hold it)
__global__ void k_fw_scatter(const uint64_t* __restrict__ off, const uint32_t* __restrict__ col,
                             const uint32_t* __restrict__ w, uint32_t k, uint32_t kp, uint32_t* __restrict__ M,
                             uint32_t* __restrict__ wide) {
    bool wd = false;
    for (uint32_t a = blockIdx.x; a < k; a += gridDim.x)
        for (uint64_t j = off[a] + threadIdx.x; j < off[a + 1]; j += blockDim.x) {
            uint32_t b = col[j];
            wd |= w[j] >= INFF;
            if (b != a) atomicMin(&M[(size_t)a * kp + b], w[j]);
        }
    if (wd && wide) atomicExch(wide, 1u);
}

// Tiles are T x T = 64 x 64; a CTA of 256 threads gives each thread a 4 x 4
// block (rows 4*ty.., cols 4*tx..).  Within the pivot tile and the pivot
// row / column tiles, iteration p reads row p and column p, which iteration p
// itself cannot change (D[p][p] = 0), so one barrier per p suffices.
constexpr int FT = 64;
constexpr int FQ = 4;       // 4 x 4 entries per thread
constexpr int FTH = 256;    // 16 x 16 threads
constexpr int FP = FT + 1;  // padded shared row

__device__ __forceinline__ void fw_load_tile(uint32_t (*t)[FP], const uint32_t* M, uint32_t kp, uint32_t ti,
                                             uint32_t tj) {
    for (int i = threadIdx.x; i < FT * FT; i += FTH) {
        int y = i / FT, x = i % FT;
        t[y][x] = M[((size_t)ti * FT + y) * kp + (size_t)tj * FT + x];
    }
}
__device__ __forceinline__ void fw_store_tile(uint32_t (*t)[FP], uint32_t* M, uint32_t kp, uint32_t ti, uint32_t tj) {
    for (int i = threadIdx.x; i < FT * FT; i += FTH) {
        int y = i / FT, x = i % FT;
        M[((size_t)ti * FT + y) * kp + (size_t)tj * FT + x] = t[y][x];
    }
}

// phase 1: the pivot tile against itself
template <bool FAST>
__global__ void __launch_bounds__(FTH) k_fw_phase1(uint32_t* __restrict__ M, uint32_t kp, uint32_t r,
                                                   uint32_t* __restrict__ ovf_flag) {
    __shared__ uint32_t t[FT][FP];
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    fw_load_tile(t, M, kp, r, r);
    __syncthreads();
    bool ovf = false;
    for (int p = 0; p < FT; ++p) {
        uint32_t a[FQ], b[FQ];
#pragma unroll
        for (int q = 0; q < FQ; ++q) {
            a[q] = t[ty * FQ + q][p];
            b[q] = t[p][tx * FQ + q];
        }
#pragma unroll
        for (int i = 0; i < FQ; ++i)
#pragma unroll
            for (int j = 0; j < FQ; ++j) {
                uint32_t& c = t[ty * FQ + i][tx * FQ + j];
                c = fw_relax<FAST>(c, a[i], b[j], ovf);
            }
        __syncthreads();
    }
    fw_store_tile(t, M, kp, r, r);
    if (ovf) atomicExch(ovf_flag, 1u);
}

// phase 2: tiles in pivot row r (blockIdx.y == 0) and pivot column r (blockIdx.y == 1)
template <bool FAST>
__global__ void __launch_bounds__(FTH) k_fw_phase2(uint32_t* __restrict__ M, uint32_t kp, uint32_t r,
                                                   uint32_t* __restrict__ ovf_flag) {
    __shared__ uint32_t piv[FT][FP];
    __shared__ uint32_t t[FT][FP];
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const bool is_row = blockIdx.y == 0;
    uint32_t o = blockIdx.x;
    if (o >= r) ++o;
    const uint32_t ti = is_row ? r : o, tj = is_row ? o : r;
    fw_load_tile(piv, M, kp, r, r);
    fw_load_tile(t, M, kp, ti, tj);
    __syncthreads();
    bool ovf = false;
    for (int p = 0; p < FT; ++p) {
        uint32_t a[FQ], b[FQ];
#pragma unroll
        for (int q = 0; q < FQ; ++q) {
            // row tile: min(t, piv[y][p] + t[p][x]); column tile: min(t, t[y][p] + piv[p][x])
            a[q] = is_row ? piv[ty * FQ + q][p] : t[ty * FQ + q][p];
            b[q] = is_row ? t[p][tx * FQ + q] : piv[p][tx * FQ + q];
        }
#pragma unroll
        for (int i = 0; i < FQ; ++i)
#pragma unroll
            for (int j = 0; j < FQ; ++j) {
                uint32_t& c = t[ty * FQ + i][tx * FQ + j];
                c = fw_relax<FAST>(c, a[i], b[j], ovf);
            }
        __syncthreads();
    }
    fw_store_tile(t, M, kp, ti, tj);
    if (ovf) atomicExch(ovf_flag, 1u);
}

// phase 3: every other tile from its pivot-column and pivot-row tiles; no barrier inside the p loop.
// The pivot-column tile is held transposed, so a thread reads its 4 rows of column p as one vector.
constexpr int FA = FT + 4;  // padded row of the transposed tile, 16-byte aligned
template <bool FAST>
__global__ void __launch_bounds__(FTH) k_fw_phase3(uint32_t* __restrict__ M, uint32_t kp, uint32_t r,
                                                   uint32_t* __restrict__ ovf_flag) {
    __shared__ __align__(16) uint32_t At[FT][FA];
    __shared__ __align__(16) uint32_t B[FT][FT];
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    uint32_t ti = blockIdx.y, tj = blockIdx.x;
    if (ti >= r) ++ti;
    if (tj >= r) ++tj;
    for (int i = threadIdx.x; i < FT * FT; i += FTH) {
        int y = i / FT, x = i % FT;
        At[x][y] = M[((size_t)ti * FT + y) * kp + (size_t)r * FT + x];
        B[y][x] = M[((size_t)r * FT + y) * kp + (size_t)tj * FT + x];
    }
    uint32_t c[FQ][FQ];
#pragma unroll
    for (int i = 0; i < FQ; ++i) {
        const uint4 v = *reinterpret_cast<const uint4*>(&M[((size_t)ti * FT + ty * FQ + i) * kp + (size_t)tj * FT + tx * FQ]);
        c[i][0] = v.x; c[i][1] = v.y; c[i][2] = v.z; c[i][3] = v.w;
    }
    __syncthreads();
    bool ovf = false;
#pragma unroll 8
    for (int p = 0; p < FT; ++p) {
        const uint4 av = *reinterpret_cast<const uint4*>(&At[p][ty * FQ]);
        const uint4 bv = *reinterpret_cast<const uint4*>(&B[p][tx * FQ]);
        const uint32_t a[FQ] = {av.x, av.y, av.z, av.w};
        const uint32_t b[FQ] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
        for (int i = 0; i < FQ; ++i)
#pragma unroll
            for (int j = 0; j < FQ; ++j) c[i][j] = fw_relax<FAST>(c[i][j], a[i], b[j], ovf);
    }
#pragma unroll
    for (int i = 0; i < FQ; ++i)
        *reinterpret_cast<uint4*>(&M[((size_t)ti * FT + ty * FQ + i) * kp + (size_t)tj * FT + tx * FQ]) =
            make_uint4(c[i][0], c[i][1], c[i][2], c[i][3]);
    if (!FAST && ovf) atomicExch(ovf_flag, 1u);
}

// largest entry below `none` among the k x k real entries; *missing = 1 if some entry is `none`
__global__ void k_fw_max_finite(const uint32_t* __restrict__ M, uint32_t kp, uint32_t k, uint32_t none,
                                uint32_t* __restrict__ out, uint32_t* __restrict__ missing) {
    uint32_t m = 0;
    bool miss = false;
    size_t total = (size_t)k * kp;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t c = (uint32_t)(i % kp);
        uint32_t v = M[i];
        if (c < k && v != none && v > m) m = v;
        miss |= c < k && v == none;
    }
    if (missing && __any_sync(0xffffffffu, miss) && lane_id() == 0) atomicExch(missing, 1u);
    m = block_reduce(m, [](uint32_t a, uint32_t b) { return a > b ? a : b; }, 0u);
    if (threadIdx.x == 0) atomicMax(out, m);
}

// Batched exact SSSP on the quotient CSR (multi-source Bellman-Ford): a CTA
// owns S consecutive sources and keeps dist[v][s] for all k nodes in shared
// memory; in each round one warp per node v pulls min(dist[u][s] + w(u,v))
// over its neighbours u for all S sources at once (lane = (neighbour slot,
// source)), and only v's warp writes row v.  Rounds repeat until no distance
// changes.  Exact, so the eccentricities and their maximum equal
// Floyd-Warshall's, with about rounds x entries x k work instead of k^3,
// which wins on sparse quotients.
template <int S, bool kCsrInSmem>
__global__ void __launch_bounds__(1024) k_apsp_msbf(const uint64_t* __restrict__ goff, const uint32_t* __restrict__ gcol,
                                                    const uint32_t* __restrict__ gw, uint32_t k, uint32_t nnz,
                                                    uint32_t* __restrict__ out_max, uint32_t* __restrict__ ovf_flag) {
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t* dist = sm;  // k x S
    // when it fits, the quotient CSR itself is staged in shared memory too (32-bit offsets)
    uint32_t* soff = sm + (size_t)k * S;
    uint32_t* scol = soff + (k + 1);
    uint32_t* sw = scol + nnz;
    // "some distance changed" flag of round r lives in slot r % 3: it is written during round r and
    // read after its closing barrier, and slot (r + 1) % 3 is cleared during round r, when no thread
    // can still be reading it (round r - 2) or writing it yet (round r + 1)
    __shared__ uint32_t s_changed[3];
    const uint32_t s0 = blockIdx.x * S;
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id(), nwarps = blockDim.x >> 5;
    const uint32_t my_s = lane % S, slot = lane / S;
    constexpr uint32_t kSlots = 32 / S;
    for (uint32_t i = threadIdx.x; i < k * S; i += blockDim.x) {
        const uint32_t v = i / S, s = i % S;
        dist[i] = (s0 + s == v) ? 0u : INF;
    }
    if (kCsrInSmem) {
        for (uint32_t i = threadIdx.x; i <= k; i += blockDim.x) soff[i] = (uint32_t)goff[i];
        for (uint32_t i = threadIdx.x; i < nnz; i += blockDim.x) {
            scol[i] = gcol[i];
            sw[i] = gw[i];
        }
    }
    bool ovf = false;
    if (threadIdx.x == 0) s_changed[0] = s_changed[1] = s_changed[2] = 0;
    __syncthreads();
    for (uint32_t round = 0; round < k; ++round) {
        const uint32_t slot_r = round % 3;
        if (threadIdx.x == 0) s_changed[(round + 1) % 3] = 0;
        bool changed = false;
        for (uint32_t v = warp; v < k; v += nwarps) {
            const uint32_t beg = kCsrInSmem ? soff[v] : (uint32_t)goff[v];
            const uint32_t end = kCsrInSmem ? soff[v + 1] : (uint32_t)goff[v + 1];
            uint32_t best = INF;
            for (uint32_t j = beg + slot; j < end; j += kSlots) {
                const uint32_t u = kCsrInSmem ? scol[j] : gcol[j];
                const uint32_t wj = kCsrInSmem ? sw[j] : gw[j];
                const uint32_t du = dist[u * S + my_s];
                if (du != INF) {
                    const uint64_t nd = (uint64_t)du + wj;
                    if (nd >= INF) ovf = true;
                    else best = min(best, (uint32_t)nd);
                }
            }
#pragma unroll
            for (uint32_t o = S; o < 32; o <<= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
            if (lane < S && best < dist[v * S + lane]) {
                dist[v * S + lane] = best;
                changed = true;
            }
        }
        if (__any_sync(0xffffffffu, changed) && lane == 0) s_changed[slot_r] = 1;
        __syncthreads();
        if (!s_changed[slot_r]) break;
    }
    uint32_t best = 0;
    for (uint32_t i = threadIdx.x; i < k * S; i += blockDim.x)
        if (s0 + i % S < k && dist[i] != INF && dist[i] > best) best = dist[i];
    best = block_reduce(best, [](uint32_t a, uint32_t b) { return a > b ? a : b; }, 0u);
    if (threadIdx.x == 0) atomicMax(out_max, best);
    if (__any_sync(0xffffffffu, ovf) && lane == 0) atomicExch(ovf_flag, 1u);
}

template <int S>
cldiam_status launch_msbf(uint32_t k, const uint64_t* off, const uint32_t* col, const uint32_t* w, uint64_t nnz,
                          cudaStream_t s, uint32_t* out_max, uint32_t* ovf) {
    constexpr int kMax = 220 * 1024;
    static std::atomic<bool> attr[64];  // first call per device sets the attribute (idempotent)
    int dev = 0;
    CLD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        CLD_CUDA(cudaFuncSetAttribute(k_apsp_msbf<S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax));
        CLD_CUDA(cudaFuncSetAttribute(k_apsp_msbf<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax));
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    const size_t dist_bytes = (size_t)k * S * 4;
    const size_t csr_bytes = ((size_t)k + 1 + 2 * nnz) * 4;
    const unsigned grid = (k + S - 1) / S;
    if (dist_bytes + csr_bytes <= (size_t)kMax) {
        CLD_K(K_FW, s, k_apsp_msbf<S, true><<<grid, 1024, dist_bytes + csr_bytes, s>>>(off, col, w, k, (uint32_t)nnz,
                                                                                     out_max, ovf));
    } else {
        CLD_K(K_FW, s, k_apsp_msbf<S, false><<<grid, 1024, dist_bytes, s>>>(off, col, w, k, (uint32_t)nnz, out_max, ovf));
    }
    CLD_LAUNCH_CHECK();
    return CLDIAM_OK;
}

// Batched exact SSSP on the quotient with a worklist (multi-source Bellman-Ford
// that only pushes from changed nodes): a CTA owns S consecutive sources and
// keeps dist[v][s] for all k nodes in shared memory, plus one word of change
// bits per node (bit s: dist[v][s] decreased).  In each round one warp per
// node v with change bits pushes dist[v][s] + w(v, u) to every neighbour u
// (lanes = neighbours) with a shared-memory atomicMin for each changed
// source s, and marks u for the next round when that lowers dist[u][s].
// Distances only ever decrease and stay lengths of real paths, so when no
// node is marked they are exact; the work is the number of distance
// decreases times the degree, instead of rounds x entries, which wins on
// quotients with many rounds (high hop diameter).
template <int S, bool kCsrInSmem>
__global__ void __launch_bounds__(1024) k_apsp_wl(const uint64_t* __restrict__ goff, const uint32_t* __restrict__ gcol,
                                                  const uint32_t* __restrict__ gw, uint32_t k, uint32_t nnz,
                                                  uint32_t* __restrict__ out_max, uint32_t* __restrict__ ovf_flag,
                                                  uint32_t* __restrict__ err) {
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t* dist = sm;                   // k x S
    uint32_t* chg0 = sm + (size_t)k * S;   // change bits, two rounds
    uint32_t* chg1 = chg0 + k;
    uint32_t* soff = chg1 + k;
    uint32_t* scol = soff + (k + 1);
    uint32_t* sw = scol + nnz;
    const uint32_t s0 = blockIdx.x * S;
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id(), nwarps = blockDim.x >> 5;
    for (uint32_t i = threadIdx.x; i < k * S; i += blockDim.x) {
        const uint32_t v = i / S, s = i % S;
        dist[i] = (s0 + s == v) ? 0u : INF;
    }
    for (uint32_t v = threadIdx.x; v < k; v += blockDim.x) {
        chg0[v] = (v >= s0 && v < s0 + S) ? 1u << (v - s0) : 0u;
        chg1[v] = 0;
    }
    if (kCsrInSmem) {
        for (uint32_t i = threadIdx.x; i <= k; i += blockDim.x) soff[i] = (uint32_t)goff[i];
        for (uint32_t i = threadIdx.x; i < nnz; i += blockDim.x) {
            scol[i] = gcol[i];
            sw[i] = gw[i];
        }
    }
    bool ovf = false;
    __syncthreads();
    const uint32_t max_rounds = 4 * k + 64;  // far above any real count: a guard, reported as an error
    uint32_t round = 0;
    for (;; ++round) {
        uint32_t* cur = (round & 1) ? chg1 : chg0;
        uint32_t* nxt = (round & 1) ? chg0 : chg1;
        for (uint32_t v = warp; v < k; v += nwarps) {
            const uint32_t bits = cur[v];
            if (!bits) continue;
            const uint32_t beg = kCsrInSmem ? soff[v] : (uint32_t)goff[v];
            const uint32_t end = kCsrInSmem ? soff[v + 1] : (uint32_t)goff[v + 1];
            for (uint32_t j = beg + lane; j < end; j += 32) {
                const uint32_t u = kCsrInSmem ? scol[j] : gcol[j];
                const uint32_t wj = kCsrInSmem ? sw[j] : gw[j];
                for (uint32_t b = bits; b; b &= b - 1) {
                    const uint32_t sidx = (uint32_t)__ffs(b) - 1;
                    const uint32_t dv = dist[v * S + sidx];
                    if (dv == INF) continue;
                    const uint64_t nd = (uint64_t)dv + wj;
                    if (nd >= INF) {
                        ovf = true;
                        continue;
                    }
                    uint32_t* du = &dist[u * S + sidx];
                    if ((uint32_t)nd < *du && (uint32_t)nd < atomicMin(du, (uint32_t)nd))
                        atomicOr(&nxt[u], 1u << sidx);
                }
            }
        }
        __syncthreads();
        bool any = false;
        for (uint32_t v = threadIdx.x; v < k; v += blockDim.x) {
            cur[v] = 0;
            any |= nxt[v] != 0;
        }
        if (!__syncthreads_or(any)) break;
        if (round >= max_rounds) {
            if (threadIdx.x == 0) atomicExch(err, 1u);
            break;
        }
    }
    uint32_t best = 0;
    for (uint32_t i = threadIdx.x; i < k * S; i += blockDim.x)
        if (s0 + i % S < k && dist[i] != INF && dist[i] > best) best = dist[i];
    best = block_reduce(best, [](uint32_t a, uint32_t b) { return a > b ? a : b; }, 0u);
    if (threadIdx.x == 0) atomicMax(out_max, best);
    if (__any_sync(0xffffffffu, ovf) && lane == 0) atomicExch(ovf_flag, 1u);
}

template <int S>
cldiam_status launch_wl(uint32_t k, const uint64_t* off, const uint32_t* col, const uint32_t* w, uint64_t nnz,
                        cudaStream_t s, uint32_t* out_max, uint32_t* ovf, uint32_t* err) {
    constexpr int kMax = 220 * 1024;
    static std::atomic<bool> attr[64];  // first call per device sets the attribute (idempotent)
    int dev = 0;
    CLD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        CLD_CUDA(cudaFuncSetAttribute(k_apsp_wl<S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax));
        CLD_CUDA(cudaFuncSetAttribute(k_apsp_wl<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax));
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    const size_t dist_bytes = (size_t)k * S * 4 + (size_t)k * 8;
    const size_t csr_bytes = ((size_t)k + 1 + 2 * nnz) * 4;
    const unsigned grid = (k + S - 1) / S;
    if (dist_bytes + csr_bytes <= (size_t)kMax) {
        CLD_K(K_FW, s, k_apsp_wl<S, true><<<grid, 1024, dist_bytes + csr_bytes, s>>>(off, col, w, k, (uint32_t)nnz,
                                                                                   out_max, ovf, err));
    } else {
        CLD_K(K_FW, s, k_apsp_wl<S, false><<<grid, 1024, dist_bytes, s>>>(off, col, w, k, (uint32_t)nnz, out_max, ovf,
                                                                          err));
    }
    CLD_LAUNCH_CHECK();
    return CLDIAM_OK;
}

// Blocked Floyd-Warshall over the padded kp x kp matrix M in the given form; scal[0] = overflow
// (checked form), scal[1] = largest finite distance, scal[3] = wide weight, scal[4] = unconnected pair.
template <bool FAST>
cldiam_status fw_dense(uint32_t* M, uint32_t kp, uint32_t k, uint32_t nt, const uint64_t* off, const uint32_t* col,
                       const uint32_t* w, uint32_t* scal, cudaStream_t s) {
    const uint32_t none = FAST ? INFF : INF;
    CLD_K(K_FW, s, k_fw_init<<<grid_for((size_t)kp * kp, 256), 256, 0, s>>>(M, kp, k, none));
    CLD_K(K_FW, s, k_fw_scatter<<<grid_for(k, 1, 64), 128, 0, s>>>(off, col, w, k, kp, M, FAST ? scal + 3 : nullptr));
    CLD_LAUNCH_CHECK();
    for (uint32_t r = 0; r < nt; ++r) {
        CLD_K(K_FW, s, k_fw_phase1<FAST><<<1, FTH, 0, s>>>(M, kp, r, scal));
        if (nt > 1) {
            CLD_K(K_FW, s, k_fw_phase2<FAST><<<dim3(nt - 1, 2), FTH, 0, s>>>(M, kp, r, scal));
            CLD_K(K_FW, s, k_fw_phase3<FAST><<<dim3(nt - 1, nt - 1), FTH, 0, s>>>(M, kp, r, scal));
        }
        CLD_LAUNCH_CHECK();
    }
    CLD_K(K_FW, s, k_fw_max_finite<<<grid_for((size_t)k * kp, 256), 256, 0, s>>>(M, kp, k, none, scal + 1,
                                                                                  FAST ? scal + 4 : nullptr));
    CLD_LAUNCH_CHECK();
    // algorithmic work: k^3 relaxations; bytes: the matrix read and written once per pivot round
    prof_add_bytes(K_FW, 2.0 * 4.0 * (double)kp * kp * nt);
    return CLDIAM_OK;
}

// Batched-SSSP kernel for a sparse quotient of k nodes: the worklist form with S sources per CTA while
// k x S distances and a word of change bits per node fit in shared memory (S = 8 below 2,048 nodes,
// else 4, else 1; a requested S that fits is taken), else all-node rounds with the distances alone
// (k <= 56,320), else none (dense form).
enum class SparsePlan { kNone, kWorklist8, kWorklist4, kWorklist1, kRounds1 };
SparsePlan sparse_plan(uint32_t k, uint32_t S) {
    constexpr size_t kSmem = 220 * 1024;
    const bool fit8 = (size_t)k * (8 * 4 + 8) <= kSmem, fit4 = (size_t)k * (4 * 4 + 8) <= kSmem,
               fit1 = (size_t)k * (4 + 8) <= kSmem;
    if ((S == 8 && fit8) || (S == 0 && fit8 && k < 2048)) return SparsePlan::kWorklist8;
    if ((S == 4 || S == 0 || S == 8) && fit4) return SparsePlan::kWorklist4;
    if (fit1) return SparsePlan::kWorklist1;
    if ((size_t)k * 4 <= kSmem) return SparsePlan::kRounds1;
    return SparsePlan::kNone;
}

}  // namespace

cldiam_status apsp_max_device(uint32_t k, const uint64_t* off, const uint32_t* col, const uint32_t* w, uint64_t nnz,
                              cudaStream_t s, uint64_t* phi, bool validate, uint32_t max_fw_k,
                              const cldiam_tuning& tun) {
    *phi = 0;
    if (k <= 1) return CLDIAM_OK;
    const uint32_t nt = (k + FT - 1) / FT;
    const uint32_t kp = nt * FT;
    DBuf<uint32_t> M, scal;
    CLD_TRY(scal.alloc(6, s));
    CLD_CUDA(cudaMemsetAsync(scal.get(), 0, 24, s));
    if (validate) {
        CLD_K(K_FW, s, k_fw_validate<<<grid_for((size_t)k + nnz + 1, 256), 256, 0, s>>>(off, col, k, nnz, scal.get() + 2));
        CLD_LAUNCH_CHECK();
        uint32_t bad = 0;
        CLD_CUDA(cudaMemcpyAsync(&bad, scal.get() + 2, 4, cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        if (bad) return fail(CLDIAM_ERR_INVALID_ARG, "malformed CSR (offsets or column ids)");
    }
    // sparse quotient (fewer than k^2 / 8 entries): batched SSSP, S sources per CTA with
    // k x S distances (and one word of change bits per node) in shared memory.  S = 8 below 2,048
    // nodes; above, S = 4: its half-size distance block lets two 1,024-thread CTAs share an SM (they
    // use <= 32 registers), where S = 8 fits one (R-MAT 24, k = 4,069: 3.0 -> 2.1 ms; road mesh 4096^2,
    // k = 4,357: 4.0 -> 3.4 ms)
    // (tuning: the density cut-over and the sources per CTA; a tuned cut-over never sends a quotient above
    // max_fw_k to Floyd-Warshall that the default would have solved by SSSP)
    bool sparse = (double)nnz * (double)tun.apsp_fw_density < (double)k * k;
    if (!sparse && k > max_fw_k) sparse = (double)nnz * 8.0 < (double)k * k;
    const SparsePlan plan = sparse ? sparse_plan(k, tun.apsp_sources_per_cta) : SparsePlan::kNone;
    if (plan == SparsePlan::kWorklist8) {
        CLD_TRY(launch_wl<8>(k, off, col, w, nnz, s, scal.get() + 1, scal.get(), scal.get() + 5));
    } else if (plan == SparsePlan::kWorklist4) {
        CLD_TRY(launch_wl<4>(k, off, col, w, nnz, s, scal.get() + 1, scal.get(), scal.get() + 5));
    } else if (plan == SparsePlan::kWorklist1) {
        CLD_TRY(launch_wl<1>(k, off, col, w, nnz, s, scal.get() + 1, scal.get(), scal.get() + 5));
    } else if (plan == SparsePlan::kRounds1) {
        CLD_TRY(launch_msbf<1>(k, off, col, w, nnz, s, scal.get() + 1, scal.get()));
    } else {
        if (k > max_fw_k) return fail(CLDIAM_ERR_UNSUPPORTED, "dense quotient larger than max_fw_k");
        CLD_TRY(M.alloc((size_t)kp * kp, s));
        // fast form first (scal[3] = a weight too wide for it, scal[4] = some pair left unconnected)
        CLD_TRY(fw_dense<true>(M.get(), kp, k, nt, off, col, w, scal.get(), s));
        uint32_t hf[5];
        CLD_CUDA(cudaMemcpyAsync(hf, scal.get(), 20, cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        if (hf[3] || hf[4]) {
            // disconnected pairs, or distances the fast form cannot hold: recompute with the checked form
            CLD_CUDA(cudaMemsetAsync(scal.get(), 0, 8, s));
            CLD_TRY(fw_dense<false>(M.get(), kp, k, nt, off, col, w, scal.get(), s));
        }
    }
    uint32_t h[6];
    CLD_CUDA(cudaMemcpyAsync(h, scal.get(), 24, cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    if (h[5]) return fail(CLDIAM_ERR_DIVERGED, "quotient SSSP exceeded its round limit");
    if (h[0]) return fail(CLDIAM_ERR_OVERFLOW, "a quotient distance reached 2^32 - 1");
    *phi = h[1];
    return CLDIAM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the quotient diameter, for callers that may not
// allocate device memory.  All scratch lives in one file-scope device array:
// three control words (overflow, result, validation) and, for dense inputs,
// the Floyd-Warshall matrix of up to kNoAllocMaxK x kNoAllocMaxK entries.  The
// array exists once per GPU that loads the library and stays resident until
// the process exits; every call reuses it, so calls whose work overlaps on the
// GPU race on it.
constexpr uint32_t kNoAllocMaxK = 1024;    // dense (Floyd-Warshall) inputs
constexpr uint32_t kNoAllocMaxSparseK = 51200;  // sparse inputs: distances live in shared memory
constexpr size_t kNoAllocCtlWords = 64;    // keeps the matrix 256-byte aligned
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocCtlWords + (size_t)kNoAllocMaxK * kNoAllocMaxK];

static std::mutex g_noalloc_mu;
static uint32_t* g_noalloc_ptr[64];  // device address of the scratch array, per device

cldiam_status apsp_max_noalloc(uint32_t k, const uint64_t* off, const uint32_t* col, const uint32_t* w,
                               cudaStream_t s, uint64_t* phi) {
    *phi = 0;
    int dev = 0;
    CLD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CLDIAM_ERR_UNSUPPORTED, "device ordinal above 63");
    uint32_t* scratch = nullptr;
    {
        // one-time set-up per device, with that device current: the host-side name of the
        // array is not a device address, so ask the runtime for it
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
            g_noalloc_ptr[dev] = static_cast<uint32_t*>(p);
        }
        scratch = g_noalloc_ptr[dev];
    }
    if (k <= 1) return CLDIAM_OK;
    if (!is_device_ptr(off) || !is_device_ptr(col) || !is_device_ptr(w))
        return fail(CLDIAM_ERR_INVALID_ARG, "off, col and w must be device memory (nothing is copied or allocated)");
    uint64_t nnz = 0;
    CLD_CUDA(cudaMemcpyAsync(&nnz, off + k, 8, cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    if (nnz > 0xFFFFFFFFull) return fail(CLDIAM_ERR_INVALID_ARG, "more than 2^32 - 1 entries");
    const bool sparse = (double)nnz * 8.0 < (double)k * k;
    if (sparse ? k > kNoAllocMaxSparseK : k > kNoAllocMaxK)
        return fail(CLDIAM_ERR_UNSUPPORTED, sparse ? "k above 51200, the allocation-free limit for sparse graphs"
                                                   : "k above 1024, the allocation-free limit for dense graphs");
    uint32_t* ovf = scratch + 0;
    uint32_t* best = scratch + 1;
    uint32_t* bad = scratch + 2;
    uint32_t* diverged = scratch + 3;  // the worklist SSSP's round limit
    CLD_CUDA(cudaMemsetAsync(scratch, 0, 4 * sizeof(uint32_t), s));  // the array keeps the last call's values
    k_fw_validate<<<grid_for((size_t)k + nnz + 1, 256), 256, 0, s>>>(off, col, k, nnz, bad);
    CLD_LAUNCH_CHECK();
    uint32_t h[3] = {0, 0, 0};
    CLD_CUDA(cudaMemcpyAsync(h, scratch, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    if (h[2]) return fail(CLDIAM_ERR_INVALID_ARG, "malformed CSR (offsets or column ids)");
    if (sparse) {
        // batched SSSP with the kernel and sources per CTA apsp_max_device takes by default: distances,
        // change bits (and the CSR when it fits) in shared memory, only the control words here
        switch (sparse_plan(k, 0)) {
            case SparsePlan::kWorklist8: CLD_TRY(launch_wl<8>(k, off, col, w, nnz, s, best, ovf, diverged)); break;
            case SparsePlan::kWorklist4: CLD_TRY(launch_wl<4>(k, off, col, w, nnz, s, best, ovf, diverged)); break;
            case SparsePlan::kWorklist1: CLD_TRY(launch_wl<1>(k, off, col, w, nnz, s, best, ovf, diverged)); break;
            default: CLD_TRY(launch_msbf<1>(k, off, col, w, nnz, s, best, ovf)); break;
        }
    } else {
        const uint32_t nt = (k + FT - 1) / FT;
        const uint32_t kp = nt * FT;  // <= kNoAllocMaxK
        uint32_t* M = scratch + kNoAllocCtlWords;
        k_fw_init<<<grid_for((size_t)kp * kp, 256), 256, 0, s>>>(M, kp, k, INF);
        k_fw_scatter<<<grid_for(k, 1, 64), 128, 0, s>>>(off, col, w, k, kp, M, nullptr);
        CLD_LAUNCH_CHECK();
        for (uint32_t r = 0; r < nt; ++r) {
            k_fw_phase1<false><<<1, FTH, 0, s>>>(M, kp, r, ovf);
            if (nt > 1) {
                k_fw_phase2<false><<<dim3(nt - 1, 2), FTH, 0, s>>>(M, kp, r, ovf);
                k_fw_phase3<false><<<dim3(nt - 1, nt - 1), FTH, 0, s>>>(M, kp, r, ovf);
            }
            CLD_LAUNCH_CHECK();
        }
        k_fw_max_finite<<<grid_for((size_t)k * kp, 256), 256, 0, s>>>(M, kp, k, INF, best, nullptr);
        CLD_LAUNCH_CHECK();
    }
    uint32_t hd[4] = {0, 0, 0, 0};
    CLD_CUDA(cudaMemcpyAsync(hd, scratch, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    if (hd[3]) return fail(CLDIAM_ERR_DIVERGED, "quotient SSSP exceeded its round limit");
    if (hd[0]) return fail(CLDIAM_ERR_OVERFLOW, "a distance reached 2^32 - 1");
    *phi = hd[1];
    return CLDIAM_OK;
}

}  // namespace cld
