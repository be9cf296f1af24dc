// Device-wide primitives: prefix sums, reductions and a stable LSD radix sort
// (8-bit digits, warp match-based ranking).  These realise the sorting and
// (segmented) prefix-sum building blocks that the paper's MR implementation
// relies on (Fact 1, Section 2), here within one GPU.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "common.cuh"
#include "prof.cuh"

namespace cld {

// ------------------------------------------------------------------ status
static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error_cstr() { return g_last_error.c_str(); }

cldiam_status fail(cldiam_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

cldiam_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    g_last_error = buf;
    if (e == cudaErrorMemoryAllocation) return CLDIAM_ERR_OOM;
    return CLDIAM_ERR_CUDA;
}

// ------------------------------------------------------------------ memory
static std::mutex g_pool_mu;
static bool g_pool_tuned[64];

cldiam_status dmalloc(void** p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    CLD_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !g_pool_tuned[dev]) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pool_tuned[dev]) {
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t thr = ~0ull;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
            g_pool_tuned[dev] = true;
        }
    }
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char buf[160];
        snprintf(buf, sizeof buf, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return fail(CLDIAM_ERR_OOM, buf);
    }
    return CLDIAM_OK;
}

void dfree(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

cldiam_status Pinned::alloc(size_t bytes) {
    if (h) return CLDIAM_OK;
    CLD_CUDA(cudaMallocHost(&h, bytes));
    memset(h, 0, bytes);
    return CLDIAM_OK;
}

int num_sms() {
    static int cached[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    if (cached[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 152;
    }
    return cached[dev];
}

// ------------------------------------------------------------------ scan
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_reduce(const T* __restrict__ in, size_t n, T* __restrict__ partial) {
    size_t base = (size_t)blockIdx.x * SCAN_TILE;
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        size_t idx = base + (size_t)i * SCAN_THREADS + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    s = block_reduce(s, [](T a, T b) { return a + b; }, (T)0);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <class T>
__global__ void __launch_bounds__(SCAN_THREADS)
    k_tile_scan(const T* __restrict__ in, T* __restrict__ out, size_t n, const T* __restrict__ offsets,
                T* __restrict__ total) {
    size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_ITEMS;
    T x[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        size_t idx = base + i;
        x[i] = (idx < n) ? in[idx] : (T)0;
        s += x[i];
    }
    // block exclusive scan over thread sums (explicit, avoids slot aliasing)
    __shared__ T wsum[33];
    T incl = warp_incl_scan(s);
    unsigned w = threadIdx.x >> 5, l = lane_id();
    if (l == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        T v = wsum[l];
        T vi = warp_incl_scan(v);
        wsum[l] = vi - v;
        if (l == 31) wsum[32] = vi;
    }
    __syncthreads();
    T off = (offsets ? offsets[blockIdx.x] : (T)0) + wsum[w] + incl - s;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        size_t idx = base + i;
        if (idx < n) out[idx] = off;
        off += x[i];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        *total = (offsets ? offsets[blockIdx.x] : (T)0) + wsum[32];
}

template <class T>
static cldiam_status scan_exclusive(const T* in, T* out, size_t n, T* total, cudaStream_t s) {
    if (n == 0) {
        if (total) CLD_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
        return CLDIAM_OK;
    }
    size_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        CLD_K(K_SCAN, s, k_tile_scan<T><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr, total));
        CLD_LAUNCH_CHECK();
        return CLDIAM_OK;
    }
    DBuf<T> part, part_scan;
    CLD_TRY(part.alloc(nb, s));
    CLD_TRY(part_scan.alloc(nb, s));
    CLD_K(K_SCAN, s, k_tile_reduce<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, part.get()));
    CLD_LAUNCH_CHECK();
    CLD_TRY(scan_exclusive<T>(part.get(), part_scan.get(), nb, nullptr, s));
    CLD_K(K_SCAN, s, k_tile_scan<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, part_scan.get(), total));
    CLD_LAUNCH_CHECK();
    return CLDIAM_OK;
}

cldiam_status scan_exclusive_u32(const uint32_t* in, uint32_t* out, size_t n, uint32_t* total, cudaStream_t s) {
    return scan_exclusive<uint32_t>(in, out, n, total, s);
}
cldiam_status scan_exclusive_u64(const uint64_t* in, uint64_t* out, size_t n, uint64_t* total, cudaStream_t s) {
    return scan_exclusive<uint64_t>(in, out, n, total, s);
}

// ------------------------------------------------------------------ reductions
__global__ void k_reduce_max_u32(const uint32_t* __restrict__ in, size_t n, uint32_t* out) {
    uint32_t m = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = max(m, in[i]);
    m = block_reduce(m, [](uint32_t a, uint32_t b) { return a > b ? a : b; }, 0u);
    if (threadIdx.x == 0) atomicMax(out, m);
}
__global__ void k_reduce_min_u32(const uint32_t* __restrict__ in, size_t n, uint32_t* out) {
    uint32_t m = 0xFFFFFFFFu;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = min(m, in[i]);
    m = block_reduce(m, [](uint32_t a, uint32_t b) { return a < b ? a : b; }, 0xFFFFFFFFu);
    if (threadIdx.x == 0) atomicMin(out, m);
}
__global__ void k_reduce_sum_u32(const uint32_t* __restrict__ in, size_t n, unsigned long long* out) {
    unsigned long long m = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m += in[i];
    m = block_reduce(m, [](unsigned long long a, unsigned long long b) { return a + b; }, 0ull);
    if (threadIdx.x == 0) atomicAdd(out, m);
}

cldiam_status reduce_max_u32(const uint32_t* in, size_t n, uint32_t* out, cudaStream_t s) {
    CLD_CUDA(cudaMemsetAsync(out, 0, sizeof(uint32_t), s));
    if (n == 0) return CLDIAM_OK;
    CLD_K(K_REDUCE, s, k_reduce_max_u32<<<grid_for(n, 256, 4), 256, 0, s>>>(in, n, out));
    CLD_LAUNCH_CHECK();
    return CLDIAM_OK;
}
cldiam_status reduce_min_u32(const uint32_t* in, size_t n, uint32_t* out, cudaStream_t s) {
    CLD_CUDA(cudaMemsetAsync(out, 0xFF, sizeof(uint32_t), s));
    if (n == 0) return CLDIAM_OK;
    CLD_K(K_REDUCE, s, k_reduce_min_u32<<<grid_for(n, 256, 4), 256, 0, s>>>(in, n, out));
    CLD_LAUNCH_CHECK();
    return CLDIAM_OK;
}
cldiam_status reduce_sum_u32_to_u64(const uint32_t* in, size_t n, uint64_t* out, cudaStream_t s) {
    CLD_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), s));
    if (n == 0) return CLDIAM_OK;
    CLD_K(K_REDUCE, s, k_reduce_sum_u32<<<grid_for(n, 256, 4), 256, 0, s>>>(in, n, reinterpret_cast<unsigned long long*>(out)));
    CLD_LAUNCH_CHECK();
    return CLDIAM_OK;
}

// ------------------------------------------------------------------ radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;                       // items per thread
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;    // 2048 items per tile
constexpr int RS_RADIX = 256;

// item (warp w, iteration i, lane l) of a tile sits at w*256 + i*32 + l, so
// every warp load is 32 consecutive keys.
template <class K>
__global__ void __launch_bounds__(RS_THREADS)
    k_radix_hist(const K* __restrict__ keys, size_t n, int shift, uint32_t* __restrict__ hist, uint32_t ntiles) {
    __shared__ uint32_t h[RS_RADIX];
    for (int i = threadIdx.x; i < RS_RADIX; i += RS_THREADS) h[i] = 0;
    __syncthreads();
    const uint32_t tile = blockIdx.x;
    const unsigned w = threadIdx.x >> 5, l = lane_id();
    size_t base = (size_t)tile * RS_TILE + (size_t)w * (RS_ITEMS * 32);
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        size_t idx = base + (size_t)i * 32 + l;
        bool valid = idx < n;
        uint32_t d = valid ? (uint32_t)((keys[idx] >> shift) & 0xFF) : 0x100u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && l == (unsigned)(__ffs(peers) - 1)) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_RADIX; d += RS_THREADS) hist[(size_t)d * ntiles + tile] = h[d];
}

template <class K>
__global__ void __launch_bounds__(RS_THREADS)
    k_radix_scatter(const K* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, K* __restrict__ keys_out,
                    uint32_t* __restrict__ vals_out, size_t n, int shift, const uint32_t* __restrict__ offs,
                    uint32_t ntiles) {
    __shared__ uint32_t whist[RS_WARPS][RS_RADIX];
    __shared__ uint32_t gbase[RS_RADIX];
    for (int i = threadIdx.x; i < RS_WARPS * RS_RADIX; i += RS_THREADS) (&whist[0][0])[i] = 0;
    const uint32_t tile = blockIdx.x;
    for (int d = threadIdx.x; d < RS_RADIX; d += RS_THREADS) gbase[d] = offs[(size_t)d * ntiles + tile];
    __syncthreads();
    const unsigned w = threadIdx.x >> 5, l = lane_id();
    const unsigned ltmask = lanemask_lt();
    size_t base = (size_t)tile * RS_TILE + (size_t)w * (RS_ITEMS * 32);
    K key[RS_ITEMS];
    uint32_t val[RS_ITEMS];
    uint32_t dig[RS_ITEMS];
    uint32_t rank[RS_ITEMS];
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        size_t idx = base + (size_t)i * 32 + l;
        bool valid = idx < n;
        key[i] = valid ? keys_in[idx] : (K)0;
        val[i] = valid ? vals_in[idx] : 0u;
        uint32_t d = valid ? (uint32_t)((key[i] >> shift) & 0xFF) : 0x100u;
        dig[i] = d;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned leader = __ffs(peers) - 1;
        uint32_t b = 0;
        if (valid && l == leader) {
            b = whist[w][d];
            whist[w][d] = b + (uint32_t)__popc(peers);
        }
        b = __shfl_sync(0xffffffffu, b, leader);
        rank[i] = b + (uint32_t)__popc(peers & ltmask);
        __syncwarp();
    }
    __syncthreads();
    // exclusive scan over warps, per digit
    for (int d = threadIdx.x; d < RS_RADIX; d += RS_THREADS) {
        uint32_t s = 0;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) {
            uint32_t t = whist[ww][d];
            whist[ww][d] = s;
            s += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        if (dig[i] < 0x100u) {
            uint32_t pos = gbase[dig[i]] + whist[w][dig[i]] + rank[i];
            keys_out[pos] = key[i];
            vals_out[pos] = val[i];
        }
    }
}

template <class K>
static cldiam_status radix_sort_pairs(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, size_t n,
                                      int bits, bool* in_alt, cudaStream_t s) {
    *in_alt = false;
    if (n <= 1 || bits <= 0) return CLDIAM_OK;
    if (n > 0xFFFFFFFFull) return fail(CLDIAM_ERR_UNSUPPORTED, "radix sort limited to 2^32 - 1 items");
    uint32_t ntiles = (uint32_t)((n + RS_TILE - 1) / RS_TILE);
    DBuf<uint32_t> hist;
    CLD_TRY(hist.alloc((size_t)RS_RADIX * ntiles, s));
    K* ki = keys;
    uint32_t* vi = vals;
    K* ko = keys_alt;
    uint32_t* vo = vals_alt;
    bool alt = false;
    for (int shift = 0; shift < bits; shift += 8) {
        CLD_K(K_RADIX_HIST, s, k_radix_hist<K><<<ntiles, RS_THREADS, 0, s>>>(ki, n, shift, hist.get(), ntiles));
        CLD_LAUNCH_CHECK();
        CLD_TRY(scan_exclusive_u32(hist.get(), hist.get(), (size_t)RS_RADIX * ntiles, nullptr, s));
        CLD_K(K_RADIX_SCATTER, s, k_radix_scatter<K><<<ntiles, RS_THREADS, 0, s>>>(ki, vi, ko, vo, n, shift, hist.get(), ntiles));
        CLD_LAUNCH_CHECK();
        // algorithmic bytes: histogram reads every key; scatter reads and writes every (key, value)
        prof_add_bytes(K_RADIX_HIST, (double)n * sizeof(K));
        prof_add_bytes(K_RADIX_SCATTER, 2.0 * (double)n * (sizeof(K) + sizeof(uint32_t)));
        K* tk = ki; ki = ko; ko = tk;
        uint32_t* tv = vi; vi = vo; vo = tv;
        alt = !alt;
    }
    *in_alt = alt;
    return CLDIAM_OK;
}

cldiam_status radix_sort_pairs_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                                   size_t n, int bits, bool* in_alt, cudaStream_t s) {
    return radix_sort_pairs<uint64_t>(keys, vals, keys_alt, vals_alt, n, bits, in_alt, s);
}
cldiam_status radix_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                                   size_t n, int bits, bool* in_alt, cudaStream_t s) {
    return radix_sort_pairs<uint32_t>(keys, vals, keys_alt, vals_alt, n, bits, in_alt, s);
}

}  // namespace cld
