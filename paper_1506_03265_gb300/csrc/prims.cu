// Device-wide primitives: prefix sums, reductions and a stable LSD radix sort
// (8-bit digits, warp-level ranking from bit ballots).  These realise the sorting and
// (segmented) prefix-sum building blocks that the paper's MR implementation
// relies on (Fact 1, Section 2), here within one GPU.
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

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
static std::atomic<bool> g_pool_tuned[64];  // set under g_pool_mu, read without it

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

static std::mutex g_pin_mu;
static std::vector<void*> g_pin_free;

void* pinned_take() {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        constexpr size_t kSlab = 256 * kPinnedBlock;  // slabs are never unpinned
        void* slab = nullptr;
        if (cudaHostAlloc(&slab, kSlab, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (size_t i = kSlab / kPinnedBlock; i-- > 0;) g_pin_free.push_back(static_cast<char*>(slab) + i * kPinnedBlock);
    }
    void* p = g_pin_free.back();
    g_pin_free.pop_back();
    return p;
}

void pinned_give(void* p) {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

cldiam_status Pinned::alloc(size_t bytes) {
    if (h) return CLDIAM_OK;
    if (bytes <= kPinnedBlock) {
        h = pinned_take();
        if (!h) return fail(CLDIAM_ERR_OOM, "pinned host allocation failed");
        pooled = true;
    } else {
        CLD_CUDA(cudaMallocHost(&h, bytes));
    }
    memset(h, 0, bytes);
    return CLDIAM_OK;
}

int num_sms() {
    static std::atomic<int> cached[64];  // concurrent first calls store the same value
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    if (cached[dev].load() == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev].store(v > 0 ? v : 152);
    }
    return cached[dev].load();
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

// ------------------------------------------------------------------ offsets from sorted rows
__global__ void k_offsets_from_rows(const uint32_t* __restrict__ row, uint64_t nnz, uint32_t n,
                                    uint64_t* __restrict__ off) {
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= nnz; r += (uint64_t)gridDim.x * blockDim.x) {
        // entry r opens rows row[r-1]+1 .. row[r] (all rows up to row[0] when r = 0); position nnz
        // closes rows row[nnz-1]+1 .. n
        if (r > 0 && r < nnz && row[r] == row[r - 1]) continue;
        const uint64_t lo = (r == 0) ? 0 : (uint64_t)row[r - 1] + 1;
        const uint64_t hi = (r == nnz) ? n : (uint64_t)row[r];
        for (uint64_t x = lo; x <= hi; ++x) off[x] = r;
    }
}

cldiam_status offsets_from_rows(const uint32_t* row, uint64_t nnz, uint32_t n, uint64_t* off, cudaStream_t s) {
    CLD_K(K_CSR, s, k_offsets_from_rows<<<grid_for(nnz + 1, 256), 256, 0, s>>>(row, nnz, n, off));
    CLD_LAUNCH_CHECK();
    return CLDIAM_OK;
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
// Onesweep-style LSD radix sort (8-bit digits).  One read of the keys builds
// the digit histograms of every pass; each pass is then a single kernel in
// which tile t ranks its items (warp-level, stable), publishes its
// per-digit counts, and obtains the counts of all earlier tiles by decoupled
// look-back over a per-(tile, digit) status word, so no per-pass histogram
// read or separate scan is needed.  Items are staged in shared memory in
// digit order and written out as contiguous runs.
constexpr int OS_THREADS = 256;
constexpr int OS_WARPS = OS_THREADS / 32;
template <class K, bool KV>
struct OsCfg {  // items per thread: fewer for 64-bit (key, value) pairs to keep registers (and occupancy) in check
    static constexpr int ITEMS = (sizeof(K) == 8 && KV) ? 8 : 12;
    static constexpr int TILE = OS_THREADS * ITEMS;
};
constexpr int OS_RADIX = 256;
constexpr unsigned long long OS_AGG = 1ull << 32;   // status: tile's own count
constexpr unsigned long long OS_PRE = 2ull << 32;   // status: inclusive prefix over tiles 0..t
constexpr long long OS_WAIT_CYCLES = 4000000000ll;  // ~2 s at 2 GHz: a look-back that waits longer gives up

// Digit histograms of every pass from one read of the keys: one private histogram per warp and pass
// in shared memory (warps x npass x 256 words, dynamic), so shared atomics collide only within a warp.
template <class K>
__global__ void __launch_bounds__(256) k_os_hist(const K* __restrict__ keys, size_t n, int npass, int shift0, int bits,
                                                 uint32_t* __restrict__ hist) {
    extern __shared__ uint32_t hs[];
    const unsigned w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < OS_WARPS * npass * OS_RADIX; i += blockDim.x) hs[i] = 0;
    __syncthreads();
    uint32_t* h = hs + (size_t)w * npass * OS_RADIX;
    constexpr int U = 8;  // keys loaded per thread before counting, to keep loads in flight
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = (size_t)blockIdx.x * blockDim.x + threadIdx.x; base < n; base += stride * U) {
        K kk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t i = base + (size_t)u * stride;
            kk[u] = i < n ? keys[i] : (K)0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool valid = base + (size_t)u * stride < n;
            for (int p = 0; p < npass; ++p) {
                // the last digit holds only the key bits left (bits above the key are not sorted on)
                const uint32_t dm = bits - 8 * p >= 8 ? 0xFFu : ((1u << (bits - 8 * p)) - 1u);
                const uint32_t d = (uint32_t)(kk[u] >> (shift0 + 8 * p)) & dm;
                if (valid) atomicAdd(&h[p * OS_RADIX + d], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * OS_RADIX; i += blockDim.x) {
        uint32_t c = 0;
        for (int ww = 0; ww < OS_WARPS; ++ww) c += hs[(size_t)ww * npass * OS_RADIX + i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// exclusive scan of each pass's 256 digit counts (one block, 256 threads)
__global__ void k_os_hist_scan(uint32_t* __restrict__ hist, int npass) {
    __shared__ uint32_t wsum[OS_WARPS];
    const unsigned d = threadIdx.x, w = d >> 5, l = lane_id();
    for (int p = 0; p < npass; ++p) {
        uint32_t c = hist[p * OS_RADIX + d];
        uint32_t incl = warp_incl_scan(c);
        if (l == 31) wsum[w] = incl;
        __syncthreads();
        uint32_t off = 0;
        for (unsigned ww = 0; ww < w; ++ww) off += wsum[ww];
        hist[p * OS_RADIX + d] = off + incl - c;
        __syncthreads();
    }
}

// Digit (key >> shift) & dm (dm = 0xFF, or fewer bits in the last pass of a key whose width is not a
// multiple of 8).  For 64-bit keys HI says shift >= 32 (uniform per pass), so the digit comes from one
// 32-bit word, or from a funnel shift of the two when it may straddle them.
template <class K, bool HI>
__device__ __forceinline__ uint32_t os_digit(K k, uint32_t sh, uint32_t dm) {
    if constexpr (sizeof(K) == 8) {
        const uint32_t lo = (uint32_t)k, hi = (uint32_t)((uint64_t)k >> 32);
        if constexpr (HI) return (hi >> sh) & dm;
        else return __funnelshift_r(lo, hi, sh) & dm;
    } else {
        return ((uint32_t)k >> sh) & dm;
    }
}

// Narrows peers to the lanes whose digit bits B..7 equal this lane's.  plo holds digit bits 0..3 at the
// top bit of its bytes 0..3 (bit j at bit 8j + 7), phi bits 4..7 likewise, so a byte permute of the pair
// {phi, plo} whose selector nibbles are 8 + b (sign-replicate mode, source byte b) spreads digit bit b over
// the whole word m; the ballot of m != 0 is the lanes with bit b set, and m picks it or its complement.
template <int B>
__device__ __forceinline__ unsigned os_peers(uint32_t plo, uint32_t phi, unsigned peers) {
    uint32_t m;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(m) : "r"(plo), "r"(phi), "n"(0x1111 * (8 + B)));
    const unsigned bb = __ballot_sync(0xffffffffu, m != 0u);
    peers &= ~(bb ^ m);
    if constexpr (B < 7) return os_peers<B + 1>(plo, phi, peers);
    else return peers;
}

// Loads one tile's items, every load issued before ranking so they are in flight together, and ranks them.
// FULL: every thread holds all OS_ITEMS items, so the per-item bounds tests go (and with them the spills
// that the generic form needs at 64 registers).  Stable warp-local ranks: peers with the same digit,
// counted in item order then lane order; the peer mask is the AND of one ballot per digit bit (a fixed
// cost; a match instruction costs more the more distinct digits a warp holds, which is most of them for
// these keys); every peer reads the running count (one broadcast word) and writes back the same new count
// (in the last tile only the highest valid peer does).
template <class K, bool KV, bool HI, int OS_ITEMS, bool FULL>
__device__ __forceinline__ void os_load_rank(const K* __restrict__ kt, const uint32_t* __restrict__ vt, uint32_t rem,
                                             uint32_t lbase, unsigned l, unsigned ltmask, uint32_t sh, uint32_t dm,
                                             uint32_t* __restrict__ wh, K (&key)[OS_ITEMS],
                                             uint32_t (&val)[KV ? OS_ITEMS : 1],
                                             uint32_t (&rank_pk)[(OS_ITEMS + 1) / 2]) {
#pragma unroll
    for (int i = 0; i < OS_ITEMS; ++i) {
        const uint32_t li = lbase + (uint32_t)i * 32;
        if constexpr (FULL) {
            key[i] = kt[li];
            if constexpr (KV) val[i] = vt[li];
        } else {
            key[i] = li < rem ? kt[li] : (K)0;
            if constexpr (KV) val[i] = li < rem ? vt[li] : 0u;
        }
    }
#pragma unroll
    for (int i = 0; i < OS_ITEMS; ++i) {
        const bool valid = FULL || lbase + (uint32_t)i * 32 < rem;
        const uint32_t d = os_digit<K, HI>(key[i], sh, dm);
        unsigned peers = 0xFFFFFFFFu;
        if constexpr (!FULL) {  // the last tile: items past the end form their own group
            const unsigned vb = __ballot_sync(0xffffffffu, valid);
            peers = valid ? vb : ~vb;
        }
        peers = os_peers<0>((d & 0xFu) * 0x10204080u, (d & 0xF0u) * 0x01020408u, peers);
        const uint32_t cur = wh[d];
        __syncwarp();
        if constexpr (FULL) wh[d] = cur + (uint32_t)__popc(peers);  // every peer stores the same value
        else if (valid && (peers >> l) == 1u) wh[d] = cur + (uint32_t)__popc(peers);
        const uint32_t rk = valid ? cur + (uint32_t)__popc(peers & ltmask) : 0xFFFFu;
        if (i % 2 == 0) rank_pk[i / 2] = rk;
        else rank_pk[i / 2] |= rk << 16;
        __syncwarp();
    }
}

// KV: items carry a 32-bit value (vin/vout); otherwise keys only.  sh = shift mod 32 (HI: shift >= 32).
template <class K, bool KV, bool HI, int OS_ITEMS = OsCfg<K, KV>::ITEMS, int OS_TILE = OsCfg<K, KV>::TILE>
__global__ void __launch_bounds__(OS_THREADS, 4)
    k_os_pass(const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
              uint32_t* __restrict__ vout, size_t n, uint32_t sh, uint32_t dm, const uint32_t* __restrict__ goff,
              unsigned long long* __restrict__ status, uint32_t* __restrict__ tile_ctr, uint32_t* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char os_smem[];
    K* s_key = reinterpret_cast<K*>(os_smem);
    uint32_t* s_val = reinterpret_cast<uint32_t*>(os_smem + sizeof(K) * OS_TILE);
    // whist[w][d]: first the count of digit d among warp w's items, then the tile position of warp w's
    // first d item; gdiff[d]: output position of the tile's first d item minus its tile position
    __shared__ uint32_t whist[OS_WARPS][OS_RADIX];
    __shared__ uint32_t gdiff[OS_RADIX];
    __shared__ uint32_t wsum[OS_WARPS];
    __shared__ uint32_t s_tile;
    const unsigned tid = threadIdx.x, w = tid >> 5, l = lane_id();
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);  // tiles in start order: earlier tiles are running or done
    for (int i = tid; i < OS_WARPS * OS_RADIX; i += OS_THREADS) (&whist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const size_t tbase = (size_t)tile * OS_TILE;
    const uint32_t rem = (uint32_t)min((size_t)OS_TILE, n - tbase);  // items in this tile
    const K* kt = kin + tbase;
    const uint32_t* vt = KV ? vin + tbase : nullptr;
    const uint32_t lbase = w * (OS_ITEMS * 32) + l;  // tile position of this thread's item 0 (warp-striped)
    const unsigned ltmask = lanemask_lt();

    K key[OS_ITEMS];
    uint32_t val[KV ? OS_ITEMS : 1];
    uint32_t rank_pk[(OS_ITEMS + 1) / 2];  // warp-local ranks (< 32 * OS_ITEMS) as 16-bit halves; 0xFFFF = no item
    // full tiles (all but the last) take the form without bounds tests
    if (rem == (uint32_t)OS_TILE)
        os_load_rank<K, KV, HI, OS_ITEMS, true>(kt, vt, rem, lbase, l, ltmask, sh, dm, whist[w], key, val, rank_pk);
    else
        os_load_rank<K, KV, HI, OS_ITEMS, false>(kt, vt, rem, lbase, l, ltmask, sh, dm, whist[w], key, val, rank_pk);
    __syncthreads();

    // per digit (thread d): tile count, publication, tile-local scan, look-back
    const unsigned d = tid;
    const uint32_t g0 = goff[d];
    uint32_t cnt = 0;
#pragma unroll
    for (int ww = 0; ww < OS_WARPS; ++ww) cnt += whist[ww][d];
    volatile unsigned long long* vst = status;
    if (tile == 0) vst[d] = OS_PRE | cnt;
    else vst[(size_t)tile * OS_RADIX + d] = OS_AGG | cnt;
    uint32_t tst;
    {
        const uint32_t incl = warp_incl_scan(cnt);
        if (l == 31) wsum[w] = incl;
        __syncthreads();
        uint32_t off = 0;
        for (unsigned ww = 0; ww < w; ++ww) off += wsum[ww];
        tst = off + incl - cnt;
    }
    {
        uint32_t run = tst;  // only thread d touches column d of whist here
#pragma unroll
        for (int ww = 0; ww < OS_WARPS; ++ww) {
            const uint32_t cw = whist[ww][d];
            whist[ww][d] = run;
            run += cw;
        }
    }
    __syncthreads();
    // stage in digit order (tile positions suffice; digits recomputed from the keys); the keys are dead
    // before the look-back
#pragma unroll
    for (int i = 0; i < OS_ITEMS; ++i) {
        const uint32_t rk = (rank_pk[i / 2] >> (16 * (i % 2))) & 0xFFFFu;
        if (rem == (uint32_t)OS_TILE || rk != 0xFFFFu) {
            const uint32_t dd = os_digit<K, HI>(key[i], sh, dm);
            const uint32_t pos = whist[w][dd] + rk;
            s_key[pos] = key[i];
            if constexpr (KV) s_val[pos] = val[i];
        }
    }
    uint32_t excl = 0;
    if (tile > 0) {
        // windowed look-back: read the statuses of LB earlier tiles at once, add their counts
        // back to the first inclusive prefix; wait (bounded) only on a tile not yet published
        constexpr int LB = 8;
        const long long t0 = clock64();
        long long t = (long long)tile - 1;
        bool done = false, timed_out = false;
        while (!done && !timed_out) {
            unsigned long long sw[LB];
#pragma unroll
            for (int j = 0; j < LB; ++j)
                sw[j] = (t - j >= 0) ? (unsigned long long)vst[(size_t)(t - j) * OS_RADIX + d] : (unsigned long long)OS_PRE;
#pragma unroll
            for (int j = 0; j < LB; ++j) {
                if (done || timed_out) break;
                while ((sw[j] & ~0xFFFFFFFFull) == 0) {
                    if (clock64() - t0 > OS_WAIT_CYCLES) {
                        atomicExch(err, 1u);
                        timed_out = true;
                        break;
                    }
                    __nanosleep(32);
                    sw[j] = vst[(size_t)(t - j) * OS_RADIX + d];
                }
                excl += (uint32_t)sw[j];
                if ((sw[j] & ~0xFFFFFFFFull) == OS_PRE) done = true;
            }
            t -= LB;
        }
        vst[(size_t)tile * OS_RADIX + d] = OS_PRE | (excl + cnt);
    }
    gdiff[d] = g0 + excl - tst;  // modulo 2^32; positions are < 2^32
    __syncthreads();
    // write out: consecutive threads take consecutive staged items, i.e. runs of equal digits
    if (rem == (uint32_t)OS_TILE) {
#pragma unroll
        for (int j = 0; j < OS_ITEMS; ++j) {
            const uint32_t i = (uint32_t)j * OS_THREADS + tid;
            const K k = s_key[i];
            const uint32_t pos = gdiff[os_digit<K, HI>(k, sh, dm)] + i;
            kout[pos] = k;
            if constexpr (KV) vout[pos] = s_val[i];
        }
    } else {
        for (uint32_t i = tid; i < rem; i += OS_THREADS) {
            const K k = s_key[i];
            const uint32_t pos = gdiff[os_digit<K, HI>(k, sh, dm)] + i;
            kout[pos] = k;
            if constexpr (KV) vout[pos] = s_val[i];
        }
    }
}

// LSD sort of n items on key bits [shift0, shift0 + bits); vals == nullptr sorts keys only.
template <class K>
static cldiam_status radix_sort_impl(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, size_t n, int shift0,
                                     int bits, bool* in_alt, cudaStream_t s, uint32_t* err_dev = nullptr,
                                     const K* first_in = nullptr, uint32_t* hist_in = nullptr) {
    *in_alt = false;
    if (n <= 1 || bits <= 0) {
        if (first_in && n) CLD_CUDA(cudaMemcpyAsync(keys, first_in, n * sizeof(K), cudaMemcpyDeviceToDevice, s));
        return CLDIAM_OK;
    }
    if (n > 0xFFFFFFFFull) return fail(CLDIAM_ERR_UNSUPPORTED, "radix sort limited to 2^32 - 1 items");
    const bool kv = vals != nullptr;
    const int npass = (bits + 7) / 8;
    const int tile = kv ? OsCfg<K, true>::TILE : OsCfg<K, false>::TILE;
    const uint32_t ntiles = (uint32_t)((n + tile - 1) / tile);
    const size_t smem = (sizeof(K) + (kv ? sizeof(uint32_t) : 0)) * tile;
    static std::atomic<bool> attr_set[2][64];  // first call per device sets the attributes (idempotent)
    static std::atomic<bool> hist_attr_set[64];
    int dev = 0;
    CLD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_set[kv][dev]) {
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if (kv) {
            CLD_CUDA(cudaFuncSetAttribute(k_os_pass<K, true, false>, a, (int)smem));
            CLD_CUDA(cudaFuncSetAttribute(k_os_pass<K, true, true>, a, (int)smem));
        } else {
            CLD_CUDA(cudaFuncSetAttribute(k_os_pass<K, false, false>, a, (int)smem));
            CLD_CUDA(cudaFuncSetAttribute(k_os_pass<K, false, true>, a, (int)smem));
        }
        if (dev >= 0 && dev < 64) attr_set[kv][dev] = true;
    }
    DBuf<uint32_t> hist_own, ctl;
    DBuf<unsigned long long> status;
    CLD_TRY(ctl.alloc(2 * npass + 2, s));
    CLD_TRY(status.alloc((size_t)ntiles * OS_RADIX, s));
    CLD_CUDA(cudaMemsetAsync(ctl.get(), 0, (2 * npass + 2) * 4, s));
    uint32_t* hist = hist_in;
    if (!hist) {
        CLD_TRY(hist_own.alloc((size_t)npass * OS_RADIX, s));
        hist = hist_own.get();
        CLD_CUDA(cudaMemsetAsync(hist, 0, (size_t)npass * OS_RADIX * 4, s));
        const size_t hsm = (size_t)OS_WARPS * npass * OS_RADIX * 4;  // <= 64 KB (at most 8 passes)
        if (dev < 0 || dev >= 64 || !hist_attr_set[dev]) {
            CLD_CUDA(cudaFuncSetAttribute(k_os_hist<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          8 * OS_WARPS * OS_RADIX * 4));
            if (dev >= 0 && dev < 64) hist_attr_set[dev] = true;
        }
        CLD_K(K_RADIX_HIST, s, k_os_hist<K><<<grid_for(n, 256, 4), 256, hsm, s>>>(first_in ? first_in : keys, n, npass,
                                                                                  shift0, bits, hist));
        prof_add_bytes(K_RADIX_HIST, (double)n * sizeof(K));
    }
    CLD_K(K_RADIX_HIST, s, k_os_hist_scan<<<1, OS_RADIX, 0, s>>>(hist, npass));
    CLD_LAUNCH_CHECK();
    // first_in (keys only): the first pass reads it and writes keys_alt, so first_in is never written
    const K* ki = first_in ? first_in : keys;
    uint32_t* vi = vals;
    K* ko = keys_alt;
    uint32_t* vo = vals_alt;
    bool alt = false;
    for (int p = 0; p < npass; ++p) {
        CLD_CUDA(cudaMemsetAsync(status.get(), 0, (size_t)ntiles * OS_RADIX * 8, s));
        const int shift = shift0 + 8 * p;
        const bool hi = sizeof(K) == 8 && shift >= 32;
        const uint32_t sh = (uint32_t)shift & 31u;
        const uint32_t dm = bits - 8 * p >= 8 ? 0xFFu : ((1u << (bits - 8 * p)) - 1u);  // key bits only
        const uint32_t* go = hist + p * OS_RADIX;
        uint32_t* tc = ctl.get() + p;
        uint32_t* er = err_dev ? err_dev : ctl.get() + 2 * npass;
        if (kv && hi) {
            CLD_K(K_RADIX_SCATTER, s, k_os_pass<K, true, true><<<ntiles, OS_THREADS, smem, s>>>(ki, vi, ko, vo, n, sh, dm, go,
                                                                                              status.get(), tc, er));
        } else if (kv) {
            CLD_K(K_RADIX_SCATTER, s, k_os_pass<K, true, false><<<ntiles, OS_THREADS, smem, s>>>(ki, vi, ko, vo, n, sh, dm, go,
                                                                                               status.get(), tc, er));
        } else if (hi) {
            CLD_K(K_RADIX_SCATTER, s, k_os_pass<K, false, true><<<ntiles, OS_THREADS, smem, s>>>(ki, nullptr, ko, nullptr, n,
                                                                                               sh, dm, go, status.get(), tc, er));
        } else {
            CLD_K(K_RADIX_SCATTER, s, k_os_pass<K, false, false><<<ntiles, OS_THREADS, smem, s>>>(ki, nullptr, ko, nullptr, n,
                                                                                                sh, dm, go, status.get(), tc, er));
        }
        CLD_LAUNCH_CHECK();
        // algorithmic bytes: every item (key and value) read once and written once
        prof_add_bytes(K_RADIX_SCATTER, 2.0 * (double)n * (sizeof(K) + (kv ? sizeof(uint32_t) : 0)));
        const K* done_in = ki;
        ki = ko;
        ko = (first_in && p == 0) ? keys : const_cast<K*>(done_in);  // first_in is never written
        uint32_t* tv = vi; vi = vo; vo = tv;
        alt = !alt;
    }
    *in_alt = alt;
    if (err_dev) return CLDIAM_OK;  // the caller reads the look-back error word with its next result
    uint32_t herr = 0;
    CLD_CUDA(cudaMemcpyAsync(&herr, ctl.get() + 2 * npass, 4, cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    if (herr) return fail(CLDIAM_ERR_TIMEOUT, "radix sort look-back wait expired");
    return CLDIAM_OK;
}

// ------------------------------------------------------------------ unique runs of a sorted sequence
// Two passes over sorted (key, value) pairs: the first counts each tile's run
// heads (ballots), an exclusive scan turns the counts into each tile's first
// output index, and the second gives the heads consecutive indices r and
// writes them; for each run the minimum value is folded in with one store per
// run inside a warp, or one atomicMin per run piece per warp otherwise.
// Output per unique key: row_out[r] = key / div (if row_out), col_out[r*cs] =
// key % div, w_out[r*cs] = min value (w_out pre-filled with 0xFFFFFFFF).
// Keys >= sentinel are ignored (they sort last).
// With off_out, the run heads also write the CSR offsets of rows
// 0..nrows: off_out[q] = index of the first unique key with row >= q (a head
// fills the rows after its predecessor's row up to its own; the last run
// fills the rows after it with the total).
constexpr int UQ_THREADS = 256;
constexpr int UQ_ITEMS = 8;
constexpr int UQ_TILE = UQ_THREADS * UQ_ITEMS;

// heads of each tile (first pass)
template <class K>
__global__ void __launch_bounds__(UQ_THREADS) k_unique_count(const K* __restrict__ keys, size_t cnt,
                                                              K sentinel, uint32_t* __restrict__ heads) {
    __shared__ uint32_t s_w[UQ_THREADS / 32];
    const unsigned tid = threadIdx.x, w = tid >> 5, l = lane_id();
    const size_t base = (size_t)blockIdx.x * UQ_TILE + (size_t)w * (UQ_ITEMS * 32);
    K key[UQ_ITEMS];
#pragma unroll
    for (int i = 0; i < UQ_ITEMS; ++i) {
        const size_t idx = base + (size_t)i * 32 + l;
        key[i] = idx < cnt ? keys[idx] : sentinel;
    }
    uint32_t run = 0;
#pragma unroll
    for (int i = 0; i < UQ_ITEMS; ++i) {
        const size_t idx = base + (size_t)i * 32 + l;
        K prev = __shfl_up_sync(0xffffffffu, key[i], 1);
        if (l == 0) prev = (idx > 0 && idx < cnt) ? keys[idx - 1] : sentinel;
        run += (uint32_t)__popc(__ballot_sync(0xffffffffu, key[i] < sentinel && (idx == 0 || prev != key[i])));
    }
    if (l == 0) s_w[w] = run;
    __syncthreads();
    if (tid == 0) {
        uint32_t t = 0;
        for (int ww = 0; ww < UQ_THREADS / 32; ++ww) t += s_w[ww];
        heads[blockIdx.x] = t;
    }
}

// second pass: tile t's heads get indices from first[t] on
template <class K>
__global__ void __launch_bounds__(UQ_THREADS, 4)
    k_unique_write(const K* __restrict__ keys, const uint32_t* __restrict__ vals, size_t cnt, K sentinel,
                   uint64_t div, uint32_t* __restrict__ row_out, uint32_t* __restrict__ col_out,
                   uint32_t* __restrict__ w_out, int cs, uint64_t* __restrict__ off_out, uint32_t nrows,
                   const uint32_t* __restrict__ first) {
    __shared__ uint32_t s_woff[UQ_THREADS / 32], s_prefix;
    const unsigned tid = threadIdx.x, w = tid >> 5, l = lane_id();
    const uint32_t tile = blockIdx.x;
    const size_t base = (size_t)tile * UQ_TILE + (size_t)w * (UQ_ITEMS * 32);
    K key[UQ_ITEMS];
    uint32_t val[UQ_ITEMS];
#pragma unroll
    for (int i = 0; i < UQ_ITEMS; ++i) {
        const size_t idx = base + (size_t)i * 32 + l;
        key[i] = idx < cnt ? keys[idx] : sentinel;
        val[i] = idx < cnt ? vals[idx] : 0xFFFFFFFFu;
    }
    uint32_t head_bits = 0, run = 0;
    uint32_t ex[UQ_ITEMS];
#pragma unroll
    for (int i = 0; i < UQ_ITEMS; ++i) {
        const size_t idx = base + (size_t)i * 32 + l;
        K prev = __shfl_up_sync(0xffffffffu, key[i], 1);
        if (l == 0) prev = (idx > 0 && idx < cnt) ? keys[idx - 1] : sentinel;
        const bool f = key[i] < sentinel && (idx == 0 || prev != key[i]);
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        ex[i] = run + (uint32_t)__popc(bal & lanemask_lt());
        run += (uint32_t)__popc(bal);
        head_bits |= (f ? 1u : 0u) << i;
    }
    if (l == 0) s_woff[w] = run;
    __syncthreads();
    if (w == 0) {
        uint32_t acc = 0, my_off = 0;
        for (int ww = 0; ww < UQ_THREADS / 32; ++ww) {
            const uint32_t t = s_woff[ww];
            if ((int)l == ww) my_off = acc;
            acc += t;
        }
        __syncwarp();
        if (l < UQ_THREADS / 32) s_woff[l] = my_off;
        if (l == 0) s_prefix = first[tile];
    }
    __syncthreads();
    const uint32_t tbase = s_prefix + s_woff[w];
    // Run minima: a head stores its run's key and its own value, then (after a block barrier, so the
    // stores come first) every other item of a run folds its value in with atomicMin.  The one run
    // that may continue into the next tile has its head fold in with atomicMin too (w_out holds
    // 0xFFFFFFFF beforehand), as do items whose run began in an earlier tile.
    const size_t tend = min(cnt, (size_t)(tile + 1) * UQ_TILE);
    const K lastkey = keys[tend - 1];
    const bool crosses = tend < cnt && keys[tend] == lastkey && lastkey < sentinel;
    const auto row_of = [&](K kk) -> uint64_t { return (uint64_t)kk / div; };
#pragma unroll
    for (int i = 0; i < UQ_ITEMS; ++i) {
        const size_t idx = base + (size_t)i * 32 + l;
        const bool valid = key[i] < sentinel;
        K before = __shfl_up_sync(0xffffffffu, key[i], 1);
        if (l == 0) before = idx > 0 ? keys[idx - 1] : sentinel;
        const uint32_t f = (head_bits >> i) & 1u;
        if (!valid || !f) continue;
        const uint32_t r = tbase + ex[i];
        if (crosses && key[i] == lastkey) atomicMin(&w_out[(size_t)r * cs], val[i]);
        else w_out[(size_t)r * cs] = val[i];
        const uint64_t q = row_of(key[i]);
        if (row_out) row_out[r] = (uint32_t)q;
        col_out[(size_t)r * cs] = (uint32_t)((uint64_t)key[i] - q * div);
        if (off_out) {
            const uint64_t q0 = idx == 0 ? 0ull : row_of(before) + 1ull;  // rows after the previous run's row
            for (uint64_t qq = q0; qq <= q && qq <= nrows; ++qq) off_out[qq] = r;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < UQ_ITEMS; ++i) {
        const size_t idx = base + (size_t)i * 32 + l;
        const bool valid = key[i] < sentinel;
        K after = __shfl_down_sync(0xffffffffu, key[i], 1);
        if (l == 31) after = (idx + 1 < cnt) ? keys[idx + 1] : sentinel;
        if (!valid) continue;
        const uint32_t f = (head_bits >> i) & 1u;
        const uint32_t r = tbase + ex[i] + f - 1u;
        if (!f) atomicMin(&w_out[(size_t)r * cs], val[i]);
        // the last run: the remaining rows end at the total
        if (off_out && !(after < sentinel))
            for (uint64_t qq = row_of(key[i]) + 1; qq <= nrows; ++qq) off_out[qq] = (uint64_t)r + 1;
    }
}

template <class K>
static cldiam_status unique_min_sorted(const K* keys, const uint32_t* vals, size_t cnt, K sentinel,
                                       uint64_t div, uint32_t* row_out, uint32_t* col_out,
                                       uint32_t* w_out, int cs, uint64_t* off_out, uint32_t nrows,
                                       uint32_t* total_dev, cudaStream_t s) {
    if (cnt == 0) {
        CLD_CUDA(cudaMemsetAsync(total_dev, 0, 4, s));
        if (off_out) CLD_CUDA(cudaMemsetAsync(off_out, 0, ((size_t)nrows + 1) * 8, s));
        return CLDIAM_OK;
    }
    if (cnt > 0xFFFFFFFFull) return fail(CLDIAM_ERR_UNSUPPORTED, "more than 2^32 - 1 items");
    const uint32_t ntiles = (uint32_t)((cnt + UQ_TILE - 1) / UQ_TILE);
    DBuf<uint32_t> heads, first;
    CLD_TRY(heads.alloc(ntiles, s));
    CLD_TRY(first.alloc(ntiles, s));
    CLD_K(K_CSR, s, k_unique_count<K><<<ntiles, UQ_THREADS, 0, s>>>(keys, cnt, sentinel, heads.get()));
    CLD_LAUNCH_CHECK();
    CLD_TRY(scan_exclusive_u32(heads.get(), first.get(), ntiles, total_dev, s));
    CLD_K(K_CSR, s, k_unique_write<K><<<ntiles, UQ_THREADS, 0, s>>>(keys, vals, cnt, sentinel, div,
                                                                     row_out, col_out, w_out, cs, off_out, nrows,
                                                                     first.get()));
    CLD_LAUNCH_CHECK();
    uint32_t total = 0;
    CLD_CUDA(cudaMemcpyAsync(&total, total_dev, 4, cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    if (off_out && total == 0) CLD_CUDA(cudaMemsetAsync(off_out, 0, ((size_t)nrows + 1) * 8, s));  // no valid key
    return CLDIAM_OK;
}

// ------------------------------------------------------------------ de-duplication of packed edge items
// Items (a << vb | b) << wb | w with wb = 64 - 2 vb, sorted on their (a, b) bits; ~0 marks a dropped item
// (self-loop) and sorts last.  Two passes over tiles of 2,048 items: the first counts each tile's run
// heads, an exclusive scan gives each tile its first head index, and the second flags the heads again
// and writes them out.  (A one-pass form with a decoupled look-back over the tile counts was slower: its
// tiles wait on each other while the extra read of the two-pass form streams at full bandwidth.)
constexpr int UP_THREADS = 256;
constexpr int UP_WARPS = UP_THREADS / 32;
constexpr int UP_ITEMS = 8;
constexpr int UP_TILE = UP_THREADS * UP_ITEMS;

// Head flag of a packed item: kept and not sharing (row, col) with its predecessor (~0 before position 0).
__device__ __forceinline__ bool up_head(uint64_t prev, uint64_t x, uint64_t same_lim, uint64_t valid_lim) {
    return x < valid_lim && (prev ^ x) >= same_lim;
}

// First pass of the two-pass form: run heads per tile (CTAs loop over tiles).  With hist2 the heads'
// b digits are counted too, into per-warp shared histograms (dynamic, warps x npass x 256 words)
// flushed once per CTA.
__global__ void __launch_bounds__(UP_THREADS) k_unique_packed_count(const uint64_t* __restrict__ items, uint32_t cnt,
                                                                    int vb, uint32_t ntiles, uint32_t* __restrict__ heads,
                                                                    uint32_t* __restrict__ hist2) {
    extern __shared__ uint32_t uh[];
    __shared__ uint32_t s_w[UP_WARPS];
    const unsigned tid = threadIdx.x, w = tid >> 5, l = lane_id();
    const int wb = 64 - 2 * vb;
    const int npass = (vb + 7) / 8;
    if (hist2) {
        for (int i = tid; i < UP_WARPS * npass * 256; i += UP_THREADS) uh[i] = 0;
    }
    uint32_t* h = uh + w * npass * 256;
    const uint64_t same_lim = 1ull << wb, valid_lim = ~0ull << wb;
    const uint32_t wstart = w * (UP_ITEMS * 32);
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t tbase = (uint64_t)tile * UP_TILE;
        const uint32_t rem = (uint32_t)min((uint64_t)UP_TILE, (uint64_t)cnt - tbase);
        const uint64_t* it = items + tbase;
        uint64_t x[UP_ITEMS];
#pragma unroll
        for (int i = 0; i < UP_ITEMS; ++i) {
            const uint32_t li = wstart + (uint32_t)i * 32 + l;
            x[i] = li < rem ? it[li] : ~0ull;
        }
        uint64_t carry = ~0ull;
        if (l == 0 && wstart < rem && tbase + wstart > 0) carry = it[(int64_t)wstart - 1];
        uint32_t run = 0;
        __syncthreads();  // the histograms are zeroed; s_w of the previous tile has been read
#pragma unroll
        for (int i = 0; i < UP_ITEMS; ++i) {
            const uint64_t rot = __shfl_sync(0xffffffffu, x[i], (l + 31) & 31);
            const uint64_t prev = l == 0 ? carry : rot;
            carry = rot;
            const bool hd = up_head(prev, x[i], same_lim, valid_lim);
            run += (uint32_t)__popc(__ballot_sync(0xffffffffu, hd));
            if (hist2 && hd) {
                for (int p = 0; p < npass; ++p) {
                    const int left = vb - 8 * p;
                    const uint32_t dm = left >= 8 ? 0xFFu : ((1u << left) - 1u);
                    atomicAdd(&h[p * 256 + ((uint32_t)(x[i] >> (wb + 8 * p)) & dm)], 1u);
                }
            }
        }
        if (l == 0) s_w[w] = run;
        __syncthreads();
        if (tid == 0) {
            uint32_t t = 0;
            for (int ww = 0; ww < UP_WARPS; ++ww) t += s_w[ww];
            heads[tile] = t;
        }
    }
    if (hist2) {
        __syncthreads();
        for (int i = tid; i < npass * 256; i += UP_THREADS) {
            uint32_t c = 0;
            for (int ww = 0; ww < UP_WARPS; ++ww) c += uh[ww * npass * 256 + i];
            if (c) atomicAdd(&hist2[i], c);
        }
    }
}

// De-duplication that keeps packed items: out[r] = the r-th distinct (row, col) with its smallest weight.
// Items of one run differ only in their weight bits, so the run minimum is the 64-bit minimum of the items:
// heads store their item, the other members of runs headed in the tile fold theirs in with atomicMin after
// a block barrier, and the tile's last run is followed into later tiles by one warp.
__global__ void __launch_bounds__(UP_THREADS, 4)
    k_unique_items(const uint64_t* __restrict__ items, uint32_t cnt, int vb, unsigned long long* __restrict__ out,
                   uint32_t* __restrict__ total, const uint32_t* __restrict__ first, uint32_t* __restrict__ ustart,
                   uint32_t* __restrict__ uend) {
    __shared__ uint32_t s_woff[UP_WARPS];
    __shared__ uint32_t s_first, s_count;
    const unsigned tid = threadIdx.x, w = tid >> 5, l = lane_id();
    const uint32_t tile = blockIdx.x;
    const uint64_t tbase = (uint64_t)tile * UP_TILE;
    const uint32_t rem = (uint32_t)min((uint64_t)UP_TILE, (uint64_t)cnt - tbase);
    const int wb = 64 - 2 * vb;
    const uint64_t same_lim = 1ull << wb, valid_lim = ~0ull << wb;
    const uint32_t wstart = w * (UP_ITEMS * 32);
    const uint64_t* it = items + tbase;
    uint64_t x[UP_ITEMS];
#pragma unroll
    for (int i = 0; i < UP_ITEMS; ++i) {
        const uint32_t li = wstart + (uint32_t)i * 32 + l;
        x[i] = li < rem ? it[li] : ~0ull;
    }
    uint64_t carry = ~0ull;
    if (l == 0 && wstart < rem && tbase + wstart > 0) carry = it[(int64_t)wstart - 1];
    uint32_t head = 0, run = 0;
    uint32_t ex_pk[UP_ITEMS / 4];
    uint32_t newrow = 0;  // bit i: item i heads a run whose row (the a bits) differs from the previous item's
#pragma unroll
    for (int i = 0; i < UP_ITEMS; ++i) {
        const uint64_t rot = __shfl_sync(0xffffffffu, x[i], (l + 31) & 31);
        const uint64_t prev = l == 0 ? carry : rot;
        carry = rot;
        const bool f = up_head(prev, x[i], same_lim, valid_lim);
        if (f && (prev >= valid_lim || (prev ^ x[i]) >> (wb + vb) != 0)) newrow |= 1u << i;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const uint32_t ex = run + (uint32_t)__popc(bal & lanemask_lt());
        run += (uint32_t)__popc(bal);
        if (i % 4 == 0) ex_pk[i / 4] = ex;
        else ex_pk[i / 4] |= ex << (8 * (i % 4));
        head |= (f ? 1u : 0u) << i;
    }
    if (l == 0) s_woff[w] = run;
    __syncthreads();
    if (w == 0) {
        const uint32_t v = l < UP_WARPS ? s_woff[l] : 0u;
        const uint32_t incl = warp_incl_scan(v);
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, UP_WARPS - 1);
        const uint32_t excl = first[tile];
        if (l < UP_WARPS) s_woff[l] = excl + incl - v;
        if (l == 0) {
            s_first = excl;
            s_count = tot;
            if (tile == gridDim.x - 1) *total = excl + tot;
        }
    }
    __syncthreads();
    const uint32_t woff = s_woff[w], tfirst = s_first;
#pragma unroll
    for (int i = 0; i < UP_ITEMS; ++i)
        if ((head >> i) & 1u) {
            const uint32_t r = woff + ((ex_pk[i / 4] >> (8 * (i % 4))) & 0xFFu);
            out[r] = x[i];
            // run bounds of the rows: a distinct edge whose row differs from the previous one's starts its
            // row's run and ends the previous row's (the last row's end is set after the pass)
            if (ustart && ((newrow >> i) & 1u)) {
                ustart[(uint32_t)(x[i] >> (wb + vb))] = r;
                if (r > 0) {
                    // the previous distinct edge is any item before this one in the run order: the item at
                    // position (tile start + this item's position) - 1 of the sorted input
                    const uint32_t li = wstart + (uint32_t)i * 32 + l;
                    const uint64_t pv = items[tbase + li - 1];
                    uend[(uint32_t)(pv >> (wb + vb))] = r;
                }
            }
        }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < UP_ITEMS; ++i) {
        const uint32_t li = wstart + (uint32_t)i * 32 + l;
        if (li >= rem || x[i] >= valid_lim || ((head >> i) & 1u)) continue;
        const uint32_t before = woff + ((ex_pk[i / 4] >> (8 * (i % 4))) & 0xFFu);  // heads before the item
        if (before > tfirst) atomicMin(&out[before - 1], (unsigned long long)x[i]);
    }
    // the tile's last run continuing into later tiles: scan forward while the key repeats
    if (w == UP_WARPS - 1 && rem == (uint32_t)UP_TILE && s_count > 0 && tbase + UP_TILE < cnt) {
        const uint64_t last = __shfl_sync(0xffffffffu, x[UP_ITEMS - 1], 31);
        if (last < valid_lim) {
            unsigned long long mn = ~0ull;
            for (uint64_t p = tbase + UP_TILE;; p += 32) {
                const uint64_t y = p + l < cnt ? items[p + l] : ~0ull;
                const unsigned same = __ballot_sync(0xffffffffu, y < valid_lim && (y ^ last) < same_lim);
                const unsigned take = ~same ? (unsigned)(__ffs(~same) - 1) : 32u;
                if (l < take) mn = min(mn, (unsigned long long)y);
                if (take < 32) break;
            }
            mn = warp_min(mn);
            if (l == 0 && mn != ~0ull) atomicMin(&out[tfirst + s_count - 1], mn);
        }
    }
}

// the last row's run ends at the number of distinct edges
__global__ void k_last_uend(const uint64_t* __restrict__ out, const uint32_t* __restrict__ total, int shift,
                            uint32_t* __restrict__ uend) {
    const uint32_t t = *total;
    if (t > 0) uend[(uint32_t)(out[t - 1] >> shift)] = t;
}

cldiam_status unique_items_u64(const uint64_t* items, size_t cnt, int vb, uint64_t* out, uint32_t* total_dev,
                               cudaStream_t s, uint32_t* hist2, uint32_t* ustart, uint32_t* uend) {
    if (cnt == 0) {
        CLD_CUDA(cudaMemsetAsync(total_dev, 0, 4, s));
        return CLDIAM_OK;
    }
    if (cnt > 0xFFFFFFFFull - UP_TILE) return fail(CLDIAM_ERR_UNSUPPORTED, "too many items");
    if (vb < 1 || vb > 32) return fail(CLDIAM_ERR_INVALID_ARG, "packed items need 1..32 id bits");
    const uint32_t ntiles = (uint32_t)((cnt + UP_TILE - 1) / UP_TILE);
    DBuf<uint32_t> heads, first;
    CLD_TRY(heads.alloc(ntiles, s));
    CLD_TRY(first.alloc(ntiles, s));
    const size_t usm = hist2 ? (size_t)UP_WARPS * ((vb + 7) / 8) * 256 * 4 : 0;  // <= 32 KB
    CLD_K(K_CSR, s, k_unique_packed_count<<<grid_for((size_t)ntiles * UP_THREADS, UP_THREADS, 4), UP_THREADS, usm, s>>>(
                        items, (uint32_t)cnt, vb, ntiles, heads.get(), hist2));
    CLD_LAUNCH_CHECK();
    CLD_TRY(scan_exclusive_u32(heads.get(), first.get(), ntiles, nullptr, s));
    CLD_K(K_CSR, s, k_unique_items<<<ntiles, UP_THREADS, 0, s>>>(items, (uint32_t)cnt, vb,
                                                                 reinterpret_cast<unsigned long long*>(out), total_dev,
                                                                 first.get(), ustart, uend));
    if (ustart) CLD_K(K_CSR, s, k_last_uend<<<1, 1, 0, s>>>(out, total_dev, 64 - vb, uend));
    CLD_LAUNCH_CHECK();
    return CLDIAM_OK;
}

cldiam_status unique_min_sorted_u64(const uint64_t* keys, const uint32_t* vals, size_t cnt, uint64_t sentinel,
                                    uint64_t div, uint32_t* row_out, uint32_t* col_out, uint32_t* w_out, int cs,
                                    uint64_t* off_out, uint32_t nrows, uint32_t* total_dev, cudaStream_t s) {
    return unique_min_sorted<uint64_t>(keys, vals, cnt, sentinel, div, row_out, col_out, w_out, cs, off_out,
                                       nrows, total_dev, s);
}
cldiam_status unique_min_sorted_u32(const uint32_t* keys, const uint32_t* vals, size_t cnt, uint32_t sentinel,
                                    uint64_t div, uint32_t* row_out, uint32_t* col_out, uint32_t* w_out, int cs,
                                    uint64_t* off_out, uint32_t nrows, uint32_t* total_dev, cudaStream_t s) {
    return unique_min_sorted<uint32_t>(keys, vals, cnt, sentinel, div, row_out, col_out, w_out, cs, off_out,
                                       nrows, total_dev, s);
}

cldiam_status radix_sort_pairs_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                                   size_t n, int bits, bool* in_alt, cudaStream_t s) {
    return radix_sort_impl<uint64_t>(keys, vals, keys_alt, vals_alt, n, 0, bits, in_alt, s);
}
cldiam_status radix_sort_keys_u64(uint64_t* keys, uint64_t* keys_alt, size_t n, int shift0, int bits, bool* in_alt,
                                  cudaStream_t s, uint32_t* err_dev, const uint64_t* first_in, uint32_t* hist_in) {
    return radix_sort_impl<uint64_t>(keys, nullptr, keys_alt, nullptr, n, shift0, bits, in_alt, s, err_dev, first_in,
                                     hist_in);
}
cldiam_status radix_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                                   size_t n, int bits, bool* in_alt, cudaStream_t s) {
    return radix_sort_impl<uint32_t>(keys, vals, keys_alt, vals_alt, n, 0, bits, in_alt, s);
}

}  // namespace cld
