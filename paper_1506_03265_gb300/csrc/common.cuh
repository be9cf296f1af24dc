// Internal helpers of the CL-DIAM CUDA library: status plumbing, stream-
// ordered device buffers, warp/block primitives and the Philox4x32-10 draw.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "cldiam.h"

namespace cld {

constexpr uint64_t kInfKey = ~0ull;         // node without a center: (inf, nil)
constexpr uint32_t kNone = 0xFFFFFFFFu;      // no center / unreachable distance
constexpr uint32_t kDeltaMax = 0x80000000u;  // Delta saturates at 2^31
constexpr uint32_t kMaxStages = 100000u;
constexpr double kGamma = 2.772588722239781;  // 4 ln 2 (Algorithm 1)

// ---------------------------------------------------------------- status
void set_error(const std::string& msg);
cldiam_status fail(cldiam_status s, const std::string& msg);
cldiam_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define CLD_CUDA(x)                                                      \
    do {                                                                 \
        cudaError_t e_ = (x);                                            \
        if (e_ != cudaSuccess) return cld::cuda_fail(e_, #x, __FILE__, __LINE__); \
    } while (0)

#define CLD_TRY(x)                            \
    do {                                      \
        cldiam_status s_ = (x);               \
        if (s_ != CLDIAM_OK) return s_;       \
    } while (0)

#define CLD_LAUNCH_CHECK() CLD_CUDA(cudaGetLastError())

// ---------------------------------------------------------------- memory
// Stream-ordered allocation from the device's default memory pool (kept warm:
// its release threshold is raised once, so repeated calls reuse memory).
cldiam_status dmalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);

template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { release(); }
    cldiam_status alloc(size_t count, cudaStream_t stream) {
        release();
        s = stream;
        n = count;
        if (count == 0) return CLDIAM_OK;
        return dmalloc(reinterpret_cast<void**>(&p), count * sizeof(T), stream);
    }
    void release() {
        if (p) dfree(p, s);
        p = nullptr;
        n = 0;
    }
    T* get() const { return p; }
    T* detach() {
        T* q = p;
        p = nullptr;
        n = 0;
        return q;
    }
};

// Per-call small host<->device counter block in pinned memory.  Blocks of up
// to kPinnedBlock bytes come from a process-wide free list of pinned slabs
// (pinning and unpinning memory is slow and cudaFreeHost synchronises the
// device); larger ones are pinned individually.
constexpr size_t kPinnedBlock = 256;
void* pinned_take();
void pinned_give(void* p);
struct Pinned {
    void* h = nullptr;
    bool pooled = false;
    ~Pinned() {
        if (!h) return;
        if (pooled) pinned_give(h);
        else cudaFreeHost(h);
    }
    cldiam_status alloc(size_t bytes);
};

// ---------------------------------------------------------------- launch sizing
int num_sms();
inline unsigned grid_for(size_t n, int block, int max_blocks_per_sm = 8) {
    size_t b = (n + block - 1) / block;
    size_t cap = (size_t)num_sms() * max_blocks_per_sm;
    if (b > cap) b = cap;
    if (b == 0) b = 1;
    return (unsigned)b;
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11).  Ten rounds of two 32x32->64 multiplies with the round constants
// 0xD2511F53 / 0xCD9E8D57 and a Weyl key schedule (0x9E3779B9, 0xBB67AE85).
struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ inline void mulhilo32(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
#ifdef __CUDA_ARCH__
    hi = __umulhi(a, b);
    lo = a * b;
#else
    uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
#endif
}

__host__ __device__ inline U4 philox4x32_10(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t h0, l0, h1, l1;
        mulhilo32(0xD2511F53u, c0, h0, l0);
        mulhilo32(0xCD9E8D57u, c2, h1, l1);
        uint32_t n0 = h1 ^ c1 ^ k0;
        uint32_t n2 = h0 ^ c3 ^ k1;
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// ---------------------------------------------------------------- warp / block helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}
template <class T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}
// inclusive warp scan
template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if ((int)lane_id() >= o) v += u;
    }
    return v;
}

// Warp-aggregated append: every lane with `pred` gets a unique slot from
// *counter (one atomic per warp).  Must be called by all lanes of the warp.
__device__ __forceinline__ uint32_t warp_append(uint32_t* counter, bool pred) {
    unsigned mask = __ballot_sync(0xffffffffu, pred);
    if (mask == 0) return 0;
    unsigned leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane_id() == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + __popc(mask & lanemask_lt());
}

// Block-aggregated append: one global atomicAdd per CTA.  Returns this
// thread's slot when `pred`.  Every thread of the block must call it (it
// synchronises the block); `scratch` is caller shared memory of 33 words.
__device__ __forceinline__ uint32_t block_append(uint32_t* counter, bool pred, uint32_t* scratch) {
    const unsigned mask = __ballot_sync(0xffffffffu, pred);
    const unsigned w = threadIdx.x >> 5, l = lane_id(), nw = blockDim.x >> 5;
    if (l == 0) scratch[w] = (uint32_t)__popc(mask);
    __syncthreads();
    if (w == 0) {
        const uint32_t v = l < nw ? scratch[l] : 0u;
        const uint32_t incl = warp_incl_scan(v);
        if (l < nw) scratch[l] = incl - v;
        if (l == 31) scratch[32] = incl ? atomicAdd(counter, incl) : 0u;
    }
    __syncthreads();
    const uint32_t slot = scratch[32] + scratch[w] + (uint32_t)__popc(mask & lanemask_lt());
    __syncthreads();
    return slot;
}

// Block-wide reduction helpers (blockDim.x multiple of 32, <= 1024).
template <class T, class Op>
__device__ T block_reduce(T v, Op op, T identity) {
    __shared__ T red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    unsigned w = threadIdx.x >> 5;
    if (lane_id() == 0) red[w] = v;
    __syncthreads();
    unsigned nw = blockDim.x >> 5;
    v = (threadIdx.x < nw) ? red[threadIdx.x] : identity;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;  // valid in thread 0
}

// ---------------------------------------------------------------- timers and acquire loads
// nanoseconds of the GPU's global timer (bounds every wait on another CTA)
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// ---------------------------------------------------------------- L2 eviction priorities
// A graph sweep streams adjacency that is read once per step; the node state
// it looks up (keys, stamps) is far smaller and reused by every entry.  The
// streamed lines are loaded with the evict-first policy (and no L1
// allocation), the node state with evict-last, so that the state stays in L2
// while the adjacency passes through.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint2 ld_stream_u2(const uint2* p, uint64_t pol) {
    uint2 r;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                 : "=r"(r.x), "=r"(r.y)
                 : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t* p, uint64_t pol) {
    uint32_t r;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint64_t ld_stream_u64(const uint64_t* p, uint64_t pol) {
    uint64_t r;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint32_t ld_nc_keep_u32(const uint32_t* p, uint64_t pol) {
    uint32_t r;
    asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    return r;
}
// read-only for the whole kernel (a snapshot): may be cached in L1
__device__ __forceinline__ unsigned long long ld_nc_keep_u64(const unsigned long long* p, uint64_t pol) {
    unsigned long long r;
    asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(pol));
    return r;
}
// mutable node state read as a filter: through L1.  A stale line can only hold an older, larger key (keys
// never rise within a kernel), so the filter lets through extra candidates, never drops a winning one.
__device__ __forceinline__ unsigned long long ld_keep_u64(const unsigned long long* p, uint64_t pol) {
    unsigned long long r;
    asm volatile("ld.global.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint32_t ld_keep_u32(const uint32_t* p, uint64_t pol) {
    uint32_t r;
    asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    return r;
}
// mutable node state: L2 only (other CTAs write it in the same kernel)
__device__ __forceinline__ unsigned long long ld_cg_keep_u64(const unsigned long long* p, uint64_t pol) {
    unsigned long long r;
    asm volatile("ld.global.cg.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ unsigned long long atom_min_keep_u64(unsigned long long* p, unsigned long long v,
                                                                uint64_t pol) {
    unsigned long long old;
    asm volatile("atom.global.min.L2::cache_hint.u64 %0, [%1], %2, %3;" : "=l"(old) : "l"(p), "l"(v), "l"(pol)
                 : "memory");
    return old;
}
__device__ __forceinline__ void red_min_keep_u64(unsigned long long* p, unsigned long long v, uint64_t pol) {
    asm volatile("red.global.min.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}

// ---------------------------------------------------------------- device-wide primitives (prims.cu)
// Exclusive prefix sum of n values; *total (device pointer, may be null) gets the sum.
cldiam_status scan_exclusive_u32(const uint32_t* in, uint32_t* out, size_t n, uint32_t* total, cudaStream_t s);
cldiam_status scan_exclusive_u64(const uint64_t* in, uint64_t* out, size_t n, uint64_t* total, cudaStream_t s);
// Max / sum reductions into a device scalar (which the call initialises).
cldiam_status reduce_max_u32(const uint32_t* in, size_t n, uint32_t* out, cudaStream_t s);
cldiam_status reduce_sum_u32_to_u64(const uint32_t* in, size_t n, uint64_t* out, cudaStream_t s);
cldiam_status reduce_min_u32(const uint32_t* in, size_t n, uint32_t* out, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the
// key.  Buffers *_alt are scratch of the same size; on return *result_in_alt
// tells which pair of buffers holds the sorted sequence.
cldiam_status radix_sort_pairs_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                                   size_t n, int bits, bool* result_in_alt, cudaStream_t s);
cldiam_status radix_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                                   size_t n, int bits, bool* result_in_alt, cudaStream_t s);
// Stable LSD radix sort of 64-bit keys alone on key bits [shift0, shift0 + bits).  With err_dev the
// call does not synchronise: a look-back wait that expired sets *err_dev (device word) instead of
// returning TIMEOUT, for the caller to read with its next result.  With first_in the n input keys are
// read from there (never written) and keys / keys_alt serve only as the ping-pong buffers.  With hist_in
// the digit counts of every pass (ceil(bits / 8) x 256 words, in pass order, digits as the sort takes
// them) were accumulated by the producer of the keys: the sort scans them in place instead of reading
// the keys once more to count.
cldiam_status radix_sort_keys_u64(uint64_t* keys, uint64_t* keys_alt, size_t n, int shift0, int bits,
                                  bool* result_in_alt, cudaStream_t s, uint32_t* err_dev = nullptr,
                                  const uint64_t* first_in = nullptr, uint32_t* hist_in = nullptr);

// Unique keys of a sorted sequence with the minimum value of each run:
// row_out[r] = key / div (row_out may be null), col_out[r*cs] = key % div,
// w_out[r*cs] = run minimum (w_out must hold 0xFFFFFFFF beforehand);
// keys >= sentinel are skipped; *total_dev = number of unique keys.  With
// off_out (may be null), off_out[0..nrows] = CSR offsets of the rows.
cldiam_status unique_min_sorted_u64(const uint64_t* keys, const uint32_t* vals, size_t cnt, uint64_t sentinel,
                                    uint64_t div, uint32_t* row_out, uint32_t* col_out, uint32_t* w_out, int cs,
                                    uint64_t* off_out, uint32_t nrows, uint32_t* total_dev, cudaStream_t s);
cldiam_status unique_min_sorted_u32(const uint32_t* keys, const uint32_t* vals, size_t cnt, uint32_t sentinel,
                                    uint64_t div, uint32_t* row_out, uint32_t* col_out, uint32_t* w_out, int cs,
                                    uint64_t* off_out, uint32_t nrows, uint32_t* total_dev, cudaStream_t s);
// De-duplication of packed edge items (a << vb | b) << (64 - 2 vb) | w sorted on their (a, b) bits (~0 marks
// a dropped item): out[r] = the r-th distinct (a, b) item with its smallest weight; *total_dev = their
// number.  With hist2 (ceil(vb / 8) x 256 words, zeroed) the counting pass also adds up the 8-bit digits
// of every distinct item's b (bits [wb, wb + vb)), pass by pass: the histograms of a following sort on b.
cldiam_status unique_items_u64(const uint64_t* items, size_t cnt, int vb, uint64_t* out, uint32_t* total_dev,
                               cudaStream_t s, uint32_t* hist2 = nullptr, uint32_t* ustart = nullptr,
                               uint32_t* uend = nullptr);

// CSR offsets off[0..n] of entries whose (sorted) row ids are row[0..nnz):
// off[u] = index of the first entry with row >= u.  No atomics, no scan.
cldiam_status offsets_from_rows(const uint32_t* row, uint64_t nnz, uint32_t n, uint64_t* off, cudaStream_t s);

inline int bits_for(uint64_t max_value) {  // bits needed to represent values <= max_value
    int b = 0;
    while (b < 64 && (max_value >> b) != 0) ++b;
    return b;
}

}  // namespace cld
