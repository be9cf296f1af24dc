// Phi(G_C) (Section 4): the largest finite shortest-path distance of the
// quotient graph, by exact blocked Floyd-Warshall over the dense k x k
// distance matrix in (min, +) arithmetic on the integer ALUs (min-plus is not
// a tensor-core contraction).
//
// Blocked FW with 32 x 32 tiles (Venkataraman, Sahni, Mukhopadhyaya): for
// each pivot tile r, (1) close the diagonal tile, (2) update the tiles of
// row r and column r through it, (3) update every other tile from its row-r
// and column-r tiles.  Entries are uint32 with 0xFFFFFFFF = no path; a sum
// of two finite entries that reaches 2^32 - 1 raises the overflow flag
// instead of wrapping.
#include "internal.cuh"
#include "prof.cuh"

namespace cld {

namespace {

constexpr int T = 32;
constexpr uint32_t INF = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t relax_min(uint32_t c, uint32_t a, uint32_t b, bool& ovf) {
    uint32_t s = a + b;
    bool carry = s < a;
    bool finite = (a != INF) & (b != INF);
    ovf |= finite & (carry | (s == INF));
    return (carry | !finite) ? c : (s < c ? s : c);
}

__global__ void k_fw_init(uint32_t* __restrict__ M, uint32_t kp, uint32_t k) {
    size_t total = (size_t)kp * kp;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t r = (uint32_t)(i / kp), c = (uint32_t)(i % kp);
        M[i] = (r == c) ? 0u : INF;
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

__global__ void k_fw_scatter(const uint64_t* __restrict__ off, const uint32_t* __restrict__ col,
                             const uint32_t* __restrict__ w, uint32_t k, uint32_t kp, uint32_t* __restrict__ M) {
    for (uint32_t a = blockIdx.x; a < k; a += gridDim.x)
        for (uint64_t j = off[a] + threadIdx.x; j < off[a + 1]; j += blockDim.x) {
            uint32_t b = col[j];
            if (b != a) atomicMin(&M[(size_t)a * kp + b], w[j]);
        }
}

// phase 1: the pivot tile against itself
__global__ void __launch_bounds__(T* T) k_fw_phase1(uint32_t* __restrict__ M, uint32_t kp, uint32_t r,
                                                    uint32_t* __restrict__ ovf_flag) {
    __shared__ uint32_t t[T][T + 1];
    const int y = threadIdx.x / T, x = threadIdx.x % T;
    size_t base = (size_t)r * T * kp + (size_t)r * T;
    t[y][x] = M[base + (size_t)y * kp + x];
    __syncthreads();
    bool ovf = false;
    for (int p = 0; p < T; ++p) {
        uint32_t v = relax_min(t[y][x], t[y][p], t[p][x], ovf);
        __syncthreads();
        t[y][x] = v;
        __syncthreads();
    }
    M[base + (size_t)y * kp + x] = t[y][x];
    if (ovf) atomicExch(ovf_flag, 1u);
}

// phase 2: tiles in pivot row r and pivot column r
__global__ void __launch_bounds__(T* T) k_fw_phase2(uint32_t* __restrict__ M, uint32_t kp, uint32_t r, uint32_t nt,
                                                    uint32_t* __restrict__ ovf_flag) {
    __shared__ uint32_t piv[T][T + 1];
    __shared__ uint32_t t[T][T + 1];
    const int y = threadIdx.x / T, x = threadIdx.x % T;
    uint32_t idx = blockIdx.x;  // 0..nt-2 row tiles, nt-1..2nt-3 column tiles
    bool is_row = idx < nt - 1;
    uint32_t o = is_row ? idx : idx - (nt - 1);
    if (o >= r) ++o;
    uint32_t ti = is_row ? r : o, tj = is_row ? o : r;
    size_t pb = (size_t)r * T * kp + (size_t)r * T;
    size_t tb = (size_t)ti * T * kp + (size_t)tj * T;
    piv[y][x] = M[pb + (size_t)y * kp + x];
    t[y][x] = M[tb + (size_t)y * kp + x];
    __syncthreads();
    bool ovf = false;
    for (int p = 0; p < T; ++p) {
        // row tile: t[y][x] = min(t, piv[y][p] + t[p][x]); column tile: min(t, t[y][p] + piv[p][x])
        uint32_t a = is_row ? piv[y][p] : t[y][p];
        uint32_t b = is_row ? t[p][x] : piv[p][x];
        uint32_t v = relax_min(t[y][x], a, b, ovf);
        __syncthreads();
        t[y][x] = v;
        __syncthreads();
    }
    M[tb + (size_t)y * kp + x] = t[y][x];
    if (ovf) atomicExch(ovf_flag, 1u);
}

// phase 3: every other tile from its pivot-column and pivot-row tiles
__global__ void __launch_bounds__(T* T) k_fw_phase3(uint32_t* __restrict__ M, uint32_t kp, uint32_t r, uint32_t nt,
                                                    uint32_t* __restrict__ ovf_flag) {
    __shared__ uint32_t A[T][T + 1];
    __shared__ uint32_t B[T][T + 1];
    const int y = threadIdx.x / T, x = threadIdx.x % T;
    uint32_t ti = blockIdx.y, tj = blockIdx.x;
    if (ti >= r) ++ti;
    if (tj >= r) ++tj;
    A[y][x] = M[((size_t)ti * T + y) * kp + (size_t)r * T + x];
    B[y][x] = M[((size_t)r * T + y) * kp + (size_t)tj * T + x];
    size_t ci = ((size_t)ti * T + y) * kp + (size_t)tj * T + x;
    uint32_t c = M[ci];
    __syncthreads();
    bool ovf = false;
#pragma unroll 8
    for (int p = 0; p < T; ++p) c = relax_min(c, A[y][p], B[p][x], ovf);
    M[ci] = c;
    if (ovf) atomicExch(ovf_flag, 1u);
}

__global__ void k_fw_max_finite(const uint32_t* __restrict__ M, uint32_t kp, uint32_t k, uint32_t* __restrict__ out) {
    uint32_t m = 0;
    size_t total = (size_t)k * kp;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t c = (uint32_t)(i % kp);
        uint32_t v = M[i];
        if (c < k && v != INF && v > m) m = v;
    }
    m = block_reduce(m, [](uint32_t a, uint32_t b) { return a > b ? a : b; }, 0u);
    if (threadIdx.x == 0) atomicMax(out, m);
}

}  // namespace

cldiam_status apsp_max_device(uint32_t k, const uint64_t* off, const uint32_t* col, const uint32_t* w, uint64_t nnz,
                              cudaStream_t s, uint64_t* phi, bool validate) {
    *phi = 0;
    if (k <= 1) return CLDIAM_OK;
    const uint32_t nt = (k + T - 1) / T;
    const uint32_t kp = nt * T;
    DBuf<uint32_t> M, scal;
    CLD_TRY(scal.alloc(3, s));
    CLD_CUDA(cudaMemsetAsync(scal.get(), 0, 12, s));
    if (validate) {
        CLD_K(K_FW, s, k_fw_validate<<<grid_for((size_t)k + nnz + 1, 256), 256, 0, s>>>(off, col, k, nnz, scal.get() + 2));
        CLD_LAUNCH_CHECK();
        uint32_t bad = 0;
        CLD_CUDA(cudaMemcpyAsync(&bad, scal.get() + 2, 4, cudaMemcpyDeviceToHost, s));
        CLD_CUDA(cudaStreamSynchronize(s));
        if (bad) return fail(CLDIAM_ERR_INVALID_ARG, "malformed CSR (offsets or column ids)");
    }
    CLD_TRY(M.alloc((size_t)kp * kp, s));
    CLD_K(K_FW, s, k_fw_init<<<grid_for((size_t)kp * kp, 256), 256, 0, s>>>(M.get(), kp, k));
    CLD_K(K_FW, s, k_fw_scatter<<<grid_for(k, 1, 64), 128, 0, s>>>(off, col, w, k, kp, M.get()));
    CLD_LAUNCH_CHECK();
    for (uint32_t r = 0; r < nt; ++r) {
        CLD_K(K_FW, s, k_fw_phase1<<<1, T * T, 0, s>>>(M.get(), kp, r, scal.get()));
        if (nt > 1) {
            CLD_K(K_FW, s, k_fw_phase2<<<2 * (nt - 1), T * T, 0, s>>>(M.get(), kp, r, nt, scal.get()));
            CLD_K(K_FW, s, k_fw_phase3<<<dim3(nt - 1, nt - 1), T * T, 0, s>>>(M.get(), kp, r, nt, scal.get()));
        }
        CLD_LAUNCH_CHECK();
    }
    CLD_K(K_FW, s, k_fw_max_finite<<<grid_for((size_t)k * kp, 256), 256, 0, s>>>(M.get(), kp, k, scal.get() + 1));
    CLD_LAUNCH_CHECK();
    uint32_t h[2];
    CLD_CUDA(cudaMemcpyAsync(h, scal.get(), 8, cudaMemcpyDeviceToHost, s));
    CLD_CUDA(cudaStreamSynchronize(s));
    if (h[0]) return fail(CLDIAM_ERR_OVERFLOW, "a quotient distance reached 2^32 - 1");
    *phi = h[1];
    return CLDIAM_OK;
}

}  // namespace cld
