// transpose.cu -- the tall-and-skinny entry (section II: the row-block form of
// the distributed SVD).  A tall A (rows x cols, cols <= 1024) is split into
// row blocks; A^T is then short and fat and its column blocks are A's row
// blocks, so the column-block path runs unchanged on A^T.  This file forms
// the CSC of A^T (the CSR of A) from the CSC of A on the device:
//   1. count the entries of every row (atomics),
//   2. exclusive scan of the counts into the column pointers of A^T,
//   3. scatter every entry into its row's segment (atomic slot, any order),
//   4. order every segment by column: an entry's place is the number of
//      entries of its row with a smaller column (columns within a row are
//      distinct), so the result is the unique sorted CSC of A^T.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rk {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanTile = 2 * kScanThreads;

__global__ void __launch_bounds__(kThreads)
k_t_count(const int32_t* __restrict__ row_idx, int64_t nnz, int32_t* __restrict__ cnt) {
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * kThreads)
        atomicAdd(cnt + row_idx[e], 1);
}

// Exclusive scan of n int32 counts into int64 offsets, tile by tile: local
// offsets and the tile totals.
__global__ void __launch_bounds__(kScanThreads)
k_t_scan_tiles(const int32_t* __restrict__ cnt, int64_t n, int64_t* __restrict__ out,
               int64_t* __restrict__ tile_sum) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const int64_t i0 = base + 2 * threadIdx.x, i1 = i0 + 1;
    const int64_t a = i0 < n ? cnt[i0] : 0, b = i1 < n ? cnt[i1] : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = a + b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int64_t before = (warp ? warp_tot[warp - 1] : 0) + incl - (a + b);
    if (i0 < n) out[i0] = before;
    if (i1 < n) out[i1] = before + a;
    if (threadIdx.x == kScanThreads - 1) tile_sum[blockIdx.x] = warp_tot[31];
}

// Exclusive scan of the tile totals in place (one CTA, contiguous runs per
// thread) and the grand total into out[n].
__global__ void __launch_bounds__(kScanThreads)
k_t_scan_totals(int64_t* __restrict__ tile_sum, int64_t ntiles, int64_t* __restrict__ out,
                int64_t n) {
    __shared__ int64_t scan[kScanThreads];
    const int64_t per = ceil_div(ntiles, kScanThreads);
    const int64_t a = std::min<int64_t>(ntiles, (int64_t)threadIdx.x * per);
    const int64_t b = std::min<int64_t>(ntiles, a + per);
    int64_t s = 0;
    for (int64_t i = a; i < b; ++i) s += tile_sum[i];
    scan[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        const int64_t add = threadIdx.x >= (unsigned)off ? scan[threadIdx.x - off] : 0;
        __syncthreads();
        scan[threadIdx.x] += add;
        __syncthreads();
    }
    int64_t run = scan[threadIdx.x] - s;
    for (int64_t i = a; i < b; ++i) {
        const int64_t t = tile_sum[i];
        tile_sum[i] = run;
        run += t;
    }
    if (threadIdx.x == kScanThreads - 1) out[n] = scan[kScanThreads - 1];
}

__global__ void __launch_bounds__(kThreads)
k_t_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ tile_sum) {
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kThreads)
        out[i] += tile_sum[i / kScanTile];
}

// Every entry of A into its row's segment of A^T.  The entry's column (a
// column of A: at most 1024 of them) is found by binary search over A's
// column pointers held in shared memory.  cnt[r] counts down the free slots.
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_t_scatter(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
            const V* __restrict__ vals, int cols, int64_t nnz,
            const int64_t* __restrict__ t_ptr, int32_t* __restrict__ cnt,
            int32_t* __restrict__ tmp_idx, V* __restrict__ tmp_val) {
    __shared__ int64_t cp[kMaxM + 1];
    for (int i = threadIdx.x; i <= cols; i += kThreads) cp[i] = col_ptr[i];
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * kThreads) {
        int lo = 0, hi = cols;  // cp[lo] <= e < cp[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (cp[mid] <= e) lo = mid; else hi = mid;
        }
        const int r = row_idx[e];
        const int64_t pos = t_ptr[r] + atomicSub(cnt + r, 1) - 1;
        tmp_idx[pos] = lo;
        tmp_val[pos] = vals[e];
    }
}

// Place every scattered entry at its rank by column inside its segment.
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_t_order(const int64_t* __restrict__ t_ptr, int64_t rows, int64_t nnz,
          const int32_t* __restrict__ tmp_idx, const V* __restrict__ tmp_val,
          int32_t* __restrict__ t_idx, V* __restrict__ t_val) {
    for (int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x; q < nnz;
         q += (int64_t)gridDim.x * kThreads) {
        int64_t lo = 0, hi = rows;  // t_ptr[lo] <= q < t_ptr[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (t_ptr[mid] <= q) lo = mid; else hi = mid;
        }
        const int64_t s0 = t_ptr[lo], s1 = t_ptr[lo + 1];
        const int32_t c = tmp_idx[q];
        int64_t rank = 0;
        for (int64_t u = s0; u < s1; ++u) rank += tmp_idx[u] < c;
        t_idx[s0 + rank] = c;
        t_val[s0 + rank] = tmp_val[q];
    }
}

unsigned grid_for(int64_t n, int64_t cap) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kThreads), cap));
}

}  // namespace

size_t transpose_scratch_words(int64_t rows) { return (size_t)ceil_div(rows, kScanTile) + 1; }

cudaError_t launch_transpose_csc(const int64_t* col_ptr, const int32_t* row_idx, const void* vals,
                                 int value_type, int64_t rows, int cols, int64_t nnz,
                                 int32_t* cnt, int64_t* tile_sum, int32_t* tmp_idx,
                                 void* tmp_val, int64_t* t_ptr, int32_t* t_idx, void* t_val,
                                 cudaStream_t s) {
    if (cols < 1 || cols > kMaxM || rows < 1) return cudaErrorInvalidValue;
    const int64_t ntiles = ceil_div(rows, kScanTile);
    RK_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)rows, s));
    const unsigned ge = grid_for(nnz, 152 * 64);
    if (nnz > 0) k_t_count<<<ge, kThreads, 0, s>>>(row_idx, nnz, cnt);
    RK_CUDA_TRY(cudaGetLastError());
    k_t_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, s>>>(cnt, rows, t_ptr, tile_sum);
    RK_CUDA_TRY(cudaGetLastError());
    k_t_scan_totals<<<1, kScanThreads, 0, s>>>(tile_sum, ntiles, t_ptr, rows);
    RK_CUDA_TRY(cudaGetLastError());
    k_t_scan_add<<<grid_for(rows, 152 * 64), kThreads, 0, s>>>(t_ptr, rows, tile_sum);
    RK_CUDA_TRY(cudaGetLastError());
    if (nnz == 0) return cudaSuccess;
    if (value_type == 0) {
        k_t_scatter<float><<<ge, kThreads, 0, s>>>(col_ptr, row_idx,
                                                   static_cast<const float*>(vals), cols, nnz,
                                                   t_ptr, cnt, tmp_idx,
                                                   static_cast<float*>(tmp_val));
        RK_CUDA_TRY(cudaGetLastError());
        k_t_order<float><<<ge, kThreads, 0, s>>>(t_ptr, rows, nnz, tmp_idx,
                                                 static_cast<const float*>(tmp_val), t_idx,
                                                 static_cast<float*>(t_val));
    } else {
        k_t_scatter<double><<<ge, kThreads, 0, s>>>(col_ptr, row_idx,
                                                    static_cast<const double*>(vals), cols, nnz,
                                                    t_ptr, cnt, tmp_idx,
                                                    static_cast<double*>(tmp_val));
        RK_CUDA_TRY(cudaGetLastError());
        k_t_order<double><<<ge, kThreads, 0, s>>>(t_ptr, rows, nnz, tmp_idx,
                                                  static_cast<const double*>(tmp_val), t_idx,
                                                  static_cast<double*>(t_val));
    }
    return cudaGetLastError();
}

}  // namespace rk
