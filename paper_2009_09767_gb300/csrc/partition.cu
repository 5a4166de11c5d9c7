// partition.cu -- Algorithm 1 (column-block split, lonely-node scan) and
// Algorithm 2 (RandomChecker) of Ranky (arXiv 2009.09767, section III).
//
// The paper scans the dense index space (d, m, n) to find lonely nodes: rows
// with no non-zero inside block d.  Here one pass over the stored entries
// marks, per block, which rows are occupied (an M-bit set per block); a row
// is lonely in block d when its bit is clear there but set in some block
// (rows empty in all of A are not fixed: the paper assumes rank(A) = M).
#include "common.cuh"
#include "kernels.h"

namespace rk {

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC 2011):
// ten rounds of the two published multipliers, key advanced by the published
// Weyl increments between rounds.
__device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a = c[0], b = c[2];
        const uint32_t hi_a = __umulhi(0xD2511F53u, a), lo_a = 0xD2511F53u * a;
        const uint32_t hi_b = __umulhi(0xCD9E8D57u, b), lo_b = 0xCD9E8D57u * b;
        c[0] = hi_b ^ c[1] ^ k0;
        c[1] = lo_b;
        c[2] = hi_a ^ c[3] ^ k1;
        c[3] = lo_a;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// RandomChecker: "find a random column in block d" for lonely row m.  The draw
// is counted by (m, d) and keyed by the seed; the first output word is mapped
// onto the block's width by a 32.32 fixed-point multiply.
__device__ inline int64_t random_column(uint64_t seed, int d, int m, int64_t lo, int64_t w) {
    uint32_t c[4] = {(uint32_t)m, (uint32_t)d, 0u, 0u};
    philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    return lo + (int64_t)(((uint64_t)c[0] * (uint64_t)w) >> 32);
}

// ---------------------------------------------------------------------------
// Occupancy: one CTA per column chunk (chunks never straddle a block).  All
// entries of a chunk belong to one block, so the chunk is a contiguous slice
// of row_idx/vals that is streamed once, coalesced.  Each warp ORs into its
// own shared bit set; the warps' sets are merged and ORed into the block's
// global set at the end.
__global__ void __launch_bounds__(kThreads)
k_occupancy(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
            const void* __restrict__ vals, int value_type, int M,
            const int32_t* __restrict__ chunk_block, const int64_t* __restrict__ chunk_col_lo,
            const int64_t* __restrict__ chunk_col_hi, uint32_t* __restrict__ occ) {
    constexpr int kWarps = kThreads / 32;
    __shared__ uint32_t bits[kWarps][kMaxM / 32];
    const int W = (M + 31) >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = lane; i < W; i += 32) bits[warp][i] = 0u;
    __syncthreads();
    const int c = blockIdx.x;
    const int d = chunk_block[c];
    const int64_t e0 = col_ptr[chunk_col_lo[c]], e1 = col_ptr[chunk_col_hi[c]];
    if (value_type == 0) {
        const float* v = static_cast<const float*>(vals);
        for (int64_t e = e0 + threadIdx.x; e < e1; e += kThreads) {
            const int r = row_idx[e];
            if (v[e] != 0.0f) atomicOr(&bits[warp][r >> 5], 1u << (r & 31));
        }
    } else {
        const double* v = static_cast<const double*>(vals);
        for (int64_t e = e0 + threadIdx.x; e < e1; e += kThreads) {
            const int r = row_idx[e];
            if (v[e] != 0.0) atomicOr(&bits[warp][r >> 5], 1u << (r & 31));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += kThreads) {
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) acc |= bits[w][i];
        if (acc) atomicOr(&occ[(int64_t)d * W + i], acc);
    }
}

cudaError_t launch_occupancy(const int64_t* col_ptr, const int32_t* row_idx, const void* vals,
                             int value_type, int M, int nchunks, const int32_t* chunk_block,
                             const int64_t* chunk_col_lo, const int64_t* chunk_col_hi,
                             uint32_t* occ, cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    k_occupancy<<<nchunks, kThreads, 0, s>>>(col_ptr, row_idx, vals, value_type, M, chunk_block,
                                             chunk_col_lo, chunk_col_hi, occ);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Lonely flags and RandomChecker patches, one CTA of 1024 threads.  Words are
// numbered (d, w) block-major, each thread owns a contiguous run of words, so
// a block-wide exclusive scan of per-thread counts puts patches in (block,
// row) order.
__global__ void __launch_bounds__(1024)
k_lonely_patches(const uint32_t* __restrict__ occ, int D, int M, const int64_t* __restrict__ bounds,
                 int random, uint64_t seed, uint32_t* __restrict__ row_ne,
                 uint32_t* __restrict__ lonely, PatchRec* __restrict__ patches,
                 int64_t* __restrict__ patch_ofs, PatchRec* __restrict__ ext_patches,
                 int64_t* __restrict__ ext_npatches) {
    __shared__ uint32_t ne[kMaxM / 32];
    __shared__ int64_t scan[1024];
    const int W = (M + 31) >> 5;
    const uint32_t last_mask = (M & 31) ? ((1u << (M & 31)) - 1u) : 0xffffffffu;
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        uint32_t acc = 0;
        for (int d = 0; d < D; ++d) acc |= occ[(int64_t)d * W + i];
        ne[i] = acc;
        row_ne[i] = acc;
    }
    __syncthreads();
    const int64_t total_words = (int64_t)D * W;
    const int64_t per = (total_words + blockDim.x - 1) / blockDim.x;
    const int64_t w0 = min(total_words, (int64_t)threadIdx.x * per);
    const int64_t w1 = min(total_words, w0 + per);
    int64_t cnt = 0;
    for (int64_t gw = w0; gw < w1; ++gw) {
        const int w = (int)(gw % W);
        uint32_t lon = ~occ[gw] & ne[w];
        if (w == W - 1) lon &= last_mask;
        lonely[gw] = lon;
        cnt += __popc(lon);
    }
    scan[threadIdx.x] = cnt;
    __syncthreads();
    // inclusive Hillis-Steele scan over 1024 counts
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        int64_t add = threadIdx.x >= (unsigned)off ? scan[threadIdx.x - off] : 0;
        __syncthreads();
        scan[threadIdx.x] += add;
        __syncthreads();
    }
    const int64_t total = scan[blockDim.x - 1];
    int64_t pos = scan[threadIdx.x] - cnt;
    if (!random) {
        if (threadIdx.x == 0) {
            for (int d = 0; d <= D; ++d) patch_ofs[d] = 0;
            if (ext_npatches) *ext_npatches = 0;
        }
        return;
    }
    for (int64_t gw = w0; gw < w1; ++gw) {
        const int d = (int)(gw / W), w = (int)(gw % W);
        if (w == 0) patch_ofs[d] = pos;
        uint32_t lon = lonely[gw];
        const int64_t lo = bounds[d], width = bounds[d + 1] - bounds[d];
        while (lon) {
            const int bit = __ffs(lon) - 1;
            lon &= lon - 1;
            const int m = w * 32 + bit;
            PatchRec p;
            p.row = m;
            p.block = d;
            p.col = random_column(seed, d, m, lo, width);
            patches[pos] = p;
            if (ext_patches) ext_patches[pos] = p;
            ++pos;
        }
    }
    if (threadIdx.x == 0) {
        patch_ofs[D] = total;
        if (ext_npatches) *ext_npatches = total;
    }
}

cudaError_t launch_lonely_patches(const uint32_t* occ, int D, int M, const int64_t* bounds,
                                  int random, uint64_t seed, uint32_t* row_ne, uint32_t* lonely,
                                  PatchRec* patches, int64_t* patch_ofs, PatchRec* ext_patches,
                                  int64_t* ext_npatches, cudaStream_t s) {
    k_lonely_patches<<<1, 1024, 0, s>>>(occ, D, M, bounds, random, seed, row_ne, lonely, patches,
                                        patch_ofs, ext_patches, ext_npatches);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CSC structure check: one thread per column.
__global__ void k_check_csc(int M, int64_t N, int64_t nnz, const int64_t* __restrict__ col_ptr,
                            const int32_t* __restrict__ row_idx, int32_t* bad) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0 && (col_ptr[0] != 0 || col_ptr[N] != nnz)) atomicOr(bad, 1);
    if (j >= N) return;
    const int64_t a = col_ptr[j], b = col_ptr[j + 1];
    if (a > b || a < 0 || b > nnz) { atomicOr(bad, 2); return; }
    int prev = -1;
    for (int64_t e = a; e < b; ++e) {
        const int r = row_idx[e];
        if (r < 0 || r >= M) { atomicOr(bad, 4); return; }
        if (r <= prev) { atomicOr(bad, 8); return; }
        prev = r;
    }
}

cudaError_t launch_check_csc(int M, int64_t N, int64_t nnz, const int64_t* col_ptr,
                             const int32_t* row_idx, int32_t* bad, cudaStream_t s) {
    const int64_t blocks = ceil_div(N, kThreads);
    k_check_csc<<<(unsigned)blocks, kThreads, 0, s>>>(M, N, nnz, col_ptr, row_idx, bad);
    return cudaGetLastError();
}

}  // namespace rk
