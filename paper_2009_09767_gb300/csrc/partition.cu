// partition.cu -- Algorithm 1 (column-block split, lonely-node scan) and
// Algorithm 2 (RandomChecker) of Ranky (arXiv 2009.09767, section III).
//
// The paper scans the dense index space (d, m, n) to find lonely nodes: rows
// with no non-zero inside block d.  Here one pass over the stored entries
// marks, per block, which rows are occupied (an M-bit set per block); a row
// is lonely in block d when its bit is clear there but set in some block
// (rows empty in all of A are not fixed: the paper assumes rank(A) = M).
#include <algorithm>

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
// Lonely flags and rank-fix slots, one CTA of 1024 threads.  Words are
// numbered (d, w) block-major, each thread owns a contiguous run of words, so
// a block-wide exclusive scan of per-thread counts puts the lonely nodes in
// (block, row) order.  mode 0: flags only; 1: RandomChecker patches; 2: one
// slot per lonely node with col = -1 (filled by the neighbour pick) and
// lonely_any = rows lonely in some block.
__global__ void __launch_bounds__(1024)
k_lonely_patches(const uint32_t* __restrict__ occ, int D, int M, const int64_t* __restrict__ bounds,
                 int mode, uint64_t seed, uint32_t* __restrict__ row_ne,
                 uint32_t* __restrict__ lonely, PatchRec* __restrict__ patches,
                 int64_t* __restrict__ patch_ofs, PatchRec* __restrict__ ext_patches,
                 int64_t* __restrict__ ext_npatches, uint32_t* __restrict__ lonely_any) {
    __shared__ uint32_t ne[kMaxM / 32];
    __shared__ int64_t scan[1024];
    const int W = (M + 31) >> 5;
    const uint32_t last_mask = (M & 31) ? ((1u << (M & 31)) - 1u) : 0xffffffffu;
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        uint32_t acc = 0, all = 0xffffffffu;
        for (int d = 0; d < D; ++d) {
            const uint32_t o = occ[(int64_t)d * W + i];
            acc |= o;
            all &= o;
        }
        ne[i] = acc;
        row_ne[i] = acc;
        if (lonely_any) lonely_any[i] = acc & ~all;
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
    if (mode == 0) {
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
            p.col = mode == 1 ? random_column(seed, d, m, lo, width) : -1;
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
                                  int mode, uint64_t seed, uint32_t* row_ne, uint32_t* lonely,
                                  PatchRec* patches, int64_t* patch_ofs, PatchRec* ext_patches,
                                  int64_t* ext_npatches, uint32_t* lonely_any, cudaStream_t s) {
    k_lonely_patches<<<1, 1024, 0, s>>>(occ, D, M, bounds, mode, seed, row_ne, lonely, patches,
                                        patch_ofs, ext_patches, ext_npatches, lonely_any);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// NeighborChecker (Algorithm 3) and neighbourRandomChecker (Algorithm 4).
//
// For lonely row m of block d the algorithm lists, once per shared column,
// every row c that is non-zero beside m in another block, then, once per
// list entry, every column of block d where c is non-zero, and inserts a 1
// at a column drawn from that multiset.  Row m has no entry in block d, so c
// is listed C[m][c] times, C the co-occurrence counts of the rows over all
// columns, and column n of block d is listed w(n) = sum of C[m][c] over the
// stored non-zeros (c, n).  The pick needs row m of C and one pass over
// block d's entries.  The 64-bit Philox word x of counter (m, d, 1, 0)
// selects entry r = floor(x T / 2^64), T = sum w, of the list ordered by
// column: the column where the running sum of w first exceeds r.  Every list
// is formed from the input A (an insertion never feeds another node's list).
// An empty list gives no insertion, or, for neighbourRandomChecker, the
// RandomChecker column.

__device__ inline bool nonzero_at(const void* vals, int vt, int64_t e) {
    return vt == 0 ? static_cast<const float*>(vals)[e] != 0.0f
                   : static_cast<const double*>(vals)[e] != 0.0;
}

__device__ inline bool bit_set(const uint32_t* bits, int r) { return (bits[r >> 5] >> (r & 31)) & 1u; }

// C[a][b] += 1 for every column where rows a and b are both non-zero, for the
// rows a lonely in some block (other rows of C are not formed).  A thread per
// column; columns longer than kLightCooc entries are queued and taken by a
// warp each.
constexpr int kLightCooc = 32;

__global__ void __launch_bounds__(kThreads)
k_row_cooc(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
           const void* __restrict__ vals, int vt, int64_t N, int M,
           const uint32_t* __restrict__ lonely_any, unsigned long long* __restrict__ C) {
    __shared__ int64_t heavy[kThreads];
    __shared__ int nheavy;
    if (threadIdx.x == 0) nheavy = 0;
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (j < N) {
        const int64_t e0 = col_ptr[j], e1 = col_ptr[j + 1];
        if (e1 - e0 > kLightCooc) {
            heavy[atomicAdd(&nheavy, 1)] = j;
        } else {
            for (int64_t a = e0; a < e1; ++a) {
                const int ra = row_idx[a];
                if (!bit_set(lonely_any, ra) || !nonzero_at(vals, vt, a)) continue;
                unsigned long long* Crow = C + (int64_t)ra * M;
                for (int64_t b = e0; b < e1; ++b)
                    if (nonzero_at(vals, vt, b)) atomicAdd(Crow + row_idx[b], 1ull);
            }
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int h = warp; h < nheavy; h += kThreads / 32) {
        const int64_t jj = heavy[h];
        const int64_t e0 = col_ptr[jj], e1 = col_ptr[jj + 1];
        for (int64_t a = e0; a < e1; ++a) {
            const int ra = row_idx[a];
            if (!bit_set(lonely_any, ra) || !nonzero_at(vals, vt, a)) continue;
            unsigned long long* Crow = C + (int64_t)ra * M;
            for (int64_t b = e0 + lane; b < e1; b += 32)
                if (nonzero_at(vals, vt, b)) atomicAdd(Crow + row_idx[b], 1ull);
        }
    }
}

// Exclusive prefix sum over the CTA (kThreads threads, one value each) and
// the CTA total.  warp_tot: kThreads/32 words of shared memory.
__device__ inline unsigned long long cta_exclusive_scan(unsigned long long v,
                                                        unsigned long long* warp_tot,
                                                        unsigned long long& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned long long before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
        const unsigned long long t = warp_tot[w];
        if (w < warp) before += t;
        all += t;
    }
    __syncthreads();
    total = all;
    return before + incl - v;
}

// One CTA per slot (persistent over the slots): row m's counts in shared
// memory, each thread sums the weights of a contiguous run of block d's
// entries, a CTA scan places the runs, and the thread whose run holds entry
// r finds it and its column (binary search over col_ptr).
__global__ void __launch_bounds__(kThreads)
k_neighbor_pick(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                const void* __restrict__ vals, int vt, int M, int D,
                const int64_t* __restrict__ bounds, const unsigned long long* __restrict__ C,
                int fallback, uint64_t seed, PatchRec* __restrict__ slots,
                const int64_t* __restrict__ slot_ofs) {
    __shared__ unsigned long long crow[kMaxM];
    __shared__ unsigned long long warp_tot[kThreads / 32];
    const int64_t nslots = slot_ofs[D];
    for (int64_t sl = blockIdx.x; sl < nslots; sl += gridDim.x) {
        const int m = slots[sl].row, d = slots[sl].block;
        for (int i = threadIdx.x; i < M; i += kThreads) crow[i] = C[(int64_t)m * M + i];
        __syncthreads();
        const int64_t lo = bounds[d], hi = bounds[d + 1];
        const int64_t e0 = col_ptr[lo], e1 = col_ptr[hi];
        const int64_t per = ceil_div(e1 - e0, kThreads);
        const int64_t a = min(e1, e0 + (int64_t)threadIdx.x * per), b = min(e1, a + per);
        unsigned long long w = 0;
        for (int64_t e = a; e < b; ++e)
            if (nonzero_at(vals, vt, e)) w += crow[row_idx[e]];
        unsigned long long T;
        const unsigned long long before = cta_exclusive_scan(w, warp_tot, T);
        if (T == 0) {
            if (threadIdx.x == 0) slots[sl].col = fallback ? random_column(seed, d, m, lo, hi - lo) : -1;
        } else {
            uint32_t c[4] = {(uint32_t)m, (uint32_t)d, 1u, 0u};
            philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
            const unsigned long long x = (unsigned long long)c[0] | ((unsigned long long)c[1] << 32);
            const unsigned long long r = __umul64hi(x, T);
            if (r >= before && r - before < w) {
                unsigned long long acc = before;
                int64_t hit = a;
                for (int64_t e = a; e < b; ++e) {
                    if (!nonzero_at(vals, vt, e)) continue;
                    acc += crow[row_idx[e]];
                    if (acc > r) { hit = e; break; }
                }
                int64_t jl = lo, jh = hi;  // col_ptr[jl] <= hit < col_ptr[jh]
                while (jh - jl > 1) {
                    const int64_t mid = (jl + jh) >> 1;
                    if (col_ptr[mid] <= hit) jl = mid; else jh = mid;
                }
                slots[sl].col = jl;
            }
        }
        __syncthreads();  // crow is reloaded for the next slot
    }
}

// Drop the empty slots (col < 0), keeping (block, row) order; patch_ofs[d] =
// patches before block d.  One CTA of 1024 threads, contiguous slot runs.
__global__ void __launch_bounds__(1024)
k_patch_compact(const PatchRec* __restrict__ slots, const int64_t* __restrict__ slot_ofs, int D,
                PatchRec* __restrict__ patches, int64_t* __restrict__ patch_ofs,
                PatchRec* __restrict__ ext_patches, int64_t* __restrict__ ext_npatches) {
    __shared__ int64_t scan[1024];
    const int64_t n = slot_ofs[D];
    const int64_t per = ceil_div(n, 1024);
    const int64_t a = min(n, (int64_t)threadIdx.x * per), b = min(n, a + per);
    int64_t cnt = 0;
    for (int64_t i = a; i < b; ++i) cnt += slots[i].col >= 0;
    scan[threadIdx.x] = cnt;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int64_t add = threadIdx.x >= (unsigned)off ? scan[threadIdx.x - off] : 0;
        __syncthreads();
        scan[threadIdx.x] += add;
        __syncthreads();
    }
    const int64_t total = scan[1023];
    int64_t pos = scan[threadIdx.x] - cnt;
    for (int64_t i = a; i < b; ++i) {
        const PatchRec p = slots[i];
        if (p.col < 0) continue;
        patches[pos] = p;
        if (ext_patches) ext_patches[pos] = p;
        ++pos;
    }
    for (int d = threadIdx.x; d <= D; d += 1024) {
        const int64_t q = slot_ofs[d];
        int64_t v = total;
        if (q < n) {
            const int t = (int)(q / per);
            v = t ? scan[t - 1] : 0;
            for (int64_t i = (int64_t)t * per; i < q; ++i) v += slots[i].col >= 0;
        }
        patch_ofs[d] = v;
    }
    if (threadIdx.x == 0 && ext_npatches) *ext_npatches = total;
}

cudaError_t launch_neighbor_patches(const int64_t* col_ptr, const int32_t* row_idx,
                                    const void* vals, int value_type, int M, int64_t N, int D,
                                    const int64_t* bounds, const uint32_t* lonely_any,
                                    unsigned long long* cooc, int fallback, uint64_t seed,
                                    PatchRec* slots, const int64_t* slot_ofs, PatchRec* patches,
                                    int64_t* patch_ofs, PatchRec* ext_patches,
                                    int64_t* ext_npatches, cudaStream_t s) {
    RK_CUDA_TRY(cudaMemsetAsync(cooc, 0, sizeof(unsigned long long) * (size_t)M * M, s));
    k_row_cooc<<<(unsigned)ceil_div(N, kThreads), kThreads, 0, s>>>(col_ptr, row_idx, vals,
                                                                      value_type, N, M,
                                                                      lonely_any, cooc);
    RK_CUDA_TRY(cudaGetLastError());
    int dev = 0, sms = 152;
    RK_CUDA_TRY(cudaGetDevice(&dev));
    RK_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t grid = std::min<int64_t>((int64_t)D * M, (int64_t)sms * 8);
    k_neighbor_pick<<<(unsigned)std::max<int64_t>(grid, 1), kThreads, 0, s>>>(
        col_ptr, row_idx, vals, value_type, M, D, bounds, cooc, fallback, seed, slots, slot_ofs);
    RK_CUDA_TRY(cudaGetLastError());
    k_patch_compact<<<1, 1024, 0, s>>>(slots, slot_ofs, D, patches, patch_ofs, ext_patches,
                                       ext_npatches);
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
