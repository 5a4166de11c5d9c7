// gram.cu -- block cross products A'^i A'^i^T in FP64 (Ranky, arXiv
// 2009.09767, Eq. 2: the quantity the proxy matrix reproduces).
//
// A column a_j adds the outer product a_j a_j^T, so a block's cross product
// costs sum_j k_j (k_j + 1) / 2 multiply-adds over its columns of k_j
// entries: the work that sparsity leaves, none of the dense M x w product.
// One CTA streams a column chunk (all in one block) and scatters the
// upper-triangle products of its columns with FP64 atomic adds into the
// block's M x M matrix (row-major, padded to Mp).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rk {

// Columns with up to kLight entries are taken by one thread each (their
// k (k + 1) / 2 products issued back to back); longer ones are queued and
// taken by a warp each, lanes over the second index.
namespace {
constexpr int kLight = 32;
}

__global__ void __launch_bounds__(kThreads)
k_gram(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
       const void* __restrict__ vals, int value_type, int Mp,
       const int32_t* __restrict__ chunk_block, const int64_t* __restrict__ chunk_col_lo,
       const int64_t* __restrict__ chunk_col_hi, double* __restrict__ G) {
    __shared__ int64_t heavy[kThreads * 4];
    __shared__ int nheavy;
    const int c = blockIdx.x;
    const int d = chunk_block[c];
    double* Gd = G + (int64_t)d * Mp * Mp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kThreads / 32;
    if (threadIdx.x == 0) nheavy = 0;
    __syncthreads();
    const int64_t lo = chunk_col_lo[c], hi = chunk_col_hi[c];
    for (int64_t j = lo + threadIdx.x; j < hi; j += kThreads) {
        const int64_t e0 = col_ptr[j], e1 = col_ptr[j + 1];
        if (e1 - e0 > kLight) {
            const int h = atomicAdd(&nheavy, 1);
            if (h < kThreads * 4) { heavy[h] = j; continue; }
        }
        for (int64_t a = e0; a < e1; ++a) {
            const double va = load_val(vals, value_type, a);
            if (va == 0.0) continue;
            double* row = Gd + (int64_t)row_idx[a] * Mp;
            for (int64_t b = a; b < e1; ++b) {
                const double vb = load_val(vals, value_type, b);
                if (vb != 0.0) atomicAdd(row + row_idx[b], va * vb);
            }
        }
    }
    __syncthreads();
    const int nh = min(nheavy, kThreads * 4);
    for (int h = warp; h < nh; h += kWarps) {
        const int64_t j = heavy[h];
        const int64_t e0 = col_ptr[j], e1 = col_ptr[j + 1];
        for (int64_t a = e0; a < e1; ++a) {
            const int ra = row_idx[a];
            const double va = load_val(vals, value_type, a);
            if (va == 0.0) continue;
            double* row = Gd + (int64_t)ra * Mp;
            for (int64_t b = a + lane; b < e1; b += 32) {
                const double vb = load_val(vals, value_type, b);
                if (vb != 0.0) atomicAdd(row + row_idx[b], va * vb);
            }
        }
    }
}

cudaError_t launch_gram(const int64_t* col_ptr, const int32_t* row_idx, const void* vals,
                        int value_type, int Mp, int nchunks, const int32_t* chunk_block,
                        const int64_t* chunk_col_lo, const int64_t* chunk_col_hi, double* G,
                        cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    k_gram<<<nchunks, kThreads, 0, s>>>(col_ptr, row_idx, vals, value_type, Mp, chunk_block,
                                        chunk_col_lo, chunk_col_hi, G);
    return cudaGetLastError();
}

// RandomChecker insertions: column col of block d becomes a + sum_i e_{m_i}
// over the patches (m_i, col).  Its outer product gains a e_m^T + e_m a^T for
// each patch, e_m e_m^T, and e_{m_i} e_{m_j}^T for each pair of patches that
// share the column.  One warp per patch.
__global__ void __launch_bounds__(kThreads)
k_gram_patches(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
               const void* __restrict__ vals, int value_type, int Mp, int D,
               const PatchRec* __restrict__ patches, const int64_t* __restrict__ patch_ofs,
               int max_patches, double* __restrict__ G) {
    const int64_t total = patch_ofs[D];
    const int64_t i = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= total) return;
    const PatchRec p = patches[i];
    double* Gd = G + (int64_t)p.block * Mp * Mp;
    const int m = p.row;
    if (lane == 0) atomicAdd(Gd + (int64_t)m * Mp + m, 1.0);
    const int64_t e0 = col_ptr[p.col], e1 = col_ptr[p.col + 1];
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        const int r = row_idx[e];
        const double v = load_val(vals, value_type, e);
        if (v == 0.0) continue;
        if (r == m) {
            atomicAdd(Gd + (int64_t)m * Mp + m, 2.0 * v);
        } else {
            const int lo = min(r, m), hi = max(r, m);
            atomicAdd(Gd + (int64_t)lo * Mp + hi, v);
        }
    }
    const int64_t q0 = patch_ofs[p.block], q1 = patch_ofs[p.block + 1];
    for (int64_t q = i + 1 + lane; q < q1; q += 32) {
        const PatchRec o = patches[q];
        if (o.col == p.col) {
            const int lo = min(o.row, m), hi = max(o.row, m);
            atomicAdd(Gd + (int64_t)lo * Mp + hi, 1.0);
        }
    }
    (void)q0;
}

cudaError_t launch_gram_patches(const int64_t* col_ptr, const int32_t* row_idx, const void* vals,
                                int value_type, int Mp, int D, const PatchRec* patches,
                                const int64_t* patch_ofs, int max_patches, double* G,
                                cudaStream_t s) {
    if (max_patches <= 0) return cudaSuccess;
    const int64_t blocks = ceil_div((int64_t)max_patches * 32, kThreads);
    k_gram_patches<<<(unsigned)blocks, kThreads, 0, s>>>(col_ptr, row_idx, vals, value_type, Mp, D,
                                                         patches, patch_ofs, max_patches, G);
    return cudaGetLastError();
}

__global__ void k_symmetrize(double* __restrict__ G, int Mp) {
    double* Gm = G + (int64_t)blockIdx.y * Mp * Mp;
    const int64_t n = (int64_t)Mp * Mp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / Mp), j = (int)(e % Mp);
        if (i > j) Gm[e] = Gm[(int64_t)j * Mp + i];
    }
}

cudaError_t launch_symmetrize(double* G, int nmat, int Mp, cudaStream_t s) {
    const int64_t n = (int64_t)Mp * Mp;
    const int bx = (int)std::min<int64_t>(ceil_div(n, kThreads), 1024);
    k_symmetrize<<<dim3(bx, nmat), kThreads, 0, s>>>(G, Mp);
    return cudaGetLastError();
}

template <typename S, typename D>
__global__ void k_convert(const S* __restrict__ src, D* __restrict__ dst, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = (D)src[e];
}

cudaError_t launch_convert_f64_f32(const double* src, float* dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int bx = (int)std::min<int64_t>(ceil_div(n, kThreads), 4096);
    k_convert<double, float><<<bx, kThreads, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_convert_f32_f64(const float* src, double* dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int bx = (int)std::min<int64_t>(ceil_div(n, kThreads), 4096);
    k_convert<float, double><<<bx, kThreads, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace rk
