// spmm.cu -- right singular vectors V = A'^T U_k S_k^-1 (the paper lists the
// right vectors as future work, section V; they follow from A' = U S V^T).
//
// Row j of V (k contiguous values) is the combination of the rows of
// W = U_k S_k^-1 picked by column j's entries: V[j,:] = sum_e a_e W[row_e,:].
// One warp owns a column; each lane holds 16-byte slices of the output row,
// so a warp writes 512 contiguous bytes per store with streaming stores (V is
// written once and never re-read).  W (M x k) stays in L2 / L1.  The kernel
// is bound by the store of V: N * k * sizeof(T) bytes.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rk {

namespace {

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ void fma_vec(typename Vec<T>::type& acc, T a, const typename Vec<T>::type& w);
template <>
__device__ __forceinline__ void fma_vec<float>(float4& acc, float a, const float4& w) {
    acc.x = fmaf(a, w.x, acc.x); acc.y = fmaf(a, w.y, acc.y);
    acc.z = fmaf(a, w.z, acc.z); acc.w = fmaf(a, w.w, acc.w);
}
template <>
__device__ __forceinline__ void fma_vec<double>(double2& acc, double a, const double2& w) {
    acc.x = fma(a, w.x, acc.x); acc.y = fma(a, w.y, acc.y);
}

template <typename T, typename VT>
__device__ __forceinline__ T load_as(const void* vals, int64_t e) {
    return (T) static_cast<const VT*>(vals)[e];
}

// vector path: k % Vec<T>::n == 0 and k / Vec<T>::n <= 32 CPL.  A warp
// loads up to 32 of the column's entries at once (one per lane) and
// broadcasts them; each lane accumulates its CPL slices of the output row in
// one pass over the entries, so every W load of an entry issues together and
// a column costs a few dependent memory trips, not one per slice.
template <typename T, typename VT, int CPL>
__global__ void __launch_bounds__(256)
k_spmm_vec(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
           const void* __restrict__ vals, int64_t N, int k, const T* __restrict__ W,
           T* __restrict__ V) {
    using V4 = typename Vec<T>::type;
    constexpr int NV = Vec<T>::n;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int kv = k / NV;                 // vectors per row
    for (int64_t j = warp; j < N; j += nwarps) {
        const int64_t e0 = col_ptr[j], e1 = col_ptr[j + 1];
        V4 acc[CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            if constexpr (NV == 4) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            else acc[q] = make_double2(0.0, 0.0);
        }
        for (int64_t eb = e0; eb < e1; eb += 32) {
            const int n = (int)min((int64_t)32, e1 - eb);
            int my_r = 0;
            T my_a = T(0);
            if (lane < n) {
                my_r = __ldg(row_idx + eb + lane);
                my_a = load_as<T, VT>(vals, eb + lane);
            }
            for (int i = 0; i < n; ++i) {
                const int r = __shfl_sync(0xffffffffu, my_r, i);
                const T a = __shfl_sync(0xffffffffu, my_a, i);
                const V4* wr = reinterpret_cast<const V4*>(W + (int64_t)r * k);
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    const int c = lane + 32 * q;
                    if (c < kv) fma_vec<T>(acc[q], a, __ldg(wr + c));
                }
            }
        }
        V4* out = reinterpret_cast<V4*>(V + j * (int64_t)k);
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const int c = lane + 32 * q;
            if (c < kv) __stcs(out + c, acc[q]);
        }
    }
}

template <typename T, typename VT>
__global__ void __launch_bounds__(256)
k_spmm_scalar(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
              const void* __restrict__ vals, int64_t N, int k, const T* __restrict__ W,
              T* __restrict__ V) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = warp; j < N; j += nwarps) {
        const int64_t e0 = col_ptr[j], e1 = col_ptr[j + 1];
        for (int c = lane; c < k; c += 32) {
            T acc = T(0);
            for (int64_t e = e0; e < e1; ++e) {
                const int r = __ldg(row_idx + e);
                acc += load_as<T, VT>(vals, e) * __ldg(W + (int64_t)r * k + c);
            }
            __stcs(V + j * (int64_t)k + c, acc);
        }
    }
}

template <typename T>
__global__ void k_spmm_patches(const PatchRec* __restrict__ patches, const int64_t* __restrict__ np,
                               int k, const T* __restrict__ W, T* __restrict__ V) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= *np) return;
    const PatchRec p = patches[i];
    for (int c = lane; c < k; c += 32)
        atomicAdd(V + p.col * (int64_t)k + c, W[(int64_t)p.row * k + c]);
}

}  // namespace

template <typename T>
cudaError_t launch_spmm(const int64_t* col_ptr, const int32_t* row_idx, const void* vals,
                        int value_type, int64_t N, int k, const T* W, T* V, cudaStream_t s) {
    if (N <= 0 || k <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = ceil_div(N * 32, 256);
    const int grid = (int)std::min<int64_t>(want, (int64_t)sms * 16);
    const int kv = (k % Vec<T>::n) == 0 ? k / Vec<T>::n : -1;
    auto go = [&](auto vt_tag) {
        using VT = decltype(vt_tag);
        if (kv > 0 && kv <= 32) k_spmm_vec<T, VT, 1><<<grid, 256, 0, s>>>(col_ptr, row_idx, vals, N, k, W, V);
        else if (kv > 0 && kv <= 64) k_spmm_vec<T, VT, 2><<<grid, 256, 0, s>>>(col_ptr, row_idx, vals, N, k, W, V);
        else if (kv > 0 && kv <= 128) k_spmm_vec<T, VT, 4><<<grid, 256, 0, s>>>(col_ptr, row_idx, vals, N, k, W, V);
        else if (kv > 0 && kv <= 256) k_spmm_vec<T, VT, 8><<<grid, 256, 0, s>>>(col_ptr, row_idx, vals, N, k, W, V);
        else k_spmm_scalar<T, VT><<<grid, 256, 0, s>>>(col_ptr, row_idx, vals, N, k, W, V);
    };
    if (value_type == 0) go(float{});
    else go(double{});
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spmm_patches(const PatchRec* patches, const int64_t* npatches_dev,
                                int max_patches, int k, const T* W, T* V, cudaStream_t s) {
    if (max_patches <= 0 || k <= 0) return cudaSuccess;
    const int64_t blocks = ceil_div((int64_t)max_patches * 32, 256);
    k_spmm_patches<T><<<(unsigned)blocks, 256, 0, s>>>(patches, npatches_dev, k, W, V);
    return cudaGetLastError();
}

template cudaError_t launch_spmm<float>(const int64_t*, const int32_t*, const void*, int, int64_t,
                                        int, const float*, float*, cudaStream_t);
template cudaError_t launch_spmm<double>(const int64_t*, const int32_t*, const void*, int, int64_t,
                                         int, const double*, double*, cudaStream_t);
template cudaError_t launch_spmm_patches<float>(const PatchRec*, const int64_t*, int, int,
                                                const float*, float*, cudaStream_t);
template cudaError_t launch_spmm_patches<double>(const PatchRec*, const int64_t*, int, int,
                                                 const double*, double*, cudaStream_t);

}  // namespace rk
