// static_scratch.cu -- right singular vectors without any device allocation.
//
// svd_right_vectors_static computes V = A'^T U_k S_k^-1 (the last stage of
// svd_run) from singular values and left vectors the caller already holds.
// Its only scratch, the weights W = U_k S_k^-1, lives in a file-scope device
// array instead of memory from cudaMalloc.  It exists for callers that must
// not allocate device memory on their call path: services that carve the GPU
// into fixed budgets at start-up and refuse any allocation afterwards, and
// latency-bound callers that cannot afford cudaMalloc's implicit device-wide
// synchronisation or its failure under memory pressure.
//
// Limits and sharing rules (also stated in include/ranky.h):
//   * the array holds kStaticScratchBytes; M * k * sizeof(element of V) above
//     that is rejected with SVD_ERR_UNSUPPORTED before any work is enqueued;
//   * every GPU that loads the library keeps the array until the process
//     exits;
//   * all calls on a device share the one array and it keeps the last call's
//     contents; each call rewrites every weight it reads, so nothing needs
//     clearing, but calls whose kernels overlap on the GPU (different streams
//     without ordering between them) race on the array;
//   * the first call on each device looks up the array's device address with
//     cudaGetSymbolAddress (a host-side name of a __device__ variable is not a
//     device address); make that first call before any stream capture.
#include <algorithm>
#include <mutex>

#include "../../include/ranky.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)4 << 20;   // 4 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// W[m][i] = U[m, i] / sigma_i where sigma_i^2 is above the rank tolerance,
// else 0 (the same rule svd_run applies: rank_tol^2 when rank_tol > 0, else
// max(M, N) * eps64 * sigma_1^2).  U is column-major M x k.
template <typename T>
__global__ void k_weights_static(const double* __restrict__ sigma, const double* __restrict__ U,
                                 int M, int k, double lam_tol_abs, int64_t tol_scale,
                                 T* __restrict__ W) {
    const double s1 = sigma[0];
    const double tau = lam_tol_abs > 0.0 ? lam_tol_abs
                                         : (double)tol_scale * 2.220446049250313e-16 * s1 * s1;
    const int64_t n = (int64_t)M * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e / k), i = (int)(e % k);
        const double si = sigma[i];
        W[e] = si * si > tau ? (T)(U[(int64_t)i * M + m] / si) : (T)0;
    }
}

template <typename T>
cudaError_t run_static(int M, int64_t N, int value_type, const int64_t* col_ptr,
                       const int32_t* row_idx, const void* vals, int k, const double* sigma,
                       const double* U, double rank_tol, const svd_patch* patches,
                       const int64_t* npatches, int max_patches, T* V, cudaStream_t s) {
    void* addr = nullptr;
    cudaError_t e = scratch_address(&addr);
    if (e != cudaSuccess) return e;
    T* W = static_cast<T*>(addr);
    const int64_t n = (int64_t)M * k;
    const int grid = (int)std::min<int64_t>(rk::ceil_div(n, 256), 1024);
    const double lam_abs = rank_tol > 0 ? rank_tol * rank_tol : 0.0;
    const int64_t tol_scale = (int64_t)M > N ? (int64_t)M : N;
    k_weights_static<T><<<grid, 256, 0, s>>>(sigma, U, M, k, lam_abs, tol_scale, W);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = rk::launch_spmm<T>(col_ptr, row_idx, vals, value_type, N, k, W, V, s);
    if (e != cudaSuccess) return e;
    if (patches && npatches && max_patches > 0)
        e = rk::launch_spmm_patches<T>(reinterpret_cast<const rk::PatchRec*>(patches), npatches,
                                       max_patches, k, W, V, s);
    return e;
}

}  // namespace

extern "C" svd_status svd_right_vectors_static(int32_t M, int64_t N, int64_t nnz,
                                               int32_t value_type, const int64_t* d_col_ptr,
                                               const int32_t* d_row_idx, const void* d_vals,
                                               int32_t k, const double* d_sigma,
                                               const double* d_U, double rank_tol,
                                               const svd_patch* d_patches,
                                               const int64_t* d_npatches, int64_t max_patches,
                                               int32_t v_type, void* d_V, void* stream) {
    if (M < 1 || N < 1 || nnz < 0 || k < 1 || k > M || (int64_t)k > N) return SVD_ERR_INVALID_ARG;
    if (value_type != SVD_VALUE_F32 && value_type != SVD_VALUE_F64) return SVD_ERR_INVALID_ARG;
    if (v_type != SVD_VALUE_F32 && v_type != SVD_VALUE_F64) return SVD_ERR_INVALID_ARG;
    if (!d_col_ptr || !d_sigma || !d_U || !d_V || (nnz > 0 && (!d_row_idx || !d_vals)))
        return SVD_ERR_INVALID_ARG;
    if ((d_patches == nullptr) != (d_npatches == nullptr) || max_patches < 0 ||
        max_patches > (int64_t)1 << 30)
        return SVD_ERR_INVALID_ARG;
    const size_t elem = v_type == SVD_VALUE_F32 ? sizeof(float) : sizeof(double);
    if ((size_t)M * (size_t)k * elem > kStaticScratchBytes) return SVD_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (v_type == SVD_VALUE_F32)
        e = run_static<float>(M, N, value_type, d_col_ptr, d_row_idx, d_vals, k, d_sigma, d_U,
                              rank_tol, d_patches, d_npatches, (int)max_patches,
                              static_cast<float*>(d_V), s);
    else
        e = run_static<double>(M, N, value_type, d_col_ptr, d_row_idx, d_vals, k, d_sigma, d_U,
                               rank_tol, d_patches, d_npatches, (int)max_patches,
                               static_cast<double*>(d_V), s);
    return e == cudaSuccess ? SVD_OK : SVD_ERR_CUDA;
}
