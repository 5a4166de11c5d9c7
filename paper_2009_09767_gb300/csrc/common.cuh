// common.cuh -- shared device helpers of the sm_103a column-block SVD.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define RK_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return _e;                   \
    } while (0)

namespace rk {

constexpr int kMaxM = 1024;          // rows supported by the block kernels
constexpr int kThreads = 256;

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double value = 5.9604644775390625e-8; };   // 2^-24
template <> struct Eps<double> { static constexpr double value = 1.1102230246251565e-16; }; // 2^-53

__device__ inline double load_val(const void* vals, int value_type, int64_t e) {
    return value_type == 0 ? (double)static_cast<const float*>(vals)[e]
                           : static_cast<const double*>(vals)[e];
}

// Block of column j given D+1 boundaries (binary search, boundaries sorted).
__device__ inline int block_of(const int64_t* bounds, int D, int64_t j) {
    int lo = 0, hi = D;  // invariant bounds[lo] <= j < bounds[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (bounds[mid] <= j) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace rk
