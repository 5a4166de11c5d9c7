// dense.cu -- FP64 dense stages of the column-block SVD (Ranky, arXiv
// 2009.09767): batched products, the eigenbasis refinement used by the mixed
// precision mode, eigenvalue sort and numerical rank, the proxy matrix
// P = [U^1 S^1 | ... | U^D S^D] (section III) and its cross product P P^T
// (Eq. 3), and the final outputs.
//
// FP64 arithmetic on this part runs on the FP64 pipes, whose rate is far below
// the FP32 one, so every product here is compute-bound at any tile shape that
// keeps the operands in shared memory.
#include <cooperative_groups.h>
#include <cfloat>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rk {

// ---------------------------------------------------------------------------
// Batched row-major DGEMM, 64x64 tile, 16-deep k slices, 4x4 outputs/thread.
namespace {
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256)
k_dgemm(int m, int n, int k, double alpha, const double* __restrict__ A, int64_t lda,
        int64_t strideA, int tA, const double* __restrict__ B, int64_t ldb, int64_t strideB,
        int tB, double beta, double* __restrict__ C, int64_t ldc, int64_t strideC, int sym) {
    // sym: the product is known to be symmetric (m == n): only tiles on or
    // above the diagonal are computed and each is written to both halves.
    if (sym && blockIdx.x < blockIdx.y) return;
    __shared__ double As[GK][GT + 1];
    __shared__ double Bs[GK][GT + 1];
    const int bz = blockIdx.z;
    A += (int64_t)bz * strideA;
    B += (int64_t)bz * strideB;
    C += (int64_t)bz * strideC;
    const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int kk = 0; kk < k; kk += GK) {
        for (int it = threadIdx.x; it < GK * GT; it += 256) {
            int kq, iq;
            if (tA) { iq = it % GT; kq = it / GT; } else { kq = it % GK; iq = it / GK; }
            const int gi = i0 + iq, gk = kk + kq;
            double v = 0.0;
            if (gi < m && gk < k) v = tA ? A[(int64_t)gk * lda + gi] : A[(int64_t)gi * lda + gk];
            As[kq][iq] = v;
        }
        for (int it = threadIdx.x; it < GK * GT; it += 256) {
            int kq, jq;
            if (tB) { kq = it % GK; jq = it / GK; } else { jq = it % GT; kq = it / GT; }
            const int gj = j0 + jq, gk = kk + kq;
            double v = 0.0;
            if (gj < n && gk < k) v = tB ? B[(int64_t)gj * ldb + gk] : B[(int64_t)gk * ldb + gj];
            Bs[kq][jq] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < GK; ++q) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[q][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[q][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gi = i0 + ty + 16 * r;
        if (gi >= m) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int gj = j0 + tx + 16 * c;
            if (gj >= n) continue;
            double* cp = C + (int64_t)gi * ldc + gj;
            const double v = beta == 0.0 ? alpha * acc[r][c] : alpha * acc[r][c] + beta * *cp;
            *cp = v;
            if (sym && blockIdx.x != blockIdx.y) C[(int64_t)gj * ldc + gi] = v;
        }
    }
}
}  // namespace

cudaError_t launch_dgemm(int nb, int m, int n, int k, double alpha, const double* A, int64_t lda,
                         int64_t strideA, int tA, const double* B, int64_t ldb, int64_t strideB,
                         int tB, double beta, double* C, int64_t ldc, int64_t strideC,
                         cudaStream_t s, int sym) {
    if (nb <= 0 || m <= 0 || n <= 0) return cudaSuccess;
    if (sym && m != n) return cudaErrorInvalidValue;
    dim3 grid((unsigned)ceil_div(n, GT), (unsigned)ceil_div(m, GT), (unsigned)nb);
    k_dgemm<<<grid, 256, 0, s>>>(m, n, k, alpha, A, lda, strideA, tA, B, ldb, strideB, tB, beta,
                                 C, ldc, strideC, sym);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Eigenbasis refinement (Ogita & Aishima, "Iterative refinement for symmetric
// eigenvalue decomposition", Japan J. Indust. Appl. Math. 35, 2018), one step
// for each of nmat matrices.  Rows of X are the approximate eigenvectors.
//   R = I - X X^T,  S = X G X^T,  lam_i = S_ii / (1 - R_ii),
//   delta = 2 (|S - diag(lam)| + |G| |R|)   (Frobenius bounds),
//   E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) if |lam_i - lam_j| > delta
//        = R_ij / 2                             otherwise,
//   X_new = X + E^T X   (rows), i.e. columns X + X E.
namespace {
// Per matrix: eigenvalue estimates lam_i = S_ii / (X X^T)_ii and the cluster
// threshold delta = 2 (|S - diag(lam)|_2 + max|lam| |offdiag(R)|_2).  The
// diagonal of R = I - X X^T only rescales the vectors, which the division
// above already accounts for, so only its off-diagonal part enters delta.
// The two 2-norms are estimated by power iteration on the symmetric matrices
// (in FP32: only the magnitude matters), scaled up by 1.5 against the
// iteration's underestimate.
constexpr int kPowerIters = 8;

// One matrix per cluster of CS CTAs (CS <= 16): CTA c owns rows
// [c Mp / CS, (c + 1) Mp / CS) of both matrices and computes that chunk of
// every product; the chunks and the partial norms are exchanged through the
// cluster's shared memory.  Every CTA keeps the whole iterate.
__global__ void __launch_bounds__(256)
k_oa_norms(const double* __restrict__ W1, const double* __restrict__ W3, int Mp, int CS,
           double* __restrict__ lam, double* __restrict__ norms) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = (int)cluster.block_rank();
    const int mat = blockIdx.x / CS;
    const double* XX = W1 + (int64_t)mat * Mp * Mp;
    const double* S = W3 + (int64_t)mat * Mp * Mp;
    double* L = lam + (int64_t)mat * Mp;
    const int rows = Mp / CS, r0 = crank * rows;
    __shared__ float vs[kMaxM], vr[kMaxM];
    __shared__ float ys[kMaxM], yr[kMaxM];     // this CTA's chunk (first `rows` entries)
    __shared__ double lrow[kMaxM];
    __shared__ float part[3][8];
    __shared__ float pnorm[3];                  // this CTA's |y_s|^2, |y_r|^2, lmax
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float lmax = 0.f;
    for (int q = threadIdx.x; q < rows; q += 256) {
        const int i = r0 + q;
        const double xx = XX[(int64_t)i * Mp + i];
        const double l = xx > 0.0 ? S[(int64_t)i * Mp + i] / xx : 0.0;
        L[i] = l;
        lrow[q] = l;
        lmax = fmaxf(lmax, (float)fabs(l));
    }
    for (int i = threadIdx.x; i < Mp; i += 256) {
        // deterministic start vector with all components non-zero
        const float v0 = 1.0f + 0.5f * (float)((i * 2654435761u) >> 28) / 16.0f;
        vs[i] = v0;
        vr[i] = v0;
    }
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if (lane == 0) part[2][warp] = lmax;
    __syncthreads();
    float ns = 0.f, nr = 0.f;
    for (int it = 0; it < kPowerIters; ++it) {
        // y = B v on this CTA's rows, B = S - diag(lam) and B = -offdiag(X X^T)
        for (int q = warp; q < rows; q += 8) {
            const int i = r0 + q;
            float as = 0.f, ar = 0.f;
            const double li = lrow[q];
            for (int j = lane; j < Mp; j += 32) {
                const double s_ij = S[(int64_t)i * Mp + j] - (i == j ? li : 0.0);
                const double r_ij = i == j ? 0.0 : -XX[(int64_t)i * Mp + j];
                as = fmaf((float)s_ij, vs[j], as);
                ar = fmaf((float)r_ij, vr[j], ar);
            }
            for (int o = 16; o > 0; o >>= 1) {
                as += __shfl_xor_sync(0xffffffffu, as, o);
                ar += __shfl_xor_sync(0xffffffffu, ar, o);
            }
            if (lane == 0) { ys[q] = as; yr[q] = ar; }
        }
        __syncthreads();
        // partial |y|^2 of the chunk; |v|^2 from the whole local iterate
        float ps = 0.f, pr = 0.f, qs = 0.f, qr = 0.f;
        for (int q = threadIdx.x; q < rows; q += 256) { ps += ys[q] * ys[q]; pr += yr[q] * yr[q]; }
        for (int i = threadIdx.x; i < Mp; i += 256) { qs += vs[i] * vs[i]; qr += vr[i] * vr[i]; }
        for (int o = 16; o > 0; o >>= 1) {
            ps += __shfl_xor_sync(0xffffffffu, ps, o); pr += __shfl_xor_sync(0xffffffffu, pr, o);
            qs += __shfl_xor_sync(0xffffffffu, qs, o); qr += __shfl_xor_sync(0xffffffffu, qr, o);
        }
        __shared__ float pv[2][8];
        if (lane == 0) { part[0][warp] = ps; part[1][warp] = pr; pv[0][warp] = qs; pv[1][warp] = qr; }
        __syncthreads();
        if (threadIdx.x == 0) {
            float a = 0.f, b = 0.f, lm = 0.f;
            for (int w = 0; w < 8; ++w) { a += part[0][w]; b += part[1][w]; lm = fmaxf(lm, part[2][w]); }
            pnorm[0] = a; pnorm[1] = b; pnorm[2] = lm;
        }
        cluster.sync();
        // totals over the cluster, then the whole normalised y from the owners
        float a = 0.f, b = 0.f, c = 0.f, d = 0.f;
        for (int w = 0; w < 8; ++w) { c += pv[0][w]; d += pv[1][w]; }
        for (int r = 0; r < CS; ++r) {
            const float* pn = cluster.map_shared_rank(pnorm, r);
            a += pn[0]; b += pn[1];
        }
        ns = c > 0.f ? sqrtf(a / c) : 0.f;     // |B v| / |v|
        nr = d > 0.f ? sqrtf(b / d) : 0.f;
        const float fs = a > 0.f ? rsqrtf(a) : 0.f, fr = b > 0.f ? rsqrtf(b) : 0.f;
        for (int i = threadIdx.x; i < Mp; i += 256) {
            const int r = i / rows, q = i - r * rows;
            vs[i] = cluster.map_shared_rank(ys, r)[q] * fs;
            vr[i] = cluster.map_shared_rank(yr, r)[q] * fr;
        }
        // every CTA has read the chunks before they are overwritten
        cluster.sync();
    }
    if (crank == 0 && threadIdx.x == 0) {
        float lm = 0.f;
        for (int r = 0; r < CS; ++r) lm = fmaxf(lm, cluster.map_shared_rank(pnorm, r)[2]);
        norms[mat] = 2.0 * 1.5 * ((double)ns + (double)lm * (double)nr);
    }
    // keep the shared memory alive until rank 0 has read it
    cluster.sync();
}

// Rows of X back to unit length: the refinement keeps the rows orthogonal to
// first order, but sum_k E_ki^2 from pairs with a small gap lengthens row i at
// second order; the direction is what the step improved, the length is known.
__global__ void k_normalize_rows(double* __restrict__ X, int Mp, int64_t nrows) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= nrows) return;
    double* x = X + row * Mp;
    double ss = 0.0;
    for (int j = lane; j < Mp; j += 32) ss = fma(x[j], x[j], ss);
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (ss <= 0.0) return;
    const double f = 1.0 / sqrt(ss);
    for (int j = lane; j < Mp; j += 32) x[j] *= f;
}

__global__ void k_oa_E(double* __restrict__ W1, const double* __restrict__ W3, int Mp,
                       const double* __restrict__ lam, const double* __restrict__ norms) {
    const int mat = blockIdx.y;
    double* XX = W1 + (int64_t)mat * Mp * Mp;
    const double* S = W3 + (int64_t)mat * Mp * Mp;
    const double* L = lam + (int64_t)mat * Mp;
    const double delta = norms[mat];
    const int64_t n = (int64_t)Mp * Mp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / Mp), j = (int)(e % Mp);
        const double r = (i == j ? 1.0 : 0.0) - XX[e];
        const double gap = L[j] - L[i];
        XX[e] = fabs(gap) > delta ? (S[e] + L[j] * r) / gap : 0.5 * r;
    }
}
}  // namespace

// T = G X^T from the sparse block instead of the dense G (G = sum_j a_j a_j^T
// over the block's columns): T = sum_j a_j (X a_j)^T.  One warp per column j
// forms y = X a_j from the rows of X^T picked by the column's entries, then
// adds v_e * y to row r_e of T for every entry (r_e, v_e) (FP64 atomics).
// Cost 2 * nnz * Mp multiply-adds instead of the dense Mp^3.
namespace {
constexpr int kYPerLane = 8;   // FP64 accumulators per lane (256 columns of T per pass)

__global__ void __launch_bounds__(256)
k_transpose(const double* __restrict__ X, double* __restrict__ XT, int Mp) {
    __shared__ double tile[32][33];
    const int64_t off = (int64_t)blockIdx.z * Mp * Mp;
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int r = ty; r < 32; r += 8) tile[r][tx] = X[off + (int64_t)(by + r) * Mp + bx + tx];
    __syncthreads();
    for (int r = ty; r < 32; r += 8) XT[off + (int64_t)(bx + r) * Mp + by + tx] = tile[tx][r];
}

__global__ void __launch_bounds__(256)
k_sparse_gxt(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
             const void* __restrict__ vals, int value_type, int Mp,
             const int32_t* __restrict__ chunk_block, const int64_t* __restrict__ chunk_lo,
             const int64_t* __restrict__ chunk_hi, const double* __restrict__ XT,
             double* __restrict__ T) {
    const int c = blockIdx.x;
    const int d = chunk_block[c];
    const int64_t mm = (int64_t)Mp * Mp;
    const double* XTd = XT + d * mm;
    double* Td = T + d * mm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t j = chunk_lo[c] + warp; j < chunk_hi[c]; j += 8) {
        const int64_t e0 = col_ptr[j], e1 = col_ptr[j + 1];
        if (e0 == e1) continue;
        for (int i0 = 0; i0 < Mp; i0 += 32 * kYPerLane) {
            double y[kYPerLane];
#pragma unroll
            for (int q = 0; q < kYPerLane; ++q) y[q] = 0.0;
            for (int64_t e = e0; e < e1; ++e) {
                const double v = load_val(vals, value_type, e);
                const double* xr = XTd + (int64_t)row_idx[e] * Mp + i0 + lane;
#pragma unroll
                for (int q = 0; q < kYPerLane; ++q)
                    if (i0 + lane + 32 * q < Mp) y[q] = fma(v, xr[32 * q], y[q]);
            }
            for (int64_t e = e0; e < e1; ++e) {
                const double v = load_val(vals, value_type, e);
                double* tr = Td + (int64_t)row_idx[e] * Mp + i0 + lane;
#pragma unroll
                for (int q = 0; q < kYPerLane; ++q)
                    if (i0 + lane + 32 * q < Mp) atomicAdd(tr + 32 * q, v * y[q]);
            }
        }
    }
}
}  // namespace

cudaError_t launch_refine(const double* G, double* X, double* Xn, double* lam, int nmat,
                          int Mp, double* W1, double* W2, double* W3, double* norms,
                          cudaStream_t s, const SparseBlocks* sp, OzOperand* oz,
                          const RRWork* rr) {
    const int64_t st = (int64_t)Mp * Mp;
    if (sp) {
        // X^T staged in W3 for the sparse product
        k_transpose<<<dim3(Mp / 32, Mp / 32, nmat), 256, 0, s>>>(X, W3, Mp);
        RK_CUDA_TRY(cudaGetLastError());
    }
    if (oz) {
        // exact-slice products (oz[0], oz[1] hold the operands): X sliced once
        // for W1 = X X^T and S = X (G X^T)
        OzOperand& xa = oz[0];
        OzOperand& ob = oz[1];
        RK_CUDA_TRY(launch_oz_split(nmat, Mp, Mp, X, Mp, st, 0, nullptr, 5, xa, s));
        RK_CUDA_TRY(launch_oz_gemm(nmat, Mp, Mp, xa, xa, 1.0, 0.0, W1, Mp, st, 1, s));
        if (sp) {
            // W2 = T = G X^T from the sparse columns; W3 = X T (B rows = columns of T)
            RK_CUDA_TRY(cudaMemsetAsync(W2, 0, sizeof(double) * st * nmat, s));
            if (sp->nchunks > 0) {
                k_sparse_gxt<<<sp->nchunks, 256, 0, s>>>(sp->col_ptr, sp->row_idx, sp->vals,
                                                         sp->value_type, Mp, sp->chunk_block,
                                                         sp->chunk_lo, sp->chunk_hi, W3, W2);
                RK_CUDA_TRY(cudaGetLastError());
            }
            RK_CUDA_TRY(launch_oz_split(nmat, Mp, Mp, W2, Mp, st, 1, nullptr, 5, ob, s));
            RK_CUDA_TRY(launch_oz_gemm(nmat, Mp, Mp, xa, ob, 1.0, 0.0, W3, Mp, st, 1, s));
        } else {
            // W2 = X G (G symmetric: its rows are the B rows), W3 = W2 X^T
            RK_CUDA_TRY(launch_oz_split(nmat, Mp, Mp, G, Mp, st, 0, nullptr, 5, ob, s));
            RK_CUDA_TRY(launch_oz_gemm(nmat, Mp, Mp, xa, ob, 1.0, 0.0, W2, Mp, st, 0, s));
            RK_CUDA_TRY(launch_oz_split(nmat, Mp, Mp, W2, Mp, st, 0, nullptr, 5, ob, s));
            RK_CUDA_TRY(launch_oz_gemm(nmat, Mp, Mp, ob, xa, 1.0, 0.0, W3, Mp, st, 1, s));
        }
    } else {
        // W1 = X X^T (symmetric)
        RK_CUDA_TRY(launch_dgemm(nmat, Mp, Mp, Mp, 1.0, X, Mp, st, 0, X, Mp, st, 1, 0.0, W1, Mp, st, s, 1));
        if (sp) {
            // W2 = G X^T from the sparse blocks (X^T in W3), then W3 = X W2
            RK_CUDA_TRY(cudaMemsetAsync(W2, 0, sizeof(double) * st * nmat, s));
            if (sp->nchunks > 0) {
                k_sparse_gxt<<<sp->nchunks, 256, 0, s>>>(sp->col_ptr, sp->row_idx, sp->vals,
                                                         sp->value_type, Mp, sp->chunk_block,
                                                         sp->chunk_lo, sp->chunk_hi, W3, W2);
                RK_CUDA_TRY(cudaGetLastError());
            }
            RK_CUDA_TRY(launch_dgemm(nmat, Mp, Mp, Mp, 1.0, X, Mp, st, 0, W2, Mp, st, 0, 0.0, W3, Mp, st, s, 1));
        } else {
            // W2 = X G, W3 = W2 X^T = X G X^T (symmetric)
            RK_CUDA_TRY(launch_dgemm(nmat, Mp, Mp, Mp, 1.0, X, Mp, st, 0, G, Mp, st, 0, 0.0, W2, Mp, st, s));
            RK_CUDA_TRY(launch_dgemm(nmat, Mp, Mp, Mp, 1.0, W2, Mp, st, 0, X, Mp, st, 1, 0.0, W3, Mp, st, s, 1));
        }
    }
    if (rr) {
        // estimates, clusters, Rayleigh-Ritz inside them (X, S (W3), X X^T
        // (W1) and lam in place; W2, dead after the products, holds the
        // cluster rotations), then E over W1
        RK_CUDA_TRY(launch_cluster_rr(*rr, nmat, Mp, X, W3, W1, W2, lam, norms, s));
    } else {
        // cluster size: enough CTAs to cover the GPU, a divisor of Mp, <= 16
        int cs = 1;
        while (cs < 16 && nmat * cs < 304 && Mp % (2 * cs) == 0) cs *= 2;
        if (cs > 8)
            RK_CUDA_TRY(cudaFuncSetAttribute(k_oa_norms, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nmat * cs), 1, 1);
        cfg.blockDim = dim3(256, 1, 1);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        RK_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_oa_norms, (const double*)W1, (const double*)W3, Mp, cs,
                                       lam, norms));
        const int bx = (int)std::min<int64_t>(ceil_div(st, 256), 1024);
        k_oa_E<<<dim3(bx, nmat), 256, 0, s>>>(W1, W3, Mp, lam, norms);
        RK_CUDA_TRY(cudaGetLastError());
    }
    // Xn = X + E^T X
    RK_CUDA_TRY(cudaMemcpyAsync(Xn, X, sizeof(double) * st * nmat, cudaMemcpyDeviceToDevice, s));
    if (oz) {
        // the correction is small: three slices (relative 2^-23) are ample
        RK_CUDA_TRY(launch_oz_split(nmat, Mp, Mp, W1, Mp, st, 1, nullptr, 3, oz[0], s));
        RK_CUDA_TRY(launch_oz_split(nmat, Mp, Mp, X, Mp, st, 1, nullptr, 3, oz[1], s));
        RK_CUDA_TRY(launch_oz_gemm(nmat, Mp, Mp, oz[0], oz[1], 1.0, 1.0, Xn, Mp, st, 0, s));
    } else {
        RK_CUDA_TRY(launch_dgemm(nmat, Mp, Mp, Mp, 1.0, W1, Mp, st, 1, X, Mp, st, 0, 1.0, Xn, Mp, st, s));
    }
    const int64_t rows = (int64_t)nmat * Mp;
    k_normalize_rows<<<(unsigned)ceil_div(rows * 32, 256), 256, 0, s>>>(Xn, Mp, rows);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sort eigenvalues descending (ties by index), numerical rank, sigma.
namespace {
__global__ void __launch_bounds__(1024)
k_sort_rank(const double* __restrict__ lam, const float* __restrict__ lam32,
            const double* __restrict__ diag64, const float* __restrict__ diag32, int M, int Mp,
            const int64_t* __restrict__ bounds, int64_t width_all, double rank_tol,
            double* __restrict__ sigma_sorted, int32_t* __restrict__ perm,
            int32_t* __restrict__ rank) {
    __shared__ double key[kMaxM];
    __shared__ int idx[kMaxM];
    __shared__ int cnt;
    const int mat = blockIdx.x;
    int n = 1;
    while (n < M) n <<= 1;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v = -DBL_MAX;
        if (i < M) {
            const int64_t o = (int64_t)mat * Mp;
            if (lam) v = lam[o + i];
            else if (lam32) v = (double)lam32[o + i];
            else if (diag64) v = diag64[(int64_t)mat * Mp * Mp + (int64_t)i * Mp + i];
            else v = (double)diag32[(int64_t)mat * Mp * Mp + (int64_t)i * Mp + i];
        }
        key[i] = v;
        idx[i] = i;
    }
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    // bitonic sort: descending key, ascending index on ties
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const double ki = key[i], kj = key[j];
                    const int ii = idx[i], ij = idx[j];
                    // "i before j" in the final order
                    const bool i_first = ki > kj || (ki == kj && ii < ij);
                    if (desc != i_first) {
                        key[i] = kj; key[j] = ki;
                        idx[i] = ij; idx[j] = ii;
                    }
                }
            }
            __syncthreads();
        }
    }
    const int64_t width = bounds ? bounds[mat + 1] - bounds[mat] : width_all;
    const double lmax = fmax(key[0], 0.0);
    const double tau = rank_tol > 0.0 ? rank_tol * rank_tol
                                      : (double)((int64_t)M > width ? (int64_t)M : width) * 2.220446049250313e-16 * lmax;
    int local = 0;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const double v = key[i];
        sigma_sorted[(int64_t)mat * M + i] = v > 0.0 ? sqrt(v) : 0.0;
        perm[(int64_t)mat * M + i] = idx[i];
        if (v > tau) ++local;
    }
    atomicAdd(&cnt, local);
    __syncthreads();
    // a block of w columns has rank <= min(M, w): never report more
    if (threadIdx.x == 0) rank[mat] = (int)min((int64_t)cnt, min((int64_t)M, width));
}
}  // namespace

cudaError_t launch_sort_rank(const double* lam, const float* lam32, const double* diag64,
                             const float* diag32, int nmat, int M, int Mp, const int64_t* bounds,
                             int64_t width_all, double rank_tol, double* sigma_sorted,
                             int32_t* perm, int32_t* rank, cudaStream_t s) {
    k_sort_rank<<<nmat, 1024, 0, s>>>(lam, lam32, diag64, diag32, M, Mp, bounds, width_all,
                                      rank_tol, sigma_sorted, perm, rank);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Proxy P = [U^1[:, :r_1] S^1 | ... ], column-major M x R with R = sum r_i.
namespace {
__global__ void k_proxy_ofs(const int32_t* __restrict__ rank, int D, int keep_max,
                            int64_t* __restrict__ ofs) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int64_t acc = 0;
        for (int d = 0; d < D; ++d) {
            ofs[d] = acc;
            acc += keep_max > 0 ? min(rank[d], keep_max) : rank[d];
        }
        ofs[D] = acc;
    }
}

__global__ void k_proxy(const double* __restrict__ X64, const float* __restrict__ X32,
                        const double* __restrict__ sigma_sorted, const int32_t* __restrict__ perm,
                        const int32_t* __restrict__ rank, int M, int Mp, int keep_max,
                        const int64_t* __restrict__ ofs, double* __restrict__ P) {
    const int d = blockIdx.y;
    const int r = keep_max > 0 ? min(rank[d], keep_max) : rank[d];
    const int64_t base = ofs[d];
    const int64_t mo = (int64_t)d * Mp * Mp;
    for (int j = blockIdx.x; j < r; j += gridDim.x) {
        const int src = perm[(int64_t)d * M + j];
        const double sg = sigma_sorted[(int64_t)d * M + j];
        double* col = P + (base + j) * (int64_t)M;
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            const double x = X64 ? X64[mo + (int64_t)src * Mp + m] : (double)X32[mo + (int64_t)src * Mp + m];
            col[m] = x * sg;
        }
    }
}
}  // namespace

cudaError_t launch_proxy(const double* X64, const float* X32, const double* sigma_sorted,
                         const int32_t* perm, const int32_t* rank, int D, int M, int Mp,
                         int64_t* proxy_ofs, double* P, cudaStream_t s, int keep_max) {
    k_proxy_ofs<<<1, 32, 0, s>>>(rank, D, keep_max, proxy_ofs);
    RK_CUDA_TRY(cudaGetLastError());
    const int bx = M < 64 ? M : 64;
    k_proxy<<<dim3(bx, D), 128, 0, s>>>(X64, X32, sigma_sorted, perm, rank, M, Mp, keep_max,
                                        proxy_ofs, P);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// One level of the tree merge: the weighted bases Y_c (Mp x Mp, row j =
// sigma_cj times the eigenvector of the j-th largest eigenvalue of child c,
// for j below the child's kept rank; zero otherwise, and for the padding
// children c >= nchild), then S_node = sum over its `arity` consecutive
// children of Y_c^T Y_c (the children's proxy columns are the rows of Y_c:
// S_node = P_node P_node^T, Eq. 3, without forming P).
namespace {
__global__ void k_tree_weights(const double* __restrict__ X64, const double* __restrict__ sigma_sorted,
                               const int32_t* __restrict__ perm, const int32_t* __restrict__ rank,
                               int nchild, int M, int Mp, int keep_max, double* __restrict__ Y) {
    const int c = blockIdx.y;
    const int64_t mm = (int64_t)Mp * Mp;
    double* Yc = Y + (int64_t)c * mm;
    int kept = 0;
    if (c < nchild) kept = keep_max > 0 ? min(rank[c], keep_max) : rank[c];
    for (int j = blockIdx.x; j < Mp; j += gridDim.x) {
        double sg = 0.0;
        const double* x = nullptr;
        if (j < kept) {
            sg = sigma_sorted[(int64_t)c * M + j];
            x = X64 + (int64_t)c * mm + (int64_t)perm[(int64_t)c * M + j] * Mp;
        }
        for (int m = threadIdx.x; m < Mp; m += blockDim.x)
            Yc[(int64_t)j * Mp + m] = (x && m < M) ? sg * x[m] : 0.0;
    }
}
}  // namespace

cudaError_t launch_tree_level(const double* X64, const double* sigma_sorted, const int32_t* perm,
                              const int32_t* rank, int nchild, int arity, int M, int Mp,
                              int keep_max, double* Y, double* S, OzOperand* oz, cudaStream_t s) {
    const int nnode = (int)ceil_div(nchild, arity);
    const int64_t mm = (int64_t)Mp * Mp;
    k_tree_weights<<<dim3(std::min(Mp, 128), nnode * arity), 128, 0, s>>>(
        X64, sigma_sorted, perm, rank, nchild, M, Mp, keep_max, Y);
    RK_CUDA_TRY(cudaGetLastError());
    const int64_t k = (int64_t)arity * Mp;
    if (oz) {
        // A = the stacked Y of a node read transposed: Mp rows (coordinates) x
        // arity Mp k (the children's proxy columns)
        RK_CUDA_TRY(launch_oz_split(nnode, Mp, k, Y, Mp, arity * mm, 1, nullptr, 5, oz[0], s));
        return launch_oz_gemm(nnode, Mp, Mp, oz[0], oz[0], 1.0, 0.0, S, Mp, mm, 1, s);
    }
    return launch_dgemm(nnode, Mp, Mp, (int)k, 1.0, Y, Mp, arity * mm, 1, Y, Mp, arity * mm, 0,
                        0.0, S, Mp, mm, s, 1);
}

// ---------------------------------------------------------------------------
// S = P P^T over the R proxy columns (R read on the device), split over R.
namespace {
__global__ void __launch_bounds__(256)
k_merge_partial(const double* __restrict__ P, const int64_t* __restrict__ ofs, int D, int M,
                int64_t kc, double* __restrict__ partial, int Mp) {
    const int ntile = (M + GT - 1) / GT;
    // upper-triangle tile (ti <= tj) from the linear index
    int t = blockIdx.x, ti = 0;
    while (t >= ntile - ti) { t -= ntile - ti; ++ti; }
    const int tj = ti + t;
    const int split = blockIdx.y;
    const int64_t R = ofs[D];
    const int64_t k0 = (int64_t)split * kc, k1 = min(R, k0 + kc);
    __shared__ double As[GK][GT + 1];
    __shared__ double Bs[GK][GT + 1];
    const int i0 = ti * GT, j0 = tj * GT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int64_t kk = k0; kk < k1; kk += GK) {
        for (int it = threadIdx.x; it < GK * GT; it += 256) {
            const int iq = it % GT, kq = it / GT;
            const int64_t gk = kk + kq;
            const bool ok = gk < k1;
            As[kq][iq] = (ok && i0 + iq < M) ? P[gk * M + i0 + iq] : 0.0;
            Bs[kq][iq] = (ok && j0 + iq < M) ? P[gk * M + j0 + iq] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < GK; ++q) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[q][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[q][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
    double* out = partial + (int64_t)split * Mp * Mp;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gi = i0 + ty + 16 * r;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int gj = j0 + tx + 16 * c;
            if (gi < Mp && gj < Mp) out[(int64_t)gi * Mp + gj] = acc[r][c];
        }
    }
}

__global__ void k_merge_reduce(const double* __restrict__ partial, int nsplit, int M, int Mp,
                               double* __restrict__ S) {
    const int64_t n = (int64_t)Mp * Mp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / Mp), j = (int)(e % Mp);
        double v = 0.0;
        if (i < M && j < M) {
            const int a = min(i, j), b = max(i, j);
            const int64_t src = (int64_t)a * Mp + b;
            for (int sp = 0; sp < nsplit; ++sp) v += partial[(int64_t)sp * n + src];
        }
        S[e] = v;
    }
}
}  // namespace

int merge_gram_splits(int M, int64_t Rmax) {
    const int ntile = (M + GT - 1) / GT;
    const int upper = ntile * (ntile + 1) / 2;
    int64_t want = ceil_div(600, upper);
    const int64_t cap = ceil_div(Rmax, 256);
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

cudaError_t launch_merge_gram(const double* P, const int64_t* proxy_ofs, int D, int M, int Mp,
                              int64_t Rmax, double* partial, int nsplit, double* S,
                              cudaStream_t s, OzOperand* oz) {
    if (oz) {
        // exact-slice product over the proxy columns (P is column-major M x R)
        RK_CUDA_TRY(launch_oz_split(1, M, Rmax, P, M, 0, 1, proxy_ofs + D, 5, *oz, s));
        RK_CUDA_TRY(launch_oz_gemm(1, M, M, *oz, *oz, 1.0, 0.0, partial, Mp, 0, 1, s, nsplit,
                                   (int64_t)Mp * Mp));
    } else {
        const int ntile = (M + GT - 1) / GT;
        const int upper = ntile * (ntile + 1) / 2;
        const int64_t kc = round_up(ceil_div(Rmax, nsplit), GK);
        k_merge_partial<<<dim3(upper, nsplit), 256, 0, s>>>(P, proxy_ofs, D, M, kc, partial, Mp);
        RK_CUDA_TRY(cudaGetLastError());
    }
    const int64_t n = (int64_t)Mp * Mp;
    const int bx = (int)std::min<int64_t>(ceil_div(n, 256), 2048);
    k_merge_reduce<<<bx, 256, 0, s>>>(partial, nsplit, M, Mp, S);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Outputs: sigma, U (column-major, sign rule), rank, W = U_k S_k^-1 (row-major M x k).
namespace {
template <typename TW>
__global__ void __launch_bounds__(256)
k_finalize(const double* __restrict__ X64, const float* __restrict__ X32,
           const double* __restrict__ sigma_sorted, const int32_t* __restrict__ perm, int M,
           int Mp, int k, double lam_tol_abs, int64_t tol_scale, double* __restrict__ d_sigma,
           double* __restrict__ d_U, int32_t* __restrict__ d_rank, TW* __restrict__ W) {
    const int i = blockIdx.x;
    const double s1 = sigma_sorted[0];
    const double tau = lam_tol_abs > 0.0 ? lam_tol_abs
                                         : (double)tol_scale * 2.220446049250313e-16 * s1 * s1;
    if (i == 0 && threadIdx.x == 0) {
        int r = 0;
        for (int j = 0; j < M; ++j) r += sigma_sorted[j] * sigma_sorted[j] > tau;
        *d_rank = r;
    }
    const int src = perm[i];
    __shared__ double bv[256];
    __shared__ int bi[256];
    double best = -1.0;
    int barg = M;
    for (int m = threadIdx.x; m < M; m += 256) {
        const double x = X64 ? X64[(int64_t)src * Mp + m] : (double)X32[(int64_t)src * Mp + m];
        const double a = fabs(x);
        if (a > best) { best = a; barg = m; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = barg;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double ov = bv[threadIdx.x + o];
            const int oi = bi[threadIdx.x + o];
            if (ov > bv[threadIdx.x] || (ov == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = ov;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const int am = bi[0];
    const double xam = X64 ? X64[(int64_t)src * Mp + am] : (double)X32[(int64_t)src * Mp + am];
    const double sg = xam < 0.0 ? -1.0 : 1.0;
    const double si = sigma_sorted[i];
    const bool keep = si * si > tau;
    if (threadIdx.x == 0) d_sigma[i] = si;
    for (int m = threadIdx.x; m < M; m += 256) {
        const double x = sg * (X64 ? X64[(int64_t)src * Mp + m] : (double)X32[(int64_t)src * Mp + m]);
        d_U[(int64_t)i * M + m] = x;
        W[(int64_t)m * k + i] = keep ? (TW)(x / si) : (TW)0;
    }
}
}  // namespace

cudaError_t launch_finalize(const double* X64, const float* X32, const double* sigma_sorted,
                            const int32_t* perm, int M, int Mp, int k, double lam_tol_abs,
                            int64_t tol_scale, double* d_sigma, double* d_U, int32_t* d_rank,
                            double* W64, float* W32, cudaStream_t s) {
    if (W64)
        k_finalize<double><<<k, 256, 0, s>>>(X64, X32, sigma_sorted, perm, M, Mp, k, lam_tol_abs,
                                             tol_scale, d_sigma, d_U, d_rank, W64);
    else
        k_finalize<float><<<k, 256, 0, s>>>(X64, X32, sigma_sorted, perm, M, Mp, k, lam_tol_abs,
                                            tol_scale, d_sigma, d_U, d_rank, W32);
    return cudaGetLastError();
}

}  // namespace rk
