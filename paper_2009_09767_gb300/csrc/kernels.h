// kernels.h -- host-side launchers of the column-block SVD kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rk {

struct PatchRec {       // matches svd_patch in include/ranky.h
    int32_t row;
    int32_t block;
    int64_t col;
};

// ---- partition.cu: Algorithm 1 split + lonely scan, Algorithm 2 -------------
// chunk_block[c] / chunk_col[c .. c+1]: column chunks that never straddle a block.
cudaError_t launch_occupancy(const int64_t* col_ptr, const int32_t* row_idx, const void* vals,
                             int value_type, int M, int nchunks, const int32_t* chunk_block,
                             const int64_t* chunk_col_lo, const int64_t* chunk_col_hi,
                             uint32_t* occ, cudaStream_t s);
// occ: D x W words (W = ceil(M/32)).  Writes row_ne (W words), lonely (D x W),
// and, by mode, nothing more (0), RandomChecker patches (1) or one slot with
// col = -1 per lonely node (2), in (block, row) order with per-block offsets;
// lonely_any (W words, may be null) = rows lonely in some block.
cudaError_t launch_lonely_patches(const uint32_t* occ, int D, int M, const int64_t* bounds,
                                  int mode, uint64_t seed, uint32_t* row_ne, uint32_t* lonely,
                                  PatchRec* patches, int64_t* patch_ofs, PatchRec* ext_patches,
                                  int64_t* ext_npatches, uint32_t* lonely_any, cudaStream_t s);
// Algorithms 3-4 over the slots of mode 2: row co-occurrence counts (cooc,
// M x M, cleared here), a column per slot (or none; RandomChecker's when
// fallback), then the filled slots compacted into patches / patch_ofs (and
// the caller's copy).  Three kernels.
cudaError_t launch_neighbor_patches(const int64_t* col_ptr, const int32_t* row_idx,
                                    const void* vals, int value_type, int M, int64_t N, int D,
                                    const int64_t* bounds, const uint32_t* lonely_any,
                                    unsigned long long* cooc, int fallback, uint64_t seed,
                                    PatchRec* slots, const int64_t* slot_ofs, PatchRec* patches,
                                    int64_t* patch_ofs, PatchRec* ext_patches,
                                    int64_t* ext_npatches, cudaStream_t s);

// ---- gram.cu: Eq. 2 block cross products --------------------------------------
// G: D x Mp x Mp FP64 (upper triangle accumulated; must be zero on entry).
cudaError_t launch_gram(const int64_t* col_ptr, const int32_t* row_idx, const void* vals,
                        int value_type, int Mp, int nchunks, const int32_t* chunk_block,
                        const int64_t* chunk_col_lo, const int64_t* chunk_col_hi, double* G,
                        cudaStream_t s);
cudaError_t launch_gram_patches(const int64_t* col_ptr, const int32_t* row_idx, const void* vals,
                                int value_type, int Mp, int D, const PatchRec* patches,
                                const int64_t* patch_ofs, int max_patches, double* G, cudaStream_t s);
// Mirror the upper triangle into the lower one, in place, for nmat matrices.
cudaError_t launch_symmetrize(double* G, int nmat, int Mp, cudaStream_t s);
cudaError_t launch_convert_f64_f32(const double* src, float* dst, int64_t n, cudaStream_t s);
cudaError_t launch_convert_f32_f64(const float* src, double* dst, int64_t n, cudaStream_t s);

// ---- jacobi.cu: block two-sided Jacobi eigensolver ----------------------------
// G (nmat x Mp x Mp, symmetric, overwritten by its diagonalised form) and
// Vt (nmat x Mp x Mp, rows = eigenvectors on exit).  sweeps[mat] receives the
// sweep count, negative when max_sweeps ran out.  The FP32 solver needs
// work = jacobi_work_bytes(nmat, Mp) bytes of device memory (the published
// pair rotations); the FP64 one ignores it.
// cluster (FP32 solver): CTAs per matrix, 0 = the occupancy model's choice.
template <typename T>
cudaError_t launch_jacobi(T* G, T* Vt, int nmat, int Mp, int max_sweeps, double tol,
                          int32_t* sweeps, cudaStream_t s, void* work = nullptr, int cluster = 0);
size_t jacobi_work_bytes(int nmat, int Mp);
// Padded order of an M x M problem (a multiple of 32).
int jacobi_pad(int M);

// One matrix of a persistent batched solve: G and Vt (Mp x Mp, element type of
// the launch), the sweep counter it reports to.
struct JacobiItem {
    void* G;
    void* Vt;
    int32_t* sweeps;
    void* work;        // FP32: jacobi_work_bytes(1, Mp) bytes
    int32_t Mp;
    int32_t max_sweeps;  // this matrix's sweep cap (> 0; else the launch's)
};
// Largest Mp one persistent worker CTA can hold.
int jacobi_item_max_mp(bool fp64);
// Persistent workers over nitems matrices of order <= max_mp (items in device
// memory; next is a device int used as the work counter).
template <typename T>
cudaError_t launch_jacobi_items(const JacobiItem* items, int nitems, int max_mp, int* next,
                                int max_sweeps, double tol, cudaStream_t s);

// ---- dense.cu: FP64 batched products, refinement, sort/rank, proxy, merge ----
// C[b] = alpha * op(A[b]) op(B[b]) + beta * C[b], row-major, op = transpose if t*.
cudaError_t launch_dgemm(int nb, int m, int n, int k, double alpha, const double* A, int64_t lda,
                         int64_t strideA, int tA, const double* B, int64_t ldb, int64_t strideB,
                         int tB, double beta, double* C, int64_t ldc, int64_t strideC,
                         cudaStream_t s, int sym = 0);
// FP64-accurate products on the bf16 tensor cores (ozaki.cu).  An operand is
// a stack of S integer slices (bf16 bits) per row with the row's magnitude
// bound, rows padded to OZ_ROW_PAD and k to OZ_K_PAD (zeros).
constexpr int OZ_ROW_PAD = 128;
constexpr int OZ_K_PAD = 32;
struct OzOperand {
    uint16_t* slices;                // [nb][S][rows_pad][kpad]
    unsigned long long* amax;        // [nb][rows_pad] bits of max |x| per row
    int S;
    int rows;
    int rows_pad;
    int64_t kpad;
    int tc = 1;                      // products on tcgen05/TMEM (ozaki_tc.cu), else mma.sync
    int* err = nullptr;              // device word set when a bounded wait of the tcgen05 kernel ran out
};
int64_t oz_operand_elems(int nb, int S, int rows, int64_t k);
// Split nb matrices (rows x k logical; element (r, c) at src[r ld + c], or at
// src[c ld + r] when trans) into S = 3 or 5 slices.  kdev, when given, holds
// the number of valid k on the device (the rest reads as zero).
cudaError_t launch_oz_split(int nb, int rows, int64_t k, const double* src, int64_t ld,
                            int64_t stride, int trans, const int64_t* kdev, int S, OzOperand& op,
                            cudaStream_t s);
// C = alpha A B^T + beta C for nb matrices (m x n, row-major ldc).  With
// nsplit > 1 the k range is split and split z writes C + z strideSplit (beta
// then applies per split).  sym: only tiles on or above the diagonal are
// formed and mirrored.
cudaError_t launch_oz_gemm(int nb, int m, int n, const OzOperand& A, const OzOperand& B,
                           double alpha, double beta, double* C, int64_t ldc, int64_t strideC,
                           int sym, cudaStream_t s, int nsplit = 1, int64_t strideSplit = 0);
// The same product with tcgen05.mma (accumulators in TMEM); bit for bit the
// result of the mma.sync kernel.  err (may be null) is set to 1 when a
// bounded wait ran out (the CTA then stops without writing its tile).
cudaError_t launch_oz_gemm_tc(int nb, int m, int n, const OzOperand& A, const OzOperand& B,
                              double alpha, double beta, double* C, int64_t ldc, int64_t strideC,
                              int sym, cudaStream_t s, int nsplit, int64_t strideSplit, int* err);
// The sparse blocks behind block cross products (for G X^T without the dense G).
struct SparseBlocks {
    const int64_t* col_ptr;
    const int32_t* row_idx;
    const void* vals;
    int value_type;
    int nchunks;
    const int32_t* chunk_block;
    const int64_t* chunk_lo;
    const int64_t* chunk_hi;
};
// One Ogita-Aishima refinement step for nmat symmetric matrices G with
// approximate eigenvector rows X (Mp x Mp).  Xn receives the refined rows,
// lam the eigenvalue estimates.  W1..W3 are Mp x Mp scratch per matrix.
// With sp, G X^T is formed from the sparse columns (G itself unused); with
// oz (two operand buffers of nmat x 5 slices x Mp x Mp) every product runs on
// the tensor cores through exact slices instead of the FP64 pipes.
// Cluster Rayleigh-Ritz work (cluster_rr.cu): per matrix the sorted member
// order (Mp), cluster starts and sizes (Mp/2 each) and the cluster count.
struct RRWork {
    int32_t* order;
    int32_t* cstart;
    int32_t* csize;
    int32_t* ncl;
    int32_t* cid;      // per matrix, Mp: cluster of each index (-1: none)
    int32_t* rowmax;   // per matrix, Mp: FP32 upper bound of each row's link test (bits)
    double kappa;      // pairs whose first-order mixing estimate is >= 1/kappa are clustered
    int M;             // indices >= M are padding and never clustered
    int stagger = 0;   // odd refinement steps: long runs are cut half a piece later
};
// With rr, the rows of each cluster of strongly mixed estimates are first
// replaced by the Ritz vectors of the projected problem (X is updated in
// place, and S, X X^T and lam with it), then every other pair takes the
// first-order correction (the published step's cluster threshold and its
// norm estimates are not used).
cudaError_t launch_refine(const double* G, double* X, double* Xn, double* lam, int nmat,
                          int Mp, double* W1, double* W2, double* W3, double* norms,
                          cudaStream_t s, const SparseBlocks* sp = nullptr,
                          OzOperand* oz = nullptr, const RRWork* rr = nullptr);
// Estimates, clusters, Rayleigh-Ritz and the correction E written over B
// (five kernels); Tg is Mp x Mp scratch per matrix, lmax one double per matrix.
cudaError_t launch_cluster_rr(const RRWork& w, int nmat, int Mp, double* X, double* S, double* B,
                              double* Tg, double* lam, double* lmax, cudaStream_t s);
size_t rr_smem_bytes();
// Per matrix: sort eigenvalues (lam, or the diagonal of Gdiag when lam is null)
// of the first M indices descending, rank by tolerance, write sigma
// (sqrt(max(lam,0))) sorted, the permutation and the rank.
// width[b] = block width (for the default tolerance), rank_tol > 0 overrides.
cudaError_t launch_sort_rank(const double* lam, const float* lam32, const double* diag64,
                             const float* diag32, int nmat, int M, int Mp, const int64_t* bounds,
                             int64_t width_all, double rank_tol, double* sigma_sorted,
                             int32_t* perm, int32_t* rank, cudaStream_t s);
// keep_max > 0: at most that many columns per block (the truncation k').
cudaError_t launch_proxy(const double* X64, const float* X32, const double* sigma_sorted,
                         const int32_t* perm, const int32_t* rank, int D, int M, int Mp,
                         int64_t* proxy_ofs, double* P, cudaStream_t s, int keep_max = 0);
// One tree-merge level: nchild children (eigenvector rows X64, sorted sigma,
// permutation, rank, as launch_sort_rank leaves them) -> ceil(nchild / arity)
// node matrices S (Mp x Mp each).  Y holds ceil(nchild / arity) * arity
// Mp x Mp matrices of scratch; with oz, the products are exact-slice ones
// (oz[0] must hold nnode x 5 slices of Mp x arity Mp), else FP64.  Two or
// four kernels.
cudaError_t launch_tree_level(const double* X64, const double* sigma_sorted, const int32_t* perm,
                              const int32_t* rank, int nchild, int arity, int M, int Mp,
                              int keep_max, double* Y, double* S, OzOperand* oz, cudaStream_t s);
// S = P P^T (M x M, stored Mp x Mp), split over the R columns.
cudaError_t launch_merge_gram(const double* P, const int64_t* proxy_ofs, int D, int M, int Mp,
                              int64_t Rmax, double* partial, int nsplit, double* S, cudaStream_t s,
                              OzOperand* oz = nullptr);
int merge_gram_splits(int M, int64_t Rmax);
// Final sort, sign rule, outputs and the SpMM weights W = U_k S_k^-1.
cudaError_t launch_finalize(const double* X64, const float* X32, const double* sigma_sorted,
                            const int32_t* perm, int M, int Mp, int k, double lam_tol_abs,
                            int64_t tol_scale, double* d_sigma, double* d_U, int32_t* d_rank,
                            double* W64, float* W32, cudaStream_t s);

// ---- spmm.cu: V = A'^T W ------------------------------------------------------
template <typename T>
cudaError_t launch_spmm(const int64_t* col_ptr, const int32_t* row_idx, const void* vals,
                        int value_type, int64_t N, int k, const T* W, T* V, cudaStream_t s);
template <typename T>
cudaError_t launch_spmm_patches(const PatchRec* patches, const int64_t* npatches_dev,
                                int max_patches, int k, const T* W, T* V, cudaStream_t s);

// ---- transpose.cu: CSC of A^T from the CSC of a tall A ---------------------------
// A is rows x cols (cols <= 1024); writes t_ptr (rows + 1), t_idx and t_val
// (nnz each, the CSC of A^T with sorted row indices).  Scratch: cnt (rows
// int32), tile_sum (transpose_scratch_words(rows) int64), tmp_idx / tmp_val
// (nnz each).  Six kernels and one memset.
cudaError_t launch_transpose_csc(const int64_t* col_ptr, const int32_t* row_idx, const void* vals,
                                 int value_type, int64_t rows, int cols, int64_t nnz,
                                 int32_t* cnt, int64_t* tile_sum, int32_t* tmp_idx,
                                 void* tmp_val, int64_t* t_ptr, int32_t* t_idx, void* t_val,
                                 cudaStream_t s);
size_t transpose_scratch_words(int64_t rows);

// ---- misc ---------------------------------------------------------------------
cudaError_t launch_check_csc(int M, int64_t N, int64_t nnz, const int64_t* col_ptr,
                             const int32_t* row_idx, int32_t* bad, cudaStream_t s);

}  // namespace rk
