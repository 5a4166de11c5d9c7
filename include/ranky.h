/*
 * ranky.h -- C ABI of the GB300 (sm_103a) column-block SVD of a sparse,
 * short-and-fat matrix (Ranky, Tugay & Gunduz Oguducu, arXiv 2009.09767).
 *
 * The computation (section III of the paper, Algorithm 1):
 *   1. split A (M x N, CSC) into D column blocks A^1 .. A^D;
 *   2. find lonely nodes (rows with no non-zero inside a block) and, in the
 *      RandomChecker mode (Algorithm 2), insert A[m, col] = 1 at a random
 *      column col of that block; the default TRUNCATE mode inserts nothing
 *      and keeps only the numerically non-zero part of each block instead;
 *   3. reduced SVD of every block, A^i = U^i S^i V^i* (Eq. 1), here through
 *      the block cross product A^i A^i^T and a Jacobi eigensolver;
 *   4. proxy P = [U^1 S^1 | ... | U^D S^D] and its SVD, which gives S and U
 *      of A' (Eqs. 2-3: P P^* = A' A'^*);
 *   5. right vectors V = A'^T U S^-1 (the paper leaves these to future work).
 *
 * Conventions for every entry point:
 *   - Indices are 0-based.  CSC: col_ptr int64[N+1] (col_ptr[0] == 0,
 *     non-decreasing, col_ptr[N] == nnz), row_idx int32[nnz] strictly
 *     increasing inside each column, values float32 or float64[nnz].
 *     Stored zeros are allowed and count as zeros.
 *   - "d_" pointers are device pointers (any allocator; the caller owns
 *     them); "h_" pointers are host pointers.  Inputs are never modified.
 *   - All device work is enqueued on the caller's stream (a cudaStream_t
 *     passed as void*, NULL = legacy default stream).  Argument and shape
 *     errors are returned synchronously; errors the device detects
 *     (non-convergence) are written to the plan's status word and returned
 *     by svd_sync().
 *   - No exception crosses the ABI.  A plan is not thread-safe: one run at a
 *     time per plan; different plans may run concurrently on different
 *     streams.
 *   - Outputs: sigma descending; U column-major M x k; V row-major N x k;
 *     each u_i has its largest-magnitude entry positive (first one on a
 *     tie) and v_i takes the same sign.  Singular values whose square is at
 *     or below the rank tolerance get zero columns in V and are not counted
 *     in *rank.
 */
#ifndef RANKY_H
#define RANKY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SVD_OK = 0,
    SVD_ERR_INVALID_ARG = 1,    /* a pointer, size or field is out of range */
    SVD_ERR_INVALID_CSC = 2,    /* svd_check_csc found a malformed CSC */
    SVD_ERR_OOM = 3,            /* device or pinned host allocation failed */
    SVD_ERR_BUDGET = 4,         /* request exceeds a server's memory budget */
    SVD_ERR_CUDA = 5,           /* a CUDA runtime call failed */
    SVD_ERR_NOT_CONVERGED = 6,  /* a Jacobi solve used max_sweeps */
    SVD_ERR_TIMEOUT = 7,        /* a bounded wait ran out */
    SVD_ERR_UNSUPPORTED = 8     /* valid request outside what is built (e.g. M > 1024) */
} svd_status;

typedef enum {
    SVD_PREC_FP64 = 0,   /* everything in FP64 */
    SVD_PREC_MIXED = 1   /* FP32 block Jacobi rotations and SpMM; FP64 cross
                            products, refinement, rank decision and merge */
} svd_precision;

typedef enum {
    SVD_RANKFIX_TRUNCATE = 0,        /* no insertion; drop numerically zero block
                                        directions (default) */
    SVD_RANKFIX_RANDOM = 1,          /* RandomChecker, Algorithm 2 */
    SVD_RANKFIX_NEIGHBOR = 2,        /* NeighborChecker, Algorithm 3: for lonely row m
                                        of block d, a column of block d drawn from the
                                        multiset {n : rows c sharing a non-zero column
                                        with m in another block, once per shared
                                        column, and non-zero at (c, n)}; the 64-bit
                                        Philox word of counter (m, d, 1, 0) selects
                                        entry floor(x T / 2^64) of that list ordered
                                        by column (T its length; T < 2^64 assumed).
                                        All lists come from the input A.  An empty
                                        list inserts nothing. */
    SVD_RANKFIX_NEIGHBOR_RANDOM = 3  /* neighbourRandomChecker, Algorithm 4: as
                                        NEIGHBOR, with the RANDOM column where the
                                        neighbour list is empty */
} svd_rankfix;

typedef enum { SVD_VALUE_F32 = 0, SVD_VALUE_F64 = 1 } svd_value_type;

/* Problem description (section III: A is M x N, split into D column blocks). */
typedef struct {
    int32_t M;                       /* rows, 1 .. 1024 (any >= 1 with SVD_FLAG_TALL) */
    int64_t N;                       /* columns, >= 1 (<= 1024 with SVD_FLAG_TALL) */
    int64_t nnz;                     /* stored entries, >= 0 */
    int32_t value_type;              /* svd_value_type of the values array */
    int32_t num_blocks;              /* D, 1 .. N */
    const int64_t* block_col_bounds; /* host, D+1 boundaries (0 = b_0 < ... <
                                        b_D = N), copied at svd_plan; NULL =
                                        equal widths floor(N/D), remainder to
                                        the last block */
    int32_t k;                       /* triplets returned, 0 = min(M, N) */
    int32_t precision;               /* svd_precision */
    int32_t rank_fix;                /* svd_rankfix */
    uint64_t seed;                   /* rank-fix key (Philox4x32-10) */
    double rank_tol;                 /* > 0: absolute tolerance on singular values;
                                        <= 0: a squared singular value (eigenvalue
                                        of the cross product) counts when it is
                                        above max(M, width) * eps64 * largest */
    int32_t max_sweeps;              /* Jacobi sweep cap, <= 0 = default (40) */
    double jacobi_tol;               /* relative off-diagonal threshold, <= 0 =
                                        default (per precision) */
    int32_t refine_iters;            /* mixed mode: FP64 refinement steps of each
                                        block eigenbasis, < 0 = default (1) */
    int32_t flags;                   /* SVD_FLAG_* */
    int32_t merge_arity;             /* proxy merge: 0 or 1 = one level (section III,
                                        Fig. 1: the SVD of P = [U^1 S^1 | ... |
                                        U^D S^D]); a >= 2 = a tree in which every
                                        node merges a consecutive children (the
                                        multi-level merge of Iwen and Ong that
                                        section II describes and section III
                                        specialises): node matrix S = sum of the
                                        children's Y^T Y, Y = their S U^T, then its
                                        eigendecomposition, level by level up to
                                        the root.  P is never formed: the plan
                                        needs M * R * 8 bytes (R = sum of block
                                        ranks <= D M) less device memory.
                                        Rejected by svd_batch_create and run alone
                                        by the server. */
    int32_t jacobi_cluster;          /* mixed precision: CTAs (thread-block cluster
                                        size 1, 2, 4, 8 or 16) per block matrix in
                                        the FP32 Jacobi launch; 0 = chosen from the
                                        occupancy model (the autotuner sets it from
                                        measurements); a size that cannot be
                                        launched falls back to 0 */
    int32_t merge_rank;              /* k' > 0: every block (and tree node) passes at
                                        most its k' largest singular directions
                                        upward (the approximate truncation of the
                                        multi-level merge; k' >= k required); 0 =
                                        its numerical rank (exact) */
} svd_desc;

#define SVD_FLAG_CHECK_CSC 1   /* svd_run validates the CSC first (synchronous) */
#define SVD_FLAG_SKIP_V 2      /* do not compute V (d_V may be NULL) */
#define SVD_FLAG_TIMING 4      /* record per-stage CUDA events (SVD_Q_STAGE_MS) */
#define SVD_FLAG_DENSE_REFINE 8 /* mixed precision: form the block refinement's G X^T from the
                                 dense block cross product even when the sparse columns
                                 would be cheaper (both give the same result up to
                                 rounding; for testing and timing) */
#define SVD_FLAG_FP64_PRODUCTS 16 /* mixed precision: form the refinement products and
                                 P P^T with FP64 arithmetic instead of exact 8-bit
                                 slices on the bf16 tensor cores (for testing and
                                 timing) */
#define SVD_FLAG_LEGACY_MMA 64 /* mixed precision: run the exact-slice products on the
                                 warp-level mma.sync tensor path instead of tcgen05.mma
                                 with TMEM accumulators (bit-identical results; for
                                 testing and timing) */
#define SVD_FLAG_TALL 32       /* tall-and-skinny A: M rows (any, >= 1) and N <= 1024
                                 columns, split into num_blocks ROW blocks (the row-block
                                 form of section II); block_col_bounds then holds D+1
                                 row boundaries ending at M.  The CSC still describes A.
                                 The plan transposes it on the device and runs the
                                 column-block path on A^T.  A^T's column blocks are A's
                                 row blocks.  The outputs swap layouts:
                                   d_U  float[M*k] (MIXED) or double[M*k] (FP64),
                                        row-major left vectors U = A' V S^-1 (pass the
                                        pointer cast to double*); SVD_FLAG_SKIP_V skips
                                        them (the long side), d_U may then be NULL;
                                   d_V  double[N*k] column-major right vectors.
                                 Lonely nodes, insertions and svd_query results are
                                 those of A^T. A lonely node is a column of A with no
                                 entry inside a row block. An insertion's row is a
                                 column of A and its col is a row of A. Batches and the
                                 server return SVD_ERR_UNSUPPORTED for tall plans. */

/* One RandomChecker insertion: A'[row, col] = 1.0 (Algorithm 2). */
typedef struct {
    int32_t row;
    int32_t block;
    int64_t col;
} svd_patch;

typedef struct svd_plan_s* svd_plan_t;

/* Validate desc, allocate the plan and its device workspace (owned by the
 * plan until svd_free).  The plan fixes what section III's Algorithm 1
 * needs before it reads A: the shape, the D column blocks of the split
 * (floor(N/D) columns each, the remainder in the last, or explicit bounds),
 * the rank fix (Algorithms 2-4, or TRUNCATE) and the precision.  *device_bytes_needed (may be NULL) receives the
 * workspace size.  Returns SVD_ERR_INVALID_ARG / SVD_ERR_UNSUPPORTED /
 * SVD_ERR_OOM without allocating anything on failure. */
svd_status svd_plan(const svd_desc* desc, svd_plan_t* out, size_t* device_bytes_needed);

/* Like svd_plan, on caller-provided device workspace (256-byte aligned, at
 * least svd_plan_bytes); svd_free does not free it. */
svd_status svd_plan_ws(const svd_desc* desc, void* d_workspace, size_t workspace_bytes,
                       svd_plan_t* out);

/* Workspace size for desc without allocating (for admission control). */
svd_status svd_plan_bytes(const svd_desc* desc, size_t* device_bytes_needed);

/* Enqueue one SVD of the CSC matrix on `stream`: section III of the paper
 * for one matrix.  Algorithm 1's split and lonely-node scan, the rank fix
 * (Algorithms 2-4), the block cross products A^i A^i^T (Eq. 2) and their
 * eigensolves (the block SVDs of Eq. 1), the proxy P and the eigensolve of
 * P P^T (Eqs. 2-3), then V = A'^T U S^-1 (left to future work in section V).
 *   d_sigma   double[k]            singular values, descending
 *   d_U       double[M*k]          column-major left vectors
 *   d_V       float[N*k] (MIXED) or double[N*k] (FP64), row-major right
 *             vectors V = A'^T U S^-1; may be NULL with SVD_FLAG_SKIP_V
 *   d_rank    int32[1]             number of singular values above tolerance
 *   d_patches svd_patch[D*M]       rank-fix insertions (value 1.0) in (block,
 *             row) order (may be NULL when rank_fix is TRUNCATE)
 *   d_npatches int64[1]            number of insertions (may be NULL likewise)
 * Asynchronous; call svd_sync() (or synchronise the stream and call
 * svd_sync()) to read device-detected errors. */
svd_status svd_run(svd_plan_t plan, const int64_t* d_col_ptr, const int32_t* d_row_idx,
                   const void* d_vals, double* d_sigma, double* d_U, void* d_V,
                   int32_t* d_rank, svd_patch* d_patches, int64_t* d_npatches,
                   void* stream);

/* Same computation (section III) from HOST buffers: copies the CSC to plan-owned device
 * memory, runs, and copies sigma, U, V (unless SVD_FLAG_SKIP_V or h_V ==
 * NULL), rank and patches back.  Synchronous; pinned host memory makes the
 * copies fast but is not required.  When h_V is page-locked (cudaHostAlloc,
 * cudaHostRegister) and the rank fix is TRUNCATE, the device writes V into
 * it directly, with no staging buffer and no copy. */
svd_status svd_run_host(svd_plan_t plan, const int64_t* h_col_ptr, const int32_t* h_row_idx,
                        const void* h_vals, double* h_sigma, double* h_U, void* h_V,
                        int32_t* h_rank, svd_patch* h_patches, int64_t* h_npatches,
                        void* stream);

/* Wait for the plan's last run and return its device-detected status: a
 * Jacobi eigensolve of a block or of P P^T that used max_sweeps
 * (SVD_ERR_NOT_CONVERGED), or a bounded wait of the tensor-core product
 * that ran out (SVD_ERR_TIMEOUT). */
svd_status svd_sync(svd_plan_t plan);

/* Synchronous CSC validation (structure only): col_ptr monotone and ending at
 * nnz, rows in [0, M) and strictly increasing inside each column. */
svd_status svd_check_csc(int32_t M, int64_t N, int64_t nnz, const int64_t* d_col_ptr,
                         const int32_t* d_row_idx, void* stream);

/* Copy an intermediate of the last run to host memory (after svd_sync):
 * the quantities of Algorithm 1 and Eqs. 1-3 named below.
 * `bytes` must equal the item's size; returns SVD_ERR_INVALID_ARG otherwise. */
enum {
    SVD_Q_BLOCK_BOUNDS = 1,  /* int64[D+1] column boundaries (Algorithm 1 split) */
    SVD_Q_LONELY = 2,        /* uint8[D*M] lonely-node flags (Algorithm 1) */
    SVD_Q_ROW_NONEMPTY = 3,  /* uint8[M] rows with a non-zero anywhere in A */
    SVD_Q_BLOCK_RANKS = 4,   /* int32[D] numerical rank r_i of each block */
    SVD_Q_BLOCK_SIGMA = 5,   /* double[D*M] block singular values, descending */
    SVD_Q_BLOCK_GRAM = 6,    /* double[M*M] A^i A^i^T of block `index` (row-major) */
    SVD_Q_PROXY_COLS = 7,    /* int64[1] R = sum r_i */
    SVD_Q_PROXY = 8,         /* double[M*R] proxy P, column-major */
    SVD_Q_SWEEPS = 9,        /* int32[D+1] Jacobi sweeps per block, then the merge */
    SVD_Q_LAUNCHES = 10,     /* int64[1] kernels launched by the last run */
    SVD_Q_MERGE_GRAM = 11,   /* double[M*M] P P^T (row-major) */
    SVD_Q_STAGE_MS = 12,     /* float[9] stage times of the last run (SVD_FLAG_TIMING):
                                partition+lonely, cross products, block Jacobi,
                                block refinement, sort+proxy, P P^T, merge
                                eigensolve, outputs, V */
    SVD_Q_STAGE_TOTAL = 13   /* double[10]: per-stage milliseconds summed over the
                                runs since the previous such query, then the run
                                count; resets the sums */
};
svd_status svd_query(svd_plan_t plan, int32_t what, int64_t index, void* h_dst, size_t bytes);

/* ---- Batches (no counterpart in the paper: svd_run's section III
 * computation for many matrices): many plans in one pass (all plans' block eigensolves in one
 * persistent launch, likewise the merge eigensolves; the per-matrix stages on
 * a pool of worker streams).  Each plan keeps its own workspace; the batch
 * object adds the work lists, streams and (optionally) a CUDA graph. */
typedef struct {
    const int64_t* d_col_ptr;
    const int32_t* d_row_idx;
    const void* d_vals;
    double* d_sigma;
    double* d_U;
    void* d_V;
    int32_t* d_rank;
    svd_patch* d_patches;   /* may be NULL (with d_npatches) */
    int64_t* d_npatches;
} svd_io;

typedef struct svd_batch_s* svd_batch_t;

#define SVD_BATCH_GRAPH 1   /* capture the pass into a CUDA graph on the first run and replay
                               it on later runs that pass the same svd_io buffers (a different
                               set of buffers is captured anew) */

/* Group n plans (which must stay alive until svd_batch_free; each plan in at
 * most one batch that runs at a time). */
svd_status svd_batch_create(int32_t n, const svd_plan_t* plans, int32_t flags, svd_batch_t* out);
/* Enqueue one SVD per plan, ios[i] for plans[i] (same conventions as
 * svd_run), on `stream`; asynchronous. */
svd_status svd_batch_run(svd_batch_t batch, const svd_io* ios, void* stream);
/* Wait for the batch and return the worst device-detected status. */
svd_status svd_batch_sync(svd_batch_t batch);
/* Kernels launched by the last non-replayed run (0 if none). */
int64_t svd_batch_launches(svd_batch_t batch);
void svd_batch_free(svd_batch_t batch);

/* ---- Serving (no counterpart in the paper: svd_run's section III
 * computation for requests that arrive over time): a continuous-batching SVD service on one GPU.  A scheduler
 * thread admits submitted requests in arrival order as stream slots and room
 * in the device-memory budget free up; each admitted request gets its plan
 * workspace, CSC and outputs from one pool allocation inside the budget and
 * runs on its slot's stream (host->device copies, svd_run, device->host
 * copies), overlapping with the requests already running. */
typedef struct svd_server_s* svd_server_t;

typedef struct {
    svd_desc desc;             /* block_col_bounds (if any) is copied at submit */
    const int64_t* h_col_ptr;  /* host CSC; must stay valid until the request is done */
    const int32_t* h_row_idx;
    const void* h_vals;
    double* h_sigma;           /* host outputs (as svd_run_host); pinned memory is faster */
    double* h_U;
    void* h_V;                 /* may be NULL: V is not copied back */
    int32_t* h_rank;
} svd_request;

/* budget_bytes: device memory the service may use (allocated once);
 * max_inflight: requests on the GPU at the same time (one stream each). */
svd_status svd_server_create(size_t budget_bytes, int32_t max_inflight, svd_server_t* out);
/* Queue a request; SVD_ERR_BUDGET when it can never fit in the budget. */
svd_status svd_server_submit(svd_server_t srv, const svd_request* req, uint64_t* ticket);
/* *done = 1 once finished; *result = the request's status (SVD_OK on success). */
svd_status svd_server_poll(svd_server_t srv, uint64_t ticket, int32_t* done, svd_status* result);
/* Block until the request finishes or timeout_s passes (SVD_ERR_TIMEOUT). */
svd_status svd_server_wait(svd_server_t srv, uint64_t ticket, double timeout_s, svd_status* result);
/* Drop a request that has not been admitted yet (its result becomes
 * SVD_ERR_INVALID_ARG); running requests cannot be cancelled. */
svd_status svd_server_cancel(svd_server_t srv, uint64_t ticket);
/* Submit, admission and completion times (seconds, steady clock). */
svd_status svd_server_times(svd_server_t srv, uint64_t ticket, double* t_submit,
                            double* t_admit, double* t_done);
/* Forget a finished ticket. */
svd_status svd_server_release(svd_server_t srv, uint64_t ticket);
/* out[8]: submitted, completed, failed, rejected, running, queued, pool bytes
 * in use, peak pool bytes. */
svd_status svd_server_stats(svd_server_t srv, int64_t* out);
/* Host-side fault injection for tests: make the request with `ticket`
 * (submitted later) fail its pool allocation, or carry a malformed CSC. */
#define SVD_INJECT_ALLOC 1
#define SVD_INJECT_BAD_CSC 2
svd_status svd_server_inject(svd_server_t srv, int32_t what, uint64_t ticket);
/* Drops queued requests, waits for running ones, frees everything. */
void svd_server_destroy(svd_server_t srv);

/* Right singular vectors without any device allocation.  The paper has no
 * counterpart: this serves callers that must not allocate device memory on
 * their call path (services that split the GPU into fixed budgets at start-up
 * and refuse later allocations; latency-bound callers that cannot take
 * cudaMalloc's implicit device-wide synchronisation or its failure under
 * memory pressure).
 *
 * Computes d_V = A'^T U_k S_k^-1 (row-major N x k, float32 when v_type is
 * SVD_VALUE_F32, float64 when SVD_VALUE_F64) from a CSC matrix and the
 * singular values d_sigma (double[k], descending) and left vectors d_U
 * (double, column-major M x k) that svd_run returned; d_patches / d_npatches
 * (both NULL or both set, max_patches = capacity) add RandomChecker
 * insertions as svd_run does.  Columns whose squared singular value is at or
 * below the rank tolerance (rank_tol^2 when rank_tol > 0, else
 * max(M, N) * eps64 * sigma_1^2) are zero.
 *
 * Its scratch (the M x k weights) is a static device array of 4 MiB that
 * every GPU loading the library keeps until the process exits:
 * M * k * sizeof(V element) above 4 MiB returns SVD_ERR_UNSUPPORTED without
 * enqueuing work.  All calls on a device share the array and it keeps the
 * last call's contents; every call rewrites what it reads, but calls whose
 * kernels overlap on the GPU race on it.  The first call on each device
 * looks up the array's device address; make it before any stream capture.
 * Asynchronous on `stream`; argument errors return synchronously. */
svd_status svd_right_vectors_static(int32_t M, int64_t N, int64_t nnz, int32_t value_type,
                                    const int64_t* d_col_ptr, const int32_t* d_row_idx,
                                    const void* d_vals, int32_t k, const double* d_sigma,
                                    const double* d_U, double rank_tol,
                                    const svd_patch* d_patches, const int64_t* d_npatches,
                                    int64_t max_patches, int32_t v_type, void* d_V,
                                    void* stream);

/* ---- FP64-accurate dense product on the tensor cores -----------------------
 * C = A B^T for FP64 A (m x k, row-major, leading dimension lda) and B
 * (n x k, ldb), the product behind the merge's P P^T (section III, Eq. 3:
 * P P^* = A A^*) and the mixed-precision refinement of every block basis.
 * Each row is scaled by its power-of-two magnitude bound and cut into
 * `slices` (3 or 5) signed 8-bit integer slices (exact in bf16); every pair of
 * slices whose weights are within the kept range is multiplied on the bf16
 * tensor cores with exact integer sums, and the sums are combined in 64-bit
 * integers and converted to FP64 once (error-free splitting after Ozaki et
 * al., Numer. Algorithms 59, 2012).  The error is below about
 * 2^(2 - 8 slices) k 2^(e_i + e_j), e_i the exponent bound of row i of A, e_j
 * of row j of B (5 slices: ~2^-38 k of the row scales).
 *   m, n          1 .. 2^20; k >= 1
 *   d_C           row-major m x n (ldc >= n), overwritten
 *   flags         SVD_PRODUCT_SYM: B is A (n == m, d_B ignored); only the
 *                 upper triangle is formed, then mirrored.
 *                 SVD_PRODUCT_LEGACY_MMA: warp-level mma.sync instead of
 *                 tcgen05.mma with TMEM accumulators (bit-identical result)
 *   d_work        device scratch of svd_exact_product_bytes(...) bytes,
 *                 caller-owned; nothing is allocated
 *   d_err         device int32 (may be NULL), set to 1 when a bounded wait of
 *                 the tcgen05 kernel ran out (its tile is then not written)
 * Asynchronous on `stream`; argument errors return synchronously. */
#define SVD_PRODUCT_SYM 1
#define SVD_PRODUCT_LEGACY_MMA 2
size_t svd_exact_product_bytes(int32_t m, int32_t n, int64_t k, int32_t slices);
svd_status svd_exact_product(int32_t m, int32_t n, int64_t k, const double* d_A, int64_t lda,
                             const double* d_B, int64_t ldb, double* d_C, int64_t ldc,
                             int32_t slices, int32_t flags, void* d_work, size_t work_bytes,
                             int32_t* d_err, void* stream);

void svd_free(svd_plan_t plan);
const char* svd_status_str(svd_status s);
int32_t svd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RANKY_H */
