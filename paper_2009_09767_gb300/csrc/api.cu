// api.cu -- the C ABI (include/ranky.h): plan, run, query, free.
//
// svd_run enqueues, on the caller's stream, the steps of Ranky's Algorithm 1
// (arXiv 2009.09767, section III) followed by the right-vector product:
//   occupancy -> lonely flags (+ RandomChecker patches) -> block cross
//   products -> block eigensolves (FP64 Jacobi, or FP32 Jacobi + FP64
//   refinement) -> sort / block rank -> proxy P -> P P^T -> merge eigensolve
//   -> sigma, U, rank, W = U_k S_k^-1 -> V = A'^T W.
// Nothing is synchronised inside svd_run: block ranks, the proxy width and
// convergence are read by later kernels from device memory.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ranky.h"
#include "common.cuh"
#include "kernels.h"
#include "batch_engine.h"

using namespace rk;

namespace {
// stages timed with SVD_FLAG_TIMING (see SVD_Q_STAGE_MS)
constexpr int kStages = 9;
constexpr int kRing = 64;

}

struct svd_plan_s {
    svd_desc d{};
    int M = 0, Mp = 0, D = 0, k = 0;
    int64_t N = 0, nnz = 0;
    bool mixed = false, random = false;
    bool neighbor = false;  // Algorithm 3 (or 4 with the RandomChecker fallback)
    bool patched = false;   // any insertion mode
    bool tall = false;      // SVD_FLAG_TALL: the caller's CSC is this problem's transpose
    double jac_tol = 0.0;
    int max_sweeps = 40, refine_iters = 2, merge_refine_iters = 3;
    double rr_kappa = 32.0;    // Rayleigh-Ritz clusters: first-order mixing estimate >= 1 / rr_kappa
    std::vector<int64_t> bounds_h;
    int nchunks = 0;
    int W = 0;  // bitmap words per block
    int nsplit = 1;
    int64_t Rmax = 0;
    int arity = 0;          // tree merge: children per node (>= 2), 0 = one-level merge
    int keep = 0;           // k' > 0: directions a block / node passes upward
    int Dcap = 0;           // D rounded up to a multiple of the arity (tree scratch)

    char* arena = nullptr;
    size_t arena_bytes = 0;
    bool owns_arena = true;

    int64_t* bounds_d = nullptr;
    int32_t* chunk_block = nullptr;
    int64_t* chunk_lo = nullptr;
    int64_t* chunk_hi = nullptr;
    uint32_t* occ = nullptr;
    uint32_t* row_ne = nullptr;
    uint32_t* lonely = nullptr;
    PatchRec* patches = nullptr;
    int64_t* patch_ofs = nullptr;
    uint32_t* lonely_any = nullptr;     // neighbour modes: rows lonely in some block
    unsigned long long* cooc = nullptr; // neighbour modes: M x M row co-occurrence counts
    PatchRec* slots = nullptr;          // neighbour modes: one per lonely node
    int64_t* slot_ofs = nullptr;
    // tall plans: the caller's CSC (of the N x M transpose of this problem) for
    // the next run, and its transpose (this problem's CSC) with the scratch
    const int64_t* src_col_ptr = nullptr;
    const int32_t* src_row_idx = nullptr;
    const void* src_vals = nullptr;
    int64_t* t_ptr = nullptr;
    int32_t* t_idx = nullptr;
    char* t_val = nullptr;
    int32_t* t_cnt = nullptr;
    int64_t* t_tile = nullptr;
    int32_t* t_tmp_idx = nullptr;
    char* t_tmp_val = nullptr;
    double* G64 = nullptr;
    double* Gw64 = nullptr;    // FP64: Jacobi working copy
    double* Vt64 = nullptr;    // FP64 eigenvector rows (FP64 solve, or converted FP32 + refined)
    float* G32 = nullptr;
    float* Vt32 = nullptr;
    double* Xn = nullptr;      // refinement output
    double* RW1 = nullptr;
    double* RW2 = nullptr;
    double* RW3 = nullptr;
    double* lam = nullptr;
    double* norms = nullptr;
    double* bsig = nullptr;
    int32_t* bperm = nullptr;
    int32_t* brank = nullptr;
    int64_t* pofs = nullptr;
    double* P = nullptr;
    double* partial = nullptr;
    double* S64 = nullptr;
    double* Sw64 = nullptr;
    double* SV64 = nullptr;
    float* S32 = nullptr;
    float* SV32 = nullptr;
    double* SXn = nullptr;
    double* SR1 = nullptr;
    double* SR2 = nullptr;
    double* SR3 = nullptr;
    // exact-slice operands of the tensor-core products (mixed precision)
    bool use_oz = false;
    uint16_t* oz_sl[2] = {nullptr, nullptr};
    // published pair rotations of the FP32 solver: D blocks, then the merge
    char* jwork = nullptr;
    unsigned long long* oz_amax[2] = {nullptr, nullptr};
    double* slam = nullptr;
    double* snorm = nullptr;
    double* msig = nullptr;
    int32_t* mperm = nullptr;
    int32_t* mrank = nullptr;
    double* W64 = nullptr;
    float* W32 = nullptr;
    int32_t* sweeps = nullptr;
    int32_t* dev_err = nullptr;  // [0]: a bounded wait of the tcgen05 products ran out
    // cluster Rayleigh-Ritz of the refinement (mixed): D blocks, then the merge
    int32_t* rr_order = nullptr;
    int32_t* rr_cstart = nullptr;
    int32_t* rr_csize = nullptr;
    int32_t* rr_ncl = nullptr;
    int32_t* rr_cid = nullptr;
    int32_t* rr_rowmax = nullptr;

    // svd_run_host staging (lazily allocated)
    char* host_arena = nullptr;
    size_t host_arena_bytes = 0;

    cudaStream_t last_stream = nullptr;
    int64_t launches = 0;
    bool ran = false;
    // per-stage CUDA events (SVD_FLAG_TIMING), a ring of kRing runs so that
    // stage totals accumulate without synchronising inside svd_run
    cudaEvent_t ev[kRing][kStages + 1] = {};
    bool ev_pending[kRing] = {};
    int64_t run_index = 0;
    double stage_total[kStages] = {};
    int64_t stage_runs = 0;
    bool timing = false;
    int cur_slot = -1;
};

namespace {

constexpr int64_t kChunkCols = 512;

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carver {
    char* base;
    size_t off = 0;
    bool dry;
    template <typename T>
    T* take(size_t count) {
        const size_t at = off;
        off = align_up(off + count * sizeof(T));
        return dry ? nullptr : reinterpret_cast<T*>(base + at);
    }
};

// The short-and-fat problem a descriptor poses: A itself, or, for
// SVD_FLAG_TALL, A^T (its column blocks are the row blocks of A).
svd_desc short_fat(const svd_desc& d) {
    svd_desc t = d;
    if (d.flags & SVD_FLAG_TALL) {
        t.M = (int32_t)std::min<int64_t>(d.N, INT32_MAX);
        t.N = d.M;
    }
    return t;
}

svd_status validate_short_fat(const svd_desc* d);

svd_status validate_desc(const svd_desc* d) {
    if (!d) return SVD_ERR_INVALID_ARG;
    if ((d->flags & SVD_FLAG_TALL) && (d->M < 1 || d->N < 1)) return SVD_ERR_INVALID_ARG;
    const svd_desc t = short_fat(*d);
    return validate_short_fat(&t);
}

svd_status validate_short_fat(const svd_desc* d) {
    if (d->M < 1 || d->N < 1 || d->nnz < 0) return SVD_ERR_INVALID_ARG;
    if (d->value_type != SVD_VALUE_F32 && d->value_type != SVD_VALUE_F64) return SVD_ERR_INVALID_ARG;
    if (d->num_blocks < 1 || (int64_t)d->num_blocks > d->N) return SVD_ERR_INVALID_ARG;
    if (d->precision != SVD_PREC_FP64 && d->precision != SVD_PREC_MIXED) return SVD_ERR_INVALID_ARG;
    if (d->rank_fix < SVD_RANKFIX_TRUNCATE || d->rank_fix > SVD_RANKFIX_NEIGHBOR_RANDOM)
        return SVD_ERR_INVALID_ARG;
    if (d->k < 0) return SVD_ERR_INVALID_ARG;
    const int64_t kmax = std::min<int64_t>(d->M, d->N);
    if (d->k > kmax) return SVD_ERR_INVALID_ARG;
    if (d->M > kMaxM) return SVD_ERR_UNSUPPORTED;
    if (d->merge_arity < 0 || d->merge_rank < 0) return SVD_ERR_INVALID_ARG;
    if (d->merge_rank > 0) {
        const int64_t k = d->k > 0 ? d->k : kmax;
        if (d->merge_rank < k) return SVD_ERR_INVALID_ARG;
    }
    if (d->block_col_bounds) {
        const int64_t* b = d->block_col_bounds;
        if (b[0] != 0 || b[d->num_blocks] != d->N) return SVD_ERR_INVALID_ARG;
        for (int i = 0; i < d->num_blocks; ++i)
            if (b[i + 1] <= b[i]) return SVD_ERR_INVALID_ARG;
    }
    return SVD_OK;
}

// Lay out (or size, when dry) the plan's device workspace.
void carve(svd_plan_s* p, Carver& c) {
    const int D = p->D, M = p->M, Mp = p->Mp;
    const int64_t mm = (int64_t)Mp * Mp;
    p->bounds_d = c.take<int64_t>(D + 1);
    p->chunk_block = c.take<int32_t>(p->nchunks);
    p->chunk_lo = c.take<int64_t>(p->nchunks);
    p->chunk_hi = c.take<int64_t>(p->nchunks);
    p->occ = c.take<uint32_t>((size_t)D * p->W);
    p->row_ne = c.take<uint32_t>(p->W);
    p->lonely = c.take<uint32_t>((size_t)D * p->W);
    p->patches = c.take<PatchRec>((size_t)D * M);
    p->patch_ofs = c.take<int64_t>(D + 1);
    if (p->tall) {
        const size_t sv = p->d.value_type == SVD_VALUE_F32 ? 4 : 8;
        const int64_t nz = std::max<int64_t>(p->nnz, 1);
        p->t_ptr = c.take<int64_t>(p->N + 1);
        p->t_idx = c.take<int32_t>(nz);
        p->t_val = c.take<char>(nz * sv);
        p->t_cnt = c.take<int32_t>(p->N);
        p->t_tile = c.take<int64_t>(transpose_scratch_words(p->N));
        p->t_tmp_idx = c.take<int32_t>(nz);
        p->t_tmp_val = c.take<char>(nz * sv);
    }
    if (p->neighbor) {
        p->lonely_any = c.take<uint32_t>(p->W);
        p->cooc = c.take<unsigned long long>((size_t)M * M);
        p->slots = c.take<PatchRec>((size_t)D * M);
        p->slot_ofs = c.take<int64_t>(D + 1);
    }
    p->G64 = c.take<double>((size_t)D * mm);
    p->Vt64 = c.take<double>((size_t)D * mm);
    if (p->mixed) {
        p->G32 = c.take<float>((size_t)D * mm);
        p->Vt32 = c.take<float>((size_t)D * mm);
        p->jwork = c.take<char>(jacobi_work_bytes(D + 1, Mp));
        if (p->refine_iters > 0 || p->arity) {
            p->Xn = c.take<double>((size_t)D * mm);
            p->RW1 = c.take<double>((size_t)D * mm);
            p->RW2 = c.take<double>((size_t)std::max(D, p->Dcap) * mm);   // + tree scratch Y
            p->RW3 = c.take<double>((size_t)D * mm);
            p->lam = c.take<double>((size_t)D * Mp);
            p->norms = c.take<double>(D);
        }
    } else {
        p->Gw64 = c.take<double>((size_t)std::max(D, p->Dcap) * mm);   // + tree scratch Y
    }
    p->bsig = c.take<double>((size_t)D * M);
    p->bperm = c.take<int32_t>((size_t)D * M);
    p->brank = c.take<int32_t>(D);
    p->pofs = c.take<int64_t>(D + 1);
    p->P = c.take<double>((size_t)M * p->Rmax);
    p->partial = c.take<double>((size_t)p->nsplit * mm);
    p->S64 = c.take<double>(mm);
    p->SV64 = c.take<double>(mm);
    if (p->mixed) {
        p->S32 = c.take<float>(mm);
        p->SV32 = c.take<float>(mm);
        p->SXn = c.take<double>(mm);
        p->SR1 = c.take<double>(mm);
        p->SR2 = c.take<double>(mm);
        p->SR3 = c.take<double>(mm);
        p->slam = c.take<double>(Mp);
        p->snorm = c.take<double>(1);
        p->W32 = c.take<float>((size_t)M * std::max(p->k, 1));
    } else {
        p->Sw64 = c.take<double>(mm);
        p->W64 = c.take<double>((size_t)M * std::max(p->k, 1));
    }
    if (p->use_oz) {
        const int64_t blk = (p->refine_iters > 0 || p->arity)
                                ? oz_operand_elems(std::max(D, p->Dcap), 5, Mp, Mp) : 0;
        const int64_t mrg = std::max(oz_operand_elems(1, 5, M, p->Rmax), oz_operand_elems(1, 5, Mp, Mp));
        const int64_t rows = round_up(Mp, OZ_ROW_PAD);
        p->oz_sl[0] = c.take<uint16_t>((size_t)std::max(blk, mrg));
        p->oz_sl[1] = c.take<uint16_t>((size_t)std::max(blk, oz_operand_elems(1, 5, Mp, Mp)));
        p->oz_amax[0] = c.take<unsigned long long>((size_t)D * rows);
        p->oz_amax[1] = c.take<unsigned long long>((size_t)D * rows);
    }
    p->msig = c.take<double>(M);
    p->mperm = c.take<int32_t>(M);
    p->mrank = c.take<int32_t>(1);
    p->sweeps = c.take<int32_t>(D + 1 + (p->arity ? D : 0));   // blocks, merge, tree nodes
    p->dev_err = c.take<int32_t>(4);
    if (p->mixed) {
        p->rr_order = c.take<int32_t>((size_t)(D + 1) * Mp);
        p->rr_cstart = c.take<int32_t>((size_t)(D + 1) * (Mp / 2));
        p->rr_csize = c.take<int32_t>((size_t)(D + 1) * (Mp / 2));
        p->rr_ncl = c.take<int32_t>(D + 1);
        p->rr_cid = c.take<int32_t>((size_t)(D + 1) * Mp);
        p->rr_rowmax = c.take<int32_t>((size_t)(D + 1) * Mp);
    }
}

// Cluster Rayleigh-Ritz work of matrix `first` onwards (the D blocks from 0,
// the merge at D).
RRWork rr_work(svd_plan_s* p, int first) {
    const int Mp = p->Mp;
    return RRWork{p->rr_order + (size_t)first * Mp, p->rr_cstart + (size_t)first * (Mp / 2),
                  p->rr_csize + (size_t)first * (Mp / 2), p->rr_ncl + first,
                  p->rr_cid + (size_t)first * Mp, p->rr_rowmax + (size_t)first * Mp, p->rr_kappa,
                  p->M, 0};
}

svd_status fill_plan(const svd_desc* d, svd_plan_s* p) {
    p->d = *d;
    p->d.block_col_bounds = nullptr;
    p->M = d->M;
    p->N = d->N;
    p->nnz = d->nnz;
    p->D = d->num_blocks;
    p->k = d->k > 0 ? d->k : (int)std::min<int64_t>(d->M, d->N);
    p->mixed = d->precision == SVD_PREC_MIXED;
    p->random = d->rank_fix == SVD_RANKFIX_RANDOM;
    p->neighbor = d->rank_fix == SVD_RANKFIX_NEIGHBOR || d->rank_fix == SVD_RANKFIX_NEIGHBOR_RANDOM;
    p->patched = p->random || p->neighbor;
    p->tall = (d->flags & SVD_FLAG_TALL) != 0;
    p->use_oz = p->mixed && !(d->flags & SVD_FLAG_FP64_PRODUCTS);
    p->Mp = jacobi_pad(d->M);
    p->W = (d->M + 31) / 32;
    p->max_sweeps = d->max_sweeps > 0 ? d->max_sweeps : 40;
    p->jac_tol = d->jacobi_tol > 0 ? d->jacobi_tol : (p->mixed ? 8.0 * Eps<float>::value : 1e-14);
    p->refine_iters = d->refine_iters >= 0 ? d->refine_iters : 2;
    p->bounds_h.resize(p->D + 1);
    if (d->block_col_bounds) {
        std::copy(d->block_col_bounds, d->block_col_bounds + p->D + 1, p->bounds_h.begin());
    } else {
        const int64_t base = d->N / p->D;
        for (int i = 0; i <= p->D; ++i) p->bounds_h[i] = base * i;
        p->bounds_h[p->D] = d->N;
    }
    int64_t nch = 0;
    for (int i = 0; i < p->D; ++i)
        nch += ceil_div(p->bounds_h[i + 1] - p->bounds_h[i], kChunkCols);
    if (nch > (int64_t)1 << 30) return SVD_ERR_UNSUPPORTED;
    p->nchunks = (int)nch;
    p->arity = d->merge_arity >= 2 ? d->merge_arity : 0;
    p->keep = d->merge_rank;
    p->Dcap = p->arity ? (int)round_up(p->D, p->arity) : p->D;
    int64_t rmax = 0;
    for (int i = 0; i < p->D; ++i) {
        int64_t r = std::min<int64_t>(p->M, p->bounds_h[i + 1] - p->bounds_h[i]);
        if (p->keep > 0) r = std::min<int64_t>(r, p->keep);
        rmax += r;
    }
    // the tree merge never forms the proxy P
    p->Rmax = p->arity ? 1 : std::max<int64_t>(rmax, 1);
    p->nsplit = merge_gram_splits(p->M, p->Rmax);
    return SVD_OK;
}

#define LAUNCH(plan, n, expr)                                  \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) {                               \
            fprintf(stderr, "ranky: %s: %s\n", #expr, cudaGetErrorString(_e)); \
            cudaGetLastError();                                \
            return SVD_ERR_CUDA;                               \
        }                                                      \
        (plan)->launches += (n);                               \
    } while (0)

#define CU(expr)                                                \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) {                                \
            fprintf(stderr, "ranky: %s: %s\n", #expr, cudaGetErrorString(_e)); \
            cudaGetLastError();                                 \
            return SVD_ERR_CUDA;                                \
        }                                                       \
    } while (0)

struct RunIO {
    const int64_t* col_ptr;
    const int32_t* row_idx;
    const void* vals;
    double* sigma;
    double* U;
    void* V;
    int32_t* rank;
    svd_patch* patches;
    int64_t* npatches;
};

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return st != cudaStreamCaptureStatusNone;
}

// Stage-time events of one run (SVD_FLAG_TIMING; not while a stream is
// being captured into a graph).
void timing_begin(svd_plan_s* p, cudaStream_t s) {
    p->cur_slot = -1;
    if (!p->timing || capturing(s)) return;
    const int slot = (int)(p->run_index % kRing);
    if (p->ev_pending[slot]) {
        // the run that used this slot kRing runs ago: fold its times into the totals
        cudaEventSynchronize(p->ev[slot][kStages]);
        for (int i = 0; i < kStages; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p->ev[slot][i], p->ev[slot][i + 1]);
            p->stage_total[i] += ms;
        }
        ++p->stage_runs;
        p->ev_pending[slot] = false;
    }
    p->cur_slot = slot;
}

void mark(svd_plan_s* p, int i, cudaStream_t s) {
    if (p->cur_slot >= 0) cudaEventRecord(p->ev[p->cur_slot][i], s);
}

// Up to the block eigensolve: Algorithm 1 scan, Algorithm 2 insertions, Eq. 2
// cross products; leaves the matrices the block Jacobi works on.
svd_status phase_pre(svd_plan_s* p, const RunIO& io, cudaStream_t s) {
    const int D = p->D, M = p->M, Mp = p->Mp;
    const int64_t mm = (int64_t)Mp * Mp;
    const int vt = p->d.value_type;
    p->launches = 0;
    timing_begin(p, s);
    mark(p, 0, s);
    if (p->tall)  // the caller's CSC is of the N x M transpose: form this problem's CSC
        LAUNCH(p, 6, launch_transpose_csc(p->src_col_ptr, p->src_row_idx, p->src_vals, vt, p->N,
                                          M, p->nnz, p->t_cnt, p->t_tile, p->t_tmp_idx,
                                          p->t_tmp_val, p->t_ptr, p->t_idx, p->t_val, s));
    CU(cudaMemsetAsync(p->occ, 0, sizeof(uint32_t) * (size_t)D * p->W, s));
    LAUNCH(p, 1, launch_occupancy(io.col_ptr, io.row_idx, io.vals, vt, M, p->nchunks,
                                  p->chunk_block, p->chunk_lo, p->chunk_hi, p->occ, s));
    PatchRec* ext = reinterpret_cast<PatchRec*>(io.patches);
    if (!p->neighbor) {
        LAUNCH(p, 1, launch_lonely_patches(p->occ, D, M, p->bounds_d, p->random ? 1 : 0,
                                           p->d.seed, p->row_ne, p->lonely, p->patches,
                                           p->patch_ofs, ext, io.npatches, nullptr, s));
    } else {
        LAUNCH(p, 1, launch_lonely_patches(p->occ, D, M, p->bounds_d, 2, p->d.seed, p->row_ne,
                                           p->lonely, p->slots, p->slot_ofs, nullptr, nullptr,
                                           p->lonely_any, s));
        LAUNCH(p, 3, launch_neighbor_patches(io.col_ptr, io.row_idx, io.vals, vt, M, p->N, D,
                                             p->bounds_d, p->lonely_any, p->cooc,
                                             p->d.rank_fix == SVD_RANKFIX_NEIGHBOR_RANDOM,
                                             p->d.seed, p->slots, p->slot_ofs, p->patches,
                                             p->patch_ofs, ext, io.npatches, s));
    }
    mark(p, 1, s);
    CU(cudaMemsetAsync(p->G64, 0, sizeof(double) * (size_t)D * mm, s));
    LAUNCH(p, 1, launch_gram(io.col_ptr, io.row_idx, io.vals, vt, Mp, p->nchunks, p->chunk_block,
                             p->chunk_lo, p->chunk_hi, p->G64, s));
    if (p->patched)
        LAUNCH(p, 1, launch_gram_patches(io.col_ptr, io.row_idx, io.vals, vt, Mp, D, p->patches,
                                         p->patch_ofs, D * M, p->G64, s));
    LAUNCH(p, 1, launch_symmetrize(p->G64, D, Mp, s));
    mark(p, 2, s);
    if (!p->mixed)
        CU(cudaMemcpyAsync(p->Gw64, p->G64, sizeof(double) * D * mm, cudaMemcpyDeviceToDevice, s));
    else
        LAUNCH(p, 1, launch_convert_f64_f32(p->G64, p->G32, (int64_t)D * mm, s));
    return SVD_OK;
}

svd_status block_jacobi(svd_plan_s* p, cudaStream_t s) {
    if (!p->mixed)
        LAUNCH(p, 1, launch_jacobi<double>(p->Gw64, p->Vt64, p->D, p->Mp, p->max_sweeps,
                                           p->jac_tol, p->sweeps, s));
    else
        LAUNCH(p, 1, launch_jacobi<float>(p->G32, p->Vt32, p->D, p->Mp, p->max_sweeps, p->jac_tol,
                                          p->sweeps, s, p->jwork, p->d.jacobi_cluster));
    return SVD_OK;
}

// Kernels one refinement step launches (see launch_refine): the sparse
// route adds the transpose of X and the scatter, the exact-slice products
// two kernels per operand split.
int refine_launches(bool sparse, bool oz, int nchunks, bool rr) {
    const int scatter = sparse && nchunks > 0 ? 1 : 0;
    const int extra = rr ? 3 : 0;   // five kernels in place of the two of the norm-threshold step
    if (oz) return (sparse ? 15 + scatter : 17) + extra;
    return (sparse ? 7 + scatter : 7) + extra;
}

void oz_ops(svd_plan_s* p, OzOperand* ops) {
    const int tc = (p->d.flags & SVD_FLAG_LEGACY_MMA) ? 0 : 1;
    for (int i = 0; i < 2; ++i)
        ops[i] = OzOperand{p->oz_sl[i], p->oz_amax[i], 0, 0, 0, 0, tc, p->dev_err};
}

// The tree merge (merge_arity >= 2): every level forms the node matrices
// S_node = sum over the node's children of Y_c^T Y_c (Y_c = S_c U_c^T, the
// child's proxy columns as rows), eigensolves them as the blocks were
// (mixed: FP32 Jacobi + refinement; FP64: FP64 Jacobi), sorts and ranks
// them, and passes their bases up; the root's matrix goes to S64 for the
// merge eigensolve.  X: the blocks' eigenvector rows (FP64).
svd_status tree_merge(svd_plan_s* p, const double* X, OzOperand* oz, cudaStream_t s) {
    const int D = p->D, M = p->M, Mp = p->Mp, a = p->arity;
    const int64_t mm = (int64_t)Mp * Mp;
    int n = D, node_off = 0;
    for (;;) {
        const int nn = (int)ceil_div(n, a);
        double* Y = p->mixed ? p->RW2 : p->Gw64;
        LAUNCH(p, p->use_oz ? 4 : 2,
               launch_tree_level(X, p->bsig, p->bperm, p->brank, n, a, M, Mp, p->keep, Y,
                                 nn == 1 ? p->S64 : p->G64, p->use_oz ? oz : nullptr, s));
        if (nn == 1) break;
        int32_t* sw = p->sweeps + D + 1 + node_off;
        if (!p->mixed) {
            CU(cudaMemcpyAsync(p->Gw64, p->G64, sizeof(double) * nn * mm, cudaMemcpyDeviceToDevice, s));
            LAUNCH(p, 1, launch_jacobi<double>(p->Gw64, p->Vt64, nn, Mp, p->max_sweeps, p->jac_tol,
                                               sw, s));
            LAUNCH(p, 1, launch_sort_rank(nullptr, nullptr, p->Gw64, nullptr, nn, M, Mp, nullptr, p->N,
                                          p->d.rank_tol, p->bsig, p->bperm, p->brank, s));
            X = p->Vt64;
        } else {
            LAUNCH(p, 1, launch_convert_f64_f32(p->G64, p->G32, nn * mm, s));
            LAUNCH(p, 1, launch_jacobi<float>(p->G32, p->Vt32, nn, Mp, p->max_sweeps, p->jac_tol, sw,
                                              s, p->jwork));
            LAUNCH(p, 1, launch_convert_f32_f64(p->Vt32, p->Vt64, nn * mm, s));
            double* Xc = p->Vt64;
            double* Xn = p->Xn;
            RRWork rr = rr_work(p, 0);
            const bool use_rr = p->rr_kappa > 0;
            for (int it = 0; it < p->refine_iters; ++it) {
                rr.stagger = it & 1;
                LAUNCH(p, refine_launches(false, p->use_oz, 0, use_rr),
                       launch_refine(p->G64, Xc, Xn, p->lam, nn, Mp, p->RW1, p->RW2, p->RW3, p->norms,
                                     s, nullptr, p->use_oz ? oz : nullptr, use_rr ? &rr : nullptr));
                std::swap(Xc, Xn);
            }
            if (p->refine_iters > 0)
                LAUNCH(p, 1, launch_sort_rank(p->lam, nullptr, nullptr, nullptr, nn, M, Mp, nullptr,
                                              p->N, p->d.rank_tol, p->bsig, p->bperm, p->brank, s));
            else
                LAUNCH(p, 1, launch_sort_rank(nullptr, nullptr, nullptr, p->G32, nn, M, Mp, nullptr,
                                              p->N, p->d.rank_tol, p->bsig, p->bperm, p->brank, s));
            X = Xc;
        }
        node_off += nn;
        n = nn;
    }
    return SVD_OK;
}

// Block refinement, sort and rank, proxy P and P P^T (Eqs. 2-3); leaves the
// merge matrix for the merge eigensolve.
svd_status phase_mid(svd_plan_s* p, const RunIO& io, cudaStream_t s) {
    const int D = p->D, M = p->M, Mp = p->Mp;
    const int64_t mm = (int64_t)Mp * Mp;
    mark(p, 3, s);
    const double* Xblk64 = nullptr;
    const float* Xblk32 = nullptr;
    if (!p->mixed) {
        LAUNCH(p, 1, launch_sort_rank(nullptr, nullptr, p->Gw64, nullptr, D, M, Mp, p->bounds_d, 0,
                                      p->d.rank_tol, p->bsig, p->bperm, p->brank, s));
        Xblk64 = p->Vt64;
    } else if (p->refine_iters > 0) {
        LAUNCH(p, 1, launch_convert_f32_f64(p->Vt32, p->Vt64, (int64_t)D * mm, s));
        double* X = p->Vt64;
        double* Xn = p->Xn;
        // G X^T straight from the sparse blocks when that is cheaper than the
        // dense product (no insertions: those are only in the dense G).  The
        // scatter costs 2 nnz Mp FP64 loads and atomics; the dense route D Mp^3
        // multiply-adds, on the tensor cores with the exact-slice products
        // (measured: one scatter update costs about as much as 100 dense
        // multiply-adds there), on the FP64 pipes otherwise (about 8).
        const double dense_per_nnz = p->use_oz ? 100.0 : 8.0;
        const bool sparse = !p->patched && !(p->d.flags & SVD_FLAG_DENSE_REFINE) &&
                            dense_per_nnz * (double)p->nnz < (double)D * Mp * (double)Mp;
        const SparseBlocks sb{io.col_ptr, io.row_idx, io.vals, p->d.value_type, p->nchunks,
                              p->chunk_block, p->chunk_lo, p->chunk_hi};
        OzOperand oz[2];
        oz_ops(p, oz);
        RRWork rr = rr_work(p, 0);
        const bool use_rr = p->rr_kappa > 0;
        for (int it = 0; it < p->refine_iters; ++it) {
            rr.stagger = it & 1;
            LAUNCH(p, refine_launches(sparse, p->use_oz, p->nchunks, use_rr),
                   launch_refine(p->G64, X, Xn, p->lam, D, Mp, p->RW1, p->RW2, p->RW3,
                                       p->norms, s, sparse ? &sb : nullptr,
                                       p->use_oz ? oz : nullptr, use_rr ? &rr : nullptr));
            std::swap(X, Xn);
        }
        LAUNCH(p, 1, launch_sort_rank(p->lam, nullptr, nullptr, nullptr, D, M, Mp, p->bounds_d, 0,
                                      p->d.rank_tol, p->bsig, p->bperm, p->brank, s));
        Xblk64 = X;
    } else {
        LAUNCH(p, 1, launch_sort_rank(nullptr, nullptr, nullptr, p->G32, D, M, Mp, p->bounds_d, 0,
                                      p->d.rank_tol, p->bsig, p->bperm, p->brank, s));
        Xblk32 = p->Vt32;
    }
    mark(p, 4, s);
    OzOperand oz[2];
    oz_ops(p, oz);
    if (!p->arity) {
        LAUNCH(p, 2, launch_proxy(Xblk64, Xblk32, p->bsig, p->bperm, p->brank, D, M, Mp, p->pofs,
                                  p->P, s, p->keep));
        mark(p, 5, s);
        LAUNCH(p, p->use_oz ? 4 : 2, launch_merge_gram(p->P, p->pofs, D, M, Mp, p->Rmax, p->partial, p->nsplit,
                                       p->S64, s, p->use_oz ? oz : nullptr));
    } else {
        mark(p, 5, s);
        if (!Xblk64) {   // FP32 bases (no refinement): the tree works on FP64 rows
            LAUNCH(p, 1, launch_convert_f32_f64(p->Vt32, p->Vt64, (int64_t)D * mm, s));
            Xblk64 = p->Vt64;
        }
        svd_status st = tree_merge(p, Xblk64, oz, s);
        if (st != SVD_OK) return st;
    }
    mark(p, 6, s);
    if (!p->mixed)
        CU(cudaMemcpyAsync(p->Sw64, p->S64, sizeof(double) * mm, cudaMemcpyDeviceToDevice, s));
    else
        LAUNCH(p, 1, launch_convert_f64_f32(p->S64, p->S32, mm, s));
    return SVD_OK;
}

svd_status merge_jacobi(svd_plan_s* p, cudaStream_t s) {
    if (!p->mixed)
        LAUNCH(p, 1, launch_jacobi<double>(p->Sw64, p->SV64, 1, p->Mp, p->max_sweeps, p->jac_tol,
                                           p->sweeps + p->D, s));
    else
        LAUNCH(p, 1, launch_jacobi<float>(p->S32, p->SV32, 1, p->Mp, p->max_sweeps, p->jac_tol,
                                          p->sweeps + p->D, s,
                                          p->jwork + jacobi_work_bytes(p->D, p->Mp)));
    return SVD_OK;
}

// Merge refinement, sigma / U / rank / W, and V = A'^T W.
svd_status phase_post(svd_plan_s* p, const RunIO& io, cudaStream_t s) {
    const int D = p->D, M = p->M, Mp = p->Mp;
    const int64_t mm = (int64_t)Mp * Mp;
    const int vt = p->d.value_type;
    const double* Xm64 = nullptr;
    if (!p->mixed) {
        LAUNCH(p, 1, launch_sort_rank(nullptr, nullptr, p->Sw64, nullptr, 1, M, Mp, nullptr, p->N,
                                      p->d.rank_tol, p->msig, p->mperm, p->mrank, s));
        Xm64 = p->SV64;
    } else {
        LAUNCH(p, 1, launch_convert_f32_f64(p->SV32, p->SV64, mm, s));
        double* X = p->SV64;
        double* Xn = p->SXn;
        OzOperand oz[2];
        oz_ops(p, oz);
        RRWork rr = rr_work(p, D);
        const bool use_rr = p->rr_kappa > 0;
        for (int it = 0; it < p->merge_refine_iters; ++it) {
            rr.stagger = it & 1;
            LAUNCH(p, refine_launches(false, p->use_oz, 0, use_rr),
                   launch_refine(p->S64, X, Xn, p->slam, 1, Mp, p->SR1, p->SR2, p->SR3,
                                       p->snorm, s, nullptr, p->use_oz ? oz : nullptr,
                                       use_rr ? &rr : nullptr));
            std::swap(X, Xn);
        }
        LAUNCH(p, 1, launch_sort_rank(p->slam, nullptr, nullptr, nullptr, 1, M, Mp, nullptr, p->N,
                                      p->d.rank_tol, p->msig, p->mperm, p->mrank, s));
        Xm64 = X;
    }
    mark(p, 7, s);
    const double lam_abs = p->d.rank_tol > 0 ? p->d.rank_tol * p->d.rank_tol : 0.0;
    const int64_t tol_scale = std::max<int64_t>(M, p->N);
    LAUNCH(p, 1, launch_finalize(Xm64, nullptr, p->msig, p->mperm, M, Mp, p->k, lam_abs, tol_scale,
                                 io.sigma, io.U, io.rank, p->W64, p->W32, s));
    mark(p, 8, s);
    if (!(p->d.flags & SVD_FLAG_SKIP_V) && io.V) {
        if (p->mixed) {
            LAUNCH(p, 1, launch_spmm<float>(io.col_ptr, io.row_idx, io.vals, vt, p->N, p->k, p->W32,
                                            static_cast<float*>(io.V), s));
            if (p->patched)
                LAUNCH(p, 1, launch_spmm_patches<float>(p->patches, p->patch_ofs + D, D * M, p->k,
                                                        p->W32, static_cast<float*>(io.V), s));
        } else {
            LAUNCH(p, 1, launch_spmm<double>(io.col_ptr, io.row_idx, io.vals, vt, p->N, p->k,
                                             p->W64, static_cast<double*>(io.V), s));
            if (p->patched)
                LAUNCH(p, 1, launch_spmm_patches<double>(p->patches, p->patch_ofs + D, D * M, p->k,
                                                         p->W64, static_cast<double*>(io.V), s));
        }
    }
    mark(p, 9, s);
    if (p->cur_slot >= 0) p->ev_pending[p->cur_slot] = true;
    ++p->run_index;
    p->last_stream = s;
    p->ran = true;
    return SVD_OK;
}

svd_status run_device(svd_plan_s* p, const int64_t* col_ptr, const int32_t* row_idx,
                      const void* vals, double* d_sigma, double* d_U, void* d_V, int32_t* d_rank,
                      svd_patch* d_patches, int64_t* d_npatches, cudaStream_t s) {
    const RunIO io{col_ptr, row_idx, vals, d_sigma, d_U, d_V, d_rank, d_patches, d_npatches};
    svd_status st = phase_pre(p, io, s);
    if (st == SVD_OK) st = block_jacobi(p, s);
    if (st == SVD_OK) st = phase_mid(p, io, s);
    if (st == SVD_OK) st = merge_jacobi(p, s);
    if (st == SVD_OK) st = phase_post(p, io, s);
    return st;
}

}  // namespace

extern "C" {

int32_t svd_version(void) { return 1; }

namespace {
// workspace of svd_exact_product: the two operands' slices and row bounds
struct ProductLayout {
    size_t a_sl, b_sl, a_mx, b_mx, total;
};
ProductLayout product_layout(int32_t m, int32_t n, int64_t k, int32_t S, bool sym) {
    ProductLayout L{};
    const size_t ea = (size_t)oz_operand_elems(1, S, m, k) * sizeof(uint16_t);
    const size_t eb = sym ? 0 : (size_t)oz_operand_elems(1, S, n, k) * sizeof(uint16_t);
    L.a_sl = 0;
    L.b_sl = align_up(ea);
    L.a_mx = L.b_sl + align_up(eb);
    L.b_mx = L.a_mx + align_up(sizeof(unsigned long long) * round_up(m, OZ_ROW_PAD));
    L.total = L.b_mx + align_up(sizeof(unsigned long long) * round_up(n, OZ_ROW_PAD));
    return L;
}
}  // namespace

size_t svd_exact_product_bytes(int32_t m, int32_t n, int64_t k, int32_t slices) {
    if (m < 1 || n < 1 || k < 1 || (slices != 3 && slices != 5)) return 0;
    return product_layout(m, n, k, slices, false).total;
}

svd_status svd_exact_product(int32_t m, int32_t n, int64_t k, const double* d_A, int64_t lda,
                             const double* d_B, int64_t ldb, double* d_C, int64_t ldc,
                             int32_t slices, int32_t flags, void* d_work, size_t work_bytes,
                             int32_t* d_err, void* stream) {
    const bool sym = (flags & SVD_PRODUCT_SYM) != 0;
    if (m < 1 || n < 1 || k < 1 || m > (1 << 20) || n > (1 << 20)) return SVD_ERR_INVALID_ARG;
    if (slices != 3 && slices != 5) return SVD_ERR_INVALID_ARG;
    if (sym && n != m) return SVD_ERR_INVALID_ARG;
    if (!d_A || (!sym && !d_B) || !d_C || !d_work || lda < k || (!sym && ldb < k) || ldc < n)
        return SVD_ERR_INVALID_ARG;
    const ProductLayout L = product_layout(m, n, k, slices, sym);
    if (work_bytes < L.total) return SVD_ERR_INVALID_ARG;
    char* w = static_cast<char*>(d_work);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int tc = (flags & SVD_PRODUCT_LEGACY_MMA) ? 0 : 1;
    OzOperand a{reinterpret_cast<uint16_t*>(w + L.a_sl), reinterpret_cast<unsigned long long*>(w + L.a_mx),
                0, 0, 0, 0, tc, d_err};
    OzOperand b{reinterpret_cast<uint16_t*>(w + L.b_sl), reinterpret_cast<unsigned long long*>(w + L.b_mx),
                0, 0, 0, 0, tc, d_err};
    CU(launch_oz_split(1, m, k, d_A, lda, 0, 0, nullptr, slices, a, s));
    if (!sym) CU(launch_oz_split(1, n, k, d_B, ldb, 0, 0, nullptr, slices, b, s));
    CU(launch_oz_gemm(1, m, n, a, sym ? a : b, 1.0, 0.0, d_C, ldc, 0, sym ? 1 : 0, s));
    return SVD_OK;
}

const char* svd_status_str(svd_status s) {
    switch (s) {
        case SVD_OK: return "ok";
        case SVD_ERR_INVALID_ARG: return "invalid argument";
        case SVD_ERR_INVALID_CSC: return "invalid CSC structure";
        case SVD_ERR_OOM: return "out of memory";
        case SVD_ERR_BUDGET: return "over the memory budget";
        case SVD_ERR_CUDA: return "CUDA error";
        case SVD_ERR_NOT_CONVERGED: return "Jacobi did not converge within max_sweeps";
        case SVD_ERR_TIMEOUT: return "timeout";
        case SVD_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

svd_status svd_plan_bytes(const svd_desc* desc, size_t* bytes) {
    svd_status st = validate_desc(desc);
    if (st != SVD_OK) return st;
    svd_plan_s tmp;
    const svd_desc sf = short_fat(*desc);
    st = fill_plan(&sf, &tmp);
    if (st != SVD_OK) return st;
    Carver c{nullptr, 0, true};
    carve(&tmp, c);
    if (bytes) *bytes = c.off;
    return SVD_OK;
}

namespace {
// Create a plan on `arena` (nullptr: allocate one).
svd_status plan_create(const svd_desc* desc, void* arena, size_t arena_bytes, svd_plan_t* out,
                       size_t* bytes) {
    if (!out) return SVD_ERR_INVALID_ARG;
    *out = nullptr;
    svd_status st = validate_desc(desc);
    if (st != SVD_OK) return st;
    svd_plan_s* p = new (std::nothrow) svd_plan_s();
    if (!p) return SVD_ERR_OOM;
    const svd_desc sf = short_fat(*desc);
    st = fill_plan(&sf, p);
    if (st != SVD_OK) { delete p; return st; }
    Carver dry{nullptr, 0, true};
    carve(p, dry);
    p->arena_bytes = dry.off;
    if (arena) {
        if (arena_bytes < p->arena_bytes || (reinterpret_cast<uintptr_t>(arena) & 255u)) {
            delete p;
            return SVD_ERR_INVALID_ARG;
        }
        p->arena = static_cast<char*>(arena);
        p->owns_arena = false;
    } else if (cudaMalloc(&p->arena, p->arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return SVD_ERR_OOM;
    }
    Carver c{p->arena, 0, false};
    carve(p, c);
    // block boundaries and column chunks
    std::vector<int32_t> cb;
    std::vector<int64_t> clo, chi;
    cb.reserve(p->nchunks);
    for (int i = 0; i < p->D; ++i) {
        for (int64_t a = p->bounds_h[i]; a < p->bounds_h[i + 1]; a += kChunkCols) {
            cb.push_back(i);
            clo.push_back(a);
            chi.push_back(std::min(a + kChunkCols, p->bounds_h[i + 1]));
        }
    }
    bool ok = cudaMemcpy(p->bounds_d, p->bounds_h.data(), sizeof(int64_t) * (p->D + 1),
                         cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(p->chunk_block, cb.data(), sizeof(int32_t) * cb.size(),
                          cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(p->chunk_lo, clo.data(), sizeof(int64_t) * clo.size(),
                          cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(p->chunk_hi, chi.data(), sizeof(int64_t) * chi.size(),
                          cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemset(p->sweeps, 0, sizeof(int32_t) * (p->D + 1 + (p->arity ? p->D : 0))) ==
                   cudaSuccess;
    ok = ok && cudaMemset(p->dev_err, 0, sizeof(int32_t) * 4) == cudaSuccess;
    if (!ok) {
        if (p->owns_arena) cudaFree(p->arena);
        delete p;
        return SVD_ERR_CUDA;
    }
    if (desc->flags & SVD_FLAG_TIMING) {
        p->timing = true;
        for (int r = 0; r < kRing; ++r)
            for (int i = 0; i <= kStages; ++i) cudaEventCreate(&p->ev[r][i]);
    }
    if (bytes) *bytes = p->arena_bytes;
    *out = p;
    return SVD_OK;
}
}  // namespace

svd_status svd_plan(const svd_desc* desc, svd_plan_t* out, size_t* bytes) {
    return plan_create(desc, nullptr, 0, out, bytes);
}

svd_status svd_plan_ws(const svd_desc* desc, void* d_workspace, size_t workspace_bytes,
                       svd_plan_t* out) {
    if (!d_workspace) return SVD_ERR_INVALID_ARG;
    return plan_create(desc, d_workspace, workspace_bytes, out, nullptr);
}

svd_status svd_run(svd_plan_t p, const int64_t* d_col_ptr, const int32_t* d_row_idx,
                   const void* d_vals, double* d_sigma, double* d_U, void* d_V, int32_t* d_rank,
                   svd_patch* d_patches, int64_t* d_npatches, void* stream) {
    if (!p || !d_col_ptr || (!d_row_idx && p->nnz > 0) || (!d_vals && p->nnz > 0) || !d_sigma ||
        !d_rank)
        return SVD_ERR_INVALID_ARG;
    // short-side (FP64, column-major) and long-side outputs; a tall plan's
    // caller holds them as V and U
    double* small = p->tall ? static_cast<double*>(d_V) : d_U;
    void* big = p->tall ? static_cast<void*>(d_U) : d_V;
    if (!small) return SVD_ERR_INVALID_ARG;
    if (!big && !(p->d.flags & SVD_FLAG_SKIP_V)) return SVD_ERR_INVALID_ARG;
    if ((d_patches == nullptr) != (d_npatches == nullptr)) return SVD_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p->d.flags & SVD_FLAG_CHECK_CSC) {
        // the caller's CSC: p->M x p->N, or N' = p->M columns of p->N rows when tall
        const svd_status st =
            p->tall ? svd_check_csc((int32_t)p->N, p->M, p->nnz, d_col_ptr, d_row_idx, stream)
                    : svd_check_csc(p->M, p->N, p->nnz, d_col_ptr, d_row_idx, stream);
        if (st != SVD_OK) return st;
    }
    if (p->tall) {
        p->src_col_ptr = d_col_ptr;
        p->src_row_idx = d_row_idx;
        p->src_vals = d_vals;
        return run_device(p, p->t_ptr, p->t_idx, p->t_val, d_sigma, small, big, d_rank,
                          d_patches, d_npatches, s);
    }
    return run_device(p, d_col_ptr, d_row_idx, d_vals, d_sigma, small, big, d_rank, d_patches,
                      d_npatches, s);
}

svd_status svd_run_host(svd_plan_t p, const int64_t* h_col_ptr, const int32_t* h_row_idx,
                        const void* h_vals, double* h_sigma, double* h_U, void* h_V,
                        int32_t* h_rank, svd_patch* h_patches, int64_t* h_npatches,
                        void* stream) {
    if (!p || !h_col_ptr || (!h_row_idx && p->nnz > 0) || (!h_vals && p->nnz > 0) || !h_sigma ||
        !h_rank)
        return SVD_ERR_INVALID_ARG;
    // short-side (FP64) and long-side outputs; a tall plan's caller holds them as V and U
    double* h_small = p->tall ? static_cast<double*>(h_V) : h_U;
    void* h_big = p->tall ? static_cast<void*>(h_U) : h_V;
    if (!h_small) return SVD_ERR_INVALID_ARG;
    const int64_t ncp = (p->tall ? p->M : p->N) + 1;  // column pointers of the caller's CSC
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t sv = p->d.value_type == SVD_VALUE_F32 ? 4 : 8;
    const size_t sV = p->mixed ? 4 : 8;
    const bool want_v = h_big && !(p->d.flags & SVD_FLAG_SKIP_V);
    // A page-locked V buffer is addressable from the device (unified
    // addressing; on this part over the chip-to-chip link): the SpMM then
    // streams V straight into it and the 2 GB copy disappears.  Not with
    // rank-fix insertions, whose V correction uses atomic adds.
    void* dV_direct = nullptr;
    if (want_v && !p->patched) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, h_big) == cudaSuccess && at.type == cudaMemoryTypeHost &&
            at.devicePointer)
            dV_direct = at.devicePointer;
        cudaGetLastError();
    }
    const bool copy_v = want_v && !dV_direct;
    Carver dry{nullptr, 0, true};
    dry.take<int64_t>(ncp);
    dry.take<int32_t>(std::max<int64_t>(p->nnz, 1));
    dry.take<char>(std::max<int64_t>(p->nnz, 1) * sv);
    dry.take<double>(p->k);
    dry.take<double>((size_t)p->M * p->k);
    dry.take<char>(copy_v ? (size_t)p->N * p->k * sV : 1);
    dry.take<int32_t>(1);
    dry.take<svd_patch>((size_t)p->D * p->M);
    dry.take<int64_t>(1);
    if (dry.off > p->host_arena_bytes) {
        if (p->host_arena) cudaFree(p->host_arena);
        p->host_arena = nullptr;
        p->host_arena_bytes = 0;
        if (cudaMalloc(&p->host_arena, dry.off) != cudaSuccess) {
            cudaGetLastError();
            return SVD_ERR_OOM;
        }
        p->host_arena_bytes = dry.off;
    }
    Carver c{p->host_arena, 0, false};
    int64_t* cp = c.take<int64_t>(ncp);
    int32_t* ri = c.take<int32_t>(std::max<int64_t>(p->nnz, 1));
    char* va = c.take<char>(std::max<int64_t>(p->nnz, 1) * sv);
    double* sg = c.take<double>(p->k);
    double* U = c.take<double>((size_t)p->M * p->k);
    char* V = copy_v ? c.take<char>((size_t)p->N * p->k * sV) : static_cast<char*>(dV_direct);
    if (copy_v == false) c.take<char>(1);
    int32_t* rk_ = c.take<int32_t>(1);
    svd_patch* pt = c.take<svd_patch>((size_t)p->D * p->M);
    int64_t* np = c.take<int64_t>(1);
    CU(cudaMemcpyAsync(cp, h_col_ptr, sizeof(int64_t) * ncp, cudaMemcpyHostToDevice, s));
    if (p->nnz > 0) {
        CU(cudaMemcpyAsync(ri, h_row_idx, sizeof(int32_t) * p->nnz, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(va, h_vals, sv * p->nnz, cudaMemcpyHostToDevice, s));
    }
    const int saved = p->d.flags;
    if (!want_v) p->d.flags |= SVD_FLAG_SKIP_V;
    void* Vb = want_v ? static_cast<void*>(V) : nullptr;
    svd_status st = p->tall ? svd_run(p, cp, ri, va, sg, static_cast<double*>(Vb), U, rk_, pt,
                                      np, stream)
                            : svd_run(p, cp, ri, va, sg, U, Vb, rk_, pt, np, stream);
    p->d.flags = saved;
    if (st != SVD_OK) return st;
    CU(cudaMemcpyAsync(h_sigma, sg, sizeof(double) * p->k, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(h_small, U, sizeof(double) * p->M * p->k, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(h_rank, rk_, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (copy_v) CU(cudaMemcpyAsync(h_big, V, (size_t)p->N * p->k * sV, cudaMemcpyDeviceToHost, s));
    if (h_npatches) CU(cudaMemcpyAsync(h_npatches, np, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (h_patches)
        CU(cudaMemcpyAsync(h_patches, pt, sizeof(svd_patch) * (size_t)p->D * p->M,
                           cudaMemcpyDeviceToHost, s));
    return svd_sync(p);
}

svd_status svd_sync(svd_plan_t p) {
    if (!p) return SVD_ERR_INVALID_ARG;
    if (!p->ran) return SVD_OK;
    if (p->last_stream) CU(cudaStreamSynchronize(p->last_stream));
    const int nsw = p->D + 1 + (p->arity ? p->D : 0);
    std::vector<int32_t> sw(nsw);
    CU(cudaMemcpy(sw.data(), p->sweeps, sizeof(int32_t) * nsw, cudaMemcpyDeviceToHost));
    int32_t err = 0;
    CU(cudaMemcpy(&err, p->dev_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (err) return SVD_ERR_TIMEOUT;
    for (int32_t v : sw)
        if (v < 0) return SVD_ERR_NOT_CONVERGED;
    return SVD_OK;
}

svd_status svd_check_csc(int32_t M, int64_t N, int64_t nnz, const int64_t* d_col_ptr,
                         const int32_t* d_row_idx, void* stream) {
    if (M < 1 || N < 1 || nnz < 0 || !d_col_ptr || (nnz > 0 && !d_row_idx))
        return SVD_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t* flag = nullptr;
    CU(cudaMallocAsync(&flag, sizeof(int32_t), s));
    CU(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
    CU(launch_check_csc(M, N, nnz, d_col_ptr, d_row_idx, flag, s));
    int32_t h = 0;
    CU(cudaMemcpyAsync(&h, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(cudaFreeAsync(flag, s));
    CU(cudaStreamSynchronize(s));
    return h ? SVD_ERR_INVALID_CSC : SVD_OK;
}

svd_status svd_query(svd_plan_t p, int32_t what, int64_t index, void* h_dst, size_t bytes) {
    if (!p || !h_dst) return SVD_ERR_INVALID_ARG;
    const int D = p->D, M = p->M, Mp = p->Mp;
    if (p->last_stream) CU(cudaStreamSynchronize(p->last_stream));
    switch (what) {
        case SVD_Q_BLOCK_BOUNDS:
            if (bytes != sizeof(int64_t) * (D + 1)) return SVD_ERR_INVALID_ARG;
            memcpy(h_dst, p->bounds_h.data(), bytes);
            return SVD_OK;
        case SVD_Q_LONELY:
        case SVD_Q_ROW_NONEMPTY: {
            const bool lon = what == SVD_Q_LONELY;
            const size_t rows = lon ? (size_t)D : 1;
            if (bytes != rows * M) return SVD_ERR_INVALID_ARG;
            std::vector<uint32_t> w(rows * p->W);
            CU(cudaMemcpy(w.data(), lon ? p->lonely : p->row_ne, sizeof(uint32_t) * w.size(),
                          cudaMemcpyDeviceToHost));
            uint8_t* o = static_cast<uint8_t*>(h_dst);
            for (size_t d = 0; d < rows; ++d)
                for (int m = 0; m < M; ++m)
                    o[d * M + m] = (w[d * p->W + m / 32] >> (m % 32)) & 1u;
            return SVD_OK;
        }
        case SVD_Q_BLOCK_RANKS:
            if (bytes != sizeof(int32_t) * D) return SVD_ERR_INVALID_ARG;
            CU(cudaMemcpy(h_dst, p->brank, bytes, cudaMemcpyDeviceToHost));
            return SVD_OK;
        case SVD_Q_BLOCK_SIGMA:
            if (bytes != sizeof(double) * D * M) return SVD_ERR_INVALID_ARG;
            CU(cudaMemcpy(h_dst, p->bsig, bytes, cudaMemcpyDeviceToHost));
            return SVD_OK;
        case SVD_Q_BLOCK_GRAM:
        case SVD_Q_MERGE_GRAM: {
            const bool blk = what == SVD_Q_BLOCK_GRAM;
            if (blk && (index < 0 || index >= D)) return SVD_ERR_INVALID_ARG;
            if (bytes != sizeof(double) * M * M) return SVD_ERR_INVALID_ARG;
            const double* src = blk ? p->G64 + index * (int64_t)Mp * Mp : p->S64;
            CU(cudaMemcpy2D(h_dst, sizeof(double) * M, src, sizeof(double) * Mp, sizeof(double) * M,
                            M, cudaMemcpyDeviceToHost));
            return SVD_OK;
        }
        case SVD_Q_PROXY_COLS:
            if (bytes != sizeof(int64_t)) return SVD_ERR_INVALID_ARG;
            if (p->arity) {   // the tree merge forms no proxy
                memset(h_dst, 0, bytes);
                return SVD_OK;
            }
            CU(cudaMemcpy(h_dst, p->pofs + D, bytes, cudaMemcpyDeviceToHost));
            return SVD_OK;
        case SVD_Q_PROXY: {
            if (p->arity) return SVD_ERR_UNSUPPORTED;
            int64_t R = 0;
            CU(cudaMemcpy(&R, p->pofs + D, sizeof(int64_t), cudaMemcpyDeviceToHost));
            if (bytes != sizeof(double) * M * R) return SVD_ERR_INVALID_ARG;
            CU(cudaMemcpy(h_dst, p->P, bytes, cudaMemcpyDeviceToHost));
            return SVD_OK;
        }
        case SVD_Q_SWEEPS:
            if (bytes != sizeof(int32_t) * (D + 1)) return SVD_ERR_INVALID_ARG;
            CU(cudaMemcpy(h_dst, p->sweeps, bytes, cudaMemcpyDeviceToHost));
            return SVD_OK;
        case SVD_Q_LAUNCHES:
            if (bytes != sizeof(int64_t)) return SVD_ERR_INVALID_ARG;
            memcpy(h_dst, &p->launches, bytes);
            return SVD_OK;
        case SVD_Q_STAGE_MS: {
            if (bytes != sizeof(float) * kStages) return SVD_ERR_INVALID_ARG;
            if (!p->timing || !p->ran) return SVD_ERR_INVALID_ARG;
            const int last = (int)((p->run_index - 1) % kRing);
            float* o = static_cast<float*>(h_dst);
            for (int i = 0; i < kStages; ++i)
                CU(cudaEventElapsedTime(o + i, p->ev[last][i], p->ev[last][i + 1]));
            return SVD_OK;
        }
        case SVD_Q_STAGE_TOTAL: {
            if (bytes != sizeof(double) * (kStages + 1)) return SVD_ERR_INVALID_ARG;
            if (!p->timing) return SVD_ERR_INVALID_ARG;
            for (int r = 0; r < kRing; ++r) {
                if (!p->ev_pending[r]) continue;
                for (int i = 0; i < kStages; ++i) {
                    float ms = 0.f;
                    CU(cudaEventElapsedTime(&ms, p->ev[r][i], p->ev[r][i + 1]));
                    p->stage_total[i] += ms;
                }
                ++p->stage_runs;
                p->ev_pending[r] = false;
            }
            double* o = static_cast<double*>(h_dst);
            for (int i = 0; i < kStages; ++i) o[i] = p->stage_total[i];
            o[kStages] = (double)p->stage_runs;
            for (int i = 0; i < kStages; ++i) p->stage_total[i] = 0.0;
            p->stage_runs = 0;
            return SVD_OK;
        }
    }
    return SVD_ERR_INVALID_ARG;
}

void svd_free(svd_plan_t p) {
    if (!p) return;
    if (p->last_stream) cudaStreamSynchronize(p->last_stream);
    if (p->arena && p->owns_arena) cudaFree(p->arena);
    if (p->host_arena) cudaFree(p->host_arena);
    if (p->timing)
        for (int r = 0; r < kRing; ++r)
            for (int i = 0; i <= kStages; ++i) cudaEventDestroy(p->ev[r][i]);
    delete p;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many plans in one pass.  The per-matrix stages of the plans run
// on a pool of worker streams; all block eigensolves of all plans go to one
// persistent Jacobi launch fed from a work list (matrices of any order up to
// the worker's capacity), and the merge eigensolves to another.  Optionally
// the whole pass is captured into a CUDA graph on the first run and replayed.

struct svd_batch_s {
    std::vector<svd_plan_s*> plans;
    std::vector<cudaStream_t> streams;
    cudaEvent_t fork_ev = nullptr;
    std::vector<cudaEvent_t> join_ev;
    // work lists: [blocks f32 | blocks f64 | merges f32 | merges f64]
    JacobiItem* d_items = nullptr;
    int* d_next = nullptr;
    int count[4] = {};
    int offset[4] = {};
    int maxmp[4] = {};
    double tol[4] = {};
    int sweeps_cap = 40;
    std::vector<int> outsized;   // plans whose Mp exceeds the worker capacity
    bool use_graph = false;
    bool captured = false;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;   // graphs are captured and replayed here
    cudaEvent_t in_ev = nullptr, out_ev = nullptr;
    std::vector<RunIO> ios_seen;
    int64_t launches = 0;
    size_t item_capacity = 0;            // JacobiItems the device list holds
    JacobiItem* h_stage = nullptr;       // page-locked staging for asynchronous list uploads
};

namespace {

void fork(svd_batch_s* b, cudaStream_t s) {
    cudaEventRecord(b->fork_ev, s);
    for (cudaStream_t w : b->streams) cudaStreamWaitEvent(w, b->fork_ev, 0);
}

void join(svd_batch_s* b, cudaStream_t s) {
    for (size_t i = 0; i < b->streams.size(); ++i) {
        cudaEventRecord(b->join_ev[i], b->streams[i]);
        cudaStreamWaitEvent(s, b->join_ev[i], 0);
    }
}

svd_status batch_items(svd_batch_s* b, int first, cudaStream_t s) {
    // first = 0: block work lists, 2: merge work lists
    for (int w = first; w < first + 2; ++w) {
        if (!b->count[w]) continue;
        cudaError_t e = (w % 2 == 0)
            ? launch_jacobi_items<float>(b->d_items + b->offset[w], b->count[w], b->maxmp[w],
                                         b->d_next + w, b->sweeps_cap, b->tol[w], s)
            : launch_jacobi_items<double>(b->d_items + b->offset[w], b->count[w], b->maxmp[w],
                                          b->d_next + w, b->sweeps_cap, b->tol[w], s);
        if (e != cudaSuccess) {
            fprintf(stderr, "ranky: batched Jacobi: %s\n", cudaGetErrorString(e));
            return SVD_ERR_CUDA;
        }
        ++b->launches;
    }
    return SVD_OK;
}

svd_status batch_enqueue(svd_batch_s* b, const RunIO* ios, cudaStream_t s) {
    const size_t n = b->plans.size(), ns = b->streams.size();
    b->launches = 0;
    svd_status st = SVD_OK;
    fork(b, s);
    for (size_t i = 0; i < n && st == SVD_OK; ++i)
        st = phase_pre(b->plans[i], ios[i], b->streams[i % ns]);
    join(b, s);
    if (st != SVD_OK) return st;
    if ((st = batch_items(b, 0, s)) != SVD_OK) return st;
    for (int i : b->outsized)
        if ((st = block_jacobi(b->plans[i], s)) != SVD_OK) return st;
    fork(b, s);
    for (size_t i = 0; i < n && st == SVD_OK; ++i)
        st = phase_mid(b->plans[i], ios[i], b->streams[i % ns]);
    join(b, s);
    if (st != SVD_OK) return st;
    if ((st = batch_items(b, 2, s)) != SVD_OK) return st;
    for (int i : b->outsized)
        if ((st = merge_jacobi(b->plans[i], s)) != SVD_OK) return st;
    fork(b, s);
    for (size_t i = 0; i < n && st == SVD_OK; ++i)
        st = phase_post(b->plans[i], ios[i], b->streams[i % ns]);
    join(b, s);
    for (size_t i = 0; i < n; ++i) b->launches += b->plans[i]->launches;
    return st;
}

}  // namespace

svd_status batch_engine_create(int nstreams, size_t item_capacity, svd_batch_t* out) {
    if (!out || nstreams < 1) return SVD_ERR_INVALID_ARG;
    *out = nullptr;
    svd_batch_s* b = new (std::nothrow) svd_batch_s();
    if (!b) return SVD_ERR_OOM;
    item_capacity = std::max<size_t>(item_capacity, 1);
    bool ok = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->in_ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->out_ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    b->streams.resize(nstreams);
    b->join_ev.resize(nstreams);
    for (int i = 0; i < nstreams && ok; ++i) {
        ok = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->join_ev[i], cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaMalloc(&b->d_items, sizeof(JacobiItem) * item_capacity) == cudaSuccess &&
         cudaMalloc(&b->d_next, sizeof(int) * 4) == cudaSuccess &&
         cudaHostAlloc(&b->h_stage, sizeof(JacobiItem) * item_capacity, cudaHostAllocDefault) == cudaSuccess;
    b->item_capacity = item_capacity;
    if (!ok) {
        cudaGetLastError();
        svd_batch_free(b);
        return SVD_ERR_OOM;
    }
    *out = b;
    return SVD_OK;
}

svd_status batch_engine_assign(svd_batch_t b, int n, const svd_plan_t* plans, cudaStream_t stream) {
    if (!b || n < 1 || !plans) return SVD_ERR_INVALID_ARG;
    // (the previous plans were detached, or belong to a batch being built:
    // they are not touched here, they may be gone)
    b->plans.assign(plans, plans + n);
    b->outsized.clear();
    for (int w = 0; w < 4; ++w) { b->maxmp[w] = 0; b->tol[w] = 0.0; }
    b->sweeps_cap = 40;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    b->captured = false;
    // work lists: [blocks f32 | blocks f64 | merges f32 | merges f64]
    std::vector<JacobiItem> lists[4];
    const int cap32 = jacobi_item_max_mp(false), cap64 = jacobi_item_max_mp(true);
    for (int i = 0; i < n; ++i)
        if (plans[i] && plans[i]->arity) return SVD_ERR_UNSUPPORTED;   // tree merges run alone
    for (int i = 0; i < n; ++i) {
        svd_plan_s* p = plans[i];
        const bool f64 = !p->mixed;
        if (p->Mp > (f64 ? cap64 : cap32)) {
            b->outsized.push_back(i);
            continue;
        }
        const int64_t mm = (int64_t)p->Mp * p->Mp;
        const int wb = f64 ? 1 : 0;
        for (int d = 0; d < p->D; ++d) {
            JacobiItem it{};
            it.G = f64 ? (void*)(p->Gw64 + d * mm) : (void*)(p->G32 + d * mm);
            it.Vt = f64 ? (void*)(p->Vt64 + d * mm) : (void*)(p->Vt32 + d * mm);
            it.sweeps = p->sweeps + d;
            it.work = f64 ? nullptr : (void*)(p->jwork + jacobi_work_bytes(d, p->Mp));
            it.Mp = p->Mp;
            it.max_sweeps = p->max_sweeps;
            lists[wb].push_back(it);
        }
        JacobiItem m{};
        m.G = f64 ? (void*)p->Sw64 : (void*)p->S32;
        m.Vt = f64 ? (void*)p->SV64 : (void*)p->SV32;
        m.sweeps = p->sweeps + p->D;
        m.work = f64 ? nullptr : (void*)(p->jwork + jacobi_work_bytes(p->D, p->Mp));
        m.Mp = p->Mp;
        m.max_sweeps = p->max_sweeps;
        lists[2 + wb].push_back(m);
        for (int w : {wb, 2 + wb}) {
            b->maxmp[w] = std::max(b->maxmp[w], p->Mp);
            b->tol[w] = p->jac_tol;
        }
        b->sweeps_cap = std::max(b->sweeps_cap, p->max_sweeps);
    }
    size_t total = 0;
    for (int w = 0; w < 4; ++w) {
        b->offset[w] = (int)total;
        b->count[w] = (int)lists[w].size();
        total += lists[w].size();
    }
    if (total > b->item_capacity) return SVD_ERR_INVALID_ARG;
    if (!total) return SVD_OK;
    for (int w = 0; w < 4; ++w)
        std::copy(lists[w].begin(), lists[w].end(), b->h_stage + b->offset[w]);
    // asynchronous on the caller's stream (from page-locked staging, which is
    // not touched again before the pass that reads the lists has run), or
    // synchronous when no stream is given
    const cudaError_t e = stream ? cudaMemcpyAsync(b->d_items, b->h_stage, sizeof(JacobiItem) * total,
                                                   cudaMemcpyHostToDevice, stream)
                                 : cudaMemcpy(b->d_items, b->h_stage, sizeof(JacobiItem) * total,
                                              cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaGetLastError(); return SVD_ERR_CUDA; }
    return SVD_OK;
}

void batch_engine_detach(svd_batch_t b) {
    if (!b) return;
    for (svd_plan_s* p : b->plans)   // plans that leave the batch keep no stream of it
        for (cudaStream_t w : b->streams)
            if (p->last_stream == w || p->last_stream == b->cap_stream) p->last_stream = nullptr;
    b->plans.clear();
}

namespace {

bool same_ios(const std::vector<RunIO>& a, const RunIO* b, size_t n) {
    if (a.size() != n) return false;
    return memcmp(a.data(), b, sizeof(RunIO) * n) == 0;
}

}  // namespace

extern "C" {

svd_status svd_batch_create(int32_t n, const svd_plan_t* plans, int32_t flags, svd_batch_t* out) {
    if (!out || n < 1 || !plans) return SVD_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!plans[i]) return SVD_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (plans[i]->tall || plans[i]->arity) return SVD_ERR_UNSUPPORTED;
    size_t items = 0;
    for (int i = 0; i < n; ++i) items += (size_t)plans[i]->D + 1;
    svd_batch_t b = nullptr;
    svd_status st = batch_engine_create(std::min(n, 8), items, &b);
    if (st != SVD_OK) return st;
    b->use_graph = (flags & SVD_BATCH_GRAPH) != 0;
    st = batch_engine_assign(b, n, plans, nullptr);
    if (st != SVD_OK) {
        svd_batch_free(b);
        return st;
    }
    *out = b;
    return SVD_OK;
}

svd_status svd_batch_run(svd_batch_t b, const svd_io* ios, void* stream) {
    if (!b || !ios) return SVD_ERR_INVALID_ARG;
    const size_t n = b->plans.size();
    std::vector<RunIO> rio(n);
    for (size_t i = 0; i < n; ++i) {
        const svd_io& o = ios[i];
        svd_plan_s* p = b->plans[i];
        if (!o.d_col_ptr || (p->nnz > 0 && (!o.d_row_idx || !o.d_vals)) || !o.d_sigma || !o.d_U ||
            !o.d_rank || (!o.d_V && !(p->d.flags & SVD_FLAG_SKIP_V)) ||
            ((o.d_patches == nullptr) != (o.d_npatches == nullptr)))
            return SVD_ERR_INVALID_ARG;
        rio[i] = RunIO{o.d_col_ptr, o.d_row_idx, o.d_vals, o.d_sigma, o.d_U, o.d_V, o.d_rank,
                       o.d_patches, o.d_npatches};
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!b->use_graph) return batch_enqueue(b, rio.data(), s);
    // The graph is captured on, and replayed on, the batch's own stream, which
    // is ordered after the caller's stream (event in) and before it (event out):
    // the caller's stream may be the legacy default stream, which cannot be
    // captured.
    cudaStream_t cs = b->cap_stream;
    CU(cudaEventRecord(b->in_ev, s));
    CU(cudaStreamWaitEvent(cs, b->in_ev, 0));
    if (!(b->captured && same_ios(b->ios_seen, rio.data(), n))) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
            b->captured = false;
        }
        CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        svd_status st = batch_enqueue(b, rio.data(), cs);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(cs, &g);
        if (st != SVD_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (ce != cudaSuccess) fprintf(stderr, "ranky: batch capture: %s\n", cudaGetErrorString(ce));
            return st != SVD_OK ? st : SVD_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            fprintf(stderr, "ranky: batch graph: %s\n", cudaGetErrorString(ie));
            cudaGetLastError();
            b->exec = nullptr;
            return SVD_ERR_CUDA;
        }
        b->captured = true;
        b->ios_seen = rio;
    }
    CU(cudaGraphLaunch(b->exec, cs));
    CU(cudaEventRecord(b->out_ev, cs));
    CU(cudaStreamWaitEvent(s, b->out_ev, 0));
    for (svd_plan_s* p : b->plans) { p->last_stream = cs; p->ran = true; }
    return SVD_OK;
}

svd_status svd_batch_sync(svd_batch_t b) {
    if (!b) return SVD_ERR_INVALID_ARG;
    for (cudaStream_t w : b->streams) CU(cudaStreamSynchronize(w));
    if (b->cap_stream) CU(cudaStreamSynchronize(b->cap_stream));
    svd_status worst = SVD_OK;
    for (svd_plan_s* p : b->plans) {
        const svd_status st = svd_sync(p);
        if (st != SVD_OK) worst = st;
    }
    return worst;
}

int64_t svd_batch_launches(svd_batch_t b) { return b ? b->launches : 0; }

void svd_batch_free(svd_batch_t b) {
    if (!b) return;
    for (cudaStream_t w : b->streams)
        if (w) cudaStreamSynchronize(w);
    if (b->cap_stream) cudaStreamSynchronize(b->cap_stream);
    // the plans outlive the batch: they must not keep its streams
    for (svd_plan_s* p : b->plans)
        for (cudaStream_t w : b->streams)
            if (p->last_stream == w || p->last_stream == b->cap_stream) p->last_stream = nullptr;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (cudaStream_t w : b->streams)
        if (w) cudaStreamDestroy(w);
    for (cudaEvent_t e : b->join_ev)
        if (e) cudaEventDestroy(e);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->cap_stream) {
        cudaStreamSynchronize(b->cap_stream);
        cudaStreamDestroy(b->cap_stream);
    }
    if (b->in_ev) cudaEventDestroy(b->in_ev);
    if (b->out_ev) cudaEventDestroy(b->out_ev);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_next) cudaFree(b->d_next);
    if (b->h_stage) cudaFreeHost(b->h_stage);
    delete b;
}

}  // extern "C"
