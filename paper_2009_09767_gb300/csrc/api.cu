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
    double jac_tol = 0.0;
    int max_sweeps = 40, refine_iters = 1, merge_refine_iters = 2;
    std::vector<int64_t> bounds_h;
    int nchunks = 0;
    int W = 0;  // bitmap words per block
    int nsplit = 1;
    int64_t Rmax = 0;

    char* arena = nullptr;
    size_t arena_bytes = 0;

    int64_t* bounds_d = nullptr;
    int32_t* chunk_block = nullptr;
    int64_t* chunk_lo = nullptr;
    int64_t* chunk_hi = nullptr;
    uint32_t* occ = nullptr;
    uint32_t* row_ne = nullptr;
    uint32_t* lonely = nullptr;
    PatchRec* patches = nullptr;
    int64_t* patch_ofs = nullptr;
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
    double* slam = nullptr;
    double* snorm = nullptr;
    double* msig = nullptr;
    int32_t* mperm = nullptr;
    int32_t* mrank = nullptr;
    double* W64 = nullptr;
    float* W32 = nullptr;
    int32_t* sweeps = nullptr;
    int32_t* scratch_flag = nullptr;

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
};

namespace {

constexpr int64_t kChunkCols = 16384;

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

svd_status validate_desc(const svd_desc* d) {
    if (!d) return SVD_ERR_INVALID_ARG;
    if (d->M < 1 || d->N < 1 || d->nnz < 0) return SVD_ERR_INVALID_ARG;
    if (d->value_type != SVD_VALUE_F32 && d->value_type != SVD_VALUE_F64) return SVD_ERR_INVALID_ARG;
    if (d->num_blocks < 1 || (int64_t)d->num_blocks > d->N) return SVD_ERR_INVALID_ARG;
    if (d->precision != SVD_PREC_FP64 && d->precision != SVD_PREC_MIXED) return SVD_ERR_INVALID_ARG;
    if (d->rank_fix < SVD_RANKFIX_TRUNCATE || d->rank_fix > SVD_RANKFIX_NEIGHBOR_RANDOM)
        return SVD_ERR_INVALID_ARG;
    if (d->rank_fix == SVD_RANKFIX_NEIGHBOR || d->rank_fix == SVD_RANKFIX_NEIGHBOR_RANDOM)
        return SVD_ERR_UNSUPPORTED;
    if (d->k < 0) return SVD_ERR_INVALID_ARG;
    const int64_t kmax = std::min<int64_t>(d->M, d->N);
    if (d->k > kmax) return SVD_ERR_INVALID_ARG;
    if (d->M > kMaxM) return SVD_ERR_UNSUPPORTED;
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
    p->G64 = c.take<double>((size_t)D * mm);
    p->Vt64 = c.take<double>((size_t)D * mm);
    if (p->mixed) {
        p->G32 = c.take<float>((size_t)D * mm);
        p->Vt32 = c.take<float>((size_t)D * mm);
        if (p->refine_iters > 0) {
            p->Xn = c.take<double>((size_t)D * mm);
            p->RW1 = c.take<double>((size_t)D * mm);
            p->RW2 = c.take<double>((size_t)D * mm);
            p->RW3 = c.take<double>((size_t)D * mm);
            p->lam = c.take<double>((size_t)D * Mp);
            p->norms = c.take<double>(D);
        }
    } else {
        p->Gw64 = c.take<double>((size_t)D * mm);
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
    p->msig = c.take<double>(M);
    p->mperm = c.take<int32_t>(M);
    p->mrank = c.take<int32_t>(1);
    p->sweeps = c.take<int32_t>(D + 1);
    p->scratch_flag = c.take<int32_t>(4);
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
    p->Mp = jacobi_pad(d->M);
    p->W = (d->M + 31) / 32;
    p->max_sweeps = d->max_sweeps > 0 ? d->max_sweeps : 40;
    p->jac_tol = d->jacobi_tol > 0 ? d->jacobi_tol : (p->mixed ? 8.0 * Eps<float>::value : 1e-14);
    p->refine_iters = d->refine_iters >= 0 ? d->refine_iters : 1;
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
    int64_t rmax = 0;
    for (int i = 0; i < p->D; ++i)
        rmax += std::min<int64_t>(p->M, p->bounds_h[i + 1] - p->bounds_h[i]);
    p->Rmax = std::max<int64_t>(rmax, 1);
    p->nsplit = merge_gram_splits(p->M, p->Rmax);
    return SVD_OK;
}

#define LAUNCH(plan, n, expr)                                  \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) {                               \
            fprintf(stderr, "ranky: %s: %s\n", #expr, cudaGetErrorString(_e)); \
            return SVD_ERR_CUDA;                               \
        }                                                      \
        (plan)->launches += (n);                               \
    } while (0)

#define CU(expr)                                                \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) {                                \
            fprintf(stderr, "ranky: %s: %s\n", #expr, cudaGetErrorString(_e)); \
            return SVD_ERR_CUDA;                                \
        }                                                       \
    } while (0)

svd_status run_device(svd_plan_s* p, const int64_t* col_ptr, const int32_t* row_idx,
                      const void* vals, double* d_sigma, double* d_U, void* d_V, int32_t* d_rank,
                      svd_patch* d_patches, int64_t* d_npatches, cudaStream_t s) {
    const int D = p->D, M = p->M, Mp = p->Mp;
    const int64_t mm = (int64_t)Mp * Mp;
    const int vt = p->d.value_type;
    p->launches = 0;
    const int slot = (int)(p->run_index % kRing);
    if (p->timing && p->ev_pending[slot]) {
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
    auto mark = [&](int i) {
        if (p->timing) cudaEventRecord(p->ev[slot][i], s);
    };
    mark(0);

    CU(cudaMemsetAsync(p->occ, 0, sizeof(uint32_t) * (size_t)D * p->W, s));
    CU(cudaMemsetAsync(p->G64, 0, sizeof(double) * (size_t)D * mm, s));
    // Algorithm 1: per-block row occupancy, lonely nodes; Algorithm 2 patches
    LAUNCH(p, 1, launch_occupancy(col_ptr, row_idx, vals, vt, M, p->nchunks, p->chunk_block,
                                  p->chunk_lo, p->chunk_hi, p->occ, s));
    LAUNCH(p, 1, launch_lonely_patches(p->occ, D, M, p->bounds_d, p->random ? 1 : 0, p->d.seed,
                                       p->row_ne, p->lonely, p->patches, p->patch_ofs,
                                       reinterpret_cast<PatchRec*>(d_patches), d_npatches, s));
    mark(1);
    // Eq. 2: block cross products
    LAUNCH(p, 1, launch_gram(col_ptr, row_idx, vals, vt, Mp, p->nchunks, p->chunk_block,
                             p->chunk_lo, p->chunk_hi, p->G64, s));
    if (p->random)
        LAUNCH(p, 1, launch_gram_patches(col_ptr, row_idx, vals, vt, Mp, D, p->patches,
                                         p->patch_ofs, D * M, p->G64, s));
    LAUNCH(p, 1, launch_symmetrize(p->G64, D, Mp, s));

    mark(2);
    // Eq. 1: block eigensolves
    const double* Xblk64 = nullptr;
    const float* Xblk32 = nullptr;
    if (!p->mixed) {
        CU(cudaMemcpyAsync(p->Gw64, p->G64, sizeof(double) * D * mm, cudaMemcpyDeviceToDevice, s));
        LAUNCH(p, 1, launch_jacobi<double>(p->Gw64, p->Vt64, D, Mp, p->max_sweeps, p->jac_tol,
                                           p->sweeps, s));
        LAUNCH(p, 1, launch_sort_rank(nullptr, nullptr, p->Gw64, nullptr, D, M, Mp, p->bounds_d, 0,
                                      p->d.rank_tol, p->bsig, p->bperm, p->brank, s));
        mark(3);
        Xblk64 = p->Vt64;
    } else {
        LAUNCH(p, 1, launch_convert_f64_f32(p->G64, p->G32, (int64_t)D * mm, s));
        LAUNCH(p, 1, launch_jacobi<float>(p->G32, p->Vt32, D, Mp, p->max_sweeps, p->jac_tol,
                                          p->sweeps, s));
        mark(3);
        if (p->refine_iters > 0) {
            LAUNCH(p, 1, launch_convert_f32_f64(p->Vt32, p->Vt64, (int64_t)D * mm, s));
            double* X = p->Vt64;
            double* Xn = p->Xn;
            for (int it = 0; it < p->refine_iters; ++it) {
                LAUNCH(p, 7, launch_refine(p->G64, X, Xn, p->lam, D, Mp, p->RW1, p->RW2, p->RW3,
                                           p->norms, s));
                std::swap(X, Xn);
            }
            LAUNCH(p, 1, launch_sort_rank(p->lam, nullptr, nullptr, nullptr, D, M, Mp, p->bounds_d,
                                          0, p->d.rank_tol, p->bsig, p->bperm, p->brank, s));
            Xblk64 = X;
        } else {
            LAUNCH(p, 1, launch_sort_rank(nullptr, nullptr, nullptr, p->G32, D, M, Mp, p->bounds_d,
                                          0, p->d.rank_tol, p->bsig, p->bperm, p->brank, s));
            Xblk32 = p->Vt32;
        }
    }
    mark(4);
    // proxy P = [U^1 S^1 | ... | U^D S^D] and P P^T (Eqs. 2-3)
    LAUNCH(p, 2, launch_proxy(Xblk64, Xblk32, p->bsig, p->bperm, p->brank, D, M, Mp, p->pofs, p->P,
                              s));
    mark(5);
    LAUNCH(p, 2, launch_merge_gram(p->P, p->pofs, D, M, Mp, p->Rmax, p->partial, p->nsplit,
                                   p->S64, s));
    mark(6);
    // merge eigensolve
    const double* Xm64 = nullptr;
    if (!p->mixed) {
        CU(cudaMemcpyAsync(p->Sw64, p->S64, sizeof(double) * mm, cudaMemcpyDeviceToDevice, s));
        LAUNCH(p, 1, launch_jacobi<double>(p->Sw64, p->SV64, 1, Mp, p->max_sweeps, p->jac_tol,
                                           p->sweeps + D, s));
        LAUNCH(p, 1, launch_sort_rank(nullptr, nullptr, p->Sw64, nullptr, 1, M, Mp, nullptr, p->N,
                                      p->d.rank_tol, p->msig, p->mperm, p->mrank, s));
        Xm64 = p->SV64;
    } else {
        LAUNCH(p, 1, launch_convert_f64_f32(p->S64, p->S32, mm, s));
        LAUNCH(p, 1, launch_jacobi<float>(p->S32, p->SV32, 1, Mp, p->max_sweeps, p->jac_tol,
                                          p->sweeps + D, s));
        LAUNCH(p, 1, launch_convert_f32_f64(p->SV32, p->SV64, mm, s));
        double* X = p->SV64;
        double* Xn = p->SXn;
        for (int it = 0; it < p->merge_refine_iters; ++it) {
            LAUNCH(p, 7, launch_refine(p->S64, X, Xn, p->slam, 1, Mp, p->SR1, p->SR2, p->SR3,
                                       p->snorm, s));
            std::swap(X, Xn);
        }
        LAUNCH(p, 1, launch_sort_rank(p->slam, nullptr, nullptr, nullptr, 1, M, Mp, nullptr, p->N,
                                      p->d.rank_tol, p->msig, p->mperm, p->mrank, s));
        Xm64 = X;
    }
    mark(7);
    const double lam_abs = p->d.rank_tol > 0 ? p->d.rank_tol * p->d.rank_tol : 0.0;
    const int64_t tol_scale = std::max<int64_t>(M, p->N);
    LAUNCH(p, 1, launch_finalize(Xm64, nullptr, p->msig, p->mperm, M, Mp, p->k, lam_abs, tol_scale,
                                 d_sigma, d_U, d_rank, p->W64, p->W32, s));
    mark(8);
    // V = A'^T W
    if (!(p->d.flags & SVD_FLAG_SKIP_V) && d_V) {
        if (p->mixed) {
            LAUNCH(p, 1, launch_spmm<float>(col_ptr, row_idx, vals, vt, p->N, p->k, p->W32,
                                            static_cast<float*>(d_V), s));
            if (p->random)
                LAUNCH(p, 1, launch_spmm_patches<float>(p->patches, p->patch_ofs + D, D * M, p->k,
                                                        p->W32, static_cast<float*>(d_V), s));
        } else {
            LAUNCH(p, 1, launch_spmm<double>(col_ptr, row_idx, vals, vt, p->N, p->k, p->W64,
                                             static_cast<double*>(d_V), s));
            if (p->random)
                LAUNCH(p, 1, launch_spmm_patches<double>(p->patches, p->patch_ofs + D, D * M, p->k,
                                                         p->W64, static_cast<double*>(d_V), s));
        }
    }
    mark(9);
    if (p->timing) p->ev_pending[slot] = true;
    ++p->run_index;
    p->last_stream = s;
    p->ran = true;
    return SVD_OK;
}

}  // namespace

extern "C" {

int32_t svd_version(void) { return 1; }

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
    st = fill_plan(desc, &tmp);
    if (st != SVD_OK) return st;
    Carver c{nullptr, 0, true};
    carve(&tmp, c);
    if (bytes) *bytes = c.off;
    return SVD_OK;
}

svd_status svd_plan(const svd_desc* desc, svd_plan_t* out, size_t* bytes) {
    if (!out) return SVD_ERR_INVALID_ARG;
    *out = nullptr;
    svd_status st = validate_desc(desc);
    if (st != SVD_OK) return st;
    svd_plan_s* p = new (std::nothrow) svd_plan_s();
    if (!p) return SVD_ERR_OOM;
    st = fill_plan(desc, p);
    if (st != SVD_OK) { delete p; return st; }
    Carver dry{nullptr, 0, true};
    carve(p, dry);
    p->arena_bytes = dry.off;
    if (cudaMalloc(&p->arena, p->arena_bytes) != cudaSuccess) {
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
    ok = ok && cudaMemset(p->sweeps, 0, sizeof(int32_t) * (p->D + 1)) == cudaSuccess;
    if (!ok) {
        cudaFree(p->arena);
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

svd_status svd_run(svd_plan_t p, const int64_t* d_col_ptr, const int32_t* d_row_idx,
                   const void* d_vals, double* d_sigma, double* d_U, void* d_V, int32_t* d_rank,
                   svd_patch* d_patches, int64_t* d_npatches, void* stream) {
    if (!p || !d_col_ptr || (!d_row_idx && p->nnz > 0) || (!d_vals && p->nnz > 0) || !d_sigma ||
        !d_U || !d_rank)
        return SVD_ERR_INVALID_ARG;
    if (!d_V && !(p->d.flags & SVD_FLAG_SKIP_V)) return SVD_ERR_INVALID_ARG;
    if ((d_patches == nullptr) != (d_npatches == nullptr)) return SVD_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p->d.flags & SVD_FLAG_CHECK_CSC) {
        svd_status st = svd_check_csc(p->M, p->N, p->nnz, d_col_ptr, d_row_idx, stream);
        if (st != SVD_OK) return st;
    }
    return run_device(p, d_col_ptr, d_row_idx, d_vals, d_sigma, d_U, d_V, d_rank, d_patches,
                      d_npatches, s);
}

svd_status svd_run_host(svd_plan_t p, const int64_t* h_col_ptr, const int32_t* h_row_idx,
                        const void* h_vals, double* h_sigma, double* h_U, void* h_V,
                        int32_t* h_rank, svd_patch* h_patches, int64_t* h_npatches,
                        void* stream) {
    if (!p || !h_col_ptr || (!h_row_idx && p->nnz > 0) || (!h_vals && p->nnz > 0) || !h_sigma ||
        !h_U || !h_rank)
        return SVD_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t sv = p->d.value_type == SVD_VALUE_F32 ? 4 : 8;
    const size_t sV = p->mixed ? 4 : 8;
    const bool want_v = h_V && !(p->d.flags & SVD_FLAG_SKIP_V);
    Carver dry{nullptr, 0, true};
    dry.take<int64_t>(p->N + 1);
    dry.take<int32_t>(std::max<int64_t>(p->nnz, 1));
    dry.take<char>(std::max<int64_t>(p->nnz, 1) * sv);
    dry.take<double>(p->k);
    dry.take<double>((size_t)p->M * p->k);
    dry.take<char>(want_v ? (size_t)p->N * p->k * sV : 1);
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
    int64_t* cp = c.take<int64_t>(p->N + 1);
    int32_t* ri = c.take<int32_t>(std::max<int64_t>(p->nnz, 1));
    char* va = c.take<char>(std::max<int64_t>(p->nnz, 1) * sv);
    double* sg = c.take<double>(p->k);
    double* U = c.take<double>((size_t)p->M * p->k);
    char* V = c.take<char>(want_v ? (size_t)p->N * p->k * sV : 1);
    int32_t* rk_ = c.take<int32_t>(1);
    svd_patch* pt = c.take<svd_patch>((size_t)p->D * p->M);
    int64_t* np = c.take<int64_t>(1);
    CU(cudaMemcpyAsync(cp, h_col_ptr, sizeof(int64_t) * (p->N + 1), cudaMemcpyHostToDevice, s));
    if (p->nnz > 0) {
        CU(cudaMemcpyAsync(ri, h_row_idx, sizeof(int32_t) * p->nnz, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(va, h_vals, sv * p->nnz, cudaMemcpyHostToDevice, s));
    }
    const int saved = p->d.flags;
    if (!want_v) p->d.flags |= SVD_FLAG_SKIP_V;
    svd_status st = svd_run(p, cp, ri, va, sg, U, want_v ? V : nullptr, rk_, pt, np, stream);
    p->d.flags = saved;
    if (st != SVD_OK) return st;
    CU(cudaMemcpyAsync(h_sigma, sg, sizeof(double) * p->k, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(h_U, U, sizeof(double) * p->M * p->k, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(h_rank, rk_, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (want_v) CU(cudaMemcpyAsync(h_V, V, (size_t)p->N * p->k * sV, cudaMemcpyDeviceToHost, s));
    if (h_npatches) CU(cudaMemcpyAsync(h_npatches, np, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (h_patches)
        CU(cudaMemcpyAsync(h_patches, pt, sizeof(svd_patch) * (size_t)p->D * p->M,
                           cudaMemcpyDeviceToHost, s));
    return svd_sync(p);
}

svd_status svd_sync(svd_plan_t p) {
    if (!p) return SVD_ERR_INVALID_ARG;
    if (!p->ran) return SVD_OK;
    CU(cudaStreamSynchronize(p->last_stream));
    std::vector<int32_t> sw(p->D + 1);
    CU(cudaMemcpy(sw.data(), p->sweeps, sizeof(int32_t) * (p->D + 1), cudaMemcpyDeviceToHost));
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
            CU(cudaMemcpy(h_dst, p->pofs + D, bytes, cudaMemcpyDeviceToHost));
            return SVD_OK;
        case SVD_Q_PROXY: {
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
    if (p->arena) cudaFree(p->arena);
    if (p->host_arena) cudaFree(p->host_arena);
    if (p->timing)
        for (int r = 0; r < kRing; ++r)
            for (int i = 0; i <= kStages; ++i) cudaEventDestroy(p->ev[r][i]);
    delete p;
}

}  // extern "C"
