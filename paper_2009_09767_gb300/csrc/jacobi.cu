// jacobi.cu -- batched block two-sided Jacobi eigensolvers for the symmetric
// positive semi-definite cross products of Ranky's block SVD (arXiv
// 2009.09767, Eq. 1: A^i = U^i S^i V^i*, whose U^i and (S^i)^2 are the
// eigenvectors and eigenvalues of A^i A^i^T).
//
// Common structure:
//   * The index set 0..Mp-1 (Mp a multiple of 32) is cut into nb = Mp/16
//     blocks of 16 indices.  A round-robin (circle) schedule pairs the blocks;
//     each of the nb-1 steps of a sweep handles nb/2 disjoint block pairs.
//   * A matrix is owned by a cluster of csize CTAs.  Each pair's 32 x 32
//     sub-problem G[I+J, I+J] gets one cyclic sweep of 31 rounds x 16
//     disjoint rotations in shared memory, accumulating its rotation Q; the
//     step's rotation diag(Q_1, ..) is then applied to G and to the
//     eigenvectors.  A sweep in which no rotation passed the threshold ends
//     the solve.
//   * G and the eigenvectors live in global memory (L2-resident at these
//     sizes) and are read with L2-only loads, because other CTAs of the
//     cluster write them between barriers.  Padding indices (M..Mp-1) hold
//     zero rows and columns: they never rotate, so their eigenvectors stay
//     exact unit vectors.
//
// FP64 solver (k_jacobi<double>, k_jacobi_items<double>): one warp per pair
// solve; phase A: rows I+J of G and of Vt become Q^T times themselves (panel
// products through shared memory on the FP64 pipes), cluster barrier;
// phase B: columns I+J of G become themselves times Q, cluster barrier.
//
// FP32 solver (k_jacobi4, k_jacobi4_items): see the section below; the
// update runs as independent warp jobs on the tensor cores.
//
// Two launch forms each: one cluster per matrix (all matrices of one size),
// and persistent single-CTA workers that take matrices of any size from a
// work list (to batch many problems in one launch).
#include <cooperative_groups.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace rk {

namespace {

constexpr int kJT = 512;          // threads per CTA (16 warps)
constexpr int kB2 = 32;           // sub-problem size
constexpr int kB = kB2 / 2;       // index block size
constexpr int kMaxCluster = 16;

template <typename T> struct PairsMax;
template <> struct PairsMax<double> { static constexpr int value = 8; };

// circle schedule over n (even) items: partner pair u of round r
__device__ __forceinline__ void circle_pair(int n, int r, int u, int& a, int& b) {
    if (u == 0) {
        a = n - 1;
        b = r;
    } else {
        a = (r + u) % (n - 1);
        b = (r - u + (n - 1)) % (n - 1);
    }
    if (a > b) { const int t = a; a = b; b = t; }
}

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

template <typename T> struct V16;
template <> struct V16<double> {
    using type = double2;
    static constexpr int n = 2;
    __device__ static double get(const double2& v, int i) { return i == 0 ? v.x : v.y; }
};

template <typename T>
__device__ __forceinline__ void lds4(const T* p, T (&o)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 c = *reinterpret_cast<const double2*>(p + 2);
        o[0] = a.x; o[1] = a.y; o[2] = c.x; o[3] = c.y;
    }
}

template <typename T>
__device__ __forceinline__ void stg4(T* dst, const T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        reinterpret_cast<double2*>(dst)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(dst)[1] = make_double2(v[2], v[3]);
    }
}

// Shared-memory layout (in elements of T unless noted):
//   stage  STAGE             panel tile (16-byte aligned)
//   Q      ppc x 32 x LD     rotations of this CTA's pairs
//   sub    ppc x 32 x LD     sub-problems
//   rot    ppc x 16 x {c, s} rotation table of each warp's current round
//   pq     ppc x 16 x {p, q} (int)
template <typename T>
struct JSmem {
    static constexpr int LD = kB2 + 1;                 // odd stride: row and column access conflict-free
    static constexpr int PAD = 32 / (int)sizeof(T);    // 16-byte aligned rows, shifted banks
    static constexpr int TW = 8192 / kB2;              // row-panel tile width (256)
    static constexpr int RSLD = TW + PAD;
    static constexpr int TR = 8192 / kB2;              // column-panel tile height (256)
    static constexpr int CSLD = kB2 + 4;
    static constexpr int STAGE = (kB2 * RSLD > TR * CSLD) ? kB2 * RSLD : TR * CSLD;
    static constexpr int NSTAGE = 1;
    static constexpr size_t bytes(int ppc) {
        return sizeof(T) * ((size_t)NSTAGE * STAGE + 2ull * ppc * kB2 * LD + 2ull * ppc * kB) +
               sizeof(int) * 2ull * ppc * kB;
    }
};

// One cyclic sweep of the 32 x 32 sub-problem by one warp, accumulating Q.
// The 16 rotations of a round are independent, so each lane loads all the
// values it needs for the 16 of them before updating any: the round's shared
// memory traffic overlaps instead of forming 16 dependent chains.  A rotation
// that did not pass the threshold is the identity (c = 1, s = 0).
template <typename T>
__device__ void warp_sweep(T* sub, T* Q, T* rc, T* rs, int* rp, int* rq, T tol, T floor_abs,
                           int& rotated) {
    constexpr int LD = JSmem<T>::LD;
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < kB2 - 1; ++r) {
        T a = T(0), d = T(0), g = T(0), t = T(0);
        bool rot = false;
        int p = 0, q = 0;
        if (lane < kB) {
            circle_pair(kB2, r, lane, p, q);
            a = sub[p * LD + p];
            d = sub[q * LD + q];
            g = sub[p * LD + q];
            T c = T(1), s = T(0);
            const T ag = g < T(0) ? -g : g;
            const T rel = tol * sqrt(fabs(a) * fabs(d));
            if (ag > rel && ag > floor_abs) {
                const T zeta = (d - a) / (T(2) * g);
                const T az = zeta < T(0) ? -zeta : zeta;
                t = (zeta >= T(0) ? T(1) : T(-1)) / (az + sqrt(T(1) + zeta * zeta));
                c = rsqrt_t<T>(T(1) + t * t);
                s = t * c;
                rot = true;
                rotated = 1;
            }
            rc[lane] = c; rs[lane] = s; rp[lane] = p; rq[lane] = q;
        }
        __syncwarp();
        // rows p, q of every pair (lane = column), then columns p, q of every
        // pair and of Q (lane = row); in two halves of 8 pairs to bound the
        // registers held in flight
#pragma unroll
        for (int h = 0; h < kB; h += kB / 2) {
            T cu[kB / 2], su[kB / 2], x[kB / 2], y[kB / 2];
            int pu[kB / 2], qu[kB / 2];
#pragma unroll
            for (int u = 0; u < kB / 2; ++u) {
                cu[u] = rc[h + u]; su[u] = rs[h + u];
                circle_pair(kB2, r, h + u, pu[u], qu[u]);
            }
#pragma unroll
            for (int u = 0; u < kB / 2; ++u) { x[u] = sub[pu[u] * LD + lane]; y[u] = sub[qu[u] * LD + lane]; }
#pragma unroll
            for (int u = 0; u < kB / 2; ++u) {
                sub[pu[u] * LD + lane] = cu[u] * x[u] - su[u] * y[u];
                sub[qu[u] * LD + lane] = su[u] * x[u] + cu[u] * y[u];
            }
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < kB; h += kB / 2) {
            T cu[kB / 2], su[kB / 2], x[kB / 2], y[kB / 2];
            int pu[kB / 2], qu[kB / 2];
#pragma unroll
            for (int u = 0; u < kB / 2; ++u) {
                cu[u] = rc[h + u]; su[u] = rs[h + u];
                circle_pair(kB2, r, h + u, pu[u], qu[u]);
            }
#pragma unroll
            for (int u = 0; u < kB / 2; ++u) { x[u] = sub[lane * LD + pu[u]]; y[u] = sub[lane * LD + qu[u]]; }
#pragma unroll
            for (int u = 0; u < kB / 2; ++u) {
                sub[lane * LD + pu[u]] = cu[u] * x[u] - su[u] * y[u];
                sub[lane * LD + qu[u]] = su[u] * x[u] + cu[u] * y[u];
            }
#pragma unroll
            for (int u = 0; u < kB / 2; ++u) { x[u] = Q[lane * LD + pu[u]]; y[u] = Q[lane * LD + qu[u]]; }
#pragma unroll
            for (int u = 0; u < kB / 2; ++u) {
                Q[lane * LD + pu[u]] = cu[u] * x[u] - su[u] * y[u];
                Q[lane * LD + qu[u]] = su[u] * x[u] + cu[u] * y[u];
            }
        }
        __syncwarp();
        // the rotated 2 x 2 diagonal blocks, exactly
        if (rot) {
            sub[p * LD + p] = a - t * g;
            sub[q * LD + q] = d + t * g;
            sub[p * LD + q] = T(0);
            sub[q * LD + p] = T(0);
        }
        __syncwarp();
    }
}

__device__ __forceinline__ int gidx(int bi, int bj, int k) {
    return k < kB ? bi * kB + k : bj * kB + (k - kB);
}

// rows idx(0..31) of Mat (ld = Mp) <- Q^T * rows, over all Mp columns.
// Tiles of 32 x TW; the global loads of the next tile are issued into
// registers before the current tile is computed.
template <typename T>
__device__ void panel_rows(T* Mat, int Mp, int bi, int bj, const T* Q, T* stage) {
    using S = JSmem<T>;
    constexpr int LD = S::LD, TW = S::TW, SLD = S::RSLD;
    constexpr int VN = V16<T>::n;
    using VT = typename V16<T>::type;
    constexpr int PER = kB2 * (TW / VN) / kJT;    // vectors per thread per tile
    constexpr int CG = TW / 4;                    // 64 column groups
    const int ti = threadIdx.x / CG, tc = threadIdx.x % CG;   // ti < 8
    const int i0 = ti * 4, j0 = tc * 4;
    VT pre[PER];
    auto load = [&](int c0) {
        const int cw = min(TW, Mp - c0);
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int it = threadIdx.x + e * kJT;
            const int k = it / (TW / VN), c = (it % (TW / VN)) * VN;
            if (c < cw) pre[e] = __ldcg(reinterpret_cast<const VT*>(Mat + (int64_t)gidx(bi, bj, k) * Mp + c0 + c));
            else pre[e] = VT{};
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int it = threadIdx.x + e * kJT;
            const int k = it / (TW / VN), c = (it % (TW / VN)) * VN;
            *reinterpret_cast<VT*>(stage + k * SLD + c) = pre[e];
        }
    };
    load(0);
    stash();
    __syncthreads();
    for (int c0 = 0; c0 < Mp; c0 += TW) {
        const int cw = min(TW, Mp - c0);          // multiple of 32
        const bool more = c0 + TW < Mp;
        if (more) load(c0 + TW);
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
#pragma unroll 8
        for (int k = 0; k < kB2; ++k) {
            T qv[4], xv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) qv[i] = Q[k * LD + i0 + i];
            lds4<T>(stage + k * SLD + j0, xv);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(qv[i], xv[j], acc[i][j]);
        }
        if (j0 < cw) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                stg4<T>(Mat + (int64_t)gidx(bi, bj, i0 + i) * Mp + c0 + j0, acc[i]);
        }
        __syncthreads();
        if (more) {
            stash();
            __syncthreads();
        }
    }
}

// columns idx(0..31) of Mat <- columns * Q, over all Mp rows; tiles of TR x 32
// with the next tile's loads in flight during the current one.
template <typename T>
__device__ void panel_cols(T* Mat, int Mp, int bi, int bj, const T* Q, T* stage) {
    using S = JSmem<T>;
    constexpr int LD = S::LD, TR = S::TR, SLD = S::CSLD;
    constexpr int VN = V16<T>::n;
    using VT = typename V16<T>::type;
    constexpr int PER = TR * (kB2 / VN) / kJT;
    constexpr int JG = kB2 / 4;                   // 8 column groups
    const int tr = threadIdx.x / JG, tj = threadIdx.x % JG;   // tr < 64
    const int i0 = tr * 4, j0 = tj * 4;
    VT pre[PER];
    auto load = [&](int r0) {
        const int rh = min(TR, Mp - r0);
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int it = threadIdx.x + e * kJT;
            const int r = it / (kB2 / VN), k = (it % (kB2 / VN)) * VN;
            if (r < rh) pre[e] = __ldcg(reinterpret_cast<const VT*>(Mat + (int64_t)(r0 + r) * Mp + gidx(bi, bj, k)));
            else pre[e] = VT{};
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int it = threadIdx.x + e * kJT;
            const int r = it / (kB2 / VN), k = (it % (kB2 / VN)) * VN;
#pragma unroll
            for (int v = 0; v < VN; ++v) stage[r * SLD + k + v] = V16<T>::get(pre[e], v);
        }
    };
    load(0);
    stash();
    __syncthreads();
    for (int r0 = 0; r0 < Mp; r0 += TR) {
        const int rh = min(TR, Mp - r0);
        const bool more = r0 + TR < Mp;
        if (more) load(r0 + TR);
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
#pragma unroll 8
        for (int k = 0; k < kB2; ++k) {
            T xv[4], qv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) xv[i] = stage[(i0 + i) * SLD + k];
#pragma unroll
            for (int j = 0; j < 4; ++j) qv[j] = Q[k * LD + j0 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(xv[i], qv[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i0 + i >= rh) continue;
            stg4<T>(Mat + (int64_t)(r0 + i0 + i) * Mp + gidx(bi, bj, j0), acc[i]);
        }
        __syncthreads();
        if (more) {
            stash();
            __syncthreads();
        }
    }
}

// Barrier over the CTAs that own one matrix: the cluster, or the CTA alone.
template <bool kCluster>
__device__ __forceinline__ void owner_sync() {
    if constexpr (kCluster) cg::this_cluster().sync();
    else __syncthreads();
}

// Solve one matrix.  csize CTAs (rank crank) share it; ppc pairs per CTA.
template <typename T, bool kCluster>
__device__ void jacobi_matrix(T* __restrict__ G, T* __restrict__ Vt, int Mp, int csize, int crank,
                              int ppc, int max_sweeps, T tol, int32_t* __restrict__ sweeps_out,
                              unsigned char* smem_raw) {
    using SM = JSmem<T>;
    constexpr int LD = SM::LD;
    const int nb = Mp / kB;
    const int npairs = nb / 2;
    const int nmine = (npairs - crank + csize - 1) / csize;   // pairs of this CTA per step
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    T* stage = reinterpret_cast<T*>(smem_raw);
    T* Qs = stage + SM::NSTAGE * SM::STAGE;
    T* subs = Qs + (size_t)ppc * kB2 * LD;
    T* rcs = subs + (size_t)ppc * kB2 * LD;
    T* rss = rcs + (size_t)ppc * kB;
    int* rps = reinterpret_cast<int*>(rss + (size_t)ppc * kB);
    int* rqs = rps + (size_t)ppc * kB;
    __shared__ int rot_flag;
    __shared__ int decision;
    __shared__ T floor_sh;

    for (int64_t e = (int64_t)crank * kJT + threadIdx.x; e < (int64_t)Mp * Mp;
         e += (int64_t)csize * kJT) {
        const int i = (int)(e / Mp), j = (int)(e % Mp);
        Vt[e] = i == j ? T(1) : T(0);
    }
    // Absolute floor of the rotation threshold: rounding leaves off-diagonal
    // noise of order eps * max|G_ij| <= eps * max_i G_ii in a positive
    // semi-definite matrix, which no rotation can remove.
    if (warp == 0) {
        T dmax = T(0);
        for (int i = lane; i < Mp; i += 32) dmax = fmax(dmax, fabs(ldcg(G + (int64_t)i * Mp + i)));
        for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        if (lane == 0) {
            floor_sh = T(4) * T(Eps<T>::value) * dmax;
            rot_flag = 0;
        }
    }
    owner_sync<kCluster>();
    const T floor_abs = floor_sh;

    int sweep = 0;
    bool converged = false;
    while (sweep < max_sweeps) {
        int rotated = 0;
        for (int step = 0; step < nb - 1; ++step) {
            // phase A: warp w solves this CTA's pair w
            if (warp < nmine) {
                const int u = crank + warp * csize;
                int bi, bj;
                circle_pair(nb, step, u, bi, bj);
                T* sub = subs + (size_t)warp * kB2 * LD;
                T* Q = Qs + (size_t)warp * kB2 * LD;
                for (int i = 0; i < kB2; ++i) {
                    sub[i * LD + lane] = ldcg(G + (int64_t)gidx(bi, bj, i) * Mp + gidx(bi, bj, lane));
                    Q[i * LD + lane] = i == lane ? T(1) : T(0);
                }
                __syncwarp();
                warp_sweep<T>(sub, Q, rcs + warp * kB, rss + warp * kB, rps + warp * kB,
                              rqs + warp * kB, tol, floor_abs, rotated);
            }
            __syncthreads();
            for (int t = 0; t < nmine; ++t) {
                int bi, bj;
                circle_pair(nb, step, crank + t * csize, bi, bj);
                const T* Q = Qs + (size_t)t * kB2 * LD;
                panel_rows<T>(G, Mp, bi, bj, Q, stage);
                panel_rows<T>(Vt, Mp, bi, bj, Q, stage);
            }
            owner_sync<kCluster>();
            // phase B: columns of G
            for (int t = 0; t < nmine; ++t) {
                int bi, bj;
                circle_pair(nb, step, crank + t * csize, bi, bj);
                panel_cols<T>(G, Mp, bi, bj, Qs + (size_t)t * kB2 * LD, stage);
            }
            owner_sync<kCluster>();
        }
        ++sweep;
        // OR of the rotation flags over the owners
        if (__syncthreads_or(rotated) && threadIdx.x == 0) rot_flag = 1;
        __syncthreads();
        int any;
        if constexpr (kCluster) {
            cg::cluster_group cluster = cg::this_cluster();
            if (crank == 0 && threadIdx.x == 0) {
                int acc = 0;
                for (int r = 0; r < csize; ++r) acc |= *cluster.map_shared_rank(&rot_flag, r);
                decision = acc;
            }
            cluster.sync();
            any = *cluster.map_shared_rank(&decision, 0);
            cluster.sync();
        } else {
            any = rot_flag;
            __syncthreads();
        }
        if (threadIdx.x == 0) rot_flag = 0;
        __syncthreads();
        if (!any) { converged = true; break; }
    }
    if (crank == 0 && threadIdx.x == 0) *sweeps_out = converged ? sweep : -sweep;
}

template <typename T>
__global__ void __launch_bounds__(kJT, 1)
k_jacobi(T* __restrict__ Gall, T* __restrict__ Vtall, int Mp, int csize, int ppc, int max_sweeps,
         T tol, int32_t* __restrict__ sweeps_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int crank = (int)cg::this_cluster().block_rank();
    const int mat = blockIdx.x / csize;
    jacobi_matrix<T, true>(Gall + (int64_t)mat * Mp * Mp, Vtall + (int64_t)mat * Mp * Mp, Mp, csize,
                           crank, ppc, max_sweeps, tol, sweeps_out + mat, smem_raw);
}

// Persistent workers: each CTA takes the next matrix of the list until none is left.
template <typename T>
__global__ void __launch_bounds__(kJT, 1)
k_jacobi_items(const JacobiItem* __restrict__ items, int nitems, int* __restrict__ next,
               int max_sweeps, T tol) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int item_sh;
    for (;;) {
        if (threadIdx.x == 0) item_sh = atomicAdd(next, 1);
        __syncthreads();
        const int it = item_sh;
        __syncthreads();
        if (it >= nitems) break;
        const JacobiItem w = items[it];
        const int ppc = w.Mp / kB2;
        jacobi_matrix<T, false>(static_cast<T*>(w.G), static_cast<T*>(w.Vt), w.Mp, 1, 0, ppc,
                                w.max_sweeps > 0 ? w.max_sweeps : max_sweeps, tol, w.sweeps,
                                smem_raw);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// FP32 solver, symmetric block form.  The step's rotation is
// J = diag(Q_1, ..., Q_np) over the pair index sets P_u = I_u + J_u, so the
// new matrix is made of the 32 x 32 blocks
//   G'[P_u, P_w] = Q_u^T G[P_u, P_w] Q_w          (u <= w, mirrored below)
// and the eigenvector columns V'[:, P_u] = V[:, P_u] Q_u (V = Vt^T while the
// solve runs).  Every block is one independent warp job, with no CTA-wide
// barrier inside the update: one cluster barrier after the pair solves
// (their Q are published through L2) and one after the update.
//
// Products run on the tensor cores with f16 operands split as
// hi = f16(x), lo = f16(x - hi) and accumulated as lo*hi + hi*lo + hi*hi
// in FP32 (22 significant bits per operand, the same as a TF32 hi/lo split,
// in half as many mma instructions).  The split keeps 22 bits only while lo
// is a normal f16, i.e. for |x| >= 2^-3, so every operand is moved up the
// f16 exponent range by a power of two (exact, removed in FP32): G is scaled
// on entry so that its Gershgorin bound max_i sum_j |G_ij| (>= lambda_max,
// which bounds every entry of every iterate; the diagonal alone does not:
// it grows towards lambda_max as the solve proceeds) lies in [2^12, 2^13),
// so that |Q^T G[P_u, P_w]| <= sqrt(32) 2^13 < 2^16 stays finite; Q and V
// are split as 2^14 Q and 2^14 V.  Below 2^-3 of its scale an operand keeps an absolute
// error of 2^-25 of that scale, far under the rotation floor; without the
// shift that error reaches the floor and rotations never stop.  Q is
// published as (2^14 Q)^T (row n = column n of Q), hi then lo, 32 x 32
// halves each: both GEMM operands read from it as consecutive pairs.
constexpr int kJT4 = 256;                      // threads per CTA
constexpr int kW4 = kJT4 / 32;                 // warps per CTA
constexpr int kQWords = kB2 * kB2 / 2;         // 32-bit words of one 32 x 32 f16 matrix
constexpr float kQScale = 16384.f;             // 2^14: Q and V as split operands
constexpr float kQInv = 1.f / 16384.f;

// Update jobs may stage their global operand (32 rows x the 32 columns of
// P_u) in a per-warp shared buffer with cp.async: the next job's copy is
// in flight while the current job computes.  Rows are padded to 40 floats,
// so that the 8-byte fragment loads of a half warp hit 32 distinct banks.
constexpr int kStageLD = 40;
constexpr size_t kStageBytes = (size_t)kB2 * kStageLD * sizeof(float);

struct J4Smem {
    static constexpr int LD = kB2 + 1;
    // per warp: sub-problem, its rotation, the round's rotation table
    // (c, s, p, q per pair as one float4) and the round flags
    static constexpr size_t per_warp = sizeof(float) * 2 * kB2 * LD + sizeof(float4) * kB + sizeof(int) * 4;
    static constexpr size_t solve_bytes = per_warp * kW4;
    static constexpr size_t staged_bytes = solve_bytes + kW4 * kStageBytes;
    static constexpr size_t bytes(bool staged) { return staged ? staged_bytes : solve_bytes; }
};

// 32-bit words of solver work per matrix: np published rotations (2 kQWords
// words each) and np identity flags, rounded to 256 bytes.
__host__ __device__ inline size_t jwork_words(int Mp) {
    return (size_t)round_up((int64_t)(Mp / kB2) * (2 * kQWords + 1), 64);
}

__device__ __forceinline__ void split_h2(float x, float y, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(x, y);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(x - hf.x, y - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void mma_f16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d += A B with A = ah + al, B = bh + bl (the al*bl term is below the split)
__device__ __forceinline__ void mma_split(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                          uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    mma_f16(d, al, bh0, bh1);
    mma_f16(d, ah, bl0, bl1);
    mma_f16(d, ah, bh0, bh1);
}

// Rotation word off of a published (2^14 Q)^T from the CTA's shared copy
// (kS) or from L2.  The staged kernels store their shared copy with the
// 16-byte groups of each 16-word row XOR-ed by (row / 2) mod 4, so that the
// eight rows one fragment load touches fall in distinct banks (kSw).
template <bool kS, bool kSw>
__device__ __forceinline__ uint32_t ldq(const uint32_t* q, int off) {
    if constexpr (kS && kSw) return q[off ^ (((off >> 5) & 3) << 2)];
    else if constexpr (kS) return q[off];
    else return __ldcg(q + off);
}
__device__ __forceinline__ float2 ldcg_f2(const float* p) {
    return __ldcg(reinterpret_cast<const float2*>(p));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Stage rows row(n), n < 32, of Mat at the 32 columns of P_u = (ui, uj) into
// stg[n][k]: row(n) = P_w(n) of a block job (blk), r0 + n of a column job.
// Each 16-byte copy stays inside one 16-column half of P_u.
__device__ __forceinline__ void stage_rows(float* stg, const float* Mat, int Mp, int ui, int uj, bool blk,
                                           int wi, int wj, int r0) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = i * 32 + lane;
        const int n = c >> 3, k = (c & 7) * 4;
        const int row = blk ? gidx(wi, wj, n) : r0 + n;
        cp_async16(stg + n * kStageLD + k, Mat + (int64_t)row * Mp + gidx(ui, uj, k));
    }
    cp_async_commit();
}

// Fragments of a staged block job (B[k][n] = stg[n][k]) and of a staged
// column job (A[m][k] = stg[m][k]) in the order job_block / job_vcols take.
__device__ __forceinline__ void frag_block(const float* stg, float2 (&op)[16]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk)
#pragma unroll
        for (int nj = 0; nj < 4; ++nj)
#pragma unroll
            for (int h = 0; h < 2; ++h)
                op[(kk * 4 + nj) * 2 + h] =
                    *reinterpret_cast<const float2*>(stg + (nj * 8 + g) * kStageLD + kk * 16 + 2 * t + 8 * h);
}
__device__ __forceinline__ void frag_vcols(const float* stg, float2 (&op)[16]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk)
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            const float* r = stg + (mi * 16 + g) * kStageLD + kk * 16 + 2 * t;
            float2* o = op + (kk * 2 + mi) * 4;
            o[0] = *reinterpret_cast<const float2*>(r);
            o[1] = *reinterpret_cast<const float2*>(r + 8 * kStageLD);
            o[2] = *reinterpret_cast<const float2*>(r + 8);
            o[3] = *reinterpret_cast<const float2*>(r + 8 * kStageLD + 8);
        }
}

// Fragment coordinates (m16n8k16): g = lane / 4, t = lane % 4;
//   A (16 x 16): (g, 2t..2t+1) (g+8, 2t..) (g, 2t+8..) (g+8, 2t+8..)
//   B (16 x 8):  (k = 2t..2t+1, n = g) (k = 2t+8.., n = g)
//   C (16 x 8):  (g, 2t) (g, 2t+1) (g+8, 2t) (g+8, 2t+1)

// Block job: G[P_u, P_w] <- Q_u^T G[P_u, P_w] Q_w and its mirror.  B of the
// first product is read through the symmetry, B[k][n] = G[P_w(n)][P_u(k)],
// so every fragment is a consecutive pair.  On the diagonal (u == w) only the
// upper triangle is written, to both halves.  Staged (kSt): the B fragments
// come in op, op[(kk * 4 + nj) * 2 + h] = B[16kk + 2t + 8h][8nj + g].
template <bool kS, bool kSt>
__device__ void job_block(float* __restrict__ G, int Mp, const uint32_t* __restrict__ Qu,
                          const uint32_t* __restrict__ Qw, int ui, int uj, int wi, int wj,
                          const float2 (&op)[16]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const bool diag = ui == wi && uj == wj;
    float acc[2][4][4];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
            for (int z = 0; z < 4; ++z) acc[x][y][z] = 0.f;
    // T = Q_u^T B: A[m][k] = QT_u[m][k]
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            const int m = mi * 16 + g, kp = kk * 8 + t;
            ah[mi][0] = ldq<kS, kSt>(Qu, m * 16 + kp);
            ah[mi][1] = ldq<kS, kSt>(Qu, (m + 8) * 16 + kp);
            ah[mi][2] = ldq<kS, kSt>(Qu, m * 16 + kp + 4);
            ah[mi][3] = ldq<kS, kSt>(Qu, (m + 8) * 16 + kp + 4);
            al[mi][0] = ldq<kS, kSt>(Qu, kQWords + m * 16 + kp);
            al[mi][1] = ldq<kS, kSt>(Qu, kQWords + (m + 8) * 16 + kp);
            al[mi][2] = ldq<kS, kSt>(Qu, kQWords + m * 16 + kp + 4);
            al[mi][3] = ldq<kS, kSt>(Qu, kQWords + (m + 8) * 16 + kp + 4);
        }
        const int k = kk * 16 + 2 * t;
        const int c0 = gidx(ui, uj, k), c1 = gidx(ui, uj, k + 8);
#pragma unroll
        for (int nj = 0; nj < 4; ++nj) {
            const float* row = G + (int64_t)gidx(wi, wj, nj * 8 + g) * Mp;
            const float2 v0 = kSt ? op[(kk * 4 + nj) * 2] : ldcg_f2(row + c0);
            const float2 v1 = kSt ? op[(kk * 4 + nj) * 2 + 1] : ldcg_f2(row + c1);
            uint32_t bh0, bl0, bh1, bl1;
            split_h2(v0.x, v0.y, bh0, bl0);
            split_h2(v1.x, v1.y, bh1, bl1);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) mma_split(acc[mi][nj], ah[mi], al[mi], bh0, bh1, bl0, bl1);
        }
    }
    // out = T Q_w: A = T from the accumulators, B[k][n] = QT_w[n][k]
    float out[2][4][4];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
            for (int z = 0; z < 4; ++z) out[x][y][z] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            // T = Q_u^T B: the accumulators hold 2^14 T
            const float* c0 = acc[mi][2 * kk];
            const float* c1 = acc[mi][2 * kk + 1];
            split_h2(c0[0] * kQInv, c0[1] * kQInv, ah[mi][0], al[mi][0]);
            split_h2(c0[2] * kQInv, c0[3] * kQInv, ah[mi][1], al[mi][1]);
            split_h2(c1[0] * kQInv, c1[1] * kQInv, ah[mi][2], al[mi][2]);
            split_h2(c1[2] * kQInv, c1[3] * kQInv, ah[mi][3], al[mi][3]);
        }
#pragma unroll
        for (int nj = 0; nj < 4; ++nj) {
            const int n = nj * 8 + g, kp = kk * 8 + t;
            const uint32_t bh0 = ldq<kS, kSt>(Qw, n * 16 + kp), bh1 = ldq<kS, kSt>(Qw, n * 16 + kp + 4);
            const uint32_t bl0 = ldq<kS, kSt>(Qw, kQWords + n * 16 + kp);
            const uint32_t bl1 = ldq<kS, kSt>(Qw, kQWords + n * 16 + kp + 4);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) mma_split(out[mi][nj], ah[mi], al[mi], bh0, bh1, bl0, bl1);
        }
    }
    __syncwarp();
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int hz = 0; hz < 2; ++hz) {
            const int m = mi * 16 + g + 8 * hz;
            const int gm = gidx(ui, uj, m);
#pragma unroll
            for (int nj = 0; nj < 4; ++nj) {
                const int n = nj * 8 + 2 * t;
                const int gn = gidx(wi, wj, n);       // n, n + 1 in the same half
                const float v0 = out[mi][nj][2 * hz] * kQInv, v1 = out[mi][nj][2 * hz + 1] * kQInv;
                if (!diag) {
                    *reinterpret_cast<float2*>(G + (int64_t)gm * Mp + gn) = make_float2(v0, v1);
                    G[(int64_t)gn * Mp + gm] = v0;
                    G[(int64_t)(gn + 1) * Mp + gm] = v1;
                } else {
                    if (m <= n) {
                        G[(int64_t)gm * Mp + gn] = v0;
                        G[(int64_t)gn * Mp + gm] = v0;
                    }
                    if (m <= n + 1) {
                        G[(int64_t)gm * Mp + gn + 1] = v1;
                        G[(int64_t)(gn + 1) * Mp + gm] = v1;
                    }
                }
            }
        }
}

// Column job: V[r0..r0+31, P_u] <- V[r0..r0+31, P_u] Q_u.  Staged (kSt): the
// A fragments come in op, op[(kk * 2 + mi) * 4 + q] = rows 16mi + g (+8 for
// q odd), columns 16kk + 2t (+8 for q >= 2).
template <bool kS, bool kSt>
__device__ void job_vcols(float* __restrict__ V, int Mp, const uint32_t* __restrict__ Qu, int ui,
                          int uj, int r0, const float2 (&op)[16]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float out[2][4][4];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
            for (int z = 0; z < 4; ++z) out[x][y][z] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        const int k = kk * 16 + 2 * t;
        const int c0 = gidx(ui, uj, k), c1 = gidx(ui, uj, k + 8);
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            const float* ra = V + (int64_t)(r0 + mi * 16 + g) * Mp;
            const float* rb = ra + 8 * (int64_t)Mp;
            const float2* o = op + (kk * 2 + mi) * 4;
            const float2 x0 = kSt ? o[0] : ldcg_f2(ra + c0), x1 = kSt ? o[1] : ldcg_f2(rb + c0);
            const float2 x2 = kSt ? o[2] : ldcg_f2(ra + c1), x3 = kSt ? o[3] : ldcg_f2(rb + c1);
            split_h2(x0.x * kQScale, x0.y * kQScale, ah[mi][0], al[mi][0]);
            split_h2(x1.x * kQScale, x1.y * kQScale, ah[mi][1], al[mi][1]);
            split_h2(x2.x * kQScale, x2.y * kQScale, ah[mi][2], al[mi][2]);
            split_h2(x3.x * kQScale, x3.y * kQScale, ah[mi][3], al[mi][3]);
        }
#pragma unroll
        for (int nj = 0; nj < 4; ++nj) {
            const int n = nj * 8 + g, kp = kk * 8 + t;
            const uint32_t bh0 = ldq<kS, kSt>(Qu, n * 16 + kp), bh1 = ldq<kS, kSt>(Qu, n * 16 + kp + 4);
            const uint32_t bl0 = ldq<kS, kSt>(Qu, kQWords + n * 16 + kp);
            const uint32_t bl1 = ldq<kS, kSt>(Qu, kQWords + n * 16 + kp + 4);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) mma_split(out[mi][nj], ah[mi], al[mi], bh0, bh1, bl0, bl1);
        }
    }
    __syncwarp();
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int hz = 0; hz < 2; ++hz) {
            float* row = V + (int64_t)(r0 + mi * 16 + g + 8 * hz) * Mp;
#pragma unroll
            for (int nj = 0; nj < 4; ++nj) {
                const int gn = gidx(ui, uj, nj * 8 + 2 * t);
                *reinterpret_cast<float2*>(row + gn) =
                    make_float2(out[mi][nj][2 * hz] * (kQInv * kQInv), out[mi][nj][2 * hz + 1] * (kQInv * kQInv));
            }
        }
}

// One cyclic sweep of a 32 x 32 FP32 sub-problem by a group of K warps
// (named barrier bar, 32 K threads), accumulating Q.  Warp 0 of the group
// computes the round's 16 rotations (lanes 0..15) and, at the start of the
// next round, writes the exact 2 x 2 diagonal blocks of the rotated pairs;
// the two-sided update of the 256 2 x 2 blocks and the column pass of Q are
// split over the K warps (two barriers per round).  The rotation parameters use the fast reciprocal and square root
// (the angle only steers convergence); c is polished by one Newton step so
// that c^2 + s^2 = 1 to about an ulp (orthogonality of Q).
__device__ __forceinline__ void group_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int K>
__device__ bool group_sweep(float* sub, float* Q, float4* rot, int* act, float tol, float floor_abs,
                            int& rotated, int wi, int bar, bool cross) {
    constexpr int LD = J4Smem::LD;
    constexpr int NU = kB / K;                 // pairs per warp per pass
    constexpr int HB = NU > 8 ? 8 : NU;        // pairs held in registers at once
    const int lane = threadIdx.x & 31;
    const float tol2 = tol * tol;
    float fa = 0.f, fd = 0.f;
    int fp = -1, fq = 0;
    bool any_round = false;
    // all 496 pairs of the sub-problem in 31 rounds, or (cross) only the 256
    // pairs between its two index blocks in 16 rounds: pair u of round r is
    // (u, 16 + (u + r) mod 16)
    const int rounds = cross ? kB : kB2 - 1;
    for (int r = 0; r < rounds; ++r) {
        if (wi == 0) {
            if (fp >= 0) {
                sub[fp * LD + fp] = fa;
                sub[fq * LD + fq] = fd;
                sub[fp * LD + fq] = 0.f;
                sub[fq * LD + fp] = 0.f;
            }
            __syncwarp();
            if (lane < kB) {
                int p, q;
                if (cross) {
                    p = lane;
                    q = kB + ((lane + r) & (kB - 1));
                } else {
                    circle_pair(kB2, r, lane, p, q);
                }
                const float a = sub[p * LD + p], d = sub[q * LD + q], g = sub[p * LD + q];
                float c = 1.f, sn = 0.f;
                fp = -1;
                if (fabsf(g) > floor_abs && g * g > tol2 * fabsf(a * d)) {
                    // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (d - a) / (2 g),
                    // written without the division: t = sign(h g) 2|g| / (|h| + sqrt(h^2 + 4 g^2))
                    const float h = d - a;
                    const float rr = sqrtf(fmaf(h, h, 4.f * g * g));
                    float t = 2.f * fabsf(g) * __frcp_rn(fabsf(h) + rr);
                    if ((h < 0.f) != (g < 0.f)) t = -t;
                    const float x = fmaf(t, t, 1.f);
                    c = rsqrtf(x);
                    c = c * fmaf(-0.5f * x, c * c, 1.5f);
                    sn = t * c;
                    fa = a - t * g;
                    fd = d + t * g;
                    fp = p;
                    fq = q;
                    rotated = 1;
                }
                rot[lane] = make_float4(c, sn, __int_as_float(p), __int_as_float(q));
            }
            // a round without any rotation leaves sub and Q unchanged.  The
            // flag alternates between two slots by round parity: a warp still
            // reading round r's slot cannot see round r + 1's write, and
            // round r + 2 cannot start before every warp passed round r + 1's
            // barrier.
            const unsigned m = __ballot_sync(0xffffffffu, lane < kB && fp >= 0);
            if (lane == 0) act[r & 1] = m != 0u;
        }
        group_bar(bar, 32 * K);
        if (!act[r & 1]) continue;   // uniform over the group
        any_round = true;
        // two-sided update, one 2 x 2 block (rows p_u, q_u; columns p_w, q_w)
        // per thread: R_u^T S R_w, so no ordering between a row and a column
        // pass is needed; then columns p_w, q_w of Q (lane = row)
#pragma unroll
        for (int i = 0; i < 256 / (32 * K); ++i) {
            const int b = (wi + K * i) * 32 + lane;
            const int u = b >> 4, w = b & 15;
            const float4 ru = rot[u], rw = rot[w];
            const float cu = ru.x, su = ru.y, cw = rw.x, sw = rw.y;
            const int pu = __float_as_int(ru.z), qu = __float_as_int(ru.w);
            const int pw = __float_as_int(rw.z), qw = __float_as_int(rw.w);
            const float x11 = sub[pu * LD + pw], x12 = sub[pu * LD + qw];
            const float x21 = sub[qu * LD + pw], x22 = sub[qu * LD + qw];
            const float y11 = cu * x11 - su * x21, y21 = su * x11 + cu * x21;
            const float y12 = cu * x12 - su * x22, y22 = su * x12 + cu * x22;
            sub[pu * LD + pw] = cw * y11 - sw * y12;
            sub[pu * LD + qw] = sw * y11 + cw * y12;
            sub[qu * LD + pw] = cw * y21 - sw * y22;
            sub[qu * LD + qw] = sw * y21 + cw * y22;
        }
#pragma unroll
        for (int h = 0; h < NU; h += HB) {
            float cu[HB], su[HB], x[HB], y[HB];
            int pu[HB], qu[HB];
#pragma unroll
            for (int v = 0; v < HB; ++v) {
                const float4 ru = rot[wi + (h + v) * K];
                cu[v] = ru.x; su[v] = ru.y; pu[v] = __float_as_int(ru.z); qu[v] = __float_as_int(ru.w);
            }
#pragma unroll
            for (int v = 0; v < HB; ++v) { x[v] = Q[lane * LD + pu[v]]; y[v] = Q[lane * LD + qu[v]]; }
#pragma unroll
            for (int v = 0; v < HB; ++v) {
                Q[lane * LD + pu[v]] = cu[v] * x[v] - su[v] * y[v];
                Q[lane * LD + qu[v]] = su[v] * x[v] + cu[v] * y[v];
            }
        }
        group_bar(bar, 32 * K);
    }
    // (the last round's exact diagonal is not needed: the block is rebuilt
    // from the rotations by the update jobs)
    group_bar(bar, 32 * K);    // every warp has read the flags before they are reused
    return any_round;
}

// Load, solve and publish pair u with a group of K warps.
template <int K>
__device__ void solve_pair(const float* __restrict__ G, int Mp, int nb, int step, int u, float* sub,
                           float* Q, float4* rot, int* act, float tol, float floor_abs, int& rotated,
                           int wi, int bar, uint32_t* __restrict__ qbuf, int* __restrict__ ident) {
    constexpr int LD = J4Smem::LD;
    const int lane = threadIdx.x & 31;
    int bi, bj;
    circle_pair(nb, step, u, bi, bj);
    for (int i = wi; i < kB2; i += K) {
        sub[i * LD + lane] = __ldcg(G + (int64_t)gidx(bi, bj, i) * Mp + gidx(bi, bj, lane));
        Q[i * LD + lane] = i == lane ? 1.f : 0.f;
    }
    group_bar(bar, 32 * K);
    // the pairs inside each index block are taken at the sweep's first step
    // (every block takes part in it), the pairs between the two blocks at
    // every step: each pair once per sweep at least
    const bool moved = group_sweep<K>(sub, Q, rot, act, tol, floor_abs, rotated, wi, bar, step != 0);
    if (wi == 0 && (threadIdx.x & 31) == 0) ident[u] = moved ? 0 : 1;
    uint32_t* qo = qbuf + (size_t)u * 2 * kQWords;
    for (int w = wi; w < kB; w += K) {
        // row n = lane of (2^14 Q)^T: Q[2w][lane], Q[2w + 1][lane]
        uint32_t hi, lo;
        split_h2(Q[(2 * w) * LD + lane] * kQScale, Q[(2 * w + 1) * LD + lane] * kQScale, hi, lo);
        qo[lane * 16 + w] = hi;
        qo[kQWords + lane * 16 + w] = lo;
    }
    group_bar(bar, 32 * K);
}

// The 256 pairs between the two index blocks of pair u (16 rounds; round r
// pairs p < 16 with 16 + (p + r) mod 16) by one warp, the sub-problem in
// registers.  Lane j holds column j of the sub-problem S and of Q.  The rows
// of the second index block are shifted by one register after every round,
// so that the partner row of row p is always register 16 + p: the row
// rotations (R^T S) then use fixed registers, and the column rotations (S R,
// Q R) take the partner lane's column by shuffles.  Diagonal entries are
// tracked per lane (d_j) with the same update as the shared-memory solver
// (a - t g, d + t g); the same threshold decides each rotation.  No named
// barrier and no shared traffic but the round's 16 rotations (tab).
__device__ void solve_cross_warp(const float* __restrict__ G, int Mp, int nb, int step, int u,
                                 float tol, float floor_abs, int& rotated, uint32_t* __restrict__ qbuf,
                                 int* __restrict__ ident, float2* tab) {
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool lo = lane < kB;
    int bi, bj;
    circle_pair(nb, step, u, bi, bj);
    float sv[kB2], qv[kB2];
    {
        // column lane of S = row lane (S is symmetric in memory)
        const float* row = G + (int64_t)gidx(bi, bj, lane) * Mp;
#pragma unroll
        for (int i = 0; i < kB; i += 4) {
            const float4 a = __ldcg(reinterpret_cast<const float4*>(row + bi * kB + i));
            const float4 b = __ldcg(reinterpret_cast<const float4*>(row + bj * kB + i));
            sv[i] = a.x; sv[i + 1] = a.y; sv[i + 2] = a.z; sv[i + 3] = a.w;
            sv[kB + i] = b.x; sv[kB + i + 1] = b.y; sv[kB + i + 2] = b.z; sv[kB + i + 3] = b.w;
        }
    }
    float dg = __ldcg(G + (int64_t)gidx(bi, bj, lane) * Mp + gidx(bi, bj, lane));
#pragma unroll
    for (int i = 0; i < kB2; ++i) qv[i] = i == lane ? 1.f : 0.f;
    const float tol2 = tol * tol;
    bool moved = false;
#pragma unroll 1
    for (int r = 0; r < kB; ++r) {
        const int partner = lo ? kB + ((lane + r) & (kB - 1)) : ((lane - kB - r) & (kB - 1));
        // g = S[q][p] of pair p = lane: register 16 + p
        float g;
        {
            float x8[8], x4[4], x2[2];
#pragma unroll
            for (int k = 0; k < 8; ++k) x8[k] = (lane & 1) ? sv[kB + 2 * k + 1] : sv[kB + 2 * k];
#pragma unroll
            for (int k = 0; k < 4; ++k) x4[k] = (lane & 2) ? x8[2 * k + 1] : x8[2 * k];
#pragma unroll
            for (int k = 0; k < 2; ++k) x2[k] = (lane & 4) ? x4[2 * k + 1] : x4[2 * k];
            g = (lane & 8) ? x2[1] : x2[0];
        }
        const float dp = __shfl_sync(kFull, dg, partner);
        float c = 1.f, sn = 0.f, tg = 0.f;
        bool rot = false;
        if (lo && fabsf(g) > floor_abs && g * g > tol2 * fabsf(dg * dp)) {
            const float h = dp - dg;
            const float rr = sqrtf(fmaf(h, h, 4.f * g * g));
            float t = 2.f * fabsf(g) * __frcp_rn(fabsf(h) + rr);
            if ((h < 0.f) != (g < 0.f)) t = -t;
            const float x = fmaf(t, t, 1.f);
            c = rsqrtf(x);
            c = c * fmaf(-0.5f * x, c * c, 1.5f);
            sn = t * c;
            tg = t * g;
            rot = true;
        }
        if (__ballot_sync(kFull, rot) != 0u) {    // uniform over the warp
            moved = true;
            const float cx = __shfl_sync(kFull, c, partner);
            const float sx = __shfl_sync(kFull, sn, partner);
            const float tgx = __shfl_sync(kFull, tg, partner);
            // this lane's column: c col_p - s col_q (lane p) or s col_p + c col_q (lane q)
            const float cm = lo ? c : cx, sm = lo ? -sn : sx;
            dg = lo ? dg - tg : dg + tgx;
            if (lo) tab[lane] = make_float2(c, sn);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < kB; ++k) {
                const float2 cs = tab[k];
                const float x = sv[k], y = sv[kB + k];
                sv[k] = cs.x * x - cs.y * y;
                sv[kB + k] = cs.y * x + cs.x * y;
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < kB2; ++i) {
                const float o = __shfl_sync(kFull, sv[i], partner);
                sv[i] = fmaf(sm, o, cm * sv[i]);
            }
#pragma unroll
            for (int i = 0; i < kB2; ++i) {
                const float o = __shfl_sync(kFull, qv[i], partner);
                qv[i] = fmaf(sm, o, cm * qv[i]);
            }
        }
        // next round: register 16 + p takes the row that register 16 + p + 1 held
        const float s0 = sv[kB];
#pragma unroll
        for (int m = 0; m < kB - 1; ++m) sv[kB + m] = sv[kB + m + 1];
        sv[kB2 - 1] = s0;
    }
    if (moved) rotated = 1;
    if (lane == 0) ident[u] = moved ? 0 : 1;
    // row n = lane of (2^14 Q)^T: words w = (Q[2w][n], Q[2w + 1][n]), hi then lo
    uint32_t hw[kB], lw[kB];
#pragma unroll
    for (int w = 0; w < kB; ++w) split_h2(qv[2 * w] * kQScale, qv[2 * w + 1] * kQScale, hw[w], lw[w]);
    uint4* qh = reinterpret_cast<uint4*>(qbuf + (size_t)u * 2 * kQWords + lane * kB);
    uint4* ql = reinterpret_cast<uint4*>(qbuf + (size_t)u * 2 * kQWords + kQWords + lane * kB);
#pragma unroll
    for (int k = 0; k < kB / 4; ++k) {
        qh[k] = make_uint4(hw[4 * k], hw[4 * k + 1], hw[4 * k + 2], hw[4 * k + 3]);
        ql[k] = make_uint4(lw[4 * k], lw[4 * k + 1], lw[4 * k + 2], lw[4 * k + 3]);
    }
}

// Solve one FP32 matrix with csize CTAs (rank crank); qbuf holds the np
// published rotations (np x 2 x kQWords words).  kSt: update jobs stage
// their operands through shared memory (kStageBytes per warp after the
// solve area) and the shared copy of the rotations is swizzled.
template <bool kCluster, bool kSt>
__device__ void jacobi4_matrix(float* __restrict__ G, float* __restrict__ V, int Mp, int csize,
                               int crank, int max_sweeps, float tol, int32_t* __restrict__ sweeps_out,
                               uint32_t* __restrict__ qbuf, unsigned char* smem_raw) {
    constexpr int LD = J4Smem::LD;
    const int nb = Mp / kB, np = nb / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = csize * kW4, gwarp = crank * kW4 + warp;
    __shared__ int rot_flag;
    __shared__ int decision;
    __shared__ float scale_sh, dmax_sh;

    // scale: the Gershgorin bound max_i sum_j |G_ij| >= lambda_max, which
    // bounds every entry the solve will produce, into [2^12, 2^13); the
    // largest diagonal sets the rotation floor
    __shared__ unsigned int rowsum_bits;
    if (threadIdx.x == 0) rowsum_bits = 0u;
    __syncthreads();
    {
        float rmax = 0.f;
        for (int i = warp; i < Mp; i += kW4) {
            float acc = 0.f;
            for (int j = lane; j < Mp; j += 32) acc += fabsf(__ldcg(G + (int64_t)i * Mp + j));
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            rmax = fmaxf(rmax, acc);
        }
        if (lane == 0) atomicMax(&rowsum_bits, __float_as_uint(rmax));
    }
    __syncthreads();
    if (warp == 0) {
        float dmax = 0.f;
        for (int i = lane; i < Mp; i += 32) dmax = fmaxf(dmax, fabsf(__ldcg(G + (int64_t)i * Mp + i)));
        for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        if (lane == 0) {
            const float bound = __uint_as_float(rowsum_bits);
            int e = 0;
            if (bound > 0.f) frexpf(bound, &e);        // bound in [2^(e-1), 2^e)
            scale_sh = bound > 0.f ? ldexpf(1.f, 13 - e) : 1.f;
            dmax_sh = dmax * scale_sh;
            rot_flag = 0;
        }
    }
    __syncthreads();
    const float sc = scale_sh;
    // absolute floor of the rotation threshold (see the FP64 solver): half the
    // relative threshold, times the largest diagonal (4 eps at the default)
    const float floor_abs = 0.5f * tol * dmax_sh;
    owner_sync<kCluster>();
    for (int64_t e = (int64_t)crank * kJT4 + threadIdx.x; e < (int64_t)Mp * Mp;
         e += (int64_t)csize * kJT4) {
        const int i = (int)(e / Mp), j = (int)(e % Mp);
        V[e] = i == j ? 1.f : 0.f;
        G[e] = __ldcg(G + e) * sc;
    }
    owner_sync<kCluster>();

    // groups of kgrp warps share one pair solve (kgrp * pairs of this CTA <= 8)
    const int nmine = (np - crank + csize - 1) / csize;
    const int kgrp = nmine >= kW4 ? 1 : nmine >= 4 ? 2 : nmine >= 2 ? 4 : 8;
    const int ngroups = kW4 / kgrp, grp = warp / kgrp, wi = warp % kgrp;
    int* ident = reinterpret_cast<int*>(qbuf + (size_t)np * 2 * kQWords);   // np flags
    const bool qsmem = ((size_t)np * 2 * kQWords + np) * sizeof(uint32_t) <= J4Smem::solve_bytes;
    const int nblk = np * (np + 1) / 2;
    const int rtiles = Mp / kB2;
    const int njobs = nblk + np * rtiles;
    // The single-matrix form (a few update jobs per warp) takes its jobs
    // longest first: block jobs (two products) go round robin, then each
    // warp takes a run of column jobs (one product) that brings it to
    // ceil(products / warps); round robin over all jobs would leave the warps
    // with an extra block job two products above the rest, and every step
    // waits for the slowest.  The staged form (a dozen jobs per warp) keeps
    // round robin over all jobs, which measured faster there.
    int nbw = 0, vstart = 0, nseq = 0;
    if constexpr (!kSt) {
        const int nvj = njobs - nblk;
        const int qb = nblk / nwarps, rb = nblk % nwarps;
        nbw = qb + (gwarp < rb ? 1 : 0);
        const int cap = (2 * nblk + nvj + nwarps - 1) / nwarps;
        for (int x = 0; x < gwarp; ++x) vstart += max(0, cap - 2 * (qb + (x < rb ? 1 : 0)));
        nseq = nbw + max(0, min(cap - 2 * nbw, nvj - vstart));
    }
    int sweep = 0;
    bool converged = false;
    while (sweep < max_sweeps) {
        int rotated = 0;
        for (int step = 0; step < nb - 1; ++step) {
            // pair solves: the CTA's pairs u = crank + t csize go to groups of
            // kgrp warps; each group publishes (2^14 Q)^T (hi, lo) of its pairs
            // steps after the first: with at least 4 pairs per CTA, one warp
            // per pair in registers; otherwise (and at the first step, which
            // also takes the pairs inside each index block) groups of kgrp
            // warps in shared memory
            const bool by_warp = step != 0 && (!kSt || kgrp <= 2);
            if (by_warp) {
                float2* tab = reinterpret_cast<float2*>(smem_raw + J4Smem::per_warp * warp);
                for (int t = warp; t < nmine; t += kW4)
                    solve_cross_warp(G, Mp, nb, step, crank + t * csize, tol, floor_abs, rotated, qbuf, ident, tab);
            }
            for (int t = grp; t < nmine && !by_warp; t += ngroups) {
                const int u = crank + t * csize;
                float* gsub = reinterpret_cast<float*>(smem_raw + J4Smem::per_warp * grp);
                float* gQ = gsub + kB2 * LD;
                float4* grot = reinterpret_cast<float4*>(gQ + kB2 * LD);
                int* gact = reinterpret_cast<int*>(grot + kB);
                switch (kgrp) {
                    case 1: solve_pair<1>(G, Mp, nb, step, u, gsub, gQ, grot, gact, tol, floor_abs, rotated, wi, 1 + grp, qbuf, ident); break;
                    case 2: solve_pair<2>(G, Mp, nb, step, u, gsub, gQ, grot, gact, tol, floor_abs, rotated, wi, 1 + grp, qbuf, ident); break;
                    case 4: solve_pair<4>(G, Mp, nb, step, u, gsub, gQ, grot, gact, tol, floor_abs, rotated, wi, 1 + grp, qbuf, ident); break;
                    default: solve_pair<8>(G, Mp, nb, step, u, gsub, gQ, grot, gact, tol, floor_abs, rotated, wi, 1 + grp, qbuf, ident); break;
                }
            }
            owner_sync<kCluster>();
            // the step's rotations and identity flags into this CTA's shared
            // memory (the solve area is free now) when they fit
            const uint32_t* qsrc = qbuf;
            const int* isrc = ident;
            if (qsmem) {
                uint32_t* qs = reinterpret_cast<uint32_t*>(smem_raw);
                const int nw = np * 2 * kQWords;
                for (int w = threadIdx.x; w < nw / 4; w += kJT4)
                    reinterpret_cast<uint4*>(qs)[kSt ? w ^ ((w >> 3) & 3) : w] =
                        __ldcg(reinterpret_cast<const uint4*>(qbuf) + w);
                for (int w = threadIdx.x; w < np; w += kJT4) qs[nw + w] = (uint32_t)__ldcg(ident + w);
                __syncthreads();
                qsrc = qs;
                isrc = reinterpret_cast<const int*>(qs + nw);
            }
            auto ident_of = [&](int u) { return qsmem ? isrc[u] != 0 : __ldcg(ident + u) != 0; };
            // job j: block (u, w2) of the upper triangle when j < nblk, else
            // the column tile at rows r0 of P_u
            auto decode = [&](int j, int& u, int& w2, int& r0) {
                if (j < nblk) {
                    int r = j;
                    u = 0;
                    while (r >= np - u) { r -= np - u; ++u; }
                    w2 = u + r;
                    r0 = 0;
                    return true;
                }
                const int r = j - nblk;
                u = r / rtiles;
                w2 = u;
                r0 = (r % rtiles) * kB2;
                return false;
            };
            // a block whose two rotations are the identity (or a tile whose
            // one is) does not change
            auto skip = [&](int j) {
                int u, w2, r0;
                const bool blk = decode(j, u, w2, r0);
                return ident_of(u) && (!blk || ident_of(w2));
            };
            auto run_job = [&](bool blk, int u, int w2, int r0, const float2 (&op)[16]) {
                int ui, uj;
                circle_pair(nb, step, u, ui, uj);
                const uint32_t* qu = qsrc + (size_t)u * 2 * kQWords;
                if (blk) {
                    int wi2, wj;
                    circle_pair(nb, step, w2, wi2, wj);
                    const uint32_t* qw = qsrc + (size_t)w2 * 2 * kQWords;
                    if (qsmem) job_block<true, kSt>(G, Mp, qu, qw, ui, uj, wi2, wj, op);
                    else job_block<false, kSt>(G, Mp, qu, qw, ui, uj, wi2, wj, op);
                } else {
                    if (qsmem) job_vcols<true, kSt>(V, Mp, qu, ui, uj, r0, op);
                    else job_vcols<false, kSt>(V, Mp, qu, ui, uj, r0, op);
                }
            };
            if constexpr (kSt) {
                // the copy of job j + 1's operand runs while job j computes
                float* stg = reinterpret_cast<float*>(smem_raw + J4Smem::solve_bytes + (size_t)warp * kStageBytes);
                auto issue = [&](int j) {
                    int u, w2, r0;
                    const bool blk = decode(j, u, w2, r0);
                    int ui, uj, wi2 = 0, wj = 0;
                    circle_pair(nb, step, u, ui, uj);
                    if (blk) circle_pair(nb, step, w2, wi2, wj);
                    stage_rows(stg, blk ? G : V, Mp, ui, uj, blk, wi2, wj, r0);
                };
                auto next_job = [&](int j) {
                    while (j < njobs && skip(j)) j += nwarps;
                    return j;
                };
                int j = next_job(gwarp);
                if (j < njobs) issue(j);
                while (j < njobs) {
                    const int jn = next_job(j + nwarps);
                    float2 op[16];
                    cp_async_wait_all();
                    __syncwarp();
                    if (j < nblk) frag_block(stg, op);
                    else frag_vcols(stg, op);
                    __syncwarp();
                    if (jn < njobs) issue(jn);
                    int u, w2, r0;
                    const bool blk = decode(j, u, w2, r0);
                    run_job(blk, u, w2, r0, op);
                    j = jn;
                }
            } else {
                const float2 none[16] = {};
                for (int t = 0; t < nseq; ++t) {
                    int u, w2, r0;
                    const bool blk = decode(t < nbw ? gwarp + t * nwarps : nblk + vstart + (t - nbw), u, w2, r0);
                    if (ident_of(u) && (!blk || ident_of(w2))) continue;
                    run_job(blk, u, w2, r0, none);
                }
            }
            // (the next step's solves overwrite the shared copy: every warp of
            // this CTA has finished its jobs at the barrier below)
            owner_sync<kCluster>();
        }
        ++sweep;
        if (__syncthreads_or(rotated) && threadIdx.x == 0) rot_flag = 1;
        __syncthreads();
        int any;
        if constexpr (kCluster) {
            cg::cluster_group cluster = cg::this_cluster();
            if (crank == 0 && threadIdx.x == 0) {
                int acc = 0;
                for (int r = 0; r < csize; ++r) acc |= *cluster.map_shared_rank(&rot_flag, r);
                decision = acc;
            }
            cluster.sync();
            any = *cluster.map_shared_rank(&decision, 0);
            cluster.sync();
        } else {
            any = rot_flag;
            __syncthreads();
        }
        if (threadIdx.x == 0) rot_flag = 0;
        __syncthreads();
        if (!any) { converged = true; break; }
    }
    // unscale G; V^T into place as Vt (each unordered pair swapped once).
    // Other CTAs wrote G and V: every load here goes through L2.
    const float inv = 1.f / sc;
    for (int64_t e = (int64_t)crank * kJT4 + threadIdx.x; e < (int64_t)Mp * Mp;
         e += (int64_t)csize * kJT4) {
        G[e] = __ldcg(G + e) * inv;
        const int i = (int)(e / Mp), j = (int)(e % Mp);
        if (i < j) {
            const float a = __ldcg(V + e), b = __ldcg(V + (int64_t)j * Mp + i);
            V[e] = b;
            V[(int64_t)j * Mp + i] = a;
        }
    }
    if (crank == 0 && threadIdx.x == 0) *sweeps_out = converged ? sweep : -sweep;
}

template <bool kSt>
__global__ void __launch_bounds__(kJT4, 2)
k_jacobi4(float* __restrict__ Gall, float* __restrict__ Vall, int Mp, int csize, int max_sweeps,
          float tol, int32_t* __restrict__ sweeps_out, uint32_t* __restrict__ qall) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int crank = (int)cg::this_cluster().block_rank();
    const int mat = blockIdx.x / csize;
    jacobi4_matrix<true, kSt>(Gall + (int64_t)mat * Mp * Mp, Vall + (int64_t)mat * Mp * Mp, Mp, csize,
                         crank, max_sweeps, tol, sweeps_out + mat,
                         qall + (size_t)mat * jwork_words(Mp), smem_raw);
}

__global__ void __launch_bounds__(kJT4, 2)
k_jacobi4_items(const JacobiItem* __restrict__ items, int nitems, int* __restrict__ next,
                int max_sweeps, float tol) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int item_sh;
    for (;;) {
        if (threadIdx.x == 0) item_sh = atomicAdd(next, 1);
        __syncthreads();
        const int it = item_sh;
        __syncthreads();
        if (it >= nitems) break;
        const JacobiItem w = items[it];
        jacobi4_matrix<false, true>(static_cast<float*>(w.G), static_cast<float*>(w.Vt), w.Mp, 1, 0,
                              w.max_sweeps > 0 ? w.max_sweeps : max_sweeps, tol, w.sweeps,
                              static_cast<uint32_t*>(w.work), smem_raw);
        __syncthreads();
    }
}

// Cluster size of the FP32 solver: a step costs one pair solve (kSolve4 job
// units) plus the jobs of one warp; clusters run in waves of the hardware's
// maximum active clusters.
constexpr int kSolve4 = 4;

// The FP32 solver for several matrices stages its job operands (the copies
// hide L2 latency over many jobs per warp); a single matrix (the merge) has
// a few jobs per warp and runs the direct form.
using Jacobi4Kernel = void (*)(float*, float*, int, int, int, float, int32_t*, uint32_t*);
Jacobi4Kernel jacobi4_kernel(bool staged) { return staged ? k_jacobi4<true> : k_jacobi4<false>; }

// Clusters of cs CTAs of the FP32 solver that can be resident at once (0 if
// none can).
int active_clusters4(int cs, bool staged) {
    const Jacobi4Kernel kern = jacobi4_kernel(staged);
    const size_t smem = J4Smem::bytes(staged);
    if (cs > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs, 1, 1);
    cfg.blockDim = dim3(kJT4, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nclusters;
}

int pick_cluster4(int nmat, int Mp, bool staged) {
    const int np = Mp / kB2;
    const int64_t jobs = (int64_t)np * (np + 1) / 2 + (int64_t)np * (Mp / kB2);
    int best = -1;
    double best_cost = 1e300;
    for (int cs = 1; cs <= kMaxCluster; cs *= 2) {
        const int nclusters = active_clusters4(cs, staged);
        if (nclusters < 1) continue;
        const int nw = cs * kW4;
        const double solves = (double)((np + nw - 1) / nw);
        const double per_warp = (double)(jobs + nw - 1) / nw;
        const int64_t waves = (nmat + nclusters - 1) / nclusters;
        const double cost = (double)waves * (kSolve4 * solves + per_warp);
        if (cost <= best_cost) { best_cost = cost; best = cs; }
    }
    return best;
}

// Cluster size for nmat matrices with npairs block pairs per step.  A CTA
// owns ppc = ceil(npairs / csize) pairs; its step costs about one warp sweep
// (the pairs' warps run in parallel) plus ppc pairs of panel products, so a
// matrix takes ~ (kInner + ppc).  Clusters run in waves of the hardware's
// maximum active clusters of that size.  Minimise waves * (kInner + ppc);
// ties go to the larger cluster (lower latency per matrix).
constexpr int kInner = 2;

template <typename T>
int pick_cluster(int nmat, int npairs) {
    auto kern = k_jacobi<T>;
    int best = -1;
    int64_t best_cost = INT64_MAX;
    for (int cs = 1; cs <= kMaxCluster && cs <= npairs; cs *= 2) {
        const int ppc = (npairs + cs - 1) / cs;
        if (ppc > PairsMax<T>::value) continue;
        const size_t smem = JSmem<T>::bytes(ppc);
        if (cs > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                          cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)cs, 1, 1);
        cfg.blockDim = dim3(kJT, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
            cudaGetLastError();
            continue;
        }
        const int64_t waves = (nmat + nclusters - 1) / nclusters;
        const int64_t cost = waves * (kInner + ppc);
        if (cost <= best_cost) { best_cost = cost; best = cs; }
    }
    return best;
}

}  // namespace

int jacobi_pad(int M) { return (int)round_up(M, kB2); }

int jacobi_item_max_mp(bool fp64) { return fp64 ? kB2 * PairsMax<double>::value : kMaxM; }

size_t jacobi_work_bytes(int nmat, int Mp) {
    return (size_t)std::max(nmat, 0) * jwork_words(Mp) * sizeof(uint32_t);
}

template <typename T>
cudaError_t launch_jacobi(T* G, T* Vt, int nmat, int Mp, int max_sweeps, double tol,
                          int32_t* sweeps, cudaStream_t s, void* work, int cluster) {
    if (nmat <= 0) return cudaSuccess;
    if (Mp % kB2 != 0) return cudaErrorInvalidValue;
    const int npairs = Mp / kB2;
    if constexpr (sizeof(T) == 4) {
        if (!work) return cudaErrorInvalidValue;
        // a requested cluster size (1, 2, 4, 8 or 16) that cannot be launched
        // falls back to the occupancy model's choice
        const bool staged = nmat > 1;
        const Jacobi4Kernel kern = jacobi4_kernel(staged);
        int csize = -1;
        if (cluster >= 1 && cluster <= kMaxCluster && (cluster & (cluster - 1)) == 0 &&
            active_clusters4(cluster, staged) >= 1)
            csize = cluster;
        if (csize < 1) csize = pick_cluster4(nmat, Mp, staged);
        if (csize < 1) return cudaErrorInvalidConfiguration;
        if (csize > 8)
            RK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        RK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)J4Smem::bytes(staged)));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nmat * csize), 1, 1);
        cfg.blockDim = dim3(kJT4, 1, 1);
        cfg.dynamicSmemBytes = J4Smem::bytes(staged);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)csize;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kern, (float*)G, (float*)Vt, Mp, csize, max_sweeps,
                                  (float)tol, sweeps, static_cast<uint32_t*>(work));
    } else {
        const int csize = pick_cluster<T>(nmat, npairs);
        if (csize < 1) return cudaErrorInvalidConfiguration;
        const int ppc = (npairs + csize - 1) / csize;
        const size_t smem = JSmem<T>::bytes(ppc);
        auto kern = k_jacobi<T>;
        if (csize > 8)
            RK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        RK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nmat * csize), 1, 1);
        cfg.blockDim = dim3(kJT, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)csize;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kern, G, Vt, Mp, csize, ppc, max_sweeps, (T)tol, sweeps);
    }
}

template <typename T>
cudaError_t launch_jacobi_items(const JacobiItem* items, int nitems, int max_mp, int* next,
                                int max_sweeps, double tol, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    int dev = 0, sms = 0, per_sm = 0;
    RK_CUDA_TRY(cudaGetDevice(&dev));
    RK_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if constexpr (sizeof(T) == 4) {
        if (max_mp % kB2 != 0 || max_mp < kB2 || max_mp > kMaxM) return cudaErrorInvalidValue;
        RK_CUDA_TRY(cudaFuncSetAttribute(k_jacobi4_items, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)J4Smem::bytes(true)));
        RK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi4_items, kJT4,
                                                                  J4Smem::bytes(true)));
        const int grid = std::max(1, std::min(nitems, sms * std::max(per_sm, 1)));
        RK_CUDA_TRY(cudaMemsetAsync(next, 0, sizeof(int), s));
        k_jacobi4_items<<<grid, kJT4, J4Smem::bytes(true), s>>>(items, nitems, next, max_sweeps, (float)tol);
        return cudaGetLastError();
    } else {
        const int ppc = max_mp / kB2;
        if (max_mp % kB2 != 0 || ppc < 1 || ppc > PairsMax<T>::value) return cudaErrorInvalidValue;
        const size_t smem = JSmem<T>::bytes(ppc);
        auto kern = k_jacobi_items<T>;
        RK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kJT, smem));
        const int grid = std::max(1, std::min(nitems, sms * std::max(per_sm, 1)));
        RK_CUDA_TRY(cudaMemsetAsync(next, 0, sizeof(int), s));
        k_jacobi_items<T><<<grid, kJT, smem, s>>>(items, nitems, next, max_sweeps, (T)tol);
        return cudaGetLastError();
    }
}

template cudaError_t launch_jacobi<float>(float*, float*, int, int, int, double, int32_t*,
                                          cudaStream_t, void*, int);
template cudaError_t launch_jacobi<double>(double*, double*, int, int, int, double, int32_t*,
                                           cudaStream_t, void*, int);
template cudaError_t launch_jacobi_items<float>(const JacobiItem*, int, int, int*, int, double,
                                                cudaStream_t);
template cudaError_t launch_jacobi_items<double>(const JacobiItem*, int, int, int*, int, double,
                                                 cudaStream_t);

}  // namespace rk
