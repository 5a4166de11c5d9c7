// jacobi.cu -- batched block two-sided Jacobi eigensolver for the symmetric
// positive semi-definite cross products of Ranky's block SVD (arXiv
// 2009.09767, Eq. 1: A^i = U^i S^i V^i*, whose U^i and (S^i)^2 are the
// eigenvectors and eigenvalues of A^i A^i^T).
//
// Design (one thread-block cluster per matrix):
//   * The index set 0..Mp-1 is cut into nb = Mp/b blocks of b = B2/2 indices.
//     A round-robin (circle) schedule pairs the blocks; each of the nb-1
//     steps of a sweep handles nb/2 disjoint block pairs in parallel.
//   * For its pair (I, J) a CTA loads the B2 x B2 sub-matrix G[I+J, I+J] into
//     shared memory and runs one cyclic Jacobi sweep on it (again a circle
//     schedule: b disjoint rotations per round, each 2x2 block of the
//     sub-matrix updated from both sides by one thread), accumulating the
//     B2 x B2 orthogonal Q.
//   * Phase A: rows I+J of G and of Vt are replaced by Q^T times themselves
//     (panel products streamed through shared memory).  Cluster barrier.
//     Phase B: columns I+J of G by themselves times Q.  Cluster barrier.
//   * A sweep in which no rotation passed the threshold ends the solve.
// G and Vt stay in global memory (L2-resident at these sizes) and are read
// with L2-only loads, because other CTAs of the cluster write them between
// barriers.  Padding indices (M..Mp-1) hold zero rows/columns: they never
// rotate, so their eigenvectors stay exact unit vectors.
#include <cooperative_groups.h>

#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace rk {

namespace {

constexpr int kJT = 512;   // threads per CTA (16 warps)
constexpr int kMaxCluster = 8;

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
__device__ __forceinline__ float rsqrt_t<float>(float x) { return 1.0f / sqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

// 16-byte vectors of T
template <typename T> struct V16;
template <> struct V16<float> {
    using type = float4;
    static constexpr int n = 4;
    __device__ static float get(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
};
template <> struct V16<double> {
    using type = double2;
    static constexpr int n = 2;
    __device__ static double get(const double2& v, int i) { return i == 0 ? v.x : v.y; }
};

// Load four consecutive T from 16-byte aligned shared memory.
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

template <typename T, int B2>
struct JacobiSmem {
    static constexpr int b = B2 / 2;
    static constexpr int PAD = 16 / (int)sizeof(T);  // keeps rows 16-byte aligned
    static constexpr int LD = B2 + 1;               // sub-problem stride (odd)
    static constexpr int QLD = B2 + PAD;            // Q stride (aligned rows)
    static constexpr int TW = 8192 / B2;            // row-panel tile width
    static constexpr int RSLD = TW + PAD;           // row-panel stage stride
    static constexpr int TR = 8192 / B2;            // column-panel tile height
    static constexpr int CSLD = B2 + 1;             // column-panel stage stride
    static constexpr int STAGE = (B2 * RSLD > TR * CSLD) ? B2 * RSLD : TR * CSLD;
    static size_t bytes(int ppc) {
        return sizeof(T) * ((size_t)B2 * LD + (size_t)ppc * B2 * QLD + (size_t)STAGE) +
               sizeof(T) * 3 * b + sizeof(int) * 2 * b;
    }
};

// One cyclic sweep (B2-1 rounds) on the shared sub-matrix, accumulating Q.
// Per round: b threads compute the b disjoint rotations into a table; then
// every 2x2 block (pair u rows, pair v columns) is updated from both sides by
// one thread, and the Q columns of each pair by (row, pair) threads.
template <typename T, int B2>
__device__ void inner_sweep(T* sub, T* Q, T* cs, T* sn, T* tn, int* pp, int* qq, T tol, T floor_abs,
                            int* rotated) {
    using S = JacobiSmem<T, B2>;
    constexpr int LD = S::LD, QLD = S::QLD, b = S::b;
    for (int r = 0; r < B2 - 1; ++r) {
        if (threadIdx.x < b) {
            const int u = threadIdx.x;
            int p, q;
            circle_pair(B2, r, u, p, q);
            const T a = sub[p * LD + p], d = sub[q * LD + q], g = sub[p * LD + q];
            T c = T(1), s = T(0), t = T(0);
            const T ag = g < T(0) ? -g : g;
            const T rel = tol * sqrt(fabs(a) * fabs(d));
            if (ag > rel && ag > floor_abs) {
                const T zeta = (d - a) / (T(2) * g);
                const T az = zeta < T(0) ? -zeta : zeta;
                t = (zeta >= T(0) ? T(1) : T(-1)) / (az + sqrt(T(1) + zeta * zeta));
                c = rsqrt_t<T>(T(1) + t * t);
                s = t * c;
                *rotated = 1;
            }
            cs[u] = c; sn[u] = s; tn[u] = t; pp[u] = p; qq[u] = q;
        }
        __syncthreads();
        for (int it = threadIdx.x; it < b * b; it += kJT) {
            const int u = it / b, v = it % b;
            const int pu = pp[u], qu = qq[u], pv = pp[v], qv = qq[v];
            const T cu = cs[u], su = sn[u], cv = cs[v], sv = sn[v];
            if (u == v) {
                if (su != T(0)) {
                    const T g = sub[pu * LD + qu];
                    const T t = tn[u];
                    sub[pu * LD + pu] = sub[pu * LD + pu] - t * g;
                    sub[qu * LD + qu] = sub[qu * LD + qu] + t * g;
                    sub[pu * LD + qu] = T(0);
                    sub[qu * LD + pu] = T(0);
                }
                continue;
            }
            if (su == T(0) && sv == T(0)) continue;
            const T x00 = sub[pu * LD + pv], x01 = sub[pu * LD + qv];
            const T x10 = sub[qu * LD + pv], x11 = sub[qu * LD + qv];
            const T y00 = cu * x00 - su * x10, y01 = cu * x01 - su * x11;
            const T y10 = su * x00 + cu * x10, y11 = su * x01 + cu * x11;
            sub[pu * LD + pv] = cv * y00 - sv * y01;
            sub[pu * LD + qv] = sv * y00 + cv * y01;
            sub[qu * LD + pv] = cv * y10 - sv * y11;
            sub[qu * LD + qv] = sv * y10 + cv * y11;
        }
        // Q <- Q R on columns p, q; pair index fastest so a warp touches one row
        for (int it = threadIdx.x; it < b * B2; it += kJT) {
            const int u = it % b, row = it / b;
            const T s = sn[u];
            if (s == T(0)) continue;
            const T c = cs[u];
            const int p = pp[u], q = qq[u];
            const T x = Q[row * QLD + p], y = Q[row * QLD + q];
            Q[row * QLD + p] = c * x - s * y;
            Q[row * QLD + q] = s * x + c * y;
        }
        __syncthreads();
    }
}

// Global index of local sub-problem index k (0..B2-1) for block pair (bi, bj).
template <int B2>
__device__ __forceinline__ int gidx(int bi, int bj, int k) {
    constexpr int b = B2 / 2;
    return k < b ? bi * b + k : bj * b + (k - b);
}

// rows idx(0..B2-1) of Mat (ld = Mp) <- Q^T * rows, over all Mp columns.
// Tile: B2 rows x TW columns staged in shared memory; each thread computes a
// 4 x 4 block of outputs with 16-byte shared loads.
template <typename T, int B2>
__device__ void panel_rows(T* Mat, int Mp, int bi, int bj, const T* Q, T* stage) {
    using S = JacobiSmem<T, B2>;
    constexpr int QLD = S::QLD, TW = S::TW, SLD = S::RSLD;
    constexpr int VN = V16<T>::n;
    using VT = typename V16<T>::type;
    constexpr int CG = TW / 4;
    const int ti = threadIdx.x / CG, tc = threadIdx.x % CG;
    const int i0 = ti * 4, j0 = tc * 4;
    for (int c0 = 0; c0 < Mp; c0 += TW) {
        const int cw = min(TW, Mp - c0);   // multiple of 32 (Mp is)
        for (int it = threadIdx.x; it < B2 * (TW / VN); it += kJT) {
            const int k = it / (TW / VN), c = (it % (TW / VN)) * VN;
            VT v;
            if (c < cw) v = __ldcg(reinterpret_cast<const VT*>(Mat + (int64_t)gidx<B2>(bi, bj, k) * Mp + c0 + c));
            else v = VT{};
            *reinterpret_cast<VT*>(stage + k * SLD + c) = v;
        }
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
#pragma unroll 8
        for (int k = 0; k < B2; ++k) {
            T qv[4], xv[4];
            lds4<T>(Q + k * QLD + i0, qv);
            lds4<T>(stage + k * SLD + j0, xv);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(qv[i], xv[j], acc[i][j]);
        }
        if (j0 < cw) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                T* dst = Mat + (int64_t)gidx<B2>(bi, bj, i0 + i) * Mp + c0 + j0;
                if constexpr (sizeof(T) == 4) {
                    *reinterpret_cast<float4*>(dst) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                } else {
                    reinterpret_cast<double2*>(dst)[0] = make_double2(acc[i][0], acc[i][1]);
                    reinterpret_cast<double2*>(dst)[1] = make_double2(acc[i][2], acc[i][3]);
                }
            }
        }
        __syncthreads();
    }
}

// columns idx(0..B2-1) of Mat <- columns * Q, over all Mp rows.
template <typename T, int B2>
__device__ void panel_cols(T* Mat, int Mp, int bi, int bj, const T* Q, T* stage) {
    using S = JacobiSmem<T, B2>;
    constexpr int QLD = S::QLD, TR = S::TR, SLD = S::CSLD;
    constexpr int VN = V16<T>::n;
    using VT = typename V16<T>::type;
    constexpr int JG = B2 / 4;
    const int tr = threadIdx.x / JG, tj = threadIdx.x % JG;
    const int i0 = tr * 4, j0 = tj * 4;
    for (int r0 = 0; r0 < Mp; r0 += TR) {
        const int rh = min(TR, Mp - r0);
        for (int it = threadIdx.x; it < TR * (B2 / VN); it += kJT) {
            const int r = it / (B2 / VN), k = (it % (B2 / VN)) * VN;
            if (r < rh) {
                const VT v = __ldcg(reinterpret_cast<const VT*>(Mat + (int64_t)(r0 + r) * Mp + gidx<B2>(bi, bj, k)));
#pragma unroll
                for (int e = 0; e < VN; ++e) stage[r * SLD + k + e] = V16<T>::get(v, e);
            } else {
#pragma unroll
                for (int e = 0; e < VN; ++e) stage[r * SLD + k + e] = T(0);
            }
        }
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
#pragma unroll 8
        for (int k = 0; k < B2; ++k) {
            T xv[4], qv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) xv[i] = stage[(i0 + i) * SLD + k];
            lds4<T>(Q + k * QLD + j0, qv);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(xv[i], qv[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i0 + i >= rh) continue;
            T* dst = Mat + (int64_t)(r0 + i0 + i) * Mp + gidx<B2>(bi, bj, j0);
            if constexpr (sizeof(T) == 4) {
                *reinterpret_cast<float4*>(dst) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            } else {
                reinterpret_cast<double2*>(dst)[0] = make_double2(acc[i][0], acc[i][1]);
                reinterpret_cast<double2*>(dst)[1] = make_double2(acc[i][2], acc[i][3]);
            }
        }
        __syncthreads();
    }
}

template <typename T, int B2>
__global__ void __launch_bounds__(kJT, 1)
k_jacobi(T* __restrict__ Gall, T* __restrict__ Vtall, int Mp, int csize, int ppc, int max_sweeps,
         T tol, int32_t* __restrict__ sweeps_out) {
    using SM = JacobiSmem<T, B2>;
    constexpr int LD = SM::LD, QLD = SM::QLD;
    constexpr int b = B2 / 2;
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = (int)cluster.block_rank();
    const int mat = blockIdx.x / csize;
    T* G = Gall + (int64_t)mat * Mp * Mp;
    T* Vt = Vtall + (int64_t)mat * Mp * Mp;
    const int nb = Mp / b;
    const int npairs = nb / 2;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* stage = reinterpret_cast<T*>(smem_raw);        // 16-byte aligned
    T* Qs = stage + SM::STAGE;                            // STAGE, QLD keep alignment
    T* sub = Qs + (size_t)ppc * B2 * QLD;
    T* cs = sub + (size_t)B2 * LD;
    T* sn = cs + b;
    T* tn = sn + b;
    int* pp = reinterpret_cast<int*>(tn + b);
    int* qq = pp + b;
    __shared__ int rot_flag;
    __shared__ int decision;
    __shared__ T floor_sh;

    // Vt = I for this CTA's share of rows
    for (int64_t e = (int64_t)crank * kJT + threadIdx.x; e < (int64_t)Mp * Mp;
         e += (int64_t)csize * kJT) {
        const int i = (int)(e / Mp), j = (int)(e % Mp);
        Vt[e] = i == j ? T(1) : T(0);
    }
    // Absolute floor of the rotation threshold: rounding leaves off-diagonal
    // noise of order eps * max|G_ij| <= eps * max_i G_ii in a positive
    // semi-definite matrix, which no rotation can remove.
    if (threadIdx.x < 32) {
        T dmax = T(0);
        for (int i = threadIdx.x; i < Mp; i += 32) dmax = fmax(dmax, fabs(ldcg(G + (int64_t)i * Mp + i)));
        for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        if (threadIdx.x == 0) {
            floor_sh = T(4) * T(Eps<T>::value) * dmax;
            rot_flag = 0;
        }
    }
    cluster.sync();
    const T floor_abs = floor_sh;

    int sweep = 0;
    bool converged = false;
    while (sweep < max_sweeps) {
        for (int step = 0; step < nb - 1; ++step) {
            // phase A: solve sub-problems, update rows of G and Vt
            for (int t = 0; t < ppc; ++t) {
                const int u = crank + t * csize;
                if (u >= npairs) break;
                int bi, bj;
                circle_pair(nb, step, u, bi, bj);
                T* Q = Qs + (size_t)t * B2 * QLD;
                for (int it = threadIdx.x; it < B2 * B2; it += kJT) {
                    const int i = it / B2, j = it % B2;
                    sub[i * LD + j] = ldcg(G + (int64_t)gidx<B2>(bi, bj, i) * Mp + gidx<B2>(bi, bj, j));
                    Q[i * QLD + j] = i == j ? T(1) : T(0);
                }
                __syncthreads();
                inner_sweep<T, B2>(sub, Q, cs, sn, tn, pp, qq, tol, floor_abs, &rot_flag);
                panel_rows<T, B2>(G, Mp, bi, bj, Q, stage);
                panel_rows<T, B2>(Vt, Mp, bi, bj, Q, stage);
            }
            cluster.sync();
            // phase B: columns of G
            for (int t = 0; t < ppc; ++t) {
                const int u = crank + t * csize;
                if (u >= npairs) break;
                int bi, bj;
                circle_pair(nb, step, u, bi, bj);
                panel_cols<T, B2>(G, Mp, bi, bj, Qs + (size_t)t * B2 * QLD, stage);
            }
            cluster.sync();
        }
        ++sweep;
        // cluster-wide OR of the rotation flags
        if (crank == 0 && threadIdx.x == 0) {
            int any = 0;
            for (int r = 0; r < csize; ++r) any |= *cluster.map_shared_rank(&rot_flag, r);
            decision = any;
        }
        cluster.sync();
        const int any = *cluster.map_shared_rank(&decision, 0);
        cluster.sync();
        if (threadIdx.x == 0) rot_flag = 0;
        __syncthreads();
        if (!any) { converged = true; break; }
    }
    if (crank == 0 && threadIdx.x == 0) sweeps_out[mat] = converged ? sweep : -sweep;
}

// Cluster size for nmat matrices with npairs block pairs per step.  A CTA
// handles ppc = ceil(npairs / csize) pairs per step, so a matrix takes time
// ~ ppc; clusters run in waves of the hardware's maximum active clusters for
// that size.  Choose the size with the fewest waves * ppc (ties: the larger
// cluster, lower latency per matrix).
template <typename T, int B2>
int pick_cluster(int nmat, int npairs) {
    auto kern = k_jacobi<T, B2>;
    int best = 1;
    int64_t best_cost = INT64_MAX;
    for (int cs = 1; cs <= kMaxCluster && cs <= npairs; cs *= 2) {
        const int ppc = (npairs + cs - 1) / cs;
        const size_t smem = JacobiSmem<T, B2>::bytes(ppc);
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
        const int64_t cost = waves * ppc;
        if (cost <= best_cost) { best_cost = cost; best = cs; }
    }
    return best;
}

template <typename T, int B2>
cudaError_t launch_jacobi_b2(T* G, T* Vt, int nmat, int Mp, int max_sweeps, double tol,
                             int32_t* sweeps, cudaStream_t s) {
    const int b = B2 / 2;
    const int nb = Mp / b;
    const int npairs = nb / 2;
    const int csize = pick_cluster<T, B2>(nmat, npairs);
    const int ppc = (npairs + csize - 1) / csize;
    const size_t smem = JacobiSmem<T, B2>::bytes(ppc);
    auto kern = k_jacobi<T, B2>;
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

}  // namespace

int jacobi_pad(int M) { return M <= 32 ? 32 : (int)round_up(M, 64); }

template <typename T>
cudaError_t launch_jacobi(T* G, T* Vt, int nmat, int Mp, int max_sweeps, double tol,
                          int32_t* sweeps, cudaStream_t s) {
    if (nmat <= 0) return cudaSuccess;
    if (Mp == 32) return launch_jacobi_b2<T, 32>(G, Vt, nmat, Mp, max_sweeps, tol, sweeps, s);
    return launch_jacobi_b2<T, 64>(G, Vt, nmat, Mp, max_sweeps, tol, sweeps, s);
}

template cudaError_t launch_jacobi<float>(float*, float*, int, int, int, double, int32_t*,
                                          cudaStream_t);
template cudaError_t launch_jacobi<double>(double*, double*, int, int, int, double, int32_t*,
                                           cudaStream_t);

}  // namespace rk
