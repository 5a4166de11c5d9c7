// cluster_rr.cu -- Rayleigh-Ritz rotation inside clusters of close
// eigenvalue estimates, the part of the mixed-precision eigenbasis refinement
// that a first-order correction cannot do.
//
// The refinement step (Ogita & Aishima, Japan J. Indust. Appl. Math. 35,
// 2018) corrects the pair (i, j) of approximate eigenvectors by
// (S_ij + lam_j R_ij) / (lam_j - lam_i), which is only accurate while the
// mixing angle of the pair is small against their gap.  An FP32 Jacobi solve
// leaves pairs whose eigenvalues are closer than its stopping residual mixed
// at an angle of order one; the step then leaves them (or mis-corrects them),
// and the cross products these bases reproduce (Eqs. 2-3 of Ranky, arXiv
// 2009.09767: P P^T = sum_i A^i A^i^T) keep an error of the order of the
// FP32 residual.  The cure is the exact solution of the projected problem
// inside each cluster (the treatment of clustered eigenvalues in Ogita &
// Aishima, Japan J. Indust. Appl. Math. 36, 2019):
//
//   with X_c the rows of cluster c, S_cc = X_c G X_c^T, B_cc = X_c X_c^T:
//   B_cc = L L^T (Cholesky), C = L^-1 S_cc L^-T = Z diag(mu) Z^T (Jacobi,
//   FP64), and the rows of T_c = Z^T L^-1 X_c are the Ritz vectors: they are
//   orthonormal and T_c G T_c^T = diag(mu).
//
// The step's S = X G X^T and B = X X^T are transformed alongside
// (S <- T S T^T, B <- T B T^T, T = diag(T_c, identity elsewhere)) so that the
// first-order correction that follows sees the rotated basis.
//
// Which pairs need the exact treatment is decided pair by pair, not by one
// global threshold: the first-order correction of (i, j) has the size
// theta_ij = (|S_ij| + |lam_j| |R_ij|) / |lam_j - lam_i|, and it is accurate
// (its error is of order theta^2) while theta_ij is small.  Pairs with
// theta_ij >= 1 / kappa are linked;
// runs of linked estimates are the clusters, cut into pieces of at most
// kRRMax.  Every pair outside a common cluster then takes the first-order
// correction, whatever its gap; a single threshold from a norm bound of the
// off-diagonal part (the published step's) would put whole dense stretches of
// a spectrum into clusters.  Indices >= M (padding) never take part.
#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "kernels.h"

namespace rk {

namespace {

constexpr int kRRMax = 96;              // largest cluster solved exactly (3 x 96 x 97 doubles of shared memory)
constexpr int kRRLd = kRRMax + 1;       // odd stride: row and column access conflict-free
constexpr int kRRSweeps = 30;           // Jacobi sweep cap inside a cluster
constexpr int kRRSlots = 16;            // CTAs per matrix walking the cluster list
constexpr int kRRTile = 16;             // columns (rows) per CTA in the apply passes

__device__ __forceinline__ void rr_pair(int n, int r, int u, int& a, int& b) {
    // circle schedule over n (even) items: pair u of round r
    if (u == 0) {
        a = n - 1;
        b = r;
    } else {
        a = (r + u) % (n - 1);
        b = (r - u + (n - 1)) % (n - 1);
    }
    if (a > b) { const int t = a; a = b; b = t; }
}

// rowmax[a] >= max_{c != a} |S_ac| + |lam_c| |B_ac| (lam_c = S_cc / B_cc) as
// FP32 bits, from the high words of the FP64 entries and FP32 arithmetic
// rounded upwards: within about 4e-6 of the exact maximum, and never below
// it.  The FP64 pipe (a small fraction of the others' rate) stays idle.  A
// CTA of 8 warps takes 32 rows of one matrix, a warp a row at a time.
//
// |x| from its high word: the FP32 number with x's exponent and the top 20
// bits of its mantissa; one unit of the 20th bit more is an upper bound,
// the truncation itself a lower one.  Outside FP32's normal range: 2^-126
// (upper) or 0 (lower) below it, infinity (upper) or FLT_MAX (lower) above.
__device__ __forceinline__ float hi_abs_upper(double x) {
    const int h = __double2hiint(x) & 0x7fffffff;
    const int e = h >> 20;                       // biased FP64 exponent
    if (e >= 1151) return __int_as_float(0x7f800000);
    if (e < 897) return 0x1p-126f;
    return __uint_as_float((((unsigned)(e - 896) << 23) | ((unsigned)(h & 0xfffff) << 3)) + 8u);
}
__device__ __forceinline__ float hi_abs_lower(double x) {
    const int h = __double2hiint(x) & 0x7fffffff;
    const int e = h >> 20;
    if (e >= 1151) return FLT_MAX;
    if (e < 897) return 0.0f;
    return __uint_as_float(((unsigned)(e - 896) << 23) | ((unsigned)(h & 0xfffff) << 3));
}

__global__ void __launch_bounds__(256)
k_rr_rowmax(const double* __restrict__ S, const double* __restrict__ B, int M, int Mp,
            int32_t* __restrict__ rowmax) {
    __shared__ float lamb[kMaxM];     // >= |lam_c|
    const int b = blockIdx.y;
    const int64_t mm = (int64_t)Mp * Mp;
    const double* Sb = S + b * mm;
    const double* Bb = B + b * mm;
    for (int c = threadIdx.x; c < M; c += blockDim.x) {
        // a zero or tiny B_cc leaves no bound: the row's scan is unlimited
        const float bl = hi_abs_lower(Bb[(int64_t)c * Mp + c]);
        lamb[c] = bl > 0.0f ? __fdiv_ru(hi_abs_upper(Sb[(int64_t)c * Mp + c]), bl)
                            : __int_as_float(0x7f800000);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int a = blockIdx.x * 32 + warp; a < min(M, blockIdx.x * 32 + 32); a += 8) {
        const double* Sa = Sb + (int64_t)a * Mp;
        const double* Ba = Bb + (int64_t)a * Mp;
        float m = 0.0f;
        for (int c = lane; c < M; c += 32) {
            if (c == a) continue;
            m = fmaxf(m, __fadd_ru(hi_abs_upper(Sa[c]), __fmul_ru(lamb[c], hi_abs_upper(Ba[c]))));
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) rowmax[(int64_t)b * Mp + a] = __float_as_int(m);
    }
}

// Estimates lam_i = S_ii / B_ii (all Mp indices) and their largest magnitude;
// then the clusters: sort the first M estimates; positions q < q2 are linked
// when the first-order mixing estimate of the pair is not small,
// |lam_c - lam_a| <= kappa (|S_ac| + |lam_c| |B_ac|) (the scan from q stops
// at the first gap above kappa times the largest such numerator of row a);
// runs of linked positions are the clusters, cut into pieces of at most
// kRRMax at their largest gaps.  cid[i] = the piece of index i, -1 outside
// every piece.
// One CTA of 1024 threads per matrix (Mp <= 1024).  The scan limit of row a
// is kappa rowmax[a] (k_rr_rowmax), at least the exact maximum of the link
// test's right-hand side over the row: pairs beyond the exact maximum fail
// the test anyway, so the clusters are those of the exact limit.  The scan
// runs a warp per position, 32 candidates per ballot, with the exact FP64
// test.
__global__ void __launch_bounds__(1024)
k_rr_plan(const double* __restrict__ S, const double* __restrict__ B, int M, int Mp, double kappa,
          int stagger, double* __restrict__ lam, double* __restrict__ lmax_out,
          int32_t* __restrict__ order, int32_t* __restrict__ cstart, int32_t* __restrict__ csize,
          int32_t* __restrict__ ncl, int32_t* __restrict__ cid, const int32_t* __restrict__ rowmax_g) {
    __shared__ double key[kMaxM];
    __shared__ int id[kMaxM];
    __shared__ int reach[kMaxM];
    __shared__ float rowmax[kMaxM];
    __shared__ double wmax[32];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int64_t mm = (int64_t)Mp * Mp;
    const double* Sb = S + b * mm;
    const double* Bb = B + b * mm;
    double* L = lam + (int64_t)b * Mp;
    int32_t* cb = cid + (int64_t)b * Mp;
    double lm = 0.0;
    for (int i = tid; i < Mp; i += blockDim.x) {
        const double bii = Bb[(int64_t)i * Mp + i];
        const double l = bii > 0.0 ? Sb[(int64_t)i * Mp + i] / bii : 0.0;
        L[i] = l;
        rowmax[i] = __int_as_float(rowmax_g[(int64_t)b * Mp + i]);
        cb[i] = -1;
        if (l == l) lm = fmax(lm, fabs(l));
    }
    for (int o = 16; o > 0; o >>= 1) lm = fmax(lm, __shfl_xor_sync(0xffffffffu, lm, o));
    if ((tid & 31) == 0) wmax[tid >> 5] = lm;
    int n = 1;
    while (n < M) n <<= 1;
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
        const double v = i < M ? L[i] : DBL_MAX;
        key[i] = (v == v) ? v : DBL_MAX;   // a NaN estimate sorts last
        id[i] = i;
    }
    if (tid == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wmax[w]);
        lmax_out[b] = m;
    }
    __syncthreads();
    // bitonic sort ascending on (key, id)
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < n; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const bool gt = key[i] > key[ixj] || (key[i] == key[ixj] && id[i] > id[ixj]);
                    if (gt == up) {
                        const double tk = key[i]; key[i] = key[ixj]; key[ixj] = tk;
                        const int ti = id[i]; id[i] = id[ixj]; id[ixj] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    int32_t* ord = order + (int64_t)b * Mp;
    for (int q = tid; q < M; q += blockDim.x) ord[q] = id[q];
    {
        // reach[q] = the last position linked to q; keys are sorted, so the
        // candidates within the limit are a prefix of q + 1, q + 2, ...
        const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
        for (int q = warp; q < M; q += nw) {
            const int a = id[q];
            const double lim = kappa * (double)rowmax[a];    // no pair further than this links
            const double* Sa = Sb + (int64_t)a * Mp;
            const double* Ba = Bb + (int64_t)a * Mp;
            int r = q;
            for (int base = q + 1; base < M; base += 32) {
                const int q2 = base + lane;
                bool in = false, link = false;
                if (q2 < M) {
                    const double gap = key[q2] - key[q];
                    in = gap <= lim;
                    if (in) {
                        const int c = id[q2];
                        const double crit = kappa * (fabs(Sa[c]) + fabs(key[q2]) * fabs(Ba[c]));
                        link = gap <= crit;
                    }
                }
                const unsigned lm = __ballot_sync(0xffffffffu, link);
                if (lm != 0u) r = base + 31 - __clz(lm);
                if (__ballot_sync(0xffffffffu, q2 < M && !in) != 0u) break;
            }
            if (lane == 0) reach[q] = r;
        }
    }
    __syncthreads();
    if (tid == 0) {
        int32_t* cs = cstart + (int64_t)b * (Mp / 2);
        int32_t* cz = csize + (int64_t)b * (Mp / 2);
        int nc = 0;
        auto emit = [&](int lo, int hi) {
            if (hi - lo + 1 < 2) return;
            cs[nc] = lo;
            cz[nc] = hi - lo + 1;
            for (int q = lo; q <= hi; ++q) cb[id[q]] = nc;
            ++nc;
        };
        int i = 0;
        while (i < M) {
            int j = i, end = reach[i];
            while (j < end) { ++j; end = max(end, reach[j]); }
            // run [i, end]; longer than kRRMax: pieces of nominal length kRRMax
            // (the first one half as long when staggered), each cut at the
            // largest gap in the last quarter of its nominal span
            int len = stagger ? kRRMax / 2 : kRRMax;
            while (end - i + 1 > kRRMax) {
                int best = i + len - 1;
                double bg = -1.0;
                for (int q = i + len - kRRMax / 4; q < i + len - 1; ++q) {
                    const double g = key[q + 1] - key[q];
                    if (g > bg) { bg = g; best = q; }
                }
                emit(i, best);
                i = best + 1;
                len = kRRMax;
            }
            emit(i, end);
            i = end + 1;
        }
        ncl[b] = nc;
    }
}

// Rayleigh-Ritz inside each cluster: T_c into the rows/columns of the
// cluster's members in Tg (Mp x Mp per matrix), the Ritz values into lam.
// A cluster whose Gram is not safely positive definite is dropped (size 0).
__global__ void __launch_bounds__(256)
k_rr_solve(const double* __restrict__ S, const double* __restrict__ B, int Mp,
           const int32_t* __restrict__ order, const int32_t* __restrict__ cstart,
           int32_t* __restrict__ csize, const int32_t* __restrict__ ncl, double* __restrict__ Tg,
           double* __restrict__ lam) {
    extern __shared__ double rr_sm[];
    double* A = rr_sm;                       // S_cc, then C, then T^T
    double* Lm = A + kRRMax * kRRLd;         // B_cc, then its Cholesky factor
    double* Z = Lm + kRRMax * kRRLd;         // Y^T, then the eigenvectors
    __shared__ int ix[kRRMax];
    __shared__ double rc[kRRMax / 2], rs[kRRMax / 2], mu[kRRMax];
    __shared__ int rp[kRRMax / 2], rq[kRRMax / 2];
    __shared__ int fail, any;
    const int b = blockIdx.y, tid = threadIdx.x;
    const int half = Mp / 2;
    const int64_t mm = (int64_t)Mp * Mp;
    const double* Sb = S + b * mm;
    const double* Bb = B + b * mm;
    for (int c = blockIdx.x; c < ncl[b]; c += gridDim.x) {
        const int m = csize[(int64_t)b * half + c];
        if (m < 2 || m > kRRMax) continue;   // uniform over the CTA
        const int32_t* ord = order + (int64_t)b * Mp + cstart[(int64_t)b * half + c];
        __syncthreads();
        if (tid < m) ix[tid] = ord[tid];
        if (tid == 0) fail = 0;
        __syncthreads();
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int r = e / m, s = e % m;
            A[r * kRRLd + s] = Sb[(int64_t)ix[r] * Mp + ix[s]];
            Lm[r * kRRLd + s] = Bb[(int64_t)ix[r] * Mp + ix[s]];
        }
        __syncthreads();
        // Cholesky B_cc = L L^T (right-looking, lower triangle)
        for (int k = 0; k < m; ++k) {
            if (tid == 0) {
                const double d = Lm[k * kRRLd + k];
                if (!(d > 0.25)) fail = 1;   // rows are unit vectors: B_cc ~ I
                else Lm[k * kRRLd + k] = sqrt(d);
            }
            __syncthreads();
            if (fail) break;
            const double dk = Lm[k * kRRLd + k];
            for (int i = k + 1 + tid; i < m; i += blockDim.x) Lm[i * kRRLd + k] /= dk;
            __syncthreads();
            const int w = m - k - 1;
            for (int e = tid; e < w * w; e += blockDim.x) {
                const int i = k + 1 + e / w, j = k + 1 + e % w;
                if (j <= i) Lm[i * kRRLd + j] -= Lm[i * kRRLd + k] * Lm[j * kRRLd + k];
            }
            __syncthreads();
        }
        if (fail) {
            if (tid == 0) csize[(int64_t)b * half + c] = 0;
            continue;
        }
        // Y = L^-1 S_cc (column j by thread j), then Z = Y^T, C = L^-1 Z
        if (tid < m) {
            const int j = tid;
            for (int i = 0; i < m; ++i) {
                double v = A[i * kRRLd + j];
                for (int p = 0; p < i; ++p) v -= Lm[i * kRRLd + p] * A[p * kRRLd + j];
                A[i * kRRLd + j] = v / Lm[i * kRRLd + i];
            }
        }
        __syncthreads();
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int r = e / m, s = e % m;
            Z[r * kRRLd + s] = A[s * kRRLd + r];
        }
        __syncthreads();
        if (tid < m) {
            const int j = tid;
            for (int i = 0; i < m; ++i) {
                double v = Z[i * kRRLd + j];
                for (int p = 0; p < i; ++p) v -= Lm[i * kRRLd + p] * Z[p * kRRLd + j];
                Z[i * kRRLd + j] = v / Lm[i * kRRLd + i];
            }
        }
        __syncthreads();
        double amax = 0.0;
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int r = e / m, s = e % m;
            const double v = 0.5 * (Z[r * kRRLd + s] + Z[s * kRRLd + r]);
            A[r * kRRLd + s] = v;
            amax = fmax(amax, fabs(v));
        }
        __syncthreads();
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int r = e / m, s = e % m;
            Z[r * kRRLd + s] = r == s ? 1.0 : 0.0;
        }
        // absolute floor of the rotation test: rounding noise of C
        for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        __shared__ double wmax[8];
        if ((tid & 31) == 0) wmax[tid >> 5] = amax;
        __syncthreads();
        double cmax = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) cmax = fmax(cmax, wmax[w]);
        const double floor_abs = 1e-17 * cmax;
        // cyclic Jacobi on C (FP64), A <- J^T A J, Z <- Z J
        const int n2 = m + (m & 1);
        const int np = n2 / 2;
        for (int sweep = 0; sweep < kRRSweeps; ++sweep) {
            if (tid == 0) any = 0;
            __syncthreads();
            for (int r = 0; r < n2 - 1; ++r) {
                if (tid < np) {
                    int p, q;
                    rr_pair(n2, r, tid, p, q);
                    double c_ = 1.0, s_ = 0.0;
                    if (q < m) {
                        const double app = A[p * kRRLd + p], aqq = A[q * kRRLd + q];
                        const double apq = A[p * kRRLd + q];
                        if (fabs(apq) > floor_abs && fabs(apq) > 1e-15 * sqrt(fabs(app * aqq))) {
                            const double zeta = (aqq - app) / (2.0 * apq);
                            const double t = (zeta >= 0.0 ? 1.0 : -1.0) /
                                             (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                            c_ = 1.0 / sqrt(1.0 + t * t);
                            s_ = t * c_;
                            any = 1;
                        }
                    }
                    rc[tid] = c_; rs[tid] = s_; rp[tid] = p; rq[tid] = q;
                }
                __syncthreads();
                for (int e = tid; e < np * m; e += blockDim.x) {
                    const int u = e / m, col = e % m;
                    const int p = rp[u], q = rq[u];
                    const double c_ = rc[u], s_ = rs[u];
                    if (q >= m || s_ == 0.0) continue;
                    const double x = A[p * kRRLd + col], y = A[q * kRRLd + col];
                    A[p * kRRLd + col] = c_ * x - s_ * y;
                    A[q * kRRLd + col] = s_ * x + c_ * y;
                }
                __syncthreads();
                for (int e = tid; e < np * m; e += blockDim.x) {
                    const int u = e / m, row = e % m;
                    const int p = rp[u], q = rq[u];
                    const double c_ = rc[u], s_ = rs[u];
                    if (q >= m || s_ == 0.0) continue;
                    double x = A[row * kRRLd + p], y = A[row * kRRLd + q];
                    A[row * kRRLd + p] = c_ * x - s_ * y;
                    A[row * kRRLd + q] = s_ * x + c_ * y;
                    x = Z[row * kRRLd + p];
                    y = Z[row * kRRLd + q];
                    Z[row * kRRLd + p] = c_ * x - s_ * y;
                    Z[row * kRRLd + q] = s_ * x + c_ * y;
                }
                __syncthreads();
            }
            if (!any) break;   // uniform: read after the round's barriers
            __syncthreads();
        }
        if (tid < m) mu[tid] = A[tid * kRRLd + tid];
        __syncthreads();
        // T^T = L^-T Z: back substitution with L^T, column k by thread k
        if (tid < m) {
            const int k = tid;
            for (int i = m - 1; i >= 0; --i) {
                double v = Z[i * kRRLd + k];
                for (int p = i + 1; p < m; ++p) v -= Lm[p * kRRLd + i] * A[p * kRRLd + k];
                A[i * kRRLd + k] = v / Lm[i * kRRLd + i];
            }
        }
        __syncthreads();
        double* Tb = Tg + b * mm;
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int k = e / m, i = e % m;       // T[k][i] = (T^T)[i][k]
            Tb[(int64_t)ix[k] * Mp + ix[i]] = A[i * kRRLd + k];
        }
        if (tid < m) lam[(int64_t)b * Mp + ix[tid]] = mu[tid];
    }
}

// Rows of the cluster's members, in place: Z[c, tile] <- T_c Z[c, tile],
// for up to three matrices.  One CTA per (column tile, cluster slot, matrix).
__global__ void __launch_bounds__(256)
k_rr_rows(double* __restrict__ Z0, double* __restrict__ Z1, double* __restrict__ Z2, int Mp,
          const int32_t* __restrict__ order, const int32_t* __restrict__ cstart,
          const int32_t* __restrict__ csize, const int32_t* __restrict__ ncl,
          const double* __restrict__ Tg) {
    extern __shared__ double rr_dyn[];
    double (*Ts)[kRRLd] = reinterpret_cast<double (*)[kRRLd]>(rr_dyn);
    double (*buf)[kRRTile + 1] = reinterpret_cast<double (*)[kRRTile + 1]>(rr_dyn + kRRMax * kRRLd);
    __shared__ int ix[kRRMax];
    const int b = blockIdx.z, c0 = blockIdx.x * kRRTile, tid = threadIdx.x;
    const int half = Mp / 2;
    const int64_t mm = (int64_t)Mp * Mp;
    const double* Tb = Tg + b * mm;
    for (int c = blockIdx.y; c < ncl[b]; c += gridDim.y) {
        const int m = csize[(int64_t)b * half + c];
        if (m < 2 || m > kRRMax) continue;
        const int32_t* ord = order + (int64_t)b * Mp + cstart[(int64_t)b * half + c];
        __syncthreads();
        if (tid < m) ix[tid] = ord[tid];
        __syncthreads();
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int r = e / m, s = e % m;
            Ts[r][s] = Tb[(int64_t)ix[r] * Mp + ix[s]];
        }
        for (int z = 0; z < 3; ++z) {
            double* Zm = z == 0 ? Z0 : z == 1 ? Z1 : Z2;
            if (!Zm) continue;
            Zm += b * mm;
            __syncthreads();
            for (int e = tid; e < m * kRRTile; e += blockDim.x) {
                const int s = e / kRRTile, col = e % kRRTile;
                buf[s][col] = Zm[(int64_t)ix[s] * Mp + c0 + col];
            }
            __syncthreads();
            for (int e = tid; e < m * kRRTile; e += blockDim.x) {
                const int r = e / kRRTile, col = e % kRRTile;
                double v = 0.0;
                for (int s = 0; s < m; ++s) v = fma(Ts[r][s], buf[s][col], v);
                Zm[(int64_t)ix[r] * Mp + c0 + col] = v;
            }
        }
    }
}

// Columns of the cluster's members, in place: Z[tile, c] <- Z[tile, c] T_c^T,
// for up to two matrices (after k_rr_rows: Z <- T Z T^T).
__global__ void __launch_bounds__(256)
k_rr_cols(double* __restrict__ Z0, double* __restrict__ Z1, int Mp,
          const int32_t* __restrict__ order, const int32_t* __restrict__ cstart,
          const int32_t* __restrict__ csize, const int32_t* __restrict__ ncl,
          const double* __restrict__ Tg) {
    extern __shared__ double rr_dyn[];
    double (*Ts)[kRRLd] = reinterpret_cast<double (*)[kRRLd]>(rr_dyn);
    double (*buf)[kRRMax + 1] = reinterpret_cast<double (*)[kRRMax + 1]>(rr_dyn + kRRMax * kRRLd);
    __shared__ int ix[kRRMax];
    const int b = blockIdx.z, r0 = blockIdx.x * kRRTile, tid = threadIdx.x;
    const int half = Mp / 2;
    const int64_t mm = (int64_t)Mp * Mp;
    const double* Tb = Tg + b * mm;
    for (int c = blockIdx.y; c < ncl[b]; c += gridDim.y) {
        const int m = csize[(int64_t)b * half + c];
        if (m < 2 || m > kRRMax) continue;
        const int32_t* ord = order + (int64_t)b * Mp + cstart[(int64_t)b * half + c];
        __syncthreads();
        if (tid < m) ix[tid] = ord[tid];
        __syncthreads();
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int r = e / m, s = e % m;
            Ts[r][s] = Tb[(int64_t)ix[r] * Mp + ix[s]];
        }
        for (int z = 0; z < 2; ++z) {
            double* Zm = z == 0 ? Z0 : Z1;
            if (!Zm) continue;
            Zm += b * mm;
            __syncthreads();
            for (int e = tid; e < m * kRRTile; e += blockDim.x) {
                const int row = e / m, s = e % m;
                buf[row][s] = Zm[(int64_t)(r0 + row) * Mp + ix[s]];
            }
            __syncthreads();
            for (int e = tid; e < m * kRRTile; e += blockDim.x) {
                const int row = e / m, r = e % m;
                double v = 0.0;
                for (int s = 0; s < m; ++s) v = fma(buf[row][s], Ts[r][s], v);
                Zm[(int64_t)(r0 + row) * Mp + ix[r]] = v;
            }
        }
    }
}

// First-order correction outside the clusters, orthogonality only inside:
// E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) for i, j in different clusters
// while |E_ij| <= 1 / kappa (every pair the link test left apart satisfies
// this), R_ij / 2 otherwise: same cluster, a gap at rounding level, or a
// linked pair of a run cut into pieces.  The last are mixed at an angle a
// first-order step does not correct but scrambles; when their gap is at the
// level of the estimates' noise (long runs of repeated eigenvalues) the
// mixing costs nothing.  R = I - B, written over B.
// The numerator and the gap are formed in FP64 (both cancel); the quotient
// takes the approximate FP64 reciprocal (rcp.approx, relative error about
// 2^-20) times the numerator: E is applied through a product of three 8-bit
// slices (23 bits), and a correctly rounded FP64 division per entry would
// cost several FP64 operations on a pipe whose rate is a small fraction of
// the FP32 one.  The threshold tests compare the high words of the IEEE
// patterns (monotone in the magnitude), again off the FP64 pipe.
__device__ __forceinline__ double rcp_approx(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return r;
}

__global__ void k_rr_correction(double* __restrict__ B, const double* __restrict__ S, int Mp,
                                const double* __restrict__ lam, const double* __restrict__ lmax,
                                const int32_t* __restrict__ cid, double max_corr) {
    const int b = blockIdx.y;
    double* Bb = B + (int64_t)b * Mp * Mp;
    const double* Sb = S + (int64_t)b * Mp * Mp;
    const double* L = lam + (int64_t)b * Mp;
    const int32_t* cb = cid + (int64_t)b * Mp;
    // high words of |x| compared as integers: |gap| > tiny, |f| <= max_corr
    const int tiny_hi = __double2hiint(64.0 * 1.1102230246251565e-16 * lmax[b]) & 0x7fffffff;
    const int corr_hi = __double2hiint(max_corr) & 0x7fffffff;
    const int n = Mp * Mp;   // <= 2^20
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int i = e / Mp, j = e - i * Mp;
        const double bij = Bb[e];
        double v;
        if (i == j) {
            v = 0.5 * (1.0 - bij);
        } else {
            bool first_order = false;
            const int ci = cb[i];
            if (!(ci >= 0 && ci == cb[j])) {
                const double lj = L[j];
                const double gap = lj - L[i];
                if ((__double2hiint(gap) & 0x7fffffff) > tiny_hi) {
                    // (S_ij + lam_j R_ij) / gap, R_ij = -B_ij
                    const double f = fma(-lj, bij, Sb[e]) * rcp_approx(gap);
                    if ((__double2hiint(f) & 0x7fffffff) <= corr_hi) {   // NaN fails
                        v = f;
                        first_order = true;
                    }
                }
            }
            if (!first_order) v = -0.5 * bij;
        }
        Bb[e] = v;
    }
}

}  // namespace

size_t rr_smem_bytes() { return sizeof(double) * 3 * kRRMax * kRRLd; }

cudaError_t launch_cluster_rr(const RRWork& w, int nmat, int Mp, double* X, double* S, double* B,
                              double* Tg, double* lam, double* lmax, cudaStream_t s) {
    if (nmat <= 0) return cudaSuccess;
    if (Mp > kMaxM || Mp % kRRTile != 0 || w.M > Mp) return cudaErrorInvalidValue;
    k_rr_rowmax<<<dim3((unsigned)ceil_div(w.M, 32), nmat), 256, 0, s>>>(S, B, w.M, Mp, w.rowmax);
    RK_CUDA_TRY(cudaGetLastError());
    k_rr_plan<<<nmat, 1024, 0, s>>>(S, B, w.M, Mp, w.kappa, w.stagger, lam, lmax, w.order,
                                    w.cstart, w.csize, w.ncl, w.cid, w.rowmax);
    RK_CUDA_TRY(cudaGetLastError());
    const int smem = (int)rr_smem_bytes();
    RK_CUDA_TRY(cudaFuncSetAttribute(k_rr_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_rr_solve<<<dim3(kRRSlots, nmat), 256, smem, s>>>(S, B, Mp, w.order, w.cstart, w.csize, w.ncl,
                                                      Tg, lam);
    RK_CUDA_TRY(cudaGetLastError());
    const int srow = (int)(sizeof(double) * (kRRMax * kRRLd + kRRMax * (kRRTile + 1)));
    const int scol = (int)(sizeof(double) * (kRRMax * kRRLd + kRRTile * (kRRMax + 1)));
    RK_CUDA_TRY(cudaFuncSetAttribute(k_rr_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, srow));
    RK_CUDA_TRY(cudaFuncSetAttribute(k_rr_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, scol));
    k_rr_rows<<<dim3(Mp / kRRTile, kRRSlots, nmat), 256, srow, s>>>(X, S, B, Mp, w.order, w.cstart,
                                                                   w.csize, w.ncl, Tg);
    RK_CUDA_TRY(cudaGetLastError());
    k_rr_cols<<<dim3(Mp / kRRTile, kRRSlots, nmat), 256, scol, s>>>(S, B, Mp, w.order, w.cstart,
                                                                   w.csize, w.ncl, Tg);
    RK_CUDA_TRY(cudaGetLastError());
    const int bx = (int)std::min<int64_t>(ceil_div((int64_t)Mp * Mp, 256), 1024);
    k_rr_correction<<<dim3(bx, nmat), 256, 0, s>>>(B, S, Mp, lam, lmax, w.cid, 1.0 / w.kappa);
    return cudaGetLastError();
}

}  // namespace rk
