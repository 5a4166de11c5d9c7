/*
 * oracle.c -- plain, slow, FP64 CPU reference for the Ranky column-block SVD.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the timed CPU
 * baseline of the benchmark use it.  It shares no code, header or constant
 * table with the CUDA path.
 *
 * What it computes (Tugay & Gunduz Oguducu, "Ranky: An Approach to Solve
 * Distributed SVD on Large Sparse Matrices", arXiv 2009.09767):
 *
 *   - ro_svd_jacobi: the SVD of a dense M x N matrix (section III reads the
 *     singular values as the square roots of the eigenvalues of A A^*, and
 *     Eqs. 2-3 show that the proxy matrix reaches exactly those of the full
 *     matrix).  The method therefore reaches SVD(A') exactly up to rounding,
 *     where A' is the input plus the rank-fix insertions, so the oracle is
 *     that plain definition: a one-sided (Hestenes) Jacobi SVD that rotates
 *     pairs of rows until all rows are mutually orthogonal, with the
 *     Rutishauser rotation formulas and cyclic-by-row pair order.
 *   - ro_lonely_dense: the lonely-node scan of Algorithm 1 (a row whose
 *     entries are all zero inside a column block), written exactly as the
 *     dense triple loop of the algorithm, half-open loop bounds.
 *   - ro_gram_dense: the block cross product A^i (A^i)^* of Eq. 2 by plain
 *     summation over the block's columns.
 *   - ro_philox4x32_10 / ro_random_patch_col: RandomChecker (Algorithm 2)
 *     draws "a random column in block d".  The random numbers come from the
 *     counter-based Philox4x32-10 generator, implemented here from its
 *     published definition (Salmon, Moraes, Dror, Shaw, "Parallel random
 *     numbers: as easy as 1, 2, 3", SC 2011), keyed by the caller's seed and
 *     counted by (row, block).
 *   - ro_neighbor_list / ro_neighbor_patch_col: NeighborChecker (Algorithm 3)
 *     for one lonely row m of block d.  The two lists are built exactly as
 *     the algorithm builds them, as multisets: every row that shares a
 *     non-zero column with m in another block, once per shared column
 *     (row m itself included); then, for every list entry, every column of
 *     block d where that row is non-zero.  Readings where the algorithm's
 *     text is garbled: the second loop's row is the candidate the list entry
 *     names (not the list position), and its columns run over block d's own
 *     range.  The lists are built from the input A, before any insertion.
 *     "Choose a random column from neighbourList" is a uniform draw over the
 *     list's entries: the list is sorted ascending and entry
 *     floor(x * T / 2^64) taken, x the 64-bit Philox word (m, d, 1, 0) and
 *     T the list's length.  An empty list gives -1 (no column); Algorithm 4
 *     (neighbourRandomChecker) then takes the RandomChecker column.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011): 10 rounds of two 32x32->64 multiplies
 * with the published multipliers, key bumped by the published Weyl
 * constants between rounds. */
void ro_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    const uint32_t MUL0 = 0xD2511F53u, MUL1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)MUL0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)MUL1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) { k0 += W0; k1 += W1; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* RandomChecker (Algorithm 2): the column inserted for lonely row m of block
 * d.  Counter = (m, d, 0, 0), key = (low, high word of seed); the first
 * output word x is mapped onto the block's w columns as lo + floor(x*w/2^32). */
int64_t ro_random_patch_col(uint64_t seed, int32_t d, int32_t m, int64_t lo,
                            int64_t w) {
    uint32_t ctr[4] = {(uint32_t)m, (uint32_t)d, 0u, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    ro_philox4x32_10(ctr, key, out);
    return lo + (int64_t)(((uint64_t)out[0] * (uint64_t)w) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3 (NeighborChecker).  Growable arrays for the two lists. */
typedef struct { int64_t* v; int64_t n, cap; } ro_list;

static int ro_list_push(ro_list* l, int64_t x) {
    if (l->n == l->cap) {
        int64_t cap = l->cap ? 2 * l->cap : 64;
        int64_t* v = (int64_t*)realloc(l->v, (size_t)cap * sizeof(int64_t));
        if (!v) return -1;
        l->v = v;
        l->cap = cap;
    }
    l->v[l->n++] = x;
    return 0;
}

static int ro_cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

/* High 64 bits of the 128-bit product a*b, from four 32x32 products. */
uint64_t ro_mulhi64(uint64_t a, uint64_t b) {
    uint64_t a0 = a & 0xffffffffu, a1 = a >> 32, b0 = b & 0xffffffffu, b1 = b >> 32;
    uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
    uint64_t mid = (p00 >> 32) + (p01 & 0xffffffffu) + (p10 & 0xffffffffu);
    return p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
}

/* The neighbour list of lonely row m in block d (dense row-major M x N A,
 * D+1 column bounds), sorted ascending.  Returns its length and, when out is
 * not NULL and cap allows, copies it there; -2 when memory ran out. */
int64_t ro_neighbor_list(const double* A, int32_t M, int64_t N, const int64_t* bounds,
                         int32_t D, int32_t d, int32_t m, int64_t* out, int64_t cap) {
    ro_list cand = {0, 0, 0}, nbr = {0, 0, 0};
    int64_t len = -2;
    /* candidates: rows non-zero in a column of another block where m is */
    for (int32_t d1 = 0; d1 < D; ++d1) {
        if (d1 == d) continue;
        for (int64_t n1 = bounds[d1]; n1 < bounds[d1 + 1]; ++n1) {
            if (A[(int64_t)m * N + n1] == 0.0) continue;
            for (int32_t m1 = 0; m1 < M; ++m1)
                if (A[(int64_t)m1 * N + n1] != 0.0 && ro_list_push(&cand, m1)) goto done;
        }
    }
    /* neighbours: columns of block d where a candidate is non-zero */
    for (int64_t i = 0; i < cand.n; ++i) {
        const int64_t c = cand.v[i];
        for (int64_t n2 = bounds[d]; n2 < bounds[d + 1]; ++n2)
            if (A[c * N + n2] != 0.0 && ro_list_push(&nbr, n2)) goto done;
    }
    if (nbr.n > 1) qsort(nbr.v, (size_t)nbr.n, sizeof(int64_t), ro_cmp_i64);
    len = nbr.n;
    if (out)
        for (int64_t i = 0; i < len && i < cap; ++i) out[i] = nbr.v[i];
done:
    free(cand.v);
    free(nbr.v);
    return len;
}

/* NeighborChecker's column for lonely row m of block d: the list entry chosen
 * by the draw described in the header, or -1 when the list is empty (-2 when
 * memory ran out).  *list_len receives the list's length. */
int64_t ro_neighbor_patch_col(const double* A, int32_t M, int64_t N, const int64_t* bounds,
                              int32_t D, int32_t d, int32_t m, uint64_t seed,
                              int64_t* list_len) {
    int64_t len = ro_neighbor_list(A, M, N, bounds, D, d, m, NULL, 0);
    if (list_len) *list_len = len;
    if (len <= 0) return len == 0 ? -1 : -2;
    int64_t* lst = (int64_t*)malloc((size_t)len * sizeof(int64_t));
    if (!lst) return -2;
    ro_neighbor_list(A, M, N, bounds, D, d, m, lst, len);
    uint32_t ctr[4] = {(uint32_t)m, (uint32_t)d, 1u, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t w[4];
    ro_philox4x32_10(ctr, key, w);
    const uint64_t x = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    const int64_t col = lst[ro_mulhi64(x, (uint64_t)len)];
    free(lst);
    return col;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, lonely-node scan.  A is dense row-major M x N; bounds holds
 * D+1 column boundaries.  lonely[d*M + m] = 1 when row m has no non-zero in
 * columns [bounds[d], bounds[d+1]).  row_nonempty[m] = 1 when row m has a
 * non-zero anywhere in A. */
void ro_lonely_dense(const double* A, int32_t M, int64_t N,
                     const int64_t* bounds, int32_t D, uint8_t* lonely,
                     uint8_t* row_nonempty) {
    for (int32_t m = 0; m < M; ++m) {
        row_nonempty[m] = 0;
        for (int64_t n = 0; n < N; ++n)
            if (A[(int64_t)m * N + n] != 0.0) { row_nonempty[m] = 1; break; }
    }
    for (int32_t d = 0; d < D; ++d) {
        for (int32_t m = 0; m < M; ++m) {
            int checker = 1;
            for (int64_t n = bounds[d]; n < bounds[d + 1]; ++n) {
                if (A[(int64_t)m * N + n] != 0.0) { checker = 0; break; }
            }
            lonely[(int64_t)d * M + m] = (uint8_t)checker;
        }
    }
}

/* Eq. 2 block cross product: G = A[:, lo:hi] A[:, lo:hi]^T, plain summation
 * in column order.  G is M x M row-major. */
void ro_gram_dense(const double* A, int32_t M, int64_t N, int64_t lo,
                   int64_t hi, double* G) {
    for (int32_t i = 0; i < M; ++i)
        for (int32_t j = 0; j < M; ++j) {
            double s = 0.0;
            for (int64_t n = lo; n < hi; ++n)
                s += A[(int64_t)i * N + n] * A[(int64_t)j * N + n];
            G[(int64_t)i * M + j] = s;
        }
}

/* ------------------------------------------------------------------------ */
/* One-sided Hestenes Jacobi SVD of a dense M x N row-major matrix A.
 *
 * Rows w_p, w_q of a working copy W are rotated until <w_p, w_q> is
 * negligible against |w_p| |w_q| for every pair; then W = Sigma V^T and the
 * accumulated rotations give U, so A = U Sigma V^T.
 *
 * Outputs: sigma[M] descending; U[M*M] row-major (column i = u_i);
 * V[N*M] row-major (column i = v_i; zero where sigma_i == 0).
 * Sign rule: the largest-magnitude entry of each u_i is positive (first such
 * entry on a tie); v_i takes the same sign.
 * Returns the number of sweeps, or -1 when max_sweeps ran out. */
int ro_svd_jacobi(const double* A, int32_t M, int64_t N, double* sigma,
                  double* U, double* V, int32_t max_sweeps, double tol) {
    double* W = (double*)malloc(sizeof(double) * (size_t)M * (size_t)N);
    double* Q = (double*)malloc(sizeof(double) * (size_t)M * (size_t)M);
    double* nrm = (double*)malloc(sizeof(double) * (size_t)M);
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)M);
    if (!W || !Q || !nrm || !order) {
        free(W); free(Q); free(nrm); free(order);
        return -2;
    }
    memcpy(W, A, sizeof(double) * (size_t)M * (size_t)N);
    for (int32_t i = 0; i < M; ++i)
        for (int32_t j = 0; j < M; ++j) Q[(int64_t)i * M + j] = (i == j);

    int sweeps = 0, converged = 0;
    while (!converged && sweeps < max_sweeps) {
        int rotated = 0;
        for (int32_t p = 0; p < M - 1; ++p) {
            for (int32_t q = p + 1; q < M; ++q) {
                double* wp = W + (int64_t)p * N;
                double* wq = W + (int64_t)q * N;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int64_t n = 0; n < N; ++n) {
                    alpha += wp[n] * wp[n];
                    beta += wq[n] * wq[n];
                    gamma += wp[n] * wq[n];
                }
                if (gamma == 0.0) continue;
                if (fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta)) continue;
                rotated = 1;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) /
                           (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = c * t;
                for (int64_t n = 0; n < N; ++n) {
                    double a = wp[n], b = wq[n];
                    wp[n] = c * a - s * b;
                    wq[n] = s * a + c * b;
                }
                for (int32_t r = 0; r < M; ++r) {
                    double a = Q[(int64_t)r * M + p], b = Q[(int64_t)r * M + q];
                    Q[(int64_t)r * M + p] = c * a - s * b;
                    Q[(int64_t)r * M + q] = s * a + c * b;
                }
            }
        }
        ++sweeps;
        if (!rotated) converged = 1;
    }

    for (int32_t i = 0; i < M; ++i) {
        double s = 0.0;
        const double* wi = W + (int64_t)i * N;
        for (int64_t n = 0; n < N; ++n) s += wi[n] * wi[n];
        nrm[i] = sqrt(s);
        order[i] = i;
    }
    /* stable insertion sort, descending */
    for (int32_t i = 1; i < M; ++i) {
        int32_t k = order[i];
        int32_t j = i - 1;
        while (j >= 0 && nrm[order[j]] < nrm[k]) { order[j + 1] = order[j]; --j; }
        order[j + 1] = k;
    }
    for (int32_t i = 0; i < M; ++i) {
        int32_t src = order[i];
        double si = nrm[src];
        /* sign rule on column src of Q */
        int32_t arg = 0;
        double best = -1.0;
        for (int32_t r = 0; r < M; ++r) {
            double a = fabs(Q[(int64_t)r * M + src]);
            if (a > best) { best = a; arg = r; }
        }
        double sg = Q[(int64_t)arg * M + src] < 0.0 ? -1.0 : 1.0;
        sigma[i] = si;
        for (int32_t r = 0; r < M; ++r)
            U[(int64_t)r * M + i] = sg * Q[(int64_t)r * M + src];
        const double* ws = W + (int64_t)src * N;
        for (int64_t n = 0; n < N; ++n)
            V[n * M + i] = si > 0.0 ? sg * ws[n] / si : 0.0;
    }
    free(W); free(Q); free(nrm); free(order);
    return converged ? sweeps : -1;
}
