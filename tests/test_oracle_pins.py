"""Pins for the CPU FP64 oracle: each test checks it against something other
than itself -- values printed in the paper, closed forms, invariants, exact
rational brute force, LAPACK (through numpy) and published generator
known-answer vectors.  None of these needs a GPU."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from tests.conftest import golden_path


# --------------------------------------------------------------------------
# RandomChecker's generator (Algorithm 2) against published KAT vectors

def test_philox_known_answers():
    rows = [l.split() for l in open(golden_path("philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(w[0:4], w[4:6])
        assert [int(x) for x in out] == w[6:10]


def test_random_patch_col_in_block_and_spread():
    lo, w = 1000, 37
    cols = [oracle.random_patch_col(7, d, m, lo, w) for d in range(5) for m in range(200)]
    assert min(cols) >= lo and max(cols) < lo + w
    counts = np.bincount(np.asarray(cols) - lo, minlength=w)
    # 1000 draws over 37 bins: every bin hit, none wildly over-full
    assert counts.min() > 0 and counts.max() < 3 * 1000 / w


# --------------------------------------------------------------------------
# Algorithm 1 block split against Table I's printed block sizes

def test_block_bounds_match_table1():
    rows = [l.split() for l in open(golden_path("table1_block_sizes.txt"))
            if l.strip() and not l.startswith("#")]
    for D, width in ((int(a), int(b)) for a, b in rows):
        b = oracle.block_bounds(170897, D)
        w = np.diff(b)
        assert (w[:-1] == width).all()
        assert w[-1] == 170897 - (D - 1) * width  # remainder kept in the last block
        assert b[0] == 0 and b[-1] == 170897


def test_block_bounds_explicit_widths():
    b = oracle.block_bounds(10, 3, [2, 5, 3])
    assert b.tolist() == [0, 2, 7, 10]


# --------------------------------------------------------------------------
# Lonely-node scan (Algorithm 1) on the worked example and against the
# sparse evaluation of the same definition

def _example_matrix():
    lines = [l.split() for l in open(golden_path("lonely_example.txt"))
             if l.strip() and not l.startswith("#")]
    M, N = int(lines[0][0]), int(lines[0][1])
    A = np.zeros((M, N))
    lonely = None
    for l in lines[1:]:
        if l[0] == "lonely":
            lonely = [int(x) - 1 for x in l[1:]]
        else:
            A[int(l[0]) - 1, int(l[1]) - 1] = 1.0
    return A, lonely


def test_lonely_worked_example():
    A, expect = _example_matrix()
    lon, rne = oracle.lonely_dense(A, oracle.block_bounds(A.shape[1], 1))
    assert np.nonzero(lon[0])[0].tolist() == expect
    # the empty row is empty in all of A: RandomChecker excludes it
    assert rne.tolist() == [True, True, True, True, False]


def test_lonely_multiblock_constructed():
    A = np.zeros((5, 12))
    A[0, 0] = 1.0; A[0, 5] = 2.0      # row 0: blocks 0 and 1
    A[1, 9] = -1.0                    # row 1: block 2 only
    A[2, 1] = 0.0                     # stored zero does not count
    A[3, :] = 3.0                     # row 3: everywhere
    A[4, 3] = 0.5                     # row 4: last column of block 0 only
    lon, rne = oracle.lonely_dense(A, oracle.block_bounds(12, 3))
    assert lon.astype(int).tolist() == [[0, 1, 1, 0, 0], [0, 1, 1, 0, 1],
                                        [1, 0, 1, 0, 1]]
    assert rne.tolist() == [True, True, False, True, True]


def test_lonely_sparse_equals_dense():
    c = synth.small_lonely()
    b = oracle.block_bounds(c.N, c.num_blocks)
    A = oracle.densify(c.col_ptr, c.row_idx, c.vals, c.M, c.N)
    ld, rd = oracle.lonely_dense(A, b)
    ls, rs = oracle.lonely_sparse(c.col_ptr, c.row_idx, c.vals, c.M, b)
    assert (ld == ls).all() and (rd == rs).all()
    assert np.nonzero(ld[1])[0].tolist() == list(range(0, 64, 8))


# --------------------------------------------------------------------------
# NeighborChecker (Algorithm 3) and neighbourRandomChecker (Algorithm 4)

def _neighbor_example():
    lines = [l.split() for l in open(golden_path("neighbor_example.txt"))
             if l.strip() and not l.startswith("#")]
    M, N = int(lines[0][0]), int(lines[0][1])
    A = np.zeros((M, N))
    for l in lines[1:]:
        if l[0] == "blocks":
            bounds = np.asarray([int(x) for x in l[1:]], dtype=np.int64)
        elif l[0] == "lonely":
            d, m = int(l[1]) - 1, int(l[2]) - 1
        elif l[0] == "neighbours":
            expect = [int(x) - 1 for x in l[1:]]
        else:
            A[int(l[0]) - 1, int(l[1]) - 1] = 1.0
    return A, bounds, d, m, expect


def _draw_index(seed, d, m, T):
    """Entry of a T-long sorted list the draw selects: floor(x T / 2^64),
    x = the Philox words (m, d, 1, 0) joined low word first (exact integers)."""
    w = oracle.philox4x32_10([m, d, 1, 0], [seed & 0xFFFFFFFF, seed >> 32])
    x = int(w[0]) | (int(w[1]) << 32)
    return (x * T) >> 64


def test_neighbor_worked_example():
    A, bounds, d, m, expect = _neighbor_example()
    lon, rne = oracle.lonely_dense(A, bounds)
    assert lon[d, m] and rne[m]
    assert oracle.neighbor_list(A, bounds, d, m).tolist() == expect
    for seed in range(16):
        col, T = oracle.neighbor_patch_col(A, bounds, d, m, seed)
        assert T == len(expect)
        assert col == expect[_draw_index(seed, d, m, T)]


def test_neighbor_draw_product_exact():
    """The list entry floor(x T / 2^64) is formed from four 32-bit partial
    products; it equals the exact integer quotient for every operand size,
    including carries out of the middle words."""
    rng = np.random.default_rng(3)
    cases = [(0, 0), (2**64 - 1, 2**64 - 1), (2**64 - 1, 1), (2**32, 2**32),
             (2**63, 3), (0xFFFFFFFF, 0xFFFFFFFF), (2**64 - 1, 2**40 + 12345)]
    cases += [(int(a), int(b)) for a, b in rng.integers(0, 2**63, size=(200, 2), dtype=np.uint64)]
    cases += [(int(a) * 2 + 1, int(b) >> s) for (a, b), s in
              zip(rng.integers(0, 2**63, size=(200, 2), dtype=np.uint64), range(200))]
    for a, b in cases:
        a &= 2**64 - 1
        assert oracle.mulhi64(a, b) == (a * b) >> 64, (a, b)


def _pattern_weights(A, bounds, d, m):
    """Closed form of the neighbour list's multiplicities: column n of block d
    appears sum_c C[m, c] B[c, n] times, B the 0/1 pattern of A and C the
    co-occurrence counts B B^T over the columns outside block d."""
    B = (A != 0).astype(np.int64)
    lo, hi = int(bounds[d]), int(bounds[d + 1])
    out = np.ones(B.shape[1], dtype=bool)
    out[lo:hi] = False
    C = B[:, out] @ B[:, out].T
    return C[m] @ B[:, lo:hi]


def _random_pattern(seed, M=9, N=40, density=0.12):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, N)) * (rng.random((M, N)) < density)
    A[rng.random((M, N)) < 0.02] = 0.0
    return A


def test_neighbor_list_multiplicities_closed_form():
    for seed in range(6):
        A = _random_pattern(seed)
        bounds = oracle.block_bounds(A.shape[1], 4)
        for d in range(4):
            lo = int(bounds[d])
            for m in range(A.shape[0]):
                w = _pattern_weights(A, bounds, d, m)
                expect = np.repeat(np.arange(lo, lo + w.shape[0]), w)
                got = oracle.neighbor_list(A, bounds, d, m)
                assert got.tolist() == expect.tolist(), (seed, d, m)


def test_neighbor_choice_against_closed_form():
    for seed in range(4):
        A = _random_pattern(seed + 10)
        bounds = oracle.block_bounds(A.shape[1], 4)
        lon, rne = oracle.lonely_dense(A, bounds)
        lon &= rne[None, :]
        for d, m in zip(*np.nonzero(lon)):
            w = _pattern_weights(A, bounds, d, m)
            col, T = oracle.neighbor_patch_col(A, bounds, int(d), int(m), 99 + seed)
            assert T == int(w.sum())
            if T == 0:
                assert col == -1
            else:
                flat = np.repeat(np.arange(w.shape[0]), w) + int(bounds[d])
                assert col == int(flat[_draw_index(99 + seed, int(d), int(m), T)])


def test_neighbor_rule_membership_bruteforce():
    """Every inserted entry obeys Algorithm 3's rule, checked by brute force:
    row m is lonely in block d, the column lies in block d, and some row c
    shares a non-zero column outside block d with m and is non-zero there."""
    for seed in range(4):
        A = _random_pattern(seed + 20, M=8, N=32, density=0.15)
        bounds = oracle.block_bounds(32, 4)
        lon, rne = oracle.lonely_dense(A, bounds)
        lon &= rne[None, :]
        P = oracle.neighbor_patches(A, bounds, lon, seed)
        blk = np.searchsorted(bounds, P[:, 1], side="right") - 1
        for (m, col), d in zip(P.tolist(), blk.tolist()):
            assert lon[d, m]
            lo, hi = int(bounds[d]), int(bounds[d + 1])
            ok = False
            for c in range(A.shape[0]):
                if A[c, col] == 0:
                    continue
                for n1 in range(A.shape[1]):
                    if not (lo <= n1 < hi) and A[m, n1] != 0 and A[c, n1] != 0:
                        ok = True
            assert ok, (m, col)


def test_neighbor_empty_list_and_random_fallback():
    A = np.zeros((3, 8))
    A[0, 0] = 1.0; A[0, 5] = 1.0      # row 0 in blocks 0 and 1
    A[1, 6] = 2.0                     # row 1 only in block 1, shares nothing
    A[2, 1] = 1.0; A[2, 5] = 1.0      # row 2 shares column 5 with row 0
    bounds = oracle.block_bounds(8, 2)
    lon, rne = oracle.lonely_dense(A, bounds)
    lon &= rne[None, :]
    assert lon.astype(int).tolist() == [[0, 1, 0], [0, 0, 0]]
    # row 1 in block 0: the only candidate is itself, empty in block 0
    assert oracle.neighbor_list(A, bounds, 0, 1).tolist() == []
    assert oracle.neighbor_patch_col(A, bounds, 0, 1, 5) == (-1, 0)
    assert oracle.neighbor_patches(A, bounds, lon, 5).shape == (0, 2)
    P = oracle.neighbor_patches(A, bounds, lon, 5, fallback_random=True)
    assert P.tolist() == [[1, oracle.random_patch_col(5, 0, 1, 0, 4)]]


def test_neighbor_single_distinct_column():
    A = np.zeros((3, 8))
    A[0, 2] = 1.0; A[0, 5] = 1.0      # row 0: column 2 of block 0, column 5
    A[1, 5] = 1.0; A[1, 7] = 3.0      # row 1: lonely in block 0, shares column 5
    A[2, 6] = 1.0
    bounds = oracle.block_bounds(8, 2)
    for seed in range(8):
        assert oracle.neighbor_patch_col(A, bounds, 0, 1, seed) == (2, 1)


def test_neighbor_draw_uniform_over_entries():
    """The draw is uniform over the list's entries, not over its distinct
    columns: a column listed twice is taken twice as often as one listed
    once."""
    A = np.zeros((4, 8))
    A[:, 4] = 1.0                     # rows 0-3 share column 4 (block 1)
    A[0, 0] = 1.0                     # row 0 lists column 0
    A[1, 1] = 1.0; A[2, 1] = 1.0      # rows 1 and 2 both list column 1
    bounds = oracle.block_bounds(8, 2)  # row 3 is lonely in block 0
    assert oracle.neighbor_list(A, bounds, 0, 3).tolist() == [0, 1, 1]
    cols = [oracle.neighbor_patch_col(A, bounds, 0, 3, s)[0] for s in range(4000)]
    frac = np.mean(np.asarray(cols) == 1)
    assert abs(frac - 2 / 3) < 4 * np.sqrt(2 / 9 / 4000)


def _csc(A):
    """CSC arrays of a dense matrix (stored entries = its non-zeros)."""
    cols, rows = np.nonzero(A.T)
    col_ptr = np.zeros(A.shape[1] + 1, dtype=np.int64)
    np.add.at(col_ptr, cols + 1, 1)
    return np.cumsum(col_ptr), rows.astype(np.int32), A[rows, cols]


def test_neighbor_sparse_equals_dense():
    for seed, fb in ((0, False), (1, True), (2, False), (3, True)):
        A = _random_pattern(seed + 30, M=12, N=60, density=0.08)
        bounds = oracle.block_bounds(60, 5)
        lon, rne = oracle.lonely_dense(A, bounds)
        lon &= rne[None, :]
        P = oracle.neighbor_patches(A, bounds, lon, seed, fallback_random=fb)
        col_ptr, row_idx, vals = _csc(A)
        S = oracle.neighbor_patches_sparse(col_ptr, row_idx, vals, 12, bounds, lon, seed,
                                           fallback_random=fb)
        assert S.tolist() == P.tolist()


def test_neighbor_sparse_equals_dense_on_neighbor_mix():
    """The closed-form evaluator agrees with the literal lists on the GPU
    parity case (long columns, stored zeros, empty lists), both modes."""
    c = synth.neighbor_mix()
    b = np.concatenate([[0], np.cumsum(c.widths)]).astype(np.int64)
    A = oracle.densify(c.col_ptr, c.row_idx, c.vals, c.M, c.N)
    lon, rne = oracle.lonely_dense(A, b)
    fix = lon & rne[None, :]
    for fb in (False, True):
        P = oracle.neighbor_patches(A, b, fix, 77, fallback_random=fb)
        S = oracle.neighbor_patches_sparse(c.col_ptr, c.row_idx, c.vals, c.M, b, fix, 77,
                                           fallback_random=fb)
        assert S.tolist() == P.tolist()
    assert 0 < len(oracle.neighbor_patches(A, b, fix, 77)) < int(fix.sum())


def test_svd_tall_against_lapack_and_reconstruction():
    """The tall form returns factors of A' itself: A' = U diag(s) V^T with
    orthonormal U (M x N) and V, and s equal to LAPACK's singular values; an
    insertion given as (column of A, row of A) lands at A'[row, column]."""
    rng = np.random.default_rng(12)
    A = rng.standard_normal((300, 7)) * (rng.random((300, 7)) < 0.2)
    col_ptr, row_idx, vals = _csc(A)
    pt = np.asarray([[2, 5], [6, 299]], dtype=np.int64)
    s, U, V, sweeps = oracle.svd_tall(col_ptr, row_idx, vals, 300, 7, pt)
    assert sweeps > 0
    Ap = A.copy()
    Ap[5, 2] += 1.0
    Ap[299, 6] += 1.0
    assert U.shape == (300, 7) and V.shape == (7, 7)
    assert np.abs(U @ np.diag(s) @ V.T - Ap).max() <= 1e-12 * np.abs(Ap).max()
    assert np.abs(U.T @ U - np.eye(7)).max() <= 1e-12
    assert np.abs(s - np.linalg.svd(Ap, compute_uv=False)).max() <= 1e-12 * s[0]


def test_svd_gram_01_against_jacobi_and_closed_form():
    """The exact-cross-product SVD of a 0/1 matrix agrees with the Jacobi SVD
    (both with insertions), and reproduces a closed form: k disjoint rows of
    lengths n_1..n_k have singular values sqrt(n_i)."""
    rng = np.random.default_rng(8)
    A = (rng.random((12, 300)) < 0.05).astype(np.float64)
    col_ptr, row_idx, vals = _csc(A)
    patches = np.asarray([[3, 17], [5, 250]], dtype=np.int64)
    s, U = oracle.svd_gram_01(col_ptr, row_idx, vals, 12, 300, patches)
    sj, Uj, _, _ = oracle.svd_csc(col_ptr, row_idx, vals, 12, 300, patches)
    assert np.abs(s - sj).max() <= 1e-12 * sj[0]
    assert np.abs(np.abs(U.T @ Uj) - np.eye(12)).max() <= 1e-9
    B = np.zeros((3, 20))
    B[0, 0:4] = 1; B[1, 4:13] = 1; B[2, 13:14] = 1
    s2, U2 = oracle.svd_gram_01(*_csc(B), 3, 20)
    assert np.allclose(s2, [3.0, 2.0, 1.0], rtol=0, atol=1e-14)
    assert np.allclose(np.abs(U2), np.eye(3)[[1, 0, 2]].T, atol=1e-14)
    with pytest.raises(ValueError):
        oracle.svd_gram_01(*_csc(B * 0.5), 3, 20)


# --------------------------------------------------------------------------
# Eq. 2 block cross product and the proxy identity of Eqs. 2-3

def test_gram_dense_against_matmul_and_sum():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((7, 30)) * (rng.random((7, 30)) < 0.3)
    b = oracle.block_bounds(30, 4)
    total = np.zeros((7, 7))
    for d in range(4):
        G = oracle.gram_dense(A, int(b[d]), int(b[d + 1]))
        blk = A[:, b[d]:b[d + 1]]
        np.testing.assert_allclose(G, blk @ blk.T, rtol=0, atol=1e-14)
        total += G
    np.testing.assert_allclose(total, A @ A.T, rtol=0, atol=1e-13)


def test_proxy_identity_with_oracle_blocks():
    """Eqs. 2-3: P = [U^1 S^1 | ... | U^D S^D] has the singular values and left
    subspaces of A, for any block ranks."""
    rng = np.random.default_rng(11)
    M, N, D = 9, 40, 5
    A = rng.standard_normal((M, N)) * (rng.random((M, N)) < 0.25)
    b = oracle.block_bounds(N, D)
    cols = []
    for d in range(D):
        s, U, _, _ = oracle.svd_dense(A[:, b[d]:b[d + 1]])
        cols.append(U * s[None, :])
    P = np.concatenate(cols, axis=1)
    sA = oracle.svd_dense(A)[0]
    sP = oracle.svd_dense(P)[0]
    np.testing.assert_allclose(sP, sA, rtol=1e-12, atol=1e-13 * sA[0])
    np.testing.assert_allclose(P @ P.T, A @ A.T, rtol=0, atol=1e-12 * sA[0] ** 2)


# --------------------------------------------------------------------------
# The SVD itself: closed forms

def _check_factorization(A, s, U, V, atol):
    M, N = A.shape
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, A, rtol=0, atol=atol)
    np.testing.assert_allclose(U.T @ U, np.eye(M), rtol=0, atol=1e-13)
    pos = s > 1e-12 * max(s[0], 1e-300)
    Vp = V[:, pos]
    np.testing.assert_allclose(Vp.T @ Vp, np.eye(pos.sum()), rtol=0, atol=1e-13)
    assert (np.diff(s) <= 0).all()


def _sign_rule_holds(U):
    for i in range(U.shape[1]):
        col = U[:, i]
        j = int(np.argmax(np.abs(col)))  # first index of the maximum
        assert col[j] > 0


def test_permuted_diagonal():
    M, N = 5, 9
    A = np.zeros((M, N))
    entries = [(0, 7, -3.0), (1, 2, 0.5), (2, 8, 4.0), (3, 0, -1.25), (4, 4, 2.0)]
    for r, c, v in entries:
        A[r, c] = v
    s, U, V, _ = oracle.svd_dense(A)
    np.testing.assert_array_equal(s, [4.0, 3.0, 2.0, 1.25, 0.5])
    # u_i is the unit vector of the row holding the i-th largest |entry|, made
    # positive by the sign rule; v_i carries the entry's sign
    order = [2, 0, 4, 3, 1]
    for i, r in enumerate(order):
        e = np.zeros(M); e[r] = 1.0
        np.testing.assert_array_equal(U[:, i], e)
        c, v = entries[r][1], entries[r][2]
        f = np.zeros(N); f[c] = np.sign(v)
        np.testing.assert_array_equal(V[:, i], f)


def test_rank_one():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(6)
    y = rng.standard_normal(15)
    A = np.outer(x, y)
    s, U, V, _ = oracle.svd_dense(A)
    expect = np.linalg.norm(x) * np.linalg.norm(y)
    assert abs(s[0] - expect) <= 1e-14 * expect
    assert (s[1:] <= 1e-14 * expect).all()
    u = x / np.linalg.norm(x)
    u = u if u[np.argmax(np.abs(u))] > 0 else -u
    np.testing.assert_allclose(U[:, 0], u, atol=1e-14)
    np.testing.assert_allclose(V[:, 0] * s[0], A.T @ U[:, 0], atol=1e-13 * expect)


def test_rank_r_disjoint_supports():
    """A = sum_i s_i x_i y_i^T with orthonormal x (disjoint supports) and
    orthonormal y (disjoint supports): singular values are the s_i."""
    rng = np.random.default_rng(4)
    M, N = 8, 24
    svals = np.array([5.0, 2.0, 2.0, 0.75])   # includes an exact tie
    xs = np.zeros((M, 4)); ys = np.zeros((N, 4))
    for i in range(4):
        xs[2 * i:2 * i + 2, i] = rng.standard_normal(2)
        ys[6 * i:6 * i + 6, i] = rng.standard_normal(6)
    xs /= np.linalg.norm(xs, axis=0); ys /= np.linalg.norm(ys, axis=0)
    A = (xs * svals) @ ys.T
    s, U, V, _ = oracle.svd_dense(A)
    np.testing.assert_allclose(s[:4], svals, rtol=1e-14)
    assert (s[4:] <= 1e-14 * 5.0).all()
    # u_1 and u_4 are determined up to sign; the tie at 2.0 only as a subspace
    for i, k in ((0, 0), (3, 3)):
        assert abs(abs(U[:, i] @ xs[:, k]) - 1.0) < 1e-13
    P_true = xs[:, 1:3] @ xs[:, 1:3].T
    P_got = U[:, 1:3] @ U[:, 1:3].T
    assert np.linalg.norm(P_true - P_got, 2) < 1e-13
    _check_factorization(A, s, U, V, 1e-13 * 5.0)


def _householder(rng, n):
    Q = np.eye(n)
    for _ in range(3):
        v = rng.standard_normal(n)
        v /= np.linalg.norm(v)
        Q = Q @ (np.eye(n) - 2.0 * np.outer(v, v))
    return Q


def test_known_sigma_householder_products():
    """Q1 diag(s) Q2^T with Householder-product Q's and chosen s, including a
    cluster and tails scaled by 1e-8."""
    rng = np.random.default_rng(8)
    M, N = 10, 26
    svals = np.array([3.0, 1.0, 1.0 + 1e-10, 1.0 - 1e-10, 0.5, 0.25, 0.1,
                      3e-8, 2e-8, 1e-8])
    Q1 = _householder(rng, M)
    Q2 = _householder(rng, N)[:, :M]
    A = Q1 @ np.diag(svals) @ Q2.T
    s, U, V, _ = oracle.svd_dense(A)
    expect = np.sort(svals)[::-1]
    np.testing.assert_allclose(s, expect, rtol=0, atol=2e-15 * 3.0)
    big = expect > 1e-3
    np.testing.assert_allclose(s[big], expect[big], rtol=1e-14)
    _check_factorization(A, s, U, V, 1e-14 * 3.0)


# --------------------------------------------------------------------------
# Invariants on sparse inputs shaped like the workloads

def test_invariants_small_uniform():
    c = synth.small_uniform()
    s, U, V, sweeps = oracle.svd_csc(c.col_ptr, c.row_idx, c.vals, c.M, c.N)
    assert sweeps > 0
    fro = oracle.frobenius_sq(c.vals)
    assert abs((s ** 2).sum() - fro) <= 1e-12 * fro
    A = oracle.densify(c.col_ptr, c.row_idx, c.vals, c.M, c.N)
    _check_factorization(A, s, U, V, 1e-13 * s[0])
    _sign_rule_holds(U)
    # empty columns of A have zero rows in V
    empty = np.diff(c.col_ptr) == 0
    assert np.abs(V[empty]).max() == 0.0


def test_residuals_function():
    c = synth.small_uniform()
    s, U, V, _ = oracle.svd_csc(c.col_ptr, c.row_idx, c.vals, c.M, c.N)
    r = oracle.residuals(c.col_ptr, c.row_idx, c.vals, c.M, s, U, V)
    assert r.max() < 1e-13 * s[0]
    s2 = s.copy(); s2[3] += 1e-3
    r2 = oracle.residuals(c.col_ptr, c.row_idx, c.vals, c.M, s2, U, V)
    assert abs(r2[3] - 1e-3) < 1e-12


# --------------------------------------------------------------------------
# LAPACK through numpy: a different algorithm and implementation

@pytest.mark.parametrize("shape,density", [((6, 6), 1.0), ((12, 50), 0.3),
                                           ((30, 200), 0.05), ((40, 41), 0.5)])
def test_against_lapack(shape, density):
    rng = np.random.default_rng(hash(shape) % 2**32)
    M, N = shape
    A = rng.standard_normal((M, N)) * (rng.random((M, N)) < density)
    s, U, V, _ = oracle.svd_dense(A)
    Ul, sl, Vlt = np.linalg.svd(A, full_matrices=False)
    k = min(M, N)
    np.testing.assert_allclose(s[:k], sl, rtol=0, atol=1e-13 * sl[0])
    gaps = np.abs(np.diff(sl))
    for i in range(k):
        sep = min(gaps[i - 1] if i > 0 else np.inf, gaps[i] if i < k - 1 else np.inf)
        if sl[i] > 1e-8 * sl[0] and sep > 1e-6 * sl[0]:
            assert abs(abs(U[:, i] @ Ul[:, i]) - 1.0) < 1e-10
            assert abs(abs(V[:, i] @ Vlt[i]) - 1.0) < 1e-10


def test_transposed_operand_is_caught():
    """A non-square, non-symmetric input: U must span the column space of A and
    V the row space (a transposed operand breaks this)."""
    rng = np.random.default_rng(21)
    A = rng.standard_normal((4, 11))
    s, U, V, _ = oracle.svd_dense(A)
    assert U.shape == (4, 4) and V.shape == (11, 4)
    np.testing.assert_allclose(A @ V, U * s[None, :], atol=1e-13 * s[0])
    np.testing.assert_allclose(A.T @ U, V * s[None, :], atol=1e-13 * s[0])


# --------------------------------------------------------------------------
# Exact rational brute force on tiny inputs: eigenvalues of A A^T by
# bisection on inertia counts (Sylvester), all in exact arithmetic.

def _inertia_below(B, x):
    """Number of eigenvalues of symmetric rational B strictly below x, from the
    signs of the LDL^T pivots of B - x I (exact)."""
    n = len(B)
    A = [[B[i][j] - (x if i == j else 0) for j in range(n)] for i in range(n)]
    neg = 0
    for k in range(n):
        p = A[k][k]
        if p == 0:
            return None
        if p < 0:
            neg += 1
        for i in range(k + 1, n):
            f = A[i][k] / p
            for j in range(k + 1, n):
                A[i][j] -= f * A[k][j]
    return neg


def _exact_eigs(B, hi, bits=110):
    n = len(B)
    out = []
    for k in range(n):   # k-th smallest eigenvalue
        lo_, hi_ = Fraction(-1), Fraction(hi)
        for _ in range(bits):
            mid = (lo_ + hi_) / 2
            c = _inertia_below(B, mid)
            while c is None:
                mid += (hi_ - lo_) / 1024
                c = _inertia_below(B, mid)
            if c > k:
                hi_ = mid
            else:
                lo_ = mid
        out.append((lo_ + hi_) / 2)
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_rational_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    M, N = 4, 7
    Ai = rng.integers(-3, 4, size=(M, N)) * (rng.random((M, N)) < 0.6)
    B = [[Fraction(int(np.dot(Ai[i], Ai[j]))) for j in range(M)] for i in range(M)]
    bound = sum(abs(B[i][j]) for i in range(M) for j in range(M)) + 1
    lam = sorted((float(v) for v in _exact_eigs(B, bound)), reverse=True)
    s, _, _, _ = oracle.svd_dense(Ai.astype(np.float64))
    expect = np.sqrt(np.maximum(lam, 0.0))
    np.testing.assert_allclose(s, expect, rtol=0, atol=1e-13 * max(expect[0], 1.0))
