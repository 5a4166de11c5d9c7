"""CPU FP64 oracle for the Ranky column-block SVD (arXiv 2009.09767).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library (``paper_2009_09767_gb300``) never imports, links
or calls it, and this package never imports the product; the two share no
code.  The only module both sides use is ``synth`` (seeded input generators,
which hold none of the method's arithmetic).

What each function follows:

* ``svd_dense`` / ``svd_csc``: the SVD of A' (the input plus rank-fix
  insertions).  Section III, Eqs. 2-3: the proxy matrix reproduces A A^*, so
  the method reaches SVD(A') exactly up to rounding; the oracle is that plain
  definition, a one-sided Hestenes Jacobi SVD in ``oracle.c``.  Empty columns
  are dropped before the dense SVD: they add nothing to A A^T and their rows
  of V are zero, so this is exact.
* ``block_bounds``: the column split of Algorithm 1 (``n`` from ``(N/D)*d`` to
  ``(N/D)*(d+1)``), read as half-open ranges of width floor(N/D) with the
  remainder given to the last block so that no column is dropped.
* ``lonely_dense``: Algorithm 1's lonely-node scan, literally (dense loops).
* ``lonely_sparse``: the same definition evaluated from the non-zero list
  (used where a dense copy does not fit); pinned against ``lonely_dense``.
* ``random_patches``: RandomChecker, Algorithm 2, with Philox4x32-10 keyed by
  (seed) and counted by (row, block).  Rows that are empty in all of A are not
  lonely nodes (they are excluded from the fix).
* ``neighbor_list`` / ``neighbor_patches``: NeighborChecker, Algorithm 3,
  with the two lists built literally as multisets in ``oracle.c``, and
  neighbourRandomChecker, Algorithm 4, read as RandomChecker only where the
  neighbour list is empty (Tables II and III print identical errors, which a
  second insertion would not give).  The column is entry floor(x T / 2^64)
  of the sorted list, x the 64-bit Philox word counted by (row, block, 1).
* ``neighbor_patches_sparse``: the same choice evaluated in closed form from
  the sparsity pattern B of A: column n of block d appears
  (B B^T)[m, :] B[:, n] times in row m's neighbour list.  Used where a dense
  copy does not fit; pinned against the literal lists.
* ``gram_dense``: Eq. 2's block cross product by plain summation.
* ``svd_tall``: the row-block (tall-and-skinny) form of section II.  For a
  tall A the method splits the rows into blocks; A^T is then short and fat
  with those blocks as its column blocks, so the method reaches the SVD of
  A'^T = V S U^T, whose factors are A' = U S V^T with the roles exchanged.
  Insertions are given in A^T's coordinates (row = column of A).
* ``svd_gram_01``: the SVD of A' for matrices with small integer entries (the
  0/1 patterns of the paper's job-candidate data).  Section III reads the
  singular values as the square roots of the eigenvalues of A A^*; for an
  integer A' the cross product A'A'^T is formed exactly in FP64, so the only
  rounding is the symmetric eigensolver's (LAPACK, through numpy).  Used as
  the truth where the dense Jacobi SVD would take minutes; pinned against
  ``svd_csc``.
* ``residuals``: a-posteriori residual bounds max(|A v - s u|, |A^T u - s v|)
  for triplets of matrices too large to densify; each bounds the distance
  from s to a true singular value.

Parity is pinned by ``tests/test_oracle_pins.py`` against closed forms,
invariants, exact rational brute force on tiny inputs, LAPACK (through numpy)
and the Philox known-answer vectors.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with gcc (portable flags)."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            lib.ro_philox4x32_10.argtypes = [P, P, P]
            lib.ro_philox4x32_10.restype = None
            lib.ro_random_patch_col.argtypes = [
                ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                ctypes.c_int64, ctypes.c_int64]
            lib.ro_random_patch_col.restype = ctypes.c_int64
            lib.ro_neighbor_list.argtypes = [P, ctypes.c_int32, ctypes.c_int64, P,
                                             ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32, P, ctypes.c_int64]
            lib.ro_neighbor_list.restype = ctypes.c_int64
            lib.ro_neighbor_patch_col.argtypes = [P, ctypes.c_int32, ctypes.c_int64, P,
                                                  ctypes.c_int32, ctypes.c_int32,
                                                  ctypes.c_int32, ctypes.c_uint64, P]
            lib.ro_neighbor_patch_col.restype = ctypes.c_int64
            lib.ro_mulhi64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.ro_mulhi64.restype = ctypes.c_uint64
            lib.ro_lonely_dense.argtypes = [P, ctypes.c_int32, ctypes.c_int64, P,
                                            ctypes.c_int32, P, P]
            lib.ro_lonely_dense.restype = None
            lib.ro_gram_dense.argtypes = [P, ctypes.c_int32, ctypes.c_int64,
                                          ctypes.c_int64, ctypes.c_int64, P]
            lib.ro_gram_dense.restype = None
            lib.ro_svd_jacobi.argtypes = [P, ctypes.c_int32, ctypes.c_int64, P, P, P,
                                          ctypes.c_int32, ctypes.c_double]
            lib.ro_svd_jacobi.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Philox / RandomChecker (Algorithm 2)

def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    lib.ro_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def random_patch_col(seed: int, d: int, m: int, lo: int, w: int) -> int:
    return int(_load().ro_random_patch_col(seed, d, m, lo, w))


def random_patches(lonely: np.ndarray, bounds: np.ndarray, seed: int) -> np.ndarray:
    """RandomChecker for every lonely (block d, row m), in (d, m) order.

    Returns an int64 array of shape (P, 2) with rows (m, col): the inserted
    entry A'[m, col] = 1.0 (Algorithm 2)."""
    D, M = lonely.shape
    out = []
    for d in range(D):
        lo, hi = int(bounds[d]), int(bounds[d + 1])
        for m in range(M):
            if lonely[d, m]:
                out.append((m, random_patch_col(seed, d, m, lo, hi - lo)))
    return np.asarray(out, dtype=np.int64).reshape(-1, 2)


# --------------------------------------------------------------------------
# NeighborChecker (Algorithm 3) and neighbourRandomChecker (Algorithm 4)

def neighbor_list(A: np.ndarray, bounds: np.ndarray, d: int, m: int) -> np.ndarray:
    """Row m's neighbour list in block d (Algorithm 3, multiset), sorted."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    M, N = A.shape
    b = np.ascontiguousarray(bounds, dtype=np.int64)
    D = b.shape[0] - 1
    n = lib.ro_neighbor_list(_ptr(A), M, N, _ptr(b), D, d, m, None, 0)
    if n < 0:
        raise MemoryError("oracle: allocation failed")
    out = np.zeros(max(n, 1), dtype=np.int64)
    lib.ro_neighbor_list(_ptr(A), M, N, _ptr(b), D, d, m, _ptr(out), n)
    return out[:n]


def neighbor_patch_col(A: np.ndarray, bounds: np.ndarray, d: int, m: int,
                       seed: int) -> tuple[int, int]:
    """(column, list length) NeighborChecker picks for lonely row m of block
    d; column -1 when the list is empty."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    M, N = A.shape
    b = np.ascontiguousarray(bounds, dtype=np.int64)
    D = b.shape[0] - 1
    ln = np.zeros(1, dtype=np.int64)
    col = lib.ro_neighbor_patch_col(_ptr(A), M, N, _ptr(b), D, d, m, seed, _ptr(ln))
    if col == -2:
        raise MemoryError("oracle: allocation failed")
    return int(col), int(ln[0])


def neighbor_patches(A: np.ndarray, bounds: np.ndarray, lonely: np.ndarray, seed: int,
                     fallback_random: bool = False) -> np.ndarray:
    """NeighborChecker (fallback_random=False) or neighbourRandomChecker for
    every lonely (block d, row m) in (d, m) order.  Returns (P, 2) rows
    (m, col); a lonely node with an empty neighbour list gets no insertion,
    or the RandomChecker column with the fallback."""
    D, M = lonely.shape
    out = []
    for d in range(D):
        lo, hi = int(bounds[d]), int(bounds[d + 1])
        for m in range(M):
            if not lonely[d, m]:
                continue
            col, _ = neighbor_patch_col(A, bounds, d, m, seed)
            if col < 0 and fallback_random:
                col = random_patch_col(seed, d, m, lo, hi - lo)
            if col >= 0:
                out.append((m, col))
    return np.asarray(out, dtype=np.int64).reshape(-1, 2)


def mulhi64(a: int, b: int) -> int:
    """High 64 bits of a*b as the C oracle forms them (draw -> list entry)."""
    return int(_load().ro_mulhi64(a, b))


def _philox_u64(seed: int, d: int, m: int) -> int:
    w = philox4x32_10([m, d, 1, 0], [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])
    return int(w[0]) | (int(w[1]) << 32)


def neighbor_patches_sparse(col_ptr, row_idx, vals, M: int, bounds: np.ndarray,
                            lonely: np.ndarray, seed: int,
                            fallback_random: bool = False) -> np.ndarray:
    """``neighbor_patches`` from the non-zero list: the multiplicity of column
    n in row m's neighbour list of block d is (B B^T)[m, :] B[:, n], B the
    0/1 pattern of A (exact integer products); the drawn entry is located by
    a cumulative sum over the block's columns."""
    import scipy.sparse as sp

    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    N = col_ptr.shape[0] - 1
    keep = np.asarray(vals) != 0
    c_of = np.repeat(np.arange(N, dtype=np.int64), np.diff(col_ptr))
    B = sp.csc_matrix((np.ones(int(keep.sum()), dtype=np.int64),
                       (np.asarray(row_idx, dtype=np.int64)[keep], c_of[keep])),
                      shape=(M, N))
    C = (B @ B.T).toarray().astype(np.int64)
    D = bounds.shape[0] - 1
    out = []
    for d in range(D):
        lo, hi = int(bounds[d]), int(bounds[d + 1])
        rows = np.nonzero(lonely[d])[0]
        if rows.size == 0:
            continue
        Bd = B[:, lo:hi].tocsc()
        for r0 in range(0, rows.size, 64):
            part = rows[r0:r0 + 64]
            Wt = np.asarray((sp.csr_matrix(C[part]) @ Bd).toarray(), dtype=np.int64)
            cum = np.cumsum(Wt, axis=1)
            for i, m in enumerate(part):
                T = int(cum[i, -1])
                if T == 0:
                    if fallback_random:
                        out.append((d, int(m), random_patch_col(seed, d, int(m), lo, hi - lo)))
                    continue
                r = (_philox_u64(seed, d, int(m)) * T) >> 64
                out.append((d, int(m), lo + int(np.searchsorted(cum[i], r, side="right"))))
    out.sort()
    return np.asarray([(m, c) for _, m, c in out], dtype=np.int64).reshape(-1, 2)


# --------------------------------------------------------------------------
# Algorithm 1: block split and lonely-node scan

def block_bounds(N: int, D: int, widths=None) -> np.ndarray:
    """D+1 column boundaries.  Equal split: width floor(N/D), remainder to the
    last block.  Explicit widths must be positive and sum to N."""
    if widths is not None:
        w = np.asarray(widths, dtype=np.int64)
        assert w.shape == (D,) and (w > 0).all() and int(w.sum()) == N
        return np.concatenate([[0], np.cumsum(w)]).astype(np.int64)
    base = N // D
    b = np.arange(D + 1, dtype=np.int64) * base
    b[D] = N
    return b


def lonely_dense(A: np.ndarray, bounds: np.ndarray):
    """Algorithm 1's scan over a dense matrix.  Returns (lonely[D, M] bool,
    row_nonempty[M] bool).  The RandomChecker fix applies to lonely nodes of
    rows that are non-empty in A."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    M, N = A.shape
    b = np.ascontiguousarray(bounds, dtype=np.int64)
    D = b.shape[0] - 1
    lon = np.zeros((D, M), dtype=np.uint8)
    rne = np.zeros(M, dtype=np.uint8)
    lib.ro_lonely_dense(_ptr(A), M, N, _ptr(b), D, _ptr(lon), _ptr(rne))
    return lon.astype(bool), rne.astype(bool)


def lonely_sparse(col_ptr, row_idx, vals, M: int, bounds: np.ndarray):
    """The lonely-node definition of Algorithm 1 evaluated on the non-zero list:
    row m is lonely in block d when no stored non-zero value of row m lies in
    the block's columns."""
    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    N = col_ptr.shape[0] - 1
    D = bounds.shape[0] - 1
    cols = np.repeat(np.arange(N, dtype=np.int64), np.diff(col_ptr))
    keep = np.asarray(vals) != 0
    blk = np.searchsorted(bounds, cols[keep], side="right") - 1
    occ = np.zeros((D, M), dtype=bool)
    occ[blk, np.asarray(row_idx)[keep]] = True
    row_nonempty = occ.any(axis=0)
    return ~occ, row_nonempty


# --------------------------------------------------------------------------
# Dense helpers

def densify(col_ptr, row_idx, vals, M: int, N: int, patches=None,
            cols: np.ndarray | None = None) -> np.ndarray:
    """Dense M x len(cols) FP64 copy of A' = A + patches (patch value 1.0).
    ``cols`` selects (sorted) columns; default all N."""
    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    row_idx = np.asarray(row_idx, dtype=np.int64)
    v = np.asarray(vals, dtype=np.float64)
    if cols is None:
        cols = np.arange(N, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    pos = -np.ones(N, dtype=np.int64)
    pos[cols] = np.arange(cols.shape[0])
    A = np.zeros((M, cols.shape[0]), dtype=np.float64)
    c_of = np.repeat(np.arange(N, dtype=np.int64), np.diff(col_ptr))
    sel = pos[c_of] >= 0
    A[row_idx[sel], pos[c_of[sel]]] += v[sel]
    if patches is not None and len(patches):
        p = np.asarray(patches, dtype=np.int64).reshape(-1, 2)
        ps = pos[p[:, 1]] >= 0
        np.add.at(A, (p[ps, 0], pos[p[ps, 1]]), 1.0)
    return A


def gram_dense(A: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Eq. 2 block cross product by plain summation (oracle.c)."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    M, N = A.shape
    G = np.zeros((M, M), dtype=np.float64)
    lib.ro_gram_dense(_ptr(A), M, N, lo, hi, _ptr(G))
    return G


def svd_dense(A: np.ndarray, max_sweeps: int = 100, tol: float = 1e-15):
    """One-sided Jacobi SVD (oracle.c).  Returns (sigma[M] descending,
    U[M, M], V[N, M], sweeps); A = U diag(sigma) V^T."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    M, N = A.shape
    s = np.zeros(M, dtype=np.float64)
    U = np.zeros((M, M), dtype=np.float64)
    V = np.zeros((N, M), dtype=np.float64)
    sweeps = lib.ro_svd_jacobi(_ptr(A), M, N, _ptr(s), _ptr(U), _ptr(V),
                               max_sweeps, tol)
    if sweeps == -2:
        raise MemoryError("oracle: allocation failed")
    return s, U, V, sweeps


def nonempty_columns(col_ptr, vals, patches=None) -> np.ndarray:
    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    N = col_ptr.shape[0] - 1
    c_of = np.repeat(np.arange(N, dtype=np.int64), np.diff(col_ptr))
    nz = np.zeros(N, dtype=bool)
    nz[c_of[np.asarray(vals) != 0]] = True
    if patches is not None and len(patches):
        nz[np.asarray(patches, dtype=np.int64).reshape(-1, 2)[:, 1]] = True
    return np.nonzero(nz)[0]


def svd_csc(col_ptr, row_idx, vals, M: int, N: int, patches=None,
            max_sweeps: int = 100, tol: float = 1e-15):
    """SVD of A' from CSC.  Empty columns are dropped before the dense SVD
    (exact: they add nothing to A A^T); their rows of V are zero.
    Returns (sigma[M], U[M, M], V[N, M], sweeps)."""
    cols = nonempty_columns(col_ptr, vals, patches)
    A = densify(col_ptr, row_idx, vals, M, N, patches, cols)
    s, U, Vc, sweeps = svd_dense(A, max_sweeps, tol)
    V = np.zeros((N, M), dtype=np.float64)
    V[cols] = Vc
    return s, U, V, sweeps


def svd_tall(col_ptr, row_idx, vals, M: int, N: int, patches_t=None,
             max_sweeps: int = 100, tol: float = 1e-15):
    """SVD of a tall A' (M x N CSC, patches_t = insertions (column of A, row
    of A) in A^T's coordinates): the Jacobi SVD of A'^T with U and V
    exchanged.  Returns (sigma[N], U[M, N], V[N, N], sweeps)."""
    At = np.ascontiguousarray(densify(col_ptr, row_idx, vals, M, N).T)
    if patches_t is not None and len(patches_t):
        p = np.asarray(patches_t, dtype=np.int64).reshape(-1, 2)
        np.add.at(At, (p[:, 0], p[:, 1]), 1.0)
    s, Ut, Vt, sweeps = svd_dense(At, max_sweeps, tol)
    return s, Vt, Ut, sweeps


def svd_gram_01(col_ptr, row_idx, vals, M: int, N: int, patches=None, return_gram=False):
    """sigma (descending) and U (M x M) of A' = A + patches for an A with
    integer entries, from the exactly formed cross product A'A'^T (returned
    third with return_gram).  Raises ValueError when the entries are not
    integers or the products could leave the exactly representable range
    (2^53)."""
    import scipy.sparse as sp

    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    v = np.asarray(vals, dtype=np.float64)
    if not np.all(v == np.round(v)):
        raise ValueError("svd_gram_01 needs integer entries")
    c_of = np.repeat(np.arange(N, dtype=np.int64), np.diff(col_ptr))
    r = np.asarray(row_idx, dtype=np.int64)
    if patches is not None and len(patches):
        p = np.asarray(patches, dtype=np.int64).reshape(-1, 2)
        r = np.concatenate([r, p[:, 0]])
        c_of = np.concatenate([c_of, p[:, 1]])
        v = np.concatenate([v, np.ones(p.shape[0])])
    A = sp.csr_matrix((v.astype(np.int64), (r, c_of)), shape=(M, N))
    G = (A @ A.T).toarray()
    if np.abs(G).max() >= 2**53 / max(M, 1):
        raise ValueError("cross product outside the exact FP64 integers")
    lam, U = np.linalg.eigh(G.astype(np.float64))
    order = np.argsort(-lam, kind="stable")
    lam, U = lam[order], U[:, order]
    sigma = np.sqrt(np.maximum(lam, 0.0))
    # sign rule of the product: the largest-magnitude entry of each u is positive
    arg = np.argmax(np.abs(U), axis=0)
    U = U * np.where(U[arg, np.arange(M)] < 0, -1.0, 1.0)[None, :]
    if return_gram:
        return sigma, U, G.astype(np.float64)
    return sigma, U


# --------------------------------------------------------------------------
# Sparse FP64 products for a-posteriori checks at sizes too large to densify

def sparse_matvec(col_ptr, row_idx, vals, M: int, x: np.ndarray, patches=None):
    """A' x for x of shape (N, k); FP64."""
    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    N = col_ptr.shape[0] - 1
    c_of = np.repeat(np.arange(N, dtype=np.int64), np.diff(col_ptr))
    v = np.asarray(vals, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((M,) + x.shape[1:], dtype=np.float64)
    np.add.at(out, np.asarray(row_idx, dtype=np.int64), v[:, None] * x[c_of] if x.ndim == 2 else v * x[c_of])
    if patches is not None and len(patches):
        p = np.asarray(patches, dtype=np.int64).reshape(-1, 2)
        np.add.at(out, p[:, 0], x[p[:, 1]])
    return out


def sparse_rmatvec(col_ptr, row_idx, vals, M: int, y: np.ndarray, patches=None):
    """A'^T y for y of shape (M, k); FP64."""
    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    N = col_ptr.shape[0] - 1
    c_of = np.repeat(np.arange(N, dtype=np.int64), np.diff(col_ptr))
    v = np.asarray(vals, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    out = np.zeros((N,) + y.shape[1:], dtype=np.float64)
    r = np.asarray(row_idx, dtype=np.int64)
    np.add.at(out, c_of, v[:, None] * y[r] if y.ndim == 2 else v * y[r])
    if patches is not None and len(patches):
        p = np.asarray(patches, dtype=np.int64).reshape(-1, 2)
        np.add.at(out, p[:, 1], y[p[:, 0]])
    return out


def residuals(col_ptr, row_idx, vals, M: int, sigma, U, V, patches=None):
    """Per-triplet residual max(|A'v_i - s_i u_i|, |A'^T u_i - s_i v_i|).

    For unit u_i, v_i this bounds the distance from s_i to some true singular
    value of A' (standard residual bound through the symmetric matrix
    [[0, A'], [A'^T, 0]])."""
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    s = np.asarray(sigma, dtype=np.float64)
    Av = sparse_matvec(col_ptr, row_idx, vals, M, V, patches)
    Atu = sparse_rmatvec(col_ptr, row_idx, vals, M, U, patches)
    r1 = np.linalg.norm(Av - U * s[None, :], axis=0)
    r2 = np.linalg.norm(Atu - V * s[None, :], axis=0)
    return np.maximum(r1, r2)


def frobenius_sq(vals, patches=None) -> float:
    v = np.asarray(vals, dtype=np.float64)
    n = float(np.dot(v, v))
    if patches is not None:
        n += float(len(patches))
    return n
