"""Seeded synthetic inputs shaped like the workloads of the Ranky column-block SVD.

This module only draws matrices (CSC arrays) and request streams.  It holds
none of the method's arithmetic, and it is the one module that both the CUDA
path's tests/benchmark and the CPU oracle's tests use.

Every generator is deterministic in its seed; the default seed of workload
``k`` is ``20090976 + k``.

Workloads (sizes as named by the workload, not by the paper, whose own
539 x 170897 job-candidate matrix is private):

* ``small_uniform``      M=64, N=4096, Bernoulli(0.01) pattern, U(-1,1) values,
                         4 equal blocks of 1024, 200 columns of the second block
                         forced empty, all 64 triplets.
* ``small_lonely``       the same plus rows 0, 8, ..., 56 zeroed inside the
                         second block, so that block has 8 lonely rows.
* ``zipf_wide``          M=512, N=1e6, rank-law Zipf(1.1) column degrees capped at
                         512 and calibrated to ~512k non-zeros, uniform rows,
                         N(0,1) values, 64 blocks of 15625, all 512 triplets.
* ``large_skewed``       M=1024, N=8e6, ~80M non-zeros, row index Zipf(0.8),
                         uniform columns, U(0,1] values, 256 lognormal(0.7) block
                         widths, 16 rows zeroed inside every 5th block, k=100.
                         ``scale`` shrinks N (and the non-zero count) for tests.
* ``batch_mix``          independent matrices: M ~ U{32..256}, N ~ logU[1e3,2e5],
                         density ~ logU[0.005,0.05], N(0,1) values.
* ``neighbor_mix``       rank-fix pattern for the neighbour checkers: M=96,
                         N=3001, 7 lognormal(0.5) block widths; rows 0-47 spread
                         over all blocks (Bernoulli(0.03)), rows 48-92 living in
                         one block each (two entries; the even ones next to a
                         spread row, the odd ones in columns of their own), four
                         columns of 40 spread rows, 24 stored zeros (some beside
                         the lone rows), rows 93-95 empty.
* ``paper_bipartite``    0/1 pattern of the paper's matrix shape (539 x 170897,
                         the private job-candidate data); row m is Bernoulli(
                         density * a_m) over the columns, a_m lognormal(0, 0.5)
                         activities scaled to mean 1.  The paper does not state
                         its density, so tests sweep it.
* ``tall_skinny``        the row-block case: M=20011 rows, N=96 columns,
                         Bernoulli(0.012) pattern, N(0,1) values, 7 row blocks
                         (M not divisible by 7), columns 0, 5, ..., 45 emptied
                         inside the third row block (lonely nodes of A^T).
* ``arrival_stream``     Poisson arrivals of batch_mix-shaped requests with 5%
                         zipf_wide-shaped ones.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

SEED_BASE = 20090976


@dataclasses.dataclass
class CscCase:
    """A sparse M x N matrix in CSC form plus the run parameters that go with it."""

    name: str
    M: int
    N: int
    col_ptr: np.ndarray  # int64[N+1]
    row_idx: np.ndarray  # int32[nnz], sorted within each column, no duplicates
    vals: np.ndarray     # float32 or float64[nnz]
    num_blocks: int
    widths: Optional[np.ndarray] = None  # int64[D] or None for equal widths
    k: int = 0
    seed: int = 0

    @property
    def nnz(self) -> int:
        return int(self.row_idx.shape[0])

    def with_values(self, dtype) -> "CscCase":
        return dataclasses.replace(self, vals=self.vals.astype(dtype))


def _csc_from_mask_cols(M: int, N: int, cols: np.ndarray, rows: np.ndarray,
                        vals: np.ndarray):
    """CSC arrays from (col, row) pairs that are already sorted by (col, row)."""
    counts = np.bincount(cols, minlength=N).astype(np.int64)
    col_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=col_ptr[1:])
    return col_ptr, rows.astype(np.int32), vals


def _distinct_rows(rng: np.random.Generator, M: int, degrees: np.ndarray,
                   chunk: int = 8192):
    """For each column with degree c, c distinct rows drawn uniformly, sorted.
    Returns (local column index, row) pairs in (column, row) order."""
    out_c, out_r = [], []
    n = degrees.shape[0]
    for s in range(0, n, chunk):
        deg = degrees[s:s + chunk]
        keys = rng.random((deg.shape[0], M))
        order = np.argsort(keys, axis=1)
        take = np.arange(M)[None, :] < deg[:, None]
        sel = np.zeros((deg.shape[0], M), dtype=bool)
        np.put_along_axis(sel, order, take, axis=1)
        c, r = np.nonzero(sel)
        out_c.append(c + s)
        out_r.append(r)
    if not out_c:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(out_c), np.concatenate(out_r)


def bernoulli_csc(rng: np.random.Generator, M: int, N: int, density: float):
    """Bernoulli(density) pattern over the M x N entries, column-major.  The
    positions of the successes of the Bernoulli sequence are drawn as
    cumulative geometric gaps, which gives exactly the Bernoulli law and comes
    out sorted by (column, row).  Returns (col_ptr, row_idx)."""
    total = M * N
    if density <= 0.0 or total == 0:
        return np.zeros(N + 1, dtype=np.int64), np.zeros(0, dtype=np.int32)
    if density >= 1.0:
        pos = np.arange(total, dtype=np.int64)
    else:
        parts, last = [], -1
        while True:
            remaining = total - 1 - last
            draw = int(remaining * density + 6.0 * np.sqrt(remaining * density + 1.0) + 64)
            gaps = rng.geometric(density, size=draw).astype(np.int64)
            pos = last + np.cumsum(gaps)
            if pos[-1] >= total:
                parts.append(pos[pos < total])
                break
            parts.append(pos)
            last = int(pos[-1])
        pos = np.concatenate(parts)
    cols = pos // M
    rows = (pos % M).astype(np.int32)
    col_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.bincount(cols, minlength=N), out=col_ptr[1:])
    return col_ptr, rows


def small_uniform(seed: int = SEED_BASE + 1) -> CscCase:
    rng = np.random.default_rng(seed)
    M, N, D = 64, 4096, 4
    mask = rng.random((M, N)) < 0.01
    vals_dense = rng.uniform(-1.0, 1.0, size=(M, N))
    # 200 columns of the second block (columns 1024..2047) forced empty
    empty = 1024 + rng.choice(1024, size=200, replace=False)
    mask[:, empty] = False
    cols, rows = np.nonzero(mask.T)
    vals = vals_dense[rows, cols].astype(np.float64)
    col_ptr, row_idx, vals = _csc_from_mask_cols(M, N, cols, rows, vals)
    return CscCase("small_uniform", M, N, col_ptr, row_idx, vals, D, None, k=M,
                   seed=seed)


def small_lonely(seed: int = SEED_BASE + 1) -> CscCase:
    base = small_uniform(seed)
    zero_rows = np.arange(0, 64, 8)
    return zero_rows_in_columns(base, zero_rows, 1024, 2048, "small_lonely")


def zero_rows_in_columns(case: CscCase, rows, lo: int, hi: int,
                         name: Optional[str] = None) -> CscCase:
    """Remove every entry of the given rows inside columns [lo, hi)."""
    rows = np.asarray(rows)
    cols = np.repeat(np.arange(case.N, dtype=np.int64), np.diff(case.col_ptr))
    drop = (cols >= lo) & (cols < hi) & np.isin(case.row_idx, rows)
    keep = ~drop
    cols = cols[keep]
    col_ptr = np.zeros(case.N + 1, dtype=np.int64)
    np.cumsum(np.bincount(cols, minlength=case.N), out=col_ptr[1:])
    return dataclasses.replace(case, name=name or case.name, col_ptr=col_ptr,
                               row_idx=case.row_idx[keep], vals=case.vals[keep])


def zipf_wide(seed: int = SEED_BASE + 2, M: int = 512, N: int = 1_000_000,
              D: int = 64, target_nnz: int = 512_000, s: float = 1.1,
              dtype=np.float32) -> CscCase:
    rng = np.random.default_rng(seed)
    ranks = np.arange(1, N + 1, dtype=np.float64)
    w = ranks ** (-s)
    p = w / w.sum()
    position = rng.permutation(N)           # column that holds rank r
    draw_seed = int(rng.integers(1 << 62))

    def capped_total(T: int):
        counts = np.random.default_rng(draw_seed).multinomial(T, p)
        return np.minimum(counts, M)

    lo, hi = target_nnz, target_nnz * 64
    deg = capped_total(hi)
    for _ in range(60):
        mid = (lo + hi) // 2
        deg = capped_total(mid)
        tot = int(deg.sum())
        if abs(tot - target_nnz) <= 0.01 * target_nnz:
            break
        if tot < target_nnz:
            lo = mid
        else:
            hi = mid
    deg_by_col = np.zeros(N, dtype=np.int64)
    deg_by_col[position] = deg
    c, r = _distinct_rows(rng, M, deg_by_col)
    col_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(deg_by_col, out=col_ptr[1:])
    vals = rng.standard_normal(r.shape[0]).astype(dtype)
    return CscCase("zipf_wide", M, N, col_ptr, r.astype(np.int32), vals, D, None,
                   k=M, seed=seed)


def lognormal_widths(rng: np.random.Generator, N: int, D: int, sigma: float):
    """D positive integer widths summing to N with lognormal(0, sigma) shape
    (largest-remainder rounding)."""
    raw = np.exp(rng.normal(0.0, sigma, size=D))
    share = raw / raw.sum() * (N - D)
    base = np.floor(share).astype(np.int64)
    rem = (N - D) - int(base.sum())
    order = np.argsort(-(share - base))
    base[order[:rem]] += 1
    return base + 1


def large_skewed(seed: int = SEED_BASE + 3, M: int = 1024, N: int = 8_000_000,
                 D: int = 256, nnz_per_col: float = 10.0, s: float = 0.8,
                 k: int = 100, dtype=np.float32) -> CscCase:
    rng = np.random.default_rng(seed)
    widths = lognormal_widths(rng, N, D, 0.7)
    bounds = np.concatenate([[0], np.cumsum(widths)])
    total = int(round(nnz_per_col * N))
    pr = np.arange(1, M + 1, dtype=np.float64) ** (-s)
    pr /= pr.sum()
    cols = rng.integers(0, N, size=total, dtype=np.int64)
    rows = rng.choice(M, size=total, p=pr).astype(np.int64)
    key = np.unique(cols * M + rows)
    del cols, rows
    cols = key // M
    rows = key % M
    del key
    # every 5th block: 16 seeded rows zeroed inside the block
    drop = np.zeros(cols.shape[0], dtype=bool)
    for d in range(0, D, 5):
        zr = rng.choice(M, size=16, replace=False)
        lo, hi = bounds[d], bounds[d + 1]
        a, b = np.searchsorted(cols, [lo, hi])
        drop[a:b] |= np.isin(rows[a:b], zr)
    cols = cols[~drop]
    rows = rows[~drop]
    vals = (1.0 - rng.random(rows.shape[0])).astype(dtype)  # U(0, 1]
    col_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.bincount(cols, minlength=N), out=col_ptr[1:])
    return CscCase("large_skewed", M, N, col_ptr, rows.astype(np.int32), vals, D,
                   widths.astype(np.int64), k=k, seed=seed)


def batch_mix_shapes(rng: np.random.Generator, count: int):
    """(M, N, density) triples of the batched workload."""
    M = rng.integers(32, 257, size=count)
    N = np.exp(rng.uniform(np.log(1e3), np.log(2e5), size=count)).astype(np.int64)
    rho = np.exp(rng.uniform(np.log(0.005), np.log(0.05), size=count))
    return [(int(a), int(b), float(c)) for a, b, c in zip(M, N, rho)]


def batch_matrix(M: int, N: int, density: float, seed: int,
                 dtype=np.float32, name: str = "batch_mix") -> CscCase:
    rng = np.random.default_rng(seed)
    col_ptr, row_idx = bernoulli_csc(rng, M, N, density)
    vals = rng.standard_normal(row_idx.shape[0]).astype(dtype)
    return CscCase(name, M, N, col_ptr, row_idx, vals, 0, None, k=M, seed=seed)


def batch_mix(count: int = 2000, seed: int = SEED_BASE + 4, dtype=np.float32):
    """``count`` independent matrices (block count left to the caller)."""
    rng = np.random.default_rng(seed)
    shapes = batch_mix_shapes(rng, count)
    subseeds = rng.integers(1 << 62, size=count)
    return [batch_matrix(M, N, rho, int(ss), dtype) for (M, N, rho), ss in
            zip(shapes, subseeds)]


def neighbor_mix(seed: int = SEED_BASE + 6, dtype=np.float64) -> CscCase:
    """Pattern that exercises both outcomes of the neighbour rank fix (see
    the module docstring): lonely rows with neighbours, lonely rows whose
    neighbour lists are empty, long columns and stored zeros."""
    M, N, D = 96, 3001, 7
    rng = np.random.default_rng(seed)
    widths = lognormal_widths(rng, N, D, 0.5)
    bounds = np.concatenate([[0], np.cumsum(widths)])
    V = np.zeros((M, N))
    spread = rng.random((48, N)) < 0.03
    V[:48][spread] = rng.standard_normal(int(spread.sum()))
    for c in rng.choice(N, size=4, replace=False):
        rows = rng.choice(48, size=40, replace=False)
        V[rows, c] = rng.standard_normal(40)
    used = set()
    for m in range(48, 93):
        d = int(rng.integers(D))
        lo, hi = int(bounds[d]), int(bounds[d + 1])
        if m % 2 == 0:
            cols = [c for c in rng.permutation(np.arange(lo, hi))
                    if V[:48, c].any() and c not in used][:2]
        else:
            cols = [c for c in rng.permutation(np.arange(lo, hi))
                    if not V[:, c].any() and c not in used][:2]
        for c in cols:
            used.add(int(c))
            V[m, c] = rng.standard_normal()
    stored = V != 0
    # stored zeros: next to lone rows (they must not make neighbours) and at random
    lone_cols = [c for c in sorted(used) if not V[:48, c].any()]
    for c in rng.choice(lone_cols, size=min(12, len(lone_cols)), replace=False):
        stored[int(rng.integers(48)), c] = True
    for _ in range(12):
        stored[int(rng.integers(48)), int(rng.integers(N))] = True
    cols, rows = np.nonzero(stored.T)
    col_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.bincount(cols, minlength=N), out=col_ptr[1:])
    vals = V[rows, cols].astype(dtype)
    return CscCase("neighbor_mix", M, N, col_ptr, rows.astype(np.int32), vals, D,
                   widths.astype(np.int64), k=M, seed=seed)


def paper_bipartite(density: float, seed: int = SEED_BASE + 7, M: int = 539,
                    N: int = 170_897, activity_sigma: float = 0.5) -> CscCase:
    """0/1 bipartite pattern (values 1.0, float32) of the paper's matrix
    shape; see the module docstring."""
    rng = np.random.default_rng(seed)
    a = np.exp(rng.normal(0.0, activity_sigma, size=M))
    p = np.minimum(density * a / a.mean(), 1.0)
    cols, rows = [], []
    for m in range(M):
        c = np.nonzero(rng.random(N) < p[m])[0]
        cols.append(c)
        rows.append(np.full(c.shape[0], m, dtype=np.int64))
    cols = np.concatenate(cols)
    rows = np.concatenate(rows)
    order = np.lexsort((rows, cols))
    cols, rows = cols[order], rows[order]
    col_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.bincount(cols, minlength=N), out=col_ptr[1:])
    vals = np.ones(rows.shape[0], dtype=np.float32)
    return CscCase(f"paper_bipartite_{density:g}", M, N, col_ptr, rows.astype(np.int32), vals,
                   1, None, k=M, seed=seed)


def tall_skinny(seed: int = SEED_BASE + 8, M: int = 20011, N: int = 96, D: int = 7,
                density: float = 0.012, dtype=np.float64) -> CscCase:
    """Tall A (see the module docstring); num_blocks counts ROW blocks."""
    rng = np.random.default_rng(seed)
    col_ptr, row_idx = bernoulli_csc(rng, M, N, density)
    vals = rng.standard_normal(row_idx.shape[0]).astype(dtype)
    cols = np.repeat(np.arange(N, dtype=np.int64), np.diff(col_ptr))
    lo, hi = 2 * (M // D), 3 * (M // D)          # third row block of the equal split
    drop = (cols % 5 == 0) & (cols < 50) & (row_idx >= lo) & (row_idx < hi)
    keep = ~drop
    col_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.bincount(cols[keep], minlength=N), out=col_ptr[1:])
    return CscCase("tall_skinny", M, N, col_ptr, row_idx[keep], vals[keep], D, None, k=N,
                   seed=seed)


def random_dense_csc(rng: np.random.Generator, M: int, N: int, density: float,
                     dtype=np.float64, name: str = "random") -> CscCase:
    col_ptr, row_idx = bernoulli_csc(rng, M, N, density)
    vals = rng.standard_normal(row_idx.shape[0]).astype(dtype)
    return CscCase(name, M, N, col_ptr, row_idx, vals, 1, None, k=M)


def arrival_stream(rate: float, count: int, seed: int = SEED_BASE + 5,
                   wide_share: float = 0.05):
    """Poisson arrival times (seconds) and request shapes.  Each request is
    ('batch', M, N, density, subseed) or ('wide', subseed)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    shapes = batch_mix_shapes(rng, count)
    wide = rng.random(count) < wide_share
    subseeds = rng.integers(1 << 62, size=count)
    reqs = []
    for i in range(count):
        if wide[i]:
            reqs.append(("wide", int(subseeds[i])))
        else:
            M, N, rho = shapes[i]
            reqs.append(("batch", M, N, rho, int(subseeds[i])))
    return t, reqs
