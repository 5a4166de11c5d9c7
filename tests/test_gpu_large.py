"""Full-size and large-shape parity, in the launch configuration bench.py
times.  The dense oracle cannot run at these sizes, so each result is checked
with quantities the oracle computes from the sparse matrix in FP64:

* residual certification: for unit u_i, v_i the residual
  r_i = max(|A'v_i - s_i u_i|, |A'^T u_i - s_i v_i|) bounds the distance from
  s_i to a true singular value of A', so r_i <= tol * s_i proves the relative
  error of s_i is within tol;
* the trace identity sum s_i^2 = |A'|_F^2 (full spectra);
* angle bounds for the left vectors: the Gram residual
  |A'A'^T u_i - s_i^2 u_i| over the separation of s_i^2 from the rest of the
  spectrum bounds the sine of the angle to the true vector (Davis-Kahan);
  every vector whose sigma is separated by 1e-3 sigma_1 must be within 1e-4;
* V against A'^T U S^-1 recomputed in FP64 from the sparse matrix;
* orthonormality of U, and bit-exact lonely flags from the oracle's sparse
  evaluation of Algorithm 1's definition."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2009_09767_gb300 as rk
import synth
from tests._metrics import gram_angle_bounds, orthonormality, separated, sparse_csc

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _run(case, precision, bounds=None, k=0):
    dev = torch.device("cuda")
    p = rk.Plan(case.M, case.N, case.nnz, case.num_blocks, value_type="f32", precision=precision,
                bounds=bounds, k=k)
    o = rk.alloc_outputs(p, device=dev)
    p.run(torch.from_numpy(case.col_ptr).to(dev), torch.from_numpy(case.row_idx).to(dev),
          torch.from_numpy(case.vals).to(dev), o["sigma"], o["U"], o["V"], o["rank"],
          o["patches"], o["npatches"])
    p.sync()
    return p, o


def _certify(case, s, U, Vdev, idx, rel_tol, A=None, v_tol=None):
    """Two-sided residuals r_i <= rel_tol s_i for the triplets idx (in chunks
    of 64, FP64 sparse products); with v_tol, also |v_i - A'^T u_i / s_i|_inf
    <= v_tol |v_i|_inf."""
    A = sparse_csc(case.col_ptr, case.row_idx, case.vals, case.M) if A is None else A
    worst = 0.0
    for c0 in range(0, len(idx), 64):
        ix = np.asarray(idx[c0:c0 + 64])
        Ui = U[:, ix]
        Vi = Vdev[:, torch.as_tensor(ix, device=Vdev.device)].cpu().numpy().astype(np.float64)
        if v_tol is not None:
            W = (A.T @ Ui) / s[ix][None, :]
            dv = np.abs(Vi - W).max(axis=0) / np.abs(W).max(axis=0)
            assert float(dv.max()) <= v_tol, f"V against A'^T U S^-1: {float(dv.max()):.3e}"
        Vi = Vi / np.linalg.norm(Vi, axis=0, keepdims=True)
        r = np.maximum(np.linalg.norm(A @ Vi - Ui * s[ix][None, :], axis=0),
                       np.linalg.norm(A.T @ Ui - Vi * s[ix][None, :], axis=0))
        worst = max(worst, float(np.max(r / s[ix])))
    assert worst <= rel_tol, f"certified relative error {worst:.3e} > {rel_tol:.1e}"
    return worst


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_zipf_wide_full_size(precision):
    case = synth.zipf_wide()
    p, o = _run(case, precision)
    s = o["sigma"].cpu().numpy()
    U = o["U"].cpu().numpy().T
    V = o["V"]
    assert o["rank"].item() == 512
    assert np.all(np.diff(s) <= 0)
    A = sparse_csc(case.col_ptr, case.row_idx, case.vals, case.M)
    # every one of the 512 triplets, and V against A'^T U S^-1
    _certify(case, s, U, V, np.arange(512), 1e-4 if precision == "mixed" else 1e-6, A=A,
             v_tol=1e-5 if precision == "mixed" else 1e-10)
    # left-vector angles: Gram residual over the separation, for every
    # vector separated by 1e-3 sigma_1 from its neighbours
    bound, _ = gram_angle_bounds(A, s, U)
    sep = separated(s)
    assert len(sep) > 0
    assert float(bound[sep].max()) <= 1e-4, float(bound[sep].max())
    fro = oracle.frobenius_sq(case.vals)
    assert abs((s ** 2).sum() - fro) <= (1e-6 if precision == "mixed" else 1e-10) * fro
    assert orthonormality(U) < (1e-6 if precision == "mixed" else 1e-12)
    p.free()


def test_large_skewed_downscaled():
    N = 250_000
    case = synth.large_skewed(N=N, D=8)
    bounds = np.concatenate([[0], np.cumsum(case.widths)]).astype(np.int64)
    p, o = _run(case, "mixed", bounds=bounds, k=100)
    s = o["sigma"].cpu().numpy()
    U = o["U"].cpu().numpy().T
    V = o["V"]
    assert s.shape == (100,) and np.all(np.diff(s) <= 0)
    _certify(case, s, U, V, np.arange(100), 1e-4, v_tol=1e-5)
    assert orthonormality(U) < 1e-6
    # Algorithm 1 bookkeeping, bit exact: 16 rows zeroed inside blocks 0 and 5
    lon_ref, rne_ref = oracle.lonely_sparse(case.col_ptr, case.row_idx, case.vals, case.M, bounds)
    assert (p.query(rk.Q_LONELY).astype(bool) == lon_ref).all()
    assert (p.query(rk.Q_ROW_NONEMPTY).astype(bool) == rne_ref).all()
    ranks = p.query(rk.Q_BLOCK_RANKS)
    for d in (0, 5):
        assert lon_ref[d].sum() >= 16 and ranks[d] <= case.M - lon_ref[d].sum()
    p.free()


def test_large_skewed_full_size():
    """The large single-matrix workload at its full size: 1024 x 8e6, ~80M
    non-zeros (row index Zipf(0.8), values U(0,1]), 256 lognormal(0.7) column
    blocks with 16 rows zeroed inside every 5th block, top k = 100, mixed
    precision.  All 100 triplets certified by residuals, V against
    A'^T U S^-1, and the lonely flags of all 256 x 1024 (block, row) pairs bit
    for bit."""
    case = synth.large_skewed()
    bounds = np.concatenate([[0], np.cumsum(case.widths)]).astype(np.int64)
    assert case.num_blocks == 256 and case.N == 8_000_000
    p, o = _run(case, "mixed", bounds=bounds, k=100)
    s = o["sigma"].cpu().numpy()
    U = o["U"].cpu().numpy().T
    V = o["V"]
    assert s.shape == (100,) and np.all(np.diff(s) <= 0)
    A = sparse_csc(case.col_ptr, case.row_idx, case.vals, case.M)
    _certify(case, s, U, V, np.arange(100), 1e-4, A=A, v_tol=1e-5)
    assert orthonormality(U) < 1e-6
    lon_ref, rne_ref = oracle.lonely_sparse(case.col_ptr, case.row_idx, case.vals, case.M, bounds)
    assert (p.query(rk.Q_LONELY).astype(bool) == lon_ref).all()
    assert (p.query(rk.Q_ROW_NONEMPTY).astype(bool) == rne_ref).all()
    assert lon_ref.sum() >= 16 * (256 // 5)
    p.free()
