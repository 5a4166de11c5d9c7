"""Full-size and large-shape parity, in the launch configuration bench.py
times.  The dense oracle cannot run at these sizes, so each result is checked
with quantities the oracle computes from the sparse matrix in FP64:

* residual certification: for unit u_i, v_i the residual
  r_i = max(|A'v_i - s_i u_i|, |A'^T u_i - s_i v_i|) bounds the distance from
  s_i to a true singular value of A', so r_i <= tol * s_i proves the relative
  error of s_i is within tol;
* the trace identity sum s_i^2 = |A'|_F^2 (full spectra);
* orthonormality of U, and bit-exact lonely flags from the oracle's sparse
  evaluation of Algorithm 1's definition."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2009_09767_gb300 as rk
import synth
from tests._metrics import orthonormality

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


def _certify(case, s, U, Vdev, idx, rel_tol):
    Ui = U[:, idx]
    Vi = Vdev[:, torch.as_tensor(idx, device=Vdev.device)].cpu().numpy().astype(np.float64)
    Vi = Vi / np.linalg.norm(Vi, axis=0, keepdims=True)
    r = oracle.residuals(case.col_ptr, case.row_idx, case.vals, case.M, s[idx], Ui, Vi)
    worst = float(np.max(r / s[idx]))
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
    idx = np.unique(np.concatenate([np.arange(0, 512, 37), np.arange(505, 512)]))
    _certify(case, s, U, V, idx, 1e-4 if precision == "mixed" else 1e-6)
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
    _certify(case, s, U, V, np.arange(100), 1e-4)
    assert orthonormality(U) < 1e-6
    # Algorithm 1 bookkeeping, bit exact: 16 rows zeroed inside blocks 0 and 5
    lon_ref, rne_ref = oracle.lonely_sparse(case.col_ptr, case.row_idx, case.vals, case.M, bounds)
    assert (p.query(rk.Q_LONELY).astype(bool) == lon_ref).all()
    assert (p.query(rk.Q_ROW_NONEMPTY).astype(bool) == rne_ref).all()
    ranks = p.query(rk.Q_BLOCK_RANKS)
    for d in (0, 5):
        assert lon_ref[d].sum() >= 16 and ranks[d] <= case.M - lon_ref[d].sum()
    p.free()
