"""Singular values spread over several orders of magnitude, against their
closed form.

A = Q1 diag(s) Q2^T with orthonormal Q1 (M x M) and Q2 (N x M) from QR
factorizations of Gaussian matrices, s geometric from 1 down to 10^-p, stored
as a dense-pattern CSC in FP64 and split into 4 column blocks.  The method
works on cross products (A^i A^i^T, P P^T), which square the spread: the
squared singular values span 2p decades, so small ones are the first to lose
relative accuracy.  Asserted per sigma:
  * FP64 mode: relative error <= 1e-6 for every sigma (spreads up to 1e4);
  * mixed mode: <= 1e-4 for every sigma >= 3e-4 sigma_1, and below that the
    mode's stated envelope: its refinement products carry about 39 bits
    (five 8-bit slices), so the error of sigma_i grows as (sigma_1/sigma_i)^2:
    <= 1e-4 (3e-4 sigma_1 / sigma_i)^2.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2009_09767_gb300 as rk
from tests._metrics import subspace_check

pytestmark = pytest.mark.gpu

M, N, D = 96, 4000, 4


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    rk.load_library()
    torch.cuda.set_device(0)


def _known(p, seed):
    rng = np.random.default_rng(seed)
    Q1, _ = np.linalg.qr(rng.standard_normal((M, M)))
    Q2, _ = np.linalg.qr(rng.standard_normal((N, M)))
    s = np.logspace(0, -p, M)
    A = (Q1 * s[None, :]) @ Q2.T
    col_ptr = np.arange(0, M * (N + 1), M, dtype=np.int64)
    row_idx = np.tile(np.arange(M, dtype=np.int32), N)
    vals = np.ascontiguousarray(A.T).reshape(-1)          # column-major: CSC of a dense matrix
    return s, Q1, col_ptr, row_idx, vals


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_spread_against_closed_form(precision, p):
    s_true, Q1, col_ptr, row_idx, vals = _known(p, 300 + p)
    dev = torch.device("cuda")
    t = [torch.from_numpy(a).to(dev) for a in (col_ptr, row_idx, vals)]
    plan, res = rk.svd(*t, M, N, D, precision=precision)
    s = res["sigma"].cpu().numpy()
    U = res["U"].cpu().numpy()
    plan.free()
    rel = np.abs(s - s_true) / s_true
    print(f"\nspread 1e{p}, {precision}: max relative sigma error {rel.max():.2e} "
          f"(at sigma = {s_true[int(rel.argmax())]:.1e})")
    if precision == "fp64":
        tol = np.full(M, 1e-6)
    else:
        tol = 1e-4 * np.maximum(1.0, (3e-4 / s_true) ** 2)
    assert np.all(rel <= tol), float((rel / tol).max())
    subspace_check(U, Q1, s_true, 1e-4)
