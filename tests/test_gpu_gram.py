"""Block cross products A^i A^i^T (Eq. 2) against plain summation by the
oracle, on a ragged M (padding rows) in both precisions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2009_09767_gb300 as rk
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    rk.load_library()
    torch.cuda.set_device(0)


def _grams(case, D, precision, flags):
    dev = torch.device("cuda")
    t = [torch.from_numpy(a).to(dev) for a in (case.col_ptr, case.row_idx, case.vals)]
    plan, _ = rk.svd(*t, case.M, case.N, D, precision=precision, flags=flags | rk.FLAG_SKIP_V)
    G = [plan.query(rk.Q_BLOCK_GRAM, d) for d in range(D)]
    plan.free()
    return G


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_cluster_gram_against_summation(precision):
    rng = np.random.default_rng(31)
    case = synth.random_dense_csc(rng, 100, 3000, 0.05)
    D = 3
    b = oracle.block_bounds(case.N, D)
    A = oracle.densify(case.col_ptr, case.row_idx, case.vals, case.M, case.N)
    for d, G in enumerate(_grams(case, D, precision, 0)):
        Gr = oracle.gram_dense(A, int(b[d]), int(b[d + 1]))
        assert np.abs(G - Gr).max() <= 1e-13 * np.abs(Gr).max()
