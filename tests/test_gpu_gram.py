"""Block cross products A^i A^i^T (Eq. 2): the thread-block-cluster form
(packed triangle in distributed shared memory, one write of the full
matrix) against plain summation by the oracle, and against the global-atomic
form on the same input (equal up to the summation order).  Shapes: ragged M
(padding rows), heavy columns (Zipf column degrees, full columns), and
M = 1024, whose packed triangle takes several cluster passes."""
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


@pytest.mark.parametrize("name", ["zipf", "skewed1024"])
def test_cluster_gram_equals_atomic(name):
    if name == "zipf":
        case = synth.zipf_wide(N=100_000, D=6, target_nnz=51_200)
        D = 6
    else:
        case = synth.large_skewed(M=1024, N=40_000, D=4)
        D = 4
    g1 = _grams(case, D, "mixed", 0)
    g2 = _grams(case, D, "mixed", rk.FLAG_ATOMIC_GRAM)
    for a, c in zip(g1, g2):
        scale = np.abs(c).max()
        assert np.abs(a - c).max() <= 1e-13 * scale
        assert np.array_equal(a, a.T)
