"""The FP64-accurate tensor-core product (svd_exact_product), which forms the
merge's P P^T (section III, Eq. 3) and the products of the mixed-precision
refinement.

Two independent checks:
  * the tcgen05 kernel (TMEM accumulators) and the mma.sync kernel form the
    same exact integer sums and convert them once, so their results must be
    equal bit for bit, whatever the shapes (ragged m, n, k; k above the
    1024-deep exact run, so several accumulator drains; one slice count and
    the other; the symmetric form; grids of under and over two CTAs per SM);
  * against the FP64 product A B^T computed by numpy, the error stays within
    the splitting's bound 2^(3 - 8 S) k 2^(e_i + e_j) (e_i: the exponent bound
    of row i), with rows spanning six orders of magnitude and a zero row.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2009_09767_gb300 as rk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    rk.load_library()
    torch.cuda.set_device(0)


def _operand(rng, rows, k):
    X = rng.standard_normal((rows, k)) * (10.0 ** rng.uniform(-3, 3, size=(rows, 1)))
    if rows > 2:
        X[rows // 2] = 0.0
    return X


def _exp_bound(X):
    amax = np.abs(X).max(axis=1)
    e = np.frexp(amax)[1].astype(np.float64)   # amax < 2^e
    e[amax == 0] = 0
    return e


CASES = [  # m, n, k, slices
    (128, 32, 64, 5), (200, 77, 300, 5), (512, 512, 512, 5), (300, 130, 2500, 5),
    (64, 96, 40, 3), (1, 1, 1, 5), (257, 33, 1031, 3), (130, 500, 4096, 5),
    (200, 256, 1100, 3),
    # grids of several hundred tiles (two CTAs per SM share the device)
    (2048, 2048, 512, 5), (1100, 2300, 600, 3),
]


@pytest.mark.parametrize("m,n,k,S", CASES)
def test_tcgen05_equals_mma_sync_and_bound(m, n, k, S):
    rng = np.random.default_rng(1000 * m + n + k + S)
    A = _operand(rng, m, k)
    B = _operand(rng, n, k)
    dev = torch.device("cuda")
    tA, tB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    C_tc = rk.exact_product(tA, tB, slices=S, err=err).cpu().numpy()
    C_mma = rk.exact_product(tA, tB, slices=S, legacy=True).cpu().numpy()
    assert int(err.item()) == 0
    assert np.array_equal(C_tc, C_mma), float(np.abs(C_tc - C_mma).max())
    ref = A @ B.T
    bound = 2.0 ** (3 - 8 * S) * k * np.exp2(_exp_bound(A)[:, None] + _exp_bound(B)[None, :])
    assert np.all(np.abs(C_tc - ref) <= bound), float((np.abs(C_tc - ref) / bound).max())


@pytest.mark.parametrize("m,k,S", [(384, 700, 5), (513, 1100, 3), (96, 64, 5)])
def test_symmetric_product(m, k, S):
    rng = np.random.default_rng(7 * m + k)
    A = _operand(rng, m, k)
    tA = torch.from_numpy(A).to("cuda")
    C_tc = rk.exact_product(tA, slices=S).cpu().numpy()
    C_mma = rk.exact_product(tA, slices=S, legacy=True).cpu().numpy()
    assert np.array_equal(C_tc, C_mma)
    assert np.array_equal(C_tc, C_tc.T)
    ref = A @ A.T
    e = _exp_bound(A)
    bound = 2.0 ** (3 - 8 * S) * k * np.exp2(e[:, None] + e[None, :])
    assert np.all(np.abs(C_tc - ref) <= bound)


def test_svd_same_with_either_tensor_path():
    """The mixed-precision SVD through either product kernel: the products are
    identical, so sigma agrees to the rounding of the non-deterministic
    summation order of the cross products (1e-9 relative)."""
    import synth
    case = synth.small_uniform().with_values(np.float32)
    dev = torch.device("cuda")
    t = [torch.from_numpy(a).to(dev) for a in (case.col_ptr, case.row_idx, case.vals)]
    out = {}
    for name, flags in (("tc", 0), ("mma", rk.FLAG_LEGACY_MMA)):
        plan, res = rk.svd(*t, case.M, case.N, case.num_blocks, precision="mixed", flags=flags)
        out[name] = res["sigma"].cpu().numpy()
        plan.free()
    s = out["mma"]
    big = s > 1e-10 * s[0]
    assert np.max(np.abs(out["tc"][big] - s[big]) / s[big]) <= 1e-9
