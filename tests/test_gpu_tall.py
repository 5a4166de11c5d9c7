"""GPU parity of the tall-and-skinny entry (SVD_FLAG_TALL).

Section II's row-block form: a tall A is split into row blocks, and A^T,
which is short and fat, has those blocks as its column blocks.  The library
transposes the CSC on the device and runs the column-block path on A^T.
Compared with the oracle's SVD of A' (``oracle.svd_tall``):
- sigma within the mixed / FP64 tolerances;
- both singular subspaces within 1e-4;
- lonely flags and RandomChecker insertions, in A^T's coordinates, bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2009_09767_gb300 as rk
import synth
from tests._metrics import orthonormality, sigma_check, subspace_check

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-6, 1e-12), "mixed": (1e-4, 1e-6)}
SEED = 4242


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    rk.load_library()
    torch.cuda.set_device(0)


def _expected(case, vals64, rank_fix):
    """Lonely flags of A^T over A's row blocks and the oracle's insertions."""
    b = oracle.block_bounds(case.M, case.num_blocks)
    At = np.ascontiguousarray(oracle.densify(case.col_ptr, case.row_idx, vals64, case.M,
                                             case.N).T)
    lon, rne = oracle.lonely_dense(At, b)
    fix = lon & rne[None, :]
    patches = (oracle.random_patches(fix, b, SEED) if rank_fix == "random"
               else np.zeros((0, 2), dtype=np.int64))
    return lon, fix, patches


def _tensors(case, vdtype):
    dev = torch.device("cuda")
    return (torch.from_numpy(case.col_ptr).to(dev), torch.from_numpy(case.row_idx).to(dev),
            torch.from_numpy(np.ascontiguousarray(case.vals.astype(vdtype))).to(dev))


@pytest.mark.parametrize("precision,vdtype", [("fp64", np.float64), ("mixed", np.float32)])
@pytest.mark.parametrize("rank_fix", ["truncate", "random"])
def test_tall_against_oracle(precision, vdtype, rank_fix):
    case = synth.tall_skinny()
    vals64 = case.vals.astype(vdtype).astype(np.float64)
    plan, out = rk.svd(*_tensors(case, vdtype), case.M, case.N, case.num_blocks,
                       precision=precision, rank_fix=rank_fix, seed=SEED, flags=rk.FLAG_TALL)
    lon, fix, expect = _expected(case, vals64, rank_fix)
    assert (plan.query(rk.Q_LONELY).astype(bool) == lon).all()
    assert int(fix.sum()) == 10
    assert out["patches"].cpu().numpy().tolist() == expect.tolist()
    s_ref, U_ref, V_ref, sweeps = oracle.svd_tall(case.col_ptr, case.row_idx, vals64, case.M,
                                                  case.N, expect)
    assert sweeps > 0
    rel_tol, abs_tol = TOL[precision]
    s = out["sigma"].cpu().numpy()
    U = out["U"].cpu().numpy().astype(np.float64)    # M x k, long side
    V = out["V"].cpu().numpy()                       # N x k, FP64
    assert U.shape == (case.M, case.N) and V.shape == (case.N, case.N)
    sigma_check(s, s_ref, rel_tol, abs_tol)
    subspace_check(V, V_ref, s_ref, 1e-4)
    subspace_check(U, U_ref, s_ref, 1e-4)
    assert orthonormality(V) < (1e-12 if precision == "fp64" else 1e-6)
    assert orthonormality(U) < (1e-10 if precision == "fp64" else 1e-5)
    # the sign rule holds on the short-side (FP64) vectors
    for i in range(V.shape[1]):
        assert V[int(np.argmax(np.abs(V[:, i]))), i] > 0
    plan.free()


def test_tall_run_host_matches_run():
    case = synth.tall_skinny()
    plan, out = rk.svd(*_tensors(case, np.float32), case.M, case.N, case.num_blocks,
                       precision="mixed", rank_fix="random", seed=SEED, flags=rk.FLAG_TALL)
    k = plan.k
    sigma = np.zeros(k)
    U = np.zeros((case.M, k), np.float32)
    Vs = np.zeros((k, case.N))                       # column-major N x k
    rank = np.zeros(1, np.int32)
    patches = np.zeros((plan.D * plan.Ms, 2), np.int64)
    npatches = np.zeros(1, np.int64)
    plan.run_host(case.col_ptr, case.row_idx, case.vals.astype(np.float32), sigma, U, Vs, rank,
                  patches, npatches)
    assert np.array_equal(sigma, out["sigma"].cpu().numpy())
    assert np.array_equal(U, out["U"].cpu().numpy())
    assert np.array_equal(Vs.T, out["V"].cpu().numpy())
    assert int(npatches[0]) == 10
    plan.free()


def test_tall_plan_rejected_by_batches():
    case = synth.tall_skinny()
    plan = rk.Plan(case.M, case.N, case.nnz, case.num_blocks, flags=rk.FLAG_TALL)
    with pytest.raises(rk.RankyError):
        rk.Batch([plan])
    plan.free()
