"""The tree (multi-level) merge: merge_arity >= 2.

Section II of the paper describes the multi-level merge of Iwen and Ong, of
which section III's one-level proxy (Fig. 1) is the special case: a node's
matrix is the sum of its children's Y^T Y (Y = S U^T, the children's proxy
columns), so with every direction kept each level reproduces the cross
product of its columns exactly (Eqs. 2-3) and the root's SVD is A's.  Checked:
  * against the CPU oracle's SVD of A (sigma 1e-6 FP64 / 1e-4 mixed relative,
    subspaces 1e-4) for arities 2, 4 and 8 over 8 and 64 row-skewed blocks;
  * equal to the one-level merge's result;
  * the approximate mode (k' < rank): every returned eigenvalue of A A^T
    lies below the true one and above it minus the mass the truncation
    dropped, |A|_F^2 - sum_i sigma_i^2 (Weyl: the dropped parts are positive
    semi-definite);
  * the plan is smaller by the proxy it never forms, and batches reject it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2009_09767_gb300 as rk
import synth
from tests._metrics import sigma_check, subspace_check

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-6, 1e-12), "mixed": (1e-4, 1e-6)}


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    rk.load_library()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def skewed():
    """A row-skewed matrix of the large workload's family at a size the dense
    oracle handles: 192 x 24000, ~10 entries per column, Zipf(0.8) rows,
    16 rows zeroed inside every 5th block (64 lognormal blocks)."""
    c = synth.large_skewed(M=192, N=24_000, D=64, k=192)
    s, U, V, _ = oracle.svd_csc(c.col_ptr, c.row_idx, c.vals.astype(np.float64), c.M, c.N)
    return c, s, U


def _run(case, D, precision, **kw):
    dev = torch.device("cuda")
    t = [torch.from_numpy(a).to(dev) for a in (case.col_ptr, case.row_idx, case.vals)]
    plan, res = rk.svd(*t, case.M, case.N, D, precision=precision, flags=rk.FLAG_SKIP_V, **kw)
    out = res["sigma"].cpu().numpy(), res["U"].cpu().numpy()
    plan.free()
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("D,arity", [(8, 2), (64, 2), (64, 4), (64, 8)])
def test_tree_merge_matches_oracle(skewed, precision, D, arity):
    case, s_ref, U_ref = skewed
    s, U = _run(case, D, precision, merge_arity=arity)
    sigma_check(s, s_ref, *TOL[precision])
    subspace_check(U, U_ref, s_ref, 1e-4)
    s_flat, U_flat = _run(case, D, precision)
    sigma_check(s, s_flat, *TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tree_truncated_bounds(skewed, precision):
    case, s_ref, _ = skewed
    kprime = 48
    s, _ = _run(case, 64, precision, merge_arity=4, merge_rank=kprime, k=kprime)
    lam, lam_ref = s ** 2, s_ref[:kprime] ** 2
    dropped = oracle.frobenius_sq(case.vals) - float(lam.sum())
    assert dropped >= -1e-9 * lam_ref[0]
    slack = 1e-6 * lam_ref[0]
    assert np.all(lam <= lam_ref + slack)
    assert np.all(lam >= lam_ref - dropped - slack)
    # and it is an approximation: something was dropped at k' = 48 < rank
    assert dropped > 1e-6 * lam_ref[0]


def test_tree_plan_smaller_and_batches_reject():
    """1024 x 8e6 with 256 blocks (the large workload's shape): the tree plan
    needs at least M * R * 8 bytes less than the one-level plan."""
    kw = dict(M=1024, N=8_000_000, nnz=80_000_000, num_blocks=256, k=100, precision="mixed")
    flat = rk.plan_bytes(**kw)
    tree = rk.plan_bytes(**kw, merge_arity=4)
    assert flat - tree >= 1024 * 256 * 1024 * 8
    c = synth.batch_matrix(40, 3000, 0.02, seed=5)
    p = rk.Plan(c.M, c.N, c.nnz, 4, value_type="f32", precision="mixed", merge_arity=2)
    with pytest.raises(rk.RankyError) as e:
        rk.Batch([p])
    assert e.value.status == 8
    p.free()
