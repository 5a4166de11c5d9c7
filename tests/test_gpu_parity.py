"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle
on the same seeded inputs.

Tolerances (stated for the method's output against the oracle):
  FP64 mode   sigma relative error <= 1e-6, tiny sigma <= 1e-12 * sigma_1
  mixed mode  sigma relative error <= 1e-4, tiny sigma <= 1e-6 * sigma_1
  both        singular subspaces (U and V) within 1e-4 (principal-angle sine,
              projectors for clusters)
Integer work (block bounds, lonely flags, RandomChecker insertions) is
compared bit for bit.
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


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    rk.load_library()  # fails loudly when the CUDA library is not built
    torch.cuda.set_device(0)


def run_case(case, precision, rank_fix="truncate", seed=1234, vdtype=None, bounds=None, k=0):
    dev = torch.device("cuda")
    vals = case.vals if vdtype is None else case.vals.astype(vdtype)
    t_cp = torch.from_numpy(case.col_ptr).to(dev)
    t_ri = torch.from_numpy(case.row_idx).to(dev)
    t_v = torch.from_numpy(np.ascontiguousarray(vals)).to(dev)
    if bounds is None and case.widths is not None:
        bounds = np.concatenate([[0], np.cumsum(case.widths)]).astype(np.int64)
    plan, out = rk.svd(t_cp, t_ri, t_v, case.M, case.N, case.num_blocks, precision=precision,
                       rank_fix=rank_fix, seed=seed, bounds=bounds, k=k)
    res = {
        "sigma": out["sigma"].cpu().numpy(),
        "U": out["U"].cpu().numpy(),
        "V": out["V"].cpu().numpy().astype(np.float64),
        "rank": out["rank"],
        "patches": out["patches"].cpu().numpy(),
        "patch_blocks": out["patch_blocks"].cpu().numpy(),
        "plan": plan,
        "vals64": np.asarray(vals, dtype=np.float64),
    }
    return res


def oracle_for(case, res, patches=None):
    p = res["patches"] if patches is None else patches
    p = p if len(p) else None
    s, U, V, sweeps = oracle.svd_csc(case.col_ptr, case.row_idx, res["vals64"], case.M, case.N, p)
    assert sweeps > 0
    return s, U, V


def check_against_oracle(case, res, precision, k=None, patches=None):
    """patches: the insertions the oracle computed for this case (the CUDA
    path's own list is only compared with it, never fed to the oracle)."""
    rel_tol, abs_tol = TOL[precision]
    s_ref, U_ref, V_ref = oracle_for(case, res, patches)
    kk = len(res["sigma"]) if k is None else k
    sigma_check(res["sigma"], s_ref[:kk], rel_tol, abs_tol)
    sub_tol = 1e-4
    subspace_check(res["U"], U_ref[:, :kk], s_ref[:kk], sub_tol)
    # V only where sigma is above the rank tolerance
    r = res["rank"]
    subspace_check(res["V"][:, :min(r, kk)], V_ref[:, :min(r, kk)], s_ref[:min(r, kk)], sub_tol)
    assert orthonormality(res["U"]) < (1e-12 if precision == "fp64" else 1e-6)
    # sign rule on U
    for i in range(kk):
        col = res["U"][:, i]
        assert col[int(np.argmax(np.abs(col)))] > 0
    return s_ref, U_ref, V_ref


# --------------------------------------------------------------------------
# the small workload (64 x 4096, 4 blocks)

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_small_uniform(precision):
    case = synth.small_uniform()
    res = run_case(case, precision)
    s_ref, _, _ = check_against_oracle(case, res, precision)
    plan = res["plan"]
    # Algorithm 1 split, bit exact
    b = plan.query(rk.Q_BLOCK_BOUNDS)
    assert b.tolist() == oracle.block_bounds(case.N, case.num_blocks).tolist()
    # block cross products (Eq. 2) against plain summation
    A = oracle.densify(case.col_ptr, case.row_idx, case.vals, case.M, case.N)
    for d in range(case.num_blocks):
        G = plan.query(rk.Q_BLOCK_GRAM, d)
        Gr = oracle.gram_dense(A, int(b[d]), int(b[d + 1]))
        assert np.abs(G - Gr).max() <= 1e-13 * np.abs(Gr).max()
        # block singular values against the oracle SVD of the block
        sb = plan.query(rk.Q_BLOCK_SIGMA)[d]
        sref_b = oracle.svd_dense(A[:, b[d]:b[d + 1]])[0]
        sigma_check(sb[:len(sref_b)], sref_b, TOL[precision][0], 1e-7)
    # proxy identity (Eqs. 2-3): P P^T = A A^T
    P = plan.query(rk.Q_PROXY)
    AAt = A @ A.T
    scale = np.abs(AAt).max()
    # mixed: FP32 rotations with one FP64 refinement step of each block basis
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert np.abs(P @ P.T - AAt).max() <= tol * scale
    assert np.abs(plan.query(rk.Q_MERGE_GRAM) - AAt).max() <= tol * scale
    assert res["rank"] == int((s_ref > 1e-7 * s_ref[0]).sum())
    assert (plan.query(rk.Q_SWEEPS) > 0).all()
    assert plan.query(rk.Q_LAUNCHES)[0] > 5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_small_lonely_truncate(precision):
    case = synth.small_lonely()
    res = run_case(case, precision, "truncate")
    check_against_oracle(case, res, precision)
    plan = res["plan"]
    b = oracle.block_bounds(case.N, case.num_blocks)
    A = oracle.densify(case.col_ptr, case.row_idx, case.vals, case.M, case.N)
    lon_ref, rne_ref = oracle.lonely_dense(A, b)
    assert (plan.query(rk.Q_LONELY).astype(bool) == lon_ref).all()
    assert (plan.query(rk.Q_ROW_NONEMPTY).astype(bool) == rne_ref).all()
    ranks = plan.query(rk.Q_BLOCK_RANKS)
    # 8 rows zeroed inside the second block: its numerical rank drops by 8
    for d in range(case.num_blocks):
        sref_b = oracle.svd_dense(A[:, b[d]:b[d + 1]])[0]
        expect = int((sref_b > 1e-6 * sref_b[0]).sum())
        assert ranks[d] == expect, (d, ranks[d], expect)
    assert ranks[1] == 56
    assert len(res["patches"]) == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_small_lonely_random_checker(precision):
    case = synth.small_lonely()
    seed = 987654321012345
    res = run_case(case, precision, "random", seed=seed)
    b = oracle.block_bounds(case.N, case.num_blocks)
    A = oracle.densify(case.col_ptr, case.row_idx, case.vals, case.M, case.N)
    lon_ref, rne_ref = oracle.lonely_dense(A, b)
    fix = lon_ref & rne_ref[None, :]
    expect = oracle.random_patches(fix, b, seed)
    assert res["patches"].tolist() == expect.tolist()
    assert len(expect) == 8
    # each insertion lies in the lonely row's block (Algorithm 2)
    for (m, col), d in zip(res["patches"], res["patch_blocks"]):
        assert b[d] <= col < b[d + 1] and fix[d, m]
    check_against_oracle(case, res, precision, patches=expect)
    # after the fix every block has full row rank
    assert (res["plan"].query(rk.Q_BLOCK_RANKS) == case.M).all()


# --------------------------------------------------------------------------
# NeighborChecker (Algorithm 3) and neighbourRandomChecker (Algorithm 4)

def _case_bounds(case):
    if case.widths is not None:
        return np.concatenate([[0], np.cumsum(case.widths)]).astype(np.int64)
    return oracle.block_bounds(case.N, case.num_blocks)


@pytest.mark.parametrize("precision,vdtype", [("fp64", None), ("mixed", None),
                                              ("mixed", np.float32)])
@pytest.mark.parametrize("mode", ["neighbor", "neighbor_random"])
def test_neighbor_checkers(precision, vdtype, mode):
    """Both outcomes of the neighbour fix on one matrix: lonely rows with a
    neighbour list, lonely rows without one (no insertion, or RandomChecker's
    column), long columns, stored zeros, ragged block widths."""
    case = synth.neighbor_mix()
    seed = 0x5EED00012345
    res = run_case(case, precision, mode, seed=seed, vdtype=vdtype)
    b = _case_bounds(case)
    A = oracle.densify(case.col_ptr, case.row_idx, case.vals, case.M, case.N)
    lon, rne = oracle.lonely_dense(A, b)
    fix = lon & rne[None, :]
    expect = oracle.neighbor_patches(A, b, fix, seed, fallback_random=(mode == "neighbor_random"))
    assert res["patches"].tolist() == expect.tolist()
    if mode == "neighbor":
        assert 0 < len(expect) < int(fix.sum())
    else:
        assert len(expect) == int(fix.sum())
    blocks = np.searchsorted(b, expect[:, 1], side="right") - 1
    assert res["patch_blocks"].tolist() == blocks.tolist()
    check_against_oracle(case, res, precision, patches=expect)


def test_neighbor_checker_small_lonely():
    """Every lonely row of small_lonely has neighbours: eight insertions,
    each block at full row rank afterwards."""
    case = synth.small_lonely()
    seed = 31337
    res = run_case(case, "mixed", "neighbor", seed=seed)
    b = oracle.block_bounds(case.N, case.num_blocks)
    A = oracle.densify(case.col_ptr, case.row_idx, case.vals, case.M, case.N)
    lon, rne = oracle.lonely_dense(A, b)
    expect = oracle.neighbor_patches(A, b, lon & rne[None, :], seed)
    assert len(expect) == 8
    assert res["patches"].tolist() == expect.tolist()
    check_against_oracle(case, res, "mixed", patches=expect)
    assert (res["plan"].query(rk.Q_BLOCK_RANKS) == case.M).all()


def test_neighbor_random_zipf_scaled():
    """zipf_wide's shape at a quarter of its columns (512 x 250000, 64
    blocks of 3906, ~750 lonely nodes): every insertion bit for bit against the
    closed-form evaluation of the neighbour lists, the leading triplets by
    their residuals against A'."""
    case = synth.zipf_wide(M=512, N=250_000, D=64, target_nnz=128_000)
    seed = 2009
    res = run_case(case, "mixed", "neighbor_random", seed=seed)
    b = oracle.block_bounds(case.N, case.num_blocks)
    lon, rne = oracle.lonely_sparse(case.col_ptr, case.row_idx, case.vals, case.M, b)
    fix = lon & rne[None, :]
    expect = oracle.neighbor_patches_sparse(case.col_ptr, case.row_idx, case.vals, case.M, b,
                                            fix, seed, fallback_random=True)
    assert len(expect) == int(fix.sum()) > 0
    assert res["patches"].tolist() == expect.tolist()
    k = 8
    r = oracle.residuals(case.col_ptr, case.row_idx, res["vals64"], case.M, res["sigma"][:k],
                         res["U"][:, :k], res["V"][:, :k], patches=expect)
    assert (r <= 1e-4 * res["sigma"][0]).all(), r


# --------------------------------------------------------------------------
# ragged shapes, degenerate cases

def _random_case(M, N, density, D, seed, dtype=np.float64, empty_rows=(), name="ragged"):
    rng = np.random.default_rng(seed)
    c = synth.random_dense_csc(rng, M, N, density, dtype=dtype, name=name)
    c.num_blocks = D
    if len(empty_rows):
        c = synth.zero_rows_in_columns(c, list(empty_rows), 0, N)
    return c


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("M,N,D,density", [
    (50, 700, 3, 0.05),      # M not a multiple of the tile, N mod D != 0
    (100, 999, 7, 0.03),     # several sub-problem pairs, remainder block
    (200, 3000, 5, 0.02),    # Mp = 256: 4 pairs per step
    (33, 40, 40, 0.3),       # one column per block
    (7, 19, 2, 0.5),
    (1, 10, 3, 0.5),         # a single row
])
def test_ragged_shapes(precision, M, N, D, density):
    case = _random_case(M, N, density, D, seed=M * 1000 + N)
    res = run_case(case, precision)
    check_against_oracle(case, res, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_globally_empty_rows_and_k(precision):
    case = _random_case(40, 500, 0.05, 4, seed=7, empty_rows=(3, 17, 39))
    res = run_case(case, precision, k=30)
    s_ref, _, _ = check_against_oracle(case, res, precision, k=30)
    full = run_case(case, precision)
    assert full["rank"] == 37  # three rows empty in all of A
    assert np.abs(full["sigma"][37:]).max() == 0.0
    assert np.abs(full["V"][:, 37:]).max() == 0.0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_all_zero_matrix(precision):
    M, N = 16, 64
    case = synth.CscCase("zero", M, N, np.zeros(N + 1, np.int64), np.zeros(0, np.int32),
                         np.zeros(0, np.float64), 2)
    res = run_case(case, precision)
    assert res["rank"] == 0
    assert np.abs(res["sigma"]).max() == 0.0
    assert np.abs(res["V"]).max() == 0.0
    assert orthonormality(res["U"]) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_explicit_widths_and_f32_values(precision):
    case = _random_case(64, 2000, 0.02, 4, seed=11, dtype=np.float32)
    bounds = np.array([0, 100, 1100, 1500, 2000], np.int64)
    res = run_case(case, precision, bounds=bounds)
    assert res["plan"].query(rk.Q_BLOCK_BOUNDS).tolist() == bounds.tolist()
    check_against_oracle(case, res, precision)


def test_run_host_matches_run():
    case = synth.small_uniform()
    dev = torch.device("cuda")
    plan = rk.Plan(case.M, case.N, case.nnz, case.num_blocks, value_type="f64", precision="fp64")
    out = rk.alloc_outputs(plan)
    plan.run(torch.from_numpy(case.col_ptr).to(dev), torch.from_numpy(case.row_idx).to(dev),
             torch.from_numpy(case.vals).to(dev), out["sigma"], out["U"], out["V"], out["rank"],
             out["patches"], out["npatches"])
    plan.sync()
    hs = np.zeros(plan.k)
    hU = np.zeros((plan.k, plan.M))
    hV = np.zeros((plan.N, plan.k))
    hr = np.zeros(1, np.int32)
    plan.run_host(case.col_ptr, case.row_idx, case.vals, hs, hU, hV, hr)
    # the cross products accumulate with atomics: equal up to summation order
    np.testing.assert_allclose(hs, out["sigma"].cpu().numpy(), rtol=1e-12)
    assert np.abs(np.abs(hU.T.T @ out["U"].cpu().numpy().T).diagonal() - 1).max() < 1e-10
    np.testing.assert_allclose(np.abs(hV), np.abs(out["V"].cpu().numpy()), rtol=0, atol=1e-10)
    assert hr[0] == out["rank"].item()


def test_run_host_writes_pinned_v_directly():
    """A page-locked V buffer is written by the device in place (no staging
    copy); the result equals the device-buffer run."""
    case = synth.small_uniform().with_values(np.float32)
    dev = torch.device("cuda")
    plan = rk.Plan(case.M, case.N, case.nnz, case.num_blocks, value_type="f32", precision="mixed")
    out = rk.alloc_outputs(plan, with_patches=False)
    plan.run(torch.from_numpy(case.col_ptr).to(dev), torch.from_numpy(case.row_idx).to(dev),
             torch.from_numpy(case.vals).to(dev), out["sigma"], out["U"], out["V"], out["rank"])
    plan.sync()
    hs = torch.zeros(plan.k, dtype=torch.float64).pin_memory()
    hU = torch.zeros(plan.k, plan.M, dtype=torch.float64).pin_memory()
    hV = torch.full((plan.N, plan.k), float("nan"), dtype=torch.float32).pin_memory()
    hr = torch.zeros(1, dtype=torch.int32).pin_memory()
    plan.run_host(case.col_ptr, case.row_idx, case.vals, hs, hU, hV, hr)
    assert torch.isfinite(hV).all()                 # every entry was written
    np.testing.assert_allclose(hs.numpy(), out["sigma"].cpu().numpy(), rtol=1e-9)
    np.testing.assert_allclose(np.abs(hV.numpy()), np.abs(out["V"].cpu().numpy()), rtol=0, atol=1e-5)
    assert hr[0].item() == out["rank"].item()


def test_check_csc_rejects_malformed():
    lib = rk.load_library()
    dev = torch.device("cuda")
    good_cp = torch.tensor([0, 2, 3], dtype=torch.int64, device=dev)
    good_ri = torch.tensor([0, 2, 1], dtype=torch.int32, device=dev)
    s = rk._stream_handle(None)
    assert lib.svd_check_csc(3, 2, 3, rk._ptr(good_cp), rk._ptr(good_ri), s) == 0
    unsorted = torch.tensor([2, 0, 1], dtype=torch.int32, device=dev)
    assert lib.svd_check_csc(3, 2, 3, rk._ptr(good_cp), rk._ptr(unsorted), s) == 2
    out_of_range = torch.tensor([0, 3, 1], dtype=torch.int32, device=dev)
    assert lib.svd_check_csc(3, 2, 3, rk._ptr(good_cp), rk._ptr(out_of_range), s) == 2
    bad_end = torch.tensor([0, 2, 4], dtype=torch.int64, device=dev)
    assert lib.svd_check_csc(3, 2, 3, rk._ptr(bad_end), rk._ptr(good_ri), s) == 2


@pytest.mark.parametrize("vdtype", [np.float64, np.float32])
def test_sparse_block_refinement(vdtype):
    """Mixed precision on a very sparse matrix: the block refinement forms
    G X^T from the sparse columns (100 nnz < D Mp^2 here); forcing the dense
    cross product instead must give the same spectrum and subspaces."""
    case = _random_case(150, 400000, 0.00002, 16, seed=77, name="very_sparse")
    Mp = 160
    assert 100 * case.nnz < case.num_blocks * Mp * Mp
    res = run_case(case, "mixed", vdtype=vdtype)
    s_ref, _, _ = check_against_oracle(case, res, "mixed")
    dev = torch.device("cuda")
    vals = torch.from_numpy(np.ascontiguousarray(case.vals.astype(vdtype))).to(dev)
    _, dense = rk.svd(torch.from_numpy(case.col_ptr).to(dev), torch.from_numpy(case.row_idx).to(dev),
                      vals, case.M, case.N, case.num_blocks, precision="mixed",
                      flags=rk.FLAG_DENSE_REFINE)
    sd = dense["sigma"].cpu().numpy()
    sigma_check(res["sigma"], sd, 1e-9, 1e-9 * sd[0])
    subspace_check(res["U"], dense["U"].cpu().numpy(), sd, 1e-6)
