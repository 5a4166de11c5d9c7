"""Synthetic stand-in for the paper's experiment (section IV, Tables I-III).

The paper runs the column-block SVD on a private 539 x 170897 job-candidate
matrix, splits it into 2 to 128 blocks (Table I), fixes lonely nodes with
RandomChecker, NeighborChecker and neighbourRandomChecker, and reports
e_sigma = sum |sigma_hat - sigma| and e_u = sum |u_hat - u| over all 539
triplets.  Here the matrix is a seeded 0/1 pattern of the same shape.  The
paper gives no density, so two are used: 0.0005, where half of the
(block, row) pairs at 128 blocks are lonely, and 0.002.  Each insertion list
is the oracle's and must equal the CUDA path's bit for bit.  The truth is
the SVD of the patched matrix A' from its exactly formed integer cross
product; the paper's truth is the same SVD of A', through LAPACK.

Reported per (density, blocks, rank fix, precision):
- e_sigma and e_u in the paper's form (u_hat sign-aligned with u);
- the largest relative sigma error;
- the largest principal-angle sine (projectors inside sigma clusters);
- the largest eigen-residual |A'A'^T u_hat - sigma_hat^2 u_hat| / sigma_1^2 against
  the exact cross product.
The dataset is missing, so the values are not comparable to the paper's
tables.

Asserted, for both precisions:
- sigma within 1e-6 (FP64) / 1e-4 (mixed) relative;
- the largest principal-angle sine within 1e-4 (projectors inside sigma
  clusters), the stated tolerance of both modes;
- the eigen-residual within 1e-11 (FP64) / 1e-6 (mixed) of sigma_1^2 (a backstop:
  the observed mixed values are 1e-10 to 5e-8).
The mixed mode meets the angle bound on the dense blocks of these patterns
(many close or exactly repeated block eigenvalues) through the Rayleigh-Ritz
rotation inside clusters of strongly mixed pairs in each of its two
refinement steps; a first-order step alone left angles up to 5e-4 here.
Every case runs before the assertions, so one run prints the whole table.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2009_09767_gb300 as rk
import synth
from tests._metrics import subspace_check

pytestmark = pytest.mark.gpu

BLOCKS = (2, 3, 4, 8, 10, 16, 32, 64, 128)    # Table I's block counts
DENSITIES = (0.0005, 0.002)
MODES = ("truncate", "random", "neighbor", "neighbor_random")
SEED = 170897
TOL = {"fp64": 1e-6, "mixed": 1e-4}
RESID_TOL = {"fp64": 1e-11, "mixed": 1e-6}
ANGLE_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    rk.load_library()
    torch.cuda.set_device(0)


def paper_errors(s, U, s_ref, U_ref):
    """e_sigma and e_u in the paper's form; each u_hat takes the sign that
    aligns it with u (singular vectors are defined up to sign)."""
    e_sigma = float(np.abs(s - s_ref).sum())
    sg = np.where(np.sum(U * U_ref, axis=0) < 0, -1.0, 1.0)
    e_u = float(np.abs(U * sg[None, :] - U_ref).sum())
    return e_sigma, e_u


def eigen_residual(s, U, G):
    """max_i |G u_i - s_i^2 u_i| / s_1^2 for unit u_i."""
    R = G @ U - U * (s ** 2)[None, :]
    return float(np.linalg.norm(R, axis=0).max() / max(float(s[0]) ** 2, 1e-300))


def _angle(U, U_ref, s_ref):
    try:
        return subspace_check(U, U_ref, s_ref, np.inf)
    except AssertionError:  # not reached with an infinite tolerance
        return np.inf


def _run(case, D, mode, precision):
    dev = torch.device("cuda")
    t = [torch.from_numpy(a).to(dev) for a in (case.col_ptr, case.row_idx, case.vals)]
    plan, out = rk.svd(*t, case.M, case.N, D, precision=precision, rank_fix=mode, seed=SEED,
                       flags=rk.FLAG_SKIP_V)
    res = {"sigma": out["sigma"].cpu().numpy(), "U": out["U"].cpu().numpy(),
           "patches": out["patches"].cpu().numpy()}
    plan.free()
    return res


@pytest.mark.parametrize("density", DENSITIES)
def test_paper_tables_synthetic(density):
    case = synth.paper_bipartite(density)
    lines, failures = [], []
    for D in BLOCKS:
        b = oracle.block_bounds(case.N, D)
        lon, rne = oracle.lonely_sparse(case.col_ptr, case.row_idx, case.vals, case.M, b)
        fix = lon & rne[None, :]
        expect = {
            "truncate": np.zeros((0, 2), dtype=np.int64),
            "random": oracle.random_patches(fix, b, SEED),
            "neighbor": oracle.neighbor_patches_sparse(case.col_ptr, case.row_idx, case.vals,
                                                       case.M, b, fix, SEED),
            "neighbor_random": oracle.neighbor_patches_sparse(
                case.col_ptr, case.row_idx, case.vals, case.M, b, fix, SEED,
                fallback_random=True),
        }
        for mode in MODES:
            s_ref, U_ref, G = oracle.svd_gram_01(case.col_ptr, case.row_idx, case.vals, case.M,
                                                 case.N, expect[mode], return_gram=True)
            precisions = ["mixed"]
            if mode == "neighbor_random" and density == DENSITIES[-1]:
                precisions.append("fp64")
            for prec in precisions:
                res = _run(dataclasses.replace(case, num_blocks=D), D, mode, prec)
                tag = (density, D, mode, prec)
                if res["patches"].tolist() != expect[mode].tolist():
                    failures.append((tag, "insertions differ"))
                rel = float(np.max(np.abs(res["sigma"] - s_ref) / s_ref))
                ang = _angle(res["U"], U_ref, s_ref)
                resid = eigen_residual(res["sigma"], res["U"], G)
                e_s, e_u = paper_errors(res["sigma"], res["U"], s_ref, U_ref)
                if rel > TOL[prec]:
                    failures.append((tag, f"sigma relative error {rel:.2e}"))
                if resid > RESID_TOL[prec]:
                    failures.append((tag, f"eigen-residual {resid:.2e}"))
                if ang > ANGLE_TOL:
                    failures.append((tag, f"angle {ang:.2e}"))
                lines.append(f"| {density:g} | {D} | 539 x {int(np.diff(b)[0])} | {mode} | "
                             f"{int(fix.sum())} | {len(expect[mode])} | {prec} | {e_s:.3e} | "
                             f"{e_u:.3e} | {rel:.2e} | {ang:.2e} | {resid:.2e} |")
    print("\n| density | blocks | block size | rank fix | lonely | insertions | precision | "
          "e_sigma | e_u | max rel sigma err | max angle sine | max eigen-residual |")
    print("|---|---|---|---|---|---|---|---|---|---|---|---|")
    print("\n".join(lines))
    assert not failures, failures
