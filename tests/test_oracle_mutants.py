"""Plant plausible mistakes in a temporary copy of the oracle (CPU only) and
check that the pins catch every one of them."""
import ctypes
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (original text, planted mistake)
MUTANTS = {
    "rotation_sign": ("wq[n] = s * a + c * b;", "wq[n] = s * a - c * b;"),
    "dropped_gamma_term": ("gamma += wp[n] * wq[n];", "gamma += (n > 0) * wp[n] * wq[n];"),
    "zeta_sign": ("double zeta = (beta - alpha)", "double zeta = (alpha - beta)"),
    "u_accumulation_index": ("Q[(int64_t)r * M + q] = s * a + c * b;",
                             "Q[(int64_t)r * M + p] = s * a + c * b;"),
    "sign_rule_missing": ("double sg = Q[(int64_t)arg * M + src] < 0.0 ? -1.0 : 1.0;",
                          "double sg = 1.0;"),
    "v_unscaled": ("V[n * M + i] = si > 0.0 ? sg * ws[n] / si : 0.0;",
                   "V[n * M + i] = si > 0.0 ? sg * ws[n] : 0.0;"),
    "sort_ascending": ("nrm[order[j]] < nrm[k]", "nrm[order[j]] > nrm[k]"),
    "philox_key_bump": ("k1 += W1;", "k1 += W0;"),
    "lonely_bound": ("for (int64_t n = bounds[d]; n < bounds[d + 1]; ++n)",
                     "for (int64_t n = bounds[d]; n + 1 < bounds[d + 1]; ++n)"),
    "neighbor_own_block": ("if (d1 == d) continue;", "if (d1 == d && 0) continue;"),
    "neighbor_block_range": ("for (int64_t n2 = bounds[d]; n2 < bounds[d + 1]; ++n2)",
                             "for (int64_t n2 = 0; n2 < bounds[d + 1]; ++n2)"),
    "neighbor_unsorted": ("if (nbr.n > 1) qsort(", "if (nbr.n > 1 && 0) qsort("),
    "neighbor_draw_words": ("(uint64_t)w[0] | ((uint64_t)w[1] << 32)",
                            "(uint64_t)w[1] | ((uint64_t)w[0] << 32)"),
    "neighbor_mulhi_carry": ("(p10 >> 32) + (mid >> 32);", "(p10 >> 32);"),
    "gram_transposed": ("s += A[(int64_t)i * N + n] * A[(int64_t)j * N + n];",
                        "s += A[(int64_t)i * N + n] * A[(int64_t)n * N + j];"),
}

PINS = [
    pins.test_philox_known_answers,
    pins.test_lonely_worked_example,
    pins.test_lonely_multiblock_constructed,
    pins.test_lonely_sparse_equals_dense,
    pins.test_gram_dense_against_matmul_and_sum,
    pins.test_permuted_diagonal,
    pins.test_rank_one,
    pins.test_rank_r_disjoint_supports,
    pins.test_known_sigma_householder_products,
    pins.test_invariants_small_uniform,
    pins.test_transposed_operand_is_caught,
    pins.test_neighbor_worked_example,
    pins.test_neighbor_list_multiplicities_closed_form,
    pins.test_neighbor_choice_against_closed_form,
    pins.test_neighbor_draw_uniform_over_entries,
    pins.test_neighbor_draw_product_exact,
]


def _build_mutant(tmp_path, name):
    text = open(SRC).read()
    old, new = MUTANTS[name]
    assert text.count(old) == 1, name
    src = tmp_path / f"{name}.c"
    src.write_text(text.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-std=c11", "-o",
                           str(so), str(src), "-lm"])
    return str(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path, monkeypatch):
    so = _build_mutant(tmp_path, name)
    real = oracle._load()
    lib = ctypes.CDLL(so)
    for fn in ("ro_philox4x32_10", "ro_random_patch_col", "ro_lonely_dense",
               "ro_gram_dense", "ro_svd_jacobi", "ro_neighbor_list",
               "ro_neighbor_patch_col", "ro_mulhi64"):
        f = getattr(lib, fn)
        f.argtypes = getattr(real, fn).argtypes
        f.restype = getattr(real, fn).restype
    monkeypatch.setattr(oracle, "_lib", lib)
    failures = 0
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError, FloatingPointError):
            failures += 1
    assert failures > 0, f"no pin caught the planted mistake {name!r}"
