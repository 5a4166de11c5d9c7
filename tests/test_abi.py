"""C-ABI checks that need no GPU: the library loads, exports every function
the header declares, the Python structures match the C layout, and the
host-side argument validation answers as documented."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2009_09767_gb300 as rk
from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "ranky.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2009_09767_gb300 import _build
    _build.build()
    return rk.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    # a declaration: return type (any, with const and pointers), then the name
    names = re.findall(r"^\s*(?:const\s+)?\w+[\s*]+(svd_\w+)\s*\(", text, flags=re.M)
    # every svd_ name followed by an argument list is such a declaration
    assert set(names) == set(re.findall(r"\b(svd_\w+)\s*\(", text))
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    for n in ("svd_plan", "svd_run", "svd_free", "svd_exact_product_bytes",
              "svd_right_vectors_static"):
        assert n in names, n
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for code in range(9):
        s = lib.svd_status_str(code)
        assert s and s != b"unknown status"
    assert lib.svd_status_str(99) == b"unknown status"
    assert lib.svd_version() >= 1


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(f'''
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",
    sizeof(svd_desc), offsetof(svd_desc, N), offsetof(svd_desc, nnz),
    offsetof(svd_desc, value_type), offsetof(svd_desc, num_blocks),
    offsetof(svd_desc, block_col_bounds), offsetof(svd_desc, k),
    offsetof(svd_desc, precision), offsetof(svd_desc, rank_fix), offsetof(svd_desc, seed),
    offsetof(svd_desc, rank_tol), offsetof(svd_desc, max_sweeps),
    offsetof(svd_desc, jacobi_tol), offsetof(svd_desc, refine_iters),
    offsetof(svd_desc, flags), offsetof(svd_desc, merge_arity),
    offsetof(svd_desc, jacobi_cluster), offsetof(svd_desc, merge_rank), sizeof(svd_patch));
  return 0;
}}''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-o", str(exe), str(src)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    D = rk.SvdDesc
    expect = [ctypes.sizeof(D), D.N.offset, D.nnz.offset, D.value_type.offset,
              D.num_blocks.offset, D.block_col_bounds.offset, D.k.offset, D.precision.offset,
              D.rank_fix.offset, D.seed.offset, D.rank_tol.offset, D.max_sweeps.offset,
              D.jacobi_tol.offset, D.refine_iters.offset, D.flags.offset,
              D.merge_arity.offset, D.jacobi_cluster.offset, D.merge_rank.offset,
              ctypes.sizeof(rk.SvdPatch)]
    assert got == expect


def _bytes(lib, **kw):
    d, keep = rk.make_desc(**kw)
    out = ctypes.c_size_t(0)
    st = lib.svd_plan_bytes(ctypes.byref(d), ctypes.byref(out))
    return st, out.value


def test_plan_bytes_validation(lib):
    ok = dict(M=64, N=4096, nnz=100, num_blocks=4)
    st, n = _bytes(lib, **ok)
    assert st == 0 and n > 0
    st2, n2 = _bytes(lib, **{**ok, "num_blocks": 8})
    assert st2 == 0 and n2 > n
    bad = [
        {**ok, "M": 0}, {**ok, "N": 0}, {**ok, "nnz": -1}, {**ok, "num_blocks": 0},
        {**ok, "num_blocks": 5000}, {**ok, "k": 65}, {**ok, "k": -1},
        {**ok, "value_type": 7}, {**ok, "precision": 5}, {**ok, "rank_fix": 9},
        {**ok, "bounds": [0, 10, 10, 20, 4096]}, {**ok, "bounds": [1, 10, 20, 30, 4096]},
        {**ok, "bounds": [0, 10, 20, 30, 4095]},
    ]
    for kw in bad:
        assert _bytes(lib, **kw)[0] == 1, kw
    assert _bytes(lib, **{**ok, "M": 1025})[0] == 8
    # the neighbour modes carry their own workspace (M x M counts, one slot per lonely node)
    st3, n3 = _bytes(lib, **{**ok, "rank_fix": "neighbor"})
    assert st3 == 0 and n3 > n
    assert _bytes(lib, **{**ok, "rank_fix": "neighbor_random"}) == (0, n3)
    assert _bytes(lib, **{**ok, "bounds": [0, 1, 2, 3, 4096]})[0] == 0


def test_tall_plan_bytes_validation(lib):
    """SVD_FLAG_TALL: M is the long side (any), N <= 1024, row blocks over M."""
    tall = dict(M=100_000, N=96, nnz=5000, num_blocks=8, flags=rk.FLAG_TALL)
    st, n = _bytes(lib, **tall)
    assert st == 0 and n > 0
    # the transpose buffers: the same problem stated short and fat needs less
    st2, n2 = _bytes(lib, **{**tall, "M": 96, "N": 100_000, "flags": 0})
    assert st2 == 0 and n > n2
    assert _bytes(lib, **{**tall, "N": 1025})[0] == 8          # short side above 1024
    assert _bytes(lib, **{**tall, "num_blocks": 100_001})[0] == 1
    assert _bytes(lib, **{**tall, "k": 97})[0] == 1
    assert _bytes(lib, **{**tall, "bounds": [0] + [12_500 * i for i in range(1, 8)] +
                          [100_000]})[0] == 0
    assert _bytes(lib, **{**tall, "bounds": [0] + [12_500 * i for i in range(1, 8)] +
                          [96]})[0] == 1


def test_tree_plan_bytes(lib):
    """The tree merge (section II's multi-level proxy merge) never forms the
    one-level proxy P (M x R, R up to D*M): at the large workload's shape the
    tree plan needs at least M*M*D*8 bytes less than the one-level plan, for
    every D, and its size does not grow with the number of levels (arity)."""
    for D in (64, 256, 512):
        kw = dict(M=1024, N=8_000_000, nnz=80_000_000, num_blocks=D, k=100, precision="mixed")
        st, flat = _bytes(lib, **kw)
        assert st == 0
        trees = []
        for arity in (2, 4, 16):
            st, t = _bytes(lib, **kw, merge_arity=arity)
            assert st == 0
            trees.append(t)
        assert flat - trees[0] >= 1024 * 1024 * D * 8
        assert len(set(trees)) == 1
        # a per-node rank cap k' >= k changes nothing in the workspace either
        assert _bytes(lib, **kw, merge_arity=4, merge_rank=200) == (0, trees[0])
    small = dict(M=64, N=4096, nnz=100, num_blocks=4, k=32)
    # arity 0 and 1 are the one-level merge of section III
    assert _bytes(lib, **small, merge_arity=1) == _bytes(lib, **small)
    for kw in ({"merge_arity": -1}, {"merge_rank": -1}, {"merge_rank": 31}):
        assert _bytes(lib, **small, **kw)[0] == 1, kw


def test_null_plan_is_rejected(lib):
    assert lib.svd_sync(None) == 1
    assert lib.svd_query(None, 1, 0, None, 0) == 1
    lib.svd_free(None)
