"""svd_right_vectors_static: right singular vectors for callers that must not
allocate device memory (fixed-budget services, callers that cannot take
cudaMalloc's device-wide synchronisation).  Its weights live in the
library's static 4 MiB device array; its output must equal what svd_run
returns for the same matrix, call after call.

This file is named to be collected last, so that a run that stops at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2009_09767_gb300 as rk
import synth

pytestmark = pytest.mark.gpu


def _case(name):
    if name == "small_lonely":
        return synth.small_lonely()
    rng = np.random.default_rng(77)
    c = synth.random_dense_csc(rng, 512, 20000, 0.004, dtype=np.float32)
    c.num_blocks = 3
    return c


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("name,rank_fix", [("small_lonely", "random"), ("wide512", "truncate")])
def test_static_right_vectors_match_svd_run(precision, name, rank_fix):
    assert torch.cuda.is_available()
    dev = torch.device("cuda")
    case = _case(name)
    cp = torch.from_numpy(case.col_ptr).to(dev)
    ri = torch.from_numpy(case.row_idx).to(dev)
    va = torch.from_numpy(case.vals).to(dev)
    vt = "f32" if case.vals.dtype == np.float32 else "f64"
    plan = rk.Plan(case.M, case.N, case.nnz, case.num_blocks, value_type=vt,
                   precision=precision, rank_fix=rank_fix, seed=99)
    out = rk.alloc_outputs(plan, device=dev)
    plan.run(cp, ri, va, out["sigma"], out["U"], out["V"], out["rank"], out["patches"],
             out["npatches"])
    plan.sync()
    V_ref = out["V"].clone()
    if rank_fix == "random":
        assert int(out["npatches"].item()) > 0
    tol = 1e-6 if precision == "mixed" else 1e-12
    scale = float(V_ref.abs().max())
    for call in range(2):
        V = torch.full_like(V_ref, float("nan"))
        rk.right_vectors_static(case.M, case.N, cp, ri, va, out["sigma"], out["U"], V,
                                patches=out["patches"], npatches=out["npatches"],
                                max_patches=plan.D * plan.M)
        torch.cuda.synchronize()
        assert not torch.isnan(V).any(), call
        err = float((V - V_ref).abs().max())
        assert err <= tol * scale, (call, err, scale)
    plan.free()


def test_static_right_vectors_rejects_oversize():
    assert torch.cuda.is_available()
    lib = rk.load_library()
    f = lib.svd_right_vectors_static
    dev = torch.device("cuda")
    dummy = torch.zeros(8, dtype=torch.float64, device=dev)
    cp = torch.zeros(1025, dtype=torch.int64, device=dev)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    # 1024 x 1024 FP64 weights = 8 MiB > 4 MiB: rejected before any work
    st = f(1024, 1024, 0, 1, P(cp), None, None, 1024, P(dummy), P(dummy), 0.0, None, None, 0, 1,
           P(dummy), None)
    assert st == 8
    # 1024 x 1024 FP32 weights = 4 MiB: within the limit, argument check only
    st = f(1024, 1024, 0, 1, P(cp), None, None, 1024, None, P(dummy), 0.0, None, None, 0, 0,
           P(dummy), None)
    assert st == 1


@pytest.mark.parametrize("precision,k", [("mixed", 101), ("mixed", 100), ("fp64", 37)])
def test_static_right_vectors_top_k(precision, k):
    """Top-k calls: k < M, and k % 4 != 0 (the FP32 scalar SpMM path).  From
    the same sigma and U, the static entry's V equals svd_run's V of a top-k
    plan, and the first k columns of a full plan's V."""
    assert torch.cuda.is_available()
    dev = torch.device("cuda")
    case = _case("wide512")
    cp = torch.from_numpy(case.col_ptr).to(dev)
    ri = torch.from_numpy(case.row_idx).to(dev)
    va = torch.from_numpy(case.vals).to(dev)
    tol = 1e-6 if precision == "mixed" else 1e-12
    for kk in (k, None):
        plan = rk.Plan(case.M, case.N, case.nnz, case.num_blocks, value_type="f32",
                       precision=precision, k=kk or 0)
        o = rk.alloc_outputs(plan, device=dev)
        plan.run(cp, ri, va, o["sigma"], o["U"], o["V"], o["rank"], o["patches"], o["npatches"])
        plan.sync()
        V_ref = o["V"][:, :k]
        sig = o["sigma"][:k].contiguous()
        U = o["U"][:k].contiguous()          # k x M rows = column-major M x k
        scale = float(V_ref.abs().max())
        for call in range(2):
            V = torch.full((case.N, k), float("nan"), dtype=V_ref.dtype, device=dev)
            rk.right_vectors_static(case.M, case.N, cp, ri, va, sig, U, V, k=k)
            torch.cuda.synchronize()
            assert not torch.isnan(V).any(), (kk, call)
            assert float((V - V_ref).abs().max()) <= tol * scale, (kk, call)
        plan.free()
