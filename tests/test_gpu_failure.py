"""Device-detected failure: a Jacobi solve that runs out of sweeps.

The block and merge eigensolves stop after max_sweeps sweeps whether or not
they converged (a bounded loop on the device: nothing waits on anything), and
record a negative sweep count.  svd_sync, svd_batch_sync and the serving
loop's per-request status must report SVD_ERR_NOT_CONVERGED (6) for such a
run, and the context must stay usable: a following run with the default cap
succeeds and matches the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2009_09767_gb300 as rk
import synth
from tests._metrics import sigma_check

pytestmark = pytest.mark.gpu

NOT_CONVERGED = 6


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    rk.load_library()
    torch.cuda.set_device(0)


def _inputs(case):
    dev = torch.device("cuda")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(dev)
            for a in (case.col_ptr, case.row_idx, case.vals)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sweep_cap_reports_not_converged(precision):
    case = synth.small_uniform().with_values(np.float64)
    cp, ri, va = _inputs(case)
    plan = rk.Plan(case.M, case.N, case.nnz, case.num_blocks, value_type="f64",
                   precision=precision, max_sweeps=1)
    out = rk.alloc_outputs(plan, device="cuda")
    plan.run(cp, ri, va, out["sigma"], out["U"], out["V"], out["rank"], out["patches"],
             out["npatches"])
    with pytest.raises(rk.RankyError) as e:
        plan.sync()
    assert e.value.status == NOT_CONVERGED
    sweeps = plan.query(rk.Q_SWEEPS)
    assert (sweeps < 0).any() and np.all(np.abs(sweeps) <= 1)
    plan.free()
    # the context is intact: the default cap converges and matches the oracle
    plan2, res = rk.svd(cp, ri, va, case.M, case.N, case.num_blocks, precision=precision)
    s_ref, _, _, _ = oracle.svd_csc(case.col_ptr, case.row_idx, case.vals, case.M, case.N)
    tol = (1e-6, 1e-12) if precision == "fp64" else (1e-4, 1e-6)
    sigma_check(res["sigma"].cpu().numpy(), s_ref, *tol)
    plan2.free()


def test_batch_reports_not_converged():
    cases = [synth.batch_matrix(48, 3000, 0.02, seed=11), synth.batch_matrix(40, 5000, 0.01, seed=12)]
    plans, inputs, outs = [], [], []
    for i, c in enumerate(cases):
        # the first plan is capped at one sweep, the second is not
        p = rk.Plan(c.M, c.N, c.nnz, 2, value_type="f32", precision="mixed",
                    max_sweeps=1 if i == 0 else 0)
        plans.append(p)
        inputs.append(_inputs(c))
        outs.append(rk.alloc_outputs(p, device="cuda"))
    batch = rk.Batch(plans)
    batch.run(inputs, outs)
    with pytest.raises(rk.RankyError) as e:
        batch.sync()
    assert e.value.status == NOT_CONVERGED
    with pytest.raises(rk.RankyError):
        plans[0].sync()
    plans[1].sync()   # the uncapped member converged
    batch.free()
    for p in plans:
        p.free()


def test_server_ticket_not_converged():
    srv = rk.Server(1 << 30, max_inflight=2)
    c = synth.batch_matrix(64, 4000, 0.02, seed=13)
    o_bad = rk.host_outputs(c.M, c.N, min(c.M, c.N), "mixed")
    o_ok = rk.host_outputs(c.M, c.N, min(c.M, c.N), "mixed")
    t_bad = srv.submit(c.M, c.N, c.col_ptr, c.row_idx, c.vals, 2, o_bad, precision="mixed",
                       max_sweeps=1)
    t_ok = srv.submit(c.M, c.N, c.col_ptr, c.row_idx, c.vals, 2, o_ok, precision="mixed")
    assert srv.wait(t_bad, timeout=60.0) == NOT_CONVERGED
    assert srv.wait(t_ok, timeout=60.0) == 0
    s_ref, _, _, _ = oracle.svd_csc(c.col_ptr, c.row_idx, c.vals.astype(np.float64), c.M, c.N)
    sigma_check(o_ok["sigma"], s_ref, 1e-4, 1e-6)
    st = srv.stats()
    assert st["failed"] >= 1 and st["completed"] >= 1
    srv.release(t_bad)
    srv.release(t_ok)
    srv.close()
