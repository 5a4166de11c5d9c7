"""Serving loop (svd_server_*): continuous batching on one GPU.

* every request's result is the same alone and in a mix of concurrent
  requests (within the mixed-precision tolerance), and matches the oracle;
* admission respects the device-memory budget, and a request that can never
  fit is rejected at submit;
* queued requests can be cancelled, waits time out, and host-side injected
  faults (allocation failure, malformed CSC) fail only their own request."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2009_09767_gb300 as rk
import synth
from tests._metrics import sigma_check, subspace_check

pytestmark = pytest.mark.gpu


def _requests(n=10, seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        M = int(rng.integers(16, 160))
        N = int(rng.integers(300, 6000))
        rho = float(np.exp(rng.uniform(np.log(0.005), np.log(0.05))))
        c = synth.random_dense_csc(rng, M, N, rho, dtype=np.float32)
        c.num_blocks = int(rng.integers(1, 4))
        out.append(c)
    return out


def _submit(srv, c, precision="mixed"):
    k = min(c.M, c.N)
    o = rk.host_outputs(c.M, c.N, k, precision)
    t = srv.submit(c.M, c.N, c.col_ptr, c.row_idx, c.vals, c.num_blocks, o, precision=precision)
    return t, o


def test_same_result_alone_and_in_the_mix():
    cases = _requests()
    # alone: one request at a time on a one-slot server
    alone = []
    srv = rk.Server(2 << 30, max_inflight=1)
    for c in cases:
        t, o = _submit(srv, c)
        assert srv.wait(t) == 0
        alone.append(o)
    srv.close()
    # mixed: everything submitted at once, up to 6 on the GPU together
    srv = rk.Server(2 << 30, max_inflight=6)
    tickets = [_submit(srv, c) for c in cases]
    for (t, o), c, a in zip(tickets, cases, alone):
        assert srv.wait(t) == 0
        sigma_check(o["sigma"], a["sigma"], 1e-9, 1e-9)
        subspace_check(o["U"].T, a["U"].T, a["sigma"], 1e-6)
        s_ref, _, _, _ = oracle.svd_csc(c.col_ptr, c.row_idx, c.vals.astype(np.float64), c.M, c.N)
        sigma_check(o["sigma"], s_ref[:len(o["sigma"])], 1e-4, 1e-6)
        ts, ta, td = srv.times(t)
        assert ts <= ta <= td
    st = srv.stats()
    assert st["completed"] == len(cases) and st["failed"] == 0 and st["pool_used"] == 0
    srv.close()


def test_budget_admission_and_rejection():
    cases = _requests(6, seed=9)
    need = [rk.plan_bytes(c.M, c.N, c.nnz, c.num_blocks, value_type="f32") for c in cases]
    budget = int(2.5 * max(need)) + (8 << 20)
    srv = rk.Server(budget, max_inflight=8)
    tickets = [_submit(srv, c) for c in cases]
    for t, _ in tickets:
        assert srv.wait(t) == 0
    st = srv.stats()
    assert st["pool_peak"] <= budget and st["completed"] == len(cases)
    big = synth.random_dense_csc(np.random.default_rng(1), 1024, 200000, 0.001, dtype=np.float32)
    big.num_blocks = 64
    with pytest.raises(rk.RankyError) as err:
        _submit(srv, big)
    assert err.value.status == 4   # SVD_ERR_BUDGET
    assert srv.stats()["rejected"] == 1
    srv.close()


def test_cancel_timeout_and_injected_faults():
    heavy = synth.random_dense_csc(np.random.default_rng(3), 512, 60000, 0.01, dtype=np.float32)
    heavy.num_blocks = 8
    light = _requests(3, seed=11)
    srv = rk.Server(4 << 30, max_inflight=1)
    t0, o0 = _submit(srv, heavy)                 # occupies the single slot
    t1, o1 = _submit(srv, light[0])              # queued behind it
    t2, o2 = _submit(srv, light[1])
    assert srv.cancel(t2) == 0                   # still queued: cancelled
    call, res = srv.wait_status(t1, 0.0)         # cannot be done yet
    assert call == 7                             # SVD_ERR_TIMEOUT
    assert srv.wait(t0) == 0 and srv.wait(t1) == 0
    assert srv.wait(t2) == 1                     # cancelled requests report INVALID_ARG
    assert srv.cancel(t0) != 0                   # finished requests cannot be cancelled
    # injected faults hit only their own tickets (tickets are numbered from 1)
    srv.inject(rk.INJECT_ALLOC, 4)
    srv.inject(rk.INJECT_BAD_CSC, 5)
    t3, _ = _submit(srv, light[2])
    t4, _ = _submit(srv, light[0])
    t5, o5 = _submit(srv, light[1])
    assert (t3, t4) == (4, 5)
    assert srv.wait(t3) == 3                     # SVD_ERR_OOM
    assert srv.wait(t4) == 2                     # SVD_ERR_INVALID_CSC
    assert srv.wait(t5) == 0
    s_ref, _, _, _ = oracle.svd_csc(light[1].col_ptr, light[1].row_idx,
                                    light[1].vals.astype(np.float64), light[1].M, light[1].N)
    sigma_check(o5["sigma"], s_ref[:len(o5["sigma"])], 1e-4, 1e-6)
    st = srv.stats()
    assert st["failed"] == 3 and st["pool_used"] == 0
    for t in (t0, t1, t2, t3, t4, t5):
        srv.release(t)
    srv.close()


def test_group_member_failure_is_isolated():
    """Small requests queued together run as one batched group; a member whose
    CSC is malformed (rejected by the requested structural check) fails alone
    and its group-mates finish with correct results."""
    cases = _requests(5, seed=21)
    heavy = synth.random_dense_csc(np.random.default_rng(4), 512, 60000, 0.01, dtype=np.float32)
    heavy.num_blocks = 8
    srv = rk.Server(4 << 30, max_inflight=1)
    t_heavy, _ = _submit(srv, heavy)               # holds the only slot: the rest queue up
    tickets = []
    for i, c in enumerate(cases):
        cp = c.col_ptr.copy()
        if i == 2:
            cp[-1] += 1                            # col_ptr[N] != nnz: malformed
        k = min(c.M, c.N)
        o = rk.host_outputs(c.M, c.N, k, "mixed")
        tickets.append((srv.submit(c.M, c.N, cp, c.row_idx, c.vals, c.num_blocks, o,
                                   precision="mixed", flags=rk.FLAG_CHECK_CSC), o, c))
    assert srv.wait(t_heavy) == 0
    for i, (t, o, c) in enumerate(tickets):
        st = srv.wait(t)
        if i == 2:
            assert st == 2                         # SVD_ERR_INVALID_CSC
            continue
        assert st == 0
        s_ref, _, _, _ = oracle.svd_csc(c.col_ptr, c.row_idx, c.vals.astype(np.float64), c.M, c.N)
        sigma_check(o["sigma"], s_ref[:len(o["sigma"])], 1e-4, 1e-6)
    stats = srv.stats()
    assert stats["failed"] == 1 and stats["pool_used"] == 0
    srv.close()
