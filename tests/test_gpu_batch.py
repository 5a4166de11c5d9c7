"""Batched pass (svd_batch_*) against one-at-a-time svd_run on the same plans
and inputs, and against the CPU oracle: the batch changes where each
eigensolve runs (one persistent launch over all matrices), not the result."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2009_09767_gb300 as rk
import synth
from tests._metrics import sigma_check, subspace_check

pytestmark = pytest.mark.gpu


def _cases():
    rng = np.random.default_rng(2024)
    shapes = [(40, 900, 0.03, 1), (100, 2500, 0.02, 3), (33, 400, 0.05, 2), (256, 6000, 0.01, 4),
              (64, 1500, 0.02, 2), (7, 60, 0.2, 1)]
    out = []
    for M, N, rho, D in shapes:
        c = synth.random_dense_csc(rng, M, N, rho, dtype=np.float32)
        c.num_blocks = D
        out.append(c)
    return out


@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_single_runs_and_oracle(graph):
    dev = torch.device("cuda")
    cases = _cases()
    precisions = ["mixed", "fp64", "mixed", "mixed", "fp64", "mixed"]
    plans, inputs, outs = [], [], []
    for c, prec in zip(cases, precisions):
        p = rk.Plan(c.M, c.N, c.nnz, c.num_blocks, value_type="f32", precision=prec)
        plans.append(p)
        inputs.append((torch.from_numpy(c.col_ptr).to(dev), torch.from_numpy(c.row_idx).to(dev),
                       torch.from_numpy(c.vals).to(dev)))
        outs.append(rk.alloc_outputs(p, device=dev))
    batch = rk.Batch(plans, graph=graph)
    for rep in range(2):   # with a graph: capture, then replay
        for o in outs:
            o["sigma"].fill_(float("nan"))
        batch.run(inputs, outs)
        batch.sync()
        for c, p, o, prec in zip(cases, plans, outs, precisions):
            single = rk.alloc_outputs(p, device=dev)
            p.run(*inputs[cases.index(c)], single["sigma"], single["U"], single["V"],
                  single["rank"], single["patches"], single["npatches"])
            p.sync()
            s_b, s_1 = o["sigma"].cpu().numpy(), single["sigma"].cpu().numpy()
            assert not np.isnan(s_b).any()
            tol = 1e-9 if prec == "mixed" else 1e-11
            sigma_check(s_b, s_1, tol, 1e-9)
            subspace_check(o["U"].cpu().numpy().T, single["U"].cpu().numpy().T, s_1, 1e-6)
            s_ref, _, _, _ = oracle.svd_csc(c.col_ptr, c.row_idx, c.vals.astype(np.float64), c.M, c.N)
            sigma_check(s_b, s_ref[:len(s_b)], 1e-4 if prec == "mixed" else 1e-6,
                        1e-6 if prec == "mixed" else 1e-12)
    assert batch.launches() > 0 or graph
    batch.free()
    for p in plans:
        p.free()
