"""Launch-shape tuning of the FP32 block Jacobi (jacobi_cluster, the number of
CTAs that share one block matrix): any size gives the same SVD up to
rounding, an unlaunchable size falls back to the occupancy model's choice,
and the autotuner returns one of its candidates with a time for each."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2009_09767_gb300 as rk
import synth
from paper_2009_09767_gb300 import autotune
from tests._metrics import sigma_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    rk.load_library()
    torch.cuda.set_device(0)


def test_cluster_sizes_same_result():
    rng = np.random.default_rng(5)
    case = synth.random_dense_csc(rng, 160, 6000, 0.02, dtype=np.float32)
    dev = torch.device("cuda")
    t = [torch.from_numpy(a).to(dev) for a in (case.col_ptr, case.row_idx, case.vals)]
    s_ref, _, _, _ = oracle.svd_csc(case.col_ptr, case.row_idx, case.vals.astype(np.float64),
                                    case.M, case.N)
    for cs in (0, 1, 2, 4, 8, 16, 3, 64):   # 3 and 64 are not launchable: fall back
        plan, res = rk.svd(*t, case.M, case.N, 4, precision="mixed", jacobi_cluster=cs,
                           flags=rk.FLAG_SKIP_V)
        sigma_check(res["sigma"].cpu().numpy(), s_ref, 1e-4, 1e-6)
        plan.free()


def test_autotuner_picks_a_candidate():
    case = synth.zipf_wide(N=62_500, D=4, target_nnz=32_000)
    best, times = autotune.tune_cluster(case, reps=1)
    assert best in autotune.CLUSTER_CANDIDATES
    assert set(times) == {str(c) for c in autotune.CLUSTER_CANDIDATES}
    assert all(v > 0 for v in times.values())
