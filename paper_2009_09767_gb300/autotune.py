"""Block-width autotuner for batched SVDs.

The column-block method (Ranky, arXiv 2009.09767, section III) leaves the
block width free: every width gives the same SVD (Eqs. 2-3), but the work
does not.  Each block costs one M x M eigensolve whatever its width, while
wider blocks mean fewer, larger sparse cross products.  For a batch of many
independent matrices the best width depends on the mix of shapes, so it is
measured: a sample of the batch is run once per candidate width and the
fastest is kept.  Results are cached in a JSON file (``RANKY_AUTOTUNE_CACHE``,
default ``~/.cache/ranky_autotune.json``) keyed by the workload signature.
"""
from __future__ import annotations

import json
import math
import os
import time

# None: one block per matrix (width = N)
CANDIDATES = (None, 131072, 32768, 8192)


def blocks_for(N: int, width) -> int:
    """Number of equal-width column blocks for a matrix with N columns."""
    if width is None or width >= N:
        return 1
    return max(1, math.ceil(N / width))


def _cache_path() -> str:
    return os.environ.get("RANKY_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ranky_autotune.json"))


def signature(cases, precision: str) -> str:
    Ms = [c.M for c in cases]
    Ns = [c.N for c in cases]
    nnz = sum(c.nnz for c in cases)
    return (f"{precision}|n={len(cases)}|M={min(Ms)}-{max(Ms)}|N={min(Ns)}-{max(Ns)}|"
            f"nnz={nnz // 1000}k")


def _time_width(cases, width, precision, reps, device):
    import torch

    import paper_2009_09767_gb300 as rk
    plans, inputs, outs = [], [], []
    for c in cases:
        p = rk.Plan(c.M, c.N, c.nnz, blocks_for(c.N, width), value_type="f32", precision=precision)
        plans.append(p)
        inputs.append((torch.from_numpy(c.col_ptr).to(device), torch.from_numpy(c.row_idx).to(device),
                       torch.from_numpy(c.vals).to(device)))
        outs.append(rk.alloc_outputs(p, device=device, with_patches=False))
    batch = rk.Batch(plans)
    batch.run(inputs, outs)
    batch.sync()
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    for _ in range(reps):
        batch.run(inputs, outs)
    batch.sync()
    torch.cuda.synchronize(device)
    dt = (time.perf_counter() - t0) / reps
    batch.free()
    for p in plans:
        p.free()
    return len(cases) / dt


def tune(cases, precision: str = "mixed", sample: int = 64, reps: int = 2, device=None,
         use_cache: bool = True):
    """Return (best width or None, {width: matrices/s}) for this batch."""
    import torch
    device = device or torch.device("cuda")
    sig = signature(cases, precision)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and sig in cache:
        entry = cache[sig]
        return entry["width"], {str(k): v for k, v in entry["rates"].items()}
    step = max(1, len(cases) // sample)
    picked = cases[::step][:sample]
    rates = {}
    for w in CANDIDATES:
        rates[str(w)] = _time_width(picked, w, precision, reps, device)
    best = max(rates, key=rates.get)
    width = None if best == "None" else int(best)
    if use_cache:
        cache[sig] = {"width": width, "rates": rates}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return width, rates


# FP32 Jacobi launch shape: CTAs per block matrix (thread-block cluster size).
CLUSTER_CANDIDATES = (0, 2, 4, 8, 16)   # 0: the library's occupancy model


def tune_cluster(case, precision: str = "mixed", reps: int = 2, device=None, candidates=None):
    """Measure the block-eigensolve stage (SVD_FLAG_TIMING stage times) of
    one matrix for each Jacobi cluster size; return (best size, {size: ms}).
    The size only changes how the solver is spread over the GPU, never the
    result beyond rounding."""
    import torch

    import paper_2009_09767_gb300 as rk
    device = device or torch.device("cuda")
    cp, ri, va = (torch.from_numpy(a).to(device) for a in (case.col_ptr, case.row_idx, case.vals))
    times = {}
    for cs in candidates or CLUSTER_CANDIDATES:
        p = rk.Plan(case.M, case.N, case.nnz, case.num_blocks, value_type="f32",
                    precision=precision, flags=rk.FLAG_TIMING | rk.FLAG_SKIP_V, jacobi_cluster=cs)
        o = rk.alloc_outputs(p, device=device, with_patches=False)
        p.run(cp, ri, va, o["sigma"], o["U"], None, o["rank"])
        p.sync()
        p.query(rk.Q_STAGE_TOTAL)   # reset the stage sums
        for _ in range(reps):
            p.run(cp, ri, va, o["sigma"], o["U"], None, o["rank"])
        p.sync()
        tot = p.query(rk.Q_STAGE_TOTAL)
        times[str(cs)] = float(tot[rk.STAGES.index("block_jacobi")] / max(tot[-1], 1))
        p.free()
    best = min(times, key=times.get)
    return int(best), times
