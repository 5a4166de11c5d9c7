"""Benchmark: column-block SVD (Ranky, arXiv 2009.09767) of the zipf_wide
workload -- a 512 x 1,000,000 sparse matrix with ~512k non-zeros, rank-law
Zipf(1.1) column degrees, N(0,1) values, 64 column blocks of 15625, all 512
singular triplets -- in mixed precision (FP32 Jacobi rotations and SpMM, FP64
cross products, refinement, rank decision and merge).

One "step" is one full SVD (partition, lonely scan, block cross products,
block eigensolves, proxy, merge, outputs, V) with inputs resident on the
device.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision mixed|fp64]

Under torchrun each rank runs its own matrix on its own GPU (replicas: the
column blocks of one matrix are not spread across GPUs), so the value is the
SVDs of all ranks over the slowest rank's time.

``--impl reference`` times the CPU FP64 oracle (one-sided Jacobi SVD of the
densified matrix) on a bounded sample of the workload on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SVDs/sec & HBM GB/s at σ rel err ≤1e-4; serving p50/p99 latency vs plain FP64"
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM (Blackwell)


def fp32_peak(device) -> dict:
    """FP32 FMA peak from the device's own SM count and the maximum SM clock
    (MEASURED_PEAKS.json, else nvidia-smi's clocks.max.sm)."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz, src = None, None
    peaks = measured_peaks()
    if peaks and peaks.get("sm_max_mhz"):
        mhz, src = float(peaks["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    if mhz is None:
        try:
            out = subprocess.run(["nvidia-smi", f"--id={device.index or 0}",
                                  "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                                 capture_output=True, text=True, timeout=10).stdout
            mhz, src = float(out.strip().splitlines()[0]), "nvidia-smi clocks.max.sm"
        except (OSError, ValueError, IndexError, subprocess.SubprocessError):
            mhz, src = 2070.0, "nominal 2070 MHz"
    tf = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    return {"tflops": tf, "sms": sms, "mhz": mhz,
            "source": f"{sms} SMs (device query) x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                      f"{mhz:g} MHz ({src})"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def slowest(local_value: float, ws: int, device=None) -> float:
    """The largest value over the ranks (the slowest rank's time); the local
    value when there is one rank."""
    if ws <= 1:
        return float(local_value)
    import torch
    t = torch.tensor([float(local_value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, ws: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (replicas: every rank processes the same number)."""
    return ws * units_per_rank / seconds


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM traffic of one block-Jacobi launch, as a stored note: dram__bytes_read.sum +
# dram__bytes_write.sum of a one-pass ncu capture of the 64-block launch of the full
# zipf_wide SVD (25,573,739,008 + 38,630,312,960 bytes in 24.34 ms), with the hash of
# the kernel source it was taken on.  The line reports it (labelled as stored) only for
# that launch shape and while the source is unchanged.
JACOBI_TRAFFIC = {"source_sha256_16": "01b83a6bd1e480c5", "blocks": 64,
                  "bytes_per_launch": 25_573_739_008 + 38_630_312_960}


def source_hash(rel: str) -> str:
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def jacobi_flops(sweeps: np.ndarray, Mp: int) -> float:
    """Algorithmic FP32 flops of the block Jacobi launch.  A sweep has
    Mp/16 - 1 steps; a step with np = Mp/32 pairs updates the np (np + 1) / 2
    symmetric 32 x 32 blocks of G (two 32^3 products each), the eigenvector
    columns (np * Mp/32 products of 32^3) and solves np 32 x 32 sub-problems
    (16 rotations a round, each 6 flops on 3 x 2 x 32 values: all 31 rounds
    of a sub-problem at a sweep's first step, the 16 rounds of the pairs
    between its two index blocks at the others)."""
    n_p = Mp // 32
    steps = Mp // 16 - 1
    update = n_p * (n_p + 1) / 2 * 2 * 2 * 32 ** 3 + n_p * (Mp // 32) * 2 * 32 ** 3
    rounds = 31 + 16 * (steps - 1)
    per_sweep = steps * update + n_p * rounds * 16 * 6 * 3 * 32
    return float(np.sum(np.abs(sweeps))) * per_sweep


def accuracy_vs(s, U, s_ref, U_ref, gap=1e-3):
    """Largest relative sigma error (sigma > 1e-10 sigma_1) and the largest
    principal-angle sine over the singular vectors whose sigma is separated
    from both neighbours by gap * sigma_1 (U columns = vectors)."""
    s1 = float(s_ref[0])
    big = s_ref > 1e-10 * s1
    rel = float(np.max(np.abs(s[big] - s_ref[big]) / s_ref[big])) if big.any() else 0.0
    worst = 0.0
    n = len(s_ref)
    for i in range(n):
        if not big[i]:
            continue
        if (i > 0 and s_ref[i - 1] - s_ref[i] < gap * s1) or (i + 1 < n and s_ref[i] - s_ref[i + 1] < gap * s1):
            continue
        a = U[:, i] / max(np.linalg.norm(U[:, i]), 1e-300)
        b = U_ref[:, i] / max(np.linalg.norm(U_ref[:, i]), 1e-300)
        worst = max(worst, float(np.linalg.norm(a - (a @ b) * b)))
    return {"sigma_max_rel_err": rel, "u_max_angle_sine_separated": worst,
            "tolerance": {"sigma_rel": 1e-4, "angle": 1e-4}}


def algorithmic_bytes(case, R: int, k: int, s_v: int) -> float:
    """Bytes the SVD must move at least: the CSC read twice (cross products and
    V), the FP32 block eigenbases written and read once, the FP64 proxy and V."""
    csc = case.nnz * (4 + 4) + (case.N + 1) * 8
    return 2.0 * csc + case.num_blocks * case.M * case.M * 4 * 2 + case.M * R * 8 + case.N * k * s_v


def oracle_sample(n_cols: int, seed: int):
    """A zipf_wide-shaped sample (same row count and density law, fewer columns)."""
    import synth

    target = int(round(512_000 * n_cols / 1_000_000))
    return synth.zipf_wide(seed=seed, M=512, N=n_cols, D=max(1, n_cols // 15625),
                           target_nnz=target)


def time_oracle(case):
    import oracle

    t0 = time.perf_counter()
    s, U, V, sweeps = oracle.svd_csc(case.col_ptr, case.row_idx, case.vals, case.M, case.N)
    return time.perf_counter() - t0, sweeps


def cpu_cores_used() -> int:
    return 1  # the oracle is single-threaded C


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    n_cols = args.ref_cols
    case = oracle_sample(n_cols, 20090976 + 2)
    scale = 1_000_000 / n_cols   # one-sided Jacobi work grows linearly in the columns
    for _ in range(args.warmup):
        time_oracle(case)
    t_total = 0.0
    for _ in range(args.steps):
        t, _ = time_oracle(case)
        t_total += t
    per = t_total / args.steps
    value = 1.0 / (per * scale)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "SVD/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "zipf_wide M=512 N=1000000 nnz~512k D=64 k=512",
                   "precision": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": "SVD/s", "cores": cpu_cores_used(),
                         "kind": "oracle",
                         "sample": f"one-sided Jacobi SVD of a zipf_wide-shaped 512 x {n_cols} "
                                   f"sample ({case.nnz} nnz) per step, scaled by {scale:g} "
                                   "(work is linear in the columns) to the full workload"},
        "e2e": {"value": value, "unit": "SVD/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Other workloads (one JSON line each, rank 0 only; not the headline metric)

def _plain_one_at_a_time(cases, device, n=24):
    """The plain FP64 GPU method: one svd_run per matrix, synchronised, no
    batching or graphs.  Returns (matrices/s, per-matrix latencies in ms)."""
    import torch

    import paper_2009_09767_gb300 as rk
    lat = []
    t_all = 0.0
    for c in cases[:n]:
        p = rk.Plan(c.M, c.N, c.nnz, max(1, c.num_blocks), value_type="f32", precision="fp64")
        o = rk.alloc_outputs(p, device=device, with_patches=False)
        cp, ri, va = (torch.from_numpy(c.col_ptr).to(device), torch.from_numpy(c.row_idx).to(device),
                      torch.from_numpy(c.vals).to(device))
        p.run(cp, ri, va, o["sigma"], o["U"], o["V"], o["rank"])
        p.sync()
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        p.run(cp, ri, va, o["sigma"], o["U"], o["V"], o["rank"])
        p.sync()
        dt = time.perf_counter() - t0
        lat.append(dt * 1e3)
        t_all += dt
        p.free()
    return len(lat) / t_all, lat


def run_batch(args):
    """Batched workload: independent matrices, M ~ U{32..256}, N ~ logU[1e3, 2e5],
    density ~ logU[0.5%, 5%], N(0,1) values; block width from the autotuner;
    one batched pass (graph-replayed) per step."""
    import torch

    import paper_2009_09767_gb300 as rk
    import synth
    from paper_2009_09767_gb300 import autotune

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    cases = synth.batch_mix(args.count)
    t_gen = time.perf_counter() - t0
    print(f"# generated {len(cases)} matrices in {t_gen:.1f} s", file=sys.stderr, flush=True)
    width, rates = autotune.tune(cases, args.precision, sample=min(64, len(cases)))
    print(f"# autotuned width {width}: {rates}", file=sys.stderr, flush=True)
    for c in cases:
        c.num_blocks = autotune.blocks_for(c.N, width)
    plans, inputs, outs = [], [], []
    for c in cases:
        p = rk.Plan(c.M, c.N, c.nnz, c.num_blocks, value_type="f32", precision=args.precision)
        plans.append(p)
        inputs.append((torch.from_numpy(c.col_ptr).to(dev), torch.from_numpy(c.row_idx).to(dev),
                       torch.from_numpy(c.vals).to(dev)))
        outs.append(rk.alloc_outputs(p, device=dev, with_patches=False))
    batch = rk.Batch(plans, graph=True)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(1, args.warmup)):
        batch.run(inputs, outs, stream=stream)
    batch.sync()
    torch.cuda.synchronize(dev)
    launches = batch.launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        batch.run(inputs, outs, stream=stream)
    ev1.record(stream)
    batch.sync()
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1) / args.steps
    value = len(cases) / (ms / 1e3)
    plain_rate, plain_lat = _plain_one_at_a_time(cases, dev)
    v_entries = sum(c.N * c.M for c in cases)
    line = {
        "metric": "matrices/s (batched, " + args.precision + ")", "value": value, "unit": "SVD/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "data": "synthetic",
        "config": {"workload": f"batch_mix x{len(cases)} M 32-256 N 1e3-2e5 density 0.5-5%",
                   "precision": args.precision, "block_width": width,
                   "nnz_total": int(sum(c.nnz for c in cases)), "V_entries": int(v_entries),
                   "graph": True},
        "autotune": rates, "gpu_launches_per_pass": launches,
        "plain_fp64_one_at_a_time": {"value": plain_rate, "unit": "SVD/s",
                                     "p50_ms": float(np.percentile(plain_lat, 50)),
                                     "p99_ms": float(np.percentile(plain_lat, 99)),
                                     "sample": f"first {len(plain_lat)} matrices, svd_run + sync each"},
        "speedup_vs_plain": value / plain_rate,
        "V_write_gbs": v_entries * (4 if args.precision == "mixed" else 8) / (ms / 1e3) / 1e9,
        "generate_s": t_gen,
    }
    print(json.dumps(line), flush=True)
    batch.free()
    for p in plans:
        p.free()


def serve_sweep(prec_rates, duration, grace, max_inflight=16, seed_offset=0):
    """Serving: Poisson arrivals of batch_mix-shaped requests with 5%
    zipf_wide-shaped ones, 40 GB device budget; p50/p99 latency (arrival to
    results on the host) and completed requests/s, per (precision, rate).
    prec_rates: [(precision, rate), ...].  Requests still queued `grace`
    seconds after the last arrival are cancelled and counted as dropped."""
    import torch

    import paper_2009_09767_gb300 as rk
    import synth

    torch.cuda.set_device(0)
    rng = np.random.default_rng(synth.SEED_BASE + 5 + seed_offset)
    templates = synth.batch_mix(256, seed=synth.SEED_BASE + 5)
    for c in templates:
        c.num_blocks = 1
    wide = synth.zipf_wide()
    pinned = {}

    def outputs_for(c, prec, slot):
        key = (c.M, c.N, prec, slot)
        if key not in pinned:
            pinned[key] = rk.host_outputs(c.M, c.N, min(c.M, c.N), prec, pinned=True)
        return pinned[key]

    results = []
    for prec, rate in prec_rates:
        srv = rk.Server(40 << 30, max_inflight=max_inflight)
        n = max(1, int(rate * duration))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
        kinds = rng.random(n) < 0.05
        picks = rng.integers(0, len(templates), size=n)
        tickets = []
        t_start = time.perf_counter()
        wide_slot = 0
        for i in range(n):
            delay = t_start + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            if kinds[i]:
                c, slot = wide, wide_slot % 3
                wide_slot += 1
            else:
                c, slot = templates[picks[i]], i % 4
            o = outputs_for(c, prec, slot)
            tickets.append(srv.submit(c.M, c.N, c.col_ptr, c.row_idx, c.vals, c.num_blocks, o,
                                      precision=prec))
        # requests still queued a grace period after the last arrival are
        # cancelled, all at once, and counted as dropped (an overloaded
        # server would otherwise drain its backlog for minutes); admitted
        # ones finish
        deadline = t_start + duration + grace
        status = {}
        for t in tickets:
            call, st = srv.wait_status(t, max(0.0, deadline - time.perf_counter()))
            if call == 0:
                status[t] = st
        dropped = 0
        for t in tickets:
            if t not in status and srv.cancel(t) == 0:
                srv.wait_status(t, 60.0)
                status[t] = None
                dropped += 1
        lat, fails, last_done = [], 0, 0.0
        first = None
        for t in tickets:
            if t in status and status[t] is None:
                srv.release(t)
                continue
            st = status[t] if t in status else srv.wait(t, timeout=120.0)
            ts, ta, td = srv.times(t)
            first = ts if first is None else min(first, ts)
            last_done = max(last_done, td)
            if st != 0:
                fails += 1
            else:
                lat.append((td - ts) * 1e3)
            srv.release(t)
        stats = srv.stats()
        srv.close()
        results.append({
            "precision": prec, "rate_req_s": rate, "requests": n, "failed": fails,
            "dropped_after_grace": dropped,
            "completed_per_s": len(lat) / max(last_done - first, 1e-9) if first is not None else 0.0,
            "p50_ms": float(np.percentile(lat, 50)) if lat else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat else None,
            "pool_peak_gb": stats["pool_peak"] / 2**30})
    return results


def run_serve(args):
    """Serving sweep over args.rates for both precisions (one JSON line)."""
    rates = [float(r) for r in args.rates.split(",")]
    res = serve_sweep([(p, r) for p in ("mixed", "fp64") for r in rates], args.duration,
                      args.grace)
    out = {"metric": "serving p50/p99 latency and throughput", "unit": "ms", "data": "synthetic",
           "config": {"workload": "Poisson arrivals, 95% batch_mix-shaped, 5% zipf_wide-shaped "
                                  "(512 x 1e6), V copied back", "budget_bytes": 40 << 30,
                      "max_inflight": 16, "duration_s_per_rate": args.duration,
                      "grace_s": args.grace},
           "rates": res}
    print(json.dumps(out), flush=True)


def run_single_case(args):
    """One large (1024 x 8e6, ~80M nnz, 256 lognormal blocks, k=100), small
    (64 x 4096, 4 blocks) or tall (zipf_wide transposed: 1e6 x 512, 64 row
    blocks, through the tall entry, whose device transpose is inside the
    step) SVD, timed like the headline."""
    import torch

    import paper_2009_09767_gb300 as rk
    import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flags = rk.FLAG_TIMING
    if args.workload == "large":
        c = synth.large_skewed(N=args.large_cols, D=max(1, int(round(256 * args.large_cols / 8e6))))
        bounds = np.concatenate([[0], np.cumsum(c.widths)]).astype(np.int64)
        k = 100
    elif args.workload == "tall":
        import dataclasses

        import scipy.sparse as sp
        z = synth.zipf_wide(N=args.cols)
        # the CSC of the tall A = zipf_wide^T is zipf_wide's CSR (host set-up)
        At = sp.csc_matrix((z.vals, z.row_idx, z.col_ptr), shape=(z.M, z.N)).T.tocsc()
        At.sort_indices()
        c = dataclasses.replace(z, name="zipf_wide^T", M=z.N, N=z.M,
                                col_ptr=At.indptr.astype(np.int64),
                                row_idx=At.indices.astype(np.int32),
                                vals=At.data.astype(np.float32))
        bounds, k = None, 0
        flags |= rk.FLAG_TALL
    else:
        c = synth.small_uniform().with_values(np.float32)
        bounds, k = None, 0
    if args.legacy_mma:
        flags |= rk.FLAG_LEGACY_MMA
    p = rk.Plan(c.M, c.N, c.nnz, c.num_blocks, value_type="f32", precision=args.precision,
                bounds=bounds, k=k, flags=flags, rank_fix=args.rank_fix,
                seed=args.seed)
    o = rk.alloc_outputs(p, device=dev, with_patches=True)
    cp, ri, va = (torch.from_numpy(c.col_ptr).to(dev), torch.from_numpy(c.row_idx).to(dev),
                  torch.from_numpy(c.vals).to(dev))
    stream = torch.cuda.current_stream(dev)
    def step():
        p.run(cp, ri, va, o["sigma"], o["U"], o["V"], o["rank"], o["patches"], o["npatches"],
              stream=stream)

    for _ in range(max(1, args.warmup)):
        step()
    p.sync()
    p.query(rk.Q_STAGE_TOTAL)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    p.sync()
    ms = ev0.elapsed_time(ev1) / args.steps
    totals = p.query(rk.Q_STAGE_TOTAL)
    line = {"metric": "SVD/s (" + args.workload + ", " + args.precision + ")",
            "value": 1e3 / ms, "unit": "SVD/s", "ms_per_step": ms, "steps": args.steps,
            "config": {"workload": f"{c.name} M={c.M} N={c.N} nnz={c.nnz} D={c.num_blocks} "
                                   f"k={p.k}", "precision": args.precision,
                       "rank_fix": args.rank_fix, "insertions": int(o["npatches"].item()),
                       "products": "mma.sync" if args.legacy_mma else "tcgen05",
                       "lonely_nodes": int(p.query(rk.Q_LONELY).sum())},
            "stage_ms": {n: float(totals[i] / max(totals[-1], 1)) for i, n in enumerate(rk.STAGES)},
            "sweeps": p.query(rk.Q_SWEEPS).tolist()[-1], "rank": int(o["rank"].item()),
            "sigma_head": o["sigma"][:3].cpu().tolist()}
    print(json.dumps(line), flush=True)
    p.free()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--ref-cols", type=int, default=31250)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cols", type=int, default=1_000_000,
                    help="columns of the zipf_wide matrix (smaller cases for profiling)")
    ap.add_argument("--workload", default="zipf_wide",
                    choices=["zipf_wide", "batch", "serve", "large", "small", "tall"],
                    help="zipf_wide (default, the headline), batch (many matrices in one "
                         "pass), serve (Poisson arrivals), large (1024 x 8e6), small (64 x 4096), "
                         "tall (zipf_wide transposed, row blocks)")
    ap.add_argument("--count", type=int, default=2000, help="batch: matrices")
    ap.add_argument("--rates", default="50,100,200,400", help="serve: arrival rates (req/s)")
    ap.add_argument("--duration", type=float, default=8.0, help="serve: seconds per rate")
    ap.add_argument("--grace", type=float, default=15.0,
                    help="serve: seconds after the last arrival before queued requests are dropped")
    ap.add_argument("--large-cols", type=int, default=8_000_000, help="large: columns")
    ap.add_argument("--rank-fix", default="truncate",
                    choices=["truncate", "random", "neighbor", "neighbor_random"],
                    help="large/small: rank fix (Algorithms 2-4); the headline is truncate")
    ap.add_argument("--seed", type=int, default=1, help="rank-fix key")
    ap.add_argument("--legacy-mma", action="store_true",
                    help="large/small/tall: exact-slice products on mma.sync instead of tcgen05")
    ap.add_argument("--no-plain", action="store_true",
                    help="zipf_wide: skip the plain FP64 arm (same matrix, --precision fp64)")
    ap.add_argument("--no-serve", action="store_true",
                    help="zipf_wide: skip the bounded serving sweep")
    ap.add_argument("--serve-rates", default="mixed:100,mixed:400,fp64:100",
                    help="zipf_wide: serving sweep as precision:rate pairs")
    ap.add_argument("--serve-duration", type=float, default=2.0)
    ap.add_argument("--serve-grace", type=float, default=2.0)
    ap.add_argument("--no-tune", action="store_true",
                    help="zipf_wide: skip the Jacobi launch-shape autotuner")
    ap.add_argument("--jacobi-cluster", type=int, default=0,
                    help="zipf_wide: CTAs per block matrix of the FP32 Jacobi (skips the autotuner)")
    args = ap.parse_args()

    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "zipf_wide":
        {"batch": run_batch, "serve": run_serve, "large": run_single_case,
         "small": run_single_case, "tall": run_single_case}[args.workload](args)
        return

    import torch

    import paper_2009_09767_gb300 as rk
    import synth

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    if args.cols == 1_000_000:
        case = synth.zipf_wide(seed=synth.SEED_BASE + 2 + rank)
    else:  # same row count, density law and block width; fewer columns
        case = synth.zipf_wide(seed=synth.SEED_BASE + 2 + rank, N=args.cols,
                               D=max(1, args.cols // 15625),
                               target_nnz=int(round(512_000 * args.cols / 1_000_000)))
    vt = "f32"
    s_v = 4 if args.precision == "mixed" else 8
    cp = torch.from_numpy(case.col_ptr).to(dev)
    ri = torch.from_numpy(case.row_idx).to(dev)
    va = torch.from_numpy(case.vals).to(dev)
    # launch shape of the FP32 Jacobi (CTAs per block matrix), measured
    tuned = None
    if args.jacobi_cluster > 0:
        tuned = {"jacobi_cluster": args.jacobi_cluster, "note": "given on the command line"}
    elif args.precision == "mixed" and not args.no_tune:
        from paper_2009_09767_gb300 import autotune
        cs, cs_ms = autotune.tune_cluster(case, device=dev)
        tuned = {"jacobi_cluster": cs, "block_jacobi_ms_by_cluster": cs_ms,
                 "note": "0 = the library's occupancy model"}
    plan = rk.Plan(case.M, case.N, case.nnz, case.num_blocks, value_type=vt,
                   precision=args.precision, flags=rk.FLAG_TIMING,
                   jacobi_cluster=tuned["jacobi_cluster"] if tuned else 0)
    out = rk.alloc_outputs(plan, device=dev, with_patches=False)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.run(cp, ri, va, out["sigma"], out["U"], out["V"], out["rank"], stream=stream)

    for _ in range(args.warmup):
        step()
    plan.sync()
    plan.query(rk.Q_STAGE_TOTAL)  # reset the stage sums
    clocks = ClockSampler(dev.index) if rank == 0 else None
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    clock_info = clocks.stop() if clocks else None
    plan.sync()
    elapsed_ms = slowest(ev0.elapsed_time(ev1), ws, dev)
    totals = plan.query(rk.Q_STAGE_TOTAL)
    stage_ms = {n: float(totals[i] / max(totals[-1], 1)) for i, n in enumerate(rk.STAGES)}
    launches = int(plan.query(rk.Q_LAUNCHES)[0])
    sweeps = plan.query(rk.Q_SWEEPS)
    R = int(plan.query(rk.Q_PROXY_COLS)[0])
    rank_out = int(out["rank"].item())
    ms_per_step = elapsed_ms / args.steps
    value = job_rate(args.steps, ws, elapsed_ms / 1e3)

    # end to end through the host-buffer entry point: H2D of the CSC, D2H of
    # sigma, U, V and rank inside the timed region
    e2e = None
    if not args.no_e2e:
        h_cp = torch.from_numpy(case.col_ptr).pin_memory()
        h_ri = torch.from_numpy(case.row_idx).pin_memory()
        h_va = torch.from_numpy(case.vals).pin_memory()
        vdt = torch.float32 if args.precision == "mixed" else torch.float64
        h_s = torch.empty(plan.k, dtype=torch.float64).pin_memory()
        h_U = torch.empty(plan.k, plan.M, dtype=torch.float64).pin_memory()
        h_V = torch.empty(plan.N, plan.k, dtype=vdt).pin_memory()
        h_r = torch.empty(1, dtype=torch.int32).pin_memory()
        for _ in range(2):
            plan.run_host(h_cp, h_ri, h_va, h_s, h_U, h_V, h_r, stream=stream)
        if ws > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        n_e2e = max(3, args.steps // 2)
        for _ in range(n_e2e):
            plan.run_host(h_cp, h_ri, h_va, h_s, h_U, h_V, h_r, stream=stream)
        dt = slowest(time.perf_counter() - t0, ws, dev)
        h2d = case.col_ptr.nbytes + case.row_idx.nbytes + case.vals.nbytes
        d2h = h_s.numel() * 8 + h_U.numel() * 8 + h_V.numel() * h_V.element_size() + 4
        e2e = {"value": job_rate(n_e2e, ws, dt), "unit": "SVD/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": n_e2e}

    # roofline of the dominant kernel (block Jacobi, FP32 ALU-bound)
    Mp = 512
    jac_ms = stage_ms["block_jacobi"]
    jac_flops = jacobi_flops(sweeps[:-1], Mp)
    achieved = jac_flops / (jac_ms / 1e3) / 1e12 if jac_ms > 0 else 0.0
    jac_kernel = "k_jacobi4" if args.precision == "mixed" else "k_jacobi<double>"
    fpk = fp32_peak(dev)
    roofline = {"kernel": f"{jac_kernel} ({case.num_blocks} blocks of 512 x 512)",
                "bound": "alu",
                "achieved": achieved, "peak": fpk["tflops"], "unit": "TFLOP/s",
                "frac": achieved / fpk["tflops"], "peak_source": fpk["source"],
                "traffic": None, "kernel_ms": jac_ms, "algorithmic_flops": jac_flops}
    if (case.num_blocks == JACOBI_TRAFFIC["blocks"] and args.precision == "mixed"
            and source_hash("paper_2009_09767_gb300/csrc/jacobi.cu") == JACOBI_TRAFFIC["source_sha256_16"]):
        roofline["traffic"] = JACOBI_TRAFFIC["bytes_per_launch"]
        roofline["traffic_note"] = ("stored: ncu dram__bytes_read.sum + dram__bytes_write.sum of "
                                    "this launch shape on this source (one-pass capture)")
    bytes_per_svd = algorithmic_bytes(case, R, plan.k, s_v)
    peaks = measured_peaks()
    hbm = {"algorithmic_bytes_per_svd": bytes_per_svd,
           "gbs": bytes_per_svd * value / ws / 1e9,
           "peak_gbs": (peaks or {}).get("hbm_gbs", 6800.0),
           "peak_source": "MEASURED_PEAKS.json" if peaks else "fallback 6.8 TB/s"}
    hbm["frac"] = hbm["gbs"] / hbm["peak_gbs"]
    # HBM rooflines of the memory-side stages (stage events on the launch stream):
    # the SpMM writes V once and reads the CSC and W; the cross-product stage reads
    # the CSC and writes the FP64 cross products and their FP32 copy
    csc_bytes = case.col_ptr.nbytes + case.row_idx.nbytes + case.vals.nbytes
    v_bytes = case.N * plan.k * s_v
    g_bytes = case.num_blocks * Mp * Mp * (8 + (4 if args.precision == "mixed" else 8))
    hbm_kernels = {}
    for name, stage, nbytes in (("spmm (k_spmm_vec)", "spmm", v_bytes + csc_bytes + case.M * plan.k * s_v),
                                ("cross products (k_gram, k_symmetrize, k_convert)", "gram",
                                 g_bytes + csc_bytes)):
        ms_k = stage_ms[stage]
        gbs = nbytes / (ms_k / 1e3) / 1e9 if ms_k > 0 else 0.0
        hbm_kernels[name] = {"algorithmic_bytes": float(nbytes), "ms": ms_k, "gbs": gbs,
                             "frac": gbs / hbm["peak_gbs"]}

    # the plain FP64 GPU method on the same matrix (the comparison the metric
    # names) and the mixed result's accuracy against it
    plain = None
    if rank == 0 and ws == 1 and not args.no_plain and args.precision == "mixed":
        s_mixed = out["sigma"].cpu().numpy()
        U_mixed = out["U"].cpu().numpy().T
        pp = rk.Plan(case.M, case.N, case.nnz, case.num_blocks, value_type=vt, precision="fp64")
        po = rk.alloc_outputs(pp, device=dev, with_patches=False)
        pp.run(cp, ri, va, po["sigma"], po["U"], po["V"], po["rank"], stream=stream)
        pp.sync()
        n_plain = 2
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(n_plain):
            pp.run(cp, ri, va, po["sigma"], po["U"], po["V"], po["rank"], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        pp.sync()
        plain_ms = e0.elapsed_time(e1) / n_plain
        s64 = po["sigma"].cpu().numpy()
        U64 = po["U"].cpu().numpy().T
        pp.free()
        acc = accuracy_vs(s_mixed, U_mixed, s64, U64)
        plain = {"value": 1e3 / plain_ms, "unit": "SVD/s", "ms_per_step": plain_ms,
                 "steps": n_plain, "precision": "fp64",
                 "method": "the same library with precision=FP64, one svd_run per step, "
                           "inputs resident on the device",
                 "mixed_over_plain": value / (1e3 / plain_ms),
                 "mixed_accuracy_vs_plain": acc}

    serving = None
    if rank == 0 and ws == 1 and not args.no_serve:
        pr = []
        for item in args.serve_rates.split(","):
            prec, rate = item.split(":")
            pr.append((prec, float(rate)))
        t_srv = time.perf_counter()
        serving = {"workload": "Poisson arrivals, 95% batch_mix-shaped, 5% zipf_wide-shaped; "
                               "40 GB budget; results copied to pinned host memory",
                   "duration_s_per_rate": args.serve_duration, "grace_s": args.serve_grace,
                   "rates": serve_sweep(pr, args.serve_duration, args.serve_grace)}
        serving["wall_s"] = time.perf_counter() - t_srv

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        n_cols = 31250
        sample = oracle_sample(n_cols, synth.SEED_BASE + 2)
        t, _ = time_oracle(sample)
        scale = 1_000_000 / n_cols
        cpu = {"value": 1.0 / (t * scale), "unit": "SVD/s", "cores": cpu_cores_used(),
               "kind": "oracle",
               "sample": f"one SVD of a zipf_wide-shaped 512 x {n_cols} sample ({sample.nnz} "
                         f"nnz) took {t:.2f} s; scaled by {scale:g} (one-sided Jacobi work is "
                         "linear in the columns) to the full workload"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "SVD/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": f"zipf_wide M=512 N={case.N} nnz~{case.nnz // 1000}k "
                                   f"D={case.num_blocks} k={plan.k}",
                       "M": case.M, "N": case.N, "nnz": case.nnz, "blocks": case.num_blocks,
                       "k": plan.k, "precision": args.precision, "rank_fix": "truncate",
                       "parallelism": f"replicas x{ws}",
                       "l2": "no flush: each step writes V (N x k, >= 2 GB) and a >= 0.5 GB "
                             "workspace, far above the 129 MB L2"},
            "roofline": roofline, "hbm": hbm, "cpu_baseline": cpu, "e2e": e2e,
            "plain_fp64": plain, "serving": serving, "autotune": tuned,
            "gpu_launches": launches * args.steps, "launches_per_step": launches,
            "clocks": clock_info, "stage_ms": stage_ms, "hbm_kernels": hbm_kernels,
            "sweeps": {"blocks_min": int(np.abs(sweeps[:-1]).min()),
                       "blocks_max": int(np.abs(sweeps[:-1]).max()), "merge": int(sweeps[-1])},
            "rank": rank_out, "proxy_cols": R,
        }
        print(json.dumps(line), flush=True)
    plan.free()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
