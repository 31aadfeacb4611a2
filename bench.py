#!/usr/bin/env python
"""Throughput of the randomized block-CG solver on one GB300 (or N replicas).

Workload: the sparse SPD system of a variable-coefficient 3D 7-point diffusion
operator on a 128^3 grid (d = 2,097,152, nnz = 14,581,760, face coefficients
exp(N(0,1)), FP64 values, int32 indices), shift mu = 1e-4, b ~ N(0, I), sketch
Omega of 32 Gaussian columns (block width 33). All inputs are seeded synthetic data.

One step = one complete solve to relative residual 1e-8 (FP64 residual recomputed
from the FP64 matrix): FP32 block operator / updates, FP64 Grams, small solves and
refinement. The plain FP64 path (every block quantity in FP64, stopped at the same
1e-8) is timed beside it. value = solves/s over all ranks (weak scaling: every rank
solves its own copy of the system).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

`--workload batched` measures the batched configuration instead: 512 independent
dense SPD systems, d log-uniform in [500, 16000], FP32 storage, outlier spectra, block
widths from the autotuner. It prints its own JSON line (one step = the whole batch
solved to 1e-8).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2501_18717_gb300 import workloads as W  # noqa: E402

GRID = 128
SKETCH = 32
MU = 1e-4
TOL = 1e-8
SEED = W.BASE_SEED + 2
OMEGA_SEED = W.BASE_SEED + 3
METRIC = "solves/s at rel. residual 1e-8 and HBM GB/s per iteration, mixed vs FP64 plain"
WORKLOAD = "csr_diffusion_128^3_d2097152_nnz14581760_mu1e-4_l32"


def workload_name(grid, d, nnz):
    """The diffusion workload string for a grid size (the 128^3 default is WORKLOAD)."""
    return f"csr_diffusion_{grid}^3_d{d}_nnz{nnz}_mu1e-4_l32"
KERNEL_SOURCES = ["paper_2501_18717_gb300/csrc/k_ops.cu", "paper_2501_18717_gb300/csrc/k_block.cu",
                  "paper_2501_18717_gb300/csrc/bk_tile.cuh", "paper_2501_18717_gb300/csrc/bk_update.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="diffusion", choices=["diffusion", "batched", "dense-product", "ridge",
                                                                 "sample", "nystrom", "shrink", "csr-product"])
    ap.add_argument("--ridge-n", type=int, default=200000)
    ap.add_argument("--ridge-d", type=int, default=4096)
    ap.add_argument("--ridge-inner", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--sample-d", type=int, default=40000)
    ap.add_argument("--sample-m", type=int, default=256)
    ap.add_argument("--sample-loads", type=int, default=16)
    ap.add_argument("--sample-inner", default="ozaki", choices=["ozaki", "f32x2", "fp32", "fp64"])
    ap.add_argument("--sample-nugget", type=float, default=None)
    ap.add_argument("--sample-operator", default="stored", choices=["stored", "rbf"])
    ap.add_argument("--sample-only", action="store_true",
                    help="sampling leg: only the timed calls (no profiled, inverse-square-root or other-mode call)")
    ap.add_argument("--dense-d", type=int, default=16384)
    ap.add_argument("--dense-m", type=int, default=33)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--fp64-subset", type=int, default=32)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    # smaller cases for profiling runs (ncu); the default is the 128^3 workload
    ap.add_argument("--grid", type=int, default=GRID)
    ap.add_argument("--max-loads", type=int, default=20000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-systems result attached to the default line")
    return ap.parse_args()


def algorithmic_bytes(d, nnz, m):
    """Bytes each kernel must move per launch at FP32 block precision (m live columns)."""
    blk = d * m * 4
    return {
        "operator": nnz * (4 + 4) + (d + 1) * 4 + 2 * blk,  # A values+indices, read P, write Y
        "update_r": 3 * blk,                               # read Y, Q; write W (over Q)
        "update_p": 4 * blk + 2 * d * 8,                   # read W, P; write Q, P; x read+write (FP64)
    }


def measured_bf16_peak(sustained=True):
    """Measured dense BF16 TFLOP/s (sustained: for a kernel timed inside a long call)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            j = json.load(fh)
        k = "bf16_tflops_sustained" if sustained and "bf16_tflops_sustained" in j else "bf16_tflops"
        return float(j[k]), "measured " + k
    return (1700.0 if sustained else 1900.0), "fallback"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            j = json.load(fh)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_traffic(name):
    """ncu DRAM bytes per launch for `name`, if the committed capture matches the sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        j = json.load(fh)
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if j.get("sources_sha256") != h.hexdigest():
        return None
    return j.get("kernels", {}).get(name)


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, dev=None):
    """The maximum of a host number over the ranks of the default process group (the
    slowest replica bounds the job); the number itself without one. dev is the device
    of the collective's buffer (a CUDA device for NCCL, None for gloo on the host)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev if dev is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, steps, ms):
    """Whole-job solves/s of `world` independent replicas, each timing `steps` solves,
    from the slowest replica's time in ms."""
    return world * steps / (ms / 1e3)


# ---------------------------------------------------------------------------------- oracle
def oracle_sample(rp, ci, va, b, seconds, max_loads=60):
    """Time the FP64 oracle's block-CG recurrence on the full workload for a bounded
    number of loads; returns (seconds per load, loads run, threads)."""
    from oracle import bcg, operators
    op = operators.CSR(rp, ci, va)
    d = b.shape[0]
    om = W.omega(OMEGA_SEED, d, SKETCH)
    B = W.inner_start_block(b, om)
    # one load to learn the per-load time, then as many as fit in the budget
    t0 = time.perf_counter()
    bcg.block_cg(op, MU, B[:, 0], B[:, 1:], tol=0.0, max_loads=1)
    t1 = time.perf_counter() - t0
    n = int(max(2, min(max_loads, seconds / max(t1, 1e-3))))
    t0 = time.perf_counter()
    bcg.block_cg(op, MU, B[:, 0], B[:, 1:], tol=0.0, max_loads=n)
    dt = time.perf_counter() - t0
    threads = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        threads = max(i.get("num_threads", 1) for i in threadpool_info()) or threads
    except Exception:  # noqa: BLE001
        pass
    return dt / n, n, threads


def oracle_loads_per_solve():
    p = os.path.join(ROOT, "oracle", "loads_diffusion128.json")
    if os.path.exists(p):
        with open(p) as fh:
            return (json.load(fh)["loads_fp64_refined_1e-8"],
                    "oracle refined to 1e-8 under the library's inner stopping rule (oracle/loads_diffusion128.json)")
    return None, None


def run_reference(args, world, rank):
    """The oracle arm: each step times a fixed number of loads of the FP64 oracle's
    block-CG recurrence on the full workload (the oracle cannot finish a solve within a
    bench run). ms_per_step is that measured time; value is solves/s, the measured time
    per load times the loads the oracle needs for a refined solve to 1e-8 under the
    library's stopping rule (oracle/loads_diffusion128.json), given with its inputs
    under `extrapolation`."""
    if rank != 0:
        return
    from oracle import bcg, operators
    rp, ci, va, d = W.diffusion_csr(SEED, GRID)
    b = W.normals(SEED, W.STREAM_RHS, d)
    lps, src = oracle_loads_per_solve()
    op = operators.CSR(rp, ci, va)
    om = W.omega(OMEGA_SEED, d, SKETCH)
    B = W.inner_start_block(b, om)
    # loads per step: as many as fit in the per-step budget, at most 8
    t0 = time.perf_counter()
    bcg.block_cg(op, MU, B[:, 0], B[:, 1:], tol=0.0, max_loads=1)
    probe = time.perf_counter() - t0
    n = int(max(2, min(8, min(args.cpu_seconds, 15.0) / max(probe, 1e-3))))
    step_s = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        out = bcg.block_cg(op, MU, B[:, 0], B[:, 1:], tol=0.0, max_loads=n)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            step_s.append(dt / max(out["loads"], 1) * n)
    ms_step = statistics.median(step_s) * 1e3
    spl = ms_step / 1e3 / n
    value = (1.0 / (spl * lps)) if lps else None
    thr = threads_used()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "working set larger than L2"},
        "step": f"{n} loads of the FP64 oracle block-CG recurrence on the full workload (measured)",
        "extrapolation": {"loads_timed_per_step": n, "s_per_load": spl, "loads_per_solve": lps,
                          "ms_per_solve": spl * lps * 1e3 if lps else None, "loads_source": src},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": thr, "kind": "oracle",
                         "sample": f"each step: {n} loads of the FP64 oracle block-CG recurrence on the full "
                                   f"workload ({ms_step:.0f} ms measured); solves/s = 1/(s per load x {lps} loads "
                                   f"per solve, {src})"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------- GPU arm
BATCH_SEED = W.BASE_SEED + 5
CAL_SEED = W.BASE_SEED + 50


def run_batched(args, world, rank, local, dev):
    """512 uneven dense FP32 systems solved together to 1e-8 (mixed precision), with
    the FP64-block path timed on a size-stratified subset and scaled by sum d^2."""
    import torch
    from paper_2501_18717_gb300 import bk

    n = args.batch
    ds = [int(v) for v in W.batch_sizes(BATCH_SEED, n)]
    mats, bs = [], []
    for i, d in enumerate(ds):
        A, b = W.batch_system_torch(BATCH_SEED, i, d, dev)
        mats.append(A)
        bs.append(b)
    torch.cuda.synchronize(dev)
    xs = [torch.zeros(d, dtype=torch.float64, device=dev) for d in ds]
    ctx = bk.Context(local)
    stream = torch.cuda.Stream(dev)
    ctx.set_stream(stream.cuda_stream)

    # autotune on separately seeded calibration systems, one per size bucket
    cal_d = [int(v) for v in W.batch_sizes(CAL_SEED, 24)]
    cal = [W.batch_system_torch(CAL_SEED, i, d, dev) for i, d in enumerate(cal_d)]
    cal_x = [torch.zeros(d, dtype=torch.float64, device=dev) for d in cal_d]
    mixed = bk.default_opts(tol=TOL, sketch=-1, seed=OMEGA_SEED, inner="fp32", inner_tol=1e-5, check_every=16)
    t0 = time.perf_counter()
    cands = [8, 16, 32, 64]
    with torch.cuda.stream(stream):
        bk.autotune(ctx, bk.Batch([a for a, _ in cal], np.zeros(len(cal)), [b for _, b in cal], cal_x),
                    cands, mixed)
    tune_s = time.perf_counter() - t0
    del cal, cal_x
    import tempfile
    with tempfile.TemporaryDirectory() as tdir:
        table = {str(k): {"sketch": v[0], "product": v[1]}
                 for k, v in bk.autotune_table(ctx, os.path.join(tdir, "tune.txt")).items()}

    batch = bk.Batch(mats, np.zeros(n), bs, xs)

    def solve(opts, bt):
        with torch.cuda.stream(stream):
            return bk.solve_batched(ctx, bt, opts, check=False)

    for _ in range(args.warmup):
        solve(mixed, batch)
    torch.cuda.synchronize(dev)
    infos_all = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            infos_all.append(solve(mixed, batch))
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    value = world * n * args.steps / (ms / 1e3)
    infos = infos_all[-1]
    # one solve with every step kernel launched on the stream instead of replayed from
    # CUDA graphs: how much of a step is launch overhead (what a single persistent
    # launch could save at most)
    os.environ["BK_NO_GRAPH"] = "1"
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    sinfo = solve(mixed, batch)
    g1.record(stream)
    torch.cuda.synchronize(dev)
    del os.environ["BK_NO_GRAPH"]
    stream_ms = g0.elapsed_time(g1)
    launch_check = {"graph_replay_ms_per_solve": ms / args.steps, "stream_launch_ms_per_solve": stream_ms,
                    "stream_over_graph": stream_ms / (ms / args.steps),
                    "all_converged_stream": all(i.status == bk.BK_OK for i in sinfo)}
    rel = max(i.rel_residual for i in infos)
    ok = sum(1 for i in infos if i.status == bk.BK_OK)
    loads = [i.loads for i in infos]
    # average HBM rate over the whole solve: each load streams A once (4 d^2 bytes)
    a_bytes = sum(4.0 * d * d * l for d, l in zip(ds, loads))
    peak, peak_src = measured_peaks()
    gbs = a_bytes / (ms / args.steps / 1e3) / 1e9

    # FP64-block path on a size-stratified subset (every n/k-th system by size rank)
    fp64 = None
    if args.fp64_subset > 0:
        order = np.argsort(ds)
        sub = [int(order[j]) for j in range(0, n, max(1, n // args.fp64_subset))]
        sx = [torch.zeros(ds[i], dtype=torch.float64, device=dev) for i in sub]
        sb = bk.Batch([mats[i] for i in sub], np.zeros(len(sub)), [bs[i] for i in sub], sx)
        plain = bk.default_opts(tol=TOL, sketch=-1, seed=OMEGA_SEED, inner="fp64", inner_tol=1e-6, check_every=16)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pinfo = solve(plain, sb)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        pms = e0.elapsed_time(e1)
        frac_work = sum(ds[i] ** 2 for i in sub) / sum(d * d for d in ds)
        fp64 = {"value": n / (pms / 1e3 / frac_work), "unit": "solves/s",
                "subset": len(sub), "subset_ms": pms, "subset_share_of_sum_d2": frac_work,
                "rel_residual_max": max(i.rel_residual for i in pinfo),
                "loads_mean": float(np.mean([i.loads for i in pinfo])),
                "note": "FP64 blocks on every (n/subset)-th system by size; solves/s scaled by sum d^2"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the FP64 oracle's refined block-CG on a size-stratified subset, scaled by sum d^2
        from oracle import bcg
        order = np.argsort(ds)
        sub, spent, t_all = [], 0.0, 0.0
        # systems at the size quantiles 0, 1/5, ..., 1 (smallest first), while time lasts
        for q in np.linspace(0.0, 1.0, 6):
            i = int(order[min(n - 1, int(round(q * (n - 1))))])
            if spent > args.cpu_seconds:
                break
            A_, b_ = W.batch_system(BATCH_SEED, i, ds[i])
            sk = table.get(int(np.floor(np.log2(ds[i]))), 16)
            om = W.omega(OMEGA_SEED + i, ds[i], sk)
            t0 = time.perf_counter()
            bcg.refined_solve(A_.astype(np.float64), 0.0, b_, om, tol=TOL, inner_tol=1e-6, max_loads=5000)
            dt = time.perf_counter() - t0
            spent += dt
            t_all += dt
            sub.append(i)
        frac = sum(ds[i] ** 2 for i in sub) / sum(d * d for d in ds)
        cpu = {"value": n / (t_all / frac), "unit": "solves/s", "cores": threads_used(), "kind": "oracle",
               "sample": f"FP64 oracle refined block-CG (NumPy) on {len(sub)} systems at the size quantiles "
                         f"0, 0.2, ..., 1 (d = {[ds[i] for i in sub]}), stopping once {args.cpu_seconds:.0f} s "
                         f"were spent; solves/s scaled by their share of sum d^2 ({frac:.4f})"}
    if rank == 0:
        line = {
            "metric": "solves/s at rel. residual 1e-8, batched uneven dense systems, mixed vs FP64 plain",
            "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 block ops + f64 Gram/solve/refinement", "data": "synthetic",
            "config": {"workload": f"batched_{n}_dense_logU500-16000_fp32_outliers1e2-1e5",
                       "sum_d2_bytes_fp32": sum(4.0 * d * d for d in ds), "tol": TOL,
                       "autotune": {"candidates": cands, "table_log2d": table, "seconds": tune_s,
                                    "note": "every candidate's block width is built (64: width 65, padded 68); "
                                            "product = block-product kernel"},
                       "l2": "matrices 75 GB, far larger than L2; no flush"},
            "converged": ok, "rel_residual_max": rel, "loads_mean": float(np.mean(loads)),
            "loads_max": int(max(loads)),
            "roofline": {"bound": "hbm", "kernel": "whole solve (A streamed once per load)", "achieved": gbs,
                         "peak": peak, "unit": "GB/s", "frac": gbs / peak, "traffic": None, "peak_source": peak_src},
            "fp64_plain": fp64, "clocks": clk.summary(), "cpu_baseline": cpu,
            "launch_overhead": launch_check,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def batched_leg():
    """The batched workload's JSON line from `bench.py --workload batched` run as a child
    process (one warm-up and one timed solve of the 512 systems, FP64 subset beside)."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "batched", "--steps", "1", "--warmup", "1",
           "--no-cpu-baseline"]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
    except subprocess.TimeoutExpired:
        return {"error": "batched leg timed out"}
    for ln in r.stdout.splitlines():
        if ln.startswith("{"):
            j = json.loads(ln)
            keep = ("metric", "value", "unit", "ms_per_step", "converged", "rel_residual_max", "loads_mean",
                    "fp64_plain", "roofline", "launch_overhead")
            out = {k: j.get(k) for k in keep}
            out["autotune"] = j.get("config", {}).get("autotune")
            out["command"] = " ".join(cmd[1:])
            return out
    return {"error": f"batched leg rc={r.returncode}: {r.stderr[-300:]}"}


def run_csr_product(args, world, rank, local, dev):
    """One block product of the diffusion operator with its Gram, Y = A P + mu P and
    P^T Y (FP32 values, 33 columns in 36-wide panels), through bk_block_apply: the
    operator kernel of the headline solve in isolation, for a small ncu capture.
    value = algorithmic GB/s per call (CUDA events around the calls, so each includes
    the call's host synchronisation)."""
    import torch
    from paper_2501_18717_gb300 import bk

    rp, ci, va, d = W.diffusion_csr(SEED, args.grid)
    m = SKETCH + 1
    ld = (d + 31) // 32 * 32
    nq = (m + 3) // 4
    g = torch.Generator(device=dev)
    g.manual_seed(BATCH_SEED)
    P = torch.randn((nq, ld, 4), device=dev, dtype=torch.float32, generator=g)
    P[:, d:, :] = 0
    if m % 4:
        P[-1, :, m % 4:] = 0
    Y = torch.zeros_like(P)
    G = torch.zeros((m, m), dtype=torch.float64, device=dev)
    ctx = bk.Context(local)
    stream = torch.cuda.Stream(dev)
    ctx.set_stream(stream.cuda_stream)
    op = bk.csr_operator(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev),
                         torch.from_numpy(va.astype(np.float32)).to(dev))
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            bk.block_apply(ctx, op, MU, P, Y, G, m, ld)
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            bk.block_apply(ctx, op, MU, P, Y, G, m, ld)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1) / args.steps
    nnz = int(va.shape[0])
    gb = (8.0 * nnz + 4.0 * (d + 1) + 2 * 4.0 * d * 36) / 1e9  # the operator's per-launch bytes
    gbs = gb / (ms / 1e3)
    peak, src = measured_peaks()
    if rank == 0:
        print(json.dumps({"metric": "CSR block product + Gram (operator kernel), algorithmic GB/s per call",
                          "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                          "config": {"workload": workload_name(args.grid, d, nnz), "block_width": m},
                          "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                       "frac": gbs / peak, "traffic": None, "peak_source": src}}), flush=True)
    ctx.close()
    return 0


def run_dense_product(args, world, rank, local, dev):
    """One dense FP32 block product Y = A P + mu P with its Gram P^T Y (the tensor-core
    kernel when the rows are 16-byte aligned): A d x d Gaussian, P d x m. value = GB/s
    of A streamed per product (A is larger than L2 from d = 6000 on)."""
    import torch
    from paper_2501_18717_gb300 import bk

    d, m = args.dense_d, args.dense_m
    g = torch.Generator(device=dev)
    g.manual_seed(BATCH_SEED)
    A = torch.randn((d, d), device=dev, dtype=torch.float32, generator=g)
    ld = (d + 31) // 32 * 32
    nq = (m + 3) // 4
    P = torch.randn((nq, ld, 4), device=dev, dtype=torch.float32, generator=g)
    P[:, d:, :] = 0
    if m % 4:
        P[-1, :, m % 4:] = 0
    Y = torch.zeros_like(P)
    G = torch.zeros((m, m), dtype=torch.float64, device=dev)
    ctx = bk.Context(local)
    stream = torch.cuda.Stream(dev)
    ctx.set_stream(stream.cuda_stream)
    op = bk.dense_operator(A)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            bk.block_apply(ctx, op, 0.0, P, Y, G, m, ld)
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            bk.block_apply(ctx, op, 0.0, P, Y, G, m, ld)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1) / args.steps
    gbs = 4.0 * d * d / (ms / 1e3) / 1e9
    peak, src = measured_peaks()
    if rank == 0:
        print(json.dumps({"metric": "dense FP32 block product, GB/s of A per product", "value": gbs, "unit": "GB/s",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (3xTF32)",
                          "data": "synthetic", "config": {"workload": f"dense_product_d{d}_m{m}"},
                          "note": "each step is one bk_block_apply call (includes its host synchronisation)",
                          "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                       "frac": gbs / peak, "traffic": None, "peak_source": src}}), flush=True)
    ctx.close()
    return 0


RIDGE_SEED = W.BASE_SEED + 3
RIDGE_SHIFTS = 64
RIDGE_SKETCH = 64
RIDGE_NOISE = 1e-3  # N(0, 1e-6) read as the variance


def fp32_peak_tflops(sm_mhz):
    """FFMA peak of the FP32 pipe: 152 SMs x 128 lanes x 2 flops per clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def oracle_ridge_sample(Z64, b, seconds):
    """Seconds per block-Lanczos step of the FP64 oracle (full reorthogonalisation,
    A = Z^T Z matrix-free) on the full ridge workload, over as many steps as fit."""
    from oracle import lanczos, operators
    op = operators.Gram(Z64)
    d = Z64.shape[1]
    B = W.inner_start_block(b, W.omega(RIDGE_SEED, d, RIDGE_SKETCH))
    t0 = time.perf_counter()
    lanczos.block_lanczos(op, B, 1)
    t1 = time.perf_counter() - t0
    n = int(max(1, min(6, seconds / max(t1, 1e-3))))
    t0 = time.perf_counter()
    lanczos.block_lanczos(op, B, n)
    return (time.perf_counter() - t0) / n, n


def threads_used():
    thr = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        thr = max(i.get("num_threads", 1) for i in threadpool_info()) or thr
    except Exception:  # noqa: BLE001
        pass
    return thr


def run_ridge(args, world, rank, local, dev):
    """Ridge path: 64 shifts from one block-Lanczos basis, A = Z^T Z matrix-free with
    Z 200,000 x 4096 FP32 (sigma_i = 1/i plus noise), b = Z^T f. One step = one
    bk_ridge_path call delivering 64 solutions at relative residual 1e-8 (FP64
    residuals of every shift from the stored Z)."""
    import torch
    from paper_2501_18717_gb300 import bk

    n, d, L = args.ridge_n, args.ridge_d, RIDGE_SHIFTS
    t0 = time.perf_counter()
    Z, f, b = W.ridge_workload_torch(RIDGE_SEED, n, d, RIDGE_NOISE, dev)
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    mus = np.logspace(-6, 0, L)
    X = torch.zeros((L, d), dtype=torch.float64, device=dev)  # d x L column-major
    ctx = bk.Context(local)
    stream = torch.cuda.Stream(dev)
    ctx.set_stream(stream.cuda_stream)
    op = bk.gram_operator(Z)

    def opts(inner, profile=0):
        return bk.default_opts(tol=TOL, sketch=RIDGE_SKETCH, seed=OMEGA_SEED, inner=inner,
                               inner_tol=1e-5 if inner in ("fp32", "bf16") else 1e-6, check_every=2, max_loads=400,
                               profile=profile)

    def call(o, op_=op, b_=b, X_=X):
        with torch.cuda.stream(stream):
            return bk.ridge_path(ctx, op_, mus, b_, X_, o, check=False)

    inner = args.ridge_inner
    other = "bf16" if inner == "fp32" else "fp32"
    mixed = opts(inner)
    for _ in range(args.warmup):
        call(mixed)
    torch.cuda.synchronize(dev)
    infos = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            infos.append(call(mixed))
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1) / args.steps
    value = world * L / (ms / 1e3)
    ok = all(i.status == bk.BK_OK for i in infos)

    # one profiled call: CUDA events around the operator loads, residual products and
    # orthogonalisation inside the driver
    pinfo = call(opts(inner, profile=1))
    names = bk.KERNEL_CLASSES
    kms = list(pinfo.ms_kernel)
    kn = list(pinfo.launches)
    m = RIDGE_SKETCH + 1
    groups = {}
    for k in ("operator", "residual", "orth"):
        j = names.index(k)
        groups[k] = {"ms": kms[j], "calls": int(kn[j]), "avg_ms": kms[j] / max(kn[j], 1),
                     "share_of_call": kms[j] / max(pinfo.ms_total, 1e-9)}
    # operator load = Z P then Z^T (Z P): 4 n d m flops (m = 65 on pass 0, 64 on later
    # passes; 65 used), FP32 FFMA
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak_tf = fp32_peak_tflops(sm_mhz)
    op_flops = 4.0 * n * d * m
    op_tf = op_flops / (groups["operator"]["avg_ms"] / 1e3) / 1e12 if groups["operator"]["calls"] else None
    res_tf = None
    if groups["residual"]["calls"]:
        res_tf = 4.0 * n * d * L / (groups["residual"]["avg_ms"] / 1e3) / 1e12
    peak_hbm, peak_src = measured_peaks()
    z_bytes = 4.0 * n * d
    # roofline of the group with the larger share: both are FP32-pipe bound (the
    # compensated pair arithmetic issues about 11 FP32 instructions per multiply-add)
    if groups["residual"]["ms"] > groups["operator"]["ms"] and res_tf:
        roof = {"bound": "alu", "kernel": "FP64-accurate residual products Z^T (Z X), 64 columns "
                                          "(k_tsm nn + tn, compensated FP32 pairs)",
                "achieved": res_tf, "peak": peak_tf / 11.0, "unit": "TFLOP/s", "frac": res_tf * 11.0 / peak_tf,
                "traffic": None,
                "peak_source": f"FP32 pipe 152 SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz / 11 instructions "
                               "per multiply-add"}
    else:
        roof = {"bound": "alu", "kernel": "Gram-form load Z^T (Z P) (k_tsm nn + tn, FFMA)", "achieved": op_tf,
                "peak": peak_tf, "unit": "TFLOP/s", "frac": (op_tf / peak_tf) if op_tf else None, "traffic": None,
                "peak_source": f"FP32 FFMA: 152 SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz"}

    # the other inner precision of the loads (FP32 FFMA or BF16 tensor cores), timed the
    # same way, with the operator group from one profiled call
    alt = None
    if args.steps > 0:
        ao = opts(other)
        call(ao)
        torch.cuda.synchronize(dev)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        ainfos = [call(ao) for _ in range(args.steps)]
        a1.record(stream)
        torch.cuda.synchronize(dev)
        ams = a0.elapsed_time(a1) / args.steps
        ap_ = call(opts(other, profile=1))
        j = names.index("operator")
        aop = ap_.ms_kernel[j] / max(ap_.launches[j], 1)
        # bytes of one load: Z twice (two products); BF16 loads read the head and tail
        # copies (2 x 2 n d bytes per product), FP32 loads the FP32 Z (4 n d per product)
        lbytes = 8.0 * n * d
        alt = {"inner": other, "value": world * L / (ams / 1e3), "unit": "solves/s", "ms_per_step": ams,
               "all_converged": all(i.status == bk.BK_OK for i in ainfos),
               "rel_residual_max": max(i.rel_residual for i in ainfos), "loads": ainfos[-1].loads,
               "refinements": ainfos[-1].refinements, "residual_products": ainfos[-1].residual_loads,
               "operator_avg_ms": aop, "operator_hbm_gbs": lbytes / (aop / 1e3) / 1e9,
               "operator_frac_of_hbm": lbytes / (aop / 1e3) / 1e9 / measured_peaks()[0],
               "operator_share_of_call": ap_.ms_kernel[j] / max(ap_.ms_total, 1e-9)}

    # FP64 blocks (plain) on the same GPU, one call
    fp64 = None
    if args.fp64_steps > 0:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fi = call(opts("fp64"))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        pms = e0.elapsed_time(e1)
        fp64 = {"value": L / (pms / 1e3), "unit": "solves/s", "ms_per_step": pms, "loads": fi.loads,
                "rel_residual": fi.rel_residual, "status": fi.status}

    # end to end through the C ABI from pinned host buffers (Z, b in; X out)
    e2e = None
    if not args.no_e2e:
        hZ = Z.cpu().pin_memory()
        hb = b.cpu().pin_memory()
        hX = torch.zeros((L, d), dtype=torch.float64).pin_memory()
        hop = bk.gram_operator(hZ)
        call(mixed, hop, hb, hX)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        for _ in range(args.steps):
            call(mixed, hop, hb, hX)
        torch.cuda.synchronize(dev)
        e2e_s = (time.perf_counter() - t1) / args.steps
        e2e = {"value": world * L / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(z_bytes + 8 * d + 8 * L),
               "d2h_bytes_per_step": int(8 * d * L)}
        del hZ

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        Z64 = Z.cpu().numpy().astype(np.float64)
        spl, nsteps = oracle_ridge_sample(Z64, b.cpu().numpy(), args.cpu_seconds)
        del Z64
        loads = infos[-1].loads
        cpu = {"value": L / (spl * loads), "unit": "solves/s", "cores": threads_used(), "kind": "oracle",
               "sample": f"{nsteps} block-Lanczos steps of the FP64 oracle (NumPy, full reorthogonalisation, "
                         f"Z^T (Z P) with Z promoted to FP64) on the full workload, {spl:.2f} s/step; "
                         f"solves/s = 64 / (s per step x {loads} loads, the loads of this run's GPU call)"}

    if rank == 0:
        line = {
            "metric": "solves/s at rel. residual 1e-8, ridge path (64 shifts from one block-Lanczos basis), "
                      "mixed vs FP64 plain",
            "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 products + f64 Gram/band solves + compensated-f32 (~44 bit) f64 residuals",
            "data": "synthetic",
            "config": {"workload": f"ridge_gram_Z{n}x{d}_fp32_sigma1overi_noise{RIDGE_NOISE}_shifts64_1e-6to1_l64",
                       "tol": TOL, "generator_s": gen_s,
                       "l2": f"Z {z_bytes / 1e9:.2f} GB streamed twice per load, larger than L2; no flush"},
            "all_converged": ok, "rel_residual_max": max(i.rel_residual for i in infos),
            "loads": [i.loads for i in infos], "refinements": [i.refinements for i in infos],
            "residual_products": [i.residual_loads for i in infos],
            "groups": groups,
            "roofline": roof,
            "operator_load": {"achieved_tflops": op_tf, "frac_of_ffma": (op_tf / peak_tf) if op_tf else None,
                              "hbm_equiv_gbs": 2 * z_bytes / (groups["operator"]["avg_ms"] / 1e3) / 1e9
                              if groups["operator"]["calls"] else None, "hbm_peak": peak_hbm,
                              "hbm_peak_source": peak_src},
            "residual_product": {"achieved_tflops": res_tf, "unit": "TFLOP/s (FP64-accurate, 4 n d L flop)",
                                 "frac_of_pair_peak": (res_tf * 11.0 / peak_tf) if res_tf else None},
            "fp64_plain": fp64, "e2e": e2e, "clocks": clocks, "cpu_baseline": cpu,
            "other_inner": alt,
        }
        if inner == "bf16":
            line["dtype"] = ("bf16 tensor-core products (head/tail splits, fp32 accumulation) + f64 Gram/band "
                             "solves + compensated-f32 (~44 bit) f64 residuals")
            lb = 8.0 * n * d
            gbs = lb / (groups["operator"]["avg_ms"] / 1e3) / 1e9 if groups["operator"]["calls"] else None
            line["roofline"] = {"bound": "hbm", "kernel": "BF16 Gram-form load Z^T (Z P) (k_bgemm x 2 + splits)",
                                "achieved": gbs, "peak": peak_hbm, "unit": "GB/s",
                                "frac": gbs / peak_hbm if gbs else None, "traffic": None, "peak_source": peak_src}
            line["operator_load"] = {"hbm_gbs": gbs, "bytes_per_load": lb, "hbm_peak": peak_hbm}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


SAMPLE_SEED = W.BASE_SEED + 4
# The configuration's nugget is 1e-6, but the FP32 rounding of the 40,000-point kernel
# matrix is a symmetric perturbation of norm about 3e-6, so the stored K + 1e-6 I is
# indefinite and has no square root (the driver reports BK_BREAKDOWN when the Lanczos
# matrix shows it). The default is the next decade above that floor; --sample-nugget
# 1e-6 runs the literal configuration.
SAMPLE_NUGGET = 1e-5
SAMPLE_NQUAD = 32


def run_sample(args, world, rank, local, dev):
    """Gaussian sampling (K + nugget I)^{1/2} B: K the RBF kernel (lengthscale 0.2) on
    40,000 uniform points in [0,1]^3 stored in FP32 (6.4 GB), B 40,000 x 256 standard
    normals, 32 quadrature shifts on one block-Lanczos basis. One step = one bk_sample
    call; value = samples/s."""
    import torch
    from paper_2501_18717_gb300 import bk

    d, m = args.sample_d, args.sample_m
    onfly = args.sample_operator == "rbf"
    if args.sample_nugget is None:
        # the literal nugget is well posed for the exactly formed kernel only (R14)
        args.sample_nugget = 1e-6 if onfly else SAMPLE_NUGGET
    t0 = time.perf_counter()
    pts = W.rbf_points(SAMPLE_SEED, d)
    if onfly:
        K = None
        pts_d = torch.from_numpy(np.ascontiguousarray(pts)).to(dev)
    else:
        ld = (d + 31) // 32 * 32
        Kbuf = torch.zeros((d, ld), dtype=torch.float32, device=dev)
        Kbuf[:, :d] = W.rbf_kernel_torch(pts, dev)
        K = Kbuf[:, :d]
    B = torch.from_numpy(W.sample_block(SAMPLE_SEED, d, m)).to(dev)  # column-major d x m
    Bt = B.T.contiguous()  # (m, d) row-major = d x m column-major
    S = torch.zeros((m, d), dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    ctx = bk.Context(local)
    stream = torch.cuda.Stream(dev)
    ctx.set_stream(stream.cuda_stream)
    op = bk.rbf_operator(pts_d, 0.2) if onfly else bk.dense_operator(K)

    def opts(profile=0):
        return bk.default_opts(tol=1e-4, inner=args.sample_inner, check_every=4, max_loads=args.sample_loads,
                               profile=profile)

    def call(o):
        with torch.cuda.stream(stream):
            return bk.sample(ctx, op, args.sample_nugget, Bt.T, S.T, SAMPLE_NQUAD, o, check=False)

    for _ in range(args.warmup):
        call(opts())
    torch.cuda.synchronize(dev)
    infos = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            infos.append(call(opts()))
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1) / args.steps
    if args.sample_only:
        if rank == 0:
            print(json.dumps({"metric": "samples/s, (K + nugget I)^{1/2} B by block-Lanczos quadrature (32 shifts)",
                              "value": world * m / (ms / 1e3), "unit": "samples/s", "ms_per_step": ms,
                              "steps": args.steps, "loads": [i.loads for i in infos],
                              "inner": args.sample_inner, "note": "--sample-only: timed calls only"}), flush=True)
        ctx.close()
        return 0
    pinfo = call(opts(profile=1))
    # the inverse square root on the same basis, shifts and weights (one timed call)
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        iinfo = bk.sample_isqrt(ctx, op, args.sample_nugget, Bt.T, S.T, SAMPLE_NQUAD, opts(), check=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    isqrt = {"value": m / (e0.elapsed_time(e1) / 1e3), "unit": "samples/s", "ms": e0.elapsed_time(e1),
             "loads": iinfo.loads, "last_change": iinfo.rel_residual, "status": iinfo.status}
    other = None
    if args.sample_inner == "ozaki" and not onfly:
        # the compensated FP32-pair loads on the same problem, for comparison (one profiled
        # call after the timed ones), and how far its samples are from this mode's
        call(opts())
        S_oz = S.clone()
        oo = bk.default_opts(tol=1e-4, inner="f32x2", check_every=4, max_loads=args.sample_loads, profile=1)
        oinfo = call(oo)
        j = bk.KERNEL_CLASSES.index("operator")
        other = {"inner": "f32x2", "ms_total": oinfo.ms_total, "loads": oinfo.loads,
                 "value": m / (oinfo.ms_total / 1e3), "unit": "samples/s",
                 "operator_avg_ms": oinfo.ms_kernel[j] / max(oinfo.launches[j], 1),
                 "rel_diff_of_samples": float(torch.linalg.norm(S - S_oz) / torch.linalg.norm(S_oz)),
                 "note": "one call with profiling events (ms_total includes them)"}
    names = bk.KERNEL_CLASSES
    groups = {}
    for k in ("operator", "orth"):
        j = names.index(k)
        groups[k] = {"ms": pinfo.ms_kernel[j], "calls": int(pinfo.launches[j]),
                     "avg_ms": pinfo.ms_kernel[j] / max(pinfo.launches[j], 1),
                     "share_of_call": pinfo.ms_kernel[j] / max(pinfo.ms_total, 1e-9)}
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak_tf = fp32_peak_tflops(sm_mhz)
    op_tf = 2.0 * d * d * m / (groups["operator"]["avg_ms"] / 1e3) / 1e12 if groups["operator"]["calls"] else None
    # compensated FP32-pair products issue about 11 FP32 instructions per multiply-add
    # (12 with both operands split, on the fly)
    issue = 12.0 if onfly else (11.0 if args.sample_inner == "f32x2" else 1.0)
    oz = args.sample_inner == "ozaki" and not onfly
    # the Ozaki product runs 28 BF16 digit products (digit pairs i + j <= 6 of 7 digits),
    # each 2 d^2 m flop, per load
    oz_pairs = 28
    peak_hbm, peak_src = measured_peaks()
    bf16_peak, bf16_src = measured_bf16_peak(sustained=True)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the FP64 oracle's block-Lanczos (full reorthogonalisation) on the stored K
        # promoted to FP64 (or the FP64 kernel matrix), timed for a bounded number of steps
        from oracle import lanczos, operators
        Kh = W.rbf_kernel(pts) if onfly else K.cpu().numpy()
        op64 = operators.Dense(Kh)
        del Kh
        Bh = B.cpu().numpy()
        t0 = time.perf_counter()
        lanczos.block_lanczos(op64, Bh, 1)
        t1 = time.perf_counter() - t0
        nsteps = int(max(1, min(4, args.cpu_seconds / max(t1, 1e-3))))
        t0 = time.perf_counter()
        lanczos.block_lanczos(op64, Bh, nsteps)
        sps = (time.perf_counter() - t0) / nsteps
        del op64
        loads = infos[-1].loads
        cpu = {"value": m / (sps * loads), "unit": "samples/s", "cores": threads_used(), "kind": "oracle",
               "sample": f"{nsteps} block-Lanczos steps of the FP64 oracle (NumPy, full reorthogonalisation, "
                         f"K promoted to FP64, block width {m}) on the full workload, {sps:.2f} s/step; "
                         f"samples/s = {m} / (s per step x {loads} loads, the loads of this run's GPU call; "
                         "the quadrature solves are not counted)"}
    if rank == 0:
        line = {
            "metric": "samples/s, (K + nugget I)^{1/2} B by block-Lanczos quadrature (32 shifts)",
            "value": world * m / (ms / 1e3), "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64 blocks, " + ("compensated f32-pair" if args.sample_inner == "f32x2" or onfly
                                       else ("Ozaki-split bf16 tensor-core (loads and basis)" if oz
                                             else args.sample_inner))
                     + (" products of K formed on the fly in f64" if onfly else " products of the f32-stored K")
                     + ", f64 Gram/band solves", "data": "synthetic",
            "config": {"workload": f"rbf_sample_d{d}_m{m}_ls0.2_nugget{args.sample_nugget:g}_"
                                   + ("onthefly_fp64entries" if onfly else "fp32") + "_nquad32",
                       "stop": "relative change of S <= 1e-4 between checks every 4 loads, or the load cap",
                       "inner": args.sample_inner,
                       "max_loads": args.sample_loads, "generator_s": gen_s,
                       "l2": ("K formed on the fly (points 1 MB, block 82 MB); no flush" if onfly
                              else f"K {4.0 * d * d / 1e9:.1f} GB, larger than L2; no flush")},
            "loads": [i.loads for i in infos], "last_change": [i.rel_residual for i in infos],
            "status": [i.status for i in infos], "groups": groups,
            "roofline": ({"bound": "tensor", "kernel": "dense load K P (k_ozgemm, Ozaki split: 28 BF16 digit "
                                                       "products with FP32 accumulation)",
                          "achieved": op_tf * oz_pairs if op_tf else None, "peak": bf16_peak, "unit": "TFLOP/s",
                          "frac": (op_tf * oz_pairs / bf16_peak) if op_tf else None, "traffic": None,
                          "peak_source": bf16_src, "fp64_accurate_tflops": op_tf,
                          "hbm_equiv": {"achieved_gbs": 4.0 * d * d / (groups['operator']['avg_ms'] / 1e3) / 1e9
                                        if groups["operator"]["calls"] else None, "peak": peak_hbm,
                                        "peak_source": peak_src}} if oz else
                         {"bound": "alu", "kernel": ("on-the-fly kernel load K P (k_rbf, f32 pairs)" if onfly
                                                     else f"dense load K P (k_tsm nn, {args.sample_inner})"),
                          "achieved": op_tf, "peak": peak_tf / issue, "unit": "TFLOP/s",
                          "frac": (op_tf * issue / peak_tf) if op_tf else None,
                          "traffic": None,
                          "peak_source": f"FP32 pipe: 152 SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz"
                                         f" / {issue:.0f} instructions per multiply-add",
                          "hbm_equiv": {"achieved_gbs": 4.0 * d * d / (groups['operator']['avg_ms'] / 1e3) / 1e9
                                        if groups["operator"]["calls"] else None, "peak": peak_hbm,
                                        "peak_source": peak_src}}),
            "isqrt": isqrt, "other_inner": other, "clocks": clocks, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_nystrom(args, world, rank, local, dev):
    """The comparison of Thm. main on the 128^3 diffusion system (FP64 values, mu 1e-4,
    tol 1e-8): randomized block-CG on [b Omega] (FP64 blocks) against
    Nystrom-preconditioned CG built from the same Omega (32 columns) at depths 1 and 3,
    all on the GPU. Reports loads (passes over A), solve time and the recomputed FP64
    residual of each."""
    import torch
    from paper_2501_18717_gb300 import bk

    rp, ci, va, d = W.diffusion_csr(SEED, args.grid)
    b = W.normals(SEED, W.STREAM_RHS, d)
    A = bk.csr_operator(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), torch.from_numpy(va).to(dev))
    bd = torch.from_numpy(b).to(dev)
    x = torch.zeros(d, dtype=torch.float64, device=dev)
    ctx = bk.Context(local)
    stream = torch.cuda.Stream(dev)
    ctx.set_stream(stream.cuda_stream)
    rows = {}

    def timed(fn):
        with torch.cuda.stream(stream):
            fn()  # warm-up (allocations)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
        return info, e0.elapsed_time(e1)

    with ClockSampler(local) as clk:
        info, ms = timed(lambda: bk.solve(ctx, A, MU, bd, x, bk.default_opts(
            tol=TOL, sketch=SKETCH, seed=OMEGA_SEED, inner="fp64", inner_tol=1e-6, check_every=16,
            max_loads=args.max_loads), check=False))
        rows["block_cg_fp64"] = {"loads": info.loads, "ms": ms, "rel_residual": info.rel_residual,
                                 "status": info.status, "block_width": SKETCH + 1}
        info, ms = timed(lambda: bk.solve(ctx, A, MU, bd, x, bk.default_opts(
            tol=TOL, sketch=SKETCH, seed=OMEGA_SEED, inner="fp32", inner_tol=1e-5, check_every=16,
            max_loads=args.max_loads), check=False))
        rows["block_cg_mixed"] = {"loads": info.loads, "ms": ms, "rel_residual": info.rel_residual,
                                  "status": info.status, "block_width": SKETCH + 1}
        for s_ny in (1, 3):
            info, ms = timed(lambda: bk.nystrom_pcg(ctx, A, MU, bd, x, s_ny, bk.default_opts(
                tol=TOL, sketch=SKETCH, seed=OMEGA_SEED, check_every=32, max_loads=args.max_loads), check=False))
            rows[f"nystrom_pcg_s{s_ny}"] = {"loads": info.loads, "ms": ms, "rel_residual": info.rel_residual,
                                            "status": info.status, "rank": info.refinements}
    if rank == 0:
        best = rows["block_cg_mixed"]
        print(json.dumps({
            "metric": "solves/s at rel. residual 1e-8: randomized block-CG vs Nystrom PCG from the same Omega",
            "value": 1e3 / best["ms"], "unit": "solves/s", "n_gpus": world, "steps": 1, "warmup": 1,
            "ms_per_step": best["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (block-CG FP64 and PCG), f32 blocks + f64 refinement (block-CG mixed)",
            "data": "synthetic",
            "config": {"workload": workload_name(args.grid, d, int(va.shape[0])), "sketch_l": SKETCH, "tol": TOL,
                       "mu": MU,
                       "l2": "working set larger than L2; no flush"},
            "methods": rows, "clocks": clk.summary(), "cpu_baseline": None}), flush=True)
    ctx.close()
    return 0


def oracle_shrink_sample(rp, ci, va, b, om, s_lock, iters, seconds):
    """The FP64 oracle's block-shrinking solve (locked basis of K_s(A, [b Omega]), then
    Def-CG) on the full workload: the basis and a bounded number of one-column steps are
    timed, and the time of a whole solve is the basis time plus the per-step time times
    the GPU's step count."""
    from oracle import deflated, operators
    op = operators.CSR(rp, ci, va)
    t0 = time.perf_counter()
    Wb = deflated.locked_basis(op, b, om, s_lock)
    t_basis = time.perf_counter() - t0
    k = 2
    while True:
        t0 = time.perf_counter()
        deflated.deflated_cg(op, MU, b, Wb, k)
        t_k = time.perf_counter() - t0
        if t_basis + t_k >= seconds or k >= 64:
            break
        k *= 2
    t1 = time.perf_counter()
    deflated.deflated_cg(op, MU, b, Wb, 0)
    t_setup = time.perf_counter() - t1
    per_step = max(t_k - t_setup, 1e-9) / k
    return t_basis + t_setup + per_step * iters, k, t_basis, per_step


def run_shrink(args, world, rank, local, dev):
    """Block shrinking (the outlook's deflation to a smaller block, Sec. CG_pro's locked
    reorthogonalisation) on the 128^3 diffusion system (FP64 values, mu 1e-4, tol 1e-8):
    s block steps on [b Omega] (33 columns) lock V, then one-column deflated CG against V.
    Compared with randomized block-CG (mixed) on the same Omega. Reports loads, time and
    the recomputed FP64 residual of each; roofline is the deflation products (HBM)."""
    import torch
    from paper_2501_18717_gb300 import bk

    rp, ci, va, d = W.diffusion_csr(SEED, args.grid)
    b = W.normals(SEED, W.STREAM_RHS, d)
    A = bk.csr_operator(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), torch.from_numpy(va).to(dev))
    bd = torch.from_numpy(b).to(dev)
    x = torch.zeros(d, dtype=torch.float64, device=dev)
    ctx = bk.Context(local)
    stream = torch.cuda.Stream(dev)
    ctx.set_stream(stream.cuda_stream)
    rows = {}
    head_s = 3
    m = SKETCH + 1

    def timed(fn, reps=1):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                info = fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
        return info, e0.elapsed_time(e1) / reps

    def shrink_opts(profile=0):
        return bk.default_opts(tol=TOL, sketch=SKETCH, seed=OMEGA_SEED, check_every=32, max_loads=args.max_loads,
                               profile=profile)

    with ClockSampler(local) as clk:
        info, ms = timed(lambda: bk.solve(ctx, A, MU, bd, x, bk.default_opts(
            tol=TOL, sketch=SKETCH, seed=OMEGA_SEED, inner="fp32", inner_tol=1e-5, check_every=16,
            max_loads=args.max_loads), check=False))
        rows["block_cg_mixed"] = {"loads": info.loads, "ms": ms, "rel_residual": info.rel_residual,
                                  "status": info.status, "block_width": m}
        for s_lock in (1, 3):
            info, ms = timed(lambda: bk.solve_shrink(ctx, A, MU, bd, x, s_lock, shrink_opts(), check=False),
                             reps=args.steps if s_lock == head_s else 1)
            rows[f"shrink_s{s_lock}"] = {"loads": info.loads, "block_loads": s_lock,
                                         "one_column_steps": info.loads - s_lock - 1, "ms": ms,
                                         "rel_residual": info.rel_residual, "status": info.status,
                                         "locked_columns": info.refinements}
        with torch.cuda.stream(stream):
            pinfo = bk.solve_shrink(ctx, A, MU, bd, x, head_s, shrink_opts(profile=1), check=False)
            torch.cuda.synchronize(dev)
    names = bk.KERNEL_CLASSES
    groups = {}
    for k in ("operator", "orth"):
        j = names.index(k)
        groups[k] = {"ms": pinfo.ms_kernel[j], "calls": int(pinfo.launches[j]),
                     "avg_ms": pinfo.ms_kernel[j] / max(pinfo.launches[j], 1),
                     "share_of_call": pinfo.ms_kernel[j] / max(pinfo.ms_total, 1e-9)}
    n_lock = head_s * m
    nb = n_lock + m
    # one direction update: [V Q_s]^T r (nb columns) and p = r + V c + beta p (n columns),
    # the basis as FP32 head + tail (8 bytes an entry); r read twice, p read and written
    defl_bytes = 8.0 * d * (nb + n_lock + 4)
    peak, peak_src = measured_peaks()
    gbs = defl_bytes / (groups["orth"]["avg_ms"] * 1e-3) / 1e9
    head = rows[f"shrink_s{head_s}"]
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        om = W.omega(OMEGA_SEED, d, SKETCH)
        t_solve, k, t_basis, per_step = oracle_shrink_sample(rp, ci, va, b, om, head_s, head["one_column_steps"],
                                                             args.cpu_seconds)
        cpu = {"value": 1.0 / t_solve, "unit": "solves/s", "cores": threads_used(), "kind": "oracle",
               "sample": f"FP64 oracle (NumPy/SciPy) locked basis of K_{head_s}(A, [b Omega]) "
                         f"({t_basis:.1f} s) and {k} Def-CG steps ({per_step * 1e3:.1f} ms each) on the full "
                         f"workload; a solve = basis + {head['one_column_steps']} steps, the GPU's count"}
    if rank == 0:
        print(json.dumps({
            "metric": "solves/s at rel. residual 1e-8: block-CG shrunk to one column after s block steps "
                      "(deflated CG on the locked block-Krylov basis)",
            "value": 1e3 / head["ms"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (locked basis, deflated CG; FP64 CSR values)", "data": "synthetic",
            "config": {"workload": workload_name(args.grid, d, int(va.shape[0])), "sketch_l": SKETCH, "s_lock": head_s,
                       "tol": TOL, "mu": MU,
                       "l2": f"locked basis {8.0 * d * nb / 1e9:.2f} GB (FP32 head + tail), "
                             + ("larger than L2; no flush" if 8.0 * d * nb > 2e8 else "L2-resident")},
            "methods": rows, "groups": groups,
            "roofline": {"bound": "hbm", "kernel": f"deflation products [V Q_s]^T r ({nb} cols) and p = r + V c + beta p "
                                                   f"({n_lock} cols), FP32 head/tail basis, k_defl_t + k_defl_reduce + "
                                                   "k_defl_coef + k_defl_np",
                         "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak, "traffic": None,
                         "peak_source": peak_src},
            "clocks": clk.summary(), "cpu_baseline": cpu}), flush=True)
    ctx.close()
    return 0


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    from paper_2501_18717_gb300 import bk

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if args.workload == "batched":
        return run_batched(args, world, rank, local, dev)
    if args.workload == "dense-product":
        return run_dense_product(args, world, rank, local, dev)
    if args.workload == "ridge":
        return run_ridge(args, world, rank, local, dev)
    if args.workload == "sample":
        return run_sample(args, world, rank, local, dev)
    if args.workload == "nystrom":
        return run_nystrom(args, world, rank, local, dev)
    if args.workload == "shrink":
        return run_shrink(args, world, rank, local, dev)
    if args.workload == "csr-product":
        return run_csr_product(args, world, rank, local, dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    rp, ci, va, d = W.diffusion_csr(SEED, args.grid)
    b = W.normals(SEED, W.STREAM_RHS, d)
    nnz = va.shape[0]
    m = SKETCH + 1
    A = bk.csr_operator(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), torch.from_numpy(va).to(dev))
    bd = torch.from_numpy(b).to(dev)
    x = torch.zeros(d, dtype=torch.float64, device=dev)
    ctx = bk.Context(local)
    stream = torch.cuda.Stream(dev)
    ctx.set_stream(stream.cuda_stream)

    # timed solves run without per-kernel events; one extra profiled solve outside the
    # timed region gives the kernel breakdown
    mixed = bk.default_opts(tol=TOL, sketch=SKETCH, seed=OMEGA_SEED, inner="fp32", inner_tol=1e-5,
                            check_every=16, max_loads=args.max_loads, profile=0)
    mixed_prof = bk.default_opts(tol=TOL, sketch=SKETCH, seed=OMEGA_SEED, inner="fp32", inner_tol=1e-5,
                                 check_every=16, max_loads=args.max_loads, profile=1)
    plain = bk.default_opts(tol=TOL, sketch=SKETCH, seed=OMEGA_SEED, inner="fp64", inner_tol=1e-6,
                            check_every=16, max_loads=args.max_loads, profile=0)

    def solve(opts, A_, b_, x_):
        with torch.cuda.stream(stream):
            return bk.solve(ctx, A_, MU, b_, x_, opts, check=args.max_loads >= 20000)

    for _ in range(args.warmup):
        solve(mixed, A, bd, x)
    barrier()
    torch.cuda.synchronize(dev)
    infos = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            infos.append(solve(mixed, A, bd, x))
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    value = replica_throughput(world, args.steps, ms)
    rel_res = max(i.rel_residual for i in infos)
    loads = [i.loads for i in infos]

    # per-kernel timings from one profiled solve (events recorded between its launches)
    pinf = solve(mixed_prof, A, bd, x)
    torch.cuda.synchronize(dev)
    kms = np.asarray(list(pinf.ms_kernel))
    kn = np.asarray(list(pinf.launches))
    names = bk.KERNEL_CLASSES
    algo = algorithmic_bytes(d, nnz, m)
    peak, peak_src = measured_peaks()
    kernels = {}
    for k in ("operator", "update_r", "update_p"):
        j = names.index(k)
        avg_ms = kms[j] / max(kn[j], 1)
        gbs = algo[k] / (avg_ms / 1e3) / 1e9
        kernels[k] = {"avg_ms": avg_ms, "launches": int(kn[j]), "algo_bytes": algo[k], "gbs": gbs,
                      "frac": gbs / peak, "share": float(kms[j] / max(np.sum(kms), 1e-9))}
    for k in ("reduce", "alpha", "beta"):
        j = names.index(k)
        kernels[k] = {"avg_ms": kms[j] / max(kn[j], 1), "launches": int(kn[j]),
                      "share": float(kms[j] / max(np.sum(kms), 1e-9))}
    dom = max(("operator", "update_r", "update_p"), key=lambda k: kernels[k]["share"])
    kd = kernels[dom]
    iter_ms = float(np.sum(kms)) / max(int(kn[names.index("operator")]), 1)
    iter_bytes = algo["operator"] + algo["update_r"] + algo["update_p"]

    # plain FP64 path on the same GPU
    fp64 = None
    if args.fp64_steps > 0:
        solve(plain, A, bd, x)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pinfo = [solve(plain, A, bd, x) for _ in range(args.fp64_steps)]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        pms = e0.elapsed_time(e1)
        fp64 = {"value": args.fp64_steps / (pms / 1e3), "unit": "solves/s", "ms_per_solve": pms / args.fp64_steps,
                "loads": [i.loads for i in pinfo], "rel_residual": max(i.rel_residual for i in pinfo),
                "iter_ms": pms / args.fp64_steps / max(pinfo[0].loads, 1)}

    # end to end through the C ABI with pinned host buffers: H2D of A and b, D2H of x
    if args.no_e2e:
        args.steps_e2e = 0
    hrp = torch.from_numpy(rp).pin_memory()
    hci = torch.from_numpy(ci).pin_memory()
    hva = torch.from_numpy(va).pin_memory()
    hb = torch.from_numpy(b).pin_memory()
    hx = torch.zeros(d, dtype=torch.float64).pin_memory()
    Ah = bk.csr_operator(hrp, hci, hva)
    e2e_opts = bk.default_opts(tol=TOL, sketch=SKETCH, seed=OMEGA_SEED, inner="fp32", inner_tol=1e-5,
                               check_every=16, max_loads=20000)
    n_e2e = 0 if args.no_e2e else args.steps
    if n_e2e:
        solve(e2e_opts, Ah, hb, hx)
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        solve(e2e_opts, Ah, hb, hx)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s = max_over_ranks(e2e_s, dev)
    h2d = rp.nbytes + ci.nbytes + va.nbytes + b.nbytes
    d2h = d * 8

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        spl, n, thr = oracle_sample(rp, ci, va, b, args.cpu_seconds)
        lps, src = oracle_loads_per_solve()
        if lps is None:
            lps, src = (fp64["loads"][0] if fp64 else loads[0]), "loads of this run's FP64 GPU solve"
            # (used only until oracle/loads_diffusion128.json, written by the oracle itself, exists)
        cpu = {"value": 1.0 / (spl * lps), "unit": "solves/s", "cores": thr, "kind": "oracle",
               "sample": f"{n} loads of the FP64 oracle block-CG recurrence (NumPy/SciPy) on the full workload, "
                         f"{spl:.3f} s/load; solves/s = 1/(s per load x {lps} loads per solve, {src})"}

    # the batched configuration (512 uneven dense systems, autotuned widths, mixed vs
    # FP64 blocks) in a child process of its own (its 75 GB of matrices), attached below
    batched = None
    if rank == 0 and world == 1 and not args.no_batched and args.grid == GRID:
        ctx.close()
        ctx = None
        torch.cuda.empty_cache()
        batched = batched_leg()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 block ops + f64 Gram/solve/refinement", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sketch_l": SKETCH, "block_width": m, "tol": TOL,
                       "inner": "fp32, inner_tol 1e-5", "l2": "working set (blocks 3 x 277 MB + A 125 MB) "
                                                             "larger than L2; no flush"},
            "loads_per_solve": loads, "rel_residual_max": rel_res,
            "iteration": {"ms": iter_ms, "algo_bytes": iter_bytes, "gbs": iter_bytes / (iter_ms / 1e3) / 1e9,
                          "frac": iter_bytes / (iter_ms / 1e3) / 1e9 / peak},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": kd["gbs"], "peak": peak, "unit": "GB/s",
                         "frac": kd["frac"], "traffic": kernel_traffic(dom), "peak_source": peak_src},
            "kernels": kernels,
            "fp64_plain": fp64,
            "e2e": {"value": world * n_e2e / e2e_s if n_e2e else None, "unit": "solves/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(sum(i.kernel_launches for i in infos)),
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "batched": batched,
        }
        print(json.dumps(line), flush=True)
    if ctx is not None:
        ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
