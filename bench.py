#!/usr/bin/env python
"""Benchmark of the LOOPS hybrid SpMM on GB300: SpMM GFLOP/s (2 * nnz * N per call) and the
roofline fraction of the dominant kernel, hybrid vs CSR-only, at a stated rel-L2 against the
FP64 oracle.

Default line: the largest single-GPU workload, a batch of 512 sparse matrices of 1,000 to
65,536 rows (uniform rows, banded |i - j| <= 16, and two dense 16 x 16 blocks per 16-row
block, by index mod 3; 275.7 M nonzeros, N drawn from {16, 32, 64, 128}) in FP32, run by one
graph-captured batched call. One step is one C_m = A_m . B_m of every matrix of the batch on
operands resident in HBM; the plan (partition and layout, built once, as the paper excludes
format conversion from its timing) is made before timing. L2 is flushed (a 256 MiB write, then
a read) before every timed step; every step is timed on the device with CUDA events. The line
carries the other workloads as sub-lines (``workloads``): the FP64 Laplacian with dense blocks,
the R-MAT graph in FP16 and BF16, the GCN layer forward and backward, and the small plain CSR
case, each with its own roofline and error.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl loops|reference]
                  [--workload batched|laplacian|rmat|gcn|uniform|mixed] [--dtype ...]

Under torchrun each rank runs its own replica of the workload on its GPU (the path needs no
exchange); rank 0 prints one JSON line with the whole-job throughput (max time over ranks).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "SpMM GFLOP/s (2·nnz·N) and % HBM roofline, hybrid vs CSR-only at stated rel-L2"
HBM_NOMINAL_GBS = 8000.0
# FP64 peak of this GPU, measured: 8 independent DFMA chains per thread, 8 blocks of 256
# threads per SM, CUDA events, SM clock 2,070 MHz throughout (profiles/fp64_peak_probe.md).
FP64_PEAK_TFLOPS = 1.2033
FP64_PEAK_SOURCE = ("measured DFMA throughput, 1.2033 TFLOP/s at 2,070 MHz (profiles/fp64_peak_probe.md); "
                    "nominal 152 SMs x 2 FMA/clk x 2 FLOP x 2.07 GHz = 1.259")
TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 2e-3, "bf16": 2e-3}
BATCH_COUNT, BATCH_SEED = 512, 5


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["loops", "reference"], default="loops")
    ap.add_argument("--workload", choices=["batched", "laplacian", "rmat", "gcn", "uniform", "mixed"],
                    default="batched",
                    help="batched (default: the 512-matrix batch, with the other workloads as sub-lines) "
                         "or one workload alone, measured the same way")
    ap.add_argument("--dtype", default=None, help="batched: f32 (default) or bf16; rmat: f16 or bf16; "
                                                  "mixed: f32 or bf16")
    ap.add_argument("--N", type=int, default=64, help="laplacian: columns of B")
    ap.add_argument("--batch-count", type=int, default=BATCH_COUNT,
                    help="batched: number of matrices (smaller counts give small profiling cases)")
    ap.add_argument("--batch-kinds", default="all", choices=["all", "uniform", "banded", "blocks"],
                    help="batched: keep only the matrices of one structure (index mod 3), for profiling cases")
    ap.add_argument("--block-rows", type=int, default=0,
                    help="batched: B_r of the plan (0: autotuned, or the default with a fixed --tau)")
    ap.add_argument("--tau", type=float, default=-1.0,
                    help="batched: split threshold of the timed plan (default -1: autotuned)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="batched: skip the sub-line workloads")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def host_cores() -> int:
    """Host threads available to this process."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"loops_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)"
    return 6800.0, "fallback"


def traffic_for(kernel_key: str):
    """DRAM bytes per launch of a kernel from the committed ncu summary, if the sources it was
    captured from are unchanged since the capture (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel_key)
    if not d:
        return None
    srcs = d["sources"] if "sources" in d else {d["source"]: d["source_sha256"]}
    for src, sha in srcs.items():
        path = os.path.join(ROOT, src)
        if not os.path.exists(path) or hashlib.sha256(open(path, "rb").read()).hexdigest() != sha:
            return None
    return d["dram_bytes_per_launch"]


def max_over_ranks(torch, x: float, world: int, device) -> float:
    """The largest value of x over all ranks (the job's time is its slowest rank's)."""
    t = torch.tensor([x], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_gflops(flops_per_rank_step: float, world: int, ms_step: float) -> float:
    """Whole-job throughput: every rank processes its own replica of the step."""
    return world * flops_per_rank_step / (ms_step * 1e-3) / 1e9


def csr_alg_bytes(n_rows, n_cols, nnz, N, e, c) -> int:
    """Algorithmic bytes of one SpMM: A once (row pointers, column indices, values in the
    compute dtype), B once and C once (gathers and padding not counted)."""
    return (n_rows + 1) * 8 + nnz * (4 + e) + n_cols * N * e + n_rows * N * c


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nr = np.linalg.norm(ref)
    if nr == 0.0:
        return 0.0 if np.all(got == 0) else float("inf")
    return float(np.linalg.norm(got - ref) / nr)


def make_flush(torch):
    """L2 flush: write a 256 MiB buffer (larger than the 126 MiB L2), then read another one so
    the dirty lines are written back before the timed kernel starts, not during it."""
    flush_w = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush_r = torch.ones(64 << 20, dtype=torch.float32, device="cuda")
    flush_out = torch.empty((), dtype=torch.float32, device="cuda")

    def flush():
        flush_w.zero_()
        torch.sum(flush_r, dim=0, out=flush_out)
    return flush


def new_events(torch, n):
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    s = torch.cuda.current_stream()
    for e in evs:                 # materialise the handles
        e.record(s)
    torch.cuda.synchronize()
    return evs


def time_steps(torch, fn, steps, warmup, flush, plan=None):
    """Per-step device times (ms) of fn() with the L2 flushed before each step, and (with a
    plan) the times between its timing events [0]-[1] and [2]-[3] in each step."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    pev = [new_events(torch, 4) for _ in range(steps)] if plan is not None else None
    # the plan records timing events from the warm-up on, so a batched plan's graph already
    # holds its event nodes (later steps only repoint them) before the timed steps
    if plan is not None:
        plan.set_timing_events([e.cuda_event for e in pev[0]])
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    for k in range(steps):
        flush()
        if plan is not None:
            plan.set_timing_events([e.cuda_event for e in pev[k]])
        ev[k][0].record(stream)
        fn()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if plan is not None:
        plan.set_timing_events(None)
    step = [a.elapsed_time(b) for a, b in ev]
    p01 = [r[0].elapsed_time(r[1]) for r in pev] if pev else []
    p23 = [r[2].elapsed_time(r[3]) for r in pev] if pev else []
    return step, p01, p23


def rounded_matrix(A, fmt):
    """A with the values the plan stores: round(s_A * a) / s_A in the format (s_A the plan's
    power-of-two scale; exact undo)."""
    import oracle

    if fmt == "f64":
        return A
    s = oracle.plan_scale(A.vals, fmt)
    return W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, oracle.round_to(A.vals * s, fmt) / s)


def launches_per_step(info) -> int:
    """Library kernels one single-matrix SpMM launches: CSR part, its split-row sums, BCSR part,
    its split-block sums, the tile-level split's second CSR pass."""
    return (int(info["n_csr_rows"] > 0) + int(info["n_split_rows"] > 0) + int(info["n_row_blocks"] > 0))


def oracle_batch(mats, Bs, threads):
    """The oracle (FP64 C row loop) on every matrix of a batch, matrices spread over host
    threads (each matrix on one thread)."""
    import oracle

    with ThreadPoolExecutor(max(1, threads)) as ex:
        return list(ex.map(lambda ab: oracle.spmm(ab[0], ab[1]), zip(mats, Bs)))


# ------------------------------------------------------------------ the 512-matrix batch
def batch_inputs(count: int, fmt: str, kinds: str = "all"):
    """The batch (A_m, N_m) and its dense operands B_m (host, float32 N(0, 1), seeded per
    matrix); for BF16 the values the GPU multiplies are the BF16 roundings. kinds: all, or only
    the uniform / banded / blocks matrices (index mod 3 = 0 / 1 / 2)."""
    mats = W.batched_mix(count=count, seed=BATCH_SEED)
    Bs = [W.dense_normal(A.n_cols, N, 10_000 + m).astype(np.float32) for m, (A, N) in enumerate(mats)]
    if kinds != "all":
        k = {"uniform": 0, "banded": 1, "blocks": 2}[kinds]
        keep = [m for m in range(len(mats)) if m % 3 == k]
        mats, Bs = [mats[m] for m in keep], [Bs[m] for m in keep]
    return mats, Bs


def batch_config(count: int, fmt: str, nnz: int) -> dict:
    return {"workload": f"batch of {count} sparse matrices (1,000-65,536 rows; uniform 8-64 per row / banded "
                        f"|i-j|<=16 / two dense 16x16 blocks per 16-row block, by index mod 3), "
                        f"N in {{16,32,64,128}}, {fmt.upper()}",
            "count": count, "nnz": int(nnz), "dtype": fmt,
            "l2": "flushed before every timed step (256 MiB write, then a 256 MiB read); the batch's B and "
                  "C (4 GB in FP32) exceed L2 as well",
            "plan": "built once before timing (conversion excluded as in the paper)"}


def run_batched(args, torch, lp, flush, rank, world, hbm_peak, hbm_src):
    fmt = args.dtype or "f32"
    e = 4 if fmt == "f32" else 2
    dt = torch.float32 if fmt == "f32" else torch.bfloat16
    t0 = time.perf_counter()
    mats, Bh = batch_inputs(args.batch_count, fmt, args.batch_kinds)
    gen_s = time.perf_counter() - t0
    As = [A for A, _ in mats]
    Ns = [N for _, N in mats]
    nnz = sum(A.nnz for A in As)
    flops = sum(2.0 * A.nnz * N for A, N in mats)
    alg = sum(csr_alg_bytes(A.n_rows, A.n_cols, A.nnz, N, e, 4) for A, N in mats)
    Bd = [torch.as_tensor(B).to(dt).cuda() for B in Bh]
    Cd = [torch.empty((A.n_rows, N), device="cuda") for A, N in mats]

    t0 = time.perf_counter()
    plan = lp.BatchedPlan(As, Ns, fmt, tau=args.tau, block_rows=args.block_rows)
    plan_s = time.perf_counter() - t0
    st = plan.stats()

    # main timed region: K steps, barrier + synchronize on both sides, clocks sampled
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    for _ in range(args.warmup):
        plan.spmm(Bd, Cd)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    step, kern, red = time_steps(torch, lambda: plan.spmm(Bd, Cd), args.steps, 0, flush, plan=plan)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    if world > 1:
        torch.distributed.barrier()
    ms_step = max_over_ranks(torch, sum(step), world, "cuda") / args.steps
    value = whole_job_gflops(flops, world, ms_step)
    kern_ms = statistics.mean(kern)
    achieved = alg / (kern_ms * 1e-3) / 1e9

    # parity of the timed plan's output: every matrix against the oracle (FP64, same rounded
    # inputs); the max over matrices of the per-matrix rel-L2
    plan.spmm(Bd, Cd)
    torch.cuda.synchronize()
    rel_max = None
    if rank == 0:
        Bq = [torch.as_tensor(B).to(dt).double().numpy() for B in Bh]   # the values the GPU multiplies
        refs = oracle_batch([rounded_matrix(A, fmt) for A in As], Bq, host_cores())
        rels = [rel_l2(C.double().cpu().numpy(), R) for C, R in zip(Cd, refs)]
        rel_max = max(rels)
        del refs, Bq

    # hybrid vs CSR-only (same inputs, same accuracy), fewer steps
    variants = {}
    for name, tau in (("csr_only", math.inf), ("hybrid_tau2", 2.0)):
        vp = lp.BatchedPlan(As, Ns, fmt, tau=tau)
        torch.cuda.nvtx.range_push(f"variant:{name}")
        s_v, k_v, _ = time_steps(torch, lambda: vp.spmm(Bd, Cd), max(5, args.steps // 2), 2, flush, plan=vp)
        torch.cuda.nvtx.range_pop()
        ms = statistics.mean(s_v)
        variants[name] = {"tau": tau, "gflops": flops / (ms * 1e-3) / 1e9, "ms_per_step": ms,
                          "kernel_ms": statistics.mean(k_v), "nnz_bcsr": vp.stats()["nnz_bcsr"]}
        vp.destroy()
    plan.spmm(Bd, Cd)

    # end to end through the C ABI with pinned host buffers: every step copies all B_m in and
    # all C_m out (loops_spmm_batched_host synchronises). The host operands live back to back
    # in one pinned arena for B and one for C, as the host call's documentation advises (the
    # matrices of each pipeline group then move in one copy per direction).
    e2e = None
    if not args.no_e2e:
        arena_b = torch.empty(sum(B.size for B in Bh), dtype=dt).pin_memory()
        arena_c = torch.empty(sum(A.n_rows * N for A, N in mats), dtype=torch.float32).pin_memory()
        Bp, Cp, ob, oc = [], [], 0, 0
        for B, (A, N) in zip(Bh, mats):
            v = arena_b[ob: ob + B.size].view(B.shape)
            v.copy_(torch.as_tensor(B).to(dt))
            Bp.append(v)
            ob += B.size
            Cp.append(arena_c[oc: oc + A.n_rows * N].view(A.n_rows, N))
            oc += A.n_rows * N
        k_e2e = max(3, min(args.steps, 10))
        for _ in range(2):
            plan.spmm_host(Bp, Cp)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            plan.spmm_host(Bp, Cp)
        t_e2e = (time.perf_counter() - t0) * 1e3 / k_e2e
        h2d = int(sum(B.numel() * B.element_size() for B in Bp))
        d2h = int(sum(C.numel() * 4 for C in Cp))
        same = all(torch.equal(c.cpu(), h) for c, h in zip(Cd, Cp))
        e2e = {"value": world * flops / (t_e2e * 1e-3) / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": t_e2e,
               "link_gbs": (h2d + d2h) / (t_e2e * 1e-3) / 1e9, "matches_device_call": bool(same),
               "api": "loops_spmm_batched_host (pinned host B_m and C_m back to back in one arena each, "
                      "copied in and out every step in 16 pipelined groups, host wall clock per synchronous "
                      "call)"}
        del Bp, Cp, arena_b, arena_c

    cpu = None
    if rank == 0 and world == 1:
        cpu = batch_cpu_baseline(mats, Bh, budget_s=12.0)

    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": fmt,
            "data": "synthetic (seeded: matrices of the batch recipe, B ~ N(0,1) per matrix)",
            "config": dict(batch_config(args.batch_count, fmt, nnz), parallelism=f"replicas{world}",
                           kinds=args.batch_kinds,
                           tau_autotuned=st["tau"], block_rows=st["block_rows"], plan_build_s=plan_s,
                           input_generation_s=gen_s),
            "roofline": {"bound": "hbm", "kernel": "batched persistent kernel(s) (one graph replay)",
                         "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                         "traffic": traffic_for(f"batched_{fmt}_batch{args.batch_count}"),
                         "peak_source": hbm_src, "alg_bytes_per_launch": alg, "kernel_ms": kern_ms,
                         "partial_sum_ms": statistics.mean(red),
                         "alg_bytes": "sum over matrices of A once (row_ptr 8 B/row, 4 B index + value per "
                                      "nonzero) + B once + C once"},
            "hbm": {"alg_bytes_per_step": alg, "achieved_gbs": alg / (ms_step * 1e-3) / 1e9,
                    "frac_of_measured": alg / (ms_step * 1e-3) / 1e9 / hbm_peak,
                    "frac_of_8tbs": alg / (ms_step * 1e-3) / 1e9 / HBM_NOMINAL_GBS},
            "rel_l2_vs_oracle": rel_max, "rel_l2_what": "max over the 512 matrices of ||C - C_oracle|| / ||C_oracle||, "
                                                        "oracle in FP64 on the same rounded inputs",
            "rel_l2_tol": TOL[fmt],
            "variants": variants, "hybrid_over_csr_only": variants["csr_only"]["ms_per_step"] / ms_step,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": st["n_kernels"] * args.steps, "plan": st}
    return line


def batch_cpu_baseline(mats, Bh, budget_s=12.0):
    """The oracle as it stands on a bounded sample of the batch (every 8th matrix: all three
    structures and all N), matrices spread over all host threads, repeated for about budget_s."""
    import oracle

    oracle.build()
    threads = host_cores()
    idx = list(range(0, len(mats), 8))
    sub = [mats[i][0] for i in idx]
    Bs = [Bh[i].astype(np.float64) for i in idx]
    flops = sum(2.0 * mats[i][0].nnz * mats[i][1] for i in idx)
    reps, t_tot = 0, 0.0
    while reps < 1 or (t_tot < budget_s and reps < 50):
        t0 = time.perf_counter()
        oracle_batch(sub, Bs, threads)
        t_tot += time.perf_counter() - t0
        reps += 1
    return {"value": flops * reps / t_tot / 1e9, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
            "sample": f"every 8th matrix of the batch ({len(idx)} matrices, {flops / 1e9:.2f} GFLOP) x {reps} "
                      f"runs ({t_tot:.1f} s); FP64 C oracle, one matrix per host thread"}


# ------------------------------------------------------------------ single-matrix workloads
def single_inputs(name: str, fmt: str | None, N: int = 64):
    """(A, B, N, fmt, description, extra) of a single-matrix workload; extra holds the GCN dY."""
    if name == "laplacian":
        A, B = W.laplacian_blocks(grid=512, n_blocks=4096, block=8, seed=1, N=N)
        return A, B, N, "f64", f"laplacian512+4096x8x8 blocks, FP64, N={N}", None
    if name == "rmat":
        fmt = fmt or "f16"
        A, B = W.rmat_graph(scale=20, samples_per_node=8, seed=3, N=128)
        return A, B, 128, fmt, (f"R-MAT 2^20 (a=0.57,b=0.19,c=0.19), avg degree 16, N=128, {fmt} with per-column "
                                f"scaling"), None
    if name == "gcn":
        A, X, dY = W.gcn_graph(scale=18, samples_per_node=16, seed=4, N=256)
        A = W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.vals.astype(np.float32))
        return A, X, 256, "f32", "GCN layer: R-MAT 2^18 + I, D^-1/2 (A+I) D^-1/2, N=256, f32", dY
    if name == "uniform":
        A, B = W.uniform_rows(2000, 10, 32, seed=1)
        return A, B, 32, "f32", "uniform 2,000 x 2,000, 10 nnz/row, N=32, f32", None
    fmt = fmt or "f32"
    A, B = W.block_mix(n=1 << 20, N=64)
    return A, B, 64, fmt, (f"block mix 2^20: half the 16-row blocks two dense 16x16 blocks, the rest 16 uniform "
                           f"columns per row, N=64, {fmt}"), None


def run_single(name, args, torch, lp, flush, hbm_peak, hbm_src, steps, warmup, fmt=None, full=False):
    """One single-matrix workload: autotuned plan timed (L2 flushed per step), its dominant part's
    roofline, CSR-only and hybrid variants, rel-L2 against the oracle (and, for 16-bit formats,
    against the unrounded FP64 problem); the GCN layer adds its backward pass."""
    import oracle

    A, B, N, fmt, desc, dY = single_inputs(name, fmt, args.N)
    e = {"f64": 8, "f32": 4}.get(fmt, 2)
    c = 8 if fmt == "f64" else 4
    flops = 2.0 * A.nnz * N
    alg = csr_alg_bytes(A.n_rows, A.n_cols, A.nnz, N, e, c)
    A_r = rounded_matrix(A, fmt)
    sc = None
    if fmt in ("f16", "bf16"):
        Bq, s = oracle.scale_round_columns(B, fmt)
        B_eff = Bq * s[None, :]
        Bd = torch.as_tensor(Bq).to(torch.float16 if fmt == "f16" else torch.bfloat16).cuda()
        sc = torch.as_tensor(s, dtype=torch.float32).cuda()
    else:
        B_eff = B if fmt == "f64" else B.astype(np.float32).astype(np.float64)
        Bd = torch.as_tensor(B_eff).to(torch.float64 if fmt == "f64" else torch.float32).cuda()
    Cd = torch.empty((A.n_rows, N), dtype=torch.float64 if fmt == "f64" else torch.float32, device="cuda")
    plan = lp.Plan(A, N, fmt, tau=-1.0, want_backward=(name == "gcn"))
    inf = plan.info()
    torch.cuda.nvtx.range_push(f"workload:{name}")
    step, csr, bcsr = time_steps(torch, lambda: plan.spmm(Bd, Cd, col_scale=sc), steps, warmup, flush, plan=plan)
    torch.cuda.nvtx.range_pop()
    ms = statistics.mean(step)
    csr_ms, bcsr_ms = statistics.mean(csr), statistics.mean(bcsr)
    # dominant part: its algorithmic bytes (its rows, entries, B once, its C rows) over its time
    if csr_ms >= bcsr_ms:
        part, p_ms, rows, pnnz = "csr", csr_ms, inf["n_csr_rows"], inf["nnz_csr"]
    else:
        part, p_ms, rows, pnnz = "bcsr", bcsr_ms, inf["n_row_blocks"] * inf["block_rows"], inf["nnz_bcsr"]
    p_bytes = rows * 8 + pnnz * (4 + e) + A.n_cols * N * e + rows * N * c
    if fmt == "f64":
        ach = 2.0 * pnnz * N / (p_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": f"{part} part", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "peak_source": FP64_PEAK_SOURCE,
                "hbm_frac": p_bytes / (p_ms * 1e-3) / 1e9 / hbm_peak}
        key = "csr_spmm_f64_n64" if (part == "csr" and N == 64) else None
    else:
        ach = p_bytes / (p_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": f"{part} part", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "peak_source": hbm_src}
        key = f"{part}_{name}_{fmt}"
    roof.update(traffic=traffic_for(key) if key else None, kernel_ms=p_ms, alg_bytes_per_launch=p_bytes)
    C = plan.spmm(Bd, Cd, col_scale=sc).double().cpu().numpy()
    ref = oracle.spmm_threads(A_r, B_eff, host_cores())
    out = {"workload": desc, "dtype": fmt, "nnz": int(A.nnz), "N": N, "value": flops / (ms * 1e-3) / 1e9,
           "unit": "GFLOP/s", "ms_per_step": ms, "steps": steps, "roofline": roof,
           "hbm": {"alg_bytes_per_step": alg, "frac_of_measured": alg / (ms * 1e-3) / 1e9 / hbm_peak},
           "tau_autotuned": inf["tau"], "tile_min": inf["tile_min"],
           "shapes_autotuned": {"block_rows": inf["block_rows"], "csr_lane_vectors": inf["csr_lane_vectors"],
                                "bcsr_col_tile": inf["bcsr_col_tile"]},
           "part_ms": {"csr": csr_ms, "bcsr": bcsr_ms},
           "rel_l2_vs_oracle": rel_l2(C, ref), "rel_l2_tol": TOL[fmt],
           "gpu_launches_per_step": launches_per_step(inf)}
    if fmt in ("f16", "bf16"):
        out["rel_l2_vs_unrounded_fp64"] = rel_l2(C, oracle.spmm_threads(A, B, host_cores()))
    if full or name in ("laplacian", "mixed"):
        var = {}
        for vname, tau in (("csr_only", math.inf), ("hybrid_tau2", 2.0)):
            vp = lp.Plan(A, N, fmt, tau=tau)
            s_v, _, _ = time_steps(torch, lambda: vp.spmm(Bd, Cd, col_scale=sc), max(5, steps // 2), 2, flush)
            var[vname] = {"gflops": flops / (statistics.mean(s_v) * 1e-3) / 1e9, "ms_per_step": statistics.mean(s_v),
                          "bcsr_row_blocks": vp.info()["n_row_blocks"]}
            vp.destroy()
        # the performance model (Eq. 2 fitted to warm-up times, Eq. 3) beside the timed autotuner
        mp = lp.Plan(A, N, fmt, tau=lp.TAU_MODEL)
        mi = mp.info()
        s_m, _, _ = time_steps(torch, lambda: mp.spmm(Bd, Cd, col_scale=sc), max(5, steps // 2), 2, flush)
        var["model"] = {"tau": mi["tau"], "predicted_gflops": mi["model_gflops"],
                        "gflops": flops / (statistics.mean(s_m) * 1e-3) / 1e9, "ms_per_step": statistics.mean(s_m),
                        "bcsr_row_blocks": mi["n_row_blocks"], "coef": mi["model_coef"]}
        mp.destroy()
        out["variants"] = var
    if name == "gcn":
        dYd = torch.as_tensor(dY, dtype=torch.float32).cuda()
        dYq = dY.astype(np.float32).astype(np.float64)
        dB = torch.empty((A.n_cols, N), dtype=torch.float32, device="cuda")
        st_b, _, _ = time_steps(torch, lambda: plan.backward(dYd, Bd), steps, warmup, flush)
        bms = statistics.mean(st_b)
        dX, dv = plan.backward(dYd, Bd)
        torch.cuda.synchronize()
        bw_bytes = 2 * alg - (A.n_rows + 1) * 8       # A^T dY pass and the SDDMM pass over A's pattern
        out["backward"] = {"ms_per_step": bms, "gflops": 2 * flops / (bms * 1e-3) / 1e9,
                           "hbm_frac": bw_bytes / (bms * 1e-3) / 1e9 / hbm_peak,
                           "what": "dX = A^T dY (transposed hybrid plan) + dvals = SDDMM(dY, X^T)",
                           "rel_l2_dX_vs_oracle": rel_l2(dX.double().cpu().numpy(), oracle.spmm_t(A_r, dYq)),
                           "rel_l2_dvals_vs_oracle": rel_l2(dv.double().cpu().numpy(),
                                                            oracle.sddmm(A_r, dYq, B_eff)),
                           "rel_l2_tol": TOL[fmt]}
        del dB
    plan.destroy()
    return out


# ------------------------------------------------------------------ reference arm (the oracle)
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    threads = host_cores()
    if args.workload == "batched":
        mats, Bh = batch_inputs(args.batch_count, args.dtype or "f32", args.batch_kinds)
        idx = list(range(0, len(mats), 8))
        sub = [mats[i][0] for i in idx]
        Bs = [Bh[i].astype(np.float64) for i in idx]
        flops = sum(2.0 * mats[i][0].nnz * mats[i][1] for i in idx)
        run = lambda: oracle_batch(sub, Bs, threads)  # noqa: E731
        config = batch_config(args.batch_count, args.dtype or "f32", sum(A.nnz for A, _ in mats))
        sample = (f"every 8th matrix of the batch ({len(idx)} matrices, {flops / 1e9:.2f} GFLOP) per step; FP64 C "
                  f"oracle, one matrix per host thread")
        dtype = args.dtype or "f32"
    else:
        A, B, N, fmt, desc, _ = single_inputs(args.workload, args.dtype, args.N)
        flops = 2.0 * A.nnz * N
        run = lambda: oracle.spmm_threads(A, B, threads)  # noqa: E731
        config = {"workload": desc, "nnz": int(A.nnz), "N": N}
        sample = f"full workload per step (FP64 C oracle, rows split over {threads} host threads)"
        dtype = fmt
    for _ in range(args.warmup):
        run()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        run()
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    v = flops / t / 1e9
    line = {"metric": METRIC, "value": v, "unit": "GFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic (seeded)", "config": config,
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ main
def run_loops(args):
    import torch

    import paper_2511_08158_gb300 as lp

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        lp.build()
    if world > 1:
        torch.distributed.barrier(device_ids=[local])
    lp.load()
    import oracle
    if rank == 0:
        oracle.build()
    if world > 1:
        torch.distributed.barrier(device_ids=[local])
    flush = make_flush(torch)
    hbm_peak, hbm_src = peaks()
    if args.workload == "batched":
        line = run_batched(args, torch, lp, flush, rank, world, hbm_peak, hbm_src)
        if not args.no_sub and rank == 0 and world == 1:
            subs = {}
            k = max(5, min(args.steps, 10))
            for name, fmt in (("laplacian", None), ("rmat", "f16"), ("rmat", "bf16"), ("gcn", None),
                              ("uniform", None), ("mixed", "bf16")):
                key = name if fmt is None else f"{name}_{fmt}"
                subs[key] = run_single(name, args, torch, lp, flush, hbm_peak, hbm_src, k, 3, fmt=fmt,
                                       full=(name in ("laplacian", "mixed")))
                torch.cuda.empty_cache()
            line["workloads"] = subs
    else:
        out = run_single(args.workload, args, torch, lp, flush, hbm_peak, hbm_src, args.steps, args.warmup,
                         fmt=args.dtype, full=True)
        line = {"metric": METRIC, "value": out["value"], "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": out["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": out["dtype"], "data": "synthetic (seeded)",
                "config": {"workload": out["workload"], "nnz": out["nnz"], "N": out["N"],
                           "l2": "flushed before every timed step"},
                "roofline": out["roofline"], "detail": out,
                "gpu_launches": out["gpu_launches_per_step"] * args.steps}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_loops(args)


if __name__ == "__main__":
    main()
