#!/usr/bin/env python3
"""Benchmark of the GB300 sparsity-aware 1D SpGEMM; prints one JSON line.

Workload (the paper's squaring use case, Section 4.1, on a synthetic stand-in
for its SuiteSparse graphs): R-MAT scale 18 (262,144 vertices), edge factor 16,
(a, b, c, d) = (0.57, 0.19, 0.19, 0.05), self-loops dropped, duplicates merged,
symmetrised; C = A * A with P = 16 column blocks and fetch blocks of b = 1024
column ids.  One step runs it twice: double values 1.0 and the int64 (+, x)
path-count semiring.  GFLOP = 2 x products.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Timing: inputs resident in HBM; each timed step is bracketed by CUDA events on
the library's stream and preceded (outside the timed region) by a 256 MiB write
that evicts L2.  Under torchrun every rank runs the whole workload on its own
GPU (weak scaling), the step times are maxed over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "C=A·B GFLOP/s & % HBM roofline; learned/batched vs plain GPU time, exact C"
RMAT_SCALE = 18                # the headline workload: R-MAT scale 18, edge factor 16
P_BLOCKS, FETCH_B = 16, 1024
CPU_SAMPLE_COLS = 65536      # columns of C computed by the oracle for the CPU baseline
REF_SAMPLE_COLS = 16384      # per step of the reference arm
FLUSH_BYTES = 256 << 20      # > 2 x the 126 MiB L2
BYTES_PER_NZ = 12            # int32 row id + 8-byte value
E2E_CHUNKS = 4               # groups of column blocks in the host-buffer call


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the learned-vs-exact and batched-vs-sequential comparisons of the headline line")
    ap.add_argument("--out-dir", default=os.path.join(tempfile.gettempdir(), "spgemm1d_bench"),
                    help="where the clock samples and the tuning cache are written")
    ap.add_argument("--workload", default="rmat18",
                    choices=["rmat18", "uniform8192", "galerkin128", "galerkin_right", "similarity", "batched",
                             "structure", "bc"],
                    help="rmat18 is the headline; the others measure the remaining configurations")
    ap.add_argument("--rmat-scale", type=int, default=RMAT_SCALE,
                    help="R-MAT scale of the rmat18 workload (smaller scales for profiler captures)")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def workload_name(scale: int) -> str:
    return f"rmat_s{scale}_ef16_symmetric_squaring"


def make_workload(scale: int):
    import synth
    A = synth.rmat_symmetric(scale, 16, seed=0)
    Ai = synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, A.vals.astype(np.int64))
    return A, Ai


def workload_config(scale, products_per_run, nnzC):
    return {"workload": workload_name(scale), "P": P_BLOCKS, "b": FETCH_B,
            "runs_per_step": ["f64 values 1.0", "int64 path counts"],
            "n": 1 << scale, "nnzA": None, "products_per_run": products_per_run, "nnzC_per_run": nnzC,
            "index_types": "int32 colptr / int32 row ids", "l2": "flushed before every timed step (256 MiB write)"}


# --------------------------------------------------------------- aggregation

def aggregate(local_ms: float, local_flop: float, world: int):
    """Max step time over ranks and the flops of all ranks (weak scaling)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        f = torch.tensor([local_flop], dtype=torch.float64, device=dev)
        dist.all_reduce(f, op=dist.ReduceOp.SUM)
        return float(t.item()), float(f.item())
    return local_ms, local_flop


# ------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, out_dir: str):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------ CPU baseline

def time_oracle(A, ncols_sample: int, seed: int, nthreads: int = 0):
    """The oracle on a random sample of output columns; nthreads = 0 uses
    every host core."""
    import oracle
    rng = np.random.default_rng(seed)
    cols = np.sort(rng.choice(A.ncols, ncols_sample, replace=False))
    t0 = time.perf_counter()
    r = oracle.spgemm(A, A, cols=cols, nthreads=nthreads)
    dt = time.perf_counter() - t0
    products = int(r["flops"].sum())
    return {"value": 2.0 * products / dt / 1e9, "unit": "GFLOP/s", "cores": nthreads or oracle.max_threads(),
            "kind": "oracle",
            "sample": f"{ncols_sample} random output columns (seed {seed}) of the f64 run: {products} products, "
                      f"{dt:.2f} s", "seconds": dt, "products": products}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    A, _ = make_workload(args.rmat_scale)
    for w in range(args.warmup):
        time_oracle(A, REF_SAMPLE_COLS, seed=100 + w)
    secs, prods = [], []
    for s in range(args.steps):
        r = time_oracle(A, REF_SAMPLE_COLS, seed=s)
        secs.append(r["seconds"])
        prods.append(r["products"])
    import oracle
    val = 2.0 * sum(prods) / sum(secs) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.rmat_scale, None, None),
            "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"each step: {REF_SAMPLE_COLS} random output columns of the f64 run"},
            "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- roofline

PROFILE_SCALE = 18     # the ncu capture of the dominant kernel is taken on this R-MAT scale


def kernel_source_digest():
    """Digest of the sources of the heavy numeric kernel (its own file and the
    headers it includes): a traffic figure taken from an older build is not
    reported."""
    h = hashlib.sha256()
    for name in ("numeric.cu", "spg_internal.cuh", "cta_products.cuh", "block_ops.cuh"):
        with open(os.path.join(ROOT, "paper_2408_14558_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, alg_bytes_per_launch: float):
    """DRAM bytes per launch of `kernel`, from the committed ncu summary of a
    capture at the bench's scale (one kernel, two launches, metrics of one
    ncu pass): its mean read + write bytes, times the ratio of this run's
    algorithmic bytes to the captured launch's (1 for the same workload).
    None when there is no summary or the kernel's sources changed since it
    was taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_rmat_s{PROFILE_SCALE}.md")
    if not os.path.exists(path):
        return None, None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    a = re.search(r"algorithmic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    d = re.search(r"source_digest:\s*([0-9a-f]+)", txt)
    if not m or not a or not d or d.group(1) != kernel_source_digest():
        return None, None
    t, alg = float(m.group(1)), float(a.group(1))
    return t * alg_bytes_per_launch / alg, {"captured_scale": PROFILE_SCALE, "captured_traffic_per_launch": t,
                                           "captured_algorithmic_bytes_per_launch": alg,
                                           "summary": os.path.relpath(path, ROOT)}


def kernel_bytes(group: str, st: dict) -> float:
    """Algorithmic bytes of one launch group of one run:
    numeric heavy: write its C entries, read its B entries and A~ once;
    numeric light: the same for the light columns; symbolic: read B rows and
    A~ rows once, write one count per column; gather: read and write A~."""
    nzc_h = max(st["nnzC_heavy"], 0)
    if group == "num_heavy":
        return (BYTES_PER_NZ * (nzc_h + st["nnzB_heavy"] + st["gathered_nnz_exact"]) + 8 * st["heavy_columns"])
    if group == "num_light":
        return (BYTES_PER_NZ * (st["nnzC"] - nzc_h + st["nnzB"] - st["nnzB_heavy"] + st["gathered_nnz_exact"])
                + 8 * st["light_columns"])
    if group == "sym_heavy":
        return 4 * (st["nnzB_heavy"] + st["gathered_nnz_exact"]) + 8 * st["heavy_columns"]
    if group == "sym_light":
        return 4 * (st["nnzB"] - st["nnzB_heavy"] + st["gathered_nnz_exact"]) + 8 * st["light_columns"]
    if group == "gather":
        return 2 * BYTES_PER_NZ * st["gathered_nnz_exact"]
    return 0.0


def compulsory_bytes(st: dict) -> float:
    """B (colptr + rows + values) + gathered A once + C (rows + values + int64 colptr)."""
    return (4 * (st["n"] + 1) + BYTES_PER_NZ * st["nnzB"] + BYTES_PER_NZ * st["gathered_nnz_exact"]
            + 8 * st["sum_dtilde"] + BYTES_PER_NZ * st["nnzC"] + 8 * (st["n"] + 1))


def measured_peak_hbm():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# --------------------------------------------------------------------- main

def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "rmat18":
        import bench_workloads
        return bench_workloads.run(args)
    import torch
    import torch.distributed as dist

    import paper_2408_14558_gb300 as g
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    g.load_library()
    A, Ai = make_workload(args.rmat_scale)
    dA = g.to_device(A, ptr_dtype=torch.int32, idx_dtype=torch.int32)
    dAi = g.to_device(Ai, ptr_dtype=torch.int32, idx_dtype=torch.int32)
    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def step():
        sts = []
        for X in (dA, dAi):
            plan = g.spgemm_plan(X, X, P_BLOCKS, FETCH_B)
            colptr, nnz = g.spgemm_symbolic(plan)
            C = g.spgemm_numeric(plan, colptr)
            sts.append(g.spgemm_plan_stats(plan))
            g.spgemm_plan_destroy(plan)
            del C, colptr
        return sts

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local, args.out_dir)
    clocks.start()
    times, stats = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for s in range(args.steps):
        flush.fill_(s)
        e0.record(stream)
        sts = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        stats.append(sts)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()

    products_step = sum(st["products"] for st in stats[0])
    flop_local = 2.0 * products_step * args.steps
    total_ms, flop_all = aggregate(sum(times), flop_local, world)
    value = flop_all / (total_ms / 1e3) / 1e9
    ms_per_step = total_ms / args.steps

    # dominant kernel group and its roofline
    groups = ["gather", "sym_light", "sym_heavy", "num_light", "num_heavy"]
    per_group = {gname: statistics.mean(sum(st["ms_" + gname] for st in sts) for sts in stats) for gname in groups}
    dom = max(per_group, key=per_group.get)
    dom_bytes = sum(kernel_bytes(dom, st) for st in stats[0])        # both runs of one step
    dom_ms = per_group[dom]
    peak, peak_src = measured_peak_hbm()
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else 0.0
    kernel_name = {"num_heavy": "k_num_heavy", "num_light": "k_num_light", "sym_heavy": "k_sym_heavy",
                   "sym_light": "k_sym_light", "gather": "k_gather_copy"}[dom]
    traffic, traffic_basis = (profiled_traffic(kernel_name, dom_bytes / 2)
                              if kernel_name == "k_num_heavy" and args.rmat_scale == PROFILE_SCALE else (None, None))
    comp = sum(compulsory_bytes(st) for st in stats[0])
    path_gbs = comp / (ms_per_step / 1e3) / 1e9
    launches = sum(st["kernel_launches"] for sts in stats for st in sts)
    # compute-side roofline of the f64 run's numeric phase: every product is one
    # DMUL and, inside the shared-memory atomic add of a double, one DADD on the
    # FP64 pipe, which retires 2 lane-operations per clock per SM
    f64_num_ms = statistics.mean(sts[0]["ms_numeric"] for sts in stats)
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    fp64_peak = 2.0 * n_sm * sm_mhz * 1e6 / 1e9                       # G lane-ops/s
    fp64_achieved = 2.0 * stats[0][0]["products"] / (f64_num_ms / 1e3) / 1e9 if f64_num_ms > 0 else 0.0

    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+int64", "data": "synthetic",
            "config": workload_config(args.rmat_scale, stats[0][0]["products"], stats[0][0]["nnzC"]),
            "roofline": {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_basis": traffic_basis,
                         "algorithmic_bytes_per_launch": dom_bytes / 2,
                         "algorithmic_bytes_per_step": dom_bytes, "ms_per_step": dom_ms,
                         "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src},
            "path_roofline": {"compulsory_bytes_per_step": comp, "achieved": path_gbs, "frac": path_gbs / peak,
                              "unit": "GB/s"},
            "compute_roofline": {"bound": "fp64 pipe", "scope": "numeric phase of the f64 run",
                                 "achieved": fp64_achieved, "peak": fp64_peak, "unit": "G lane-ops/s",
                                 "frac": fp64_achieved / fp64_peak if fp64_peak else 0.0,
                                 "peak_source": f"2 FP64 lane-ops per clock per SM x {n_sm} SMs x {sm_mhz:.0f} MHz"},
            "kernel_ms_per_step": {k: round(v, 4) for k, v in per_group.items()},
            "kernel_ms_per_run": {label: {gname: round(statistics.mean(sts[ri]["ms_" + gname] for sts in stats), 4)
                                          for gname in groups + ["plan", "symbolic", "numeric"]}
                                  for ri, label in enumerate(("f64", "int64"))},
            "phase_ms_per_step": {ph: statistics.mean(sum(st["ms_" + ph] for st in sts) for sts in stats)
                                  for ph in ("plan", "symbolic", "numeric")},
            "gpu_launches": launches, "clocks": clk}
    line["config"]["nnzA"] = A.nnz

    # the host-buffer call right after the headline, before the CPU baseline and the
    # comparisons, whose much larger host arrays churn the host's memory
    if not args.no_e2e:
        try:
            line["e2e"] = run_e2e(g, torch, A, Ai, max(3, min(args.steps, 8)), world, products_step,
                                  max(st["nnzC"] for sts in stats for st in sts))
        except RuntimeError as ex:   # e.g. no room for C's pinned host pool on this machine (SpgError too)
            line["e2e"] = {"value": None, "unit": "GFLOP/s", "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                           "error": str(ex).splitlines()[0][:300]}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = time_oracle(A, CPU_SAMPLE_COLS, seed=0)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        one = time_oracle(A, CPU_SAMPLE_COLS // 16, seed=1, nthreads=1)
        line["cpu_baseline"]["single_thread"] = {k: one[k] for k in ("value", "unit", "cores", "sample")}

    if rank == 0 and world == 1 and not args.no_compare and args.rmat_scale == RMAT_SCALE:
        line.update(run_comparisons(args, torch, g))

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_comparisons(args, torch, g):
    """The two comparisons the metric names, each on its own workload and with
    its own clock record: learned nnz sizing against the exact two-pass
    multiply (C = A*A^T, 100,000 x 2^20 lognormal/Zipf rows, int64) and one
    persistent graph launch of 512 uneven products against 512 sequential
    multiplies.  Both check that the faster form gives the same C."""
    import argparse
    import bench_workloads as bw
    import synth
    sub = argparse.Namespace(steps=3, warmup=1, out_dir=args.out_dir, no_cpu_baseline=True)
    out = {}
    try:
        sim = bw.run_similarity(sub, torch, g, synth, emit=False)
        keys = ("exact_ms", "learned_ms", "learned_speedup", "exact_gflops", "learned_gflops", "recompute_rate",
                "recomputed_columns", "capacity_over_nnz", "learned_equals_exact", "clocks", "steps")
        out["learned_vs_exact"] = dict({k: sim.get(k) for k in keys}, workload=sim["config"]["workload"],
                                       products=sim["config"]["products"], nnzC=sim["config"]["nnzC"],
                                       timing="median of the timed steps, CUDA events, L2 flushed before each")
    except (RuntimeError, MemoryError) as ex:
        out["learned_vs_exact"] = {"error": str(ex).splitlines()[0][:300]}
    torch.cuda.empty_cache()
    try:
        bat = bw.run_batched(sub, torch, g, synth, emit=False)
        keys = ("ms_per_step", "sequential_ms", "speedup_vs_sequential", "value", "sequential_gflops",
                "rows_equal_sequential", "max_abs_value_diff_vs_sequential", "generation_s", "clocks", "steps")
        b = {k: bat.get(k) for k in keys}
        b["batched_ms"] = b.pop("ms_per_step")
        b["batched_gflops"] = b.pop("value")
        out["batched_vs_sequential"] = dict(b, workload=bat["config"]["workload"],
                                            products=bat["config"]["products"], tuned=bat["config"]["tuned"],
                                            timing="median of the timed steps, CUDA events, L2 flushed before each")
    except (RuntimeError, MemoryError) as ex:
        out["batched_vs_sequential"] = {"error": str(ex).splitlines()[0][:300]}
    torch.cuda.empty_cache()
    return out


def run_e2e(g, torch, A, Ai, steps, world, products_step, nnzc):
    """The same metric through the C ABI's host-buffer call: every step hands
    both runs' host matrices (pinned) to spgemm_1d_multiply_host, which copies
    them to the GPU, multiplies and puts all of C into pinned host memory
    before it returns (stored there by the numeric kernels where the GPU
    addresses the pool directly, else copied back one group of column blocks
    while the next computes).  C's host arrays come from one pinned pool sized for the larger
    product, allocated before the timed steps."""
    hosts = []
    for M in (A, Ai):
        hosts.append(g.HostCSC(M.nrows, M.ncols, torch.from_numpy(M.colptr.astype(np.int32)).pin_memory(),
                               torch.from_numpy(M.rowidx.astype(np.int32)).pin_memory(),
                               torch.from_numpy(M.vals).pin_memory(), None))
    h2d = sum(h.nbytes for h in hosts)           # B is A: each run copies its matrix once
    t0 = time.perf_counter()
    pool = g.HostPool(8 * (A.ncols + 1) + 12 * int(nnzc) + 4096)
    pin_s = time.perf_counter() - t0
    direct = g.spgemm_host_writable(pool.buf[: min(pool.buf.numel(), 1 << 20)])
    chunks = E2E_CHUNKS
    secs, d2h_total = [], 0
    for s in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2h = 0
        for h in hosts:
            C = g.spgemm_1d_multiply_host(h, h, P=P_BLOCKS, b=FETCH_B, chunks=chunks, pool=pool)
            d2h += C.nbytes
            del C
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if s > 0:                       # the first pass warms the allocator
            secs.append(dt)
            d2h_total = d2h
    local_s = statistics.mean(secs)
    t_all, flop_all = aggregate(local_s, 2.0 * products_step, world)
    return {"value": flop_all / t_all / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h_total, "steps": len(secs), "ms_per_step": 1e3 * t_all,
            "ms_per_step_min_max": [round(1e3 * min(secs), 1), round(1e3 * max(secs), 1)],
            "api": f"spgemm_1d_multiply_host (host buffers, {chunks} group(s) of column blocks)",
            "c_to_host": ("the numeric kernels store C into the pinned host pool directly" if direct else
                          "each group's C copied back by the copy engine behind the next group's numeric pass"),
            "timing": "wall clock, synchronize on both sides of each step; every byte of C is in pinned host "
                      f"memory when the call returns (pool of pinned memory allocated once, {pin_s:.1f} s)"}


if __name__ == "__main__":
    sys.exit(main())
