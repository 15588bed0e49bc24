"""The configurations other than the headline R-MAT squaring, measured through
the same C ABI (`python bench.py --workload NAME`); one JSON line each.

    uniform8192  C = A*A, 8192 x 8192, 8 uniform rows per column, f64, P=4, b=256
    galerkin128  A*P_agg then P_agg^T*(A*P_agg) on the 7-point 128^3 grid, P=32, b=2048
    similarity   C = A*A^T, A 100,000 x 2^20 lognormal rows / Zipf(1.2) columns, int32
                 values, int64 result: exact two-pass vs learned sizing (4 column chunks)
    batched      512 independent ER / R-MAT-row products (n log-uniform in
                 [1000, 200000], 4..32 per column, f64): one persistent graph
                 launch vs 512 sequential spgemm_1d_multiply calls
    galerkin_right  (R^T A) R by the column 1D path and the outer-product 1D path
    structure    CV/memA and block balance: ordering x column split
    bc           one 4096-source betweenness batch on the R-MAT scale-18 graph
Every timed region is bracketed by CUDA events on the library's stream, after
warm-up, with a 256 MiB write that evicts L2 before each timed step.  Each line
carries a ``roofline`` object for its dominant phase (the library's own event
times per phase, priced in algorithmic bytes: 12 B per nonzero read or written,
8 B per output column pointer) against the measured HBM copy bandwidth, and a
``cpu_baseline``: the oracle on the host cores on a bounded sample of the same
workload.
"""
from __future__ import annotations

import json
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
FLUSH_BYTES = 256 << 20
SIM_SAMPLE_COLS = 4096        # columns of A*A^T the oracle computes for the CPU baseline
BATCH_SAMPLE = 32             # instances of the batched workload the oracle computes
BC_SAMPLE_SOURCES = 2         # sources of the betweenness batch the oracle computes


# nvidia-smi clock records of the timed regions since the last line was emitted
_CLOCKS = []


def _merged_clocks():
    """One clock record for the timed regions of a line: the median of the
    regions' median SM clocks, the highest maximum, every throttle reason seen."""
    recs = [c for c in _CLOCKS if c]
    _CLOCKS.clear()
    if not recs:
        return None
    return {"sm_mhz": statistics.median(c["sm_mhz"] for c in recs), "sm_max_mhz": max(c["sm_max_mhz"] for c in recs),
            "samples": sum(c["samples"] for c in recs), "reasons": sorted({r for c in recs for r in c["reasons"]}),
            "regions": len(recs)}


def _emit(line):
    if "clocks" not in line:
        line["clocks"] = _merged_clocks()
    print(json.dumps(line), flush=True)


def _timer(torch, out_dir=None):
    import bench
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    out_dir = out_dir or os.path.join(os.environ.get("TMPDIR", "/tmp"), "spgemm1d_bench")

    def timed(fn, steps, warmup):
        # clocks are sampled every 200 ms from the start of the warm-up, which
        # is extended (never the timed steps) until the GPU has been busy with
        # this workload for at least 0.6 s, so that short regions get samples
        clk = bench.ClockSampler(torch.cuda.current_device(), out_dir)
        clk.start()
        t0 = time.perf_counter()
        w = 0
        while w < warmup or time.perf_counter() - t0 < 0.6:
            fn()
            torch.cuda.synchronize()
            w += 1
        out = []
        for s in range(steps):
            flush.fill_(s)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            e1.synchronize()
            out.append((e0.elapsed_time(e1), r))
        _CLOCKS.append(clk.stop())
        return out
    return timed


def _base(workload, metric, value, ms, steps, warmup, dtype, config, **extra):
    line = {"metric": metric, "value": value, "unit": "GFLOP/s", "n_gpus": 1, "steps": steps, "warmup": warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": dict(workload=workload, **config)}
    line.update(extra)
    return line


_PHASES = ("num_heavy", "num_light", "sym_heavy", "sym_light", "gather")


def _roofline(groups, kernel_names=None, note=None):
    """groups: {name: (algorithmic bytes, milliseconds)} summed over the
    multiplies of one step.  The dominant group (largest time) is reported:
    achieved = its bytes / its time, against the measured HBM copy bandwidth."""
    import bench
    peak, src = bench.measured_peak_hbm()
    name = max(groups, key=lambda k: groups[k][1])
    by, ms = groups[name]
    achieved = by / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    r = {"bound": "hbm", "kernel": (kernel_names or {}).get(name, name), "achieved": achieved, "peak": peak,
         "unit": "GB/s", "frac": achieved / peak, "traffic": None, "algorithmic_bytes_per_step": by,
         "ms_per_step": ms, "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src,
         "phase_ms": {k: v[1] for k, v in groups.items()}}
    if note:
        r["note"] = note
    return r


_KERNELS = {"num_heavy": "k_num_heavy", "num_light": "k_num_light", "sym_heavy": "k_sym_heavy",
            "sym_light": "k_sym_light", "gather": "k_gather_copy"}


def _column_groups(stats):
    """Per-phase (bytes, ms) of column-1D multiplies from their plan stats."""
    import bench
    out = {}
    for st in stats:
        for ph in _PHASES:
            by, ms = out.get(ph, (0.0, 0.0))
            out[ph] = (by + bench.kernel_bytes(ph, st), ms + st["ms_" + ph])
    return out


def _cpu_baseline(args, fn, sample, cores=None, min_seconds=3.0):
    """Time fn() (the oracle on a sample; it returns the sample's product
    count), repeated until min_seconds have passed; value = 2 * products /
    seconds in GFLOP/s."""
    if getattr(args, "no_cpu_baseline", False):
        return None
    import oracle
    products, reps = 0, 0
    t0 = time.perf_counter()
    while True:
        products += int(fn())
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= min_seconds:
            break
    rep = f" x {reps} repetitions" if reps > 1 else ""
    return {"value": 2.0 * products / dt / 1e9, "unit": "GFLOP/s",
            "cores": oracle.max_threads() if cores is None else cores, "kind": "oracle",
            "sample": f"{sample}{rep}: {products} products, {dt:.2f} s", "seconds": dt}


def _csc(synth, r):
    """A synth.CSC from an oracle result dict."""
    return synth.CSC(int(r["nrows"]), int(r["ncols"]), r["colptr"], r["rowidx"], r["vals"])


def _graph_replay_ms(torch, g, dA, dB, P, b, reps=200):
    """Average time of one captured refresh + numeric graph (same patterns,
    values re-read), after warm-up; the data stay in L2 between replays."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = g.spgemm_plan(dA, dB, P, b)
        g.spgemm_symbolic(plan)
        C = g.spgemm_numeric(plan)
        g.spgemm_plan_capture(plan, C)
        for _ in range(10):
            g.spgemm_plan_replay(plan)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            g.spgemm_plan_replay(plan)
        e1.record(s)
        e1.synchronize()
        g.spgemm_plan_destroy(plan)
    return e0.elapsed_time(e1) / reps


def _one_launch(torch, g, dA, dB, P, b, reps=50):
    """The one-launch multiply (spgemm_small_multiply) captured in a CUDA graph:
    the median time of single replays, each after a 256 MiB write that evicts
    L2 (cold), and the mean of back-to-back replays (warm: the product fits in
    L2).  Returns (cold ms, warm ms, the SmallProduct)."""
    import bench
    sp = g.SmallProduct(dA, dB, P, b)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            sp.run(s)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            sp.run(s)
        flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
        clk = bench.ClockSampler(torch.cuda.current_device(), os.path.join(os.environ.get("TMPDIR", "/tmp"),
                                                                             "spgemm1d_bench"))
        clk.start()
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 0.6:       # warm-up long enough for clock samples
            graph.replay()
            torch.cuda.synchronize()
        cold = []
        for r in range(reps):
            flush.fill_(r)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            graph.replay()
            e1.record(s)
            e1.synchronize()
            cold.append(e0.elapsed_time(e1))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(200):
            graph.replay()
        e1.record(s)
        e1.synchronize()
        _CLOCKS.append(clk.stop())
    st = sp.stats()
    assert st["status"] == 0
    return statistics.median(cold), e0.elapsed_time(e1) / 200, sp, st


def run_uniform(args, torch, g, synth):
    A = synth.uniform_columns(8192, 8, seed=0)
    dA = g.to_device(A, ptr_dtype=torch.int32, idx_dtype=torch.int32)
    timed = _timer(torch)

    def step():
        plan = g.spgemm_plan(dA, dA, 4, 256)
        cp, _ = g.spgemm_symbolic(plan)
        C = g.spgemm_numeric(plan, cp)
        st = g.spgemm_plan_stats(plan)
        g.spgemm_plan_destroy(plan)
        return st
    res = timed(step, max(args.steps, 20), max(args.warmup, 5))
    ms = statistics.median(t for t, _ in res)
    st = res[0][1]
    cold_ms, warm_ms, sp, sst = _one_launch(torch, g, dA, dA, 4, 256)
    import bench
    import oracle
    comp = bench.compulsory_bytes(st)
    peak, src = bench.measured_peak_hbm()
    ach = comp / (cold_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": "k_small_multiply (one cooperative launch, graph replay)", "achieved": ach,
            "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
            "algorithmic_bytes_per_step": comp, "ms_per_step": cold_ms,
            "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src,
            "note": "bytes: B, the gathered A columns and C once; time: one graph replay after an L2 flush"}
    cpu = _cpu_baseline(args, lambda: oracle.spgemm(A, A)["flops"].sum(), "the whole product")
    _emit(_base("uniform8192_d8_P4_b256", "C=A·A GFLOP/s (one-launch multiply, CUDA graph replay)",
                2 * st["products"] / (cold_ms / 1e3) / 1e9, cold_ms, 50, 3, "f64",
                {"products": st["products"], "nnzC": st["nnzC"]},
                roofline=roof, cpu_baseline=cpu, gpu_launches=1,
                one_launch={"cold_ms": cold_ms, "warm_ms": warm_ms, "warm_gflops": 2 * st["products"] / (warm_ms / 1e3) / 1e9,
                            "nnzC": sst["nnzC"], "sum_dtilde": sst["sum_dtilde"],
                            "fetch_blocks_chosen": sst["fetch_blocks_chosen"]},
                multi_launch={"ms": ms, "gflops": 2 * st["products"] / (ms / 1e3) / 1e9, "steps": len(res),
                              "phase_ms": {k: st["ms_" + k] for k in ("plan", "symbolic", "numeric")},
                              "gpu_launches": st["kernel_launches"],
                              "roofline": _roofline(_column_groups([st]), _KERNELS)},
                graph_replay_refresh_ms=_graph_replay_ms(torch, g, dA, dA, 4, 256),
                l2="value: median of 50 single graph replays, each after a 256 MiB write that evicts L2; "
                   "warm_ms: mean of 200 back-to-back replays (the whole product fits in L2)",
                note="value = spgemm_small_multiply (plan, symbolic and numeric in one cooperative kernel, two "
                     "clears, no host read-back) replayed from a CUDA graph; multi_launch = the plan / symbolic / "
                     "numeric calls of the column 1D path (host read-backs of sizes between phases)"))


def run_galerkin(args, torch, g, synth):
    N = 128
    A, Pg, PT = synth.poisson3d(N), synth.aggregation_2x2x2(N), synth.aggregation_2x2x2_transpose(N)
    dA, dP, dPT = (g.to_device(M, ptr_dtype=torch.int32, idx_dtype=torch.int32) for M in (A, Pg, PT))
    timed = _timer(torch)

    def step():
        plan = g.spgemm_plan(dA, dP, 32, 2048)
        cp, _ = g.spgemm_symbolic(plan)
        AP = g.spgemm_numeric(plan, cp)
        s1 = g.spgemm_plan_stats(plan)
        g.spgemm_plan_destroy(plan)
        plan = g.spgemm_plan(dPT, AP, 32, 2048)
        cp, _ = g.spgemm_symbolic(plan)
        G = g.spgemm_numeric(plan, cp)
        s2 = g.spgemm_plan_stats(plan)
        g.spgemm_plan_destroy(plan)
        return s1, s2
    res = timed(step, max(args.steps, 5), max(args.warmup, 3))
    ms = statistics.median(t for t, _ in res)
    s1, s2 = res[0][1]
    prods = s1["products"] + s2["products"]
    import oracle

    def cpu_run():
        r1 = oracle.spgemm(A, Pg)
        r2 = oracle.spgemm(PT, _csc(synth, r1))
        return r1["flops"].sum() + r2["flops"].sum()
    cpu = _cpu_baseline(args, cpu_run, "both products in full")
    _emit(_base("galerkin_7pt_128cube_P32_b2048", "P^T(A P) GFLOP/s", 2 * prods / (ms / 1e3) / 1e9, ms, len(res),
                max(args.warmup, 3), "f64",
                {"products": [s1["products"], s2["products"]], "nnzC": [s1["nnzC"], s2["nnzC"]]},
                roofline=_roofline(_column_groups([s1, s2]), _KERNELS), cpu_baseline=cpu,
                gpu_launches=s1["kernel_launches"] + s2["kernel_launches"],
                phase_ms=[{k: s["ms_" + k] for k in ("plan", "symbolic", "numeric")} for s in (s1, s2)],
                gathered_nnz=[s1["gathered_nnz_exact"], s2["gathered_nnz_exact"]],
                fetch_blocks=[[s["fetch_blocks_chosen"], s["fetch_blocks_total"]] for s in (s1, s2)],
                graph_replay_ms=_graph_replay_ms(torch, g, dA, dP, 32, 2048),
                note="graph_replay_ms = one captured value refresh + numeric pass of A*P_agg (same patterns)"))


def run_similarity(args, torch, g, synth, emit=True):
    from paper_2408_14558_gb300 import learned
    A, At = synth.lognormal_zipf_rows(seed=0)
    dA = g.to_device(A, ptr_dtype=torch.int64, idx_dtype=torch.int32)
    dAt = g.to_device(At, ptr_dtype=torch.int64, idx_dtype=torch.int32)
    chunks, P = 4, 16
    n = At.ncols
    bounds = [(i * n) // chunks for i in range(chunks + 1)]
    parts = []
    for c0, c1 in zip(bounds[:-1], bounds[1:]):
        cp = (dAt.colptr[c0:c1 + 1] - dAt.colptr[c0]).contiguous()
        s, e = int(dAt.colptr[c0]), int(dAt.colptr[c1])
        parts.append(g.DeviceCSC(At.nrows, c1 - c0, cp, dAt.rowidx[s:e], dAt.vals[s:e]))
    if os.path.exists(learned.DEFAULT_MODEL):
        model = g.spgemm_model_load(learned.DEFAULT_MODEL)
    else:
        model = None
    timed = _timer(torch)

    def run(sizing):
        stats = []
        for B in parts:
            kw = dict(sizing=g.SPG_SIZING_LEARNED, model=model) if sizing else {}
            C, status = g.spgemm_1d_multiply(dA, B, P=P // chunks, b=1024, **kw)
            stats.append(g.spgemm_last_multiply_stats())
            del C
        return stats
    ex = timed(lambda: run(False), max(args.steps, 2), max(args.warmup, 1))
    ms_exact = statistics.median(t for t, _ in ex)
    prods = sum(s["products"] for s in ex[0][1])
    nnzc = sum(s["nnzC"] for s in ex[0][1])
    extra = {"exact_ms": ms_exact, "exact_gflops": 2 * prods / (ms_exact / 1e3) / 1e9}
    if model is not None:
        le = timed(lambda: run(True), max(args.steps, 2), max(args.warmup, 1))
        ms_l = statistics.median(t for t, _ in le)
        st = le[0][1]
        rec = sum(s["recomputed_columns"] for s in st)
        cap = sum(s["learned_capacity"] for s in st)
        extra.update({"learned_ms": ms_l, "learned_gflops": 2 * prods / (ms_l / 1e3) / 1e9,
                      "learned_speedup": ms_exact / ms_l, "recomputed_columns": rec,
                      "recompute_rate": rec / n, "capacity_over_nnz": cap / nnzc})
        value, ms = extra["learned_gflops"], ms_l
        extra["roofline"] = _roofline(_column_groups(st), {**_KERNELS, "num_heavy": "k_fused_heavy"},
                                      note="learned sizing: the heavy phase is the fused pattern + value pass")
    else:
        extra["learned"] = "no model file: run python -m paper_2408_14558_gb300.learned"
        value, ms = extra["exact_gflops"], ms_exact
        extra["roofline"] = _roofline(_column_groups(ex[0][1]), _KERNELS)
    extra["roofline_exact"] = _roofline(_column_groups(ex[0][1]), _KERNELS)
    import oracle
    cols = np.sort(np.random.default_rng(0).choice(At.ncols, SIM_SAMPLE_COLS, replace=False))
    extra["cpu_baseline"] = _cpu_baseline(args, lambda: oracle.spgemm(A, At, cols=cols)["flops"].sum(),
                                          f"{SIM_SAMPLE_COLS} random columns of C (seed 0)")
    extra["gpu_launches"] = sum(s_["kernel_launches"] for s_ in (le[0][1] if model is not None else ex[0][1]))
    if model is not None:
        # outside the timed region: the learned C equals the exact C, chunk by chunk
        same = True
        for B in parts:
            Ce, _ = g.spgemm_1d_multiply(dA, B, P=P // chunks, b=1024)
            Cl, _ = g.spgemm_1d_multiply(dA, B, P=P // chunks, b=1024, sizing=g.SPG_SIZING_LEARNED, model=model)
            same = same and torch.equal(Ce.colptr, Cl.colptr) and torch.equal(Ce.rowidx, Cl.rowidx) and \
                torch.equal(Ce.vals, Cl.vals)
            del Ce, Cl
        extra["learned_equals_exact"] = bool(same)
    line = _base("similarity_AAt_100k_x_1M_lognormal_zipf", "C=A·Aᵀ GFLOP/s (learned sizing; exact alongside)",
                 value, ms, max(args.steps, 2), max(args.warmup, 1), "int64",
                 {"nnzA": A.nnz, "products": prods, "nnzC": nnzc, "column_chunks": chunks, "P": P, "b": 1024},
                 **extra)
    if not emit:
        line["clocks"] = _merged_clocks()
        return line
    _emit(line)


def run_batched(args, torch, g, synth, emit=True):
    t0 = time.time()
    pairs = synth.batch_instances(512, 1000, 200000, seed=0)
    gen_s = time.time() - t0
    As = [g.to_device(A, ptr_dtype=torch.int32, idx_dtype=torch.int32) for A, _ in pairs]
    Bs = [g.to_device(B, ptr_dtype=torch.int32, idx_dtype=torch.int32) for _, B in pairs]
    cache = os.path.join(args.out_dir, "tuning_cache.json")
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    tune = g.spgemm_batch_autotune(As, Bs, sample=64, cache_path=cache)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch = g.spgemm_batch_create(As, Bs, task_cols=tune["task_cols"], warps_per_cta=tune["warps_per_cta"])
    torch.cuda.synchronize()
    create_ms = 1e3 * (time.perf_counter() - t0)
    timed = _timer(torch)

    def run_batch():
        g.spgemm_batch_execute(batch)
    res = timed(run_batch, max(args.steps, 3), max(args.warmup, 2))
    assert g.spgemm_batch_status(batch) == g.SPG_OK
    ms_b = statistics.median(t for t, _ in res)

    def run_seq():
        prods, nbytes = 0, 0.0
        for A, B in zip(As, Bs):
            C, _ = g.spgemm_1d_multiply(A, B, P=1, b=1024)
            st = g.spgemm_last_multiply_stats()
            prods += st["products"]
            nbytes += bench.compulsory_bytes(st)
            del C
        return prods, nbytes
    import bench
    seq = timed(run_seq, 2, 1)
    ms_s = statistics.median(t for t, _ in seq)
    prods, nbytes = seq[0][1]
    info = g.spgemm_batch_info(batch)
    # outside the timed region: every instance of the batch against its own
    # sequential multiply (rows exactly; doubles to rounding, reported as the
    # largest absolute difference: the order of the additions differs)
    rows_same, worst = True, 0.0
    for i, (A, B) in enumerate(zip(As, Bs)):
        Cs, _ = g.spgemm_1d_multiply(A, B, P=1, b=1024)
        bcp, brow, bval = g.spgemm_batch_result(batch, i)
        rows_same = rows_same and torch.equal(Cs.colptr, bcp.to(Cs.colptr.dtype)) and \
            torch.equal(Cs.rowidx, brow.to(Cs.rowidx.dtype))
        if rows_same and Cs.vals.numel():
            worst = max(worst, float((Cs.vals - bval).abs().max()))
        del Cs, bcp, brow, bval
    import oracle
    pick = np.sort(np.random.default_rng(0).choice(len(pairs), BATCH_SAMPLE, replace=False))
    cpu = _cpu_baseline(args, lambda: sum(int(oracle.spgemm(*pairs[i])["flops"].sum()) for i in pick),
                        f"{BATCH_SAMPLE} random instances (seed 0)")
    roof = _roofline({"batch": (nbytes, ms_b)}, {"batch": "k_batch_persistent (3 table classes, one graph)"},
                     note="bytes: every instance's B, gathered A columns and C once; time: the whole graph launch")
    line = _base("batched_512_er_rmat_n1e3_2e5_d4_32", "batched C_j=A_j·B_j GFLOP/s (one persistent graph launch)",
                2 * prods / (ms_b / 1e3) / 1e9, ms_b, len(res), max(args.warmup, 2), "f64",
                {"instances": 512, "products": prods, "tuned": tune, "tasks": info["tasks"],
                 "grid": info["grid"], "pool_entries": info["pool_entries"]},
                roofline=roof, cpu_baseline=cpu,
                sequential_ms=ms_s, sequential_gflops=2 * prods / (ms_s / 1e3) / 1e9, speedup_vs_sequential=ms_s / ms_b,
                batch_create_ms=create_ms, generation_s=gen_s, rows_equal_sequential=bool(rows_same),
                max_abs_value_diff_vs_sequential=worst)
    if not emit:
        line["clocks"] = _merged_clocks()
        return line
    _emit(line)


def run_galerkin_right(args, torch, g, synth):
    """The right Galerkin multiplication (R^T A) R (7-point 128^3, 2x2x2
    aggregation R, P = 32, b = 2048) by the column 1D path (Algorithm 1) and
    by the outer-product 1D path (Algorithm 3), in the lexicographic ordering
    and after a random symmetric permutation of the fine grid (the same coarse
    operator), with the volumes each would move between 32 owners."""
    N, P, b = 128, 32, 2048
    A, R, RT = synth.poisson3d(N), synth.aggregation_2x2x2(N), synth.aggregation_2x2x2_transpose(N)
    timed = _timer(torch)
    out = {}
    for order in ("lexicographic", "permuted"):
        if order == "permuted":
            q = synth.random_permutation(A.ncols, seed=1)
            Ao, Ro, RTo = synth.relabel(A, q, q), synth.relabel(R, row_perm=q), synth.relabel(RT, col_perm=q)
        else:
            Ao, Ro, RTo = A, R, RT
        dA, dR, dRT = (g.to_device(M, ptr_dtype=torch.int32, idx_dtype=torch.int32) for M in (Ao, Ro, RTo))
        RtA, _ = g.spgemm_1d_multiply(dRT, dA, P, b)
        torch.cuda.synchronize()

        def col():
            C, _ = g.spgemm_1d_multiply(RtA, dR, P, b)
            return g.spgemm_last_multiply_stats(), int(C.colptr[-1])

        def outer():
            C, st = g.spgemm_outer_multiply(RtA, dR, P, b)
            return st, int(C.colptr[-1])
        rc = timed(col, max(args.steps, 5), max(args.warmup, 3))
        ro = timed(outer, max(args.steps, 5), max(args.warmup, 3))
        ms_c = statistics.median(t for t, _ in rc)
        ms_o = statistics.median(t for t, _ in ro)
        sc, nnz_c = rc[0][1]
        so, nnz_o = ro[0][1]
        assert nnz_c == nnz_o == 7 * (N // 2) ** 3 - 6 * (N // 2) ** 2
        out[order] = {"column_1d_ms": ms_c, "outer_1d_ms": ms_o, "products": sc["products"],
                      "column_1d_gflops": 2 * sc["products"] / (ms_c / 1e3) / 1e9,
                      "outer_1d_gflops": 2 * so["products"] / (ms_o / 1e3) / 1e9,
                      "column_1d_fetched_A_entries": sc["gathered_nnz_remote"],
                      "outer_1d_moved_B_entries": so["nnzB_moved"],
                      "outer_1d_moved_partial_entries": so["partial_moved"],
                      "outer_1d_partial_nnz": so["partial_nnz"],
                      "outer_1d_ms_split_local_merge": [so["ms_split"], so["ms_local"], so["ms_merge"]]}
        if order == "lexicographic":
            nnz_a, nnz_b, n = int(RtA.colptr[-1]), int(dR.colptr[-1]), dR.ncols
            roof_outer = _roofline(
                {"split": (2 * 12 * nnz_b, so["ms_split"]),
                 "local": (12 * (nnz_a + nnz_b + so["partial_nnz"]), so["ms_local"]),
                 "merge": (12 * (so["partial_nnz"] + so["nnzC"]) + 8 * (n + 1), so["ms_merge"])},
                {"split": "k_outer_count + k_outer_copy", "local": "column 1D kernels on A * B'",
                 "merge": "column 1D kernels on C' * S"},
                note="split: B read and written once; local: A, the row-split B and the partial columns once; "
                     "merge: partial columns read, C written")
            roof_col = _roofline(_column_groups([sc]), _KERNELS)
    import oracle
    RtA_h = _csc(synth, oracle.spgemm(RT, A))
    cpu = _cpu_baseline(args, lambda: oracle.spgemm(RtA_h, R)["flops"].sum(),
                        "(R^T A) R in full, lexicographic ordering")
    lex = out["lexicographic"]
    _emit(_base("galerkin_right_RtA_R_128cube_P32_b2048", "(R^T A) R GFLOP/s, column 1D vs outer-product 1D",
                lex["outer_1d_gflops"], lex["outer_1d_ms"], max(args.steps, 5), max(args.warmup, 3), "f64",
                {"nnzC": 7 * (N // 2) ** 3 - 6 * (N // 2) ** 2}, orderings=out,
                roofline=roof_outer, roofline_column_1d=roof_col, cpu_baseline=cpu,
                note="value = outer-product path, lexicographic ordering; moved/fetched entries are what a "
                     "32-owner distributed run would transfer"))


def run_structure(args, torch, g, synth):
    """The paper's "structure matters" finding on synthetic inputs: A*A for a
    banded 7-point operator (128^3) and an R-MAT graph (scale 18), each in its
    own ordering and after a random symmetric permutation, with uniform and
    flop-balanced column blocks (P = 16, b = 1024): CV/memA (mean fetched A
    volume over nnz(A)), block-granular fetch volume, the largest block's flops
    over the mean, and the multiply's time on this GPU."""
    P, b = 16, 1024
    timed = _timer(torch)
    rows, host, stats = [], {}, []
    for name, A in (("poisson3d_128", synth.poisson3d(128)), ("rmat_s18_ef16", synth.rmat_symmetric(18, 16, seed=0))):
        q = synth.random_permutation(A.ncols, seed=2)
        for order, M in (("original", A), ("permuted", synth.relabel(A, q, q))):
            host[(name, order)] = M
            dM = g.to_device(M, ptr_dtype=torch.int32, idx_dtype=torch.int32)
            for split_name, split in (("uniform", g.SPG_SPLIT_UNIFORM), ("flops", g.SPG_SPLIT_FLOPS)):
                def step():
                    plan = g.spgemm_plan(dM, dM, P, b, split=split)
                    cp, _ = g.spgemm_symbolic(plan)
                    C = g.spgemm_numeric(plan, cp)
                    blk = g.spgemm_plan_blocks(plan)
                    st = g.spgemm_plan_stats(plan)
                    g.spgemm_plan_destroy(plan)
                    return blk, st
                res = timed(step, max(args.steps, 3), max(args.warmup, 2))
                ms = statistics.median(t for t, _ in res)
                blk, st = res[0][1]
                fl = blk["flops"]
                rows.append({"matrix": name, "ordering": order, "split": split_name, "ms": ms,
                             "gflops": 2 * st["products"] / (ms / 1e3) / 1e9, "cv_mem_a": blk["cv_mem_a"],
                             "fetched_A_entries": int(blk["remote"].sum()),
                             "fetch_blocks_chosen": st["fetch_blocks_chosen"],
                             "gathered_block_volume": st["gathered_nnz_block"], "nnzA": int(M.rowidx.size),
                             "block_flops_max_over_mean": float(fl.max() / max(fl.mean(), 1))})
                stats.append(st)
    ib = max(range(len(rows)), key=lambda i: rows[i]["gflops"])
    best = rows[ib]["gflops"]
    import oracle
    M = host[(rows[ib]["matrix"], rows[ib]["ordering"])]
    cols = np.sort(np.random.default_rng(0).choice(M.ncols, min(M.ncols, 65536), replace=False))
    cpu = _cpu_baseline(args, lambda: oracle.spgemm(M, M, cols=cols)["flops"].sum(),
                        f"{cols.size} random columns (seed 0) of the fastest case's product")
    _emit(_base("structure_AxA_poisson128_rmat18_P16_b1024", "CV/memA and block balance, original vs permuted "
                "ordering, uniform vs flop split", best, rows[ib]["ms"], max(args.steps, 3),
                max(args.warmup, 2), "f64", {"P": P, "b": b}, cases=rows,
                roofline=dict(_roofline(_column_groups([stats[ib]]), _KERNELS),
                              case=f"{rows[ib]['matrix']} {rows[ib]['ordering']} {rows[ib]['split']}"),
                cpu_baseline=cpu,
                note="value = best GFLOP/s of the cases; cv_mem_a is what a 16-owner distributed run would fetch "
                     "per owner over nnz(A)"))


def run_bc(args, torch, g, synth):
    """One batch of the batched betweenness centrality (Section 3.2) on the
    R-MAT scale-18 graph: 4096 random sources (the paper's batch size),
    forward search and backward sweep, P = 16, b = 1024."""
    A = synth.rmat_symmetric(18, 16, seed=0)
    dA = g.to_device(A, ptr_dtype=torch.int32, idx_dtype=torch.int32)
    src = torch.from_numpy(np.random.default_rng(0).choice(A.ncols, 4096, replace=False).astype(np.int32))
    timed = _timer(torch)
    res = timed(lambda: g.spgemm_bc_batch(dA, src, P=16, b=1024, validate=False), max(args.steps, 2),
                max(args.warmup, 1))
    ms = statistics.median(t for t, _ in res)
    _, levels, st = res[0][1]
    prods = st["products_forward"] + st["products_backward"]
    # algorithmic bytes: every level's product reads A once, its input frontier
    # (or dependency weights) and writes the masked next frontier (or the
    # previous level's dependencies); 12 B per nonzero
    lv = list(levels) + [0]
    fwd = sum(12 * (A.nnz + lv[l] + lv[l + 1]) for l in range(len(levels)))
    bwd = sum(12 * (A.nnz + lv[l] + lv[l - 1]) for l in range(1, len(levels)))
    roof = _roofline({"forward": (fwd, st["ms_forward"]), "backward": (bwd, st["ms_backward"])},
                     {"forward": "forward search SpGEMMs (column 1D path + frontier mask)",
                      "backward": "backward sweep SpGEMMs (column 1D path + dependency update)"})
    from oracle import bc as obc
    srcs = src.numpy()[:BC_SAMPLE_SOURCES]
    per_source = prods / 4096.0
    cpu = _cpu_baseline(args, lambda: (obc.brandes(A, srcs), per_source * len(srcs))[1],
                        f"{len(srcs)} of the sources, Brandes in plain Python; products = the batch's SpGEMM "
                        f"products per source x sources", cores=1)
    _emit(_base("bc_rmat_s18_ef16_batch4096_P16_b1024", "betweenness batch GFLOP/s (forward search + backward "
                "sweep SpGEMMs)", 2 * prods / (ms / 1e3) / 1e9, ms, max(args.steps, 2), max(args.warmup, 1), "f64",
                {"sources": 4096, "levels": st["levels"], "frontier_nnz": st["frontier_nnz"],
                 "products_forward": st["products_forward"], "products_backward": st["products_backward"]},
                level_nnz=levels, ms_forward=st["ms_forward"], ms_backward=st["ms_backward"],
                spgemm_phase_ms={k: st["ms_" + k] for k in ("plan", "gather", "sym_light", "sym_heavy", "num_light",
                                                            "num_heavy")},
                multiplies=st["multiplies"], spgemm_output_nnz=st["nnzC_total"],
                roofline=roof, cpu_baseline=cpu))


def run(args):
    import torch
    sys.path.insert(0, ROOT)
    import paper_2408_14558_gb300 as g
    import synth
    g.load_library()
    fn = {"uniform8192": run_uniform, "galerkin128": run_galerkin, "galerkin_right": run_galerkin_right,
          "similarity": run_similarity, "batched": run_batched, "structure": run_structure,
          "bc": run_bc}[args.workload]
    fn(args, torch, g, synth)
    return 0
