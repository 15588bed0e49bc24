"""Batched persistent execution and the autotuner on the GPU."""
import json

import numpy as np
import pytest
import torch

import oracle
import paper_2408_14558_gb300 as g
import synth
from parity import check_values

pytestmark = pytest.mark.gpu


def small_batch(count=24, seed=3, values="f64"):
    pairs = synth.batch_instances(count, 300, 6000, seed=seed, values=values)
    As = [g.to_device(A) for A, _ in pairs]
    Bs = [g.to_device(B) for _, B in pairs]
    return pairs, As, Bs


@pytest.mark.parametrize("values", ["f64", "i64"])
@pytest.mark.parametrize("task_cols,warps", [(64, 8), (16, 4), (1000, 8)])
def test_batch_matches_oracle_and_plain(values, task_cols, warps):
    pairs, As, Bs = small_batch(values=values)
    batch = g.spgemm_batch_create(As, Bs, task_cols=task_cols, warps_per_cta=warps)
    for rep in range(2):                      # the graph resets its queue and counters every launch
        g.spgemm_batch_execute(batch)
        assert g.spgemm_batch_status(batch) == g.SPG_OK
        for i in (0, 5, len(pairs) - 1) if rep == 0 else range(len(pairs)):
            A, B = pairs[i]
            cp, ri, v = g.spgemm_batch_result(batch, i)
            ref = oracle.spgemm(A, B)
            assert np.array_equal(cp.cpu().numpy(), ref["colptr"]), i
            assert np.array_equal(ri.cpu().numpy().astype(np.int64), ref["rowidx"]), i
            check_values(v.cpu().numpy(), ref["vals"], ref["absum"], f"instance {i}")
            if rep == 1 and i < 4:
                C = g.multiply(As[i], Bs[i], P=1, b=1024)
                assert torch.equal(C.colptr, cp) and torch.equal(C.rowidx, ri)


def test_batch_timeout_is_reported_and_context_survives():
    """A numeric task waiting on a flag that nothing sets gives up after the
    timeout; the batch reports SPG_TIMEOUT and the GPU context stays usable."""
    pairs, As, Bs = small_batch(count=6)
    bad = g.spgemm_batch_create(As, Bs, timeout_ns=20_000_000, stall_instance=2)
    g.spgemm_batch_execute(bad)
    with pytest.raises(g.SpgError) as e:
        g.spgemm_batch_status(bad)
    assert e.value.status == g.SPG_TIMEOUT
    g.spgemm_batch_destroy(bad)
    good = g.spgemm_batch_create(As, Bs)
    g.spgemm_batch_execute(good)
    assert g.spgemm_batch_status(good) == g.SPG_OK
    cp, ri, v = g.spgemm_batch_result(good, 2)
    ref = oracle.spgemm(*pairs[2])
    assert np.array_equal(cp.cpu().numpy(), ref["colptr"])


def _columns(M, c0, c1):
    cp = np.asarray(M.colptr, dtype=np.int64)
    s, e = int(cp[c0]), int(cp[c1])
    return synth.CSC(M.nrows, c1 - c0, cp[c0:c1 + 1] - s, np.asarray(M.rowidx[s:e]), np.asarray(M.vals[s:e]))


@pytest.mark.parametrize("values", ["f64", "i64"])
def test_batch_with_heavy_columns_matches_oracle(values):
    """Instances whose columns exceed the largest warp table (bound > 1024)
    run as CTA tasks of the same graph: R-MAT column blocks (hub columns among
    light ones), an instance whose every column is heavy, and light instances,
    all compared with the oracle, twice (the graph resets its queues)."""
    pairs = list(synth.batch_instances(6, 300, 6000, seed=4, values=values))
    R = synth.rmat_symmetric(12, 16, seed=5, values="ones" if values == "f64" else "i64")
    for c0, c1 in ((0, 700), (700, 2100), (2100, R.ncols)):
        pairs.append((R, _columns(R, c0, c1)))
    U = synth.uniform_columns(3000, 40, seed=1, values=values)   # 1600 products per column: all heavy
    pairs.append((U, U))
    As = [g.to_device(A) for A, _ in pairs]
    Bs = [g.to_device(B) for _, B in pairs]
    fl = [oracle.features(A, B)["flops"] for A, B in pairs]
    assert any((np.minimum(f, A.nrows) > 1024).any() and (np.minimum(f, A.nrows) <= 1024).any()
               for f, (A, _) in zip(fl, pairs))
    batch = g.spgemm_batch_create(As, Bs, task_cols=64, warps_per_cta=8)
    for rep in range(2):
        g.spgemm_batch_execute(batch)
        assert g.spgemm_batch_status(batch) == g.SPG_OK
        for i, (A, B) in enumerate(pairs):
            cp, ri, v = g.spgemm_batch_result(batch, i)
            ref = oracle.spgemm(A, B)
            assert np.array_equal(cp.cpu().numpy(), ref["colptr"]), (rep, i)
            assert np.array_equal(ri.cpu().numpy().astype(np.int64), ref["rowidx"]), (rep, i)
            check_values(v.cpu().numpy(), ref["vals"], ref["absum"], f"instance {i}")
    g.spgemm_batch_destroy(batch)


def test_batch_heavy_limits():
    """Heavy columns with int32 values (the CTA tasks read A's values in the
    accumulation type) are refused with SPG_UNSUPPORTED."""
    A = synth.uniform_columns(3000, 40, seed=1, values="i32")
    dA = g.to_device(A)
    with pytest.raises(g.SpgError) as e:
        g.spgemm_batch_create([dA], [dA])
    assert e.value.status == g.SPG_UNSUPPORTED


def test_autotuners_write_and_reuse_cache(tmp_path):
    pairs, As, Bs = small_batch(count=12)
    path = str(tmp_path / "tune.json")
    best = g.spgemm_batch_autotune(As, Bs, sample=8, cache_path=path)
    assert best["task_cols"] in (16, 64, 256) and best["warps_per_cta"] in (4, 8) and best["ms"] > 0
    again = g.spgemm_batch_autotune(As, Bs, sample=8, cache_path=path)
    assert (again["task_cols"], again["warps_per_cta"]) == (best["task_cols"], best["warps_per_cta"])
    A = synth.rmat_symmetric(11, 16, seed=2)
    dA = g.to_device(A)
    pb = g.spgemm_autotune(dA, dA, P=4, b=256, cache_path=path)
    assert pb["light_max"] in (256, 512, 1024) and pb["slab_rows"] in (2048, 4096, 8192)
    cache = json.load(open(path))
    assert any("|batch|" in k for k in cache) and any("|plain|" in k for k in cache)
    C = g.multiply(dA, dA, P=4, b=256, light_max=pb["light_max"], slab_rows=pb["slab_rows"])
    ref = oracle.spgemm(A, A)
    assert np.array_equal(C.colptr.cpu().numpy(), ref["colptr"])


@pytest.mark.slow
def test_batched_512_workload_against_oracle():
    """All 512 instances of the benchmark's batch (n log-uniform in
    [1000, 200000], ER or R-MAT rows, 4..32 per column, f64; seed 0), executed
    as one persistent batch with a task size the tuner can pick, every
    instance in full against the oracle: column pointers and row ids exact,
    doubles within 1e-12 * sum |a_rk * b_kj|."""
    pairs = synth.batch_instances(512, 1000, 200000, seed=0)
    As = [g.to_device(A, ptr_dtype=torch.int32, idx_dtype=torch.int32) for A, _ in pairs]
    Bs = [g.to_device(B, ptr_dtype=torch.int32, idx_dtype=torch.int32) for _, B in pairs]
    batch = g.spgemm_batch_create(As, Bs, task_cols=16, warps_per_cta=4)
    g.spgemm_batch_execute(batch)
    assert g.spgemm_batch_status(batch) == g.SPG_OK
    for i, (A, B) in enumerate(pairs):
        cp, ri, v = g.spgemm_batch_result(batch, i)
        ref = oracle.spgemm(A, B)
        assert np.array_equal(cp.cpu().numpy(), ref["colptr"]), i
        assert np.array_equal(ri.cpu().numpy().astype(np.int64), ref["rowidx"]), i
        check_values(v.cpu().numpy(), ref["vals"], ref["absum"], f"instance {i}")
