"""The one-launch multiply (spgemm_small_multiply: Algorithm 1 on one GPU in a
single cooperative kernel) against the oracle: C element by element, the
planning volumes of Algorithms 1-2 against oracle.plan_block, its failure
reports (capacity, a column too heavy for the warp table), and replays of a
captured CUDA graph, including new values written between replays."""
import numpy as np
import pytest
import torch

import oracle
import paper_2408_14558_gb300 as g
import synth
from parity import assert_full_parity

pytestmark = pytest.mark.gpu


def planning_totals(A, B, P, b):
    bounds = oracle.block_bounds(B.ncols, P)
    tot = dict(sum_H=0, sum_dtilde=0, gathered_nnz_exact=0, gathered_nnz_block=0, fetch_blocks_chosen=0)
    for i in range(P):
        pl = oracle.plan_block(A, B, int(bounds[i]), int(bounds[i + 1]), b)
        tot["sum_H"] += int(pl["H"].sum())
        tot["sum_dtilde"] += int(pl["dtilde"].size)
        tot["gathered_nnz_exact"] += int(pl["vol_exact"])
        tot["gathered_nnz_block"] += int(pl["vol_block"])
        tot["fetch_blocks_chosen"] += int(pl["fetch"].sum())
    return tot


def run_small(A, B, P, b, **kw):
    dA = g.to_device(A, idx_dtype=torch.int32, **kw)
    dB = g.to_device(B, idx_dtype=torch.int32, **kw)
    sp = g.SmallProduct(dA, dB, P, b).run()
    return sp, sp.C(), sp.stats()


@pytest.mark.parametrize("P,b", [(1, 1024), (3, 1), (4, 64), (7, 5), (300, 16)])
@pytest.mark.parametrize("vals", ["f64", "i32", "i64big"])
def test_random_products(P, b, vals):
    rng = np.random.default_rng(P * 7 + b)
    A = synth.random_sparse(300, 257, 0.03, rng, values=vals)
    B = synth.random_sparse(257, 203, 0.03, rng, values=vals)
    ref = oracle.spgemm(A, B)
    sp, C, st = run_small(A, B, P, b)
    assert_full_parity(C, ref, f"small P={P} b={b} {vals}")
    assert st["status"] == 0 and st["nnzC"] == int(ref["colptr"][-1])
    assert st["products"] == int(ref["flops"].sum())
    want = planning_totals(A, B, P, b)
    for key, v in want.items():
        assert st[key] == v, (key, st[key], v)


def test_uniform_8192_config():
    """C = A*A, 8192 x 8192, 8 uniform rows per column, P = 4, b = 256."""
    A = synth.uniform_columns(8192, 8, seed=0)
    ref = oracle.spgemm(A, A)
    sp, C, st = run_small(A, A, 4, 256)
    assert_full_parity(C, ref, "uniform 8192")
    assert st["products"] == 8 * 8 * 8192
    want = planning_totals(A, A, 4, 256)
    assert st["sum_dtilde"] == want["sum_dtilde"] and st["fetch_blocks_chosen"] == want["fetch_blocks_chosen"]


def test_edge_shapes():
    rng = np.random.default_rng(1)
    A = synth.random_sparse(50, 40, 0.1, rng)
    empty_B = synth.CSC(40, 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    zero_B = synth.CSC(40, 6, np.zeros(7, np.int64), np.zeros(0, np.int32), np.zeros(0))
    for B in (empty_B, zero_B):
        sp, C, st = run_small(A, B, 2, 8)
        assert st["status"] == 0 and st["nnzC"] == 0
        assert torch.equal(C.colptr.cpu(), torch.zeros(B.ncols + 1, dtype=torch.int64))
    # cancellation keeps the position (structure independent of rounding)
    A2 = synth.from_dense(np.array([[1.0, 1.0], [0.0, 2.0]]))
    B2 = synth.from_dense(np.array([[1.0], [-1.0]]))
    sp, C, st = run_small(A2, B2, 1, 1)
    assert C.rowidx.cpu().tolist() == [0, 1] and C.vals.cpu().tolist() == [0.0, -2.0]


def test_failure_reports():
    rng = np.random.default_rng(2)
    A = synth.random_sparse(200, 150, 0.05, rng)
    B = synth.random_sparse(150, 120, 0.05, rng)
    ref = oracle.spgemm(A, B)
    dA, dB = g.to_device(A), g.to_device(B)
    nnz = int(ref["colptr"][-1])
    sp = g.SmallProduct(dA, dB, 2, 16, capacity=nnz - 1).run()
    st = sp.stats()
    assert st["status"] == g.SPG_OUT_OF_MEMORY and st["nnzC"] == nnz
    assert np.array_equal(sp.colptr.cpu().numpy(), ref["colptr"])     # column pointers still written
    with pytest.raises(g.SpgError):
        sp.C()
    # a column whose bound min(flops, m) exceeds the warp table (512 slots
    # in the larger class, 128 in the smaller one)
    H = synth.random_sparse(2000, 600, 0.5, rng)
    K = synth.random_sparse(600, 3, 0.9, rng)
    sp = g.SmallProduct(g.to_device(H), g.to_device(K), 1, 64, capacity=6000).run()
    assert sp.max_bound == 2000 and sp.table_log == 10
    assert sp.stats()["status"] == g.SPG_UNSUPPORTED
    M = synth.random_sparse(400, 300, 0.04, rng)      # column bounds around 150..350
    N = synth.random_sparse(300, 200, 0.04, rng)
    dM, dN = g.to_device(M), g.to_device(N)
    probe = g.SmallProduct(dM, dN, 2, 32)
    assert probe.max_bound > 128
    assert g.SmallProduct(dM, dN, 2, 32, table_log=8).run().stats()["status"] == g.SPG_UNSUPPORTED
    assert_full_parity(g.SmallProduct(dM, dN, 2, 32, table_log=10).run().C(), oracle.spgemm(M, N), "class 10")


@pytest.mark.parametrize("table_log", [8, 10])
def test_both_table_classes(table_log):
    rng = np.random.default_rng(table_log)
    A = synth.random_sparse(500, 400, 0.012, rng, values="i64big")
    B = synth.random_sparse(400, 350, 0.012, rng, values="i64big")
    sp = g.SmallProduct(g.to_device(A), g.to_device(B), 3, 16, table_log=table_log).run()
    assert sp.max_bound <= 128
    ref = oracle.spgemm(A, B)
    assert_full_parity(sp.C(), ref, f"class {table_log}")
    assert sp.nnz_bound == int(np.minimum(ref["flops"], A.nrows).sum())


def test_graph_replay_with_new_values():
    A = synth.uniform_columns(4096, 8, seed=3)
    B = synth.uniform_columns(4096, 6, seed=4)
    dA, dB = g.to_device(A), g.to_device(B)
    sp = g.SmallProduct(dA, dB, 4, 256)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        sp.run(s)                       # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        sp.run(s)
    for rep in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert_full_parity(sp.C(), oracle.spgemm(A, B), f"replay {rep}")
    # new values in place, same patterns: the next replay reads them
    B.vals = -2.0 * B.vals
    dB.vals.copy_(torch.from_numpy(B.vals))
    graph.replay()
    torch.cuda.synchronize()
    assert_full_parity(sp.C(), oracle.spgemm(A, B), "replay after new values")
