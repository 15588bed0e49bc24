"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle
on the same seeded inputs.  Structure and integers bit-exact, doubles within
1e-12 * sum |a_rk * b_kj| per entry."""
import numpy as np
import pytest
import torch

import oracle
import paper_2408_14558_gb300 as g
import synth
from parity import assert_full_parity, assert_sampled_parity, check_values, run_gpu

pytestmark = pytest.mark.gpu


# ------------------------------------------------------------- small / ragged

@pytest.mark.parametrize("P,b", [(1, 1024), (2, 1), (3, 32), (7, 5), (4, 100)])
@pytest.mark.parametrize("vals", ["f64", "i32", "i64"])
def test_random_small(P, b, vals):
    rng = np.random.default_rng(P * 31 + b)
    A = synth.random_sparse(300, 257, 0.03, rng, values=vals if vals != "i64" else "i64big")
    B = synth.random_sparse(257, 203, 0.03, rng, values=vals if vals != "i64" else "i64big")
    ref = oracle.spgemm(A, B)
    C = run_gpu(A, B, P, b)
    assert_full_parity(C, ref, f"P={P} b={b} {vals}")


@pytest.mark.parametrize("P", [63, 64, 100, 257])
def test_many_blocks(P):
    """More blocks than the plan's fixed host counters (and, for P = 257, more
    blocks than columns of B: some blocks are empty)."""
    rng = np.random.default_rng(P)
    A = synth.random_sparse(300, 257, 0.03, rng, values="f64")
    B = synth.random_sparse(257, 203, 0.03, rng, values="f64")
    ref = oracle.spgemm(A, B)
    C = run_gpu(A, B, P, 16)
    assert_full_parity(C, ref, f"P={P}")


@pytest.mark.parametrize("ptr,idx", [(torch.int32, torch.int64), (torch.int64, torch.int32), (torch.int64, torch.int64)])
def test_index_types(ptr, idx):
    rng = np.random.default_rng(7)
    A = synth.random_sparse(400, 350, 0.02, rng)
    B = synth.random_sparse(350, 420, 0.02, rng)
    ref = oracle.spgemm(A, B)
    C = run_gpu(A, B, 3, 64, ptr=ptr, idx=idx)
    assert C.rowidx.dtype == idx
    assert_full_parity(C, ref, f"ptr={ptr} idx={idx}")


@pytest.mark.parametrize("light_max,slab", [(32, 1024), (64, 2048), (1024, 1024)])
@pytest.mark.parametrize("vals", ["f64", "i64"])
def test_heavy_slabs(light_max, slab, vals):
    """Force the dense-slab bins (several slabs per column, row windows that
    start and end inside a slab) and compare everything."""
    rng = np.random.default_rng(light_max + slab)
    m = 5000
    A = synth.random_sparse(m, 600, 0.01, rng, values="f64" if vals == "f64" else "i64big")
    B = synth.random_sparse(600, 500, 0.05, rng, values="f64" if vals == "f64" else "i64big")
    ref = oracle.spgemm(A, B)
    C = run_gpu(A, B, 5, 128, light_max=light_max, slab_rows=slab)
    assert_full_parity(C, ref, f"heavy {light_max} {slab} {vals}")


@pytest.mark.parametrize("vals", ["f64", "i64"])
def test_heavy_slabs_int64_indices(vals):
    """The dense-slab kernels with int64 row ids and column pointers (their
    64-bit output-index instances), several items per column."""
    rng = np.random.default_rng(21)
    m = 9000
    A = synth.random_sparse(m, 500, 0.012, rng, values="f64" if vals == "f64" else "i64big")
    B = synth.random_sparse(500, 300, 0.12, rng, values="f64" if vals == "f64" else "i64big")
    ref = oracle.spgemm(A, B)
    assert ref["nnz"].max() > 4096          # some columns span two numeric items
    C = run_gpu(A, B, 3, 64, ptr=torch.int64, idx=torch.int64, light_max=32, slab_rows=1024)
    assert C.rowidx.dtype == torch.int64
    assert_full_parity(C, ref, f"heavy int64 indices {vals}")


def test_banded_windows():
    """Clustered rows (a banded A) give narrow row windows: light bins hold
    columns with many products but few distinct rows."""
    n = 4000
    rows, cols = [], []
    for j in range(n):
        for d in range(-20, 21):
            if 0 <= j + d < n:
                rows.append(j + d)
                cols.append(j)
    from synth import _csc_from_sorted
    A = _csc_from_sorted(n, n, np.array(cols), np.array(rows), np.random.default_rng(1).uniform(-1, 1, len(rows)))
    ref = oracle.spgemm(A, A)
    C = run_gpu(A, A, 6, 256, light_max=256, slab_rows=1024)
    assert_full_parity(C, ref, "banded")


def test_edge_cases():
    z = lambda m, n: synth.CSC(m, n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    rng = np.random.default_rng(3)
    cases = [
        (z(5, 4), z(4, 6), 2, 3),                 # no nonzeros at all
        (z(0, 3), synth.random_sparse(3, 4, 0.9, rng), 2, 1),   # m = 0
        (synth.random_sparse(4, 0, 0.5, rng), z(0, 5), 3, 2),  # k = 0
        (synth.random_sparse(6, 5, 0.5, rng), z(5, 0), 1, 2),  # n = 0
        (synth.random_sparse(1, 9, 0.7, rng), synth.random_sparse(9, 13, 0.4, rng), 7, 2),  # m = 1, P > n/2
        (synth.random_sparse(30, 20, 0.2, rng), synth.random_sparse(20, 5, 0.3, rng), 7, 1000),  # P > n, b > k
    ]
    for A, B, P, b in cases:
        ref = oracle.spgemm(A, B)
        C = run_gpu(A, B, P, b)
        assert_full_parity(C, ref, f"edge {A.nrows}x{A.ncols}x{B.ncols} P={P}")


def test_cancellation_stays_structural():
    A = synth.CSC(1, 2, np.array([0, 1, 2]), np.array([0, 0], np.int32), np.array([1.0, 1.0]))
    B = synth.CSC(2, 1, np.array([0, 2]), np.array([0, 1], np.int32), np.array([1.0, -1.0]))
    C = run_gpu(A, B, 1, 1)
    cp, ri, v = C.to_host()
    assert cp.tolist() == [0, 1] and ri.tolist() == [0] and v.tolist() == [0.0]


# ---------------------------------------------------------- phase parity

@pytest.mark.parametrize("P,b", [(4, 256), (3, 7)])
def test_planning_phases_match_oracle(P, b):
    """H_i, D~_i, the fetch blocks of Algorithm 2, A~_i and flops_j of every
    block, exported from the plan, equal the oracle's."""
    A = synth.uniform_columns(2048, 8, seed=5)
    A.colptr[100:140] = A.colptr[100]                    # make some columns of A empty
    A = synth.CSC(A.nrows, A.ncols, A.colptr, np.concatenate([A.rowidx[:A.colptr[100]], A.rowidx[A.colptr[100] + 320:]]),
                  np.concatenate([A.vals[:A.colptr[100]], A.vals[A.colptr[100] + 320:]]))
    A.colptr[140:] -= 320
    B = synth.uniform_columns(2048, 6, seed=6)
    dA, dB = g.to_device(A, ptr_dtype=torch.int32), g.to_device(B, ptr_dtype=torch.int32)
    plan = g.spgemm_plan(dA, dB, P, b)
    bounds = oracle.block_bounds(B.ncols, P)
    own = oracle.block_bounds(A.ncols, P)
    remote = 0
    for i in range(P):
        ex = g.spgemm_plan_export(plan, i)
        pl = oracle.plan_block(A, B, int(bounds[i]), int(bounds[i + 1]), b)
        dt = pl["dtilde"]
        away = dt[(dt < own[i]) | (dt >= own[i + 1])]
        remote += int(np.sum(A.colptr[away + 1] - A.colptr[away]))
        words = ex["H_bits"].cpu().numpy().view(np.uint32)
        H = np.unpackbits(words.view(np.uint8), bitorder="little")[: A.ncols]
        assert np.array_equal(H, pl["H"]), f"H_{i}"
        assert np.array_equal(ex["dtilde"].cpu().numpy(), pl["dtilde"]), f"D~_{i}"
        assert np.array_equal(ex["fetch"].cpu().numpy(), pl["fetch"]), f"fetch_{i}"
        At = oracle.gather(A, pl["dtilde"])
        assert np.array_equal(ex["At_colptr"].cpu().numpy(), At["colptr"])
        assert np.array_equal(ex["At_rowidx"].cpu().numpy().astype(np.int64), At["rowidx"])
        assert np.array_equal(ex["At_vals"].cpu().numpy(), At["vals"])
        f = oracle.features(A, B, int(bounds[i]), int(bounds[i + 1]))
        assert np.array_equal(ex["flops"].cpu().numpy(), f["flops"])
    st = g.spgemm_plan_stats(plan)
    assert st["products"] == int(oracle.features(A, B)["flops"].sum())
    assert st["gathered_nnz_remote"] == remote
    g.spgemm_plan_destroy(plan)


def test_invalid_input_is_rejected():
    rng = np.random.default_rng(0)
    A = synth.random_sparse(20, 10, 0.3, rng)
    B = synth.random_sparse(10, 8, 0.3, rng)
    bad = synth.CSC(B.nrows, B.ncols, B.colptr.copy(), B.rowidx.copy(), B.vals)
    j = int(np.flatnonzero(np.diff(bad.colptr) >= 2)[0])
    s = bad.colptr[j]
    bad.rowidx[s], bad.rowidx[s + 1] = bad.rowidx[s + 1], bad.rowidx[s]    # unsorted column
    with pytest.raises(g.SpgError) as e:
        run_gpu(A, bad, 2, 4)
    assert e.value.status == g.SPG_INVALID_INPUT
    oob = synth.CSC(B.nrows, B.ncols, B.colptr, B.rowidx.copy(), B.vals)
    oob.rowidx[-1] = B.nrows + 3                                          # row out of range
    with pytest.raises(g.SpgError) as e:
        run_gpu(A, oob, 2, 4)
    assert e.value.status == g.SPG_INVALID_INPUT
    dup = synth.CSC(B.nrows, B.ncols, B.colptr, B.rowidx.copy(), B.vals)
    dup.rowidx[s + 1] = dup.rowidx[s]                                     # repeated row in a column
    with pytest.raises(g.SpgError) as e:
        run_gpu(A, dup, 2, 4)
    assert e.value.status == g.SPG_INVALID_INPUT
    cp = B.colptr.copy()
    j2 = int(np.flatnonzero(np.diff(cp) >= 1)[-1])                        # the last non-empty column
    cp[j2], cp[j2 + 1] = cp[j2 + 1], cp[j2]                               # column pointers out of order
    with pytest.raises(g.SpgError) as e:
        run_gpu(A, synth.CSC(B.nrows, B.ncols, cp, B.rowidx, B.vals), 2, 4)
    assert e.value.status == g.SPG_INVALID_INPUT


def test_rows_may_fall_between_columns():
    """Canonical input whose row ids drop from one column to the next, also
    across empty columns and at a column holding the same first row: accepted."""
    cols = [[5, 9], [], [], [0, 9], [9], [], [1], [0, 1, 2]]
    cp = np.cumsum([0] + [len(c) for c in cols]).astype(np.int64)
    ri = np.array([r for c in cols for r in c], dtype=np.int32)
    B = synth.CSC(10, len(cols), cp, ri, np.arange(1, ri.size + 1, dtype=np.float64))
    A = synth.random_sparse(12, 10, 0.4, np.random.default_rng(2), values="small")
    assert_full_parity(run_gpu(A, B, 3, 4), oracle.spgemm(A, B), "row drops at column starts")


def test_one_call_multiply_and_stats():
    A = synth.uniform_columns(3000, 8, seed=2)
    dA = g.to_device(A)
    C, st = g.spgemm_1d_multiply(dA, dA, P=4, b=256)
    assert st == g.SPG_OK
    ref = oracle.spgemm(A, A)
    assert_full_parity(C, ref, "1d_multiply")


# -------------------------------------------------------- paper workloads

def test_uniform_8192_full():
    """8192 x 8192, 8 nonzeros per column, P = 4, b = 256: whole C compared."""
    A = synth.uniform_columns(8192, 8, seed=0)
    ref = oracle.spgemm(A, A)
    C = run_gpu(A, A, 4, 256)
    assert_full_parity(C, ref, "uniform 8192")
    assert int(ref["flops"].sum()) == 8 * 8 * 8192
    Ai = synth.uniform_columns(8192, 8, seed=0, values="i32")
    refi = oracle.spgemm(Ai, Ai)
    Ci = run_gpu(Ai, Ai, 4, 256)
    assert_full_parity(Ci, refi, "uniform 8192 int")


@pytest.mark.parametrize("scale", [12, 14])
def test_rmat_squaring_reduced(scale):
    """R-MAT squaring at reduced scale (skewed degrees: light and heavy bins),
    double and int64 path counts, whole C compared."""
    A = synth.rmat_symmetric(scale, 16, seed=0)
    Ai = synth.rmat_symmetric(scale, 16, seed=0, values="i64")
    ref = oracle.spgemm(A, A)
    C = run_gpu(A, A, 16, 1024 if scale > 12 else 256, light_max=256, slab_rows=1024)
    assert_full_parity(C, ref, f"rmat s{scale}")
    refi = oracle.spgemm(Ai, Ai)
    Ci = run_gpu(Ai, Ai, 16, 1024, light_max=256, slab_rows=1024)
    assert_full_parity(Ci, refi, f"rmat s{scale} int64")


@pytest.mark.slow
def test_rmat_s18_full_size_sampled():
    """The full R-MAT scale-18 squaring (P = 16, b = 1024) in the bench's launch
    configuration: sampled columns (the heaviest, random, light) against the
    oracle, and the double run equal to the int64 path-count run everywhere
    (all sums are integers below 2^53, so exact)."""
    A = synth.rmat_symmetric(18, 16, seed=0)
    Ai = synth.rmat_symmetric(18, 16, seed=0, values="i64")
    dA = g.to_device(A)
    C = g.multiply(dA, dA, 16, 1024)
    fl = oracle.features(A, A)["flops"]
    rng = np.random.default_rng(0)
    heavy = np.argsort(fl)[-8:]
    light = rng.choice(np.flatnonzero((fl > 0) & (fl < 2000)), 40, replace=False)
    mid = rng.choice(np.flatnonzero(fl >= 2000), 40, replace=False)
    cols = np.unique(np.concatenate([heavy, light, mid, [0, A.ncols - 1]]))
    assert_sampled_parity(C, A, A, cols, "rmat s18 f64")
    dAi = g.to_device(Ai)
    Ci = g.multiply(dAi, dAi, 16, 1024)
    assert torch.equal(C.colptr, Ci.colptr)
    assert torch.equal(C.rowidx, Ci.rowidx)
    assert torch.equal(C.vals.to(torch.int64), Ci.vals)
    assert int(C.colptr[-1]) <= int(fl.sum())


@pytest.mark.parametrize("vals", ["ones", "i64"])
def test_rmat_s18_complete_against_oracle(vals):
    """All of the R-MAT scale-18 squaring (P = 16, b = 1024, the bench's launch
    configuration and plan/symbolic/numeric calls) against the oracle, one
    column block at a time (Section 3.1: the block partition never changes the
    result): column pointers and row ids bit-exact, int64 path counts
    bit-exact, every double within 1e-12 * sum |a_rk * b_kj|."""
    A = synth.rmat_symmetric(18, 16, seed=0, values=vals)
    dA = g.to_device(A, ptr_dtype=torch.int32, idx_dtype=torch.int32)
    plan = g.spgemm_plan(dA, dA, 16, 1024)
    colptr, nnz = g.spgemm_symbolic(plan)
    C = g.spgemm_numeric(plan, colptr)
    g.spgemm_plan_destroy(plan)
    torch.cuda.synchronize()
    cp = C.colptr.cpu().numpy()
    assert cp[0] == 0 and int(cp[-1]) == nnz
    bounds = oracle.block_bounds(A.ncols, 16)
    total = 0
    for i in range(16):
        c0, c1 = int(bounds[i]), int(bounds[i + 1])
        ref = oracle.spgemm(A, A, cols=np.arange(c0, c1))
        assert np.array_equal(cp[c0:c1 + 1] - cp[c0], ref["colptr"]), f"block {i}: column pointers differ"
        e0, e1 = int(cp[c0]), int(cp[c1])
        rows = C.rowidx[e0:e1].cpu().numpy()
        assert np.array_equal(rows, ref["rowidx"].astype(np.int32)), f"block {i}: row ids differ"
        del rows
        check_values(C.vals[e0:e1].cpu().numpy(), ref["vals"], ref["absum"], f"block {i} {vals}")
        total += e1 - e0
        del ref
    assert total == nnz == 2958091137


def test_galerkin_128():
    """A (7-point, 128^3) * P_agg, then P_agg^T * (A P_agg), P = 32, b = 2048:
    both products compared in full; the coarse operator has the closed-form
    nnz 7*64^3 - 6*64^2."""
    N = 128
    A = synth.poisson3d(N)
    Pg = synth.aggregation_2x2x2(N)
    PT = synth.aggregation_2x2x2_transpose(N)
    ref1 = oracle.spgemm(A, Pg)
    dA, dP, dPT = g.to_device(A), g.to_device(Pg), g.to_device(PT)
    AP = g.multiply(dA, dP, 32, 2048)
    torch.cuda.synchronize()
    assert_full_parity(AP, ref1, "A*P_agg")
    AP_host = synth.CSC(ref1["nrows"], ref1["ncols"], ref1["colptr"], ref1["rowidx"].astype(np.int32), ref1["vals"])
    ref2 = oracle.spgemm(PT, AP_host)
    AP_dev = g.DeviceCSC(AP.nrows, AP.ncols, AP.colptr, AP.rowidx, AP.vals)
    G = g.multiply(dPT, AP_dev, 32, 2048)
    torch.cuda.synchronize()
    assert_full_parity(G, ref2, "P^T (A P)")
    assert int(G.colptr[-1]) == 7 * 64 ** 3 - 6 * 64 ** 2


def test_similarity_reduced():
    """A * A^T for lognormal rows / Zipf columns, int32 values, int64 result."""
    A, At = synth.lognormal_zipf_rows(nrows=3000, ncols=1 << 16, mean=50, cap=500, seed=4)
    ref = oracle.spgemm(A, At)
    C = run_gpu(A, At, 8, 1024, light_max=512, slab_rows=1024)
    assert_full_parity(C, ref, "similarity")


@pytest.mark.slow
def test_similarity_full_size_every_chunk_sampled():
    """C = A * A^T at full size on all four column chunks the benchmark
    multiplies (P = 4 per chunk, b = 1024, int64 column pointers): per chunk
    the heaviest columns, random ones and both ends against the oracle, the
    chunk's column counts against the oracle's, and the learned-sizing result
    identical to the exact one."""
    from paper_2408_14558_gb300 import learned
    A, At = synth.lognormal_zipf_rows(seed=0)
    dA = g.to_device(A, ptr_dtype=torch.int64, idx_dtype=torch.int32)
    dAt = g.to_device(At, ptr_dtype=torch.int64, idx_dtype=torch.int32)
    model = g.spgemm_model_load(learned.DEFAULT_MODEL)
    n, chunks = At.ncols, 4
    bounds = [(i * n) // chunks for i in range(chunks + 1)]
    rng = np.random.default_rng(7)
    for ch in range(chunks):
        c0, c1 = bounds[ch], bounds[ch + 1]
        s, e = int(dAt.colptr[c0]), int(dAt.colptr[c1])
        B = g.DeviceCSC(At.nrows, c1 - c0, (dAt.colptr[c0:c1 + 1] - s).contiguous(), dAt.rowidx[s:e],
                        dAt.vals[s:e])
        C, _ = g.spgemm_1d_multiply(dA, B, P=4, b=1024)
        f = oracle.features(A, At, c0, c1)
        cols = np.unique(np.concatenate([np.argsort(f["flops"])[-4:], rng.choice(c1 - c0, 24, replace=False),
                                         [0, c1 - c0 - 1]]))
        Bh = synth.CSC(At.nrows, c1 - c0, np.asarray(At.colptr[c0:c1 + 1], dtype=np.int64) - s,
                       np.asarray(At.rowidx[s:e]), np.asarray(At.vals[s:e]))
        assert_sampled_parity(C, A, Bh, cols, f"similarity chunk {ch}")
        Cl, _ = g.spgemm_1d_multiply(dA, B, P=4, b=1024, sizing=g.SPG_SIZING_LEARNED, model=model)
        torch.cuda.synchronize()
        assert torch.equal(Cl.colptr, C.colptr), ch
        assert torch.equal(Cl.rowidx, C.rowidx), ch
        assert torch.equal(Cl.vals, C.vals), ch
        del C, Cl, B
        torch.cuda.empty_cache()
