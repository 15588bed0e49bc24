"""The masked product C<M> = A*B (an output mask applied inside the symbolic
and numeric passes) against the oracle's definition: the unmasked product with
every entry outside the mask (or, complemented, inside it) removed."""
import numpy as np
import pytest
import torch

import oracle
import paper_2408_14558_gb300 as g
import synth
from parity import assert_full_parity, mask_from_pattern

pytestmark = pytest.mark.gpu


def masked_gpu(A, B, M, complement, P, b, words=None, **kw):
    dA, dB = g.to_device(A), g.to_device(B)
    mask = mask_from_pattern(M, words=words)
    plan = g.spgemm_plan(dA, dB, P, b, mask=mask, mask_complement=complement, **kw)
    try:
        g.spgemm_symbolic(plan)
        C = g.spgemm_numeric(plan)
    finally:
        g.spgemm_plan_destroy(plan)
    torch.cuda.synchronize()
    return C


@pytest.mark.parametrize("P,b", [(1, 1024), (3, 16)])
@pytest.mark.parametrize("vals", ["f64", "i64"])
@pytest.mark.parametrize("complement", [False, True])
def test_masked_random_small(P, b, vals, complement):
    rng = np.random.default_rng(P * 7 + b + (3 if complement else 0))
    kind = "f64" if vals == "f64" else "i64big"
    A = synth.random_sparse(300, 257, 0.03, rng, values=kind)
    B = synth.random_sparse(257, 203, 0.05, rng, values=kind)
    M = synth.random_sparse(300, 203, 0.3, rng)
    C = masked_gpu(A, B, M, complement, P, b)
    assert_full_parity(C, oracle.spgemm_masked(A, B, M, complement), f"masked P={P} b={b} {vals} c={complement}")


@pytest.mark.parametrize("vals", ["f64", "i64"])
@pytest.mark.parametrize("complement", [False, True])
def test_masked_heavy_bins(vals, complement):
    """R-MAT scale-12 squaring with small light tables and 1024-row slabs (most
    columns in the heavy bin), masked by A's own pattern (the products that
    close a triangle) or by its complement; mask rows padded by 3 words."""
    P0 = synth.rmat_symmetric(12, 16, seed=2)
    rng = np.random.default_rng(9)
    v = rng.uniform(-1, 1, P0.nnz) if vals == "f64" else rng.integers(-2**40, 2**40, P0.nnz)
    A = synth.CSC(P0.nrows, P0.ncols, P0.colptr, P0.rowidx, v)
    C = masked_gpu(A, A, A, complement, 4, 256, words=(A.nrows + 31) // 32 + 3, light_max=32, slab_rows=1024)
    ref = oracle.spgemm_masked(A, A, A, complement)
    assert_full_parity(C, ref, f"masked heavy {vals} c={complement}")


def test_full_and_empty_masks():
    rng = np.random.default_rng(11)
    A = synth.random_sparse(200, 150, 0.05, rng, values="i64")
    B = synth.random_sparse(150, 120, 0.05, rng, values="i64")
    full = synth.CSC(200, 120, np.arange(121, dtype=np.int64) * 200, np.tile(np.arange(200, dtype=np.int64), 120),
                     np.ones(200 * 120))
    empty = synth.CSC(200, 120, np.zeros(121, dtype=np.int64), np.zeros(0, dtype=np.int64), np.zeros(0))
    ref = oracle.spgemm(A, B)
    for M, c in ((full, False), (empty, True)):
        assert_full_parity(masked_gpu(A, B, M, c, 2, 64, light_max=64, slab_rows=1024), ref, f"mask c={c}")
    for M, c in ((full, True), (empty, False)):
        C = masked_gpu(A, B, M, c, 2, 64)
        assert int(C.colptr[-1]) == 0


def test_masked_refresh_and_replay():
    """A refresh and a captured replay of a masked plan re-read the mask."""
    rng = np.random.default_rng(4)
    A = synth.random_sparse(3000, 700, 0.01, rng)
    B = synth.random_sparse(700, 600, 0.04, rng)
    M = synth.random_sparse(3000, 600, 0.2, rng)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        dA, dB = g.to_device(A), g.to_device(B)
        mask = mask_from_pattern(M)
        plan = g.spgemm_plan(dA, dB, 4, 64, light_max=32, slab_rows=1024, mask=mask, mask_complement=True)
        g.spgemm_symbolic(plan)
        C = g.spgemm_numeric(plan)
        s.synchronize()
        assert_full_parity(C, oracle.spgemm_masked(A, B, M, True), "first")
        A2 = synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, rng.uniform(-1, 1, A.nnz))
        dA.vals.copy_(torch.from_numpy(np.asarray(A2.vals)))
        g.spgemm_plan_capture(plan, C)
        C.vals.zero_()
        g.spgemm_plan_replay(plan)
        s.synchronize()
        assert_full_parity(C, oracle.spgemm_masked(A2, B, M, True), "replay")
        g.spgemm_plan_destroy(plan)


def test_masked_one_call_multiply_and_errors():
    rng = np.random.default_rng(8)
    A = synth.random_sparse(100, 80, 0.05, rng)
    B = synth.random_sparse(80, 60, 0.05, rng)
    M = synth.random_sparse(100, 60, 0.5, rng)
    dA, dB = g.to_device(A), g.to_device(B)
    C, st = g.spgemm_1d_multiply(dA, dB, 2, 32, mask=mask_from_pattern(M))
    assert st == g.SPG_OK
    assert_full_parity(C, oracle.spgemm_masked(A, B, M), "one call")
    with pytest.raises(ValueError):
        g.spgemm_1d_multiply(dA, dB, 2, 32, mask=mask_from_pattern(M)[:, :2])
