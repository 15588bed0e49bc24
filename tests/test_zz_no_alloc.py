"""The entry point that allocates nothing (spgemm_count_noalloc) against the
CPU oracle and the ordinary symbolic pass.

That entry point is for callers that may not allocate device memory (their
GPU memory belongs to another allocator, or was reserved once at start-up);
it keeps its scratch in a fixed array inside the library.  Every call shares
that array, so these tests call it twice in a row on the same input, and run
a product whose A has close to the 2^20-row limit (its bitmaps cover the
whole scratch) right before small products, to check that each call starts
from a clean scratch.  This file is collected last so that a stop at the
first failure has already run every other test; it also passes when run
alone in a fresh process."""
import numpy as np
import pytest
import torch

import oracle
import paper_2408_14558_gb300 as g
import synth

pytestmark = pytest.mark.gpu


def symbolic_counts(dA, dB):
    plan = g.spgemm_plan(dA, dB, P=3, b=64)
    colptr, _ = g.spgemm_symbolic(plan)
    g.spgemm_plan_destroy(plan)
    return torch.diff(colptr)


def check(A, B, dA, dB, calls=2):
    want = torch.from_numpy(oracle.spgemm(A, B)["nnz"])
    sym = symbolic_counts(dA, dB).cpu()
    assert torch.equal(sym, want)
    for _ in range(calls):
        got = g.spgemm_count_noalloc(dA, dB).clone()
        torch.cuda.synchronize()
        assert torch.equal(got.cpu(), want)


def small_cases():
    rng = np.random.default_rng(42)
    A = synth.random_sparse(700, 500, 0.02, rng)
    B = synth.random_sparse(500, 300, 0.03, rng)
    R = synth.rmat_symmetric(12, 16, seed=3)
    U = synth.uniform_columns(4096, 8, seed=9)
    return [(A, B), (R, R), (U, U)]


def test_two_calls_in_a_row_match_oracle():
    for A, B in small_cases():
        check(A, B, g.to_device(A), g.to_device(B))


def test_large_then_small_products():
    # A with 2^20 - 5 rows: every CTA's bitmap spans (almost) the whole scratch,
    # and its columns set bits all over it; the small products that follow must
    # not see any of them.
    m = (1 << 20) - 5
    Abig = synth.uniform_columns(4096, 24, seed=5, m=m)
    Bbig = synth.uniform_columns(3000, 8, seed=6, m=4096)
    check(Abig, Bbig, g.to_device(Abig), g.to_device(Bbig), calls=1)
    for A, B in small_cases():
        check(A, B, g.to_device(A), g.to_device(B), calls=1)


def test_index_types_and_rejection():
    A = synth.uniform_columns(2000, 5, seed=1)
    dA = g.to_device(A, ptr_dtype=torch.int64, idx_dtype=torch.int64)
    want = torch.from_numpy(oracle.spgemm(A, A)["nnz"])
    assert torch.equal(g.spgemm_count_noalloc(dA, dA).cpu(), want)
    big = g.DeviceCSC((1 << 20) + 1, 3, torch.zeros(4, dtype=torch.int64, device="cuda"),
                      torch.zeros(0, dtype=torch.int32, device="cuda"), torch.zeros(0, device="cuda", dtype=torch.float64))
    small = g.DeviceCSC(3, 2, torch.zeros(3, dtype=torch.int64, device="cuda"),
                        torch.zeros(0, dtype=torch.int32, device="cuda"), torch.zeros(0, device="cuda", dtype=torch.float64))
    with pytest.raises(g.SpgError) as e:
        g.spgemm_count_noalloc(big, small)
    assert e.value.status == g.SPG_UNSUPPORTED
    # an output array of the wrong type or length is refused before any launch
    with pytest.raises(ValueError):
        g.spgemm_count_noalloc(dA, dA, nnz_out=torch.empty(A.ncols, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        g.spgemm_count_noalloc(dA, dA, nnz_out=torch.empty(A.ncols - 1, dtype=torch.int64, device="cuda"))
