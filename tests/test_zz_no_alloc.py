"""The entry point that allocates nothing (spgemm_count_noalloc) against the
ordinary symbolic pass.

That entry point is for callers that may not allocate device memory (their
GPU memory belongs to another allocator, or was reserved once at start-up);
it keeps its scratch in a fixed array inside the library.  Every call shares
that array, so these tests make two calls in a row, on different inputs, to
check that each call starts from a clean scratch.  This file is collected
last so that a stop at the first failure has already run every other test;
it also passes when run alone in a fresh process."""
import numpy as np
import pytest
import torch

import paper_2408_14558_gb300 as g
import synth

pytestmark = pytest.mark.gpu


def reference_counts(dA, dB):
    plan = g.spgemm_plan(dA, dB, P=3, b=64)
    colptr, _ = g.spgemm_symbolic(plan)
    g.spgemm_plan_destroy(plan)
    return torch.diff(colptr)


def cases():
    rng = np.random.default_rng(42)
    A = synth.random_sparse(700, 500, 0.02, rng)
    B = synth.random_sparse(500, 300, 0.03, rng)
    R = synth.rmat_symmetric(12, 16, seed=3)
    U = synth.uniform_columns(4096, 8, seed=9)
    return [(A, B), (R, R), (U, U)]


def test_two_calls_in_a_row_match_symbolic():
    for A, B in cases():
        dA, dB = g.to_device(A), g.to_device(B)
        want = reference_counts(dA, dB)
        first = g.spgemm_count_noalloc(dA, dB).clone()
        second = g.spgemm_count_noalloc(dA, dB).clone()
        torch.cuda.synchronize()
        assert torch.equal(first, want)
        assert torch.equal(second, want)


def test_index_types_and_rejection():
    A = synth.uniform_columns(2000, 5, seed=1)
    dA = g.to_device(A, ptr_dtype=torch.int64, idx_dtype=torch.int64)
    want = reference_counts(dA, dA)
    assert torch.equal(g.spgemm_count_noalloc(dA, dA), want)
    big = g.DeviceCSC((1 << 20) + 1, 3, torch.zeros(4, dtype=torch.int64, device="cuda"),
                      torch.zeros(0, dtype=torch.int32, device="cuda"), torch.zeros(0, device="cuda", dtype=torch.float64))
    small = g.DeviceCSC(3, 2, torch.zeros(3, dtype=torch.int64, device="cuda"),
                        torch.zeros(0, dtype=torch.int32, device="cuda"), torch.zeros(0, device="cuda", dtype=torch.float64))
    with pytest.raises(g.SpgError) as e:
        g.spgemm_count_noalloc(big, small)
    assert e.value.status == g.SPG_UNSUPPORTED
