"""spgemm_1d_multiply_host: host matrices in, host product out, the copies
inside the call and C streamed back group by group; against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2408_14558_gb300 as g
import synth
from parity import check_values, mask_from_pattern

pytestmark = pytest.mark.gpu


def pinned(M):
    return synth.CSC(M.nrows, M.ncols, torch.from_numpy(np.ascontiguousarray(M.colptr)).pin_memory(),
                     torch.from_numpy(np.ascontiguousarray(M.rowidx)).pin_memory(),
                     torch.from_numpy(np.ascontiguousarray(M.vals)).pin_memory())


def assert_host_parity(C, ref, where):
    assert np.array_equal(C.colptr.numpy(), ref["colptr"]), f"{where}: column pointers differ"
    assert np.array_equal(C.rowidx.numpy().astype(np.int64), ref["rowidx"]), f"{where}: row indices differ"
    check_values(C.vals.numpy(), ref["vals"], ref["absum"], where)


@pytest.mark.parametrize("P,chunks", [(1, 1), (4, 3), (7, 8), (16, 4)])
@pytest.mark.parametrize("vals", ["f64", "i32", "i64"])
def test_host_multiply_random(P, chunks, vals):
    rng = np.random.default_rng(P * 13 + chunks)
    kind = "i64big" if vals == "i64" else vals
    A = synth.random_sparse(300, 257, 0.03, rng, values=kind)
    B = synth.random_sparse(257, 203, 0.05, rng, values=kind)
    C = g.spgemm_1d_multiply_host(pinned(A), pinned(B), P=P, b=32, chunks=chunks)
    assert_host_parity(C, oracle.spgemm(A, B), f"host P={P} chunks={chunks} {vals}")
    st = g.spgemm_last_multiply_stats()
    assert st["nnzC"] == C.nnz and st["products"] == int(oracle.features(A, B)["flops"].sum())


def test_host_multiply_shared_arrays_pool_and_heavy_bins():
    """A * A with one set of host arrays (copied once), heavy bins, int64 and
    double runs into one reused pinned pool, equal to the device path."""
    A = synth.rmat_symmetric(13, 16, seed=4)
    Ai = synth.rmat_symmetric(13, 16, seed=4, values="i64")
    pool = g.HostPool(256 << 20)
    hA, hAi = pinned(A), pinned(Ai)
    for M, hM in ((A, hA), (Ai, hAi)):
        C = g.spgemm_1d_multiply_host(hM, hM, P=16, b=1024, chunks=4, light_max=64, slab_rows=1024, pool=pool)
        D = g.multiply(g.to_device(M), g.to_device(M), 16, 1024, light_max=64, slab_rows=1024)
        assert torch.equal(C.colptr, D.colptr.cpu())
        assert torch.equal(C.rowidx, D.rowidx.cpu())
        assert torch.equal(C.vals, D.vals.cpu())


def test_host_multiply_edges_and_mask():
    z = lambda m, n: synth.CSC(m, n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    rng = np.random.default_rng(6)
    for A, B in ((z(5, 4), z(4, 6)), (synth.random_sparse(6, 5, 0.5, rng), z(5, 0))):
        C = g.spgemm_1d_multiply_host(A, B, P=3, b=2, chunks=2)
        assert C.nnz == 0 and C.colptr.numel() == B.ncols + 1 and int(C.colptr[-1]) == 0
    A = synth.random_sparse(400, 300, 0.03, rng)
    B = synth.random_sparse(300, 250, 0.05, rng)
    M = synth.random_sparse(400, 250, 0.3, rng)
    C = g.spgemm_1d_multiply_host(A, B, P=6, b=16, chunks=3)
    assert_host_parity(C, oracle.spgemm(A, B), "numpy inputs")
    for comp in (False, True):
        # each group of columns reads its own columns of the mask
        C = g.spgemm_1d_multiply_host(A, B, P=6, b=16, chunks=3, mask=mask_from_pattern(M), mask_complement=comp)
        assert_host_parity(C, oracle.spgemm_masked(A, B, M, comp), f"masked c={comp}")


def test_direct_stores_and_copy_engine_agree():
    """The same product with C's host arrays page-locked (the kernels store C
    into them directly where the GPU addresses them with the same pointers)
    and pageable (C always comes back through the copy engine): both equal
    the oracle."""
    A = synth.rmat_symmetric(12, 16, seed=8)
    ref = oracle.spgemm(A, A)
    hA = pinned(A)
    pool = g.HostPool(64 << 20)
    probe = pool.take(1 << 20)
    direct = g.spgemm_host_writable(probe)
    assert not g.spgemm_host_writable(torch.empty(1 << 20, dtype=torch.uint8))   # pageable: never
    for kw in ({"pool": pool}, {"pinned": False}, {}):
        C = g.spgemm_1d_multiply_host(hA, hA, P=8, b=256, chunks=3, light_max=128, slab_rows=1024, **kw)
        assert_host_parity(C, ref, f"host arrays {kw or 'pinned'} (direct stores possible: {direct})")
