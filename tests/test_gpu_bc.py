"""GPU parity of the batched betweenness centrality (forward search and
backward sweep through the column 1D SpGEMM) against the CPU Brandes oracle:
level sizes exactly, scores within floating-point rounding."""
import numpy as np
import pytest
import torch

import paper_2408_14558_gb300 as g
import synth
from oracle import bc as obc

pytestmark = pytest.mark.gpu


def _path(n):
    rows, cols = [], []
    for a in range(n - 1):
        rows += [a + 1, a]
        cols += [a, a + 1]
    order = np.lexsort((rows, cols))
    return synth._csc_from_sorted(n, n, np.array(cols)[order], np.array(rows)[order], np.ones(len(rows)))


@pytest.mark.parametrize("P", [1, 3])
def test_bc_path_graph(P):
    n = 12
    A = _path(n)
    bc, levels, st = g.spgemm_bc_batch(g.to_device(A), torch.arange(n, dtype=torch.int32), P=P, b=4)
    assert np.allclose(bc.cpu().numpy(), [2 * i * (n - 1 - i) for i in range(n)])
    assert sum(levels) == n * n and st["levels"] == n


@pytest.mark.parametrize("scale,nsrc,P", [(9, 32, 1), (10, 64, 4), (11, 40, 7)])
def test_bc_rmat_batch(scale, nsrc, P):
    A = synth.rmat_symmetric(scale, 8, seed=scale)
    rng = np.random.default_rng(scale)
    src = rng.choice(A.ncols, nsrc, replace=False)
    ref, ref_levels = obc.brandes(A, src)
    bc, levels, st = g.spgemm_bc_batch(g.to_device(A), torch.from_numpy(src.astype(np.int32)), P=P, b=64)
    got = bc.cpu().numpy()
    assert levels == ref_levels
    assert st["frontier_nnz"] == sum(ref_levels)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-9 * max(1.0, np.abs(ref).max()))


def test_bc_accumulates_across_batches_and_rejects_bad_sources():
    A = synth.rmat_symmetric(9, 8, seed=2)
    src = np.arange(0, 40, dtype=np.int32)
    ref, _ = obc.brandes(A, src)
    dA = g.to_device(A)
    bc, _, _ = g.spgemm_bc_batch(dA, torch.from_numpy(src[:25]))
    bc, _, _ = g.spgemm_bc_batch(dA, torch.from_numpy(src[25:]), bc=bc)
    assert np.allclose(bc.cpu().numpy(), ref, rtol=1e-11, atol=1e-9 * max(1.0, ref.max()))
    with pytest.raises(g.SpgError) as e:
        g.spgemm_bc_batch(dA, torch.tensor([3, A.ncols], dtype=torch.int32))
    assert e.value.status == g.SPG_INVALID_ARGUMENT
