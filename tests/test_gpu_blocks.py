"""GPU parity of the column-block split and the per-block diagnostics: the
flop-balanced bounds, per-block flops, gathered and remote A~ nonzeros equal
the oracle's, and the product is unchanged by the split."""
import numpy as np
import pytest
import torch

import oracle
import paper_2408_14558_gb300 as g
import synth
from parity import assert_full_parity

pytestmark = pytest.mark.gpu


def skewed(rng, m, n, k):
    """Columns of B with lengths growing along j (a skewed flop profile)."""
    A = synth.random_sparse(m, k, 0.05, rng, values="f64")
    dens = np.linspace(0.005, 0.3, n)
    mask = rng.random((k, n)) < dens[None, :]
    cols, rows = np.nonzero(mask.T)          # sorted by column, then row
    B = synth._csc_from_sorted(k, n, cols.astype(np.int64), rows.astype(np.int64), rng.uniform(-1, 1, rows.size))
    return A, B


@pytest.mark.parametrize("P,b", [(4, 16), (7, 5), (1, 64)])
@pytest.mark.parametrize("split", [g.SPG_SPLIT_UNIFORM, g.SPG_SPLIT_FLOPS])
def test_split_and_block_volumes(P, b, split):
    rng = np.random.default_rng(P * 10 + split)
    A, B = skewed(rng, 300, 160, 200)
    dA, dB = g.to_device(A), g.to_device(B)
    plan = g.spgemm_plan(dA, dB, P, b, split=split)
    blk = g.spgemm_plan_blocks(plan)
    want = oracle.flop_bounds(A, B, P) if split == g.SPG_SPLIT_FLOPS else oracle.block_bounds(B.ncols, P)
    assert np.array_equal(blk["bounds"], want)
    vol = oracle.block_volumes(A, B, want, b)
    assert np.array_equal(blk["flops"], vol["flops"])
    assert np.array_equal(blk["gathered"], vol["gathered"])
    assert np.array_equal(blk["remote"], vol["remote"])
    st = g.spgemm_plan_stats(plan)
    assert st["gathered_nnz_remote"] == int(vol["remote"].sum())
    assert abs(blk["cv_mem_a"] - vol["remote"].mean() / A.rowidx.size) < 1e-12
    g.spgemm_symbolic(plan)
    C = g.spgemm_numeric(plan)
    g.spgemm_plan_destroy(plan)
    torch.cuda.synchronize()
    assert_full_parity(C, oracle.spgemm(A, B), f"split={split} P={P}")


def test_flop_split_balances_a_skewed_profile():
    """On the skewed profile the flop split's largest block is well below the
    uniform split's, and the blocks' phases still match the oracle."""
    rng = np.random.default_rng(3)
    A, B = skewed(rng, 400, 240, 300)
    dA, dB = g.to_device(A), g.to_device(B)
    P = 8
    mx = {}
    for split in (g.SPG_SPLIT_UNIFORM, g.SPG_SPLIT_FLOPS):
        plan = g.spgemm_plan(dA, dB, P, 32, split=split)
        blk = g.spgemm_plan_blocks(plan)
        mx[split] = blk["flops"].max() / max(blk["flops"].mean(), 1)
        bounds = blk["bounds"]
        for i in range(P):
            ex = g.spgemm_plan_export(plan, i)
            pl = oracle.plan_block(A, B, int(bounds[i]), int(bounds[i + 1]), 32)
            assert np.array_equal(ex["dtilde"].cpu().numpy(), pl["dtilde"])
            f = oracle.features(A, B, int(bounds[i]), int(bounds[i + 1]))
            assert np.array_equal(ex["flops"].cpu().numpy(), f["flops"])
        g.spgemm_plan_destroy(plan)
    assert mx[g.SPG_SPLIT_FLOPS] < 0.8 * mx[g.SPG_SPLIT_UNIFORM]
    assert mx[g.SPG_SPLIT_FLOPS] < 1.25


def test_more_blocks_than_columns_with_flop_split():
    rng = np.random.default_rng(5)
    A = synth.random_sparse(50, 40, 0.1, rng, values="i64")
    B = synth.random_sparse(40, 9, 0.2, rng, values="i64")
    C = g.multiply(g.to_device(A), g.to_device(B), 20, 8, split=g.SPG_SPLIT_FLOPS)
    torch.cuda.synchronize()
    assert_full_parity(C, oracle.spgemm(A, B), "P > n, flop split")
