"""GPU parity of the outer-product 1D SpGEMM (Algorithm 3) against the CPU
oracle: the result equals A*B (structure and integers bit-exact, doubles
within 1e-12 * sum |a_rk * b_kj|), and the volumes it reports equal the
oracle's enumeration."""
import numpy as np
import pytest
import torch

import oracle
import paper_2408_14558_gb300 as g
import synth
from parity import assert_full_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("P", [1, 2, 3, 7, 64])
@pytest.mark.parametrize("vals", ["f64", "i32", "i64"])
def test_outer_random_small(P, vals):
    rng = np.random.default_rng(P * 7 + len(vals))
    kind = vals if vals != "i64" else "i64big"
    A = synth.random_sparse(300, 257, 0.03, rng, values=kind)
    B = synth.random_sparse(257, 203, 0.03, rng, values=kind)
    ref = oracle.spgemm(A, B)
    C, st = g.spgemm_outer_multiply(g.to_device(A), g.to_device(B), P, 16)
    torch.cuda.synchronize()
    assert_full_parity(C, ref, f"outer P={P} {vals}")
    assert st["nnzC"] == int(ref["colptr"][-1])
    assert st["products"] == int(ref["flops"].sum())


@pytest.mark.parametrize("P", [2, 5])
def test_outer_volumes_match_oracle(P):
    rng = np.random.default_rng(40 + P)
    A = synth.random_sparse(60, 70, 0.08, rng, values="f64")
    B = synth.random_sparse(70, 50, 0.08, rng, values="f64")
    _, st = g.spgemm_outer_multiply(g.to_device(A), g.to_device(B), P, 8)
    v = oracle.outer_volumes(A, B, P)
    assert st["nnzB_moved"] == v["b_moved"]
    assert st["partial_nnz"] == v["partial_nnz"]
    assert st["partial_moved"] == v["partial_moved"]
    part = oracle.spgemm(A, oracle.outer_split(B, P))
    assert st["partial_nnz"] == int(part["colptr"][-1])


def test_outer_galerkin_right_product():
    """The paper's use: (R^T A) R with R the 2x2x2 aggregation of a 7-point
    grid (N = 32), against the oracle; P = 8 row blocks."""
    N = 32
    A = synth.poisson3d(N)
    R = synth.aggregation_2x2x2(N)
    RT = synth.aggregation_2x2x2_transpose(N)
    dRtA = g.multiply(g.to_device(RT), g.to_device(A), 8, 512)
    rta = oracle.spgemm(RT, A)
    assert_full_parity(dRtA, rta, "R^T A")
    C, st = g.spgemm_outer_multiply(dRtA, g.to_device(R), 8, 512)
    torch.cuda.synchronize()
    RtA = synth.CSC(rta["nrows"], rta["ncols"], rta["colptr"], rta["rowidx"], rta["vals"])
    ref = oracle.spgemm(RtA, R)
    assert_full_parity(C, ref, "(R^T A) R")
    M = N // 2
    assert int(C.colptr[-1]) == 7 * M ** 3 - 6 * M ** 2


def test_outer_edge_cases():
    """Empty columns of B, more row blocks than rows, and an empty B."""
    rng = np.random.default_rng(9)
    A = synth.random_sparse(40, 12, 0.3, rng, values="i64")
    B0 = synth.random_sparse(12, 30, 0.3, rng, values="i64")
    col = np.repeat(np.arange(30), np.diff(B0.colptr))
    keep = (col < 10) | (col >= 16)                     # columns 10..15 empty
    cnt = np.bincount(col[keep], minlength=30)
    B = synth.CSC(12, 30, np.concatenate([[0], np.cumsum(cnt)]).astype(B0.colptr.dtype), B0.rowidx[keep],
                  B0.vals[keep])
    ref = oracle.spgemm(A, B)
    for P in (1, 12, 40):
        C, _ = g.spgemm_outer_multiply(g.to_device(A), g.to_device(B), P, 4)
        torch.cuda.synchronize()
        assert_full_parity(C, ref, f"edge P={P}")
    E = synth.CSC(12, 5, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int64))
    C, st = g.spgemm_outer_multiply(g.to_device(A), g.to_device(E), 3, 4)
    torch.cuda.synchronize()
    assert int(C.colptr[-1]) == 0 and C.ncols == 5 and st["nnzC"] == 0
