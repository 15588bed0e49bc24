"""Repeated products with fixed patterns: spgemm_numeric_refresh and its
captured CUDA graph give the oracle's product for new values of A and B."""
import numpy as np
import pytest
import torch

import oracle
import paper_2408_14558_gb300 as g
import synth
from parity import assert_full_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("light_max,slab", [(1024, 4096), (32, 1024)])
@pytest.mark.parametrize("vals", ["f64", "i64"])
def test_refresh_and_graph_replay(light_max, slab, vals):
    rng = np.random.default_rng(light_max + len(vals))
    kind = "f64" if vals == "f64" else "i64big"
    A = synth.random_sparse(3000, 700, 0.01, rng, values=kind)
    B = synth.random_sparse(700, 600, 0.04, rng, values=kind)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        dA, dB = g.to_device(A), g.to_device(B)
        plan = g.spgemm_plan(dA, dB, 4, 64, light_max=light_max, slab_rows=slab)
        g.spgemm_symbolic(plan)
        C = g.spgemm_numeric(plan)
        s.synchronize()
        assert_full_parity(C, oracle.spgemm(A, B), "first")
        for step in range(2):
            draw = (lambda k: rng.uniform(-1, 1, k)) if vals == "f64" else (lambda k: rng.integers(-2**40, 2**40, k))
            A2 = synth.CSC(A.nrows, A.ncols, A.colptr, A.rowidx, draw(A.nnz))
            B2 = synth.CSC(B.nrows, B.ncols, B.colptr, B.rowidx, draw(B.nnz))
            dA.vals.copy_(torch.from_numpy(np.asarray(A2.vals)))
            dB.vals.copy_(torch.from_numpy(np.asarray(B2.vals)))
            if step == 0:
                g.spgemm_numeric_refresh(plan, C)
            else:
                g.spgemm_plan_capture(plan, C)
                C.vals.zero_()
                g.spgemm_plan_replay(plan)
            s.synchronize()
            assert_full_parity(C, oracle.spgemm(A2, B2), f"step {step}")
        g.spgemm_plan_destroy(plan)


def test_refresh_needs_a_numeric_pass():
    rng = np.random.default_rng(1)
    A = synth.random_sparse(50, 40, 0.1, rng)
    B = synth.random_sparse(40, 30, 0.1, rng)
    plan = g.spgemm_plan(g.to_device(A), g.to_device(B), 2, 8)
    g.spgemm_symbolic(plan)
    C = g.DeviceCSC(50, 30, plan.colptr, torch.empty(plan.nnzC, dtype=torch.int32, device="cuda"),
                    torch.empty(plan.nnzC, dtype=torch.float64, device="cuda"))
    with pytest.raises(g.SpgError) as e:
        g.spgemm_numeric_refresh(plan, C)
    assert e.value.status == g.SPG_INVALID_ARGUMENT
    with pytest.raises(g.SpgError):
        g.spgemm_plan_replay(plan)
    g.spgemm_plan_destroy(plan)
