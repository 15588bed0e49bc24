"""Learned nnz sizing on the GPU: the library's MLP kernels against the float64
oracle, training, and the learned multiply against the exact one."""
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
import paper_2408_14558_gb300 as g
from paper_2408_14558_gb300 import learned
import synth
from parity import assert_full_parity

pytestmark = pytest.mark.gpu


def rand_params(rng, scale=0.3):
    return (rng.normal(0, scale, mlp.NPARAMS)).astype(np.float32)


def test_forward_matches_oracle():
    rng = np.random.default_rng(0)
    theta = rand_params(rng)
    model = g.spgemm_model_create(1)
    g.spgemm_model_set_params(model, theta)
    X = rng.normal(0, 2, (1000, 4)).astype(np.float32)
    got = g.spgemm_model_predict(model, torch.from_numpy(X).cuda()).cpu().numpy()
    want, _ = mlp.forward(theta.astype(np.float64), X.astype(np.float64))
    assert np.allclose(got, want, rtol=1e-4, atol=1e-4 * np.abs(want).max())


def test_gradient_matches_oracle():
    rng = np.random.default_rng(1)
    theta = rand_params(rng)
    model = g.spgemm_model_create(1)
    g.spgemm_model_set_params(model, theta)
    X = rng.normal(0, 1.5, (3000, 4)).astype(np.float32)
    t = rng.normal(0, 1, 3000).astype(np.float32)
    got, loss = g.spgemm_model_gradient(model, torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
    want, wloss = mlp.gradient(theta.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    scale = np.abs(want).max()
    assert np.allclose(got, want, rtol=1e-4, atol=1e-4 * scale), np.abs(got - want).max() / scale
    assert abs(loss - wloss) <= 1e-4 * wloss


def test_one_adam_step_matches_oracle():
    rng = np.random.default_rng(2)
    theta = rand_params(rng)
    model = g.spgemm_model_create(1)
    g.spgemm_model_set_params(model, theta)
    X = rng.normal(0, 1, (512, 4)).astype(np.float32)
    t = rng.normal(0, 1, 512).astype(np.float32)
    g.spgemm_model_train(model, torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), epochs=1, batch=512, lr=1e-2)
    got = g.spgemm_model_get_params(model)
    grad, _ = mlp.gradient(theta.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    want, _, _ = mlp.adam_step(theta.astype(np.float64), grad, np.zeros(mlp.NPARAMS), np.zeros(mlp.NPARAMS), 1, 1e-2)
    # the first step moves every parameter by ~lr * sign(g): compare to 1e-4 of lr
    assert np.allclose(got, want, atol=1e-4 * 1e-2 + 1e-6)


def test_features_and_labels_match_oracle():
    A = synth.rmat_symmetric(10, 8, seed=3)
    dA = g.to_device(A)
    X, y = learned.column_data(dA, dA)
    f = oracle.features(A, A)
    C = oracle.spgemm(A, A)
    want_X = mlp.features(f["flops"], f["nnzb"], f["maxa"])
    assert np.allclose(X.cpu().numpy(), want_X, rtol=1e-6, atol=1e-6)
    assert np.allclose(y.cpu().numpy(), np.log1p(C["nnz"]), rtol=1e-6)


def small_training_set():
    return learned.training_set(learned.training_instances(count=12, nmin=1 << 11, nmax=1 << 14, seed=5))


@pytest.fixture(scope="module")
def trained():
    X, y = small_training_set()
    model = g.spgemm_model_create(7)
    l0 = g.spgemm_model_gradient(model, X, y)[1]
    l1 = g.spgemm_model_train(model, X, y, epochs=30, batch=2048, lr=3e-3)
    return model, l0, l1


def test_training_reduces_loss(trained):
    model, l0, l1 = trained
    assert l1 < 0.1 * l0 and l1 < 0.2, (l0, l1)


def test_save_load_roundtrip(trained, tmp_path):
    model = trained[0]
    path = str(tmp_path / "m.bin")
    g.spgemm_model_save(model, path)
    m2 = g.spgemm_model_load(path)
    assert np.array_equal(g.spgemm_model_get_params(m2), g.spgemm_model_get_params(model))


def learned_vs_exact(A, B, model, slack, P=4, b=256, **kw):
    dA, dB = g.to_device(A), g.to_device(B)
    Ce, _ = g.spgemm_1d_multiply(dA, dB, P=P, b=b, **kw)
    Cl, st = g.spgemm_1d_multiply(dA, dB, P=P, b=b, sizing=g.SPG_SIZING_LEARNED, model=model, learned_slack=slack,
                                  **kw)
    stats = g.spgemm_last_multiply_stats()
    torch.cuda.synchronize()
    # the fused pass's output entries: none without heavy columns, never more than C
    assert 0 <= stats["nnzC_heavy"] <= stats["nnzC"]
    if stats["heavy_columns"] == 0:
        assert stats["nnzC_heavy"] == 0
    assert torch.equal(Cl.colptr, Ce.colptr)
    assert torch.equal(Cl.rowidx, Ce.rowidx)
    if Cl.vals.dtype == torch.int64:
        assert torch.equal(Cl.vals, Ce.vals)
    return Cl, st, stats


@pytest.mark.parametrize("slack", [1.25, 1e-3, 100.0])
def test_learned_multiply_equals_exact(trained, slack):
    model = trained[0]
    cases = [
        (synth.rmat_symmetric(13, 16, seed=2), None, {"light_max": 256, "slab_rows": 1024}),
        (synth.rmat_symmetric(13, 16, seed=2, values="i64"), None, {}),
        (synth.uniform_columns(4000, 8, seed=3), None, {}),
    ]
    Az, Azt = synth.lognormal_zipf_rows(nrows=2000, ncols=1 << 15, mean=40, cap=300, seed=6)
    cases.append((Az.astype(val=np.int64), Azt.astype(val=np.int64), {"light_max": 512, "slab_rows": 2048}))
    for A, B, kw in cases:
        B = A if B is None else B
        Cl, st, stats = learned_vs_exact(A, B, model, slack, **kw)
        if slack == 1e-3:
            # capacity 1 per column: every column holding more than one entry overflows
            assert st == g.SPG_OVERFLOW_RECOMPUTED and stats["recomputed_columns"] > 0
        if A.vals.dtype.kind == "f":
            ref = oracle.spgemm(A, B)
            assert_full_parity(Cl, ref, f"learned slack={slack}")


def test_trained_model_gain(trained):
    """On a held-out instance the trained network sizes the columns to within
    a small factor of the true nnz with few recomputes; the method without it
    has to size from the exact bound (flops), far above nnz, or run the
    symbolic pass."""
    model = trained[0]
    A = synth.rmat_symmetric(12, 16, seed=5)        # held out: nnz(C) is about 1/4 of the products
    C, st, stats = learned_vs_exact(A, A, model, 1.25, P=4, b=1024)
    nnz = int(C.colptr[-1])
    products = stats["products"]
    cap = stats["learned_capacity"]
    rec = stats["recomputed_columns"] / A.ncols
    assert cap < 0.6 * products, (cap, products, nnz)
    assert cap < 3.0 * nnz and rec <= 0.15, (cap, nnz, rec)
    # an untrained network sizes worse: more recomputes or far more room
    raw = g.spgemm_model_create(123)
    C2, st2, stats2 = learned_vs_exact(A, A, raw, 1.25, P=4, b=1024)
    worse = stats2["recomputed_columns"] / A.ncols > rec + 0.05 or stats2["learned_capacity"] > 1.5 * cap
    assert worse, (stats2["recomputed_columns"], stats2["learned_capacity"], rec, cap)
