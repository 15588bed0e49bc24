"""Training data and training of the nnz-prediction model, through the C ABI.

    X, y = column_data(dA, dB)            # features and log1p(nnz) of every column of A*B
    model = spgemm_model_create(seed)
    spgemm_model_train(model, X, y, ...)   # the library's forward/backward/Adam kernels
    C, status = spgemm_1d_multiply(dA, dB, P, b, sizing=SPG_SIZING_LEARNED, model=model)

`train_default_model` builds the training set the way the library's model file
is made: squares C = A*A of seeded ER and R-MAT-row instances (n log-uniform
in [2^14, 2^18], 4..32 nonzeros per column), every column one sample.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import (SPG_SIZING_LEARNED, spgemm_model_create, spgemm_model_save, spgemm_model_train, spgemm_plan,
               spgemm_plan_destroy, spgemm_plan_features, spgemm_plan_labels, spgemm_symbolic, to_device)


def column_data(dA, dB, P: int = 1, b: int = 1024):
    """(X, y) of every output column of A*B: X = the 4 log1p features, y =
    log1p(nnz(C(:,j))) from the exact symbolic pass."""
    plan = spgemm_plan(dA, dB, P, b)
    try:
        spgemm_symbolic(plan)
        X = spgemm_plan_features(plan).clone()
        y = spgemm_plan_labels(plan).clone()
    finally:
        spgemm_plan_destroy(plan)
    return X, y


def training_instances(count: int = 200, seed: int = 1234, nmin: int = 1 << 14, nmax: int = 1 << 18):
    """Seeded square instances for training, half of each kind: ER (n
    log-uniform in [nmin, nmax], 4..32 uniform rows per column) and R-MAT
    graphs (scale uniform in [log2 nmin, log2 nmax], edge factor 4..16,
    self-loops dropped, symmetrised), whose squares compress far more."""
    import synth
    rng = np.random.default_rng(seed)
    lo, hi = int(round(math.log2(nmin))), int(round(math.log2(nmax)))
    for _ in range(count):
        if rng.random() < 0.5:
            n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
            yield synth.random_instance(n, int(rng.integers(4, 33)), "er", rng)
        else:
            yield synth.rmat_symmetric(int(rng.integers(lo, hi + 1)), int(rng.integers(4, 17)),
                                       seed=int(rng.integers(0, 2 ** 31)))


def training_set(instances, device="cuda"):
    Xs, ys = [], []
    for A in instances:
        dA = to_device(A, ptr_dtype=torch.int32, idx_dtype=torch.int32, device=device)
        X, y = column_data(dA, dA)
        keep = y > 0                      # empty output columns carry no information
        Xs.append(X[keep])
        ys.append(y[keep])
    X = torch.cat(Xs)
    y = torch.cat(ys)
    g = torch.Generator(device="cpu").manual_seed(0)
    perm = torch.randperm(y.numel(), generator=g).to(y.device)
    return X[perm].contiguous(), y[perm].contiguous()


def train_default_model(path: str | None = None, count: int = 200, epochs: int = 8, batch: int = 4096,
                        lr: float = 2e-3, seed: int = 7):
    X, y = training_set(training_instances(count))
    model = spgemm_model_create(seed)
    loss = spgemm_model_train(model, X, y, epochs=epochs, batch=batch, lr=lr)
    if path:
        spgemm_model_save(model, path)
    return model, loss, int(y.numel())


__all__ = ["column_data", "training_instances", "training_set", "train_default_model", "SPG_SIZING_LEARNED",
           "DEFAULT_MODEL"]

import os as _os

DEFAULT_MODEL = _os.path.join(_os.path.dirname(_os.path.abspath(__file__)), "models", "nnz_mlp.bin")

if __name__ == "__main__":
    import sys
    import time
    out = sys.argv[1] if len(sys.argv) > 1 else DEFAULT_MODEL
    _os.makedirs(_os.path.dirname(out), exist_ok=True)
    t0 = time.time()
    model, loss, nsamples = train_default_model(out)
    print(f"trained on {nsamples} columns of 200 instances in {time.time() - t0:.1f} s, final MSE {loss:.4f} -> {out}")
