"""Comparison helpers for GPU-vs-oracle parity (shared by the GPU tests)."""
import numpy as np
import torch

import oracle
import paper_2408_14558_gb300 as g

FP64_BOUND = 1e-12   # |c - c_ref| <= 1e-12 * sum |a_rk * b_kj| per entry


def check_values(got, want, absum, where=""):
    if want.dtype.kind in "iu":
        bad = np.flatnonzero(got.astype(np.int64) != want.astype(np.int64))
        assert bad.size == 0, f"{where}: {bad.size} integer values differ, first at {bad[:5]}"
        return
    err = np.abs(got - want)
    bound = FP64_BOUND * absum
    bad = np.flatnonzero(err > bound)
    assert bad.size == 0, (f"{where}: {bad.size} values outside 1e-12*sum|ab|, first {bad[:5]}: "
                           f"got {got[bad[:3]]} want {want[bad[:3]]} bound {bound[bad[:3]]}")


def assert_full_parity(C: "g.DeviceCSC", ref: dict, where=""):
    colptr, rowidx, vals = C.to_host()
    assert np.array_equal(colptr.astype(np.int64), ref["colptr"]), f"{where}: column pointers differ"
    assert np.array_equal(rowidx.astype(np.int64), ref["rowidx"]), f"{where}: row indices differ"
    check_values(vals, ref["vals"], ref["absum"], where)


def assert_sampled_parity(C: "g.DeviceCSC", A, B, cols, where=""):
    """Compare the sampled output columns one by one against the oracle."""
    cols = np.asarray(cols, dtype=np.int64)
    ref = oracle.spgemm(A, B, cols=cols)
    cp = C.colptr.cpu().numpy()
    assert cp[0] == 0 and np.all(np.diff(cp) >= 0), f"{where}: column pointers not monotone"
    for s, j in enumerate(cols):
        a, e = int(cp[j]), int(cp[j + 1])
        ra, re_ = int(ref["colptr"][s]), int(ref["colptr"][s + 1])
        assert e - a == re_ - ra, f"{where}: nnz of column {j}: {e - a} vs {re_ - ra}"
        rows = C.rowidx[a:e].cpu().numpy().astype(np.int64)
        assert np.array_equal(rows, ref["rowidx"][ra:re_]), f"{where}: rows of column {j} differ"
        vals = C.vals[a:e].cpu().numpy()
        check_values(vals, ref["vals"][ra:re_], None if ref["absum"] is None else ref["absum"][ra:re_],
                     f"{where} column {j}")
    return ref


def run_gpu(A, B, P, b, ptr=torch.int32, idx=torch.int32, val=None, **kw):
    dA = g.to_device(A, ptr_dtype=ptr, idx_dtype=idx, val_dtype=val)
    dB = g.to_device(B, ptr_dtype=ptr, idx_dtype=idx, val_dtype=val)
    C = g.multiply(dA, dB, P, b, **kw)
    torch.cuda.synchronize()
    return C


def mask_from_pattern(M, device="cuda", words=None):
    """Output-mask tensor (columns x words int32, bit r of column j's words =
    row r, least significant bit first) whose set bits are the host CSC M's
    pattern."""
    cp = np.asarray(M.colptr, dtype=np.int64)
    ri = np.asarray(M.rowidx, dtype=np.int64)
    W = (int(M.nrows) + 31) // 32 if words is None else int(words)
    bits = np.zeros((int(M.ncols), W), dtype=np.uint32)
    cols = np.repeat(np.arange(int(M.ncols), dtype=np.int64), np.diff(cp))
    np.bitwise_or.at(bits, (cols, ri >> 5), np.left_shift(np.uint32(1), (ri & 31).astype(np.uint32)))
    return torch.from_numpy(bits.view(np.int32)).to(device)
