"""CPU oracle for the sparsity-aware 1D SpGEMM (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  The CUDA path never imports it and it never imports the CUDA
path: the two share no code.  The arithmetic lives in ``spgemm_oracle.c`` (plain
C, double or wrapping int64, dense sparse accumulator per column); this module
only compiles it, converts arrays to int64 / double and calls it.  The MLP oracle
(float64 numpy) lives in ``oracle.mlp``.

Functions and the passages they follow:

* ``spgemm``        -- C = A*B column by column (Section 2 problem statement,
                       Algorithm 1 local multiply), plus S_rj = sum |a_rk b_kj|.
* ``plan_block``    -- H_i, D~_i = H_i AND D, fetch blocks (Algorithm 1 steps on
                       H and D~, Algorithm 2 with fixed-width blocks of b ids).
* ``gather``        -- A~_i = A(:, D~_i) (Algorithm 1, "new sparse matrix").
* ``features``      -- flops_j, nnz(B(:,j)), max / mean nnz(A(:,k)) over
                       k in B(:,j) (Section 3.2 flop count).
* ``spgemm_1d``     -- the whole of Algorithm 1 on one host: per block, plan,
                       gather, and C_i = A~_i * B_i with B_i's rows remapped to
                       A~_i's columns.
* ``block_bounds``  -- column block i is [floor(i*n/P), floor((i+1)*n/P)).
* ``flop_bounds``   -- a contiguous column split with balanced flops (the
                       per-column flop count of Section 3.2 as the weight).
* ``block_volumes`` -- per block: flops, gathered A~ nonzeros, and those of
                       columns outside the block's own column block of A (the
                       communication volume of a distributed run; CV/memA of
                       the Discussion is their mean over nnz(A)).
* ``outer_split``   -- Algorithm 3, first step: B redistributed by row blocks,
                       column (i, j) = the entries of B(:, j) in row block i.
* ``merge_matrix``  -- Algorithm 3, last step written as a product: S with
                       S[i*n + j, j] = 1 sums the partial columns of column j.
* ``outer_volumes`` -- what Algorithm 3 moves between P owners: B entries that
                       change owner, partial-product nonzeros, and partial
                       nonzeros computed away from their column's owner.
* ``spgemm_masked`` -- C<M> = A*B with a structural mask (the masked product
                       of the batched betweenness search, Section 3.2): the
                       entries of A*B whose position M's pattern holds (or,
                       complemented, does not hold).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spgemm_oracle.c")
_SO = os.path.join(_HERE, "_spgemm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_spgemm_oracle.so`` (gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


class _Csc(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64),
                ("colptr", ctypes.c_void_p), ("rowidx", ctypes.c_void_p),
                ("vals", ctypes.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int64
            lib.orc_count.argtypes = [P, P, P, I, P, P, ctypes.c_int]
            lib.orc_fill.argtypes = [P, P, P, I, P, P, P, P, ctypes.c_int, ctypes.c_int]
            lib.orc_plan_block.argtypes = [P, P, I, I, I, P, P, P, P, P, P]
            lib.orc_gather.argtypes = [P, P, I, P, P, P, ctypes.c_int]
            lib.orc_column_features.argtypes = [P, P, I, I, P, P, P]
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().orc_max_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class _Mat:
    """int64/double copies of one CSC matrix, kept alive while C reads them."""

    def __init__(self, M, mode=None):
        self.colptr = np.ascontiguousarray(M.colptr, dtype=np.int64)
        self.rowidx = np.ascontiguousarray(M.rowidx, dtype=np.int64)
        v = np.asarray(M.vals)
        if mode is None:
            mode = 0 if v.dtype.kind == "f" else 1
        self.mode = mode
        self.vals = np.ascontiguousarray(v, dtype=np.float64 if mode == 0 else np.int64)
        self.s = _Csc(int(M.nrows), int(M.ncols), self.colptr.ctypes.data,
                      self.rowidx.ctypes.data, self.vals.ctypes.data)

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _mode_of(A, B):
    fa = np.asarray(A.vals).dtype.kind == "f"
    fb = np.asarray(B.vals).dtype.kind == "f"
    if fa != fb:
        raise ValueError("A and B must both hold floating or both integer values")
    return 0 if fa else 1


def block_bounds(n: int, P: int) -> np.ndarray:
    """Column block i of B and C is [floor(i*n/P), floor((i+1)*n/P))."""
    return np.array([(i * n) // P for i in range(P + 1)], dtype=np.int64)


def spgemm(A, B, cols=None, nthreads: int = 0):
    """C(:, cols) = A * B(:, cols).

    Returns a dict with ``colptr`` (len(cols)+1, int64), ``rowidx`` (int64),
    ``vals`` (double or int64), ``absum`` (double S_rj, or None for integers),
    ``nnz`` and ``flops`` per selected column.
    """
    if A.ncols != B.nrows:
        raise ValueError("inner dimensions differ")
    lib = _load()
    mode = _mode_of(A, B)
    a, b = _Mat(A, mode), _Mat(B, mode)
    cols = np.arange(B.ncols, dtype=np.int64) if cols is None else np.ascontiguousarray(cols, dtype=np.int64)
    ns = cols.shape[0]
    nnz = np.zeros(ns, dtype=np.int64)
    flops = np.zeros(ns, dtype=np.int64)
    rc = lib.orc_count(a.ref, b.ref, _ptr(cols), ns, _ptr(nnz), _ptr(flops), nthreads)
    if rc:
        raise RuntimeError(f"orc_count failed ({rc})")
    colptr = np.zeros(ns + 1, dtype=np.int64)
    np.cumsum(nnz, out=colptr[1:])
    tot = int(colptr[-1])
    rowidx = np.zeros(tot, dtype=np.int64)
    vals = np.zeros(tot, dtype=np.float64 if mode == 0 else np.int64)
    absum = np.zeros(tot, dtype=np.float64) if mode == 0 else None
    rc = lib.orc_fill(a.ref, b.ref, _ptr(cols), ns, _ptr(colptr), _ptr(rowidx), _ptr(vals),
                      _ptr(absum), mode, nthreads)
    if rc:
        raise RuntimeError(f"orc_fill failed ({rc})")
    return {"colptr": colptr, "rowidx": rowidx, "vals": vals, "absum": absum,
            "nnz": nnz, "flops": flops, "nrows": A.nrows, "ncols": ns}


def spgemm_masked(A, B, M, complement: bool = False, cols=None):
    """C<M> = A * B(:, cols) under the structural mask M (a CSC pattern with
    C's shape; values ignored): by definition the unmasked product, then, per
    column j, only the entries whose row r satisfies (r in M(:, j)) != complement.
    Same return layout as ``spgemm``."""
    r = spgemm(A, B, cols=cols)
    cols = np.arange(B.ncols, dtype=np.int64) if cols is None else np.asarray(cols, dtype=np.int64)
    mcp = np.asarray(M.colptr, dtype=np.int64)
    mri = np.asarray(M.rowidx, dtype=np.int64)
    keep = np.zeros(r["rowidx"].shape[0], dtype=bool)
    for s, j in enumerate(cols):
        a, e = int(r["colptr"][s]), int(r["colptr"][s + 1])
        inside = np.isin(r["rowidx"][a:e], mri[mcp[j]:mcp[j + 1]])
        keep[a:e] = inside != bool(complement)
    nnz = np.array([int(keep[r["colptr"][s]:r["colptr"][s + 1]].sum()) for s in range(cols.shape[0])],
                   dtype=np.int64)
    colptr = np.zeros(cols.shape[0] + 1, dtype=np.int64)
    np.cumsum(nnz, out=colptr[1:])
    return {"colptr": colptr, "rowidx": r["rowidx"][keep], "vals": r["vals"][keep],
            "absum": None if r["absum"] is None else r["absum"][keep], "nnz": nnz, "flops": r["flops"],
            "nrows": r["nrows"], "ncols": r["ncols"]}


def plan_block(A, B, c0: int, c1: int, b: int):
    """Planning quantities of Algorithm 1 / Algorithm 2 for B(:, c0:c1)."""
    lib = _load()
    a, bb = _Mat(A), _Mat(B)
    k = int(B.nrows)
    H = np.zeros(k, dtype=np.uint8)
    dt = np.zeros(max(k, 1), dtype=np.int64)
    nd = ctypes.c_int64(0)
    nblk = (k + b - 1) // b
    fetch = np.zeros(max(nblk, 1), dtype=np.uint8)
    ve, vb = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = lib.orc_plan_block(a.ref, bb.ref, c0, c1, b, _ptr(H), _ptr(dt), ctypes.byref(nd),
                            _ptr(fetch), ctypes.byref(ve), ctypes.byref(vb))
    if rc:
        raise RuntimeError(f"orc_plan_block failed ({rc})")
    fetch = fetch[:nblk]
    chosen = np.flatnonzero(fetch)
    intervals = np.stack([chosen * b, np.minimum((chosen + 1) * b, k) - 1], axis=1) if chosen.size else np.zeros((0, 2), np.int64)
    return {"H": H, "dtilde": dt[: nd.value].copy(), "fetch": fetch, "intervals": intervals,
            "vol_exact": ve.value, "vol_block": vb.value}


def gather(A, dtilde):
    """A~ = A(:, dtilde) as a dict(colptr, rowidx, vals, nrows, ncols)."""
    lib = _load()
    a = _Mat(A)
    dtilde = np.ascontiguousarray(dtilde, dtype=np.int64)
    nd = dtilde.shape[0]
    vol = int(np.sum(a.colptr[dtilde + 1] - a.colptr[dtilde])) if nd else 0
    colptr = np.zeros(nd + 1, dtype=np.int64)
    rowidx = np.zeros(vol, dtype=np.int64)
    vals = np.zeros(vol, dtype=a.vals.dtype)
    lib.orc_gather(a.ref, _ptr(dtilde), nd, _ptr(colptr), _ptr(rowidx), _ptr(vals), 8)
    return {"colptr": colptr, "rowidx": rowidx, "vals": vals, "nrows": A.nrows, "ncols": nd}


def features(A, B, c0: int = 0, c1: int | None = None):
    """Per-column features of B(:, c0:c1): flops, nnz(B(:,j)), max nnz(A(:,k)),
    mean nnz(A(:,k)) over the stored k of B(:,j) (0 for an empty column)."""
    lib = _load()
    c1 = B.ncols if c1 is None else c1
    a, bb = _Mat(A), _Mat(B)
    n = c1 - c0
    fl = np.zeros(n, dtype=np.int64)
    nb = np.zeros(n, dtype=np.int64)
    mx = np.zeros(n, dtype=np.int64)
    lib.orc_column_features(a.ref, bb.ref, c0, c1, _ptr(fl), _ptr(nb), _ptr(mx))
    mean = np.where(nb > 0, fl / np.maximum(nb, 1), 0.0)
    return {"flops": fl, "nnzb": nb, "maxa": mx, "meana": mean}


class _View:
    def __init__(self, nrows, ncols, colptr, rowidx, vals):
        self.nrows, self.ncols = nrows, ncols
        self.colptr, self.rowidx, self.vals = colptr, rowidx, vals


def spgemm_1d(A, B, P: int, b: int, nthreads: int = 0, bounds=None):
    """Algorithm 1 on one host.  For every block i: H_i, D~_i, fetch blocks,
    A~_i = A(:, D~_i), and C_i = A~_i * B_i where row k of B_i addresses column
    map[k] of A~_i (entries of B_i on rows outside D~_i meet an empty column of
    A and contribute no product).  C is the concatenation of the C_i.  The
    column blocks are block_bounds(n, P) unless ``bounds`` (P + 1 ascending
    column ids from 0 to n) is given.
    Returns (C dict, list of per-block plan dicts)."""
    if A.ncols != B.nrows:
        raise ValueError("inner dimensions differ")
    bounds = block_bounds(B.ncols, P) if bounds is None else np.asarray(bounds, dtype=np.int64)
    k = int(B.nrows)
    parts, plans = [], []
    Bcp = np.asarray(B.colptr, dtype=np.int64)
    Brow = np.asarray(B.rowidx, dtype=np.int64)
    Bval = np.asarray(B.vals)
    for i in range(P):
        c0, c1 = int(bounds[i]), int(bounds[i + 1])
        pl = plan_block(A, B, c0, c1, b)
        At = gather(A, pl["dtilde"])
        cmap = np.full(k, -1, dtype=np.int64)
        cmap[pl["dtilde"]] = np.arange(pl["dtilde"].shape[0], dtype=np.int64)
        s, e = int(Bcp[c0]), int(Bcp[c1])
        q = cmap[Brow[s:e]]
        keep = q >= 0
        colid = np.repeat(np.arange(c1 - c0), np.diff(Bcp[c0:c1 + 1]))
        cnt = np.bincount(colid[keep], minlength=c1 - c0)
        bcp = np.zeros(c1 - c0 + 1, dtype=np.int64)
        np.cumsum(cnt, out=bcp[1:])
        Bi = _View(At["ncols"], c1 - c0, bcp, q[keep], Bval[s:e][keep])
        Ai = _View(A.nrows, At["ncols"], At["colptr"], At["rowidx"], At["vals"])
        Ci = spgemm(Ai, Bi, nthreads=nthreads)
        pl["Atilde"] = At
        pl["flops"] = Ci["flops"]
        pl["nnz"] = Ci["nnz"]
        plans.append(pl)
        parts.append(Ci)
    colptr = np.zeros(B.ncols + 1, dtype=np.int64)
    np.cumsum(np.concatenate([p["nnz"] for p in parts]) if parts else np.zeros(0, np.int64), out=colptr[1:])
    mode = _mode_of(A, B)
    C = {"colptr": colptr,
         "rowidx": np.concatenate([p["rowidx"] for p in parts]) if parts else np.zeros(0, np.int64),
         "vals": np.concatenate([p["vals"] for p in parts]) if parts else np.zeros(0, np.float64 if mode == 0 else np.int64),
         "absum": np.concatenate([p["absum"] for p in parts]) if mode == 0 and parts else None,
         "nrows": A.nrows, "ncols": B.ncols}
    return C, plans


def outer_split(B, P: int):
    """Algorithm 3, "redistribute B so that p_i owns the i-th row block": the
    k x (P*n) matrix whose column i*n + j holds the entries of B(:, j) with
    row in [floor(i*k/P), floor((i+1)*k/P)), rows and values unchanged."""
    k, n = int(B.nrows), int(B.ncols)
    rb = block_bounds(k, P)
    cp = np.asarray(B.colptr, dtype=np.int64)
    rows = np.asarray(B.rowidx, dtype=np.int64)
    vals = np.asarray(B.vals)
    col = np.repeat(np.arange(n, dtype=np.int64), np.diff(cp))
    blk = np.searchsorted(rb, rows, side="right") - 1
    key = blk * n + col
    order = np.argsort(key, kind="stable")
    colptr = np.zeros(P * n + 1, dtype=np.int64)
    np.cumsum(np.bincount(key, minlength=P * n), out=colptr[1:])
    return _View(k, P * n, colptr, rows[order], vals[order])


def merge_matrix(n: int, P: int, integer: bool = False):
    """The (P*n) x n matrix S with S[i*n + j, j] = 1: (A * outer_split(B)) * S
    adds up the P partial columns of every output column (Algorithm 3, "merge
    results")."""
    colptr = np.arange(n + 1, dtype=np.int64) * P
    rows = (np.arange(P, dtype=np.int64)[None, :] * n + np.arange(n, dtype=np.int64)[:, None]).reshape(-1)
    vals = np.ones(P * n, dtype=np.int64 if integer else np.float64)
    return _View(P * n, n, colptr, rows, vals)


def outer_volumes(A, B, P: int):
    """Volumes of Algorithm 3 among P owners, process i owning column block i
    of A, B and C (the distribution of Algorithm 1): ``b_moved`` = entries of
    B whose row block differs from their column block; ``partial_nnz`` =
    sum over i of nnz(A(:, K_i) * B(K_i, :)); ``partial_moved`` = the partial
    nonzeros of column j computed by a process i that is not j's owner.
    Plain loops over the entries; for small inputs."""
    k, n = int(B.nrows), int(B.ncols)
    rb = block_bounds(k, P)
    cb = block_bounds(n, P)
    rblock = lambda r: int(np.searchsorted(rb, r, side="right") - 1)
    cblock = lambda j: int(np.searchsorted(cb, j, side="right") - 1)
    cp = np.asarray(B.colptr, dtype=np.int64)
    rows = np.asarray(B.rowidx, dtype=np.int64)
    b_moved = 0
    for j in range(n):
        for e in range(int(cp[j]), int(cp[j + 1])):
            b_moved += rblock(int(rows[e])) != cblock(j)
    acp = np.asarray(A.colptr, dtype=np.int64)
    arow = np.asarray(A.rowidx, dtype=np.int64)
    partial_nnz = partial_moved = 0
    for j in range(n):
        per_block = {}
        for e in range(int(cp[j]), int(cp[j + 1])):
            kk = int(rows[e])
            per_block.setdefault(rblock(kk), set()).update(arow[acp[kk]:acp[kk + 1]].tolist())
        for i, rset in per_block.items():
            partial_nnz += len(rset)
            partial_moved += len(rset) if i != cblock(j) else 0
    return {"b_moved": b_moved, "partial_nnz": partial_nnz, "partial_moved": partial_moved}


def flop_bounds(A, B, P: int) -> np.ndarray:
    """Contiguous column blocks with balanced flops: bound_0 = 0, bound_P = n,
    and for 0 < i < P bound_i is the smallest j whose preceding columns hold
    at least i/P of the total flops F (P * prefix_j >= i * F in integers)."""
    fl = features(A, B)["flops"].astype(np.int64)
    n = int(B.ncols)
    pre = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(fl, out=pre[1:])
    F = int(pre[-1])
    out = np.zeros(P + 1, dtype=np.int64)
    for i in range(1, P):
        j = 0
        while j < n and P * int(pre[j]) < i * F:
            j += 1
        out[i] = j
    out[P] = n
    return out


def block_volumes(A, B, bounds, b: int = 1024):
    """Per column block [bounds[i], bounds[i+1]): flops, the nonzeros of
    A~_i = A(:, D~_i), and those among them whose column lies outside the
    block's own column block [floor(i*k/P), floor((i+1)*k/P)) of A."""
    bounds = np.asarray(bounds, dtype=np.int64)
    P = bounds.shape[0] - 1
    own = block_bounds(int(A.ncols), P)
    acp = np.asarray(A.colptr, dtype=np.int64)
    flops, gathered, remote = [], [], []
    for i in range(P):
        c0, c1 = int(bounds[i]), int(bounds[i + 1])
        pl = plan_block(A, B, c0, c1, b)
        dt = pl["dtilde"]
        ln = acp[dt + 1] - acp[dt]
        away = (dt < own[i]) | (dt >= own[i + 1])
        flops.append(int(features(A, B, c0, c1)["flops"].sum()))
        gathered.append(int(ln.sum()))
        remote.append(int(ln[away].sum()))
    return {"flops": np.array(flops, np.int64), "gathered": np.array(gathered, np.int64),
            "remote": np.array(remote, np.int64)}
