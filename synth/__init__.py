"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only draws and lays out input matrices (compressed sparse column, CSC).
It holds none of the SpGEMM arithmetic: no products, no accumulation, no
nonzero-row projection, no fetch-block logic. Every generator is a pure function
of its arguments and a seed (numpy PCG64), so the CPU oracle and the CUDA path
see the same bytes within one process, on any host.

The shapes and value distributions stand in for the paper's SuiteSparse and MIS-2
inputs (Section 4, Tables 2 and 3), which are not available:

* ``uniform_columns``   -- every column has exactly ``d`` distinct uniformly random
  rows (the "sparsest random" case the paper names as worst for 1D, Section 2.1).
* ``rmat_symmetric``    -- R-MAT graph, self-loops dropped, duplicates merged,
  symmetrised: a skewed-degree squaring input (Section 4.1).
* ``poisson3d`` / ``aggregation_2x2x2`` -- a 7-point Laplacian and a restriction
  operator with exactly one nonzero per row (Table 3's property), the AMG
  Galerkin inputs of Section 2.3.
* ``lognormal_zipf_rows`` -- rectangular similarity-style input with lognormal row
  lengths and Zipf column popularity.
* ``random_instance``   -- ER or R-MAT-row square instances with a per-matrix
  nonzeros-per-column count, used for batches and MLP training data.
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np

__all__ = [
    "CSC", "from_dense", "uniform_columns", "rmat_symmetric", "poisson3d",
    "aggregation_2x2x2", "aggregation_2x2x2_transpose", "lognormal_zipf_rows",
    "random_instance", "batch_instances", "fig1_example", "random_sparse",
]


@dataclass
class CSC:
    """A sparse matrix in compressed sparse column form.

    ``colptr`` has ``ncols + 1`` entries; column ``j`` holds rows
    ``rowidx[colptr[j]:colptr[j+1]]`` (strictly increasing) with values
    ``vals[...]`` at the same positions.
    """
    nrows: int
    ncols: int
    colptr: np.ndarray
    rowidx: np.ndarray
    vals: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    def astype(self, ptr=None, idx=None, val=None) -> "CSC":
        return CSC(self.nrows, self.ncols,
                   self.colptr.astype(ptr) if ptr is not None else self.colptr,
                   self.rowidx.astype(idx) if idx is not None else self.rowidx,
                   self.vals.astype(val) if val is not None else self.vals)

    def col(self, j: int):
        s, e = int(self.colptr[j]), int(self.colptr[j + 1])
        return self.rowidx[s:e], self.vals[s:e]


def _csc_from_sorted(nrows, ncols, cols, rows, vals, idx_dtype=np.int32) -> CSC:
    """Entries must already be sorted by (col, row) and free of duplicates."""
    counts = np.bincount(cols, minlength=ncols).astype(np.int64)
    colptr = np.zeros(ncols + 1, dtype=np.int64)
    np.cumsum(counts, out=colptr[1:])
    return CSC(int(nrows), int(ncols), colptr, rows.astype(idx_dtype), vals)


def _sort_dedup(cols, rows, nrows):
    key = cols.astype(np.int64) * np.int64(nrows) + rows.astype(np.int64)
    key = np.unique(key)
    return key // nrows, key % nrows


def from_dense(M: np.ndarray, idx_dtype=np.int32) -> CSC:
    """CSC of the nonzero entries of a dense 2-D array (column-major walk)."""
    M = np.asarray(M)
    cols, rows = np.nonzero(M.T)
    return _csc_from_sorted(M.shape[0], M.shape[1], cols, rows, M[rows, cols].copy(), idx_dtype)


def _distinct_rows(rng, d_per_col: np.ndarray, sampler, max_rounds=500):
    """Draw ``d_per_col[j]`` distinct rows for every column ``j``.

    Rows come from ``sampler(size)``; a row repeated within one column is drawn
    again, so every column ends with exactly its requested count.  Returns
    (cols, rows) sorted by (col, row).
    """
    ncols = d_per_col.shape[0]
    cols = np.repeat(np.arange(ncols, dtype=np.int64), d_per_col)
    rows = sampler(cols.shape[0])
    # (col, row) order through one int64 key (rows < 2^31, so key = col * 2^31 + row)
    key = np.sort((cols << 31) | rows)
    cols, rows = key >> 31, key & ((1 << 31) - 1)
    # Entries of the columns still holding a repeat, as positions in the
    # (col, row)-sorted arrays; a column's entries are contiguous, so re-sorting
    # only those entries keeps the whole array sorted.
    idx = np.arange(cols.shape[0])
    for _ in range(max_rounds):
        c, r = cols[idx], rows[idx]
        dup = np.zeros(idx.shape[0], dtype=bool)
        dup[1:] = (c[1:] == c[:-1]) & (r[1:] == r[:-1])
        nd = int(dup.sum())
        if nd == 0:
            return cols, rows
        r = r.copy()
        r[dup] = sampler(nd)
        bad = np.isin(c, np.unique(c[dup]))
        idx, c, r = idx[bad], c[bad], r[bad]
        rows[idx] = np.sort((c << 31) | r) & ((1 << 31) - 1)
    raise RuntimeError("could not draw distinct rows")


def uniform_columns(n: int, d: int, seed: int = 0, m: int | None = None,
                    values: str = "f64") -> CSC:
    """m x n matrix (m defaults to n); each column has exactly ``d`` distinct rows
    drawn uniformly without replacement; values uniform[-1, 1] (f64) or
    integers {1..4} (i32)."""
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    cols, rows = _distinct_rows(rng, np.full(n, d, dtype=np.int64),
                                lambda s: rng.integers(0, m, size=s, dtype=np.int64))
    vals = _draw_values(rng, cols.shape[0], values)
    return _csc_from_sorted(m, n, cols, rows, vals)


def _draw_values(rng, nnz, values):
    if values == "f64":
        return rng.uniform(-1.0, 1.0, size=nnz)
    if values == "i32":
        return rng.integers(1, 5, size=nnz, dtype=np.int32)
    if values == "i64":
        return rng.integers(1, 5, size=nnz, dtype=np.int64)
    if values == "ones":
        return np.ones(nnz, dtype=np.float64)
    raise ValueError(values)


def rmat_symmetric(scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19, d=0.05,
                   seed: int = 0, values: str = "ones") -> CSC:
    """R-MAT graph with 2**scale vertices and edge_factor * 2**scale drawn edges.

    Each edge picks one quadrant per bit level (probabilities a, b, c, d; the
    first level chooses the most significant bit).  Self-loops are dropped,
    duplicate edges merged and the pattern symmetrised (A union A^T).  Values:
    "ones" (f64 1.0) or "i64" (int64 1) -- the path-count semiring input.
    """
    n = 1 << scale
    ne = edge_factor * n
    rng = np.random.default_rng(seed)
    r = np.zeros(ne, dtype=np.int64)
    cc = np.zeros(ne, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for _ in range(scale):
        u = rng.random(ne)
        rbit = (u >= ab).astype(np.int64)
        cbit = (((u >= a) & (u < ab)) | (u >= abc)).astype(np.int64)
        r = (r << 1) | rbit
        cc = (cc << 1) | cbit
    keep = r != cc
    r, cc = r[keep], cc[keep]
    cols, rows = _sort_dedup(np.concatenate([cc, r]), np.concatenate([r, cc]), n)
    if values == "ones":
        vals = np.ones(cols.shape[0], dtype=np.float64)
    elif values == "i64":
        vals = np.ones(cols.shape[0], dtype=np.int64)
    else:
        raise ValueError(values)
    return _csc_from_sorted(n, n, cols, rows, vals)


def poisson3d(N: int) -> CSC:
    """7-point Laplacian on an N^3 grid, lexicographic v = (x*N + y)*N + z,
    diagonal 6, off-diagonals -1, neighbours outside the grid dropped (Dirichlet)."""
    n = N * N * N
    v = np.arange(n, dtype=np.int64)
    x, y, z = v // (N * N), (v // N) % N, v % N
    offs = [(-N * N, x > 0), (-N, y > 0), (-1, z > 0), (0, np.ones(n, bool)),
            (1, z < N - 1), (N, y < N - 1), (N * N, x < N - 1)]
    # column v's rows are v + off for the valid offsets, already ascending
    rows = np.stack([v + o for o, _ in offs], axis=1)
    valid = np.stack([m for _, m in offs], axis=1)
    vals = np.stack([np.full(n, 6.0 if o == 0 else -1.0) for o, _ in offs], axis=1)
    cols = np.broadcast_to(v[:, None], rows.shape)
    return _csc_from_sorted(n, n, cols[valid], rows[valid], vals[valid])


def aggregation_2x2x2(N: int) -> CSC:
    """Piecewise-constant 2x2x2 aggregation P_agg (N^3 x (N/2)^3), one nonzero
    1/sqrt(8) per row: fine vertex (x, y, z) belongs to aggregate
    (x//2, y//2, z//2), both numbered lexicographically."""
    assert N % 2 == 0
    M = N // 2
    J = np.arange(M ** 3, dtype=np.int64)
    X, Y, Z = J // (M * M), (J // M) % M, J % M
    sub = [(dx, dy, dz) for dx in (0, 1) for dy in (0, 1) for dz in (0, 1)]
    rows = np.stack([((2 * X + dx) * N + 2 * Y + dy) * N + 2 * Z + dz for dx, dy, dz in sub], axis=1)
    cols = np.broadcast_to(J[:, None], rows.shape)
    vals = np.full(rows.shape, 1.0 / math.sqrt(8.0))
    return _csc_from_sorted(N ** 3, M ** 3, cols.ravel(), rows.ravel(), vals.ravel())


def aggregation_2x2x2_transpose(N: int) -> CSC:
    """P_agg^T ((N/2)^3 x N^3): column v holds the single row agg(v)."""
    M = N // 2
    v = np.arange(N ** 3, dtype=np.int64)
    x, y, z = v // (N * N), (v // N) % N, v % N
    rows = ((x // 2) * M + y // 2) * M + z // 2
    return _csc_from_sorted(M ** 3, N ** 3, v, rows, np.full(N ** 3, 1.0 / math.sqrt(8.0)))


def lognormal_zipf_rows(nrows: int = 100_000, ncols: int = 1 << 20, mean: float = 50.0,
                        cap: int = 500, zipf_s: float = 1.2, sigma: float = 1.0,
                        seed: int = 0):
    """Rectangular int32 matrix A (nrows x ncols) and its transpose, both CSC.

    Row lengths: lognormal with the given mean (mu = ln(mean) - sigma^2/2),
    rounded and clamped to [1, cap].  Column indices: Zipf over ranks 1..ncols
    with p(r) proportional to r^-s, rank r is column r-1; a column repeated within
    a row is drawn again.  Values: uniform integers {1..4}.
    Returns (A, At) where At = A^T (the CSC of At is the CSR of A).
    """
    rng = np.random.default_rng(seed)
    mu = math.log(mean) - sigma * sigma / 2.0
    lens = np.clip(np.rint(rng.lognormal(mu, sigma, size=nrows)), 1, cap).astype(np.int64)
    cdf = np.cumsum(np.arange(1, ncols + 1, dtype=np.float64) ** (-zipf_s))
    cdf /= cdf[-1]

    def sampler(s):
        return np.minimum(np.searchsorted(cdf, rng.random(s), side="right"), ncols - 1).astype(np.int64)

    # rows of A are the columns of At: draw distinct column ids per row
    rws, cls = _distinct_rows(rng, lens, sampler)
    vals = rng.integers(1, 5, size=rws.shape[0], dtype=np.int32)
    At = _csc_from_sorted(ncols, nrows, rws, cls, vals)
    order = np.lexsort((rws, cls))
    A = _csc_from_sorted(nrows, ncols, cls[order], rws[order], vals[order].copy())
    return A, At


def random_instance(n: int, d: int, kind: str, rng, m: int | None = None,
                    values: str = "f64") -> CSC:
    """m x n instance with exactly ``d`` distinct rows per column.

    kind "er": rows uniform.  kind "rmat": each of ceil(log2 m) row bits is 1 with
    probability c + d = 0.24 (the R-MAT row marginal), rows >= m are redrawn.
    """
    m = n if m is None else m
    if kind == "er":
        def sampler(s):
            return rng.integers(0, m, size=s, dtype=np.int64)
    elif kind == "rmat":
        L = max(1, int(math.ceil(math.log2(m))))
        w = (np.int64(1) << np.arange(L - 1, -1, -1, dtype=np.int64))
        wf = w.astype(np.float64)

        def sampler(s):
            out = np.empty(s, dtype=np.int64)
            todo = np.arange(s)
            while todo.size:
                bits = rng.random((todo.size, L)) < 0.24
                r = (bits.astype(np.float64) @ wf).astype(np.int64)   # exact: sums of powers of 2 below 2^53
                ok = r < m
                out[todo[ok]] = r[ok]
                todo = todo[~ok]
            return out
    else:
        raise ValueError(kind)
    cols, rows = _distinct_rows(rng, np.full(n, min(d, m), dtype=np.int64), sampler)
    return _csc_from_sorted(m, n, cols, rows, _draw_values(rng, cols.shape[0], values))


def batch_instances(count: int, nmin: int, nmax: int, seed: int = 0, dmin: int = 4,
                    dmax: int = 32, values: str = "f64"):
    """``count`` independent (A_j, B_j) square pairs: n_j log-uniform in
    [nmin, nmax], kind ER or R-MAT-row with probability 1/2 each, and a
    nonzeros-per-column count uniform in [dmin, dmax] drawn per matrix."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        kind = "er" if rng.random() < 0.5 else "rmat"
        dA = int(rng.integers(dmin, dmax + 1))
        dB = int(rng.integers(dmin, dmax + 1))
        A = random_instance(n, dA, kind, rng, values=values)
        B = random_instance(n, dB, kind, rng, values=values)
        out.append((A, B))
    return out


def fig1_example_B0() -> CSC:
    """An 8 x 4 column block whose nonzero-row projection is the paper's
    H_0 = [1,0,1,1,0,1,0,0] (Fig. 1): rows {0, 2, 3, 5}; values 1.0."""
    cols = np.array([0, 0, 1, 2, 3, 3], dtype=np.int64)
    rows = np.array([0, 3, 2, 5, 0, 3], dtype=np.int64)
    return _csc_from_sorted(8, 4, cols, rows, np.ones(6))


def fig1_example(seed: int = 0):
    """8 x 8 matrices A and B on two column owners of 4 columns each, where B's
    first block is ``fig1_example_B0`` and every column of A is nonempty."""
    rng = np.random.default_rng(seed)
    A = random_sparse(8, 8, 0.4, rng, values="f64", min_per_col=1)
    B0 = fig1_example_B0()
    B1 = random_sparse(8, 4, 0.4, rng, values="f64")
    colptr = np.concatenate([B0.colptr, B1.colptr[1:] + B0.colptr[-1]])
    B = CSC(8, 8, colptr, np.concatenate([B0.rowidx, B1.rowidx]),
            np.concatenate([B0.vals, B1.vals]))
    return A, B


def random_sparse(m: int, n: int, density: float, rng, values: str = "f64",
                  min_per_col: int = 0, idx_dtype=np.int32) -> CSC:
    """Bernoulli(density) pattern, optionally forcing ``min_per_col`` entries in
    every column; values as in ``uniform_columns`` plus "small" (integers in
    [-3, 3] without 0, exact in f64) and "i64big" (full-range int64)."""
    mask = rng.random((m, n)) < density
    if min_per_col:
        for j in range(n):
            need = min_per_col - int(mask[:, j].sum())
            if need > 0:
                free = np.flatnonzero(~mask[:, j])
                mask[rng.choice(free, size=min(need, free.size), replace=False), j] = True
    cols, rows = np.nonzero(mask.T)
    nnz = cols.shape[0]
    if values == "small":
        v = rng.integers(1, 4, size=nnz) * rng.choice([-1, 1], size=nnz)
        vals = v.astype(np.float64)
    elif values == "i64big":
        vals = rng.integers(np.iinfo(np.int64).min, np.iinfo(np.int64).max, size=nnz, dtype=np.int64)
    else:
        vals = _draw_values(rng, nnz, values)
    return _csc_from_sorted(m, n, cols, rows, vals, idx_dtype)


def random_permutation(n: int, seed: int = 0) -> np.ndarray:
    """A seeded permutation of range(n) (an input transform for ordering studies)."""
    return np.random.default_rng(seed).permutation(n).astype(np.int64)


def relabel(M: CSC, row_perm=None, col_perm=None) -> CSC:
    """The matrix whose entry (row_perm[r], col_perm[c]) is M's entry (r, c):
    rows and columns renamed by the given permutations (None keeps them).
    Q A Q^T is relabel(A, q, q); Q R is relabel(R, row_perm=q)."""
    cp = np.asarray(M.colptr, dtype=np.int64)
    cols = np.repeat(np.arange(M.ncols, dtype=np.int64), np.diff(cp))
    rows = np.asarray(M.rowidx, dtype=np.int64)
    if row_perm is not None:
        rows = np.asarray(row_perm, dtype=np.int64)[rows]
    if col_perm is not None:
        cols = np.asarray(col_perm, dtype=np.int64)[cols]
    order = np.lexsort((rows, cols))
    out = _csc_from_sorted(M.nrows, M.ncols, cols[order], rows[order], np.asarray(M.vals)[order])
    return CSC(out.nrows, out.ncols, out.colptr, out.rowidx.astype(np.asarray(M.rowidx).dtype), out.vals)
