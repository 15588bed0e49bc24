"""Pins for the CPU oracle: each test ties it to something other than itself --
the paper's worked example, dense or brute-force arithmetic, library routines,
algebraic identities and closed forms.  No GPU is needed."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def to_dense(C, m=None):
    m = C["nrows"] if m is None else m
    n = C["ncols"]
    D = np.zeros((m, n), dtype=C["vals"].dtype)
    for j in range(n):
        s, e = C["colptr"][j], C["colptr"][j + 1]
        D[C["rowidx"][s:e], j] = C["vals"][s:e]
    return D


def pattern_dense(C):
    P = np.zeros((C["nrows"], C["ncols"]), dtype=bool)
    for j in range(C["ncols"]):
        s, e = C["colptr"][j], C["colptr"][j + 1]
        P[C["rowidx"][s:e], j] = True
    return P


def to_scipy(M):
    return sp.csc_matrix((np.asarray(M.vals), np.asarray(M.rowidx, dtype=np.int64),
                          np.asarray(M.colptr, dtype=np.int64)), shape=(M.nrows, M.ncols))


def from_scipy(S, idx=np.int32):
    S = sp.csc_matrix(S)
    S.sort_indices()
    return synth.CSC(S.shape[0], S.shape[1], S.indptr.astype(np.int64), S.indices.astype(idx), S.data.copy())


def result_as_csc(C):
    return synth.CSC(C["nrows"], C["ncols"], C["colptr"], C["rowidx"], C["vals"])


def assert_sorted_unique(C):
    for j in range(C["ncols"]):
        r = C["rowidx"][C["colptr"][j]:C["colptr"][j + 1]]
        assert np.all(np.diff(r) > 0), f"column {j} rows not strictly increasing"


# ---------------------------------------------------------------- paper example

def test_fig1_H0_and_block_fetch():
    """Fig. 1 / Section 3.1: H_0 = [1,0,1,1,0,1,0,0]; with 2 blocks of 2 column
    ids per owner, p_0 fetches blocks (0,0), (0,1) and (1,0) but not (1,1)."""
    g = json.load(open(os.path.join(GOLD, "fig1_h0.json")))
    A, B = synth.fig1_example()
    pl = oracle.plan_block(A, B, 0, 4, g["b"])
    assert pl["H"].tolist() == g["H0"]
    assert pl["dtilde"].tolist() == g["required_columns_p0"]
    assert pl["fetch"].tolist() == g["fetch_blocks_p0"]
    assert pl["intervals"].tolist() == g["fetched_intervals_p0"]
    # chosen blocks are read whole: columns 1 and 4 come along unused
    unused = int(A.colptr[2] - A.colptr[1]) + int(A.colptr[5] - A.colptr[4])
    assert pl["vol_block"] == pl["vol_exact"] + unused
    # the whole of Algorithm 1 reproduces the plain product on this example
    C1, _ = oracle.spgemm_1d(A, B, P=2, b=2)
    C = oracle.spgemm(A, B)
    assert np.array_equal(C1["colptr"], C["colptr"]) and np.array_equal(C1["rowidx"], C["rowidx"])
    assert np.array_equal(C1["vals"], C["vals"])


# ------------------------------------------------------------ dense arithmetic

@pytest.mark.parametrize("seed", range(6))
def test_dense_matmul_small_integers(seed):
    """Small-integer values make every double sum exact, so the oracle must equal
    numpy's dense product bit for bit; its pattern must equal the boolean
    product of the patterns (no cancellation is dropped)."""
    rng = np.random.default_rng(seed)
    m, k, n = rng.integers(1, 40, size=3)
    A = synth.random_sparse(m, k, 0.25, rng, values="small")
    B = synth.random_sparse(k, n, 0.25, rng, values="small")
    C = oracle.spgemm(A, B)
    assert_sorted_unique(C)
    Ad, Bd = to_dense_csc(A), to_dense_csc(B)
    assert np.array_equal(to_dense(C), Ad @ Bd)
    patt = ((Ad != 0).astype(np.int64) @ (Bd != 0).astype(np.int64)) > 0
    assert np.array_equal(pattern_dense(C), patt)
    # integer semiring on the same data
    Ci = oracle.spgemm(A.astype(val=np.int64), B.astype(val=np.int64))
    assert np.array_equal(Ci["colptr"], C["colptr"]) and np.array_equal(Ci["rowidx"], C["rowidx"])
    assert np.array_equal(to_dense(Ci), (Ad @ Bd).astype(np.int64))


def to_dense_csc(M):
    D = np.zeros((M.nrows, M.ncols), dtype=np.asarray(M.vals).dtype)
    for j in range(M.ncols):
        r, v = M.col(j)
        D[r, j] = v
    return D


def test_brute_force_triple_loop_with_cancellation():
    """Brute force over (r, k, j) on tiny inputs, including explicit zeros and
    sums that cancel: every position with at least one product is present."""
    rng = np.random.default_rng(11)
    for trial in range(25):
        m, k, n = rng.integers(1, 7, size=3)
        A = synth.random_sparse(m, k, 0.5, rng, values="small")
        B = synth.random_sparse(k, n, 0.5, rng, values="small")
        A.vals[rng.random(A.nnz) < 0.2] = 0.0        # stored zeros stay structural
        Ad, Bd = to_dense_csc(A), to_dense_csc(B)
        Am = np.zeros((m, k), bool)
        Bm = np.zeros((k, n), bool)
        for j in range(k):
            Am[A.col(j)[0], j] = True
        for j in range(n):
            Bm[B.col(j)[0], j] = True
        C = oracle.spgemm(A, B)
        for j in range(n):
            want_rows, want_vals = [], []
            for r in range(m):
                terms = [Ad[r, kk] * Bd[kk, j] for kk in range(k) if Am[r, kk] and Bm[kk, j]]
                if terms:
                    want_rows.append(r)
                    want_vals.append(sum(terms))
            s, e = C["colptr"][j], C["colptr"][j + 1]
            assert C["rowidx"][s:e].tolist() == want_rows
            assert C["vals"][s:e].tolist() == want_vals
    # an explicit cancelling case: [1 1] * [1; -1] = 0, still one stored entry
    A = synth.CSC(1, 2, np.array([0, 1, 2]), np.array([0, 0], np.int32), np.array([1.0, 1.0]))
    B = synth.CSC(2, 1, np.array([0, 2]), np.array([0, 1], np.int32), np.array([1.0, -1.0]))
    C = oracle.spgemm(A, B)
    assert C["colptr"].tolist() == [0, 1] and C["vals"].tolist() == [0.0] and C["absum"].tolist() == [2.0]


def test_int64_semiring_wraps_modulo_2_64():
    """The integer semiring is exact arithmetic modulo 2^64 (Python big ints)."""
    rng = np.random.default_rng(5)
    for trial in range(10):
        m, k, n = rng.integers(1, 6, size=3)
        A = synth.random_sparse(m, k, 0.6, rng, values="i64big")
        B = synth.random_sparse(k, n, 0.6, rng, values="i64big")
        C = oracle.spgemm(A, B)
        Ad = [[0] * k for _ in range(m)]
        Bd = [[0] * n for _ in range(k)]
        for j in range(k):
            for r, v in zip(*A.col(j)):
                Ad[r][j] = int(v)
        for j in range(n):
            for r, v in zip(*B.col(j)):
                Bd[r][j] = int(v)
        got = to_dense(C)
        for r in range(m):
            for j in range(n):
                s = sum(Ad[r][kk] * Bd[kk][j] for kk in range(k)) % (1 << 64)
                if s >= 1 << 63:
                    s -= 1 << 64
                assert int(got[r, j]) == s


# ------------------------------------------------------------------ identities

@pytest.mark.parametrize("seed", range(4))
def test_transpose_identity(seed):
    """(AB)^T = B^T A^T, the transposes taken by scipy; same terms in the same
    k order, so equal bit for bit."""
    rng = np.random.default_rng(100 + seed)
    A = synth.random_sparse(50, 37, 0.08, rng)
    B = synth.random_sparse(37, 61, 0.08, rng)
    C = oracle.spgemm(A, B)
    At, Bt = from_scipy(to_scipy(A).T), from_scipy(to_scipy(B).T)
    Ct = oracle.spgemm(Bt, At)
    lhs = sp.csc_matrix(to_scipy(result_as_csc(C)).T)
    lhs.sort_indices()
    assert np.array_equal(lhs.indptr, Ct["colptr"]) and np.array_equal(lhs.indices, Ct["rowidx"])
    assert np.array_equal(lhs.data, Ct["vals"])


def test_identity_is_neutral():
    """A*I = A and I*A = A."""
    rng = np.random.default_rng(3)
    A = synth.random_sparse(40, 30, 0.1, rng)
    I30 = synth.CSC(30, 30, np.arange(31), np.arange(30, dtype=np.int32), np.ones(30))
    I40 = synth.CSC(40, 40, np.arange(41), np.arange(40, dtype=np.int32), np.ones(40))
    for C in (oracle.spgemm(A, I30), oracle.spgemm(I40, A)):
        assert np.array_equal(C["colptr"], A.colptr)
        assert np.array_equal(C["rowidx"], A.rowidx)
        assert np.array_equal(C["vals"], A.vals)


@pytest.mark.parametrize("P", [1, 2, 3, 7])
@pytest.mark.parametrize("b", [1, 2, 5, 32, 1000])
def test_union_of_blocks_equals_unpartitioned(P, b):
    """Algorithm 1 on P blocks (gather A~_i, multiply A~_i * B_i, concatenate)
    gives exactly the plain product: the partition and the fetch blocks only
    choose which data is touched (Section 3.1)."""
    rng = np.random.default_rng(P * 1000 + b)
    A = synth.random_sparse(45, 40, 0.07, rng)
    B = synth.random_sparse(40, 33, 0.07, rng)
    C = oracle.spgemm(A, B)
    C1, plans = oracle.spgemm_1d(A, B, P, b)
    for key in ("colptr", "rowidx", "vals", "absum"):
        assert np.array_equal(C1[key], C[key]), key
    assert len(plans) == P


def test_flop_identity_and_nnz_bound():
    """Section 3.2: the number of products is the inner product of the column
    counts of A with the row counts of B, and nnz(C) <= products."""
    rng = np.random.default_rng(8)
    for _ in range(5):
        A = synth.random_sparse(60, 50, 0.1, rng)
        B = synth.random_sparse(50, 70, 0.1, rng)
        C = oracle.spgemm(A, B)
        colnnz_A = np.diff(A.colptr)
        rownnz_B = np.bincount(B.rowidx, minlength=B.nrows)
        products = int(colnnz_A @ rownnz_B)
        assert int(C["flops"].sum()) == products
        assert int(C["colptr"][-1]) <= products
        f = oracle.features(A, B)
        assert np.array_equal(f["flops"], C["flops"])
        assert np.array_equal(f["nnzb"], np.diff(B.colptr))


def _features_by_loop(A, B):
    """flops_j, nnz(B(:,j)), max and mean nnz(A(:,k)) over the stored k of
    B(:,j), by a plain Python loop over B's columns reading A's column counts."""
    acount = np.diff(np.asarray(A.colptr, dtype=np.int64))
    fl, nb, mx, mean = [], [], [], []
    for j in range(B.ncols):
        ks = [int(k) for k in B.rowidx[B.colptr[j]:B.colptr[j + 1]]]
        lens = [int(acount[k]) for k in ks]
        fl.append(sum(lens))
        nb.append(len(ks))
        mx.append(max(lens) if lens else 0)
        mean.append(sum(lens) / len(lens) if lens else 0.0)
    return np.array(fl), np.array(nb), np.array(mx), np.array(mean)


def test_features_against_direct_loop():
    """Section 3.2 features of every output column (flops, nnz(B(:,j)), max and
    mean nnz of the contributing A columns) equal a plain loop, on random inputs
    and on hand-built columns: an empty column, a column whose largest A column
    comes last, one whose largest comes first, and one that only touches an
    empty column of A (max 0, not the maximum over B's values or over all A)."""
    rng = np.random.default_rng(17)
    cases = [(synth.random_sparse(80, 60, 0.08, rng, values="i32"),
              synth.random_sparse(60, 90, 0.06, rng, values="i32")) for _ in range(3)]
    # A: column k has k % 5 entries (column 0, 5, 10 empty); its values are
    # large so that a max over values, not counts, would differ.
    dA = np.zeros((12, 12))
    for k in range(12):
        dA[: k % 5, k] = 100.0 + k
    # B's columns: empty; rows {0, 1, 2, 4} (largest A column, 4 entries, last);
    # rows {9, 1} stored ascending as {1, 9} (largest = column 9, 4 entries, last);
    # rows {4, 6} (largest first); row {5} (an empty A column); all of A's columns.
    dB = np.zeros((12, 5))
    for j, ks in enumerate([[], [0, 1, 2, 4], [1, 9], [4, 6], [5]]):
        for k in ks:
            dB[k, j] = 7.0
    A_hand, B_hand = synth.from_dense(dA), synth.from_dense(dB)
    cases.append((A_hand, B_hand))
    for A, B in cases:
        f = oracle.features(A, B)
        fl, nb, mx, mean = _features_by_loop(A, B)
        assert np.array_equal(f["flops"], fl)
        assert np.array_equal(f["nnzb"], nb)
        assert np.array_equal(f["maxa"], mx)
        assert np.allclose(f["meana"], mean, rtol=0, atol=1e-12)
    f = oracle.features(A_hand, B_hand)
    assert f["maxa"].tolist() == [0, 4, 4, 4, 0]
    assert f["flops"].tolist() == [0, 0 + 1 + 2 + 4, 1 + 4, 4 + 1, 0]
    # a sub-range of columns gives the same rows of the table
    g = oracle.features(A_hand, B_hand, 1, 4)
    assert g["maxa"].tolist() == [4, 4, 4]


def test_pattern_matches_scipy_all_ones_product():
    """With all-ones values nothing cancels, so the oracle's pattern equals the
    pattern of scipy's product (a library routine)."""
    rng = np.random.default_rng(21)
    A = synth.random_sparse(300, 200, 0.02, rng, values="ones")
    B = synth.random_sparse(200, 250, 0.02, rng, values="ones")
    C = oracle.spgemm(A, B)
    S = sp.csc_matrix(to_scipy(A) @ to_scipy(B))
    S.sort_indices()
    assert np.array_equal(S.indptr, C["colptr"]) and np.array_equal(S.indices, C["rowidx"])
    assert np.array_equal(S.data, C["vals"])


# ------------------------------------------------------------- Algorithm 2

@pytest.mark.parametrize("seed", range(5))
def test_block_fetch_contract(seed):
    """Algorithm 2: the chosen intervals cover every required column, M <= K,
    every chosen block holds a required column, and the volumes are ordered
    exact <= block-granular <= nnz(A)."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(1, 300))
    A = synth.random_sparse(80, k, 0.03, rng)
    B = synth.random_sparse(k, 90, 0.01, rng)
    for b in (1, 3, 32, 64, 1000):
        for c0, c1 in ((0, 90), (10, 40), (50, 50)):
            pl = oracle.plan_block(A, B, c0, c1, b)
            H = np.zeros(k, np.uint8)
            for j in range(c0, c1):
                H[B.col(j)[0]] = 1
            assert np.array_equal(pl["H"], H)
            nonempty = np.diff(A.colptr) > 0
            assert pl["dtilde"].tolist() == np.flatnonzero(H.astype(bool) & nonempty).tolist()
            K = (k + b - 1) // b
            assert pl["fetch"].shape[0] == K and pl["fetch"].sum() <= K
            for h in pl["dtilde"]:
                assert any(lo <= h <= hi for lo, hi in pl["intervals"])
            for lo, hi in pl["intervals"]:
                assert np.any((pl["dtilde"] >= lo) & (pl["dtilde"] <= hi))
            assert pl["vol_exact"] <= pl["vol_block"] <= A.nnz
            At = oracle.gather(A, pl["dtilde"])
            assert int(At["colptr"][-1]) == pl["vol_exact"]


# ------------------------------------------------------------- closed forms

@pytest.mark.parametrize("N", [4, 8])
def test_galerkin_closed_form(N):
    """7-point Laplacian (diag 6, off-diagonal -1) and 2x2x2 aggregation with
    entries 1/sqrt(8).  Row v of A*P_agg: 3/sqrt(8) on its own aggregate (6 minus
    its 3 neighbours inside the aggregate) and -1/sqrt(8) on each aggregate
    reached through an outer face; nnz(A*P_agg) = 4N^3 - 6N^2.  The coarse
    operator P^T A P is the (N/2)^3 7-point operator with diagonal 3 and face
    off-diagonals -1/2, nnz = 7M^3 - 6M^2 with M = N/2."""
    A = synth.poisson3d(N)
    Pg = synth.aggregation_2x2x2(N)
    PT = synth.aggregation_2x2x2_transpose(N)
    AP = oracle.spgemm(A, Pg)
    assert int(AP["colptr"][-1]) == 4 * N ** 3 - 6 * N ** 2
    s8 = 1.0 / math.sqrt(8.0)
    M = N // 2
    D = to_dense(AP)
    for v in range(N ** 3):
        x, y, z = v // (N * N), (v // N) % N, v % N
        want = {((x // 2) * M + y // 2) * M + z // 2: 3 * s8}
        for axis, c in ((0, x), (1, y), (2, z)):
            step = -1 if c % 2 == 0 else 1          # the outer neighbour along this axis
            cc = c + step
            if 0 <= cc < N:
                xyz = [x, y, z]
                xyz[axis] = cc
                want[((xyz[0] // 2) * M + xyz[1] // 2) * M + xyz[2] // 2] = -s8
        nz = np.flatnonzero(D[v] != 0)
        assert sorted(want) == nz.tolist()
        for J, val in want.items():
            assert abs(D[v, J] - val) <= 1e-15
    APc = result_as_csc(AP)
    G = oracle.spgemm(PT, APc)
    assert int(G["colptr"][-1]) == 7 * M ** 3 - 6 * M ** 2
    Gd = to_dense(G)
    for I in range(M ** 3):
        X, Y, Z = I // (M * M), (I // M) % M, I % M
        for J in range(M ** 3):
            X2, Y2, Z2 = J // (M * M), (J // M) % M, J % M
            dist = abs(X - X2) + abs(Y - Y2) + abs(Z - Z2)
            want = 3.0 if dist == 0 else (-0.5 if dist == 1 else 0.0)
            assert abs(Gd[I, J] - want) <= 1e-12 * max(1.0, abs(want)) * 8


def test_graph_squaring_properties():
    """Squaring a symmetric 0/1 graph: C is symmetric, C_ii = deg(i), and the
    double run (values 1.0) equals the int64 path-count run exactly."""
    A = synth.rmat_symmetric(9, 8, seed=1)
    Ai = synth.rmat_symmetric(9, 8, seed=1, values="i64")
    C = oracle.spgemm(A, A)
    Ci = oracle.spgemm(Ai, Ai)
    assert np.array_equal(C["colptr"], Ci["colptr"]) and np.array_equal(C["rowidx"], Ci["rowidx"])
    assert np.array_equal(C["vals"].astype(np.int64), Ci["vals"])
    S = to_scipy(result_as_csc(C))
    assert (S != S.T).nnz == 0
    deg = np.diff(A.colptr)
    assert np.array_equal(S.diagonal(), deg.astype(np.float64))


def test_similarity_product_diagonal():
    """C = A*A^T for an integer matrix: symmetric with C_ii = sum_k a_ik^2."""
    A, At = synth.lognormal_zipf_rows(nrows=300, ncols=2000, mean=8, cap=40, seed=2)
    C = oracle.spgemm(A.astype(val=np.int64), At.astype(val=np.int64))
    S = to_scipy(result_as_csc(C))
    assert (S != S.T).nnz == 0
    sq = np.zeros(300, np.int64)
    for j in range(At.ncols):
        r, v = At.col(j)
        sq[j] = int(np.sum(v.astype(np.int64) ** 2))
    assert np.array_equal(S.diagonal(), sq)


# ---------------------------------------------------------------- edge cases

def test_empty_and_degenerate_shapes():
    z = lambda m, n: synth.CSC(m, n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    for m, k, n in ((0, 0, 0), (3, 0, 4), (0, 5, 2), (4, 5, 0), (3, 4, 5)):
        C = oracle.spgemm(z(m, k), z(k, n))
        assert C["colptr"].tolist() == [0] * (n + 1)
    rng = np.random.default_rng(0)
    A = synth.random_sparse(1, 6, 0.5, rng)
    B = synth.random_sparse(6, 1, 0.5, rng)
    C = oracle.spgemm(A, B)
    assert C["colptr"][-1] <= 1
    with pytest.raises(ValueError):
        oracle.spgemm(z(3, 4), z(5, 2))
    C1, plans = oracle.spgemm_1d(z(3, 4), z(4, 5), P=3, b=2)
    assert C1["colptr"].tolist() == [0] * 6 and all(p["dtilde"].size == 0 for p in plans)


# ------------------------------------------------- Algorithm 3 (outer product)

@pytest.mark.parametrize("P", [1, 2, 3, 7, 60])
def test_outer_split_times_merge_matrix_is_B(P):
    """Summing the row blocks back together gives B: scipy's product of the
    split matrix and S equals B entry for entry (P = 60 exceeds k's blocks
    of more than one row, so some blocks are empty)."""
    rng = np.random.default_rng(P)
    B = synth.random_sparse(53, 41, 0.12, rng, values="i64")
    Bs = oracle.outer_split(B, P)
    S = oracle.merge_matrix(B.ncols, P, integer=True)
    back = sp.csc_matrix(to_scipy(Bs) @ to_scipy(S))
    ref = to_scipy(B)
    assert (back != ref).nnz == 0
    assert np.array_equal(np.sort(back.indices), np.sort(ref.indices))


@pytest.mark.parametrize("P", [1, 4, 5])
def test_outer_split_columns_hold_their_row_block(P):
    """Column i*n + j holds exactly the entries of B(:, j) with row in
    [floor(i*k/P), floor((i+1)*k/P)), in ascending row order."""
    rng = np.random.default_rng(10 + P)
    B = synth.random_sparse(37, 29, 0.2, rng, values="f64")
    Bs = oracle.outer_split(B, P)
    k, n = B.nrows, B.ncols
    for i in range(P):
        lo, hi = (i * k) // P, ((i + 1) * k) // P
        for j in range(n):
            s, e = B.colptr[j], B.colptr[j + 1]
            rows = B.rowidx[s:e]
            sel = (rows >= lo) & (rows < hi)
            c = i * n + j
            got = Bs.rowidx[Bs.colptr[c]:Bs.colptr[c + 1]]
            assert np.array_equal(got, rows[sel])
            assert np.array_equal(Bs.vals[Bs.colptr[c]:Bs.colptr[c + 1]], B.vals[s:e][sel])


def test_outer_partial_products_are_dense_block_products():
    """Column (i, j) of A * outer_split(B) equals the dense product
    A[:, K_i] @ B[K_i, j], and the partial columns add up to A @ B."""
    rng = np.random.default_rng(3)
    A = synth.random_sparse(24, 30, 0.2, rng, values="i32")
    B = synth.random_sparse(30, 17, 0.2, rng, values="i32")
    P = 4
    Ad, Bd = to_dense_csc(A).astype(np.int64), to_dense_csc(B).astype(np.int64)
    Cp = to_dense(oracle.spgemm(A, oracle.outer_split(B, P)))
    k, n = B.nrows, B.ncols
    total = np.zeros((A.nrows, n), dtype=np.int64)
    for i in range(P):
        lo, hi = (i * k) // P, ((i + 1) * k) // P
        blk = Ad[:, lo:hi] @ Bd[lo:hi, :]
        assert np.array_equal(Cp[:, i * n:(i + 1) * n], blk)
        total += blk
    assert np.array_equal(total, Ad @ Bd)


def test_outer_volumes_brute_force():
    """The volume counters against direct enumeration with dense matrices."""
    rng = np.random.default_rng(5)
    A = synth.random_sparse(20, 25, 0.25, rng, values="f64")
    B = synth.random_sparse(25, 18, 0.25, rng, values="f64")
    P = 3
    v = oracle.outer_volumes(A, B, P)
    Ad, Bd = to_dense_csc(A) != 0, to_dense_csc(B) != 0
    k, n = B.nrows, B.ncols
    rblk = [max(i for i in range(P) if (i * k) // P <= r) for r in range(k)]
    cblk = [max(i for i in range(P) if (i * n) // P <= j) for j in range(n)]
    assert v["b_moved"] == sum(1 for r in range(k) for j in range(n) if Bd[r, j] and rblk[r] != cblk[j])
    pn = pm = 0
    for i in range(P):
        lo, hi = (i * k) // P, ((i + 1) * k) // P
        pat = (Ad[:, lo:hi].astype(int) @ Bd[lo:hi, :].astype(int)) > 0
        pn += int(pat.sum())
        pm += int(sum(pat[:, j].sum() for j in range(n) if cblk[j] != i))
    assert v["partial_nnz"] == pn and v["partial_moved"] == pm


# ------------------------------------------------ planning diagnostics

@pytest.mark.parametrize("P", [1, 3, 8])
def test_flop_bounds_balance(P):
    """The flop-balanced split: contiguous, from 0 to n, and every block holds
    at most F/P plus one column's flops (greedy bound), checked against flops
    recounted by brute force over B's entries."""
    rng = np.random.default_rng(P)
    A = synth.random_sparse(60, 50, 0.1, rng, values="f64")
    B = synth.random_sparse(50, 70, 0.1, rng, values="f64")
    bd = oracle.flop_bounds(A, B, P)
    assert bd[0] == 0 and bd[-1] == B.ncols and np.all(np.diff(bd) >= 0)
    acnt = np.diff(A.colptr)
    fl = np.array([sum(int(acnt[k]) for k in B.rowidx[B.colptr[j]:B.colptr[j + 1]]) for j in range(B.ncols)])
    F = int(fl.sum())
    for i in range(P):
        blk = int(fl[bd[i]:bd[i + 1]].sum())
        assert blk <= F / P + fl.max() + 1e-9
        # the boundary is the first column where the running total reaches i/P
        if 0 < i < P:
            pre = np.concatenate([[0], np.cumsum(fl)])
            assert P * pre[bd[i]] >= i * F and (bd[i] == 0 or P * pre[bd[i] - 1] < i * F)


def test_block_volumes_and_explicit_bounds():
    """Per-block volumes against brute force on dense patterns, and the 1D
    multiply with explicit bounds equals the unpartitioned product."""
    rng = np.random.default_rng(11)
    A = synth.random_sparse(40, 36, 0.12, rng, values="small")
    B = synth.random_sparse(36, 30, 0.12, rng, values="small")
    bd = np.array([0, 4, 4, 19, 30])
    v = oracle.block_volumes(A, B, bd, b=5)
    Ad, Bd = to_dense_csc(A) != 0, to_dense_csc(B) != 0
    own = oracle.block_bounds(A.ncols, 4)
    for i in range(4):
        need = Bd[:, bd[i]:bd[i + 1]].any(axis=1) & Ad.any(axis=0)     # H_i and D
        cnt = Ad.sum(axis=0)
        assert v["gathered"][i] == int(cnt[need].sum())
        ks = np.flatnonzero(need)
        assert v["remote"][i] == int(sum(cnt[k] for k in ks if not own[i] <= k < own[i + 1]))
        assert v["flops"][i] == int(sum(cnt[k] for j in range(bd[i], bd[i + 1]) for k in np.flatnonzero(Bd[:, j])))
    C, _ = oracle.spgemm_1d(A, B, 4, 5, bounds=bd)
    ref = oracle.spgemm(A, B)
    assert np.array_equal(C["colptr"], ref["colptr"]) and np.array_equal(C["rowidx"], ref["rowidx"])
    assert np.array_equal(C["vals"], ref["vals"])


# ------------------------------------------------ betweenness centrality

def _undirected(n, edges):
    rows, cols = [], []
    for a, b in edges:
        rows += [a, b]
        cols += [b, a]
    order = np.lexsort((rows, cols))
    return synth._csc_from_sorted(n, n, np.array(cols)[order], np.array(rows)[order], np.ones(len(rows)))


def test_bc_path_graph_closed_form():
    """On a path of n vertices every source counts vertex i as a shortest-path
    interior exactly for the targets on its far side: summed over all sources,
    bc(i) = 2 * i * (n - 1 - i)."""
    from oracle import bc as obc
    n = 9
    A = _undirected(n, [(i, i + 1) for i in range(n - 1)])
    bc, levels = obc.brandes(A, range(n))
    assert np.allclose(bc, [2 * i * (n - 1 - i) for i in range(n)])
    assert sum(levels) == n * n


def test_bc_star_and_cycle():
    """Star: the centre lies on every leaf-to-leaf path (bc = (n-1)(n-2) over
    ordered pairs), leaves on none.  Cycle of 6: ordered pairs at distance 2
    (12, one path, one interior vertex) give 12, pairs at distance 3 (6, two
    paths of two interior vertices, weight 1/2 each) give 12; by symmetry each
    vertex gets 24 / 6 = 4."""
    from oracle import bc as obc
    n = 7
    A = _undirected(n, [(0, i) for i in range(1, n)])
    bc, _ = obc.brandes(A, range(n))
    assert np.isclose(bc[0], (n - 1) * (n - 2)) and np.allclose(bc[1:], 0)
    C = _undirected(6, [(i, (i + 1) % 6) for i in range(6)])
    bc, _ = obc.brandes(C, range(6))
    assert np.allclose(bc, 4.0)


def test_bc_matches_networkx_subset():
    """A random graph and a subset of sources against networkx's subset
    betweenness (sources x all targets), which for undirected graphs halves
    the sum: ours = 2 * networkx."""
    nx = pytest.importorskip("networkx")
    from oracle import bc as obc
    rng = np.random.default_rng(4)
    n = 60
    edges = {(int(a), int(b)) for a, b in rng.integers(0, n, (150, 2)) if a != b}
    edges = {(min(a, b), max(a, b)) for a, b in edges}
    A = _undirected(n, sorted(edges))
    src = [0, 5, 17, 33, 59]
    bc, _ = obc.brandes(A, src)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from(edges)
    ref = nx.betweenness_centrality_subset(G, src, list(range(n)), normalized=False)
    assert np.allclose(bc, 2 * np.array([ref[v] for v in range(n)]))


# ------------------------------------------------------------- masked product

def _dense_pattern(M):
    P = np.zeros((M.nrows, M.ncols), dtype=bool)
    for j in range(M.ncols):
        P[np.asarray(M.rowidx[M.colptr[j]:M.colptr[j + 1]], dtype=np.int64), j] = True
    return P


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("complement", [False, True])
def test_masked_product_equals_dense_masked_matmul(seed, complement):
    """C<M> against dense arithmetic: small integers (exact in doubles), the
    structure from the boolean product of the patterns, masked entry by entry."""
    rng = np.random.default_rng(seed)
    A = synth.random_sparse(23, 17, 0.2, rng, values="small")
    B = synth.random_sparse(17, 11, 0.25, rng, values="small")
    M = synth.random_sparse(23, 11, 0.4, rng, values="f64")
    C = oracle.spgemm_masked(A, B, M, complement=complement)
    assert_sorted_unique(C)
    Da = np.zeros((23, 17))
    Db = np.zeros((17, 11))
    for j in range(17):
        Da[A.rowidx[A.colptr[j]:A.colptr[j + 1]], j] = A.vals[A.colptr[j]:A.colptr[j + 1]]
    for j in range(11):
        Db[B.rowidx[B.colptr[j]:B.colptr[j + 1]], j] = B.vals[B.colptr[j]:B.colptr[j + 1]]
    struct = (_dense_pattern(A).astype(int) @ _dense_pattern(B).astype(int)) > 0
    keep = struct & (_dense_pattern(M) != complement)
    assert np.array_equal(pattern_dense(C), keep)
    assert np.array_equal(to_dense(C)[keep], (Da @ Db)[keep])


def test_masked_product_partitions_the_product():
    """C<M> and C<not M> are disjoint and together give A*B exactly; a full
    mask (or an empty complemented one) leaves A*B unchanged."""
    rng = np.random.default_rng(5)
    A = synth.random_sparse(40, 30, 0.1, rng, values="i64")
    B = synth.random_sparse(30, 25, 0.1, rng, values="i64")
    M = synth.random_sparse(40, 25, 0.3, rng, values="i64")
    full = oracle.spgemm(A, B)
    inside = oracle.spgemm_masked(A, B, M)
    outside = oracle.spgemm_masked(A, B, M, complement=True)
    Pi, Po = pattern_dense(inside), pattern_dense(outside)
    assert not np.any(Pi & Po)
    assert np.array_equal(Pi | Po, pattern_dense(full))
    assert np.array_equal(to_dense(inside) + to_dense(outside), to_dense(full))
    ones = synth.CSC(40, 25, np.arange(26, dtype=np.int64) * 40, np.tile(np.arange(40, dtype=np.int64), 25),
                     np.ones(1000))
    empty = synth.CSC(40, 25, np.zeros(26, dtype=np.int64), np.zeros(0, dtype=np.int64), np.zeros(0))
    for C in (oracle.spgemm_masked(A, B, ones), oracle.spgemm_masked(A, B, empty, complement=True)):
        assert np.array_equal(C["colptr"], full["colptr"])
        assert np.array_equal(C["rowidx"], full["rowidx"])
        assert np.array_equal(C["vals"], full["vals"])


def test_masked_product_is_one_bfs_level():
    """With A a graph and F the current frontier of several sources, A*F
    under the complement of the visited pattern is the next BFS level: checked
    against networkx shortest-path lengths."""
    import networkx as nx
    A = synth.rmat_symmetric(7, 4, seed=3)
    G = nx.Graph()
    G.add_nodes_from(range(A.ncols))
    for v in range(A.ncols):
        for u in A.rowidx[A.colptr[v]:A.colptr[v + 1]]:
            G.add_edge(int(u), v)
    srcs = [0, 5, 17]
    dist = [nx.single_source_shortest_path_length(G, s) for s in srcs]

    def level_csc(d):
        rows = [sorted(v for v, l in dist[c].items() if l == d) for c in range(len(srcs))]
        cp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
        ri = np.array([v for r in rows for v in r], dtype=np.int64)
        return synth.CSC(A.nrows, len(srcs), cp, ri, np.ones(ri.shape[0]))

    def visited_csc(d):
        rows = [sorted(v for v, l in dist[c].items() if l <= d) for c in range(len(srcs))]
        cp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
        ri = np.array([v for r in rows for v in r], dtype=np.int64)
        return synth.CSC(A.nrows, len(srcs), cp, ri, np.ones(ri.shape[0]))
    for d in range(4):
        nxt = oracle.spgemm_masked(A, level_csc(d), visited_csc(d), complement=True)
        want = level_csc(d + 1)
        assert np.array_equal(nxt["colptr"], want.colptr), d
        assert np.array_equal(nxt["rowidx"], want.rowidx), d
