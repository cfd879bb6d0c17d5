"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test ties the oracle to the mathematics of C = A*B (paper Sec. 2,
Fig. "RowWise_SpGEMM"), to the flop definition and the row partition of
Sec. 4.1 (Fig. "RowsToThreads"), or to closed forms of the workloads:
hand-worked products, dense matrix multiplication on tiny inputs, brute
force over all 0/1 3x3 pairs, closed forms for Erdos-Renyi and AMG inputs,
Freivalds identities, a library cross-check and permutation invariance.
"""
import numpy as np
import pytest

import oracle
from paper_1804_01698_gb300 import inputs
from paper_1804_01698_gb300.inputs import CSR


def csr_from_dense(d: np.ndarray) -> CSR:
    d = np.asarray(d)
    m, n = d.shape
    mask = d != 0
    rp = np.zeros(m + 1, np.int32)
    rp[1:] = np.cumsum(mask.sum(axis=1))
    rows, cols = np.nonzero(mask)
    return CSR(m, n, rp, cols.astype(np.int32), d[rows, cols])


def csr_from_pattern(pattern: np.ndarray, vals: np.ndarray) -> CSR:
    """CSR with stored entries where pattern is True and values taken from vals (may be 0)."""
    m, n = pattern.shape
    rp = np.zeros(m + 1, np.int32)
    rp[1:] = np.cumsum(pattern.sum(axis=1))
    rows, cols = np.nonzero(pattern)
    return CSR(m, n, rp, cols.astype(np.int32), vals[rows, cols])


def to_dense(c: CSR, dtype=None) -> np.ndarray:
    out = np.zeros((c.nrows, c.ncols), dtype=dtype or c.vals.dtype)
    rows = np.repeat(np.arange(c.nrows), np.diff(c.row_ptr))
    out[rows, c.col_idx] = c.vals
    return out


def pattern_of(c: CSR) -> np.ndarray:
    out = np.zeros((c.nrows, c.ncols), dtype=bool)
    rows = np.repeat(np.arange(c.nrows), np.diff(c.row_ptr))
    out[rows, c.col_idx] = True
    return out


def assert_rows_sorted_unique(c: CSR):
    for i in range(c.nrows):
        seg = c.col_idx[c.row_ptr[i]:c.row_ptr[i + 1]]
        assert np.all(np.diff(seg) > 0), f"row {i} not strictly increasing"


# ---------------------------------------------------------------- flop (Sec. 4.1)

def test_row_flop_hand_example():
    # A's rows touch B rows {0,1}, {}, {1,2}; B row lengths are 2, 0, 3.
    a = csr_from_dense(np.array([[1, 1, 0], [0, 0, 0], [0, 1, 1]], dtype=np.int64))
    b = csr_from_dense(np.array([[1, 1, 0, 0], [0, 0, 0, 0], [1, 1, 1, 0]], dtype=np.int64))
    assert oracle.row_flop(a, b).tolist() == [2, 0, 3]


@pytest.mark.parametrize("seed", range(5))
def test_row_flop_is_pattern_times_row_lengths(seed):
    rng = np.random.default_rng(seed)
    pa = rng.random((30, 25)) < 0.2
    pb = rng.random((25, 40)) < 0.3
    a = csr_from_pattern(pa, np.ones(pa.shape))
    b = csr_from_pattern(pb, np.ones(pb.shape))
    expect = pa.astype(np.int64) @ pb.sum(axis=1).astype(np.int64)
    assert np.array_equal(oracle.row_flop(a, b), expect)


def test_rows_to_threads_hand_examples():
    # prefix sums 0,1,2,3,4; average 2 per thread -> thread 1 starts at row 2
    assert oracle.rows_to_threads(np.array([1, 1, 1, 1]), 2).tolist() == [0, 2, 4]
    # prefix 0,5,5,5,6,7,8; average 4 -> first prefix >= 4 is at row 1
    assert oracle.rows_to_threads(np.array([5, 0, 0, 1, 1, 1]), 2).tolist() == [0, 1, 6]
    # all-zero flop: every boundary is row 0
    assert oracle.rows_to_threads(np.zeros(3, np.int64), 3).tolist() == [0, 0, 0, 3]


# ---------------------------------------------------------------- products

def test_hand_worked_product():
    # row 0 = 1*B[0] + 2*B[2] = [0,4,0] + [14,0,0]; row 1 empty; row 2 = 3*B[1] = [15,0,18]
    a = csr_from_dense(np.array([[1, 0, 2], [0, 0, 0], [0, 3, 0]], dtype=np.int64))
    b = csr_from_dense(np.array([[0, 4, 0], [5, 0, 6], [7, 0, 0]], dtype=np.int64))
    c, _ = oracle.spgemm(a, b)
    assert c.row_ptr.tolist() == [0, 2, 2, 4]
    assert c.col_idx.tolist() == [0, 1, 0, 2]
    assert c.vals.tolist() == [14, 4, 15, 18]
    cf, absb = oracle.spgemm(a.astype(np.float64), b.astype(np.float64))
    assert cf.vals.tolist() == [14.0, 4.0, 15.0, 18.0]
    assert absb.tolist() == [14.0, 4.0, 15.0, 18.0]


def test_structural_zero_is_kept():
    # 1*1 + 1*(-1) = 0, but the entry is structurally present (inserted on presence).
    a = CSR(1, 2, np.array([0, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, 1.0]))
    b = CSR(2, 1, np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([1.0, -1.0]))
    c, absb = oracle.spgemm(a, b)
    assert c.nnz == 1 and c.vals[0] == 0.0 and absb[0] == 2.0
    assert oracle.symbolic(a, b).tolist() == [1]


@pytest.mark.parametrize("seed", range(12))
def test_dense_parity_int64(seed):
    rng = np.random.default_rng(100 + seed)
    m, n, k = rng.integers(1, 40, size=3)
    pa = rng.random((m, n)) < rng.uniform(0.05, 0.6)
    pb = rng.random((n, k)) < rng.uniform(0.05, 0.6)
    va = rng.integers(-9, 10, size=(m, n))
    vb = rng.integers(-9, 10, size=(n, k))
    a = csr_from_pattern(pa, va)
    b = csr_from_pattern(pb, vb)
    c, _ = oracle.spgemm(a, b)
    expect_pattern = (pa.astype(np.int64) @ pb.astype(np.int64)) > 0
    assert np.array_equal(pattern_of(c), expect_pattern)
    expect_vals = (np.where(pa, va, 0) @ np.where(pb, vb, 0)).astype(np.int64)
    assert np.array_equal(to_dense(c), np.where(expect_pattern, expect_vals, 0))
    assert_rows_sorted_unique(c)
    assert np.array_equal(oracle.symbolic(a, b), expect_pattern.sum(axis=1))


@pytest.mark.parametrize("seed", range(8))
def test_dense_parity_f64(seed):
    rng = np.random.default_rng(200 + seed)
    m, n, k = rng.integers(1, 48, size=3)
    pa = rng.random((m, n)) < 0.3
    pb = rng.random((n, k)) < 0.3
    va = rng.uniform(-1, 1, size=(m, n))
    vb = rng.uniform(-1, 1, size=(n, k))
    a = csr_from_pattern(pa, va)
    b = csr_from_pattern(pb, vb)
    c, absb = oracle.spgemm(a, b)
    da, db = np.where(pa, va, 0.0), np.where(pb, vb, 0.0)
    expect = da @ db
    scale = np.abs(da) @ np.abs(db)
    got = to_dense(c)
    pat = pattern_of(c)
    assert np.array_equal(pat, (pa.astype(int) @ pb.astype(int)) > 0)
    assert np.all(np.abs(got - expect) <= 1e-13 * scale + 1e-300)
    got_abs = to_dense(c.with_vals(absb))
    assert np.all(np.abs(got_abs - scale) <= 1e-13 * scale)


def test_bruteforce_all_01_3x3_pairs():
    # Every 0/1 pattern pair (2^9 x 2^9).  Values carry the position so that a
    # transposed operand or a swapped index shows up: a_ij = 1 + 3i + j, b_ij = 10 + 3i + j.
    pats = ((np.arange(512)[:, None] >> np.arange(9)) & 1).astype(bool).reshape(512, 3, 3)
    wa = (1 + np.arange(9)).reshape(3, 3)
    wb = (10 + np.arange(9)).reshape(3, 3)
    stacked = pats.reshape(512 * 3, 3)
    a = csr_from_pattern(stacked, np.tile(wa, (512, 1)))
    da = np.where(pats, wa, 0)                       # (512, 3, 3)
    for q in range(512):
        pb = pats[q]
        b = csr_from_pattern(pb, wb)
        c, _ = oracle.spgemm(a, b)
        expect = np.einsum("pij,jk->pik", da, np.where(pb, wb, 0)).reshape(512 * 3, 3)
        expect_pat = (np.einsum("pij,jk->pik", pats.astype(int), pb.astype(int)) > 0).reshape(512 * 3, 3)
        assert np.array_equal(pattern_of(c), expect_pat)
        assert np.array_equal(to_dense(c), expect)


def test_int64_wraps_modulo_2_64():
    a = CSR(1, 2, np.array([0, 2], np.int32), np.array([0, 1], np.int32),
            np.array([2 ** 62, 3], dtype=np.int64))
    b = CSR(2, 1, np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32),
            np.array([4, -5], dtype=np.int64))
    c, _ = oracle.spgemm(a, b)
    expect = (2 ** 62 * 4 + 3 * -5) % 2 ** 64
    expect = expect - 2 ** 64 if expect >= 2 ** 63 else expect
    assert int(c.vals[0]) == expect == -15


def test_empty_shapes():
    z = CSR(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    c, _ = oracle.spgemm(z, z)
    assert c.nrows == 0 and c.nnz == 0
    a = CSR(3, 0, np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0))
    b = CSR(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    c, _ = oracle.spgemm(a, b)
    assert c.row_ptr.tolist() == [0, 0, 0, 0] and c.ncols == 5


def test_out_of_range_index_is_rejected():
    a = CSR(1, 2, np.array([0, 1], np.int32), np.array([2], np.int32), np.ones(1))
    b = CSR(2, 2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32), np.ones(2))
    with pytest.raises(ValueError):
        oracle.spgemm(a, b)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n,k", [(4096, 8), (512, 3), (64, 32)])
def test_er_exact_closed_forms(n, k):
    a = inputs.er_exact(n, k, seed=inputs.SEED_BASE)
    rl = np.diff(a.row_ptr)
    assert np.all(rl == k)
    for i in range(0, n, max(1, n // 64)):
        seg = a.col_idx[a.row_ptr[i]:a.row_ptr[i + 1]]
        assert len(np.unique(seg)) == k
    flop = oracle.row_flop(a, a)
    assert np.all(flop == k * k) and flop.sum() == n * k * k
    c, _ = oracle.spgemm(a, a)
    nnz = np.diff(c.row_ptr)
    assert np.all(nnz <= min(k * k, n)) and np.all(nnz >= k)
    assert c.nnz <= flop.sum()
    assert_rows_sorted_unique(c)


def amg_nnz_closed_form(g: int) -> int:
    e = g - 2 if g % 2 == 0 else g - 1
    return g ** 3 + 3 * g * g * e


@pytest.mark.parametrize("g", [2, 3, 5, 6, 8, 9])
def test_amg_closed_forms(g):
    a = inputs.poisson7(g)
    p = inputs.aggregation(g)
    assert a.nnz == 7 * g ** 3 - 6 * g ** 2
    flop = oracle.row_flop(a, p)
    assert flop.sum() == 7 * g ** 3 - 6 * g ** 2      # P has exactly one entry per row
    c, _ = oracle.spgemm(a, p)
    assert c.nnz == amg_nnz_closed_form(g)
    # C*1 = A*(P*1) = A*1 exactly (small integers); interior rows sum to zero.
    csum = np.add.reduceat(c.vals, c.row_ptr[:-1]) if c.nnz else np.zeros(c.nrows)
    csum[np.diff(c.row_ptr) == 0] = 0
    asum = np.add.reduceat(a.vals, a.row_ptr[:-1])
    assert np.array_equal(csum, asum)


# ---------------------------------------------------------------- invariants

def _spmv(c: CSR, x: np.ndarray) -> np.ndarray:
    rows = np.repeat(np.arange(c.nrows), np.diff(c.row_ptr))
    out = np.zeros(c.nrows, dtype=np.result_type(c.vals, x))
    np.add.at(out, rows, c.vals * x[c.col_idx])
    return out


def test_freivalds_int64_exact():
    a = inputs.rmat(10, 8, seed=7, kind="ints", dtype=np.int64)
    c, _ = oracle.spgemm(a, a)
    x = np.random.default_rng(0).integers(-50, 50, size=a.ncols)
    assert np.array_equal(_spmv(c, x), _spmv(a, _spmv(a, x)))
    # 1^T C = (1^T A) B
    rows_c = np.zeros(c.ncols, np.int64)
    np.add.at(rows_c, c.col_idx, c.vals)
    ya = np.zeros(a.ncols, np.int64)
    np.add.at(ya, a.col_idx, a.vals)
    yb = np.zeros(a.ncols, np.int64)
    np.add.at(yb, a.col_idx, np.repeat(ya, np.diff(a.row_ptr)) * a.vals)
    assert np.array_equal(rows_c, yb)


def test_freivalds_f64_within_bound():
    a = inputs.rmat(10, 8, seed=8)
    c, absb = oracle.spgemm(a, a)
    x = np.random.default_rng(1).uniform(-1, 1, size=a.ncols)
    lhs = _spmv(c, x)
    rhs = _spmv(a, _spmv(a, x))
    absa = a.with_vals(np.abs(a.vals))
    bound = _spmv(absa, _spmv(absa, np.abs(x)))
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * bound + 1e-300)


def test_scipy_crosscheck_rmat():
    sp = pytest.importorskip("scipy.sparse")
    a = inputs.rmat(11, 16, seed=9, kind="ones")
    c, _ = oracle.spgemm(a, a)
    sa = sp.csr_matrix((a.vals, a.col_idx, a.row_ptr), shape=(a.nrows, a.ncols))
    sc = (sa @ sa).tocsr()
    sc.sort_indices()
    assert np.array_equal(sc.indptr, c.row_ptr) and np.array_equal(sc.indices, c.col_idx)
    assert np.array_equal(sc.data, c.vals)          # positive integers: exact
    flop = oracle.row_flop(a, a).sum()
    assert c.nnz <= flop


def test_unsorted_inputs_and_relabelled_columns():
    a = inputs.rmat(9, 8, seed=10)
    c, _ = oracle.spgemm(a, a)
    # shuffling the stored order inside rows changes nothing but rounding
    s = inputs.shuffle_rows(a, seed=11)
    cs, absb = oracle.spgemm(s, s)
    assert np.array_equal(cs.row_ptr, c.row_ptr) and np.array_equal(cs.col_idx, c.col_idx)
    assert np.all(np.abs(cs.vals - c.vals) <= 1e-12 * absb)
    # relabelling B's columns by pi relabels C's columns by pi
    pi = inputs.column_permutation(a.ncols, seed=12)
    bp = inputs.relabel_columns(a, pi)
    cp, _ = oracle.spgemm(a, bp)
    assert np.array_equal(cp.row_ptr, c.row_ptr)
    for i in range(c.nrows):
        lo, hi = c.row_ptr[i], c.row_ptr[i + 1]
        order = np.argsort(pi[c.col_idx[lo:hi]])
        assert np.array_equal(cp.col_idx[lo:hi], pi[c.col_idx[lo:hi]][order])
        assert np.array_equal(cp.vals[lo:hi], c.vals[lo:hi][order])


def test_multithreaded_matches_single():
    a = inputs.rmat(12, 16, seed=13)
    c1, b1 = oracle.spgemm(a, a, nthreads=1)
    c4, b4 = oracle.spgemm(a, a, nthreads=4)
    assert np.array_equal(c1.row_ptr, c4.row_ptr) and np.array_equal(c1.col_idx, c4.col_idx)
    assert np.array_equal(c1.vals, c4.vals) and np.array_equal(b1, b4)
    ai = a.with_vals(inputs.values(a.nnz, 3, "ints"))
    d1, _ = oracle.spgemm(ai, ai, nthreads=1)
    d3, _ = oracle.spgemm(ai, ai, nthreads=3)
    assert np.array_equal(d1.vals, d3.vals)


def test_selected_rows_match_full_product():
    a = inputs.rmat(10, 16, seed=14)
    c, absb = oracle.spgemm(a, a)
    rows = np.array([5, 0, 1023, 17, 17])
    s, sabs = oracle.spgemm_rows(a, a, rows)
    for t, i in enumerate(rows):
        assert np.array_equal(s.col_idx[s.row_ptr[t]:s.row_ptr[t + 1]], c.col_idx[c.row_ptr[i]:c.row_ptr[i + 1]])
        assert np.array_equal(s.vals[s.row_ptr[t]:s.row_ptr[t + 1]], c.vals[c.row_ptr[i]:c.row_ptr[i + 1]])


# ---------------------------------------------------------------- generators

def test_generators_shapes():
    r = inputs.rmat(8, 4, seed=1)
    assert r.nrows == r.ncols == 256 and 0 < r.nnz <= 4 * 256
    assert r.col_idx.min() >= 0 and r.col_idx.max() < 256
    assert np.all(np.abs(r.vals) < 1.0)
    f = inputs.frontier(1000, 64, seed=2)
    per_col = np.bincount(f.col_idx, minlength=64)
    assert per_col.min() >= 1 and per_col.max() <= 4
    # determinism: same seed, same matrix
    r2 = inputs.rmat(8, 4, seed=1)
    assert np.array_equal(r.col_idx, r2.col_idx) and np.array_equal(r.vals, r2.vals)
    # G500 skew: row 0 gets the most mass for a=0.57
    big = inputs.rmat(12, 16, seed=3)
    rl = np.diff(big.row_ptr)
    assert rl[0] == rl.max()


# ---------------------------------------------------------------- triangle counting L*U (Sec. 5.6)

def _triangles_from_lu(L, U, G):
    """sum over stored g_ij of (L*U)_ij, halved: each triangle a < b < c has
    its wedge b-a-c counted at (b, c) and (c, b)."""
    C, _ = oracle.spgemm(L, U)
    dense_c = np.zeros((G.nrows, G.nrows))
    rows = np.repeat(np.arange(C.nrows), np.diff(C.row_ptr))
    dense_c[rows, C.col_idx] = C.vals
    grow = np.repeat(np.arange(G.nrows), np.diff(G.row_ptr))
    return dense_c[grow, G.col_idx].sum() / 2, C


def test_triangle_count_from_lu_equals_trace_of_cube():
    """Pinned by dense linear algebra: trace(G^3) / 6 counts the triangles
    of an undirected simple graph."""
    L, U, G = inputs.triangle_lu(9, 8, seed=601)
    tri, _ = _triangles_from_lu(L, U, G)
    d = np.zeros((G.nrows, G.nrows))
    d[np.repeat(np.arange(G.nrows), np.diff(G.row_ptr)), G.col_idx] = 1.0
    assert np.array_equal(d, d.T) and not d.diagonal().any()
    assert tri == np.trace(d @ d @ d) / 6
    assert tri > 100


def test_lu_of_the_complete_graph_is_min_of_the_indices():
    """K_n: (L*U)_ij = #{k < min(i, j)} = min(i, j), stored for i, j >= 1;
    C(n, 3) triangles."""
    n = 12
    rows, cols = np.nonzero(~np.eye(n, dtype=bool))
    rp, ci = inputs.from_coo(n, n, rows, cols)
    G = inputs.CSR(n, n, rp, ci, np.ones(len(ci)))
    G = inputs.permute_symmetric(G, inputs.degree_order(G))
    L, U = inputs.triangular_split(G)
    tri, C = _triangles_from_lu(L, U, G)
    assert tri == n * (n - 1) * (n - 2) / 6
    assert C.nnz == (n - 1) * (n - 1)
    r = np.repeat(np.arange(n), np.diff(C.row_ptr))
    assert np.array_equal(C.vals, np.minimum(r, C.col_idx).astype(float))


def test_lu_of_a_star_has_one_entry():
    """A star on n vertices has no triangle; ordered by degree its centre is
    last, and (L*U) holds only (centre, centre) = n - 1."""
    n = 9
    rows = np.concatenate([np.zeros(n - 1, np.int64), np.arange(1, n)])
    cols = np.concatenate([np.arange(1, n), np.zeros(n - 1, np.int64)])
    rp, ci = inputs.from_coo(n, n, rows, cols)
    G = inputs.CSR(n, n, rp, ci, np.ones(len(ci)))
    order = inputs.degree_order(G)
    assert order[-1] == 0
    G = inputs.permute_symmetric(G, order)
    L, U = inputs.triangular_split(G)
    tri, C = _triangles_from_lu(L, U, G)
    assert tri == 0
    assert C.nnz == 1 and C.col_idx[0] == n - 1 and C.vals[0] == n - 1
    assert np.diff(C.row_ptr)[n - 1] == 1


def test_degree_order_and_split():
    L, U, G = inputs.triangle_lu(8, 8, seed=602)
    deg = np.diff(G.row_ptr)
    assert np.all(np.diff(deg) >= 0)
    assert L.nnz == U.nnz == G.nnz // 2
    for M, lower in ((L, True), (U, False)):
        r = np.repeat(np.arange(M.nrows), np.diff(M.row_ptr))
        assert np.all(M.col_idx < r) if lower else np.all(M.col_idx > r)
    # U is L transposed
    lt = sorted(zip(L.col_idx.tolist(), np.repeat(np.arange(L.nrows), np.diff(L.row_ptr)).tolist()))
    ut = list(zip(np.repeat(np.arange(U.nrows), np.diff(U.row_ptr)).tolist(), U.col_idx.tolist()))
    assert lt == ut


def test_duplicate_columns_are_summed_like_the_dense_product():
    """Duplicate columns inside input rows (a precondition violation) are
    summed: the result equals the dense product of the duplicate-summed
    matrices, and each output column appears once."""
    rng = np.random.default_rng(141)
    for _ in range(20):
        m, n, k = rng.integers(1, 12, 3)
        rows = rng.integers(0, m, 40)
        A = CSR(int(m), int(n), *_coo_to_csr(int(m), rows, rng.integers(0, n, 40)), rng.integers(-3, 4, 40).astype(np.int64))
        rows = rng.integers(0, n, 40)
        B = CSR(int(n), int(k), *_coo_to_csr(int(n), rows, rng.integers(0, k, 40)), rng.integers(-3, 4, 40).astype(np.int64))
        C, _ = oracle.spgemm(A, B)
        assert np.array_equal(_dense(C), _dense(A) @ _dense(B))
        for i in range(C.nrows):
            cs = C.col_idx[C.row_ptr[i]:C.row_ptr[i + 1]]
            assert len(set(cs.tolist())) == len(cs)


def _coo_to_csr(m, rows, cols):
    """Row pointers and columns of (row, col) pairs kept with repeats, rows in order."""
    order = np.argsort(rows, kind="stable")
    rp = np.zeros(m + 1, np.int32)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp).astype(np.int32), cols[order].astype(np.int32)


def _dense(M):
    d = np.zeros((M.nrows, M.ncols), dtype=np.int64)
    for i in range(M.nrows):
        for j in range(M.row_ptr[i], M.row_ptr[i + 1]):
            d[i, M.col_idx[j]] += M.vals[j]
    return d
