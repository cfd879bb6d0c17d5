"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Covers every step of the path: the row flop pass (bit-exact), the row bins
(a permutation obeying the bin rule), the symbolic counts and row_ptr
(bit-exact), the numeric values (int64 bit-exact, FP within tolerance) in
sorted and unsorted mode, on the named workloads at full size and on edge
cases: empty shapes, empty rows, heavy rows beyond the shared array,
heavy rows on global-memory tables, unsorted inputs, structural zeros,
int64 wrap-around and invalid input.
"""
import json
import hashlib
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1804_01698_gb300 import inputs
from paper_1804_01698_gb300.inputs import CSR
from gpu_helpers import assert_matches_oracle, gpu_product, sort_rows_on_device

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "workloads.json")))
HASH_CAPS = [32, 64, 128, 256, 512, 1536, 3072, 6144, 12288]
DT = {"i64": torch.int64, "f32": torch.float32, "f64": torch.float64}


def int_valued(m: CSR, seed: int, lo=-3, hi=3) -> CSR:
    v = (inputs.draw_bits(seed, 9, np.arange(m.nnz, dtype=np.uint64)) % np.uint64(hi - lo + 1)).astype(np.int64) + lo
    return m.with_vals(v)


def host_vals(m: CSR, dtype) -> CSR:
    return m.astype({torch.int64: np.int64, torch.float32: np.float32, torch.float64: np.float64}[dtype])


# ------------------------------------------------------------ a1, a2, a3, a4

def expected_sym_bin(bound: int, k: int):
    """The documented symbolic bin rule: hash bins by key bound, column bitmaps
    for rows above max(512, ceil(k/32)/2) when B has at most 2^18 columns,
    global tables above the largest shared-memory table otherwise."""
    if bound <= 0:
        return None
    if k <= 1 << 18 and bound > max(512, (k + 31) // 32 // 2):
        return 10 if bound > 24576 else 11
    for b, cap in enumerate(HASH_CAPS):
        if bound <= cap:
            return b
    return 9 if bound <= 24576 else 12


@pytest.mark.parametrize("name", ["er", "rmat", "tall"])
def test_flop_bins_counts_rowptr(name):
    from paper_1804_01698_gb300 import binding as sg
    if name == "er":
        A = B = inputs.er_exact(4096, 8, seed=1)
    elif name == "rmat":
        A = B = inputs.rmat(13, 16, seed=2)
    else:
        A = inputs.rmat(14, 16, seed=3, kind="ones")
        B = inputs.frontier(A.ncols, 1024, seed=3, kind="ones", dtype=np.float64)
    dA, dB = sg.to_device(A), sg.to_device(B)
    with sg.Plan(dA, dB, True) as plan:
        flop = plan.row_flop().cpu().numpy()
        ref_flop = oracle.row_flop(A, B)
        assert np.array_equal(flop, ref_flop)                                  # a1 bit-exact
        perm, offs = plan.sym_bins()
        perm = perm.cpu().numpy()
        bound = np.minimum(ref_flop, B.ncols)
        assert sorted(perm.tolist()) == np.nonzero(bound > 0)[0].tolist()     # a2: a permutation
        expect = np.array([-1 if b is None else b for b in (expected_sym_bin(int(x), B.ncols) for x in bound)])
        for b in range(len(offs) - 1):                                        # a2: the bin rule
            rows = perm[offs[b]:offs[b + 1]]
            assert np.all(expect[rows] == b), b
            assert len(rows) == int((expect == b).sum()), b
        nnz_c = plan.symbolic()
        ref_nnz = oracle.symbolic(A, B)
        assert np.array_equal(plan.row_nnz().cpu().numpy(), ref_nnz)          # a3 bit-exact
        rp = plan.c_row_ptr.cpu().numpy()
        assert rp[0] == 0 and np.array_equal(np.diff(rp), ref_nnz)            # a4 bit-exact
        assert nnz_c == ref_nnz.sum()
        st = plan.stats()
        assert st["total_flop"] == ref_flop.sum() and st["max_row_flop"] == ref_flop.max()
        assert st["status"] == 0


# ------------------------------------------------------------ a5, a6: named workloads at full size

def _golden_check(C, name):
    g = GOLDEN[name]
    rp = C.row_ptr.cpu().numpy()
    ci, _ = sort_rows_on_device(C)
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(rp, dtype=np.int32).tobytes())
    h.update(np.ascontiguousarray(ci.cpu().numpy(), dtype=np.int32).tobytes())
    assert int(rp[-1]) == g["nnz_c"]
    assert h.hexdigest() == g["c_structure_sha256"]


def test_er4096_sorted_f64():
    A, B, _ = inputs.workload("er4096_k8_f64")
    C, stats = gpu_product(A, B, torch.float64, True)
    assert stats["total_flop"] == 4096 * 64
    assert_matches_oracle(C, A, B, True)
    _golden_check(C, "er4096_k8_f64")


@pytest.fixture(scope="module")
def rmat16():
    A, B, _ = inputs.workload("rmat16_ef16_f64")
    return A, B, oracle.spgemm(A, B, nthreads=os.cpu_count() or 8)


@pytest.mark.parametrize("sorted_output", [True, False])
def test_rmat16_f64(rmat16, sorted_output):
    A, B, expect = rmat16
    C, stats = gpu_product(A, B, torch.float64, sorted_output)
    assert stats["total_flop"] == GOLDEN["rmat16_ef16_f64"]["total_flop"]
    # every kind of bin takes part: hash bins, both bitmap bins, all three
    # bitmap item classes (small, medium, large)
    # (rows of bound above 1024 = 2048 bitmap words / 2 take bitmaps)
    assert all(stats["sym_bin_rows"][b] > 0 for b in range(6))
    assert stats["sym_bin_rows"][10] > 0 and stats["sym_bin_rows"][11] > 0
    assert all(stats["num_bin_rows"][b] > 0 for b in range(6))
    assert all(stats["num_bin_rows"][b] > 0 for b in (9, 11, 12))
    assert sum(stats["num_bin_flop"]) == stats["total_flop"]
    assert_matches_oracle(C, A, B, sorted_output, expect=expect)
    _golden_check(C, "rmat16_ef16_f64")


def test_rmat18_frontier_f32_and_int64():
    A, B, _ = inputs.workload("rmat18_frontier1024_f32")
    expect = oracle.spgemm(A, B, nthreads=os.cpu_count() or 8)
    C, _ = gpu_product(A, B, torch.float32, False)
    assert_matches_oracle(C, A, B, False, expect=expect)
    _golden_check(C, "rmat18_frontier1024_f32")
    Ai, Bi = A.astype(np.int64), B.astype(np.int64)
    Ci, _ = gpu_product(Ai, Bi, torch.int64, False)
    assert_matches_oracle(Ci, Ai, Bi, False)


# ------------------------------------------------------------ value types x modes on mid-size inputs

@pytest.mark.parametrize("dt", ["i64", "f32", "f64"])
@pytest.mark.parametrize("sorted_output", [True, False])
@pytest.mark.parametrize("shape", ["rmat12", "er", "rect"])
def test_dtypes_modes(dt, sorted_output, shape):
    dtype = DT[dt]
    if shape == "rmat12":
        A = inputs.rmat(12, 16, seed=21)
        B = A
    elif shape == "er":
        A = inputs.er_exact(3000, 11, seed=22, ncols=5000)
        B = inputs.er_exact(5000, 7, seed=23, ncols=777)
    else:  # ragged rectangular product, rows of very different lengths
        A = inputs.rmat(11, 24, seed=24, abcd=(0.45, 0.25, 0.15, 0.15))
        A = CSR(A.nrows, A.ncols, A.row_ptr, A.col_idx, A.vals)
        B = inputs.er_exact(A.ncols, 5, seed=25, ncols=3001)
    if dt != "f64":  # small integers: exact in float32 and int64
        A, B = int_valued(A, 31), int_valued(B, 32)
    A, B = host_vals(A, dtype), host_vals(B, dtype)
    C, _ = gpu_product(A, B, dtype, sorted_output)
    assert_matches_oracle(C, A, B, sorted_output)


def test_float32_uniform_values_within_tolerance():
    A = inputs.er_exact(2048, 8, seed=41, dtype=np.float32)
    C, _ = gpu_product(A, A, torch.float32, True)
    assert_matches_oracle(C, A, A, True)


# ------------------------------------------------------------ heavy rows

def _heavy_rows(nrows_a, entries, ncols_b, b_row_len, seed):
    """A: nrows_a rows of `entries` distinct columns; B: rows of b_row_len random columns."""
    A = inputs.er_exact(nrows_a, entries, seed=seed, ncols=entries * 4)
    B = inputs.er_exact(entries * 4, b_row_len, seed=seed + 1, ncols=ncols_b)
    return A, B


# More FP64 values than any block's shared memory holds (227 KB per block).
SHARED_F64_MAX = 232448 // 8


def _widest_row(C) -> int:
    return int((C.row_ptr[1:] - C.row_ptr[:-1]).max())


@pytest.mark.parametrize("dt", ["f64", "i64"])
def test_bitmap_rows_beyond_the_shared_array(dt):
    """Rows with more entries than the large class's shared array: the first
    ranks accumulate in shared memory, the others straight into C."""
    dtype = DT[dt]
    A, B = _heavy_rows(6, 64, 65536, 1000, seed=61)     # ~40k entries per row
    if dt == "i64":
        A, B = int_valued(A, 62), int_valued(B, 63)
    A, B = host_vals(A, dtype), host_vals(B, dtype)
    C, st = gpu_product(A, B, dtype, True)
    assert st["sym_bin_rows"][10] == 6 and st["num_bin_rows"][9] == 6   # one work item per row
    assert _widest_row(C) > SHARED_F64_MAX
    assert_matches_oracle(C, A, B, True)


@pytest.mark.parametrize("b_order", ["sorted", "shuffled"])
@pytest.mark.parametrize("shape", ["wide", "wide_and_parts"])
def test_wide_rows_with_sorted_and_unsorted_b(b_order, shape):
    """Rows beyond the shared array, with column-sorted and with shuffled rows
    of B, and such rows also split into parts of their stored a_ik (every
    part adds its shared ranks and its other ranks into C)."""
    if shape == "wide":
        A, B = _heavy_rows(6, 64, 65536, 1000, seed=71)      # ~40k entries per row
    else:
        A, B = _heavy_rows(2, 2048, 65536, 1000, seed=72)    # ~65k entries, 2M flop: also parts
    if b_order == "shuffled":
        B = inputs.shuffle_rows(B, seed=73)
    C, st = gpu_product(A, B, torch.float64, True)
    assert _widest_row(C) > SHARED_F64_MAX
    if shape == "wide":
        assert st["num_bin_rows"][9] == A.nrows
    else:
        assert st["num_bin_rows"][9] > A.nrows
    assert_matches_oracle(C, A, B, True)


@pytest.mark.parametrize("sorted_output", [True, False])
@pytest.mark.parametrize("dt", ["f64", "i64", "f32"])
def test_global_table_rows(sorted_output, dt):
    dtype = DT[dt]
    # 2^20 columns: too many for bitmaps; flop 40k per row -> global tables;
    # plus rows of flop ~20k -> the 32768-slot block bin.
    A1, B1 = _heavy_rows(5, 40, 1 << 20, 1000, seed=71)
    A2 = inputs.er_exact(7, 20, seed=73, ncols=160)
    A = CSR(12, 160, np.concatenate([A1.row_ptr, A2.row_ptr[1:] + A1.nnz]).astype(np.int32),
            np.concatenate([A1.col_idx, A2.col_idx]), np.concatenate([A1.vals, A2.vals]))
    B = B1
    if dt != "f64":
        A, B = int_valued(A, 74), int_valued(B, 75)
    A, B = host_vals(A, dtype), host_vals(B, dtype)
    C, st = gpu_product(A, B, dtype, sorted_output)
    assert st["sym_bin_rows"][12] == 5 and st["sym_bin_rows"][9] == 7
    assert st["num_bin_rows"][10] >= 5
    assert_matches_oracle(C, A, B, sorted_output)


# ------------------------------------------------------------ edge cases

def _csr(m, n, rows):
    rp = np.zeros(m + 1, np.int32)
    cols, vals = [], []
    for i, r in enumerate(rows):
        rp[i + 1] = rp[i] + len(r)
        cols += [c for c, _ in r]
        vals += [v for _, v in r]
    return CSR(m, n, rp, np.array(cols, np.int32), np.array(vals, np.float64))


@pytest.mark.parametrize("shape", [(0, 5, 3), (4, 0, 3), (4, 5, 0), (3, 3, 3)])
def test_empty_shapes(shape):
    m, n, k = shape
    A = CSR(m, n, np.zeros(m + 1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = CSR(n, k, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    for one_shot in (False, True):
        C, _ = gpu_product(A, B, torch.float64, True, one_shot=one_shot)
        assert C.nrows == m and C.nnz == 0
        assert np.array_equal(C.row_ptr.cpu().numpy(), np.zeros(m + 1, np.int32))


def test_empty_rows_and_structural_zero():
    A = _csr(4, 3, [[], [(0, 1.0), (1, 1.0)], [], [(2, 2.0)]])
    B = _csr(3, 2, [[(0, 1.0)], [(0, -1.0)], [(1, 3.0)]])
    C, _ = gpu_product(A, B, torch.float64, True)
    assert C.row_ptr.cpu().tolist() == [0, 0, 1, 1, 2]
    assert C.col_idx.cpu().tolist() == [0, 1]
    assert C.vals.cpu().tolist() == [0.0, 6.0]          # 1*1 + 1*(-1) kept as a stored zero


def test_int64_wraps_like_the_oracle():
    A = CSR(1, 2, np.array([0, 2], np.int32), np.array([0, 1], np.int32), np.array([2 ** 62, 3], np.int64))
    B = CSR(2, 1, np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([4, -5], np.int64))
    C, _ = gpu_product(A, B, torch.int64, True)
    assert C.vals.cpu().tolist() == [-15]


def test_unsorted_inputs_give_the_same_product():
    A = inputs.rmat(12, 16, seed=81)
    S = inputs.shuffle_rows(A, seed=82)
    expect = oracle.spgemm(A, A, nthreads=8)
    for sorted_output in (True, False):
        C, _ = gpu_product(S, S, torch.float64, sorted_output)
        assert_matches_oracle(C, S, S, sorted_output, expect=expect)


def test_one_shot_entry_point():
    A = inputs.rmat(11, 16, seed=91)
    C, _ = gpu_product(A, A, torch.float64, True, one_shot=True)
    assert_matches_oracle(C, A, A, True)


def test_tiny_random_products_against_oracle():
    rng = np.random.default_rng(5)
    for t in range(25):
        m, n, k = (int(x) for x in rng.integers(1, 70, size=3))
        A = CSR(m, n, *_rand_csr(rng, m, n))
        B = CSR(n, k, *_rand_csr(rng, n, k))
        for dt in (torch.int64, torch.float64):
            Ah = A if dt == torch.float64 else int_valued(A, t)
            Bh = B if dt == torch.float64 else int_valued(B, t + 100)
            C, _ = gpu_product(host_vals(Ah, dt), host_vals(Bh, dt), dt, bool(t % 2))
            assert_matches_oracle(C, host_vals(Ah, dt), host_vals(Bh, dt), bool(t % 2))


def _rand_csr(rng, m, n):
    dens = rng.uniform(0.0, 0.5)
    mask = rng.random((m, n)) < dens
    rp = np.zeros(m + 1, np.int32)
    rp[1:] = np.cumsum(mask.sum(1))
    r, c = np.nonzero(mask)
    return rp, c.astype(np.int32), rng.uniform(-1, 1, size=len(c))


@pytest.mark.parametrize("where", ["A", "B"])
def test_out_of_range_column_is_an_error_not_a_fault(where):
    from paper_1804_01698_gb300 import binding as sg
    A = inputs.er_exact(64, 4, seed=101)
    B = inputs.er_exact(64, 4, seed=102)
    bad = (A if where == "A" else B)
    ci = bad.col_idx.copy()
    ci[7] = 64 + 5                                   # one column past the end
    bad = CSR(bad.nrows, bad.ncols, bad.row_ptr, ci, bad.vals)
    A, B = (bad, B) if where == "A" else (A, bad)
    dA, dB = sg.to_device(A), sg.to_device(B)
    with pytest.raises(sg.SpgemmError) as ei:
        with sg.Plan(dA, dB, True) as plan:
            plan.symbolic()
    assert ei.value.status == -2                     # SPGEMM_ERR_INVALID_CSR
    # the context is still usable
    C, _ = gpu_product(inputs.er_exact(64, 4, seed=103), inputs.er_exact(64, 4, seed=104), torch.float64, True)
    assert C.nnz > 0


@pytest.mark.parametrize("sorted_output", [True, False])
def test_block_rows_wider_than_the_sort_window(sorted_output):
    # ~1200 products per row: block bins.  B has 2^20 columns and half of each
    # row's entries spread over all of them, so every row of C spans far more
    # than the 131072-column window of the bitmap sort: the bitonic fallback.
    A = inputs.er_exact(300, 30, seed=121, ncols=400)
    B1 = inputs.er_exact(400, 40, seed=122, ncols=1 << 20)
    narrow = inputs.er_exact(400, 40, seed=123, ncols=3000)
    B = CSR(400, 1 << 20, B1.row_ptr, np.where(np.arange(B1.nnz) % 40 < 20, B1.col_idx, narrow.col_idx).astype(np.int32),
            B1.vals)
    C, st = gpu_product(A, B, torch.float64, sorted_output)
    assert sum(st["num_bin_rows"][5:9]) > 0
    assert_matches_oracle(C, A, B, sorted_output)


@pytest.mark.parametrize("far", [False, True])
def test_warp_rows_sorted_by_bucket_rank_and_by_the_fallback(far):
    """Sorted warp-bin rows of 33..256 entries are ranked through buckets of
    the row's column range; a row whose columns crowd one bucket (a cluster
    plus one far column) takes the bitonic network instead.  Both must give
    the oracle's sorted rows."""
    rng = np.random.default_rng(7 if far else 8)
    n, k = 600, 70000
    rows, cols = [], []
    for i in range(n):
        width = 40 + (i % 200)                      # row sizes 40 .. 239 entries
        base = int(rng.integers(0, k - 5000))
        if far:                                      # cluster of `width` consecutive columns + one far column
            cs = list(range(base, base + width)) + [k - 1 - (i % 7)]
        else:                                        # spread over the whole range
            cs = rng.choice(k, size=width, replace=False).tolist()
        rows += [i] * len(cs)
        cols += cs
    rp, ci = inputs.from_coo(n, k, np.array(rows), np.array(cols))
    B = CSR(n, k, rp, ci, rng.uniform(-1, 1, len(ci)))
    A = inputs.er_exact(300, 1, seed=9, ncols=n)     # each row of C is one row of B
    for dt in (torch.float64, torch.int64):
        a, b = (A, B) if dt == torch.float64 else (A.with_vals(np.arange(A.nnz) % 5 - 2),
                                                    B.with_vals(np.arange(B.nnz) % 7 - 3))
        C, stats = gpu_product(a, b, dt, True)
        assert stats["status"] == 0
        assert_matches_oracle(C, a, b, True)


@pytest.mark.parametrize("sorted_output", [True, False])
@pytest.mark.parametrize("dt", ["f64", "i64", "f32"])
def test_heavy_bitmap_row_split_over_blocks(dt, sorted_output):
    """A row whose flop dwarfs its output (600,000 products onto at most
    5,000 columns) is split over several blocks by ranges of its stored
    a_ik; their partial sums meet in C through global atomics.  Lighter
    bitmap rows beside it stay whole."""
    rng = np.random.default_rng(31)
    kb, nb = 5000, 20000
    B = inputs.er_exact(nb, 30, seed=32, ncols=kb)
    rows = [np.full(nb, 0)] + [np.full(50 * r, r) for r in range(1, 8)]
    cols = [np.arange(nb)] + [rng.choice(nb, size=50 * r, replace=False) for r in range(1, 8)]
    rp, ci = inputs.from_coo(8, nb, np.concatenate(rows), np.concatenate(cols))
    A = CSR(8, nb, rp, ci, rng.uniform(-1, 1, len(ci)))
    if dt != "f64":   # small integers: exact in int64 and float32
        A = A.with_vals(rng.integers(-2, 3, A.nnz).astype(np.float64))
        B = B.with_vals(rng.integers(-2, 3, B.nnz).astype(np.float64))
        if dt == "i64":
            A, B = A.astype(np.int64), B.astype(np.int64)
    C, stats = gpu_product(A, B, DT[dt], sorted_output)
    assert stats["status"] == 0
    assert stats["max_row_flop"] == 600000
    assert sum(stats["num_bin_rows"][b] for b in (9, 11, 12)) > 7   # items: the split row counts its parts
    assert_matches_oracle(C, A, B, sorted_output)


@pytest.mark.parametrize("scheme", [("chunk4", "low"), ("linear", "low"), ("chunk4", "high")])
@pytest.mark.parametrize("sorted_output", [True, False])
@pytest.mark.parametrize("dt", ["f64", "i64"])
@pytest.mark.parametrize("shape", ["rmat12", "er", "global"])
def test_chunked_probing_gives_the_same_product(shape, dt, sorted_output, scheme):
    """SPGEMM_PROBE_CHUNK4 (4-slot chunks, Sec. 4.2.2) and SPGEMM_HASH_LOW_BITS
    (the remainder form of Sec. 4.2.1) in every kind of hash table: warp and block tables in shared memory
    (R-MAT, ER) and global tables (B with 2^20 columns)."""
    dtype = DT[dt]
    if shape == "rmat12":
        A = B = inputs.rmat(12, 16, seed=81)
    elif shape == "er":
        A = inputs.er_exact(3000, 11, seed=82, ncols=5000)
        B = inputs.er_exact(5000, 7, seed=83, ncols=777)
    else:
        A, B = _heavy_rows(5, 40, 1 << 20, 1000, seed=84)
    if dt != "f64":
        A, B = int_valued(A, 85), int_valued(B, 86)
    A, B = host_vals(A, dtype), host_vals(B, dtype)
    C, st = gpu_product(A, B, dtype, sorted_output, probe=scheme[0], hash=scheme[1])
    assert st["status"] == 0
    if shape == "global":
        assert st["sym_bin_rows"][12] == 5 and st["num_bin_rows"][10] >= 5
    assert_matches_oracle(C, A, B, sorted_output)


@pytest.mark.parametrize("sorted_output", [True, False])
@pytest.mark.parametrize("dt", ["f64", "i64"])
def test_block_bins_below_the_bitmap_threshold(dt, sorted_output):
    """B with 2^18 columns: rows take bitmaps only above a bound of 4096
    (2^13 words / 2), so rows of bound 600 .. 4000 fill the block hash bins
    of 2048, 4096 and 8192 slots, beside warp-bin and bitmap rows."""
    k = 1 << 18
    B = inputs.er_exact(3000, 20, seed=95, ncols=k)
    rng = np.random.default_rng(96)
    degs = [30, 60, 100, 150, 200, 2, 10, 400] * 6          # flop 20 * deg
    rows = np.concatenate([np.full(d, i) for i, d in enumerate(degs)])
    cols = np.concatenate([rng.choice(3000, size=d, replace=False) for d in degs])
    rp, ci = inputs.from_coo(len(degs), 3000, rows, cols)
    A = CSR(len(degs), 3000, rp, ci, rng.uniform(-1, 1, len(ci)))
    if dt != "f64":
        A, B = int_valued(A, 97), int_valued(B, 98)
    A, B = host_vals(A, DT[dt]), host_vals(B, DT[dt])
    C, st = gpu_product(A, B, DT[dt], sorted_output)
    assert st["status"] == 0
    assert all(st["sym_bin_rows"][b] > 0 for b in (5, 6, 7))
    assert all(st["num_bin_rows"][b] > 0 for b in (5, 6, 7))
    assert st["sym_bin_rows"][11] > 0                      # the rows of bound 8000
    assert_matches_oracle(C, A, B, sorted_output)


@pytest.mark.parametrize("sorted_output", [True, False])
@pytest.mark.parametrize("dt", ["f64", "i64"])
def test_duplicate_columns_in_input_rows_are_summed(dt, sorted_output):
    """Duplicate columns inside an input row break the CSR precondition; both
    the oracle and the GPU sum them (a repeated a_ik repeats its products, a
    repeated b_kj adds twice into one output column).  Light rows (hash
    tables) and heavy rows (bitmaps) both see duplicates."""
    rng = np.random.default_rng(131)
    n, k = 400, 3000

    def with_dups(m, ncols, seed):
        r = np.random.default_rng(seed)
        rows, cols = [], []
        for i in range(m.nrows):
            cs = m.col_idx[m.row_ptr[i]:m.row_ptr[i + 1]].tolist()
            if cs and i % 3 == 0:
                cs = cs + r.choice(cs, size=max(1, len(cs) // 4)).tolist()   # repeat some columns
            rows += [i] * len(cs)
            cols += cs
        order = np.lexsort((np.array(cols), np.array(rows)))
        rp = np.zeros(m.nrows + 1, np.int32)
        np.add.at(rp, np.array(rows)[order] + 1, 1)
        return CSR(m.nrows, ncols, np.cumsum(rp).astype(np.int32), np.array(cols, np.int32)[order],
                   r.uniform(-1, 1, len(cols)))

    A = with_dups(inputs.er_exact(n, 6, seed=132, ncols=n), n, 133)
    heavy = np.zeros(n, bool)
    heavy[:5] = True                                  # five rows of A reach every row of B
    rp = np.concatenate([[0], np.cumsum(np.where(heavy, n, np.diff(A.row_ptr)))]).astype(np.int32)
    ci = np.concatenate([np.arange(n) if heavy[i] else A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]] for i in range(n)])
    A = CSR(n, n, rp, ci.astype(np.int32), rng.uniform(-1, 1, len(ci)))
    B = with_dups(inputs.er_exact(n, 30, seed=134, ncols=k), k, 135)
    if dt != "f64":
        A, B = int_valued(A, 136), int_valued(B, 137)
    A, B = host_vals(A, DT[dt]), host_vals(B, DT[dt])
    C, st = gpu_product(A, B, DT[dt], sorted_output)
    assert st["status"] == 0
    assert st["sym_bin_rows"][10] + st["sym_bin_rows"][11] >= 5     # the heavy rows took bitmaps
    assert_matches_oracle(C, A, B, sorted_output)


def test_product_with_more_than_2_31_flop():
    """R-MAT scale 18 A*A: total flop 2.9e9 (beyond int32), about 1e9 output
    entries, B at the bitmap column limit (2^18).  Every row count is
    compared with the oracle's symbolic phase, and 300 sampled rows (the
    heaviest among them) entry by entry."""
    from paper_1804_01698_gb300 import binding as sg
    A = inputs.rmat(18, 16, seed=141)
    flop = oracle.row_flop(A, A)
    assert int(flop.sum()) > 2**31
    dA = sg.to_device(A)
    with sg.Plan(dA, dA, True) as plan:
        nnz = plan.symbolic()
        C = plan.numeric()
        st = plan.stats()
    torch.cuda.synchronize()
    assert st["status"] == 0
    assert st["total_flop"] == int(flop.sum())
    expect_rows = oracle.symbolic(A, A, nthreads=os.cpu_count() or 8)
    rp = C.row_ptr.cpu().numpy()
    assert np.array_equal(np.diff(rp), expect_rows)
    assert nnz == int(expect_rows.sum())
    rng = np.random.default_rng(142)
    sample = np.unique(np.concatenate([np.argsort(flop)[-20:], rng.choice(A.nrows, 280, replace=False)]))
    ref, absb = oracle.spgemm_rows(A, A, sample, nthreads=os.cpu_count() or 8)
    for t, i in enumerate(sample):
        lo, hi = int(rp[i]), int(rp[i + 1])
        r0, r1 = int(ref.row_ptr[t]), int(ref.row_ptr[t + 1])
        assert hi - lo == r1 - r0
        ci = C.col_idx[lo:hi].cpu().numpy()
        cv = C.vals[lo:hi].cpu().numpy()
        assert np.array_equal(ci, ref.col_idx[r0:r1])
        assert np.all(np.abs(cv - ref.vals[r0:r1]) <= 1e-12 * absb[r0:r1])


@pytest.mark.parametrize("sorted_output", [True, False])
@pytest.mark.parametrize("dt", ["f64", "i64"])
def test_heavy_symbolic_row_split_over_blocks(dt, sorted_output):
    """A heavy bitmap row (bound 65536) with 600,000 products takes four
    symbolic blocks: each ORs its part of the row's columns into the saved
    bitmap and the last one counts them.  Its output (about 65,000 entries)
    then exceeds the numeric large class's shared array."""
    rng = np.random.default_rng(151)
    nb, kb = 20000, 1 << 16
    B = inputs.er_exact(nb, 30, seed=152, ncols=kb)
    rows = [np.zeros(nb, np.int64)] + [np.full(40 * r, r) for r in range(1, 6)]
    cols = [np.arange(nb)] + [rng.choice(nb, size=40 * r, replace=False) for r in range(1, 6)]
    rp, ci = inputs.from_coo(6, nb, np.concatenate(rows), np.concatenate(cols))
    A = CSR(6, nb, rp, ci, rng.uniform(-1, 1, len(ci)))
    if dt != "f64":
        A, B = int_valued(A, 153), int_valued(B, 154)
    A, B = host_vals(A, DT[dt]), host_vals(B, DT[dt])
    C, st = gpu_product(A, B, DT[dt], sorted_output)
    assert st["status"] == 0
    assert st["sym_bin_rows"][10] == 1 and st["max_row_flop"] == 600000
    assert_matches_oracle(C, A, B, sorted_output)
