"""GPU parity of two paths that change which entries the kernels visit, never
the product: long rows of B taken whole inside bitmap rows of A (their
column bitmaps ORed in the symbolic phase), and the compacted A that leaves
out the stored a_ik whose row of B is empty.

Every case is compared with the CPU oracle element by element (int64
bit-exact, FP within the stated tolerance), sorted and unsorted, and the
plan statistics show that the path under test really ran.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_1804_01698_gb300 import inputs
from paper_1804_01698_gb300.inputs import CSR
from gpu_helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu

DT = {"i64": torch.int64, "f32": torch.float32, "f64": torch.float64}


def int_valued(m: CSR, seed: int, lo=-3, hi=3) -> CSR:
    v = (inputs.draw_bits(seed, 9, np.arange(m.nnz, dtype=np.uint64)) % np.uint64(hi - lo + 1)).astype(np.int64) + lo
    return m.with_vals(v)


def host_vals(m: CSR, dtype) -> CSR:
    return m.astype({torch.int64: np.int64, torch.float32: np.float32, torch.float64: np.float64}[dtype])


def product(A, B, dt, sorted_output, tuning):
    from paper_1804_01698_gb300 import binding as sg
    dA = sg.to_device(A, "cuda", dt)
    dB = dA if B is A else sg.to_device(B, "cuda", dt)
    with sg.Plan(dA, dB, sorted_output, tuning=tuning) as plan:
        plan.symbolic()
        C = plan.numeric()
        st = plan.stats()
    torch.cuda.synchronize()
    assert st["status"] == 0, st
    return C, st


def typed(m: CSR, dt: str, seed: int) -> CSR:
    # f32 and int64 take small integers (exact sums); f64 keeps U(-1, 1)
    return host_vals(m if dt == "f64" else int_valued(m, seed), DT[dt])


@pytest.mark.parametrize("dt", ["f64", "f32", "i64"])
@pytest.mark.parametrize("sorted_output", [True, False])
@pytest.mark.parametrize("long_min", [1, 8, 64])
def test_long_rows_in_bitmap_rows(dt, sorted_output, long_min):
    A = typed(inputs.rmat(12, 16, seed=401), dt, 402)
    C, st = product(A, A, DT[dt], sorted_output, {"long_row_min": long_min, "bitmap_min_bound": 256})
    assert st["sym_bin_rows"][10] + st["sym_bin_rows"][11] > 0       # bitmap rows exist
    assert st["long_rows"] > 0 and st["long_entries"] > 0              # and took long rows of B
    assert_matches_oracle(C, A, A, sorted_output)


def test_long_rows_off_and_default_agree_with_the_oracle():
    A = inputs.rmat(13, 16, seed=403)
    for tuning in ({"long_row_min": -1}, None):
        C, st = product(A, A, torch.float64, True, tuning)
        assert (st["long_rows"] == 0) == (tuning is not None)
        assert_matches_oracle(C, A, A, True)


@pytest.mark.parametrize("dt", ["f64", "i64"])
@pytest.mark.parametrize("shape", ["wide", "parts"])
def test_long_rows_with_wide_and_split_rows(dt, shape):
    """Every row of B long: a heavy row of A whose output exceeds the large
    class's shared array (the ranks beyond it go straight into C), or whose
    flop is large next to its output (split into parts adding into C)."""
    if shape == "wide":
        B = inputs.er_exact(2000, 40, seed=404, ncols=60000)   # row 0 of A: ~44K distinct columns
        rows = np.concatenate([np.zeros(2000, np.int64), [1, 1, 2]])
        cols = np.concatenate([np.arange(2000), [5, 9, 7]])
        m = 3
    else:
        B = inputs.er_exact(20000, 30, seed=405, ncols=5000)   # row 0: 600K products onto <= 5000 columns
        rows = np.concatenate([np.zeros(20000, np.int64), [1, 1, 2]])
        cols = np.concatenate([np.arange(20000), [5, 9, 7]])
        m = 3
    rp, ci = inputs.from_coo(m, B.nrows, rows, cols)
    A = CSR(m, B.nrows, rp, ci, np.random.default_rng(406).uniform(-1, 1, len(ci)))
    A, B = typed(A, dt, 407), typed(B, dt, 408)
    for sorted_output in (True, False):
        C, st = product(A, B, DT[dt], sorted_output, {"long_row_min": 16})
        assert st["long_rows"] == B.nrows
        if shape == "wide":
            assert st["num_bin_rows"][9] == 1                           # large class: the one wide row
            assert int((C.row_ptr[1:] - C.row_ptr[:-1]).max()) > 232448 // 8
        assert_matches_oracle(C, A, B, sorted_output)


@pytest.mark.parametrize("b_order", ["sorted", "shuffled"])
def test_wide_row_with_sorted_and_unsorted_rows_of_b(b_order):
    """A heavy row of A whose output exceeds the large class's shared array
    (its first ranks accumulate in shared memory, the others straight into
    C), with B's rows sorted by column and in shuffled order: both give the
    oracle's C."""
    B = inputs.er_exact(3000, 40, seed=441, ncols=60000)      # row 0 of A: about 52K distinct columns
    if b_order == "shuffled":
        rng = np.random.default_rng(442)
        ci, v = B.col_idx.copy(), B.vals.copy()
        for k in range(B.nrows):
            a, b = B.row_ptr[k], B.row_ptr[k + 1]
            perm = rng.permutation(b - a)
            ci[a:b], v[a:b] = ci[a:b][perm], v[a:b][perm]
        B = CSR(B.nrows, B.ncols, B.row_ptr, ci, v)
    rows = np.concatenate([np.zeros(3000, np.int64), [1, 1, 2]])
    cols = np.concatenate([np.arange(3000), [5, 9, 7]])
    rp, aci = inputs.from_coo(3, B.nrows, rows, cols)
    A = CSR(3, B.nrows, rp, aci, np.random.default_rng(443).uniform(-1, 1, len(aci)))
    for sorted_output in (True, False):
        C, st = product(A, B, torch.float64, sorted_output, None)
        assert st["num_bin_rows"][9] == 1                               # large class: the one wide row
        assert int((C.row_ptr[1:] - C.row_ptr[:-1]).max()) > 232448 // 8
        assert_matches_oracle(C, A, B, sorted_output)


@pytest.mark.parametrize("dt", ["f64", "i64"])
def test_long_rows_with_repeated_columns(dt):
    """Repeated columns inside a row of B (a precondition violation both sides
    sum): the symbolic phase's bitmap OR counts such a column once, as the
    hash tables do, and the numeric phase adds every product."""
    rng = np.random.default_rng(409)
    n, k = 300, 4000
    rows, cols = [], []
    for i in range(n):
        cs = rng.choice(k, 40, replace=False).tolist()
        if i % 4 == 0:
            cs += cs[:5]                                  # five repeated columns
        rows += [i] * len(cs)
        cols += cs
    order = np.lexsort((np.array(cols), np.array(rows)))
    brp = np.zeros(n + 1, np.int32)
    np.add.at(brp, np.array(rows)[order] + 1, 1)
    B = CSR(n, k, np.cumsum(brp).astype(np.int32), np.array(cols, np.int32)[order], rng.uniform(-1, 1, len(cols)))
    arp, aci = inputs.from_coo(4, n, np.repeat(np.arange(4), n), np.tile(np.arange(n), 4))
    A = CSR(4, n, arp, aci, rng.uniform(-1, 1, len(aci)))
    A, B = typed(A, dt, 410), typed(B, dt, 411)
    for sorted_output in (True, False):
        C, st = product(A, B, DT[dt], sorted_output, {"long_row_min": 1})
        assert st["long_rows"] == n
        assert_matches_oracle(C, A, B, sorted_output)


@pytest.mark.parametrize("graph", [False, True])
def test_long_rows_follow_new_values_in_repeated_numeric(graph):
    from paper_1804_01698_gb300 import binding as sg
    A = inputs.rmat(12, 16, seed=412)
    dA = sg.to_device(A)
    with sg.Plan(dA, dA, True, tuning={"long_row_min": 8, "bitmap_min_bound": 256}) as plan:
        plan.symbolic()
        C = plan.numeric()
        assert plan.stats()["long_rows"] > 0
        for run in range(3):
            A2 = A.with_vals(np.random.default_rng(413 + run).uniform(-1, 1, A.nnz))
            dA.vals.copy_(torch.from_numpy(A2.vals))
            C = plan.numeric_graph(C) if graph else plan.numeric(C.col_idx, C.vals)
            torch.cuda.synchronize()
            assert_matches_oracle(C, A2, A2, True)


@pytest.mark.parametrize("dt", ["f32", "i64"])
@pytest.mark.parametrize("sorted_output", [True, False])
def test_compacted_a_for_frontier_products(dt, sorted_output):
    """A * F with F a BFS-frontier stack (1-4 entries per column): almost every
    row of F is empty, so the phases walk the compacted A."""
    A = typed(inputs.rmat(13, 16, seed=414, dtype=np.float32, kind="ones"), dt, 415)
    F = typed(inputs.frontier(A.ncols, 256, seed=416), dt, 417)
    C, st = product(A, F, DT[dt], sorted_output, None)
    assert st["nnz_a_walked"] < A.nnz // 2
    assert_matches_oracle(C, A, F, sorted_output)


@pytest.mark.parametrize("dt", ["f64", "i64"])
@pytest.mark.parametrize("sorted_output", [True, False])
def test_compacted_a_with_crowded_tiles(dt, sorted_output):
    """B's rows are empty but for its 64 lowest, which R-MAT's hub rows of A
    select again and again: fewer than half of A's entries select a non-empty
    row of B (so A is compacted), while the tiles of the hub rows hold more
    kept entries than the flop pass lists per tile (so the compaction walks
    those tiles again) and hub rows span several tiles."""
    A = typed(inputs.rmat(12, 16, seed=431), dt, 432)
    n = A.ncols
    rows = np.repeat(np.arange(64), 3)
    cols = inputs.draw_bits(433, 7, np.arange(rows.size, dtype=np.uint64)) % np.uint64(n)
    rp, ci = inputs.from_coo(n, n, rows, cols.astype(np.int64))
    Bm = typed(CSR(n, n, rp, ci, np.ones(len(ci))), dt, 434)
    aci = A.col_idx
    kept = int((aci < 64).sum())
    assert 0 < kept < A.nnz // 2
    rp_a = A.row_ptr.astype(np.int64)
    in_first_tile = int((aci[: min(A.nnz, 2048)] < 64).sum())
    assert in_first_tile > 128                      # the first tile's kept entries overflow its list
    C, st = product(A, Bm, DT[dt], sorted_output, None)
    assert st["nnz_a_walked"] == kept
    assert_matches_oracle(C, A, Bm, sorted_output)


def test_compacted_a_follows_new_values():
    from paper_1804_01698_gb300 import binding as sg
    A = inputs.rmat(12, 16, seed=418)
    F = inputs.frontier(A.ncols, 128, seed=419, dtype=np.float64, kind="uniform")
    dA, dF = sg.to_device(A), sg.to_device(F)
    with sg.Plan(dA, dF, False) as plan:
        plan.symbolic()
        C = plan.numeric()
        assert plan.stats()["nnz_a_walked"] < A.nnz // 2
        for run in range(2):
            A2 = A.with_vals(np.random.default_rng(420 + run).uniform(-1, 1, A.nnz))
            dA.vals.copy_(torch.from_numpy(A2.vals))
            C = plan.numeric(C.col_idx, C.vals)
            torch.cuda.synchronize()
            assert_matches_oracle(C, A2, F, False)


@pytest.mark.parametrize("tuning", [{"warp_load_pct": 90, "block_load_pct": 90},
                                    {"warp_load_pct": 10, "block_load_pct": 20},
                                    {"warp_load_pct": 95, "bitmap_min_bound": -1}])
@pytest.mark.parametrize("sorted_output", [True, False])
def test_hash_table_load_factors(tuning, sorted_output):
    A = inputs.rmat(12, 16, seed=421)
    C, st = product(A, A, torch.float64, sorted_output, tuning)
    assert_matches_oracle(C, A, A, sorted_output)
