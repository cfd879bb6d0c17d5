"""spgemm_numeric_rows: the numeric phase of a range of rows of C only.

Rows of C are independent (Fig. "RowWise_SpGEMM"), so one call per range
over disjoint ranges that cover every row must give the oracle's product,
and a call must write nothing outside its own rows.  Each case fills C with
sentinels, computes a middle range first and checks it against the oracle
row by row while every other row still holds its sentinels, then computes
the rest and compares the whole product.  The inputs reach every kind of
numeric kernel whose blocks skip rows outside the range: warp and block
hash rows (R-MAT scale 13), bitmap rows beyond the shared array, in parts, a
bitmap row split over blocks whose values are zeroed before its parts add
into them, and rows in global-memory tables."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import TOL, assert_matches_oracle
from paper_1804_01698_gb300 import inputs
from paper_1804_01698_gb300.inputs import CSR

pytestmark = pytest.mark.gpu

SENT_COL = -7
SENT_VAL = {torch.float64: 1e300, torch.float32: 3e38, torch.int64: -123456789}


def _heavy_rows(nrows_a, entries, ncols_b, b_row_len, seed):
    A = inputs.er_exact(nrows_a, entries, seed=seed, ncols=entries * 4)
    B = inputs.er_exact(entries * 4, b_row_len, seed=seed + 1, ncols=ncols_b)
    return A, B


def _split_row_product():
    """Row 0: 600,000 products onto at most 5,000 columns, split over blocks."""
    rng = np.random.default_rng(31)
    kb, nb = 5000, 20000
    B = inputs.er_exact(nb, 30, seed=32, ncols=kb)
    rows = [np.full(nb, 0)] + [np.full(50 * r, r) for r in range(1, 8)]
    cols = [np.arange(nb)] + [rng.choice(nb, size=50 * r, replace=False) for r in range(1, 8)]
    rp, ci = inputs.from_coo(8, nb, np.concatenate(rows), np.concatenate(cols))
    return CSR(8, nb, rp, ci, rng.uniform(-1, 1, len(ci))), B


def _global_rows():
    """5 rows over 2^20 columns (global tables) and 7 lighter rows."""
    A1, B = _heavy_rows(5, 40, 1 << 20, 1000, seed=71)
    A2 = inputs.er_exact(7, 20, seed=73, ncols=160)
    A = CSR(12, 160, np.concatenate([A1.row_ptr, A2.row_ptr[1:] + A1.nnz]).astype(np.int32),
            np.concatenate([A1.col_idx, A2.col_idx]), np.concatenate([A1.vals, A2.vals]))
    return A, B


CASES = {
    "rmat13": lambda: (inputs.rmat(13, 16, seed=inputs.SEED_BASE + 81),) * 2,
    "split_row": _split_row_product,
    "wide_rows_in_parts": lambda: _heavy_rows(3, 2048, 65536, 1000, seed=72),
    "global_tables": _global_rows,
}


def _middle(m: int) -> tuple[int, int]:
    return (m // 3, max(m // 3 + 1, 2 * m // 3)) if m >= 3 else (0, m)


def _check_rows(C, ref, absb, r0: int, r1: int, dt):
    """Rows [r0, r1) equal the oracle's (sorted output); all other entries
    still hold the sentinels."""
    rp = ref.row_ptr
    e0, e1 = int(rp[r0]), int(rp[r1])
    ci = C.col_idx.cpu().numpy()
    cv = C.vals.cpu().numpy()
    assert np.array_equal(ci[e0:e1], ref.col_idx[e0:e1]), "col_idx of the range differs"
    if dt == torch.int64:
        assert np.array_equal(cv[e0:e1], ref.vals[e0:e1].astype(np.int64))
    else:
        err = np.abs(cv[e0:e1].astype(np.float64) - ref.vals[e0:e1])
        assert not (err > TOL[dt] * absb[e0:e1]).any(), "values of the range outside tolerance"
    outside = np.r_[0:e0, e1:len(ci)]
    assert np.all(ci[outside] == SENT_COL), "a column outside the range was written"
    assert np.all(cv[outside] == SENT_VAL[dt]), "a value outside the range was written"


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("dt", [torch.float64, torch.int64])
def test_row_ranges_write_only_their_rows_and_cover_the_product(case, dt):
    from paper_1804_01698_gb300 import binding as sg
    A, B = CASES[case]()
    if dt == torch.int64:
        rng = np.random.default_rng(A.nnz)
        A = A.with_vals(rng.integers(-3, 4, A.nnz).astype(np.int64))
        B = A if case == "rmat13" else B.with_vals(rng.integers(-3, 4, B.nnz).astype(np.int64))
    ref, absb = oracle.spgemm(A, B, nthreads=8)
    dA = sg.to_device(A, "cuda", dt)
    dB = dA if case == "rmat13" else sg.to_device(B, "cuda", dt)
    with sg.Plan(dA, dB, True) as plan:
        nnz = plan.symbolic()
        C = sg.DeviceCSR(A.nrows, B.ncols, plan.c_row_ptr,
                         torch.full((nnz,), SENT_COL, dtype=torch.int32, device="cuda"),
                         torch.full((nnz,), SENT_VAL[dt], dtype=dt, device="cuda"))
        m = A.nrows
        r0, r1 = _middle(m)
        plan.numeric_rows(r0, r1, C)
        plan.numeric_rows(r1, r1, C)                 # empty range: nothing
        torch.cuda.synchronize()
        assert plan.stats()["status"] == 0
        _check_rows(C, ref, absb, r0, r1, dt)
        plan.numeric_rows(r1, m, C)
        plan.numeric_rows(0, r0, C)
        torch.cuda.synchronize()
        assert plan.stats()["status"] == 0
        assert_matches_oracle(C, A, B, True, expect=(ref, absb))
        # every row again: split rows are zeroed again before their parts add
        plan.numeric_rows(0, m, C)
        torch.cuda.synchronize()
        assert_matches_oracle(C, A, B, True, expect=(ref, absb))


def test_unsorted_ranges_cover_the_product():
    from paper_1804_01698_gb300 import binding as sg
    A = inputs.rmat(13, 16, seed=inputs.SEED_BASE + 82)
    dA = sg.to_device(A, "cuda", torch.float64)
    with sg.Plan(dA, dA, False) as plan:
        nnz = plan.symbolic()
        C = sg.DeviceCSR(A.nrows, A.ncols, plan.c_row_ptr, torch.empty(nnz, dtype=torch.int32, device="cuda"),
                         torch.empty(nnz, dtype=torch.float64, device="cuda"))
        bounds = [0, 17, 1000, 1001, 4096, A.nrows]
        for lo, hi in zip(bounds[1:], bounds[2:]):
            plan.numeric_rows(lo, hi, C)
        plan.numeric_rows(0, 17, C)
        torch.cuda.synchronize()
        assert plan.stats()["status"] == 0
    assert_matches_oracle(C, A, A, False)


def test_range_outside_the_rows_is_refused():
    from paper_1804_01698_gb300 import binding as sg
    A = inputs.er_exact(64, 4, seed=91, ncols=64)
    dA = sg.to_device(A, "cuda", torch.float64)
    with sg.Plan(dA, dA, True) as plan:
        plan.symbolic()
        C = plan.numeric()
        for lo, hi in [(-1, 3), (5, 4), (0, 65)]:
            with pytest.raises(sg.SpgemmError):
                plan.numeric_rows(lo, hi, C)
        torch.cuda.synchronize()
