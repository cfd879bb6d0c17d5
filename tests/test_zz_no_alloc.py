"""GPU test of spgemm_symbolic_noalloc, the entry point for callers that
cannot allocate device memory while they run (for example code inside an
allocator callback, or a loop that must never reach the CUDA allocator).

It is called through the C ABI.  Its row pointers and nnz(C) are compared,
bit for bit, with the CPU oracle's row counts and with those of the regular
entry point (spgemm_plan_create + spgemm_symbolic), on several calls in a
row: each call reuses the static scratch array the previous one left
behind.  The file sorts last so that a failure here comes after every other
test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1804_01698_gb300 import inputs
from paper_1804_01698_gb300.inputs import CSR

pytestmark = pytest.mark.gpu

NOALLOC_MAX_KEYS = (1 << 17) - 1   # largest row key bound min(flop_i, ncols(B)) the call accepts


def regular_row_ptr(sg, dA, dB):
    with sg.Plan(dA, dB, True) as plan:
        nnz = plan.symbolic()
        rp = plan.c_row_ptr.clone()
    torch.cuda.synchronize()
    return rp, nnz


def oracle_row_ptr(A, B):
    counts = oracle.symbolic(A, B, nthreads=8)
    rp = np.zeros(A.nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return rp


def noalloc_row_ptr(sg, dA, dB):
    lib = sg.library()
    rp = torch.full((dA.nrows + 1,), -7, dtype=torch.int32, device=dA.row_ptr.device)
    a, b = dA.desc(), dB.desc()
    nnz = ctypes.c_int64(-1)
    status = lib.spgemm_symbolic_noalloc(ctypes.byref(a), ctypes.byref(b), rp.data_ptr(), ctypes.byref(nnz),
                                         torch.cuda.current_stream().cuda_stream or None)
    torch.cuda.synchronize()
    return status, rp, int(nnz.value)


def check_against_both(sg, A, B, call):
    dA = sg.to_device(A)
    dB = dA if B is A else sg.to_device(B)
    want = oracle_row_ptr(A, B)
    ref_rp, ref_nnz = regular_row_ptr(sg, dA, dB)
    status, rp, nnz = noalloc_row_ptr(sg, dA, dB)
    assert status == 0, (call, sg.spgemm_status_string(status), sg.library().spgemm_last_error())
    assert nnz == int(want[-1]) == ref_nnz, call
    assert np.array_equal(rp.cpu().numpy().astype(np.int64), want), f"row_ptr differs from the oracle on call {call}"
    assert torch.equal(rp, ref_rp), f"row_ptr differs from spgemm_symbolic on call {call}"


def wide_row_operands(seed: int):
    """A few rows of A whose key bound is exactly the largest the call accepts
    (min(flop_i, ncols(B)) = 131071: the whole 2^17-slot table), holding a few
    tens of thousands of distinct keys, beside short rows."""
    rng = np.random.default_rng(seed)
    ncols_b, nb, per, span = NOALLOC_MAX_KEYS, 96, 4096, 40000
    b_cols = [np.sort(rng.choice(span, per, replace=False)) for _ in range(nb)]
    b_cols[0] = np.sort(rng.choice(ncols_b, per, replace=False))   # one B row spread over all columns
    brp = np.arange(nb + 1, dtype=np.int32) * per
    B = CSR(nb, ncols_b, brp, np.concatenate(b_cols).astype(np.int32), rng.uniform(-1, 1, nb * per))
    rows = [np.arange(64), np.arange(32, 96), np.array([3]), np.array([5, 7]), np.arange(0, 96, 2)]
    arp = np.zeros(len(rows) + 1, dtype=np.int32)
    arp[1:] = np.cumsum([len(r) for r in rows])
    A = CSR(len(rows), nb, arp, np.concatenate(rows).astype(np.int32), rng.uniform(-1, 1, int(arp[-1])))
    return A, B


def test_noalloc_matches_oracle_and_regular_symbolic():
    from paper_1804_01698_gb300 import binding as sg
    A, B = wide_row_operands(seed=303)
    bounds = np.minimum(oracle.row_flop(A, B), B.ncols)
    assert bounds.max() == NOALLOC_MAX_KEYS                # the table-size edge is reached
    assert oracle.symbolic(A, B).max() > 20000             # rows of tens of thousands of keys
    rm = inputs.rmat(12, 16, seed=301)
    er = inputs.er_exact(3000, 9, seed=302)
    for call, (X, Y) in enumerate([(rm, rm), (er, er), (A, B), (rm, rm)]):   # consecutive calls
        check_against_both(sg, X, Y, call)
    # the binding wrapper gives the same answer once more
    dA = sg.to_device(rm)
    rp = torch.empty(dA.nrows + 1, dtype=torch.int32, device=dA.row_ptr.device)
    assert sg.spgemm_symbolic_noalloc(dA, dA, rp) == int(oracle_row_ptr(rm, rm)[-1])
    with pytest.raises(ValueError):
        sg.spgemm_symbolic_noalloc(dA, dA, rp[:-1])         # one element short


def test_noalloc_refuses_rows_beyond_its_table():
    from paper_1804_01698_gb300 import binding as sg
    # one row touching 200 B rows of 1000 distinct columns among 2^20: bound 200000 > 131071
    A = inputs.er_exact(1, 200, seed=311, ncols=400)
    B = inputs.er_exact(400, 1000, seed=312, ncols=1 << 20)
    dA, dB = sg.to_device(A), sg.to_device(B)
    status, _, _ = noalloc_row_ptr(sg, dA, dB)
    assert status == -1                                   # SPGEMM_ERR_INVALID_ARGUMENT
    assert b"131071" in sg.library().spgemm_last_error()
    # the device is still usable and the next call is right
    check_against_both(sg, inputs.er_exact(500, 6, seed=313), inputs.er_exact(500, 6, seed=313), "after refusal")


def test_noalloc_rejects_malformed_csr():
    from paper_1804_01698_gb300 import binding as sg
    good = inputs.er_exact(600, 8, seed=321)
    # a column index outside A (= ncols) in one row, and a last row pointer past nnz
    bad_col = CSR(good.nrows, good.ncols, good.row_ptr.copy(), good.col_idx.copy(), good.vals)
    bad_col.col_idx[17] = good.ncols
    bad_rp = CSR(good.nrows, good.ncols, good.row_ptr.copy(), good.col_idx, good.vals)
    bad_rp.row_ptr[-1] = good.nnz + 5
    dG = sg.to_device(good)
    for X in (bad_col, bad_rp):
        dX = sg.to_device(X)
        status, _, _ = noalloc_row_ptr(sg, dX, dG)
        assert status == -2                               # SPGEMM_ERR_INVALID_CSR
    check_against_both(sg, good, good, "after malformed input")
