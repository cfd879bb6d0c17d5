"""GPU test of spgemm_symbolic_noalloc, the entry point for callers that
cannot allocate device memory while they run (for example code inside an
allocator callback, or a loop that must never reach the CUDA allocator).

It is called through the C ABI and its row pointers and nnz(C) are compared
with those of the regular entry point (spgemm_plan_create + spgemm_symbolic),
bit for bit, on two calls in a row: the second call reuses the static
scratch array the first one left behind.  The file sorts last so that a
failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1804_01698_gb300 import inputs

pytestmark = pytest.mark.gpu


def regular_row_ptr(sg, dA, dB):
    with sg.Plan(dA, dB, True) as plan:
        nnz = plan.symbolic()
        rp = plan.c_row_ptr.clone()
    torch.cuda.synchronize()
    return rp, nnz


def noalloc_row_ptr(sg, dA, dB):
    lib = sg.library()
    rp = torch.full((dA.nrows + 1,), -7, dtype=torch.int32, device=dA.row_ptr.device)
    a, b = dA.desc(), dB.desc()
    nnz = ctypes.c_int64(-1)
    status = lib.spgemm_symbolic_noalloc(ctypes.byref(a), ctypes.byref(b), rp.data_ptr(), ctypes.byref(nnz),
                                         torch.cuda.current_stream().cuda_stream or None)
    torch.cuda.synchronize()
    return status, rp, int(nnz.value)


def test_noalloc_matches_regular_symbolic_twice():
    from paper_1804_01698_gb300 import binding as sg
    cases = [inputs.rmat(12, 16, seed=301), inputs.er_exact(3000, 9, seed=302)]
    for call, A in enumerate(cases):          # two calls in a row, different products
        dA = sg.to_device(A)
        ref_rp, ref_nnz = regular_row_ptr(sg, dA, dA)
        status, rp, nnz = noalloc_row_ptr(sg, dA, dA)
        assert status == 0, (call, sg.spgemm_status_string(status), sg.library().spgemm_last_error())
        assert nnz == ref_nnz
        assert torch.equal(rp, ref_rp), f"row_ptr differs on call {call}"
    # the binding wrapper gives the same answer once more
    dA = sg.to_device(cases[0])
    rp = torch.empty(dA.nrows + 1, dtype=torch.int32, device=dA.row_ptr.device)
    assert sg.spgemm_symbolic_noalloc(dA, dA, rp) == regular_row_ptr(sg, dA, dA)[1]


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
    C = inputs.er_exact(500, 6, seed=313)
    dC = sg.to_device(C)
    ref_rp, ref_nnz = regular_row_ptr(sg, dC, dC)
    status, rp, nnz = noalloc_row_ptr(sg, dC, dC)
    assert status == 0 and nnz == ref_nnz and torch.equal(rp, ref_rp)
