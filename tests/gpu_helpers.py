"""Shared helpers of the GPU parity tests: run the CUDA path through the
binding and compare its output with the CPU oracle, element by element.

Comparison rule: row_ptr and col_idx bit-exact (rows of an unsorted result
are sorted first, on the device, by torch as test-side post-processing);
int64 values bit-exact; float64 within 1e-12 * (|A|*|B|)_ij and float32
within 1e-5 * (|A|*|B|)_ij, the scale (|A|*|B|)_ij being computed by the
oracle beside C.  Sorted results must have strictly increasing columns.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_1804_01698_gb300.inputs import CSR

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def gpu_product(A: CSR, B: CSR, dtype, sorted_output: bool, one_shot: bool = False, probe: str = "linear",
                hash: str = "high"):
    from paper_1804_01698_gb300 import binding as sg
    dA = sg.to_device(A, "cuda", dtype)
    dB = sg.to_device(B, "cuda", dtype)
    if one_shot:
        C = sg.spgemm(dA, dB, sorted_output)
        torch.cuda.synchronize()
        return C, None
    with sg.Plan(dA, dB, sorted_output, probe=probe, hash=hash) as plan:
        plan.symbolic()
        C = plan.numeric()
        stats = plan.stats()
        torch.cuda.synchronize()
    assert stats["status"] == 0, stats
    return C, stats


def sort_rows_on_device(C) -> tuple[torch.Tensor, torch.Tensor]:
    """Column-sort every row of a device CSR (key = row * ncols + col)."""
    n = C.nnz
    if n == 0:
        return C.col_idx, C.vals
    rows = torch.repeat_interleave(torch.arange(C.nrows, device=C.row_ptr.device, dtype=torch.int64),
                                   (C.row_ptr[1:] - C.row_ptr[:-1]).to(torch.int64), output_size=n)
    key = rows * max(C.ncols, 1) + C.col_idx.to(torch.int64)
    order = torch.sort(key).indices
    return C.col_idx[order], C.vals[order]


def assert_matches_oracle(C, A: CSR, B: CSR, sorted_output: bool, expect=None, nthreads: int = 8):
    """Compare device CSR C with the oracle's A*B (or a precomputed (C, absbound))."""
    if expect is None:
        expect = oracle.spgemm(A, B, nthreads=nthreads)
    ref, absb = expect
    rp = C.row_ptr.cpu().numpy()
    assert rp.shape == ref.row_ptr.shape
    assert np.array_equal(rp, ref.row_ptr), "row_ptr differs"
    if sorted_output:
        ci, cv = C.col_idx, C.vals
        if C.nnz > 1:
            d = (ci[1:] - ci[:-1]).cpu().numpy()
            rows = np.repeat(np.arange(C.nrows), np.diff(rp))
            same_row = rows[1:] == rows[:-1]
            assert np.all(d[same_row] > 0), "sorted output has a non-increasing column"
    else:
        ci, cv = sort_rows_on_device(C)
    ci = ci.cpu().numpy()
    cv = cv.cpu().numpy()
    assert np.array_equal(ci, ref.col_idx), "col_idx differs"
    dt = C.vals.dtype
    if dt == torch.int64:
        assert np.array_equal(cv, ref.vals.astype(np.int64)), "int64 values differ"
    else:
        err = np.abs(cv.astype(np.float64) - ref.vals)
        bound = TOL[dt] * absb
        bad = err > bound
        assert not bad.any(), f"{int(bad.sum())} values outside tolerance; worst {float((err - bound).max())}"
