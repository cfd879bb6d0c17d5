"""Repeated numeric phases on one plan (same structure, new values), plain
and replayed through a CUDA graph: every run must give the oracle's product
for the values of that run."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_1804_01698_gb300 import inputs
from paper_1804_01698_gb300.inputs import CSR
from gpu_helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu


def _new_values(M: CSR, seed: int, integer: bool) -> CSR:
    rng = np.random.default_rng(seed)
    v = rng.integers(-3, 4, M.nnz).astype(np.int64) if integer else rng.uniform(-1, 1, M.nnz)
    return M.with_vals(v)


@pytest.mark.parametrize("sorted_output", [True, False])
@pytest.mark.parametrize("dt", [torch.float64, torch.int64])
@pytest.mark.parametrize("shape", ["rmat13", "heavy_split"])
def test_repeated_numeric_plain_and_graph(shape, dt, sorted_output):
    from paper_1804_01698_gb300 import binding as sg
    integer = dt == torch.int64
    if shape == "rmat13":                      # hash bins and bitmap rows
        A = B = inputs.rmat(13, 16, seed=161)
    else:                                      # a bitmap row split over blocks
        B = inputs.er_exact(20000, 30, seed=162, ncols=5000)
        rp, ci = inputs.from_coo(3, 20000, np.concatenate([np.zeros(20000, np.int64), [1, 1, 2]]),
                                 np.concatenate([np.arange(20000), [5, 9, 7]]))
        A = CSR(3, 20000, rp, ci, np.ones(len(ci)))
    A, B = _new_values(A, 1, integer), _new_values(B, 2, integer)
    dA, dB = sg.to_device(A, "cuda", dt), sg.to_device(B, "cuda", dt)
    same = shape == "rmat13"
    if same:
        dB = dA
    with sg.Plan(dA, dB, sorted_output) as plan:
        plan.symbolic()
        C = plan.numeric()
        torch.cuda.synchronize()
        assert_matches_oracle(C, A, A if same else B, sorted_output)
        for run in range(4):
            A2 = _new_values(A, 10 + run, integer)
            B2 = A2 if same else _new_values(B, 20 + run, integer)
            dA.vals.copy_(torch.from_numpy(A2.vals).to(dt))
            if not same:
                dB.vals.copy_(torch.from_numpy(B2.vals).to(dt))
            if run % 2 == 0:
                C = plan.numeric(C.col_idx, C.vals)     # plain re-run into the same buffers
            else:
                C = plan.numeric_graph(C)               # captured once, then replayed
            torch.cuda.synchronize()
            assert plan.stats()["status"] == 0
            assert_matches_oracle(C, A2, B2, sorted_output)
        for run in range(2):                           # replay again with new values
            A3 = _new_values(A, 30 + run, integer)
            B3 = A3 if same else _new_values(B, 40 + run, integer)
            dA.vals.copy_(torch.from_numpy(A3.vals).to(dt))
            if not same:
                dB.vals.copy_(torch.from_numpy(B3.vals).to(dt))
            C = plan.numeric_graph(C)
            torch.cuda.synchronize()
            assert_matches_oracle(C, A3, B3, sorted_output)


def test_numeric_graph_needs_a_numeric_first_and_no_timing():
    from paper_1804_01698_gb300 import binding as sg
    dA = sg.to_device(inputs.er_exact(500, 5, seed=163))
    with sg.Plan(dA, dA, True) as plan:
        plan.symbolic()
        C = sg.DeviceCSR(dA.nrows, dA.ncols, plan.c_row_ptr,
                         torch.empty(plan.nnz_c, dtype=torch.int32, device="cuda"),
                         torch.empty(plan.nnz_c, dtype=torch.float64, device="cuda"))
        with pytest.raises(sg.SpgemmError) as ei:
            plan.numeric_graph(C)
        assert ei.value.status == -5
    with sg.Plan(dA, dA, True, timing=True) as plan:
        plan.symbolic()
        C = plan.numeric()
        with pytest.raises(sg.SpgemmError) as ei:
            plan.numeric_graph(C)
        assert ei.value.status == -1
