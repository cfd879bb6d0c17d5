"""The seeded workload generators still produce the inputs the golden file
was written from: shapes, nnz and the per-row flop statistics (paper
Sec. 4.1, Fig. "RowsToThreads" step 1) recomputed here on the CPU from the
generated operands alone.  A drift in a generator fails here, before the GPU
tests compare digests of C."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

from paper_1804_01698_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "workloads.json")))


@pytest.mark.parametrize("name", sorted(GOLDEN))
def test_generated_inputs_match_the_golden_record(name):
    g = GOLDEN[name]
    A, B, _ = inputs.workload(name)
    assert (A.nrows, A.ncols, B.ncols) == (g["m"], g["n"], g["k"])
    assert (A.nnz, B.nnz) == (g["nnz_a"], g["nnz_b"])
    blen = np.diff(B.row_ptr.astype(np.int64))
    per_entry = blen[A.col_idx]
    rows = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr.astype(np.int64)))
    flop = np.bincount(rows, weights=per_entry, minlength=A.nrows).astype(np.int64)
    assert int(flop.sum()) == g["total_flop"]
    assert int(flop.max()) == g["max_row_flop"]
    assert int((flop == 0).sum()) == g["zero_flop_rows"]
    assert g["nnz_c"] <= g["total_flop"]
