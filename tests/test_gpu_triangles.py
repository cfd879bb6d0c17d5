"""Triangle counting's product L*U (Sec. 5.6) on the GPU: the undirected
graph of an R-MAT matrix, relabelled by increasing degree and split into
strictly lower L and strictly upper U.  C = L*U matches the oracle (sorted
and unsorted; int64 bit-exact), and the triangle count read from the GPU's
C, sum over stored g_ij of c_ij / 2, equals trace(G^3)/6 on a graph small
enough for dense matrices."""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1804_01698_gb300 import inputs
from gpu_helpers import assert_matches_oracle, gpu_product, sort_rows_on_device

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def masked_sum_halved(C, G) -> float:
    """sum over stored g_ij of c_ij, halved (test-side post-processing)."""
    n = G.nrows
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(C.row_ptr.cpu().numpy()))
    keys_c = rows * n + C.col_idx.cpu().numpy().astype(np.int64)
    grows = np.repeat(np.arange(n, dtype=np.int64), np.diff(G.row_ptr))
    keys_g = grows * n + G.col_idx.astype(np.int64)
    order = np.argsort(keys_c)
    pos = np.searchsorted(keys_c[order], keys_g)
    pos = np.minimum(pos, len(order) - 1)
    hit = keys_c[order][pos] == keys_g
    vals = C.vals.cpu().numpy()[order][pos]
    return float(vals[hit].sum()) / 2


@pytest.mark.parametrize("sorted_output", [True, False])
@pytest.mark.parametrize("dt", [torch.float64, torch.int64])
def test_lu_matches_oracle(dt, sorted_output):
    L, U, _ = inputs.triangle_lu(12, 16, seed=611)
    if dt == torch.int64:
        L, U = L.astype(np.int64), U.astype(np.int64)
    C, stats = gpu_product(L, U, dt, sorted_output)
    assert stats["status"] == 0
    assert_matches_oracle(C, L, U, sorted_output)


def test_triangle_count_from_the_gpu_product():
    L, U, G = inputs.triangle_lu(10, 8, seed=612)
    C, _ = gpu_product(L, U, torch.int64, True)
    d = np.zeros((G.nrows, G.nrows))
    d[np.repeat(np.arange(G.nrows), np.diff(G.row_ptr)), G.col_idx] = 1.0
    expect = np.trace(d @ d @ d) / 6
    assert expect > 1000
    assert masked_sum_halved(C, G) == expect


def test_full_size_tc_rmat16():
    L, U, _ = inputs.workload("tc_rmat16_lu_f64")
    g = json.load(open(os.path.join(HERE, "golden", "workloads.json")))["tc_rmat16_lu_f64"]
    C, stats = gpu_product(L, U, torch.float64, True)
    assert stats["total_flop"] == g["total_flop"]
    assert stats["max_row_flop"] == g["max_row_flop"]
    assert_matches_oracle(C, L, U, True)
    rp = C.row_ptr.cpu().numpy()
    ci, _ = sort_rows_on_device(C)
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(rp, dtype=np.int32).tobytes())
    h.update(np.ascontiguousarray(ci.cpu().numpy(), dtype=np.int32).tobytes())
    assert int(rp[-1]) == g["nnz_c"]
    assert h.hexdigest() == g["c_structure_sha256"]
