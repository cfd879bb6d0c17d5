"""Batch graphs: every product of a batch in one CUDA graph launch.

Each product is compared with the CPU oracle element by element, on several
waves, after replays with new values, with heavy rows that need the global
tables, and after a replay whose product outgrew the planned pool (reported
as an error, and the next replay right again)."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

from paper_1804_01698_gb300 import inputs
from paper_1804_01698_gb300.inputs import CSR
from gpu_helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu


def _check_all(g, As, Bs, sorted_output):
    for p in range(len(As)):
        assert_matches_oracle(g.product(p), As[p], Bs[p], sorted_output)


@pytest.mark.parametrize("sorted_output", [True, False])
def test_batch_graph_matches_the_oracle_over_several_waves_and_replays(sorted_output):
    from paper_1804_01698_gb300 import binding as sg
    import oracle
    mats = inputs.er_batch(24, seed=501, n_hi=3000)
    nnzs = [int(oracle.symbolic(m, m).sum()) for m in mats]
    wave = max(max(nnzs), sum(nnzs) // 3)             # at least two waves, every product fits one
    dev = [sg.to_device(m) for m in mats]
    with sg.BatchGraph(dev, dev, sorted_output, wave_nnz=wave) as g:
        info = g.info()
        assert info["waves"] >= 2 and info["kernel_nodes"] > 0
        g.launch()
        g.wait()
        _check_all(g, mats, mats, sorted_output)
        for run in range(2):                       # new values, same structure: one launch each
            new = [m.with_vals(np.random.default_rng(502 + run * 50 + i).uniform(-1, 1, m.nnz))
                   for i, m in enumerate(mats)]
            for d, m in zip(dev, new):
                d.vals.copy_(torch.from_numpy(m.vals))
            g.launch()
            g.wait()
            _check_all(g, new, new, sorted_output)
        assert g.info()["kernel_nodes"] == info["kernel_nodes"]


@pytest.mark.parametrize("dt", [torch.float64, torch.int64])
def test_batch_graph_heavy_rows_take_global_tables(dt):
    from paper_1804_01698_gb300 import binding as sg
    # product 0: row 0 of A reaches 2000 rows of B spread over 60000 columns
    # (about 44K distinct keys: above the shared-memory tables)
    B0 = inputs.er_exact(2000, 40, seed=511, ncols=60000)
    rp, ci = inputs.from_coo(3, 2000, np.concatenate([np.zeros(2000, np.int64), [1, 2]]),
                             np.concatenate([np.arange(2000), [5, 7]]))
    A0 = CSR(3, 2000, rp, ci, np.ones(len(ci)))
    A1 = inputs.er_exact(700, 6, seed=512)
    As, Bs = [A0, A1], [B0, A1]
    if dt == torch.int64:
        As = [m.with_vals(np.random.default_rng(513 + i).integers(-3, 4, m.nnz)) for i, m in enumerate(As)]
        Bs = [Bs[0].with_vals(np.random.default_rng(515).integers(-3, 4, Bs[0].nnz)), As[1]]
    dA = [sg.to_device(m, "cuda", dt) for m in As]
    dB = [sg.to_device(Bs[0], "cuda", dt), dA[1]]
    with sg.BatchGraph(dA, dB, True) as g:
        g.launch()
        g.wait()
        _check_all(g, As, Bs, True)


def test_batch_graph_reports_a_product_that_outgrew_its_pool():
    from paper_1804_01698_gb300 import binding as sg
    n = 512
    A = inputs.er_exact(n, 4, seed=521)
    B = inputs.er_exact(n, 4, seed=522, ncols=4 * n)
    # B with disjoint rows: every row of A*B then has the largest count, 16
    wide = CSR(n, 4 * n, B.row_ptr.copy(), np.arange(4 * n, dtype=np.int32), B.vals)
    import oracle
    base = int(oracle.symbolic(A, B).sum())
    assert base + 1 < int(oracle.symbolic(A, wide).sum()) == 16 * n  # the wide product outgrows the pool
    dA, dB = sg.to_device(A), sg.to_device(B)
    with sg.BatchGraph([dA], [dB], True, pool_slack=0.0) as g:
        g.launch()
        g.wait()
        assert_matches_oracle(g.product(0), A, B, True)
        dB.col_idx.copy_(torch.from_numpy(wide.col_idx))             # same shape, more entries in C
        g.launch()
        with pytest.raises(sg.SpgemmError) as ei:
            g.wait()
        assert ei.value.status == -3                                  # SPGEMM_ERR_OUT_OF_MEMORY
        dB.col_idx.copy_(torch.from_numpy(B.col_idx))                # back to the planned structure
        g.launch()
        g.wait()
        assert_matches_oracle(g.product(0), A, B, True)


def test_batch_graph_rejects_timing_and_bad_arguments():
    from paper_1804_01698_gb300 import binding as sg
    lib = sg.library()
    A = sg.to_device(inputs.er_exact(100, 4, seed=531))
    a = (sg.CsrDesc * 1)(A.desc())
    h = ctypes.c_void_p()
    assert lib.spgemm_bgraph_create(ctypes.byref(h), 1, a, a, 2, sg.SPGEMM_TIMING, None, None, 0, 0.0) == -1
    assert lib.spgemm_bgraph_create(ctypes.byref(h), 1, a, a, 2, 0, None, None, -1, 0.0) == -1
    assert lib.spgemm_bgraph_create(ctypes.byref(h), 1, a, a, 2, 0, None, None, 0, -0.5) == -1
    assert lib.spgemm_bgraph_create(ctypes.byref(h), 0, a, a, 2, 0, None, None, 0, 0.0) == -1
    assert h.value is None
