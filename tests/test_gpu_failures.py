"""Failures injected on the host, checked on the GPU without faulting it:
an allocator that returns NULL, an nnz(C) limit below the product's size
(the int32-overflow path reached on a small input), and the probe counters
of SPGEMM_COUNT_PROBES, whose totals are fixed by the inputs."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

from paper_1804_01698_gb300 import inputs
from gpu_helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fail_at", [0, 1, 2])
def test_allocator_failure_is_reported(fail_at):
    """The one-shot entry point asks its allocator for row_ptr, then col_idx
    and vals; a NULL at any of them gives SPGEMM_ERR_OUT_OF_MEMORY."""
    from paper_1804_01698_gb300 import binding as sg
    lib = sg.library()
    A = sg.to_device(inputs.er_exact(500, 6, seed=121))
    keep, calls = [], [0]

    def alloc(nbytes, _ctx):
        calls[0] += 1
        if calls[0] - 1 == fail_at:
            return None
        t = torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device="cuda")
        keep.append(t)
        return t.data_ptr()

    cb = sg.ALLOC_FN(alloc)
    a = A.desc()
    rp, ci, cv, nnz = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
    rc = lib.spgemm(ctypes.byref(a), ctypes.byref(a), sg._DTYPES[torch.float64], sg.SPGEMM_SORTED, None, cb, None,
                    ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(cv), ctypes.byref(nnz))
    torch.cuda.synchronize()
    assert rc == -3
    C = sg.spgemm(A, A, True)        # the context stays usable
    torch.cuda.synchronize()
    assert C.nnz > 0


def test_nnz_limit_reaches_the_overflow_path():
    from paper_1804_01698_gb300 import binding as sg
    M = inputs.er_exact(2000, 8, seed=122)
    A = sg.to_device(M)
    with sg.Plan(A, A, True) as p:
        nnz = p.symbolic()
    with sg.Plan(A, A, True, tuning={"max_nnz_c": nnz - 1}) as p:
        with pytest.raises(sg.SpgemmError) as ei:
            p.symbolic()
        assert ei.value.status == -4
    with sg.Plan(A, A, True, tuning={"max_nnz_c": nnz}) as p:
        assert p.symbolic() == nnz
        C = p.numeric()
    torch.cuda.synchronize()
    assert_matches_oracle(C, M, M, True)


@pytest.mark.parametrize("probe", ["linear", "chunk4"])
def test_probe_counters(probe):
    """Every product of a hash-table row is one insertion in each phase, so
    inserts = flop when no row takes a bitmap; an insertion reads at least
    one slot (chunk).  With one key per row, every insertion finds its slot
    at the first probe."""
    from paper_1804_01698_gb300 import binding as sg
    M = inputs.er_exact(3000, 12, seed=123)
    A = sg.to_device(M)
    with sg.Plan(A, A, True, probe=probe, count_probes=True, tuning={"bitmap_min_bound": -1}) as p:
        p.symbolic()
        C = p.numeric()
        st = p.stats()
    torch.cuda.synchronize()
    assert st["status"] == 0
    assert st["sym_inserts"] == st["total_flop"] == st["num_inserts"]
    assert st["sym_inserts"] <= st["sym_probes"] <= 4 * st["sym_inserts"]
    assert st["num_inserts"] <= st["num_probes"] <= 4 * st["num_inserts"]
    assert_matches_oracle(C, M, M, True)
    I = inputs.CSR(1000, 1000, np.arange(1001, dtype=np.int32), np.arange(1000, dtype=np.int32), np.ones(1000))
    dI = sg.to_device(I)
    with sg.Plan(dI, dI, True, probe=probe, count_probes=True) as p:
        p.symbolic()
        p.numeric()
        st = p.stats()
    torch.cuda.synchronize()
    assert st["sym_probes"] == st["sym_inserts"] == 1000
    assert st["num_probes"] == st["num_inserts"] == 1000
    with sg.Plan(dI, dI, True, probe=probe) as p:   # counting off: the counters stay at zero
        p.symbolic()
        p.numeric()
        st = p.stats()
    assert st["sym_probes"] == st["num_inserts"] == 0
