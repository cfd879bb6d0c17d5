"""spgemm_host: operands and result in host memory, the copy of C to the
host overlapped with the numeric phase block of rows by block of rows.
Checked element by element against the oracle for every blocking (the
result must not depend on it), the value types and orders, empty and
degenerate blockings, the host arena, the error paths, and the full-size
R-MAT scale 16 product in the configuration bench.py times end to end."""
from __future__ import annotations

import os

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import assert_matches_oracle
from paper_1804_01698_gb300 import inputs
from paper_1804_01698_gb300.inputs import CSR

pytestmark = pytest.mark.gpu


def _on_device(C: CSR):
    from paper_1804_01698_gb300 import binding as sg
    return sg.DeviceCSR(C.nrows, C.ncols, torch.from_numpy(np.array(C.row_ptr)).cuda(),
                        torch.from_numpy(np.array(C.col_idx)).cuda(), torch.from_numpy(np.array(C.vals)).cuda())


def _typed(m: CSR, dtype) -> CSR:
    if dtype == np.int64:
        rng = np.random.default_rng(m.nnz + 7)
        return CSR(m.nrows, m.ncols, m.row_ptr, m.col_idx, rng.integers(-3, 4, size=m.nnz).astype(np.int64))
    return CSR(m.nrows, m.ncols, m.row_ptr, m.col_idx, m.vals.astype(dtype))


@pytest.mark.parametrize("row_blocks", [0, 1, 2, 3, 7, 1 << 20])
def test_every_blocking_gives_the_oracle_product(row_blocks):
    from paper_1804_01698_gb300 import binding as sg
    A = inputs.rmat(12, 16, seed=inputs.SEED_BASE + 31)
    C = sg.spgemm_host(A, A, True, row_blocks=row_blocks)
    assert_matches_oracle(_on_device(C), A, A, True)


@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.int64])
@pytest.mark.parametrize("sorted_output", [True, False])
def test_rectangular_product_types_and_orders(dtype, sorted_output):
    from paper_1804_01698_gb300 import binding as sg
    A = _typed(inputs.rmat(11, 12, seed=inputs.SEED_BASE + 32), dtype)
    B = _typed(inputs.er_exact(A.ncols, 9, seed=inputs.SEED_BASE + 33, ncols=3000), dtype)
    C = sg.spgemm_host(A, B, sorted_output, row_blocks=3)
    assert C.vals.dtype == np.dtype(dtype)
    assert_matches_oracle(_on_device(C), A, B, sorted_output)


def test_all_flop_in_one_row_leaves_empty_blocks():
    """One hub row holds nearly all the flop: the equal-flop blocks around it
    are empty and skipped."""
    from paper_1804_01698_gb300 import binding as sg
    rng = np.random.default_rng(5)
    m, n, k = 50, 400, 2000
    rows = [np.arange(n)] + [rng.choice(n, 1, replace=False) for _ in range(m - 1)]
    rp = np.zeros(m + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    A = CSR(m, n, rp, np.concatenate(rows).astype(np.int32), rng.uniform(-1, 1, int(rp[-1])))
    B = inputs.er_exact(n, 20, seed=6, ncols=k)
    C = sg.spgemm_host(A, B, True, row_blocks=8)
    assert_matches_oracle(_on_device(C), A, B, True)


@pytest.mark.parametrize("shape", [(0, 5, 3), (4, 0, 3), (4, 5, 0), (3, 3, 3)])
@pytest.mark.parametrize("row_blocks", [0, 3])
def test_empty_shapes(shape, row_blocks):
    from paper_1804_01698_gb300 import binding as sg
    m, n, k = shape
    A = CSR(m, n, np.zeros(m + 1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = CSR(n, k, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    C = sg.spgemm_host(A, B, True, row_blocks=row_blocks)
    assert C.nrows == m and C.ncols == k and C.nnz == 0
    assert np.array_equal(C.row_ptr, np.zeros(m + 1, np.int32))


def test_arena_holds_the_result_and_is_reused():
    from paper_1804_01698_gb300 import binding as sg
    A = inputs.rmat(11, 16, seed=inputs.SEED_BASE + 34)
    ref = oracle.spgemm(A, A)
    nnz = ref[0].nnz
    arena = sg.HostArena(sg.HostArena.bytes_for(A.nrows, nnz, 8))
    for _ in range(2):
        arena.reset()
        C = sg.spgemm_host(A, A, True, row_blocks=2, arena=arena)
        base = arena.buf.data_ptr()
        assert base <= C.col_idx.ctypes.data < base + arena.buf.numel()
        assert_matches_oracle(_on_device(C), A, A, True, expect=ref)
    small = sg.HostArena(sg.HostArena.bytes_for(A.nrows, nnz, 8) // 2)
    with pytest.raises(sg.SpgemmError) as ei:
        sg.spgemm_host(A, A, True, arena=small)
    assert ei.value.status == -3


def test_pinned_tensor_operands():
    from paper_1804_01698_gb300 import binding as sg
    A = inputs.rmat(11, 16, seed=inputs.SEED_BASE + 35)
    P = CSR(A.nrows, A.ncols, torch.from_numpy(A.row_ptr).pin_memory(), torch.from_numpy(A.col_idx).pin_memory(),
            torch.from_numpy(A.vals).pin_memory())
    C = sg.spgemm_host(P, P, False, row_blocks=4)
    assert_matches_oracle(_on_device(C), A, A, False)


def test_malformed_operands_are_errors():
    from paper_1804_01698_gb300 import binding as sg
    A = inputs.rmat(9, 8, seed=3)
    short = CSR(A.nrows, A.ncols, A.row_ptr.copy(), A.col_idx, A.vals)
    short.row_ptr[-1] -= 1                        # row_ptr[m] != nnz: refused on the host
    with pytest.raises(sg.SpgemmError) as ei:
        sg.spgemm_host(short, A, True, row_blocks=2)
    assert ei.value.status == -2
    bad = CSR(A.nrows, A.ncols, A.row_ptr, A.col_idx.copy(), A.vals)
    bad.col_idx[len(bad.col_idx) // 2] = A.ncols + 5   # out of range: the device check reports it
    with pytest.raises(sg.SpgemmError) as ei:
        sg.spgemm_host(bad, A, True, row_blocks=2)
    assert ei.value.status == -2
    C = sg.spgemm_host(A, A, True, row_blocks=2)  # the context is still usable
    assert_matches_oracle(_on_device(C), A, A, True)


def test_rmat16_full_size_end_to_end():
    """The workload bench.py times end to end: R-MAT scale 16, EF 16, A*A,
    FP64, sorted, pinned operands, the default blocking, a pinned arena."""
    from paper_1804_01698_gb300 import binding as sg
    A, B, _ = inputs.workload("rmat16_ef16_f64")
    expect = oracle.spgemm(A, B, nthreads=os.cpu_count() or 8)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()  # noqa: E731
    P = CSR(A.nrows, A.ncols, pin(A.row_ptr), pin(A.col_idx), pin(A.vals))
    arena = sg.HostArena(sg.HostArena.bytes_for(A.nrows, expect[0].nnz, 8))
    C = sg.spgemm_host(P, P, True, arena=arena)
    assert_matches_oracle(_on_device(C), A, B, True, expect=expect)


def test_device_pointers_are_refused():
    """A's row pointers are read on the host, so device arrays are refused
    with an argument error instead of a host fault."""
    import ctypes
    from paper_1804_01698_gb300 import binding as sg
    A = inputs.rmat(8, 8, seed=4)
    dA = sg.to_device(A)
    lib = sg.library()
    d = dA.desc()
    out = [ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()]
    nnz = ctypes.c_int64()
    cb = sg.ALLOC_FN(lambda n, c: None)
    status = lib.spgemm_host(ctypes.byref(d), ctypes.byref(d), sg.SPGEMM_F64, sg.SPGEMM_SORTED, None, 0, cb, None,
                             ctypes.byref(out[0]), ctypes.byref(out[1]), ctypes.byref(out[2]), ctypes.byref(nnz))
    assert status == -1
    assert b"device memory" in lib.spgemm_last_error()
    torch.cuda.synchronize()
