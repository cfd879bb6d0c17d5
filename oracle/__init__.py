"""CPU oracle for Gustavson row-wise SpGEMM (paper Sec. 2 and Sec. 4.1).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
CPU-baseline leg of the benchmark are the only callers.  The GPU library
never imports this package, and this package never imports the GPU library.

The arithmetic lives in ``spgemm_oracle.c`` (plain C, dense sparse
accumulator, built with gcc without FMA contraction).  This module builds it
on first use and marshals numpy arrays to it.

Functions:
  * ``row_flop(A, B)``: flop[i] = sum over stored a_ik of nnz(b_k*)
    (Sec. 4.1, Fig. "RowsToThreads", step 1).
  * ``rows_to_threads(flop, t)``: the paper's flop-balanced row partition
    (Sec. 4.1, Fig. "RowsToThreads", step 2).
  * ``symbolic(A, B)``: nnz of each output row (two-phase method, Sec. 2).
  * ``spgemm(A, B)``: C = A*B with column-sorted rows; for floating-point
    inputs also returns (|A|*|B|) at every stored entry of C, the scale of
    the tolerance used when comparing against a GPU result.
  * ``spgemm_rows(A, B, rows)``: the same restricted to selected rows.

Floating-point inputs are widened to float64 and summed in float64;
integer inputs are summed as int64 with wrap-around.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spgemm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/liboracle.so and return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            I64, P = ctypes.c_int64, ctypes.c_void_p
            lib.oracle_row_flop.argtypes = [I64, P, P, I64, P, P]
            lib.oracle_symbolic_rows.argtypes = [I64, I64, P, P, I64, P, P, I64, P]
            lib.oracle_numeric_rows_f64.argtypes = [I64, I64, P, P, P, I64, P, P, P, I64, P, P, P, P]
            lib.oracle_numeric_rows_i64.argtypes = [I64, I64, P, P, P, I64, P, P, P, I64, P, P, P]
            lib.oracle_rows_to_threads.argtypes = [I64, P, I64, P]
            lib.oracle_phase_mt.argtypes = [ctypes.c_int, I64, P, P, P, P, I64, P, P, P, I64, P, P, P, P, P]
            for f in (lib.oracle_row_flop, lib.oracle_symbolic_rows, lib.oracle_numeric_rows_f64,
                      lib.oracle_numeric_rows_i64, lib.oracle_rows_to_threads, lib.oracle_phase_mt):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc} (index out of range or no memory)")


def is_integer(vals: np.ndarray) -> bool:
    return np.issubdtype(np.asarray(vals).dtype, np.integer)


def row_flop(A, B) -> np.ndarray:
    """flop[i] = sum over stored a_ik of nnz(b_k*) (Sec. 4.1)."""
    if A.ncols != B.nrows:
        raise ValueError("inner dimensions differ")
    lib = _load()
    arp, aci, brp = _c32(A.row_ptr), _c32(A.col_idx), _c32(B.row_ptr)
    flop = np.zeros(A.nrows, dtype=np.int64)
    _check(lib.oracle_row_flop(A.nrows, _p(arp), _p(aci), B.nrows, _p(brp), _p(flop)), "row_flop")
    return flop


def rows_to_threads(flop: np.ndarray, t: int) -> np.ndarray:
    """offset[0..t]: thread tid owns rows offset[tid]..offset[tid+1]-1 (Sec. 4.1, step 2)."""
    lib = _load()
    flop = np.ascontiguousarray(flop, dtype=np.int64)
    off = np.zeros(t + 1, dtype=np.int64)
    _check(lib.oracle_rows_to_threads(len(flop), _p(flop), t, _p(off)), "rows_to_threads")
    return off


def symbolic(A, B, nthreads: int = 1) -> np.ndarray:
    """nnz_row[i] = number of distinct columns in row i of A*B."""
    if A.ncols != B.nrows:
        raise ValueError("inner dimensions differ")
    lib = _load()
    arp, aci, brp, bci = _c32(A.row_ptr), _c32(A.col_idx), _c32(B.row_ptr), _c32(B.col_idx)
    nnz = np.zeros(A.nrows, dtype=np.int32)
    if nthreads <= 1:
        _check(lib.oracle_symbolic_rows(0, A.nrows, _p(arp), _p(aci), B.nrows, _p(brp), _p(bci), B.ncols,
                                        _p(nnz)), "symbolic")
    else:
        off = rows_to_threads(row_flop(A, B), nthreads)
        _check(lib.oracle_phase_mt(0, nthreads, _p(off), _p(arp), _p(aci), None, B.nrows, _p(brp), _p(bci),
                                   None, B.ncols, _p(nnz), None, None, None, None), "symbolic_mt")
    return nnz


def spgemm(A, B, nthreads: int = 1):
    """C = A*B (rows column-sorted). Returns (CSR, absbound) where absbound is
    (|A|*|B|) at each stored entry of C for floating-point inputs, else None."""
    from paper_1804_01698_gb300.inputs import CSR

    if A.ncols != B.nrows:
        raise ValueError("inner dimensions differ")
    lib = _load()
    arp, aci, brp, bci = _c32(A.row_ptr), _c32(A.col_idx), _c32(B.row_ptr), _c32(B.col_idx)
    nnz = symbolic(A, B, nthreads)
    crp = np.zeros(A.nrows + 1, dtype=np.int64)
    np.cumsum(nnz, out=crp[1:])
    if crp[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz(C) exceeds int32 indexing")
    crp = crp.astype(np.int32)
    total = int(crp[-1])
    cci = np.zeros(total, dtype=np.int32)
    integer = is_integer(A.vals)
    if integer != is_integer(B.vals):
        raise ValueError("A and B must both be integer or both floating point")
    if integer:
        av = np.ascontiguousarray(A.vals, dtype=np.int64)
        bv = np.ascontiguousarray(B.vals, dtype=np.int64)
        cv = np.zeros(total, dtype=np.int64)
        cabs = None
    else:
        av = np.ascontiguousarray(A.vals, dtype=np.float64)
        bv = np.ascontiguousarray(B.vals, dtype=np.float64)
        cv = np.zeros(total, dtype=np.float64)
        cabs = np.zeros(total, dtype=np.float64)
    if nthreads <= 1:
        if integer:
            rc = lib.oracle_numeric_rows_i64(0, A.nrows, _p(arp), _p(aci), _p(av), B.nrows, _p(brp), _p(bci),
                                             _p(bv), B.ncols, _p(crp), _p(cci), _p(cv))
        else:
            rc = lib.oracle_numeric_rows_f64(0, A.nrows, _p(arp), _p(aci), _p(av), B.nrows, _p(brp), _p(bci),
                                             _p(bv), B.ncols, _p(crp), _p(cci), _p(cv), _p(cabs))
    else:
        off = rows_to_threads(row_flop(A, B), nthreads)
        rc = lib.oracle_phase_mt(2 if integer else 1, nthreads, _p(off), _p(arp), _p(aci), _p(av), B.nrows,
                                 _p(brp), _p(bci), _p(bv), B.ncols, None, _p(crp), _p(cci), _p(cv), _p(cabs))
    _check(rc, "numeric")
    return CSR(A.nrows, B.ncols, crp, cci, cv), cabs


def select_rows(A, rows: np.ndarray):
    """CSR made of the given rows of A, in the given order (pure data movement)."""
    from paper_1804_01698_gb300.inputs import CSR

    rows = np.asarray(rows, dtype=np.int64)
    starts = A.row_ptr[rows].astype(np.int64)
    lens = A.row_ptr[rows + 1].astype(np.int64) - starts
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    idx = np.repeat(starts - rp[:-1], lens) + np.arange(int(rp[-1]), dtype=np.int64)
    return CSR(len(rows), A.ncols, rp.astype(np.int32), A.col_idx[idx], A.vals[idx])


def spgemm_rows(A, B, rows: np.ndarray, nthreads: int = 1):
    """Rows `rows` of A*B, as a CSR with len(rows) rows (and the abs bound)."""
    return spgemm(select_rows(A, rows), B, nthreads)
