"""Thin Python binding of libspgemm_gb300.so (the C ABI of include/spgemm.h).

Only argument marshalling happens here: torch tensors provide device memory
and the CUDA stream, and every step of the product runs in the library's
CUDA kernels.  The functions keep the C names:

    spgemm_plan_create, spgemm_symbolic, spgemm_numeric, spgemm_plan_destroy,
    spgemm_plan_stats, spgemm_plan_workspace_bytes, spgemm_plan_row_flop,
    spgemm_plan_sym_bins, spgemm_plan_row_nnz, spgemm, spgemm_status_string

Importing this module loads the library; it raises if the library has not
been built (there is no fallback).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

_LIB = None

SPGEMM_I64, SPGEMM_F32, SPGEMM_F64 = 0, 1, 2
SPGEMM_UNSORTED, SPGEMM_SORTED, SPGEMM_VALIDATE, SPGEMM_TIMING, SPGEMM_SERIAL = 0, 1, 2, 4, 8
SPGEMM_PROBE_CHUNK4 = 16
SPGEMM_COUNT_PROBES = 32
SPGEMM_HASH_LOW_BITS = 64
_HASHES = {"high": 0, "low": SPGEMM_HASH_LOW_BITS}
_PROBES = {"linear": 0, "chunk4": SPGEMM_PROBE_CHUNK4}
MAX_BINS = 24

_DTYPES = {torch.int64: SPGEMM_I64, torch.float32: SPGEMM_F32, torch.float64: SPGEMM_F64}
_TORCH = {v: k for k, v in _DTYPES.items()}


class SpgemmError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = library()
        msg = lib.spgemm_status_string(status).decode()
        detail = lib.spgemm_last_error().decode()
        super().__init__(f"{where}: {msg} ({status})" + (f": {detail}" if detail else ""))
        self.status = status


class CsrDesc(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("vals", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("total_flop", ctypes.c_int64), ("max_row_flop", ctypes.c_int64), ("nnz_c", ctypes.c_int64),
                ("n_sym_bins", ctypes.c_int32), ("n_num_bins", ctypes.c_int32),
                ("sym_bin_rows", ctypes.c_int64 * MAX_BINS), ("num_bin_rows", ctypes.c_int64 * MAX_BINS),
                ("sym_bin_table", ctypes.c_int32 * MAX_BINS), ("num_bin_table", ctypes.c_int32 * MAX_BINS),
                ("workspace_bytes", ctypes.c_int64), ("kernel_launches", ctypes.c_int32), ("state", ctypes.c_int32),
                ("sym_bin_flop", ctypes.c_int64 * MAX_BINS), ("num_bin_flop", ctypes.c_int64 * MAX_BINS),
                ("sym_probes", ctypes.c_int64), ("sym_inserts", ctypes.c_int64),
                ("num_probes", ctypes.c_int64), ("num_inserts", ctypes.c_int64),
                ("nnz_a_walked", ctypes.c_int64), ("long_rows", ctypes.c_int64), ("long_entries", ctypes.c_int64)]


class Tuning(ctypes.Structure):
    _fields_ = [("lanes_per_entry", ctypes.c_int32), ("reserved", ctypes.c_int32), ("bitmap_min_bound", ctypes.c_int64),
                ("max_nnz_c", ctypes.c_int64), ("long_row_min", ctypes.c_int64), ("warp_load_pct", ctypes.c_int32),
                ("block_load_pct", ctypes.c_int32)]


TUNING_KEYS = ("lanes_per_entry", "bitmap_min_bound", "max_nnz_c", "long_row_min", "warp_load_pct", "block_load_pct")


def _tuning(t):
    """A spgemm_tuning from a dict with keys among TUNING_KEYS (None: defaults;
    a missing key takes the default, 0)."""
    if t is None:
        return None
    unknown = set(t) - set(TUNING_KEYS)
    if unknown:
        raise ValueError(f"unknown tuning keys {sorted(unknown)}")
    return Tuning(int(t.get("lanes_per_entry", 0)), 0, int(t.get("bitmap_min_bound", 0)), int(t.get("max_nnz_c", 0)),
                  int(t.get("long_row_min", 0)), int(t.get("warp_load_pct", 0)), int(t.get("block_load_pct", 0)))


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("ms", ctypes.c_float), ("launches", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)

EXPORTED = ("spgemm_plan_create", "spgemm_symbolic", "spgemm_numeric", "spgemm_plan_destroy",
            "spgemm_plan_workspace_bytes", "spgemm_plan_stats", "spgemm_plan_row_flop", "spgemm_plan_sym_bins",
            "spgemm_plan_row_nnz", "spgemm_plan_kernel_times", "spgemm", "spgemm_status_string",
            "spgemm_last_error", "spgemm_symbolic_noalloc", "spgemm_batch_create", "spgemm_batch_symbolic",
            "spgemm_batch_numeric", "spgemm_batch_destroy", "spgemm_plan_create_tuned", "spgemm_batch_create_tuned",
            "spgemm_numeric_graph", "spgemm_host", "spgemm_bgraph_create", "spgemm_bgraph_launch",
            "spgemm_bgraph_wait", "spgemm_bgraph_product_nnz", "spgemm_bgraph_product_copy", "spgemm_bgraph_info",
            "spgemm_bgraph_destroy", "spgemm_numeric_rows")


def library_path() -> str:
    return _build.LIB


def library():
    """Load the library (once).  Raises if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"the CUDA SpGEMM library is not built ({path}); run __graft_entry__.build() "
                           "or python -m paper_1804_01698_gb300.build")
    lib = ctypes.CDLL(path)
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.spgemm_plan_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(CsrDesc), ctypes.POINTER(CsrDesc), I32,
                                       ctypes.c_uint, P]
    lib.spgemm_plan_create_tuned.argtypes = [ctypes.POINTER(P), ctypes.POINTER(CsrDesc), ctypes.POINTER(CsrDesc),
                                             I32, ctypes.c_uint, P, ctypes.POINTER(Tuning)]
    lib.spgemm_symbolic.argtypes = [P, P, ctypes.POINTER(I64)]
    lib.spgemm_numeric.argtypes = [P, P, P, P]
    lib.spgemm_numeric_graph.argtypes = [P, P, P, P]
    lib.spgemm_numeric_rows.argtypes = [P, I64, I64, P, P, P]
    lib.spgemm_plan_destroy.argtypes = [P]
    lib.spgemm_plan_workspace_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    lib.spgemm_plan_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.spgemm_plan_row_flop.argtypes = [P, P]
    lib.spgemm_plan_sym_bins.argtypes = [P, P, P]
    lib.spgemm_plan_row_nnz.argtypes = [P, P]
    lib.spgemm_plan_kernel_times.argtypes = [P, ctypes.POINTER(KernelTime), I32, ctypes.POINTER(I32)]
    lib.spgemm_batch_create.argtypes = [ctypes.POINTER(P), I64, ctypes.POINTER(CsrDesc), ctypes.POINTER(CsrDesc), I32,
                                        ctypes.c_uint, P]
    lib.spgemm_batch_create_tuned.argtypes = [ctypes.POINTER(P), I64, ctypes.POINTER(CsrDesc),
                                              ctypes.POINTER(CsrDesc), I32, ctypes.c_uint, P, ctypes.POINTER(Tuning)]
    lib.spgemm_batch_symbolic.argtypes = [P, P, ctypes.POINTER(I64), P]
    lib.spgemm_batch_numeric.argtypes = [P, P, P, P]
    lib.spgemm_batch_destroy.argtypes = [P]
    lib.spgemm_batch_plan.argtypes = [P]
    lib.spgemm_batch_plan.restype = P
    lib.spgemm_symbolic_noalloc.argtypes = [ctypes.POINTER(CsrDesc), ctypes.POINTER(CsrDesc), P, ctypes.POINTER(I64), P]
    lib.spgemm.argtypes = [ctypes.POINTER(CsrDesc), ctypes.POINTER(CsrDesc), I32, ctypes.c_uint, P, ALLOC_FN, P,
                           ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(I64)]
    lib.spgemm_host.argtypes = [ctypes.POINTER(CsrDesc), ctypes.POINTER(CsrDesc), I32, ctypes.c_uint, P, I32, ALLOC_FN,
                                P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(I64)]
    lib.spgemm_bgraph_create.argtypes = [ctypes.POINTER(P), I64, ctypes.POINTER(CsrDesc), ctypes.POINTER(CsrDesc),
                                         I32, ctypes.c_uint, P, ctypes.POINTER(Tuning), I64, ctypes.c_double]
    lib.spgemm_bgraph_launch.argtypes = [P, P]
    lib.spgemm_bgraph_wait.argtypes = [P]
    lib.spgemm_bgraph_product_nnz.argtypes = [P, I64, ctypes.POINTER(I64)]
    lib.spgemm_bgraph_product_copy.argtypes = [P, I64, P, P, P, P]
    lib.spgemm_bgraph_info.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]
    lib.spgemm_bgraph_destroy.argtypes = [P]
    for name in EXPORTED:
        getattr(lib, name).restype = ctypes.c_int
    lib.spgemm_status_string.argtypes = [I32]
    lib.spgemm_status_string.restype = ctypes.c_char_p
    lib.spgemm_last_error.argtypes = []
    lib.spgemm_last_error.restype = ctypes.c_char_p
    _LIB = lib
    return lib


def _check(status: int, where: str):
    if status != 0:
        raise SpgemmError(status, where)


@dataclass
class DeviceCSR:
    """CSR matrix in device memory (torch tensors: int32 row_ptr/col_idx, values)."""

    nrows: int
    ncols: int
    row_ptr: torch.Tensor
    col_idx: torch.Tensor
    vals: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.col_idx.numel())

    def desc(self) -> CsrDesc:
        return CsrDesc(self.nrows, self.ncols, self.nnz, self.row_ptr.data_ptr(),
                       self.col_idx.data_ptr() if self.nnz else None, self.vals.data_ptr() if self.nnz else None)

    def to_host(self):
        from .inputs import CSR
        return CSR(self.nrows, self.ncols, self.row_ptr.cpu().numpy(), self.col_idx.cpu().numpy(),
                   self.vals.cpu().numpy())


class _Caller:
    """The caller's current stream, read once per call, against the stream a
    plan or batch runs on.  When they are the same stream (the usual case)
    every method below is a no-op; entering torch.cuda.stream and reading
    the current stream cost microseconds each, a large share of a small
    product."""

    __slots__ = ("stream", "cur", "same")

    def __init__(self, stream):
        self.stream = stream
        try:
            # (stream id, device index, device type) of the current stream,
            # without building a Stream object
            sid, dev, _ = torch._C._cuda_getCurrentStream(stream.device_index)
            self.same = sid == stream.stream_id and dev == stream.device_index
            self.cur = None if self.same else torch.cuda.current_stream(stream.device)
        except AttributeError:
            self.cur = torch.cuda.current_stream(stream.device)
            self.same = self.cur == stream

    def on(self):
        """Context for allocations that belong to the plan's stream in torch's
        caching allocator."""
        return contextlib.nullcontext() if self.same else torch.cuda.stream(self.stream)

    def before(self) -> None:
        """Work queued on the plan's stream starts after what the caller's
        stream has queued so far (the operands may still be in flight there)."""
        if not self.same:
            self.stream.wait_stream(self.cur)

    def after(self, *tensors) -> None:
        """Results written on the plan's stream, used on the caller's: the
        caller's stream waits for the plan's, and the tensors' memory (which
        belongs to the plan's stream) is not reused before the caller's work
        on them has finished (torch's caching allocator only tracks the
        allocating stream otherwise)."""
        if self.same:
            return
        self.cur.wait_stream(self.stream)
        for t in tensors:
            if t is not None and t.numel() > 0:
                t.record_stream(self.cur)


def hand_over(stream, *tensors) -> None:
    """Results written on `stream`, used on the caller's current stream (see
    _Caller.after)."""
    _Caller(stream).after(*tensors)


def _after_caller(stream) -> None:
    """Work queued on `stream` starts after the caller's queued work."""
    _Caller(stream).before()


def to_device(m, device="cuda", dtype=None, non_blocking=False) -> DeviceCSR:
    """Copy a host CSR (paper_1804_01698_gb300.inputs.CSR) to the device."""
    vals = torch.from_numpy(np.ascontiguousarray(m.vals))
    if dtype is not None:
        vals = vals.to(dtype)
    rp = torch.from_numpy(np.ascontiguousarray(m.row_ptr, dtype=np.int32))
    ci = torch.from_numpy(np.ascontiguousarray(m.col_idx, dtype=np.int32))
    return DeviceCSR(m.nrows, m.ncols, rp.to(device, non_blocking=non_blocking),
                     ci.to(device, non_blocking=non_blocking), vals.to(device, non_blocking=non_blocking))


def _stream_ptr(stream) -> int | None:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


class Plan:
    """A plan for C = A*B; methods mirror spgemm_symbolic / spgemm_numeric."""

    def __init__(self, A: DeviceCSR, B: DeviceCSR, sorted_output: bool = True, stream=None, timing: bool = False,
                 serial: bool = False, probe: str = "linear", tuning: dict | None = None, count_probes: bool = False,
                 hash: str = "high"):
        self.lib = library()
        if A.vals.dtype != B.vals.dtype or A.vals.dtype not in _DTYPES:
            raise TypeError("A and B must share a value dtype among int64, float32, float64")
        self.A, self.B = A, B
        self.dtype = A.vals.dtype
        self.device = A.row_ptr.device
        if stream is None:  # the caller's own stream: nothing to wait for
            self.stream = torch.cuda.current_stream(self.device)
        else:
            self.stream = stream
            _after_caller(stream)
        flags = (SPGEMM_SORTED if sorted_output else SPGEMM_UNSORTED) | (SPGEMM_TIMING if timing else 0) | \
            (SPGEMM_SERIAL if serial else 0) | _PROBES[probe] | _HASHES[hash] | \
            (SPGEMM_COUNT_PROBES if count_probes else 0)
        self._a, self._b = A.desc(), B.desc()
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            self._tuning = _tuning(tuning)
            _check(self.lib.spgemm_plan_create_tuned(ctypes.byref(h), ctypes.byref(self._a), ctypes.byref(self._b),
                                                     _DTYPES[self.dtype], flags, _stream_ptr(self.stream),
                                                     ctypes.byref(self._tuning) if self._tuning else None),
                   "spgemm_plan_create_tuned")
        self.handle = h
        self.c_row_ptr = None
        self.nnz_c = None

    def symbolic(self) -> int:
        c = _Caller(self.stream)
        with c.on():
            self.c_row_ptr = torch.empty(self.A.nrows + 1, dtype=torch.int32, device=self.device)
        nnz = ctypes.c_int64()
        with torch.cuda.device(self.device):
            _check(self.lib.spgemm_symbolic(self.handle, self.c_row_ptr.data_ptr(), ctypes.byref(nnz)),
                   "spgemm_symbolic")
        self.nnz_c = int(nnz.value)
        c.after(self.c_row_ptr)
        return self.nnz_c

    def numeric(self, c_col_idx: torch.Tensor | None = None, c_vals: torch.Tensor | None = None) -> DeviceCSR:
        c = _Caller(self.stream)
        with c.on():
            if c_col_idx is None:
                c_col_idx = torch.empty(max(self.nnz_c, 0), dtype=torch.int32, device=self.device)
            if c_vals is None:
                c_vals = torch.empty(max(self.nnz_c, 0), dtype=self.dtype, device=self.device)
        # the plan's stream must not run ahead of work the caller queued on the
        # operands (new values) or on these buffers
        c.before()
        with torch.cuda.device(self.device):
            _check(self.lib.spgemm_numeric(self.handle, self.c_row_ptr.data_ptr(),
                                           c_col_idx.data_ptr() if self.nnz_c else None,
                                           c_vals.data_ptr() if self.nnz_c else None), "spgemm_numeric")
        c.after(self.c_row_ptr, c_col_idx, c_vals)
        return DeviceCSR(self.A.nrows, self.B.ncols, self.c_row_ptr, c_col_idx, c_vals)

    def numeric_rows(self, row_begin: int, row_end: int, C: DeviceCSR) -> DeviceCSR:
        """Numeric phase of rows row_begin .. row_end-1 only, into C's buffers
        (from an earlier numeric() or allocated for nnz_c entries); every other
        row's entries are left as they are."""
        c = _Caller(self.stream)
        c.before()
        with torch.cuda.device(self.device):
            _check(self.lib.spgemm_numeric_rows(self.handle, row_begin, row_end, self.c_row_ptr.data_ptr(),
                                                C.col_idx.data_ptr() if self.nnz_c else None,
                                                C.vals.data_ptr() if self.nnz_c else None), "spgemm_numeric_rows")
        c.after(C.col_idx, C.vals)
        return C

    def numeric_graph(self, C: DeviceCSR) -> DeviceCSR:
        """Numeric phase again into C's buffers through a CUDA graph (captured
        on the first call for these buffers, replayed afterwards).  Only the
        values of A and B may have changed since the first numeric()."""
        c = _Caller(self.stream)
        c.before()
        with torch.cuda.device(self.device):
            _check(self.lib.spgemm_numeric_graph(self.handle, self.c_row_ptr.data_ptr(),
                                                 C.col_idx.data_ptr() if self.nnz_c else None,
                                                 C.vals.data_ptr() if self.nnz_c else None), "spgemm_numeric_graph")
        c.after(C.col_idx, C.vals)
        return C

    def stats(self) -> dict:
        s = Stats()
        status = self.lib.spgemm_plan_stats(self.handle, ctypes.byref(s))
        out = {name: getattr(s, name) for name, _ in Stats._fields_}
        for key in ("sym_bin_rows", "sym_bin_table", "sym_bin_flop"):
            out[key] = list(getattr(s, key))[: s.n_sym_bins]
        for key in ("num_bin_rows", "num_bin_table", "num_bin_flop"):
            out[key] = list(getattr(s, key))[: s.n_num_bins]
        out["status"] = status
        return out

    def kernel_times(self) -> dict:
        """{kernel name: (milliseconds, launches)} for plans created with timing=True."""
        buf = (KernelTime * 64)()
        n = ctypes.c_int()
        _check(self.lib.spgemm_plan_kernel_times(self.handle, buf, 64, ctypes.byref(n)), "spgemm_plan_kernel_times")
        return {buf[j].name.decode(): (float(buf[j].ms), int(buf[j].launches)) for j in range(min(n.value, 64))}

    def workspace_bytes(self) -> int:
        v = ctypes.c_size_t()
        _check(self.lib.spgemm_plan_workspace_bytes(self.handle, ctypes.byref(v)), "spgemm_plan_workspace_bytes")
        return int(v.value)

    def row_flop(self) -> torch.Tensor:
        c = _Caller(self.stream)
        with c.on():
            out = torch.empty(self.A.nrows, dtype=torch.int64, device=self.device)
        _check(self.lib.spgemm_plan_row_flop(self.handle, out.data_ptr()), "spgemm_plan_row_flop")
        c.after(out)
        return out

    def sym_bins(self):
        s = Stats()
        self.lib.spgemm_plan_stats(self.handle, ctypes.byref(s))
        offs = (ctypes.c_int64 * (s.n_sym_bins + 1))()
        c = _Caller(self.stream)
        with c.on():
            perm = torch.empty(max(self.A.nrows, 1), dtype=torch.int32, device=self.device)
        _check(self.lib.spgemm_plan_sym_bins(self.handle, perm.data_ptr(), offs), "spgemm_plan_sym_bins")
        c.after(perm)
        offsets = list(offs)
        return perm[: offsets[-1]], offsets

    def row_nnz(self) -> torch.Tensor:
        c = _Caller(self.stream)
        with c.on():
            out = torch.empty(self.A.nrows, dtype=torch.int32, device=self.device)
        _check(self.lib.spgemm_plan_row_nnz(self.handle, out.data_ptr()), "spgemm_plan_row_nnz")
        c.after(out)
        return out

    def destroy(self):
        if getattr(self, "handle", None):
            self.lib.spgemm_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def spgemm_plan_create(A: DeviceCSR, B: DeviceCSR, sorted_output: bool = True, stream=None,
                       timing: bool = False, serial: bool = False) -> Plan:
    return Plan(A, B, sorted_output, stream, timing, serial)


def spgemm_plan_kernel_times(plan: Plan) -> dict:
    return plan.kernel_times()


def spgemm_symbolic(plan: Plan) -> int:
    return plan.symbolic()


def spgemm_numeric(plan: Plan, c_col_idx=None, c_vals=None) -> DeviceCSR:
    return plan.numeric(c_col_idx, c_vals)


def spgemm_plan_destroy(plan: Plan) -> None:
    plan.destroy()


def spgemm_plan_stats(plan: Plan) -> dict:
    return plan.stats()


def spgemm_plan_workspace_bytes(plan: Plan) -> int:
    return plan.workspace_bytes()


def spgemm_plan_row_flop(plan: Plan) -> torch.Tensor:
    return plan.row_flop()


def spgemm_plan_sym_bins(plan: Plan):
    return plan.sym_bins()


def spgemm_plan_row_nnz(plan: Plan) -> torch.Tensor:
    return plan.row_nnz()


def spgemm_status_string(status: int) -> str:
    return library().spgemm_status_string(status).decode()


def spgemm_symbolic_noalloc(A: DeviceCSR, B: DeviceCSR, c_row_ptr: torch.Tensor, stream=None) -> int:
    """Row pointers of C = A*B into the caller's c_row_ptr (int32, A.nrows+1, on A's
    device) without any device allocation by the library; returns nnz(C).
    For callers that must not allocate device memory while they run: the
    library uses a static device array instead (one call at a time per GPU)."""
    lib = library()
    dev = A.row_ptr.device
    if (c_row_ptr.dtype != torch.int32 or not c_row_ptr.is_contiguous() or c_row_ptr.numel() < A.nrows + 1
            or c_row_ptr.device != dev):
        raise ValueError(f"c_row_ptr must be a contiguous int32 tensor of at least {A.nrows + 1} elements on {dev}")
    a, b = A.desc(), B.desc()
    nnz = ctypes.c_int64()
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    _after_caller(s)
    with torch.cuda.device(A.row_ptr.device):
        _check(lib.spgemm_symbolic_noalloc(ctypes.byref(a), ctypes.byref(b), c_row_ptr.data_ptr(), ctypes.byref(nnz),
                                           _stream_ptr(s)), "spgemm_symbolic_noalloc")
    return int(nnz.value)


def spgemm(A: DeviceCSR, B: DeviceCSR, sorted_output: bool = True, stream=None) -> DeviceCSR:
    """One-shot C = A*B through the C entry point spgemm(); C's buffers are
    torch tensors allocated through the allocator callback."""
    lib = library()
    if A.vals.dtype != B.vals.dtype or A.vals.dtype not in _DTYPES:
        raise TypeError("A and B must share a value dtype among int64, float32, float64")
    device = A.row_ptr.device
    keep: dict[int, torch.Tensor] = {}

    s = stream if stream is not None else torch.cuda.current_stream(device)
    c = _Caller(s)

    def _alloc(nbytes, _ctx):
        with c.on():
            t = torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)
        keep[t.data_ptr()] = t
        return t.data_ptr()

    cb = ALLOC_FN(_alloc)
    a, b = A.desc(), B.desc()
    rp, ci, cv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    nnz = ctypes.c_int64()
    c.before()
    with torch.cuda.device(device):
        status = lib.spgemm(ctypes.byref(a), ctypes.byref(b), _DTYPES[A.vals.dtype],
                            SPGEMM_SORTED if sorted_output else SPGEMM_UNSORTED, _stream_ptr(s), cb, None,
                            ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(cv), ctypes.byref(nnz))
    _check(status, "spgemm")
    n = int(nnz.value)
    rpt = keep[rp.value][: (A.nrows + 1) * 4].view(torch.int32)
    cit = keep[ci.value][: n * 4].view(torch.int32)
    esz = torch.empty(0, dtype=A.vals.dtype).element_size()
    cvt = keep[cv.value][: n * esz].view(A.vals.dtype)
    c.after(rpt, cit, cvt)
    return DeviceCSR(A.nrows, B.ncols, rpt, cit, cvt)


class HostArena:
    """Page-locked host memory for spgemm_host's results: one pinned buffer,
    allocated once, handed out in 256-byte aligned pieces.  Pinning memory
    costs far more than the product, so a caller that runs many products
    keeps one arena and calls reset() before each call (the previous
    results are overwritten then)."""

    def __init__(self, nbytes: int):
        self.buf = torch.empty(int(nbytes), dtype=torch.uint8).pin_memory()
        self.off = 0

    @staticmethod
    def bytes_for(nrows: int, nnz: int, value_size: int) -> int:
        """Arena size that holds one result of nrows rows and nnz entries."""
        return 3 * 256 + (nrows + 1) * 4 + max(nnz * 4, 16) + max(nnz * value_size, 16)

    def alloc(self, nbytes: int):
        start = (self.off + 255) // 256 * 256
        if start + nbytes > self.buf.numel():
            return None
        self.off = start + nbytes
        return self.buf[start:start + nbytes]

    def reset(self) -> None:
        self.off = 0


def _host_array(x, dtype=None):
    """A CPU torch tensor over a host array (numpy arrays are wrapped, not copied)."""
    t = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x))
    if t.device.type != "cpu" or not t.is_contiguous():
        raise ValueError("spgemm_host takes contiguous host arrays")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return t


def spgemm_host(A, B, sorted_output: bool = True, row_blocks: int = 0, arena: HostArena | None = None,
                stream=None, device=None):
    """C = A*B with A, B and C in host memory, through the C entry point
    spgemm_host(): the copy of C to the host overlaps the numeric phase,
    block of rows by block of rows.

    A and B are host CSR matrices (paper_1804_01698_gb300.inputs.CSR or
    anything with nrows, ncols and row_ptr/col_idx/vals as numpy arrays or
    CPU tensors; pinned tensors let the copies overlap).  C is returned as
    an inputs.CSR whose arrays live in `arena` (or in freshly pinned
    buffers when no arena is given).  row_blocks=0 lets the library choose."""
    lib = library()
    from .inputs import CSR
    arp, aci = _host_array(A.row_ptr, torch.int32), _host_array(A.col_idx, torch.int32)
    brp, bci = _host_array(B.row_ptr, torch.int32), _host_array(B.col_idx, torch.int32)
    av, bv = _host_array(A.vals), _host_array(B.vals)
    if av.dtype != bv.dtype or av.dtype not in _DTYPES:
        raise TypeError("A and B must share a value dtype among int64, float32, float64")
    same = A is B
    dev = torch.device("cuda") if device is None else torch.device(device)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    keep: dict[int, torch.Tensor] = {}

    def _alloc(nbytes, _ctx):
        n = max(int(nbytes), 16)
        t = arena.alloc(n) if arena is not None else torch.empty(n, dtype=torch.uint8).pin_memory()
        if t is None:
            return None
        keep[t.data_ptr()] = t
        return t.data_ptr()

    def desc(m, rp, ci, v):
        nnz = int(ci.numel())
        return CsrDesc(m.nrows, m.ncols, nnz, rp.data_ptr(), ci.data_ptr() if nnz else None,
                       v.data_ptr() if nnz else None)

    a = desc(A, arp, aci, av)
    b = a if same else desc(B, brp, bci, bv)
    cb = ALLOC_FN(_alloc)
    rp, ci, cv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    nnz = ctypes.c_int64()
    with torch.cuda.device(dev):
        status = lib.spgemm_host(ctypes.byref(a), ctypes.byref(b), _DTYPES[av.dtype],
                                 SPGEMM_SORTED if sorted_output else SPGEMM_UNSORTED, _stream_ptr(s), int(row_blocks),
                                 cb, None, ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(cv), ctypes.byref(nnz))
    _check(status, "spgemm_host")
    n = int(nnz.value)
    rpt = keep[rp.value][: (A.nrows + 1) * 4].view(torch.int32)
    cit = keep[ci.value][: n * 4].view(torch.int32)
    cvt = keep[cv.value][: n * av.element_size()].view(av.dtype)
    return CSR(A.nrows, B.ncols, rpt.numpy(), cit.numpy(), cvt.numpy())


class Batch:
    """Independent products C_p = A_p * B_p run as one plan (block-diagonal
    packing on the device); mirrors spgemm_batch_create / _symbolic / _numeric."""

    def __init__(self, As, Bs, sorted_output: bool = True, stream=None, timing: bool = False, serial: bool = False,
                 probe: str = "linear", tuning: dict | None = None, hash: str = "high"):
        self.lib = library()
        if len(As) != len(Bs) or not As:
            raise ValueError("need the same positive number of A and B operands")
        self.dtype = As[0].vals.dtype
        if self.dtype not in _DTYPES or any(m.vals.dtype != self.dtype for m in list(As) + list(Bs)):
            raise TypeError("all operands must share one value dtype among int64, float32, float64")
        self.As, self.Bs = list(As), list(Bs)
        self.device = As[0].row_ptr.device
        if stream is None:  # the caller's own stream: nothing to wait for
            self.stream = torch.cuda.current_stream(self.device)
        else:
            self.stream = stream
            _after_caller(stream)
        flags = (SPGEMM_SORTED if sorted_output else SPGEMM_UNSORTED) | (SPGEMM_TIMING if timing else 0) | \
            (SPGEMM_SERIAL if serial else 0) | _PROBES[probe] | _HASHES[hash]
        n = len(As)
        self._a = (CsrDesc * n)(*[m.desc() for m in As])
        self._b = (CsrDesc * n)(*[m.desc() for m in Bs])
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            self._tuning = _tuning(tuning)
            _check(self.lib.spgemm_batch_create_tuned(ctypes.byref(h), n, self._a, self._b, _DTYPES[self.dtype], flags,
                                                      _stream_ptr(self.stream),
                                                      ctypes.byref(self._tuning) if self._tuning else None),
                   "spgemm_batch_create_tuned")
        self.handle = h
        self.nprod = n
        self.m = sum(a.nrows for a in As)
        self.c_row_ptr = None
        self.nnz_c = None
        self.row_off = None

    def symbolic(self) -> int:
        c = _Caller(self.stream)
        with c.on():
            self.c_row_ptr = torch.empty(self.m + 1, dtype=torch.int32, device=self.device)
        nnz = ctypes.c_int64()
        off = (ctypes.c_int64 * (self.nprod + 1))()
        with torch.cuda.device(self.device):
            _check(self.lib.spgemm_batch_symbolic(self.handle, self.c_row_ptr.data_ptr(), ctypes.byref(nnz), off),
                   "spgemm_batch_symbolic")
        c.after(self.c_row_ptr)
        self.nnz_c = int(nnz.value)
        self.row_off = list(off)
        return self.nnz_c

    def numeric(self):
        """Returns (c_row_ptr, c_col_idx, c_vals) of the packed C; columns are local to each product."""
        c = _Caller(self.stream)
        with c.on():
            ci = torch.empty(max(self.nnz_c, 0), dtype=torch.int32, device=self.device)
            cv = torch.empty(max(self.nnz_c, 0), dtype=self.dtype, device=self.device)
        with torch.cuda.device(self.device):
            _check(self.lib.spgemm_batch_numeric(self.handle, self.c_row_ptr.data_ptr(),
                                                 ci.data_ptr() if self.nnz_c else None,
                                                 cv.data_ptr() if self.nnz_c else None), "spgemm_batch_numeric")
        self.c_col_idx, self.c_vals = ci, cv
        c.after(self.c_row_ptr, ci, cv)
        return self.c_row_ptr, ci, cv

    def product(self, p: int, row_ptr_host=None) -> DeviceCSR:
        """Product p of the batch as a DeviceCSR view (row_ptr rebased to 0),
        for use on the current stream (which may differ from the batch's)."""
        hand_over(self.stream, self.c_row_ptr, self.c_col_idx, self.c_vals)
        r0, r1 = self.row_off[p], self.row_off[p + 1]
        rp = self.c_row_ptr[r0:r1 + 1]
        if row_ptr_host is not None:
            e0, e1 = int(row_ptr_host[r0]), int(row_ptr_host[r1])
        else:
            e0, e1 = int(rp[0].item()), int(rp[-1].item())
        return DeviceCSR(r1 - r0, self.Bs[p].ncols, rp - e0, self.c_col_idx[e0:e1], self.c_vals[e0:e1])

    def workspace_bytes(self) -> int:
        v = ctypes.c_size_t()
        _check(self.lib.spgemm_plan_workspace_bytes(self.lib.spgemm_batch_plan(self.handle), ctypes.byref(v)),
               "spgemm_plan_workspace_bytes")
        return int(v.value)

    def plan_stats(self) -> dict:
        s = Stats()
        status = self.lib.spgemm_plan_stats(self.lib.spgemm_batch_plan(self.handle), ctypes.byref(s))
        out = {name: getattr(s, name) for name, _ in Stats._fields_}
        for key in ("sym_bin_rows", "sym_bin_table", "sym_bin_flop"):
            out[key] = list(getattr(s, key))[: s.n_sym_bins]
        for key in ("num_bin_rows", "num_bin_table", "num_bin_flop"):
            out[key] = list(getattr(s, key))[: s.n_num_bins]
        out["status"] = status
        return out

    def kernel_times(self) -> dict:
        buf = (KernelTime * 64)()
        n = ctypes.c_int()
        _check(self.lib.spgemm_plan_kernel_times(self.lib.spgemm_batch_plan(self.handle), buf, 64, ctypes.byref(n)),
               "spgemm_plan_kernel_times")
        return {buf[j].name.decode(): (float(buf[j].ms), int(buf[j].launches)) for j in range(min(n.value, 64))}

    def destroy(self):
        if getattr(self, "handle", None):
            self.lib.spgemm_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def spgemm_batch_create(As, Bs, sorted_output: bool = True, stream=None, timing: bool = False) -> Batch:
    return Batch(As, Bs, sorted_output, stream, timing)


def spgemm_batch_symbolic(batch: Batch) -> int:
    return batch.symbolic()


def spgemm_batch_numeric(batch: Batch):
    return batch.numeric()


def spgemm_batch_destroy(batch: Batch) -> None:
    batch.destroy()


class BatchGraph:
    """Independent products C_p = A_p * B_p, all of them in one CUDA graph
    launch; mirrors spgemm_bgraph_create / _launch / _wait / _product_*.
    The operands stay borrowed (their tensors must outlive the object):
    every launch recomputes every product from their current contents."""

    def __init__(self, As, Bs, sorted_output: bool = True, stream=None, probe: str = "linear",
                 tuning: dict | None = None, hash: str = "high", wave_nnz: int = 0, pool_slack: float = 0.0):
        self.lib = library()
        if len(As) != len(Bs) or not As:
            raise ValueError("need the same positive number of A and B operands")
        self.dtype = As[0].vals.dtype
        if self.dtype not in _DTYPES or any(m.vals.dtype != self.dtype for m in list(As) + list(Bs)):
            raise TypeError("all operands must share one value dtype among int64, float32, float64")
        self.As, self.Bs = list(As), list(Bs)
        self.device = As[0].row_ptr.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        flags = (SPGEMM_SORTED if sorted_output else SPGEMM_UNSORTED) | _PROBES[probe] | _HASHES[hash]
        n = len(As)
        self._a = (CsrDesc * n)(*[m.desc() for m in As])
        self._b = (CsrDesc * n)(*[m.desc() for m in Bs])
        h = ctypes.c_void_p()
        _after_caller(self.stream)
        with torch.cuda.device(self.device):
            self._tuning = _tuning(tuning)
            _check(self.lib.spgemm_bgraph_create(ctypes.byref(h), n, self._a, self._b, _DTYPES[self.dtype], flags,
                                                 _stream_ptr(self.stream),
                                                 ctypes.byref(self._tuning) if self._tuning else None,
                                                 int(wave_nnz), float(pool_slack)), "spgemm_bgraph_create")
        self.handle = h
        self.nprod = n

    def launch(self):
        """One cudaGraphLaunch of the whole batch on the object's stream (no host sync)."""
        with torch.cuda.device(self.device):
            _check(self.lib.spgemm_bgraph_launch(self.handle, _stream_ptr(self.stream)), "spgemm_bgraph_launch")

    def wait(self):
        with torch.cuda.device(self.device):
            _check(self.lib.spgemm_bgraph_wait(self.handle), "spgemm_bgraph_wait")

    def info(self) -> dict:
        w, k, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib.spgemm_bgraph_info(self.handle, ctypes.byref(w), ctypes.byref(k), ctypes.byref(b)),
               "spgemm_bgraph_info")
        return {"waves": w.value, "kernel_nodes": k.value, "bytes": b.value}

    def product(self, p: int) -> DeviceCSR:
        """C_p of the last launch (after wait()), copied into new tensors."""
        nnz = ctypes.c_int64()
        _check(self.lib.spgemm_bgraph_product_nnz(self.handle, p, ctypes.byref(nnz)), "spgemm_bgraph_product_nnz")
        A, B = self.As[p], self.Bs[p]
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            rp = torch.empty(A.nrows + 1, dtype=torch.int32, device=self.device)
            ci = torch.empty(max(nnz.value, 0), dtype=torch.int32, device=self.device)
            cv = torch.empty(max(nnz.value, 0), dtype=self.dtype, device=self.device)
            _check(self.lib.spgemm_bgraph_product_copy(self.handle, p, rp.data_ptr(),
                                                       ci.data_ptr() if nnz.value else None,
                                                       cv.data_ptr() if nnz.value else None,
                                                       _stream_ptr(self.stream)), "spgemm_bgraph_product_copy")
        return DeviceCSR(A.nrows, B.ncols, rp, ci, cv)

    def destroy(self):
        if self.handle:
            self.lib.spgemm_bgraph_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
