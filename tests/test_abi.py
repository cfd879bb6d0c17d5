"""CPU checks of the C ABI: the library builds, loads and exports every
function include/spgemm.h declares, the ctypes mirrors match the C struct
layouts, and argument validation that happens before any CUDA call."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1804_01698_gb300 import build as sgbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spgemm.h")


@pytest.fixture(scope="module")
def lib():
    sgbuild.build()
    from paper_1804_01698_gb300 import binding
    return binding.library()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SPGEMM_API\s+(?:const\s+)?\w+\s*\*?\s*(spgemm\w*)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("spgemm_plan_create", "spgemm_symbolic", "spgemm_numeric", "spgemm", "spgemm_plan_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", sgbuild.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_struct_layout_matches_c(tmp_path):
    from paper_1804_01698_gb300 import binding
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "spgemm.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(spgemm_csr), offsetof(spgemm_csr, vals),"
        " sizeof(spgemm_stats), offsetof(spgemm_stats, sym_bin_table), offsetof(spgemm_stats, workspace_bytes),"
        " offsetof(spgemm_stats, num_bin_flop)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    S, C = binding.Stats, binding.CsrDesc
    assert got == [ctypes.sizeof(C), C.vals.offset, ctypes.sizeof(S), S.sym_bin_table.offset,
                   S.workspace_bytes.offset, S.num_bin_flop.offset]


def test_tuning_layout_matches_c(tmp_path):
    from paper_1804_01698_gb300 import binding
    src = tmp_path / "tuning.c"
    fields = [name for name, _ in binding.Tuning._fields_]
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "spgemm.h"\nint main(void){printf("%zu'
                   + " %zu" * len(fields) + '\\n", sizeof(spgemm_tuning)'
                   + "".join(f", offsetof(spgemm_tuning, {f})" for f in fields) + "); return 0;}\n")
    exe = tmp_path / "tuning"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    T = binding.Tuning
    assert got == [ctypes.sizeof(T)] + [getattr(T, f).offset for f in fields]
    S = binding.Stats
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "spgemm.h"\nint main(void){printf("%zu %zu\\n",'
                   ' sizeof(spgemm_stats), offsetof(spgemm_stats, long_entries)); return 0;}\n')
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    assert got == [ctypes.sizeof(S), S.long_entries.offset]


def test_status_strings(lib):
    assert lib.spgemm_status_string(0) == b"ok"
    assert b"overflow" in lib.spgemm_status_string(-4)
    assert lib.spgemm_status_string(12345) == b"unknown status"


def test_argument_validation_before_any_cuda_call(lib):
    from paper_1804_01698_gb300 import binding
    a = binding.CsrDesc(2, 3, 0, 16, None, None)
    b = binding.CsrDesc(4, 3, 0, 16, None, None)        # inner dimensions differ (3 != 4)
    h = ctypes.c_void_p()
    assert lib.spgemm_plan_create(ctypes.byref(h), ctypes.byref(a), ctypes.byref(b), 2, 1, None) == -1
    assert h.value is None
    b_ok = binding.CsrDesc(3, 3, 0, 16, None, None)
    assert lib.spgemm_plan_create(ctypes.byref(h), ctypes.byref(a), ctypes.byref(b_ok), 7, 1, None) == -1  # dtype
    assert lib.spgemm_plan_create(ctypes.byref(h), ctypes.byref(a), ctypes.byref(b_ok), 2, 1 << 12, None) == -1  # flags
    neg = binding.CsrDesc(-1, 3, 0, 16, None, None)
    assert lib.spgemm_plan_create(ctypes.byref(h), ctypes.byref(neg), ctypes.byref(b_ok), 2, 1, None) == -1
    nnz_no_ptr = binding.CsrDesc(2, 3, 5, 16, None, None)
    assert lib.spgemm_plan_create(ctypes.byref(h), ctypes.byref(nnz_no_ptr), ctypes.byref(b_ok), 2, 1, None) == -1
    assert lib.spgemm_plan_create(None, ctypes.byref(a), ctypes.byref(b_ok), 2, 1, None) == -1
    assert lib.spgemm_plan_destroy(None) == 0
    assert lib.spgemm_symbolic(None, None, None) == -1
    assert lib.spgemm_numeric(None, None, None, None) == -1
    assert lib.spgemm_numeric_rows(None, 0, 1, None, None, None) == -1


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    from paper_1804_01698_gb300 import binding
    monkeypatch.setattr(binding, "_LIB", None)
    monkeypatch.setattr(binding, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        binding.library()


def test_host_entry_point_checks_before_any_cuda_call(lib):
    """spgemm_host validates its arguments, and the host row pointers of A
    that index its row blocks, before it touches the device."""
    import numpy as np
    from paper_1804_01698_gb300 import binding
    rp = np.array([0, 1, 3], dtype=np.int32)           # 2 rows, 3 entries
    ci = np.array([0, 1, 2], dtype=np.int32)
    v = np.ones(3)
    a = binding.CsrDesc(2, 3, 3, rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
    b_bad = binding.CsrDesc(4, 3, 0, rp.ctypes.data, None, None)   # 3 != 4
    b_ok = binding.CsrDesc(3, 3, 0, np.zeros(4, np.int32).ctypes.data, None, None)
    calls = []

    def alloc(nbytes, _ctx):
        calls.append(nbytes)
        return None

    cb = binding.ALLOC_FN(alloc)
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    out = [P(), P(), P()]
    nnz = I64(-1)

    def call(A, B, dtype=2, flags=1, alloc_fn=cb):
        return lib.spgemm_host(ctypes.byref(A), ctypes.byref(B), dtype, flags, None, 0, alloc_fn, None,
                               ctypes.byref(out[0]), ctypes.byref(out[1]), ctypes.byref(out[2]), ctypes.byref(nnz))

    assert call(a, b_bad) == -1                         # inner dimensions differ
    assert call(a, b_ok, dtype=9) == -1                 # value type
    assert call(a, b_ok, flags=4) == -1                 # SPGEMM_TIMING needs a plan the caller keeps
    assert b"TIMING" in lib.spgemm_last_error()
    assert call(a, b_ok, alloc_fn=ctypes.cast(None, binding.ALLOC_FN)) == -1   # no allocator
    short = np.array([0, 1, 2], dtype=np.int32)        # row_ptr[m] = 2 != nnz = 3
    a_short = binding.CsrDesc(2, 3, 3, short.ctypes.data, ci.ctypes.data, v.ctypes.data)
    assert call(a_short, b_ok) == -2
    assert b"row_ptr" in lib.spgemm_last_error()
    assert calls == [] and nnz.value == 0 and all(o.value is None for o in out)
