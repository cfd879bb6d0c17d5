"""Writes tests/golden/workloads.json from the CPU oracle only.

For each named workload (seeded synthetic inputs) it records the sizes, the
total and maximum row flop (Sec. 4.1), nnz(C) and a SHA-256 digest of C's
row_ptr and col_idx (column-sorted rows).  GPU tests compare against these
numbers bit for bit.  Run:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1804_01698_gb300 import inputs  # noqa: E402


def digest(c) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(c.row_ptr, dtype=np.int32).tobytes())
    h.update(np.ascontiguousarray(c.col_idx, dtype=np.int32).tobytes())
    return h.hexdigest()


def main():
    out = {}
    for name in inputs.WORKLOADS:
        t0 = time.time()
        a, b, _ = inputs.workload(name)
        flop = oracle.row_flop(a, b)
        c, _ = oracle.spgemm(a, b, nthreads=os.cpu_count() or 1)
        out[name] = dict(m=a.nrows, n=a.ncols, k=b.ncols, nnz_a=a.nnz, nnz_b=b.nnz,
                         total_flop=int(flop.sum()), max_row_flop=int(flop.max()),
                         zero_flop_rows=int((flop == 0).sum()),
                         nnz_c=c.nnz, max_row_nnz_c=int(np.diff(c.row_ptr).max()),
                         c_structure_sha256=digest(c))
        print(name, out[name], f"{time.time() - t0:.1f}s", flush=True)
    with open(os.path.join(HERE, "workloads.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
