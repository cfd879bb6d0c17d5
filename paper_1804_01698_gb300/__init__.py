"""GB300-native hash SpGEMM (row-wise Gustavson with hash-table accumulation).

    from paper_1804_01698_gb300 import binding as sg   # loads the CUDA library
    C = sg.spgemm(A, B, sorted_output=True)

``inputs`` holds the seeded synthetic workload generators, ``build`` the
in-tree nvcc build, ``binding`` the thin ctypes layer over the C ABI of
include/spgemm.h.  Nothing is imported eagerly, so the input generators
work on machines without CUDA.
"""

__all__ = ["inputs", "build", "binding"]
