"""Multi-rank forms of the path (one process per GPU).

Rows of C are independent, so the product shards by rows: every rank takes
a contiguous block of A's rows, holds all of B, and computes its block of C
alone.  The blocks are balanced by flop exactly as Fig. "RowsToThreads"
(Sec. 4.1) balances rows over threads: a prefix sum of the row flop and a
lower-bound search for each rank's first row.  The only exchange is an
all-gather of the blocks' nnz (one int64 per rank), which places each
block's row pointers and entries in the global C.

Independent products (batches, a serving stream) shard by product with no
exchange at all, and the benchmark's timing takes the maximum over ranks
(`max_over_ranks`).
"""
from __future__ import annotations

import numpy as np


def row_partition(flop: np.ndarray, parts: int) -> np.ndarray:
    """First row of each of `parts` contiguous row blocks of about equal flop
    (Fig. "RowsToThreads" step 2); offsets[parts] = number of rows."""
    flop = np.asarray(flop, dtype=np.int64)
    m = len(flop)
    if parts < 1:
        raise ValueError("parts must be positive")
    ps = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(flop, out=ps[1:])
    total = int(ps[-1])
    offsets = np.empty(parts + 1, dtype=np.int64)
    offsets[0], offsets[parts] = 0, m
    for r in range(1, parts):
        # first row whose flop prefix reaches r/parts of the total
        offsets[r] = np.searchsorted(ps[:m], (total * r) // parts, side="left")
    return np.maximum.accumulate(offsets)


def row_block(A, lo: int, hi: int):
    """Rows lo..hi-1 of a host CSR as a CSR of their own."""
    from .inputs import CSR
    e0, e1 = int(A.row_ptr[lo]), int(A.row_ptr[hi])
    return CSR(hi - lo, A.ncols, (A.row_ptr[lo:hi + 1] - e0).astype(np.int32), A.col_idx[e0:e1], A.vals[e0:e1])


def device_row_block(dA, lo: int, hi: int):
    """Rows lo..hi-1 of a DeviceCSR as a view (row pointers rebased)."""
    from .binding import DeviceCSR
    rp = dA.row_ptr[lo:hi + 1]
    e0, e1 = int(rp[0].item()), int(rp[-1].item())
    return DeviceCSR(hi - lo, dA.ncols, rp - e0, dA.col_idx[e0:e1], dA.vals[e0:e1])


def sharded_spgemm(A, B, flop, rank: int, world: int, product, all_gather_nnz):
    """This rank's block of C = A*B.

    `flop` is the row flop of A*B (any rank can compute it; Sec. 4.1),
    `product(A_block, B)` computes a block's product, `all_gather_nnz(n)`
    returns every rank's nnz in rank order (a collective).  Returns
    (row0, nnz0, C_block): the block's first row and first entry in C."""
    offs = row_partition(flop, world)
    lo, hi = int(offs[rank]), int(offs[rank + 1])
    C = product(A, lo, hi, B)
    nnz = list(all_gather_nnz(int(C.nnz)))
    return lo, int(sum(nnz[:rank])), C


def max_over_ranks(value: float, world: int, dist=None, device=None) -> float:
    """Largest `value` over the ranks (the benchmark's step time)."""
    if world <= 1 or dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
