"""Multi-rank host logic on the CPU (gloo, world size 2): the flop-balanced
row partition (Fig. "RowsToThreads" with ranks in place of threads), the
row-sharded product whose only exchange is an all-gather of the blocks'
nnz, and the benchmark's max-over-ranks timing.  Each rank's block product
is the oracle here; on GPUs it is the library's plan on the block."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1804_01698_gb300 import inputs
from paper_1804_01698_gb300.shard import max_over_ranks, row_block, row_partition, sharded_spgemm


@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_row_partition_is_rows_to_threads(parts):
    rng = np.random.default_rng(parts)
    for flop in (rng.integers(0, 50, 200), np.zeros(7, np.int64), np.array([10**6] + [1] * 99),
                 rng.zipf(1.5, 300).clip(max=10**5)):
        offs = row_partition(flop, parts)
        assert offs.tolist() == oracle.rows_to_threads(np.asarray(flop, np.int64), parts).tolist()
        assert offs[0] == 0 and offs[-1] == len(flop) and np.all(np.diff(offs) >= 0)
        total = int(np.sum(flop))
        for r in range(parts):   # a block exceeds its share by less than one row
            blk = int(np.sum(flop[offs[r]:offs[r + 1]]))
            assert blk <= total / parts + (int(np.max(flop)) if len(flop) else 0)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A = inputs.rmat(9, 8, seed=91)
        B = inputs.er_exact(A.ncols, 5, seed=92, ncols=300)
        flop = oracle.row_flop(A, B)

        def product(A_, lo, hi, B_):
            return oracle.spgemm(row_block(A_, lo, hi), B_)[0]

        def all_gather_nnz(n):
            out = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
            dist.all_gather(out, torch.tensor([n], dtype=torch.int64))
            return [int(t.item()) for t in out]

        row0, nnz0, C = sharded_spgemm(A, B, flop, rank, world, product, all_gather_nnz)
        full, _ = oracle.spgemm(A, B)
        ok = (np.array_equal(C.row_ptr + full.row_ptr[row0], full.row_ptr[row0:row0 + C.nrows + 1])
              and nnz0 == int(full.row_ptr[row0])
              and np.array_equal(C.col_idx, full.col_idx[nnz0:nnz0 + C.nnz])
              and np.allclose(C.vals, full.vals[nnz0:nnz0 + C.nnz], rtol=0, atol=1e-12))
        slowest = max_over_ranks(1.5 + rank, world, dist)
        q.put((rank, ok, C.nrows, slowest))
    finally:
        dist.destroy_process_group()


def test_row_sharded_product_on_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [True, True]
    assert res[0][2] + res[1][2] == 512           # the blocks cover every row
    assert res[0][2] > 0 and res[1][2] > 0
    assert [r[3] for r in res] == [2.5, 2.5]      # max over ranks seen by both
