"""Autotuner: picks a plan's tuning (spgemm_tuning) by timing candidates.

The decisions a plan exposes are the lanes that share one stored a_ik in
the block kernels' row loop (G), the symbolic bound above which rows take
the column-bitmap path, the hash probing (one slot or chunks of four per
probe) and the hash (low or high bits of the product); the better choices
depend on the input's collision factor.  Defaults come from rules measured on R-MAT
and ER products; `autotune` times a grid of candidates on the caller's own
product (or a sample batch) with CUDA events and returns the fastest.  The
result of a product does not depend on the tuning, only its time.
"""
from __future__ import annotations

import statistics

import torch

from . import binding as sg

DEFAULT_GRID = [{"lanes_per_entry": g, "bitmap_min_bound": b, "probe": pr, "hash": h}
                for g in (0, 32) for b in (0, 512, 2048, -1) for pr in ("linear", "chunk4") for h in ("low", "high")]


def _split(candidate):
    """(plan keyword arguments: probe and hash schemes, spgemm_tuning dict) of a candidate."""
    t = dict(candidate)
    return {"probe": t.pop("probe", "linear"), "hash": t.pop("hash", "high")}, t


def _time(run, steps: int, stream) -> float:
    run()  # warm-up
    ts = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def autotune(A, B, sorted_output: bool = True, candidates=None, steps: int = 3, stream=None):
    """Times whole products (plan, symbolic, C allocation, numeric) of A*B
    for every candidate tuning; returns (best tuning, [(tuning, ms), ...])."""
    stream = stream if stream is not None else torch.cuda.current_stream(A.row_ptr.device)

    def run_with(t):
        kw, tuning = _split(t)

        def run():
            with sg.Plan(A, B, sorted_output, stream=stream, tuning=tuning, **kw) as p:
                p.symbolic()
                p.numeric()
        return run

    table = [(t, _time(run_with(t), steps, stream)) for t in (candidates or DEFAULT_GRID)]
    return min(table, key=lambda r: r[1])[0], table


def autotune_batch(As, Bs, sorted_output: bool = True, candidates=None, steps: int = 3, stream=None):
    """As autotune, for one packed batch of products (a sample of a larger
    stream of products of the same kind)."""
    stream = stream if stream is not None else torch.cuda.current_stream(As[0].row_ptr.device)

    def run_with(t):
        kw, tuning = _split(t)

        def run():
            with sg.Batch(As, Bs, sorted_output, stream=stream, tuning=tuning, **kw) as b:
                b.symbolic()
                b.numeric()
        return run

    table = [(t, _time(run_with(t), steps, stream)) for t in (candidates or DEFAULT_GRID)]
    return min(table, key=lambda r: r[1])[0], table
