"""The batched and served workloads at their full sizes, in the launch
configuration bench.py times, checked on sampled products against the
oracle: the 2000 Erdos-Renyi products A_i*A_i packed into waves of
< 2^31 flop, and a serving stream with the full size ranges (n up to 65536,
AMG grids up to 48^3)."""
from __future__ import annotations

import os

import numpy as np
import pytest
import torch

import oracle
from paper_1804_01698_gb300 import inputs
from gpu_helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu


def _waves(flops, limit=2**31 - 1):
    waves, cur, tot = [], [], 0
    for i, f in enumerate(flops):
        if cur and tot + f > limit:
            waves.append(cur)
            cur, tot = [], 0
        cur.append(i)
        tot += f
    return waves + ([cur] if cur else [])


def test_batch_er2000_sampled_products():
    from paper_1804_01698_gb300 import binding as sg
    mats = inputs.er_batch(2000, seed=inputs.SEED_BASE + 3)
    flops = [m.nrows * (m.nnz // m.nrows) ** 2 for m in mats]
    waves = _waves(flops)
    assert len(waves) >= 4
    rng = np.random.default_rng(171)
    biggest = int(np.argmax(flops))
    checked = 0
    for w in waves:
        dm = [sg.to_device(mats[i]) for i in w]
        with sg.Batch(dm, dm, True) as b:
            b.symbolic()
            b.numeric()
            st = b.plan_stats()
            torch.cuda.synchronize()
            assert st["status"] == 0 and st["total_flop"] == sum(flops[i] for i in w)
            rp = b.c_row_ptr.cpu().numpy()
            picks = set(rng.choice(len(w), size=min(6, len(w)), replace=False).tolist())
            if biggest in w:
                picks.add(w.index(biggest))
            for q in sorted(picks):
                M = mats[w[q]]
                assert_matches_oracle(b.product(q, rp), M, M, True, nthreads=os.cpu_count() or 8)
                checked += 1
        del dm
        torch.cuda.empty_cache()
    assert checked >= 20


def test_serving_stream_full_size_ranges_sampled():
    from paper_1804_01698_gb300 import binding as sg
    from paper_1804_01698_gb300.serve import GpuBackend, Request, Server
    mix = inputs.serving_mix(200, seed=inputs.SEED_BASE + 5)
    reqs = []
    for i, (A, B) in enumerate(mix):
        dA = sg.to_device(A)
        dB = dA if B is A else sg.to_device(B)
        reqs.append(Request(i, dA, dB, 0.0, int(np.diff(B.row_ptr)[A.col_idx].sum())))
    st = Server(GpuBackend(sorted_output=True), mem_cap=40 << 30, max_batch=64, max_inflight=3).run(
        reqs, keep_results=True)
    torch.cuda.synchronize()
    assert sorted(c.rid for c in st.completions) == list(range(200))
    by_rid = {c.rid: c.result for c in st.completions}
    rng = np.random.default_rng(172)
    amg = [i for i, (A, B) in enumerate(mix) if A is not B]
    big_amg = max(amg, key=lambda i: mix[i][0].nrows)
    for i in sorted(set(rng.choice(200, 20, replace=False).tolist()) | {big_amg}):
        A, B = mix[i]
        assert_matches_oracle(by_rid[i], A, B, True, nthreads=os.cpu_count() or 8)


def test_serving_stream_poisson_arrivals_sampled():
    """The same stream arriving as a Poisson process near the server's
    capacity: batches of varying sizes overlap on several streams while
    new ones are prepared and finished ones retired."""
    from paper_1804_01698_gb300 import binding as sg
    from paper_1804_01698_gb300.serve import GpuBackend, Request, Server
    mix = inputs.serving_mix(200, seed=inputs.SEED_BASE + 9)
    arrivals = inputs.poisson_arrivals(200, 3000.0, inputs.SEED_BASE + 9)
    reqs = []
    for i, (A, B) in enumerate(mix):
        dA = sg.to_device(A)
        dB = dA if B is A else sg.to_device(B)
        reqs.append(Request(i, dA, dB, float(arrivals[i]), int(np.diff(B.row_ptr)[A.col_idx].sum())))
    st = Server(GpuBackend(sorted_output=False), mem_cap=40 << 30, max_batch=16, max_inflight=3).run(
        reqs, keep_results=True)
    torch.cuda.synchronize()
    assert sorted(c.rid for c in st.completions) == list(range(200))
    assert st.batches > 10
    by_rid = {c.rid: c.result for c in st.completions}
    rng = np.random.default_rng(173)
    for i in sorted(rng.choice(200, 25, replace=False).tolist()):
        A, B = mix[i]
        assert_matches_oracle(by_rid[i], A, B, False, nthreads=os.cpu_count() or 8)
