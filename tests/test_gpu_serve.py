"""The serving loop on the GPU: every request of a mix of Erdos-Renyi A*A
and AMG-style A*P products, served in continuous batches on several
streams, matches the oracle, and is the same as the product computed alone
(structure identical, values within the tolerance of the comparison rule)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1804_01698_gb300 import inputs
from gpu_helpers import assert_matches_oracle, sort_rows_on_device

pytestmark = pytest.mark.gpu


def make_requests(count, seed, rate, sg):
    from paper_1804_01698_gb300.serve import Request
    mix = inputs.serving_mix(count, seed, g_lo=4, g_hi=20, n_lo=64, n_hi=4096)
    arrivals = inputs.poisson_arrivals(count, rate, seed) if rate else np.zeros(count)
    reqs = []
    for i, (A, B) in enumerate(mix):
        dA = sg.to_device(A, "cuda", torch.float64)
        dB = dA if B is A else sg.to_device(B, "cuda", torch.float64)
        flop = int(np.diff(B.row_ptr)[A.col_idx].sum())
        reqs.append(Request(i, dA, dB, float(arrivals[i]), flop))
    return mix, reqs


@pytest.mark.parametrize("sorted_output", [True, False])
def test_served_mix_matches_the_oracle_and_the_product_alone(sorted_output):
    from paper_1804_01698_gb300 import binding as sg
    from paper_1804_01698_gb300.serve import GpuBackend, Server
    mix, reqs = make_requests(40, seed=11, rate=0.0, sg=sg)
    backend = GpuBackend(sorted_output=sorted_output, nstreams=3)
    stats = Server(backend, mem_cap=1 << 30, max_batch=8, max_inflight=3).run(reqs, keep_results=True)
    torch.cuda.synchronize()
    assert sorted(c.rid for c in stats.completions) == list(range(40))
    assert stats.batches >= 5
    by_rid = {c.rid: c.result for c in stats.completions}
    for i, (A, B) in enumerate(mix):
        C = by_rid[i]
        assert_matches_oracle(C, A, B, sorted_output)
        alone = sg.spgemm(reqs[i].A, reqs[i].B, sorted_output)
        torch.cuda.synchronize()
        assert torch.equal(alone.row_ptr, C.row_ptr)
        if sorted_output:
            ca, va, cb, vb = alone.col_idx, alone.vals, C.col_idx, C.vals
        else:
            ca, va = sort_rows_on_device(alone)
            cb, vb = sort_rows_on_device(C)
        assert torch.equal(ca, cb)
        _, absb = oracle.spgemm(A, B, nthreads=4)
        err = (va - vb).abs().cpu().numpy()
        assert np.all(err <= 2e-12 * absb)


def test_admission_under_a_tight_cap_and_arrivals_over_time():
    from paper_1804_01698_gb300 import binding as sg
    from paper_1804_01698_gb300.serve import GpuBackend, Server, serve_one_by_one
    mix, reqs = make_requests(24, seed=12, rate=2000.0, sg=sg)
    backend = GpuBackend(sorted_output=True, nstreams=2)
    cap = 4 << 20
    stats = Server(backend, mem_cap=cap, max_batch=16, max_inflight=2).run(reqs, keep_results=True)
    torch.cuda.synchronize()
    assert len(stats.completions) == 24
    big = 0
    for r in reqs:      # a single request above the cap is admitted alone
        h = backend.prepare([r])
        big = max(big, backend.bytes(h))
        backend.release(h)
    assert stats.peak_mem <= max(cap, big)
    for c in stats.completions:
        A, B = mix[c.rid]
        assert_matches_oracle(c.result, A, B, True)
    base = serve_one_by_one(GpuBackend(sorted_output=True, nstreams=1), reqs)
    assert base.batches == 24 and len(base.completions) == 24
