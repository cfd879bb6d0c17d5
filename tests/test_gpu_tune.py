"""Tuned plans (spgemm_tuning) and the autotuner on the GPU: every tuning
gives the oracle's product (the tuning moves rows between kernels, never
changes the result), out-of-range tunings are rejected, and the autotuner
returns one of its candidates."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_1804_01698_gb300 import inputs
from gpu_helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tuning", [
    {"lanes_per_entry": 4}, {"lanes_per_entry": 32}, {"bitmap_min_bound": 256}, {"bitmap_min_bound": 2048},
    {"bitmap_min_bound": -1}, {"lanes_per_entry": 8, "bitmap_min_bound": 100000}, {"long_row_min": 1},
    {"long_row_min": -1}, {"long_row_min": 32, "bitmap_min_bound": 256}, {"warp_load_pct": 75, "block_load_pct": 90},
    {"warp_load_pct": 25, "block_load_pct": 50}])
@pytest.mark.parametrize("sorted_output", [True, False])
def test_every_tuning_gives_the_same_product(tuning, sorted_output):
    from paper_1804_01698_gb300 import binding as sg
    A = inputs.rmat(12, 16, seed=111)
    dA = sg.to_device(A)
    with sg.Plan(dA, dA, sorted_output, tuning=tuning) as p:
        p.symbolic()
        C = p.numeric()
        st = p.stats()
    torch.cuda.synchronize()
    assert st["status"] == 0
    if tuning.get("bitmap_min_bound") == -1:
        assert st["sym_bin_rows"][10] == 0 and st["sym_bin_rows"][11] == 0
    if tuning.get("bitmap_min_bound") == 256:
        assert st["sym_bin_rows"][11] > 0
    assert_matches_oracle(C, A, A, sorted_output)


@pytest.mark.parametrize("bad", [{"lanes_per_entry": 5}, {"lanes_per_entry": 64}, {"bitmap_min_bound": -2},
                                 {"long_row_min": -2}, {"warp_load_pct": 4}, {"block_load_pct": 96},
                                 {"warp_load_pct": -1}])
def test_out_of_range_tuning_is_rejected(bad):
    from paper_1804_01698_gb300 import binding as sg
    dA = sg.to_device(inputs.er_exact(100, 4, seed=112))
    with pytest.raises(sg.SpgemmError) as ei:
        sg.Plan(dA, dA, True, tuning=bad)
    assert ei.value.status == -1
    with pytest.raises(ValueError):
        sg.Plan(dA, dA, True, tuning={"no_such_knob": 1})


def test_autotune_returns_a_candidate():
    from paper_1804_01698_gb300 import binding as sg
    from paper_1804_01698_gb300.tune import autotune, autotune_batch
    dA = sg.to_device(inputs.rmat(11, 16, seed=113))
    cands = [{"lanes_per_entry": 0, "bitmap_min_bound": 0}, {"lanes_per_entry": 16, "bitmap_min_bound": 2048},
             {"lanes_per_entry": 32, "bitmap_min_bound": -1, "probe": "chunk4", "hash": "low"}]
    best, table = autotune(dA, dA, True, candidates=cands, steps=2)
    assert best in cands and len(table) == 3 and all(ms > 0 for _, ms in table)
    mats = [sg.to_device(m) for m in inputs.er_batch(6, seed=114, n_hi=3000)]
    best, table = autotune_batch(mats, mats, True, candidates=cands[:2], steps=2)
    assert best in cands[:2] and len(table) == 2


def test_model_seeded_autotune_times_its_best_predictions():
    from paper_1804_01698_gb300 import binding as sg
    from paper_1804_01698_gb300.tune import model_autotune
    dA = sg.to_device(inputs.rmat(12, 16, seed=115))
    best, table, meas = model_autotune(dA, dA, True, top=2, steps=2)
    assert meas["c_sym"] >= 1.0 and meas["c_num"] >= 1.0 and 0 < meas["rho"] <= 1.0
    assert 2 <= len(table) <= 6 and best in [c for c, _, _ in table]
    assert all(pred > 0 and ms > 0 for _, pred, ms in table)
    kw, tuning = (lambda t: ({"probe": t.pop("probe", "linear"), "hash": t.pop("hash", "high")}, t))(dict(best))
    with sg.Plan(dA, dA, True, tuning=tuning, **kw) as p:     # the pick still gives the oracle's product
        p.symbolic()
        C = p.numeric()
    torch.cuda.synchronize()
    assert_matches_oracle(C, inputs.rmat(12, 16, seed=115), inputs.rmat(12, 16, seed=115), True)
