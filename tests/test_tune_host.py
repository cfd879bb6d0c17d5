"""Host logic of the autotuner and of the tuning argument, on the CPU: the
candidate grid covers every combination once, and every candidate turns into
plan arguments the binding and the C validation accept."""
from __future__ import annotations

import itertools

import pytest

from paper_1804_01698_gb300 import binding as sg
from paper_1804_01698_gb300 import tune


def test_grid_is_the_full_product_of_the_choices_once():
    keys = [(c["lanes_per_entry"], c["bitmap_min_bound"], c["probe"], c["hash"]) for c in tune.DEFAULT_GRID]
    assert len(keys) == len(set(keys)) == 32
    assert set(keys) == set(itertools.product((0, 32), (0, 512, 2048, -1), ("linear", "chunk4"), ("low", "high")))


@pytest.mark.parametrize("candidate", tune.DEFAULT_GRID)
def test_every_candidate_maps_to_valid_plan_arguments(candidate):
    kw, tuning = tune._split(candidate)
    assert set(kw) == {"probe", "hash"}
    assert kw["probe"] in sg._PROBES and kw["hash"] in sg._HASHES
    t = sg._tuning(tuning)
    # the rules spgemm_plan_create_tuned checks
    assert t.lanes_per_entry in (0, 4, 8, 16, 32)
    assert t.reserved == 0 and t.bitmap_min_bound >= -1 and 0 <= t.max_nnz_c <= 2**31 - 1
    assert candidate == {**tuning, **kw}          # nothing lost in the split


def test_split_defaults_and_tuning_validation():
    kw, tuning = tune._split({"lanes_per_entry": 8})
    assert kw == {"probe": "linear", "hash": "high"} and tuning == {"lanes_per_entry": 8}
    assert sg._tuning(None) is None
    t = sg._tuning({})
    assert (t.lanes_per_entry, t.bitmap_min_bound, t.max_nnz_c) == (0, 0, 0)
    assert (t.long_row_min, t.warp_load_pct, t.block_load_pct) == (0, 0, 0)
    t = sg._tuning({"long_row_min": 64, "warp_load_pct": 60, "block_load_pct": 80})
    assert (t.long_row_min, t.warp_load_pct, t.block_load_pct) == (64, 60, 80)
    with pytest.raises(ValueError):
        sg._tuning({"lanes": 8})


# ------------------------------------------------------------ model-seeded tuning (Eq. 2)

def test_host_bin_rule_matches_the_library_rule():
    import numpy as np
    assert tune.hash_caps() == [32, 64, 128, 256, 512, 1536, 3072, 6144, 12288]
    assert tune.hash_caps(80, 90)[0] == 51 and tune.hash_caps(80, 90)[5] == 1843
    k = 1 << 16
    assert tune.bitmap_threshold(k) == 1024 and tune.bitmap_threshold(1 << 19) == 0
    assert tune.bitmap_threshold(k, -1) == 0 and tune.bitmap_threshold(k, 300) == 300
    caps = tune.bitmap_caps(k)
    assert caps[0] < caps[1] < caps[2] and all(c % 256 == 0 for c in caps)
    flop = np.array([0, 1, 32, 33, 512, 513, 1024, 1025, 24576, 30000, 90000])
    nnz = np.array([0, 1, 30, 33, 400, 500, 900, 1000, 20000, 25000, caps[2] + 5])
    sym, num, win = tune.bin_kinds(flop, nnz, k, {})
    assert list(sym) == [-1, 0, 0, 0, 0, 1, 1, 2, 2, 3, 3]            # bitmap above 1024, heavy above 24576
    cls = [2 if z <= caps[0] else 3 if z <= caps[1] else 4 for z in nnz[7:]]
    assert list(num) == [-1, 0, 0, 0, 0, 0, 1] + cls
    assert list(win) == [1] * 11                                       # one pass per row, also beyond the array
    sym, num, win = tune.bin_kinds(flop, nnz, 1 << 20, {})            # too many columns for bitmaps
    assert list(sym) == [-1, 0, 0, 0, 0, 1, 1, 1, 1, 4, 4]            # global tables above 24576
    assert list(num) == [-1, 0, 0, 0, 0, 0, 1, 1, 5, 5, 5]


def test_model_reproduces_its_calibration_and_follows_the_load():
    import numpy as np
    rng = np.random.default_rng(7)
    k = 1 << 16
    flop = rng.integers(1, 40000, 6000)
    nnz = (flop * 0.6).astype(np.int64) + 1
    sym, num, win = tune.bin_kinds(flop, nnz, k, {})
    names = {0: ("sym_warp_1024", "num_warp_1024"), 1: ("sym_block_2048", "num_block_2048")}
    kt = {}
    words = (k + 31) // 32
    # synthetic kernel times: 1 ns per product in hash kinds; bitmap classes
    # 0.3 ns per product plus 2 ns per word of every row
    for ph, (kinds, pre) in enumerate(((sym, "sym"), (num, "num"))):
        for j, nm in enumerate(tune.SYM_KINDS if ph == 0 else tune.NUM_KINDS):
            sel = kinds == j
            f = float((flop[sel] * (win[sel] if ph == 1 else 1)).sum())
            if not f:
                continue
            rows = float((win[sel] if ph == 1 else np.ones(sel.sum())).sum())
            ms = f * 0.3e-6 + rows * words * 2e-6 if nm.startswith("bitmap") else f * 1e-6
            kt[f"{pre}_{nm}"] = ms
    model = tune.calibrate(kt, flop, nnz, k, (1.25, 1.26))
    total = sum(kt.values())
    assert abs(tune.predict_ms(model, flop, nnz, k, {}) - total) < 1e-6 * total
    assert abs(model["w"][1] - 2e-6) < 1e-8                            # the word cost is recovered
    # lower table loads shorten probes: hash-heavy inputs are predicted faster
    fast = tune.predict_ms(model, flop, nnz, k, {"warp_load_pct": 30, "block_load_pct": 50})
    slow = tune.predict_ms(model, flop, nnz, k, {"warp_load_pct": 80, "block_load_pct": 95})
    assert fast < total < slow
    assert tune.linear_probe_cost(0.0) == 1.0 and tune.linear_probe_cost(0.5) == 1.5
    assert len(tune.MODEL_GRID) == 175 and all(set(c) == {"bitmap_min_bound", "warp_load_pct", "block_load_pct"}
                                                for c in tune.MODEL_GRID)
    for c in tune.MODEL_GRID:                                          # every candidate is a valid tuning
        t = sg._tuning(c)
        assert t.warp_load_pct == 0 or 5 <= t.warp_load_pct <= 95
