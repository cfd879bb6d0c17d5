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
