"""Autotuner host logic (no GPU): cache keys, cache round trip, choice rule."""
import json

import pytest

from paper_2401_11882_gb300 import autotune
from paper_2401_11882_gb300.ops import TileConfig


def test_keys_bucket_by_powers_of_two():
    a = autotune.forward_key("GB300", "hard_sigmoid", 2, 64, 65536)
    b = autotune.forward_key("GB300", "hard_sigmoid", 2, 60, 40000)
    c = autotune.forward_key("GB300", "hard_sigmoid", 2, 65, 65536)
    assert a == b and a != c
    assert autotune._bucket(1) == 1 and autotune._bucket(3) == 4 and autotune._bucket(64) == 64


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "t.json"
    monkeypatch.setenv("DRT_TUNE_CACHE", str(path))
    assert autotune.load_cache() == {}
    autotune.save_cache({"k": {"tile": {"warps_per_cta": 4, "cands_per_unit": 32,
                                        "ctas_per_sm": 0, "cull_invalid": False}}})
    assert json.load(open(path))["k"]["tile"]["warps_per_cta"] == 4
    path.write_text("not json")
    assert autotune.load_cache() == {}


def test_pick_best_prefers_fastest_then_earliest():
    a, b, c = TileConfig(4, 16), TileConfig(8, 32), TileConfig(8, 64)
    assert autotune.pick_best([(a, 3.0), (b, 1.0), (c, 2.0)]) == b
    assert autotune.pick_best([(a, 1.0), (b, 1.0)]) == a


def test_candidate_sets_are_valid():
    for t in autotune.FORWARD_CANDIDATES + autotune.BATCH_CANDIDATES:
        assert 1 <= t.warps_per_cta <= 8 and t.ctas_per_sm >= 0 and t.cands_per_unit >= 0
