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


def test_tune_batch_times_every_candidate_and_returns_the_fastest(monkeypatch):
    # the plan is replaced by a stand-in: no GPU; each candidate's time comes from a table
    import paper_2401_11882_gb300.batched as batched
    built = []

    class FakeDescent:
        def __init__(self, batch, tile=None, **kw):
            built.append(tile)
            self.tile = tile

        def run(self, n):
            pass

        def close(self):
            pass

    monkeypatch.setattr(batched, "BatchedDescent", FakeDescent)
    cands = [TileConfig(4, 0, 0), TileConfig(8, 0, 1), TileConfig(8, 0, 2)]
    ms = {cands[0]: 5.0, cands[1]: 2.0, cands[2]: 3.0}

    def timer(fn, reps):
        fn()
        return ms[built[-1]]

    best, timings = autotune.tune_batch(object(), candidates=cands, timer=timer,
                                        return_timings=True)
    assert best == cands[1] and built == cands
    assert [t for _, t in timings] == [5.0, 2.0, 3.0]
    assert autotune.tune_batch(object(), candidates=cands, timer=timer) == cands[1]
