"""Host logic of the autotuner (no GPU): candidate grid, size classes, cache
persistence and the choice of the fastest candidate."""
import json

import pytest

from paper_2402_15253_gb300 import autotune as at


def test_candidate_grids_are_valid():
    b = at.candidates(True)
    s = at.candidates(False)
    assert len(b) == 14 and len(s) == 9
    assert all(at.valid(c) for c in b + s)
    assert at.DEFAULT in b
    assert not at.valid((16, 256, 512, 21)) and not at.valid((32, 32, 512, 21))
    assert not at.valid((32, 256, 384, 21)) and not at.valid((32, 256, 512, 70))
    assert not at.valid((32, 256, 512))


def test_size_classes_and_keys():
    assert [at.size_class(x) for x in (0, 1, 2, 3, 4, 1023, 1024)] == [0, 0, 1, 1, 2, 9, 10]
    k1 = at.cache_key("GB300", "peelone", "batched", 1000, 5000, 64)
    k2 = at.cache_key("GB300", "peelone", "batched", 1023, 8000, 127)
    k3 = at.cache_key("GB300", "histocore", "batched", 1000, 5000, 64)
    assert k1 == k2 and k1 != k3


def test_tune_picks_the_fastest_and_warms_up():
    calls = []
    fake = {(32, 128, 256, 21): 5.0, (64, 256, 512, 21): 2.0, (128, 1024, 512, 62): 2.0}

    def run(c):
        calls.append(c)
        return fake[c]

    best, timings = at.tune(run, list(fake), reps=3)
    assert best == (64, 256, 512, 21)                  # first of the tied minima
    assert timings == fake
    assert len(calls) == 3 * 4                          # one warm-up + 3 runs each
    with pytest.raises(ValueError):
        at.tune(run, [(8, 256, 512, 21)])


def test_staged_search_follows_the_best():
    # time = distance from (64, 128, 256, 23); the staged search must reach it
    def run(c):
        return abs(c[0] - 64) + abs(c[1] - 128) + abs(c[2] - 256) + abs(c[3] - 23)
    best, timings = at.tune_staged(run, at.stages(True), reps=1)
    assert best == (64, 128, 256, 23)
    assert len(timings) == 14                    # the stage-1 winner is not timed twice
    best1, _ = at.tune_staged(run, at.stages(False), reps=1)
    assert best1 == (64, 128, 512, 21)                   # single graphs keep CTA size and clusters


def test_cache_round_trip(tmp_path, monkeypatch):
    path = str(tmp_path / "sub" / "tuning.json")
    monkeypatch.setenv("PICO_TUNING_CACHE", path)
    assert at.load_cache() == {}
    at.save_cache({"a": [32, 256, 512, 21]})
    at.save_cache({"b": [64, 128, 256, 62]})
    d = json.load(open(path))
    assert d == {"a": [32, 256, 512, 21], "b": [64, 128, 256, 62]}
    (tmp_path / "bad.json").write_text("{not json")
    assert at.load_cache(str(tmp_path / "bad.json")) == {}
