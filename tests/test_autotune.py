"""The batched autotuner's host side (no GPU): the entry lookup the library applies, the cache's
JSON round trip, the ctypes table, and the committed cache's coverage."""
import ctypes
import json
import os

import pytest

from paper_2112_09017_gb300 import autotune

E = [{"n_lo": 129, "n_hi": 256, "aspect_lo": 0.0, "aspect_hi": 1.5, "tile_n": 128, "slice_stages": 4},
     {"n_lo": 129, "n_hi": 256, "aspect_lo": 1.5, "aspect_hi": 1e9, "tile_n": 256, "slice_stages": 2},
     {"n_lo": 200, "n_hi": 1024, "aspect_lo": 0.0, "aspect_hi": 1e9, "tile_n": 256, "slice_stages": 4}]


def test_first_matching_entry_wins_with_inclusive_bounds():
    assert autotune.choice_for(E, 129, 129) is E[0]
    assert autotune.choice_for(E, 256, 256) is E[0]           # n_hi inclusive
    assert autotune.choice_for(E, 384, 256) is E[0]           # m/n = 1.5 belongs to the first entry
    assert autotune.choice_for(E, 512, 256) is E[1]
    assert autotune.choice_for(E, 300, 300) is E[2]
    assert autotune.choice_for(E, 128, 128) is None           # below every range: the plan's options
    assert autotune.choice_for(None, 300, 300) is None


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "TUNING_DIR", str(tmp_path))
    res = {"gpu": "Some GPU 9000", "planes": 3, "prec": "bf16x6", "entries": E, "measured": []}
    path = autotune.save(res)
    assert os.path.basename(path) == "some_gpu_9000_p3.json"
    assert autotune.load("Some GPU 9000") == E
    assert autotune.load("Other GPU") is None


def test_ctypes_table_matches_entries():
    from paper_2112_09017_gb300 import polar
    arr = polar.tune_table(E)
    assert len(arr) == 3
    assert (arr[1].n_lo, arr[1].n_hi, arr[1].tile_n, arr[1].slice_stages) == (129, 256, 256, 2)
    assert arr[1].aspect_lo == 1.5
    assert ctypes.sizeof(polar.polar_tune_entry_t) == 40


def test_committed_cache_covers_the_tiled_sizes():
    """Every committed table assigns a legal choice to every size the grouped launches see (n from
    129 to 1024, m = n or 2n) and records the candidates it measured."""
    files = [f for f in os.listdir(autotune.TUNING_DIR) if f.endswith(".json")] if os.path.isdir(
        autotune.TUNING_DIR) else []
    if not files:
        pytest.skip("no committed tuning cache")
    for f in files:
        d = json.load(open(os.path.join(autotune.TUNING_DIR, f)))
        for n in range(129, 1025, 7):
            for m in (n, 2 * n):
                e = autotune.choice_for(d["entries"], m, n)
                assert e is not None, (f, m, n)
                assert e["tile_n"] in (128, 256) and 1 <= e["slice_stages"] <= 8
        for b in d["measured"]:
            assert any(c["ok"] for c in b["candidates"])
