"""Autotuner host logic (no GPU): workload classes, the JSON cache, the k choice rule and the candidate shapes."""
import json

import numpy as np

from paper_1502_01916_gb300 import make_codec, SIMPLE
from paper_1502_01916_gb300.tune import (CANDIDATES, cache_key, candidates_for, load_cache, pick_k, save_cache,
                                         workload_class)


def test_workload_classes():
    assert workload_class(np.full(1000, 12)) == "short-single"
    assert workload_class(np.full(1000, 300)) == "mid-single"
    assert workload_class(np.full(10, 100_000)) == "long-multi"
    assert workload_class(np.array([], np.uint32)) == "empty"


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert load_cache(path) == {}
    key = cache_key("GB300", make_codec(SIMPLE, 32), np.full(10, 5000), True)
    assert key.endswith("|long-multi|ids") and key.startswith("GB300|GS/k32")
    save_cache(path, {key: {"shape": [11, 2, 32, 0], "ms": 1.5}})
    assert load_cache(path)[key]["shape"] == [11, 2, 32, 0]
    with open(path, "w") as f:
        f.write("not json")
    assert load_cache(path) == {}


def test_pick_k_prefers_speed_then_size():
    fast4 = {4: {"ms": 1.0, "bits_per_int": 14.0}, 32: {"ms": 2.0, "bits_per_int": 12.0}}
    assert pick_k(fast4) == 4
    fast32 = {4: {"ms": 2.0, "bits_per_int": 11.0}, 32: {"ms": 1.7, "bits_per_int": 12.0}}
    assert pick_k(fast32) == 32
    tie = {4: {"ms": 1.000, "bits_per_int": 11.0}, 32: {"ms": 1.005, "bits_per_int": 12.0}}
    assert pick_k(tie) == 4  # within 1%: the smaller index
    tie32 = {4: {"ms": 1.005, "bits_per_int": 13.0}, 32: {"ms": 1.000, "bits_per_int": 12.0}}
    assert pick_k(tie32) == 32


def test_candidate_shapes_are_in_range():
    """Every candidate is a valid launch shape for its k (gc.h: 1..23 decoding
    warps at k = 32, 1..15 at k = 4; 1..8 blocks per SM; 1..32 records per
    claim; a ring of 0 (all that fits) or at least 12 KB), and the library
    default is among them."""
    for k, limit in ((32, 23), (4, 15)):
        shapes = candidates_for(k)
        assert shapes is CANDIDATES[k] and len(set(shapes)) == len(shapes)
        for w, b, c, st in shapes:
            assert 1 <= w <= limit and 1 <= b <= 8 and 1 <= c <= 32 and (st == 0 or st >= 12288)
    assert (7, 3, 32, 0) in candidates_for(32) and (7, 2, 32, 0) in candidates_for(4)
