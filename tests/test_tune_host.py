"""Autotuner host logic (no GPU): workload classes and the JSON cache."""
import json

import numpy as np

from paper_1502_01916_gb300 import make_codec, SIMPLE
from paper_1502_01916_gb300.tune import cache_key, load_cache, save_cache, workload_class


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
