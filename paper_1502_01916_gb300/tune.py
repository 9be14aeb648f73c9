"""Autotuner of the persistent decoder's launch shape.

The decoder's speed on a given index depends on how many decoding warps
share a block's staging warp and ring, how many blocks share an SM, how many
plan records a block claims per atomic, and how deep the staging ring is
(how many bytes of compressed data each block keeps in flight). This module
times gc_decode_plan on the caller's resident index for a small grid of
those shapes, keeps the fastest, and caches it in a JSON file keyed by the
device, the codec and the workload class (how long the index's lists are),
so that a server or benchmark tunes once per kind of index. The chosen
shape is registered with the library (gc_set_launch), so that later decode
calls given no launch shape use it.

The vector width k is a property of the encoded index, not of the launch:
choose_k encodes the same lists at k = 4 and k = 32, tunes each, and
reports both rates beside their sizes, for an index builder to pick from.
"""
from __future__ import annotations

import json
import os
import threading

import numpy as np

from . import gc as _gc

# (decoding warps per block, blocks per SM, records per claim, ring bytes; 0 = all that fits)
CANDIDATES = {
    32: [(7, 3, 32, 0), (6, 3, 32, 0), (8, 3, 32, 0), (5, 4, 32, 0), (4, 4, 32, 0), (9, 2, 32, 0), (11, 2, 32, 0),
         (7, 3, 16, 0), (7, 3, 32, 16384)],
    4: [(7, 2, 32, 0), (7, 2, 32, 24576), (7, 2, 16, 0), (3, 4, 32, 0), (15, 1, 32, 0)],
}


def candidates_for(k: int):
    return CANDIDATES[32 if k == 32 else 4]


_lock = threading.Lock()


def workload_class(lengths) -> str:
    """Short (most lists fit one tile), mixed, or long lists: the median
    list length and the share of ints in lists of more than one tile."""
    L = np.asarray(lengths, dtype=np.int64)
    if len(L) == 0:
        return "empty"
    med = float(np.median(L))
    multi = float(L[L > _gc.TILE_INTS].sum()) / max(1, int(L.sum()))
    size = "short" if med < 64 else "mid" if med < 1024 else "long"
    share = "multi" if multi > 0.5 else "single"
    return f"{size}-{share}"


def cache_key(device_name: str, codec, lengths, restore: bool) -> str:
    return f"{device_name}|{_gc.codec_name(codec)}|{workload_class(lengths)}|{'ids' if restore else 'gaps'}"


def default_cache_path() -> str:
    base = os.environ.get("GC_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "gc_tune.json")
    return base


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(index, plan=None, restore_docids: bool = True, candidates=None, reps: int = 3, cache_path: str | None = None,
         use_cache: bool = True, register: bool = True):
    """The fastest launch shape for decoding `index` (a gc.Index) and its
    timings; registered with the library for the index's codec unless
    register is False. Returns (gc_launch, {"key", "best_ms", "ms": {shape:
    ms}, "cached"})."""
    import torch
    dev = index.data.device
    name = torch.cuda.get_device_name(dev)
    key = cache_key(name, index.codec, index.lengths, restore_docids)
    path = cache_path or default_cache_path()
    if use_cache:
        with _lock:
            hit = load_cache(path).get(key)
        if hit and len(hit.get("shape", ())) == 4:
            launch = _gc.gc_launch(*hit["shape"])
            if register:
                _gc.gc_set_launch(index.codec, restore_docids, launch)
            return launch, {"key": key, "best_ms": hit["ms"], "ms": {}, "cached": True}
    plan = plan if plan is not None else _gc.plan_index(index)
    out = torch.empty(max(1, index.out_ints), dtype=torch.int32, device=dev)
    scratch = torch.empty(_gc.gc_decode_plan_scratch_size(index.max_tiles), dtype=torch.uint8, device=dev)
    st = _gc.new_status(dev)
    times = {}
    for shape in candidates or candidates_for(index.codec.k):
        launch = _gc.gc_launch(*shape)
        _gc.decode_index(index, out=out, restore_docids=restore_docids, launch=launch, scratch=scratch, status=st,
                         plan=plan, check=False)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for s, e in ev:
            s.record()
            _gc.decode_index(index, out=out, restore_docids=restore_docids, launch=launch, scratch=scratch,
                             status=st, plan=plan, check=False)
            e.record()
        torch.cuda.synchronize(dev)
        times[shape] = float(np.median([s.elapsed_time(e) for s, e in ev]))
    _gc.check_status(st, "tuning decode")
    best = min(times, key=times.get)
    if register:
        _gc.gc_set_launch(index.codec, restore_docids, _gc.gc_launch(*best))
    if use_cache:
        with _lock:
            cache = load_cache(path)
            cache[key] = {"shape": list(best), "ms": times[best]}
            save_cache(path, cache)
    return _gc.gc_launch(*best), {"key": key, "best_ms": times[best],
                                  "ms": {"x".join(map(str, sh)): t for sh, t in times.items()}, "cached": False}


def choose_k(kind: int, d_gaps, lengths, out_offsets=None, restore_docids: bool = True, reps: int = 3,
             register: bool = True, **codec_kw):
    """Encode the lists at k = 4 and at k = 32 (same codec kind and
    parameters), tune the launch shape of each, and time each index's decode
    with its best shape. Returns (k, {k: {"ms", "bits_per_int", "shape"}}),
    k the faster one (the smaller index on a tie within 1%)."""
    by_k = {}
    for k in (4, 32):
        idx = _gc.encode_index(_gc.make_codec(kind, k, **codec_kw), d_gaps, lengths, out_offsets=out_offsets)
        plan = _gc.plan_index(idx)
        launch, info = tune(idx, plan, restore_docids, reps=reps, use_cache=False, register=register)
        by_k[k] = {"ms": info["best_ms"], "bits_per_int": 8.0 * idx.compressed_bytes() / max(1, idx.total_ints),
                   "shape": [launch.warps_per_block, launch.blocks_per_sm, launch.items_per_claim,
                             launch.stage_bytes]}
        del idx, plan
    return pick_k(by_k), by_k


def pick_k(by_k: dict) -> int:
    """The k of the faster decode ({k: {"ms", "bits_per_int"}} for k = 4
    and 32); within 1% of each other, the smaller index."""
    a, b = by_k[4], by_k[32]
    if abs(a["ms"] - b["ms"]) <= 0.01 * min(a["ms"], b["ms"]):
        return 4 if a["bits_per_int"] <= b["bits_per_int"] else 32
    return 4 if a["ms"] < b["ms"] else 32
