"""Seeded synthetic inputs for the decode path and its oracle.

Both the CPU oracle and the CUDA library consume what this module makes; it
holds none of the compression method's arithmetic (see ``synth.cpp``). The
workload recipes mirror the paper's test collections (Table V: 25M / 50M
documents; Section 7.1: "over 90% of d-gaps fit in 8 bits") with synthetic
stand-ins, because the TREC / Wikipedia / Twitter datasets are not available.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libsynth.so")
_lib = None
_lock = threading.Lock()

U32P = ctypes.POINTER(ctypes.c_uint32)
U64P = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the generator library with g++ (host code only)."""
    src = os.path.join(_HERE, "synth.cpp")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                           src, "-o", tmp])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_raw_u64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, U64P]
            lib.synth_geometric_gaps.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, U32P]
            lib.synth_mixed_runs.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_uint32, U32P]
            lib.synth_zipf_lengths.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_uint64, U32P]
            lib.synth_zipf_lengths.restype = ctypes.c_uint64
            lib.synth_lognormal_lengths.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                                    ctypes.c_double, ctypes.c_uint64, U32P]
            lib.synth_lognormal_lengths.restype = ctypes.c_uint64
            lib.synth_uniform_index.argtypes = [ctypes.c_uint64, ctypes.c_uint64, U32P, U64P,
                                                ctypes.c_uint64, U32P, ctypes.c_int]
            lib.synth_clustered_index.argtypes = [ctypes.c_uint64, ctypes.c_uint64, U32P, U64P,
                                                  ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                                  U32P, U32P, ctypes.c_int]
            lib.synth_tf_index.argtypes = [ctypes.c_uint64, ctypes.c_uint64, U32P, U64P, ctypes.c_double,
                                           U32P, ctypes.c_int]
            lib.synth_uniform_u32.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.c_uint32, U32P]
            lib.synth_width_mix.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_uint32, U32P]
            _lib = lib
    return _lib


def _p32(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    return a.ctypes.data_as(U32P)


def _p64(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags.c_contiguous
    return a.ctypes.data_as(U64P)


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


# ---------------------------------------------------------------- primitives

def raw_u64(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    _load().synth_raw_u64(seed, count, _p64(out))
    return out


def geometric_gaps(seed: int, n: int, mean: float) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    if n:
        _load().synth_geometric_gaps(seed, n, mean, _p32(out))
    return out


def mixed_runs(seed: int, n: int, run_len: int = 256, geo_mean: float = 8.0,
               frac_uniform: float = 0.1, umax: int = 1 << 20) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    if n:
        _load().synth_mixed_runs(seed, n, run_len, geo_mean, frac_uniform, umax, _p32(out))
    return out


def uniform_u32(seed: int, n: int, lo: int = 0, hi: int = 0xFFFFFFFF) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    if n:
        _load().synth_uniform_u32(seed, n, lo, hi, _p32(out))
    return out


def width_mix(seed: int, n: int, wlo: int = 0, whi: int = 32) -> np.ndarray:
    """Values whose bit widths are uniform in [wlo, whi]: exercises every width."""
    out = np.empty(n, dtype=np.uint32)
    if n:
        _load().synth_width_mix(seed, n, wlo, whi, _p32(out))
    return out


def zipf_lengths(seed: int, nlists: int, C: float, s: float = 1.1, cap: int = 1 << 22) -> np.ndarray:
    out = np.empty(nlists, dtype=np.uint32)
    _load().synth_zipf_lengths(seed, nlists, C, s, cap, _p32(out))
    return out


def lognormal_lengths(seed: int, nlists: int, median: float = 12.0, sigma: float = 1.5,
                      cap: int = 1 << 24) -> np.ndarray:
    out = np.empty(nlists, dtype=np.uint32)
    _load().synth_lognormal_lengths(seed, nlists, median, sigma, cap, _p32(out))
    return out


def offsets_of(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(len(lengths) + 1, dtype=np.uint64)
    np.cumsum(lengths, dtype=np.uint64, out=off[1:])
    return off


def padded_offsets(lengths: np.ndarray, align: int) -> np.ndarray:
    """Starts of lists laid out back to back, each at a multiple of `align`
    ints (len = nlists + 1; the last entry is the layout's length)."""
    span = (np.asarray(lengths, dtype=np.uint64) + (align - 1)) // align * align
    off = np.zeros(len(span) + 1, dtype=np.uint64)
    np.cumsum(span, out=off[1:])
    if len(span):
        off[-1] = off[-2] + np.uint64(lengths[-1])
    return off


def uniform_index(seed: int, lengths: np.ndarray, universe: int, out: np.ndarray | None = None,
                  threads: int | None = None, align: int = 1):
    """Each list: sorted uniform sample without replacement from [0, universe), as d-gaps.

    Returns (gaps, offsets) with offsets[i] the start of list i (len = nlists + 1).
    With align > 1 every list starts at a multiple of `align` ints and the ints
    between lists are 0; list i is gaps[offsets[i]:offsets[i] + lengths[i]]
    (its contents do not depend on the layout).
    ``out`` may be a preallocated uint32 array (for instance pinned host memory).
    """
    lengths = np.ascontiguousarray(lengths, dtype=np.uint32)
    off = offsets_of(lengths) if align == 1 else padded_offsets(lengths, align)
    total = int(off[-1])
    if out is None:
        out = np.empty(total, dtype=np.uint32) if align == 1 else np.zeros(total, dtype=np.uint32)
    assert out.size >= total
    if len(lengths):
        _load().synth_uniform_index(seed, len(lengths), _p32(lengths), _p64(off[:-1].copy()),
                                    universe, _p32(out), threads or _threads())
    return out[:total], off


def tf_index(seed: int, lengths: np.ndarray, mean: float = 2.0, align: int = 1, threads: int | None = None):
    """Term frequencies for lists of the given lengths: values >= 1, geometric
    with mean `mean`, one seeded stream per list. Returns (tfs, offsets) laid
    out as uniform_index lays out gaps (align > 1: each list at a multiple of
    `align` ints, zeros between lists)."""
    lengths = np.ascontiguousarray(lengths, dtype=np.uint32)
    off = offsets_of(lengths) if align == 1 else padded_offsets(lengths, align)
    total = int(off[-1])
    out = np.empty(total, dtype=np.uint32) if align == 1 else np.zeros(total, dtype=np.uint32)
    if len(lengths):
        _load().synth_tf_index(seed, len(lengths), _p32(lengths), _p64(off[:-1].copy()), float(mean), _p32(out),
                               threads or _threads())
    return out, off


def clustered_index(seed: int, max_lengths: np.ndarray, universe: int, run_mean: float = 16.0,
                    jump_mean: float = 5000.0, threads: int | None = None):
    """Clustered docIDs (runs of consecutive docs, geometric jumps), as d-gaps.

    Lists stop early when a docID would reach the universe end; returns
    (gaps, offsets, actual_lengths).
    """
    max_lengths = np.ascontiguousarray(max_lengths, dtype=np.uint32)
    n = len(max_lengths)
    lib = _load()
    actual = np.zeros(n, dtype=np.uint32)
    zero_off = np.zeros(n, dtype=np.uint64)
    if n:
        lib.synth_clustered_index(seed, n, _p32(max_lengths), _p64(zero_off), universe, run_mean,
                                  jump_mean, _p32(actual), None, threads or _threads())
    off = offsets_of(actual)
    out = np.empty(int(off[-1]), dtype=np.uint32)
    if n:
        lib.synth_clustered_index(seed, n, _p32(actual), _p64(off[:-1].copy()), universe, run_mean,
                                  jump_mean, _p32(actual), _p32(out), threads or _threads())
    return out, off, actual


# ---------------------------------------------------------------- workloads
# The five workloads of the decode path (sizes as in the project's configs).

def single_list_geometric(n: int = 65536, mean: float = 20.0, seed: int = 0) -> np.ndarray:
    """One posting list whose d-gaps are geometric (mean 20): 65,536 docIDs."""
    return geometric_gaps(seed, n, mean)


def single_list_mixed(n: int = 1 << 26, seed: int = 0) -> np.ndarray:
    """2^26 d-gaps in runs of 256: 90% geometric mean 8, 10% uniform in [1, 2^20]."""
    return mixed_runs(seed, n, 256, 8.0, 0.1, 1 << 20)


ZIPF_C = 3.0406e8  # C of the rank law L_r = C r^-1.1 for ~1.5e9 postings over 1e6 lists


def zipf_index_lengths(nlists: int = 1_000_000, seed: int = 0, C: float = ZIPF_C) -> np.ndarray:
    """Rank-law (Zipf s=1.1) list lengths clipped to [1, 2^22], shuffled."""
    return zipf_lengths(seed, nlists, C, 1.1, 1 << 22)


def zipf_index(nlists: int = 1_000_000, universe: int = 25_000_000, seed: int = 0,
               C: float = ZIPF_C, out: np.ndarray | None = None, align: int = 1):
    lengths = zipf_index_lengths(nlists, seed, C)
    gaps, off = uniform_index(seed + 1, lengths, universe, out=out, align=align)
    return gaps, off, lengths


def clustered_short_index(nlists: int = 4_000_000, universe: int = 50_000_000, seed: int = 0):
    """Log-normal lengths (median 12, sigma 1.5), clustered docIDs (runs mean 16, jumps mean 5000)."""
    maxlen = lognormal_lengths(seed, nlists, 12.0, 1.5, 1 << 24)
    return clustered_index(seed + 1, maxlen, universe, 16.0, 5000.0)


def serving_trace(lengths: np.ndarray, rate: float, duration: float, seed: int = 0,
                  mmin: int = 2, mmax: int = 8):
    """Poisson arrivals at ``rate`` req/s for ``duration`` s; each request picks
    m ~ U{mmin..mmax} lists with probability proportional to length^0.5.

    Returns (arrival_times_s, request_offsets, list_ids).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nexp = int(rate * duration * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate, size=nexp))
    t = t[t < duration]
    m = rng.integers(mmin, mmax + 1, size=len(t))
    w = np.sqrt(lengths.astype(np.float64))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    offs = np.zeros(len(t) + 1, dtype=np.int64)
    np.cumsum(m, out=offs[1:])
    ids = np.searchsorted(cdf, rng.random(int(offs[-1])), side="right").astype(np.int64)
    ids = np.minimum(ids, len(lengths) - 1)
    return t, offs, ids
