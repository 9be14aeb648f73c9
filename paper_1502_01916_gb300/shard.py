"""Sharding the decode across GPUs (one process per GPU).

Posting lists are independent, so an index shards by list: each rank takes a
contiguous range of lists, balanced by compressed bytes (what its decode
reads), and decodes it with no exchange at all. A single list too long for
one GPU shards by tile: each rank decodes a contiguous range of the list's
1024-int tiles, and the ranks exchange one number each, the sum of their
range's gaps modulo 2^32; the exclusive scan of those sums over the ranks is
the docID before each rank's range (the prefix sum of Sec 2.1.1 across
shards). That is the path's only exchange step.

Nothing here touches the data: the decoding is the library's (or, in the
CPU tests, the oracle's).
"""
from __future__ import annotations

import numpy as np


def partition_lists(list_bytes, nranks: int) -> np.ndarray:
    """Boundaries b[0] = 0 <= ... <= b[nranks] = nlists: rank r takes lists
    [b[r], b[r+1]), the cuts placed where the running total of bytes crosses
    r / nranks of the whole."""
    w = np.asarray(list_bytes, dtype=np.float64)
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    cum = np.concatenate(([0.0], np.cumsum(w)))
    total = cum[-1]
    cuts = [int(np.searchsorted(cum, total * r / nranks, side="left")) for r in range(1, nranks)]
    b = np.array([0] + cuts + [len(w)], dtype=np.int64)
    return np.maximum.accumulate(b)


def split_tiles(ntiles: int, nranks: int) -> np.ndarray:
    """Tile boundaries of one list shared by nranks ranks, as even as whole
    tiles allow."""
    return np.array([(ntiles * r) // nranks for r in range(nranks + 1)], dtype=np.int64)


def carry_in(gap_sum: int, group=None) -> int:
    """The docID before this rank's range: the sum, modulo 2^32, of the gap
    sums of the ranks before it (one all-gather of one value per rank)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    mine = torch.tensor([int(gap_sum) & 0xFFFFFFFF], dtype=torch.int64, device=dev)
    allv = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(allv, mine, group=group)
    return int(sum(int(v.item()) for v in allv[:rank])) & 0xFFFFFFFF
