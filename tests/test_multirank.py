"""The multi-GPU path on CPU ranks (gloo, world size 2 and 3): an index sharded
by list decodes with no exchange, and one list sharded by tile range restores
the same docIDs after one exchange of per-rank gap sums. Each rank decodes its
shard with the CPU oracle; the concatenation of the shards must equal the
whole decode."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1502_01916_gb300.shard import partition_lists, split_tiles


def test_partition_lists_covers_and_balances():
    rng = np.random.default_rng(0)
    w = rng.pareto(1.1, size=5000) * 1000
    for n in (1, 2, 3, 8):
        b = partition_lists(w, n)
        assert b[0] == 0 and b[-1] == len(w) and (np.diff(b) >= 0).all()
        share = np.array([w[b[r]:b[r + 1]].sum() for r in range(n)])
        assert abs(share.sum() - w.sum()) < 1e-6 * w.sum()
        # no rank exceeds its fair share by more than the largest list
        assert share.max() <= w.sum() / n + w.max() + 1e-9


def test_split_tiles_even():
    b = split_tiles(10, 3)
    assert list(b) == [0, 3, 6, 10]
    assert list(split_tiles(2, 4)) == [0, 0, 1, 1, 2]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle as O
    import synth
    from paper_1502_01916_gb300.shard import carry_in, partition_lists, split_tiles

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    codec = O.Codec(O.PFD, 32)
    # (1) an index sharded by list: decode the own range of lists, no exchange
    lens = synth.zipf_index_lengths(400, 3, 3e4)
    gaps, off = synth.uniform_index(9, lens, 1_000_000)
    encs = [O.encode(codec, gaps[off[i]:off[i + 1]]) for i in range(len(lens))]
    b = partition_lists([len(c) + 4 * len(d) for c, d in encs], world)
    mine = [O.prefix_sum(O.decode(codec, *encs[i], int(lens[i]))) for i in range(b[rank], b[rank + 1])]
    part = np.concatenate(mine) if mine else np.zeros(0, np.uint32)
    np.save(os.path.join(out_dir, f"lists_{rank}.npy"), part)
    # (2) one list sharded by tile range: decode the own tiles' gaps, exchange
    # the gap sums, restore docIDs from the carry-in
    g = synth.mixed_runs(11, 100_003, 256, 8.0, 0.1, 1 << 20)
    ctrl, data = O.encode(codec, g)
    gaps_all = O.decode(codec, ctrl, data, len(g))  # each rank decodes the whole list's streams
    nt = O.tile_index(codec, ctrl, len(g)).shape[0]
    tb = split_tiles(nt, world)
    lo, hi = int(tb[rank]) * 1024, min(int(tb[rank + 1]) * 1024, len(g))
    seg = gaps_all[lo:hi]
    base = carry_in(int(seg.astype(np.uint64).sum()))
    ids = (np.cumsum(seg.astype(np.uint64)) + base) & 0xFFFFFFFF
    np.save(os.path.join(out_dir, f"list_{rank}.npy"), ids.astype(np.uint32))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_decode_on_cpu_ranks(world, tmp_path):
    import oracle as O
    import synth
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    codec = O.Codec(O.PFD, 32)
    lens = synth.zipf_index_lengths(400, 3, 3e4)
    gaps, off = synth.uniform_index(9, lens, 1_000_000)
    want = np.concatenate([O.prefix_sum(gaps[off[i]:off[i + 1]]) for i in range(len(lens))])
    got = np.concatenate([np.load(tmp_path / f"lists_{r}.npy") for r in range(world)])
    assert (got == want).all()
    g = synth.mixed_runs(11, 100_003, 256, 8.0, 0.1, 1 << 20)
    got = np.concatenate([np.load(tmp_path / f"list_{r}.npy") for r in range(world)])
    assert (got == O.prefix_sum(g)).all()
