"""Interleaved decode of a list's docID and term-frequency streams (the
paper's TF columns, Sec 7.3) on the GPU, through the C ABI.

An index holds each list twice: its d-gaps (list i) and its TFs (list N + i,
values >= 1, geometric with mean 2). gc_plan_interleave plans the pairs tile
by tile (d-gap tile 0, TF tile 0, d-gap tile 1, ...), and one decode with
restore_docids = GC_RESTORE_PER_RECORD writes every list's docIDs (the
oracle's prefix sums) and its TFs (the values themselves) to their own
places. Lists of every size class: one int, partial tiles, whole tiles, and
many tiles. A pair whose d-gap tiles carry no skip entries, and a pair of
lists of different lengths, are refused with their error codes.

Integer work: bit-exact, no tolerance."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_1502_01916_gb300 import build
    build.build()
    import paper_1502_01916_gb300 as gc
    return gc


def pair_index(gc, codec, seed, nlists=160):
    rng = np.random.default_rng(seed)
    lens = rng.integers(1, 4000, size=nlists).astype(np.uint32)
    lens[:7] = [1, 31, 1023, 1024, 1025, 9000, 40000]
    rng.shuffle(lens)
    gaps, off = synth.uniform_index(seed, lens, 3_000_000)
    tfs, toff = synth.tf_index(seed + 1, lens, 2.0)
    both = np.concatenate([gaps, tfs])
    idx = gc.encode_index(codec, torch.from_numpy(both.view(np.int32).copy()).cuda(), np.concatenate([lens, lens]))
    return idx, lens, gaps, off, tfs, toff


CODECS = [(0, 32, {}), (3, 32, {}), (1, 32, {"cg": 8, "ld": 2}), (2, 32, {}), (0, 4, {}), (3, 4, {}),
          (1, 4, {"cg": 1, "ld": 0})]


@pytest.mark.parametrize("kind,k,kw", CODECS, ids=lambda x: str(x))
def test_interleaved_docids_and_tfs(gc, kind, k, kw):
    codec = gc.make_codec(kind, k, **kw)
    idx, lens, gaps, off, tfs, toff = pair_index(gc, codec, 41 + 3 * kind + k)
    N = len(lens)
    total = int(off[-1])
    pairs = np.stack([np.arange(N), N + np.arange(N)], axis=1)
    outs = np.stack([off[:-1], total + toff[:-1]], axis=1).astype(np.uint64)
    plan = gc.plan_interleave(idx, pairs, outs)
    nt = gc.tiles_of(codec, lens)
    assert int(plan.count[0].item()) == 2 * int(nt.sum())
    assert int(plan.count[1].item()) == 0  # every d-gap tile has its skip entry
    # records alternate tile by tile, the TF ones raw
    w = plan.work.cpu().numpy().view(gc.WORK_DTYPE)[:2 * int(nt.sum())]
    raw = (w["shape"] & np.uint32(gc.WORK_RAW)) != 0
    assert (raw == (w["list"] >= N)).all()
    assert (w["list"][0::2] + N == w["list"][1::2]).all() and (w["tile"][0::2] == w["tile"][1::2]).all()
    out = torch.full((2 * total,), -3, dtype=torch.int32, device="cuda")
    for _ in range(2):  # the plan is reused
        gc.decode_index(idx, out=out, restore_docids=gc.RESTORE_PER_RECORD, plan=plan)
        got = gc.as_u32(out)
        for i in range(N):
            a, n = int(off[i]), int(lens[i])
            assert (got[a:a + n] == O.prefix_sum(gaps[a:a + n])).all(), f"docIDs of list {i}"
            t = total + int(toff[i])
            assert (got[t:t + n] == tfs[int(toff[i]):int(toff[i]) + n]).all(), f"TFs of list {i}"


def test_interleave_needs_skip_entries(gc):
    codec = gc.make_codec(0, 32)
    idx, lens, gaps, off, tfs, toff = pair_index(gc, codec, 5, nlists=40)
    t = idx.tiles.view(torch.int32).view(-1, 8)
    t[:, 6] = 0  # base
    t[:, 7] = 0  # flags
    N = len(lens)
    with pytest.raises(gc.GcError) as ei:
        gc.plan_interleave(idx, np.stack([np.arange(N), N + np.arange(N)], axis=1),
                           np.zeros((N, 2), np.uint64))
    assert ei.value.code == 6  # GC_ERR_UNSUPPORTED


def test_interleave_refuses_lists_of_different_lengths(gc):
    codec = gc.make_codec(3, 32)
    idx, lens, gaps, off, tfs, toff = pair_index(gc, codec, 7, nlists=40)
    i = int(np.argmax(lens != lens[0]))
    assert lens[i] != lens[0]
    with pytest.raises(gc.GcError) as ei:
        gc.plan_interleave(idx, np.array([[0, len(lens) + i]]), np.zeros((1, 2), np.uint64))
    assert ei.value.code == 1  # GC_ERR_INVALID
