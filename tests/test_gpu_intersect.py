"""AND queries (gc_intersect) against the plain definition: the docIDs two
lists have in common, in increasing order (the lists' docIDs are the prefix
sums of their gaps; numpy's set intersection of those is the expected
result). Indexes of every codec at k = 4 and 32, with skip entries; pairs
of short and long lists, identical lists, empty lists and lists whose
docID ranges do not meet."""
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


def index_lists(seed, universe):
    rng = np.random.default_rng(seed)
    lens = rng.integers(1, 5000, size=120).astype(np.uint32)
    lens[:10] = [0, 1, 2, 1023, 1024, 1025, 40000, 90000, 3, 0]
    gaps, off = synth.uniform_index(seed, lens, universe)
    # one list confined to the top of the universe (its range meets few others)
    top = np.sort(rng.choice(np.arange(universe - 5000, universe), 2000, replace=False)).astype(np.uint32)
    g = np.diff(np.concatenate(([0], top))).astype(np.uint32)
    lens = np.append(lens, np.uint32(len(g)))
    gaps = np.concatenate((gaps, g))
    off = np.append(off, off[-1] + len(g))
    return lens, gaps, off


CODECS = [(O.SIMPLE, 32, {}), (O.PFD, 32, {"zeta": 0.1}), (O.AFOR, 32, {}), (O.SCHEME, 32, {"cg": 8, "ld": 2}),
          (O.SIMPLE, 4, {}), (O.PFD, 4, {"zeta": 0.1})]


@pytest.mark.parametrize("kind,k,kw", CODECS, ids=lambda x: repr(x))
def test_intersect_matches_set_intersection(gc, kind, k, kw):
    universe = 400_000
    lens, gaps, off = index_lists(7 + k + kind, universe)
    idx = gc.encode_index(gc.make_codec(kind, k, **kw), torch.from_numpy(gaps.view(np.int32)).cuda(), lens)
    ids = [O.prefix_sum(gaps[off[i]:off[i + 1]]) for i in range(len(lens))]
    rng = np.random.default_rng(kind * 10 + k)
    n = len(lens)
    pairs = [(0, 7), (7, 0), (7, 7), (6, 7), (1, 7), (4, 5), (n - 1, 7), (n - 1, 3), (9, 9), (2, 8)]
    pairs += [tuple(int(x) for x in rng.integers(0, n, 2)) for _ in range(150)]
    res, counts, offs = gc.intersect(idx, pairs)
    for q, (i, j) in enumerate(pairs):
        want = np.intersect1d(ids[i], ids[j]).astype(np.uint32)
        got = res[int(offs[q]):int(offs[q]) + int(counts[q])]
        assert int(counts[q]) == len(want), (q, i, j)
        assert (got == want).all(), (q, i, j)


def test_intersect_without_skip_entries_is_refused(gc):
    """Tile records without skip entries cannot bound a tile's docIDs: the
    call reports GC_ERR_UNSUPPORTED instead of guessing."""
    lens, gaps, off = index_lists(3, 400_000)
    idx = gc.encode_index(gc.make_codec(O.SIMPLE, 32), torch.from_numpy(gaps.view(np.int32)).cuda(), lens)
    t = idx.tiles.view(torch.int32).view(-1, 8).clone()
    t[:, 7] = 0  # clear the flags word of every record
    idx.tiles = t.view(torch.uint8).reshape(-1)
    with pytest.raises(gc.GcError) as ei:
        gc.intersect(idx, [(4, 7)])
    assert ei.value.code == 6
