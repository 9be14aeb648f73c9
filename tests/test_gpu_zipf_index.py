"""The batched decode at the shape of the rank-law (Zipf) index, on the GPU.

A scaled copy of the benchmark's index: 100,000 lists over 25M documents
with rank-law lengths L_r = C r^-1.1 (C = 3.0406e7, a tenth of the
benchmark's), clipped to [1, 2^22], so that it keeps the benchmark's mix of
one-tile lists, partial tiles and lists of millions of docIDs (lists longer
than 2^16 included); every list a sorted uniform sample, at a 16-byte
aligned output offset. It is encoded on the GPU with Group-Simple and
Group-PFD at k = 32, planned once, and decoded in one persistent launch with
the shape the autotuner picks; then

- every docID equals the oracle's prefix sum of its list's gaps;
- every list's control and data streams equal the oracle's encoding byte
  for byte;
- the serving loop over this resident index returns, for every request of a
  Poisson trace (2-8 lists drawn with probability proportional to
  length^0.5), the oracle's docIDs of its lists, and the same docIDs when a
  request is served alone.

Integer work: bit-exact, no tolerance."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

NLISTS, UNIVERSE, C = 100_000, 25_000_000, 3.0406e7


@pytest.fixture(scope="module")
def gc():
    from paper_1502_01916_gb300 import build
    build.build()
    import paper_1502_01916_gb300 as gc
    return gc


@pytest.fixture(scope="module")
def zipf():
    """(gaps, offsets, lengths, oracle docIDs per list)."""
    gaps, off, lengths = synth.zipf_index(NLISTS, UNIVERSE, 0, C=C, align=4)
    assert int(lengths.max()) > 1 << 16 and int(lengths.min()) >= 1
    ids = [O.prefix_sum(gaps[int(off[i]):int(off[i]) + int(lengths[i])]) for i in range(len(lengths))]
    return gaps, off, lengths, ids


@pytest.fixture(scope="module")
def indexes(gc, zipf):
    gaps, off, lengths, _ = zipf
    d = torch.from_numpy(gaps.view(np.int32)).cuda()
    out = {}
    for kind in (gc.SIMPLE, gc.PFD):
        out[kind] = gc.encode_index(gc.make_codec(kind, 32, zeta=0.1), d, lengths, out_offsets=off[:-1])
    del d
    return out


@pytest.mark.parametrize("kind", [0, 3], ids=["GS", "PFD"])
def test_zipf_index_every_docid_with_tuned_shape(gc, zipf, indexes, kind):
    from paper_1502_01916_gb300.tune import tune
    gaps, off, lengths, ids = zipf
    idx = indexes[kind]
    plan = gc.plan_index(idx)
    launch, info = tune(idx, plan, use_cache=False, reps=1)
    assert not info["cached"]
    out = torch.full((int(off[-1]),), -7, dtype=torch.int32, device="cuda")
    for _ in range(2):  # the plan is reused
        gc.decode_index(idx, out=out, launch=launch, plan=plan)
        got = gc.as_u32(out)
        for i in range(len(lengths)):
            a = int(off[i])
            assert (got[a:a + int(lengths[i])] == ids[i]).all(), f"list {i}"
        # the padding between lists is never written
        pad = np.ones(len(got), bool)
        for i in range(len(lengths)):
            pad[int(off[i]):int(off[i]) + int(lengths[i])] = False
        assert (got[pad] == np.uint32(0xFFFFFFF9)).all()


@pytest.mark.parametrize("kind", [0, 3], ids=["GS", "PFD"])
def test_zipf_index_streams_byte_identical(gc, zipf, indexes, kind):
    gaps, off, lengths, _ = zipf
    idx = indexes[kind]
    oc = O.Codec(kind, 32, zeta=0.1)
    lists = idx.lists.cpu().numpy().view(gc.LIST_DTYPE)
    ctrl_pool, data_pool = idx.ctrl.cpu().numpy(), gc.as_u32(idx.data)
    for i in range(len(lengths)):
        ctrl, data = O.encode(oc, gaps[int(off[i]):int(off[i]) + int(lengths[i])])
        d = lists[i]
        assert int(d["ctrl_bytes"]) == len(ctrl) and int(d["data_words"]) == len(data), f"list {i}"
        assert ctrl_pool[d["ctrl_off"]:d["ctrl_off"] + len(ctrl)].tobytes() == ctrl.tobytes(), f"list {i}"
        assert (data_pool[d["data_off"]:d["data_off"] + len(data)] == data).all(), f"list {i}"


def test_serving_over_the_zipf_index(gc, zipf, indexes):
    from paper_1502_01916_gb300.serve import Request, Server, poisson_trace
    gaps, off, lengths, ids = zipf
    idx = indexes[gc.PFD]
    reqs = poisson_trace(idx.lengths, 50_000.0, 0.006, seed=11)
    assert len(reqs) > 150
    biggest = max(int(idx.lengths[r.lists].sum()) for r in reqs)

    def collect(into):
        return lambda r, view: into.__setitem__(r.rid, gc.as_u32(view).copy())

    mixed = {}
    srv = Server(idx, arena_ints=2 * biggest + (1 << 20), streams=3)
    srv.run(reqs, on_complete=collect(mixed), time_limit=60.0)
    assert srv.batches > 5
    for r in reqs:
        want = np.concatenate([ids[li] for li in r.lists.tolist()])
        assert (mixed[r.rid] == want).all(), f"request {r.rid} in the mix"
    alone = {}
    for r in reqs[:10]:
        Server(idx, arena_ints=biggest + 16, streams=1).run([Request(r.rid, 0.0, r.lists)],
                                                           on_complete=collect(alone), time_limit=60.0)
        assert (alone[r.rid] == mixed[r.rid]).all(), f"request {r.rid} alone vs in the mix"
