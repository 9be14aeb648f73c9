"""The serving loop on the GPU: every request's docIDs are the same when it
is served alone and when it is served in a mix with others (several batches
in flight on several streams, a small arena that makes requests wait for
space), and equal the oracle's prefix sums of its lists. Integer work: no
tolerance."""
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


def _index(gc, kind, k, seed, nlists=200):
    rng = np.random.default_rng(seed)
    lens = rng.integers(1, 5000, size=nlists).astype(np.uint32)
    lens[:4] = [1, 1024, 1025, 40_000]
    gaps, off = synth.uniform_index(seed, lens, 2_000_000)
    d = torch.from_numpy(gaps.view(np.int32).copy()).cuda()
    return gc.encode_index(gc.make_codec(kind, k, zeta=0.1), d, lens), gaps, off


@pytest.mark.parametrize("kind,k", [(0, 32), (3, 32), (3, 4)])
def test_each_request_same_alone_and_in_the_mix(gc, kind, k):
    from paper_1502_01916_gb300.serve import Request, Server
    idx, gaps, off = _index(gc, kind, k, 31 + kind + k)
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(80):
        m = int(rng.integers(2, 9))
        lists = rng.choice(idx.nlists, size=m, replace=False).astype(np.uint32)
        reqs.append(Request(i, float(rng.uniform(0, 0.002)), lists))
    want = {r.rid: np.concatenate([O.prefix_sum(gaps[off[li]:off[li + 1]]) for li in r.lists.tolist()])
            for r in reqs}
    biggest = max(int(idx.lengths[r.lists].sum()) for r in reqs)

    def collect(into):
        return lambda r, view: into.__setitem__(r.rid, gc.as_u32(view).copy())

    mixed = {}
    srv = Server(idx, arena_ints=2 * biggest + 4096, streams=3, max_requests=6, max_lists=64, max_tiles=1 << 14)
    srv.run(reqs, on_complete=collect(mixed), time_limit=20.0)
    assert srv.batches > 10  # many batches, several in flight
    for r in reqs:
        assert (mixed[r.rid] == want[r.rid]).all(), f"request {r.rid} in the mix"
    alone = {}
    for r in reqs[:12]:
        one = Request(r.rid, 0.0, r.lists)
        Server(idx, arena_ints=biggest + 16, streams=1, max_lists=16, max_tiles=1 << 12).run(
            [one], on_complete=collect(alone), time_limit=20.0)
        assert (alone[r.rid] == mixed[r.rid]).all(), f"request {r.rid} alone vs in the mix"


def test_one_launch_per_list_baseline_matches(gc):
    from paper_1502_01916_gb300.serve import Request, serve_one_launch_per_list
    idx, gaps, off = _index(gc, 0, 32, 77, nlists=50)
    reqs = [Request(i, 0.0, np.array([i, i + 1], np.uint32)) for i in range(10)]
    wall, done = serve_one_launch_per_list(idx, reqs, time_limit=20.0)
    assert all(r.done >= 0 for r in done) and wall > 0
