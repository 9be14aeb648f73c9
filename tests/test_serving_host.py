"""Host-side logic of the serving loop (no GPU): the arena allocator never
hands out overlapping live ranges and always fits a request into an empty
arena; batches take requests in arrival order within their limits."""
from collections import deque

import numpy as np
import pytest

from paper_1502_01916_gb300.serve import Request, RingArena, form_batch


@pytest.mark.parametrize("seed", range(5))
def test_ring_arena_against_occupancy_map(seed):
    rng = np.random.default_rng(seed)
    size = 1000
    arena = RingArena(size)
    live = deque()  # (offset, n)
    occ = np.zeros(size, bool)
    for _ in range(4000):
        if live and (rng.random() < 0.45 or arena.used > 0.9 * size):
            off, n = live.popleft()
            assert occ[off:off + n].all()
            occ[off:off + n] = False
            arena.free_oldest()
            continue
        n = int(rng.integers(1, 300))
        was_empty = not live
        off = arena.alloc(n)
        if off is None:
            assert not was_empty, "an empty arena takes any request that fits its size"
            continue
        assert 0 <= off and off + n <= size
        assert not occ[off:off + n].any(), "live ranges never overlap"
        occ[off:off + n] = True
        live.append((off, n))
    while live:
        live.popleft()
        arena.free_oldest()
    assert arena.used == 0 and arena.live == 0


def test_ring_arena_refuses_more_than_its_size():
    assert RingArena(10).alloc(11) is None


@pytest.mark.parametrize("seed", range(3))
def test_ring_arena_available_is_exact(seed):
    """available() is the largest request alloc() takes at that moment."""
    rng = np.random.default_rng(seed)
    arena = RingArena(500)
    for _ in range(2000):
        if arena.live and rng.random() < 0.4:
            arena.free_oldest()
            continue
        room = arena.available()
        probe = RingArena(500)
        probe.pos, probe.used, probe.held = arena.pos, arena.used, type(arena.held)(arena.held)
        assert probe.alloc(room) is not None or room == 0
        probe = RingArena(500)
        probe.pos, probe.used, probe.held = arena.pos, arena.used, type(arena.held)(arena.held)
        assert probe.alloc(room + 1) is None
        arena.alloc(int(rng.integers(1, 120)))


def _req(i, lists, ints, tiles):
    r = Request(i, 0.0, np.arange(lists, dtype=np.uint32))
    r.ints, r.tiles = ints, tiles
    return r


def test_form_batch_limits_and_offsets():
    pending = deque(_req(i, 3, 100, 5) for i in range(10))
    arena = RingArena(10_000)
    taken, units = form_batch(pending, arena, max_requests=4, max_lists=100, max_tiles=100)
    assert [r.rid for r in taken] == [0, 1, 2, 3] and units == 400
    assert [r.out for r in taken] == [0, 100, 200, 300]
    taken, _ = form_batch(pending, arena, max_requests=100, max_lists=7, max_tiles=100)
    assert [r.rid for r in taken] == [4, 5]  # 3 + 3 lists; a third would pass 7
    taken, _ = form_batch(pending, arena, max_requests=100, max_lists=100, max_tiles=12)
    assert [r.rid for r in taken] == [6, 7]  # 5 + 5 tiles


def test_form_batch_waits_for_arena_space():
    pending = deque(_req(i, 2, 600, 1) for i in range(3))
    arena = RingArena(1000)
    taken, _ = form_batch(pending, arena, 1, 100, 100)
    assert [r.rid for r in taken] == [0]
    assert not taken[0].waited
    taken, units = form_batch(pending, arena, 1, 100, 100)
    assert taken == [] and units == 0 and len(pending) == 2  # no room until request 0 is given back
    assert pending[0].waited and not pending[1].waited  # an admission stall, counted once per request
    arena.free_oldest()
    taken, _ = form_batch(pending, arena, 1, 100, 100)
    assert [r.rid for r in taken] == [1] and taken[0].waited


def test_batch_limits_are_not_admission_stalls():
    """A request left for the next batch by the batch's list or tile limit
    did not wait for arena room."""
    pending = deque(_req(i, 2, 10, 1) for i in range(3))
    taken, _ = form_batch(pending, RingArena(1000), 2, 100, 100)
    assert [r.rid for r in taken] == [0, 1] and not pending[0].waited


def test_latency_summary_counts_served_and_waits():
    from paper_1502_01916_gb300.serve import latency_summary
    rs = [_req(i, 2, 10, 1) for i in range(4)]
    for i, r in enumerate(rs[:3]):
        r.arrival, r.done = 0.0, 0.001 * (i + 1)
    rs[1].waited = True
    lengths = np.full(10, 5, np.uint32)
    s = latency_summary(rs, 1.0, lengths, offered=4)
    assert s["requests"] == 4 and s["served"] == 3 and s["admission_waits"] == 1
    assert abs(s["max_ms"] - 3.0) < 1e-9


def test_form_batch_never_asks_more_than_the_arena_holds():
    """A batch stops at the arena's room, so requests that are each small but
    together larger than the arena still get served (the first alone)."""
    pending = deque(_req(i, 2, 600, 1) for i in range(3))
    arena = RingArena(1000)
    taken, _ = form_batch(pending, arena, 10, 100, 100)
    assert [r.rid for r in taken] == [0]
    arena.free_oldest()
    taken, _ = form_batch(pending, arena, 10, 100, 100)
    assert [r.rid for r in taken] == [1]


def test_form_batch_rejects_a_request_larger_than_a_batch():
    with pytest.raises(ValueError):
        form_batch(deque([_req(0, 50, 10, 1)]), RingArena(100), 10, 10, 10)
