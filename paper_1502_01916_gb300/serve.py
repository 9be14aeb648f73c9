"""Continuous-batching decode server over an index resident on the device.

Query processing decodes the posting lists of a query's terms (the paper's
query-processing experiments decode, for each query, the lists of its terms
and restore their docIDs, Sec 7.4). A server receives such requests
continuously. This module keeps one index (its pools and tile records)
resident on the GPU and serves requests of several lists each:

- requests are admitted while the output arena (the device memory that holds
  decoded lists until the caller has read them) has room for their ints and
  the batch's plan has room for their tiles; by default the arena takes half
  of the device memory free when the server starts, at most 4 GiB (the
  paper sets no admission rule: this one bounds the server by the memory it
  may hold, not by a request count). A request that has to wait for arena
  room is counted as an admission stall;
- whatever has arrived and fits is decoded as one batch: gc_plan_select
  builds the work records of exactly those lists, aimed at the requests'
  places in the arena, and gc_decode_plan decodes them in one persistent
  launch;
- batches go to a few CUDA streams in turn, so a batch that arrives while
  others are still on the GPU starts at once and overlaps them;
- a batch is complete when its event has completed; arena space is given
  back in batch order.

Everything that touches the data runs in the C library; this module only
schedules. The arena allocator and the batch former are plain Python and are
tested without a GPU.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque

import numpy as np

from . import gc as _gc


# ------------------------------------------------------------ host logic

class RingArena:
    """First-in first-out allocator over `size` units: allocations are
    contiguous, handed out in order, and given back in the same order. One
    that would run past the end starts at 0 and also holds the units it
    skipped, until it is given back."""

    def __init__(self, size: int):
        self.size = int(size)
        self.pos = 0
        self.used = 0
        self.held = deque()  # units each live allocation gives back, oldest first

    def alloc(self, n: int):
        """Offset of n contiguous units, or None when they do not fit now."""
        n = int(n)
        if n > self.size:
            return None
        if self.used == 0:
            self.pos = 0
        wrap = self.pos + n > self.size
        pad = self.size - self.pos if wrap else 0
        if self.used + pad + n > self.size:
            return None
        off = 0 if wrap else self.pos
        self.pos = off + n
        self.used += pad + n
        self.held.append(pad + n)
        return off

    def available(self) -> int:
        """The largest n that alloc(n) would take now."""
        if self.used == 0:
            return self.size
        here = min(self.size - self.pos, self.size - self.used)  # without wrapping
        wrapped = self.pos - self.used                           # from offset 0
        return max(here, wrapped, 0)

    def free_oldest(self):
        self.used -= self.held.popleft()

    @property
    def live(self) -> int:
        return len(self.held)


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float              # seconds from the start of the run
    lists: np.ndarray           # list indexes into the index
    ints: int = 0
    tiles: int = 0
    out: int = -1               # offset of its first int in the arena
    done: float = -1.0          # completion time (seconds from the start)
    waited: bool = False        # it once found the arena without room for it


def form_batch(pending: deque, arena: RingArena, max_requests: int, max_lists: int, max_tiles: int):
    """Take requests from the head of `pending` (in arrival order) while they
    fit the batch limits and the room the arena has now; each gets its arena
    offset. Returns the requests taken (none when even the first does not fit
    yet) and the arena units they hold. The first request left behind for
    want of arena room is marked as having waited."""
    room = arena.available()
    taken, lists, tiles, need = [], 0, 0, 0
    while pending and len(taken) < max_requests:
        r = pending[0]
        if len(r.lists) > max_lists or r.tiles > max_tiles or r.ints > arena.size:
            raise ValueError(f"request {r.rid} is larger than one batch")
        if lists + len(r.lists) > max_lists or tiles + r.tiles > max_tiles:
            break
        if need + r.ints > room:
            r.waited = True
            break
        taken.append(r)
        lists += len(r.lists)
        tiles += r.tiles
        need += r.ints
        pending.popleft()
    if not taken:
        return [], 0
    off = arena.alloc(need)
    assert off is not None  # within available()
    for r in taken:
        r.out = off
        off += r.ints
    return taken, need


def tiles_of(lengths: np.ndarray, k: int) -> np.ndarray:
    rows = (lengths.astype(np.int64) + k - 1) // k
    tr = _gc.TILE_INTS // k
    return (rows + tr - 1) // tr


def poisson_trace(lengths: np.ndarray, rate: float, duration: float, seed: int = 0, mmin: int = 2, mmax: int = 8):
    """Requests of the serving workload: Poisson arrivals at `rate` per second
    for `duration` seconds, each of m ~ U{mmin..mmax} lists drawn with
    probability proportional to length^0.5 (the generator lives in synth)."""
    import synth
    t, offs, ids = synth.serving_trace(lengths, rate, duration, seed, mmin, mmax)
    return [Request(i, float(t[i]), ids[offs[i]:offs[i + 1]].astype(np.uint32)) for i in range(len(t))]


# ------------------------------------------------------------ the server

class _Slot:
    """One stream with the buffers of one batch in flight."""

    def __init__(self, torch, dev, max_lists, max_tiles, ring: int = 4):
        self.stream = torch.cuda.Stream(device=dev)
        # host selection arrays in a small ring: a batch's pinned bytes are not
        # rewritten while its copy may still be reading them
        self.ring = ring
        self.turn = 0
        self.h_sel = [torch.empty(max_lists, dtype=torch.int32, pin_memory=True) for _ in range(ring)]
        self.h_out = [torch.empty(max_lists, dtype=torch.int64, pin_memory=True) for _ in range(ring)]
        self.d_sel = torch.empty(max_lists, dtype=torch.int32, device=dev)
        self.d_out = torch.empty(max_lists, dtype=torch.int64, device=dev)
        self.work = torch.empty(max(1, max_tiles) * _gc.WORK_BYTES, dtype=torch.uint8, device=dev)
        self.count = torch.zeros(2, dtype=torch.int64, device=dev)
        self.scratch = torch.empty(_gc.gc_decode_plan_scratch_size(max_tiles), dtype=torch.uint8, device=dev)
        self.status = torch.zeros(2, dtype=torch.int32, device=dev)
        self.event = torch.cuda.Event()
        self.batch = None  # (requests, units) while in flight


class Server:
    """Serves decode requests over `index` (a resident gc.Index)."""

    def __init__(self, index, arena_ints: int | None = None, streams: int = 3, max_requests: int = 2048,
                 max_lists: int = 16384, max_tiles: int = 1 << 18, restore_docids: bool = True,
                 launch=None, device=None):
        import torch
        self.torch = torch
        self.index = index
        self.dev = index.data.device if device is None else torch.device(device)
        if arena_ints is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            arena_ints = min(free // 2, 4 << 30) // 4
        self.k = index.codec.k
        self.tiles = tiles_of(index.lengths, self.k)
        self.arena = torch.empty(max(1, arena_ints), dtype=torch.int32, device=self.dev)
        self.alloc = RingArena(arena_ints)
        self.max_requests, self.max_lists, self.max_tiles = max_requests, max_lists, max_tiles
        self.restore = restore_docids
        self.launch = launch
        self.slots = [_Slot(torch, self.dev, max_lists, max_tiles) for _ in range(streams)]
        self.order = deque()  # slots with a batch in flight, oldest first
        self.launches = 0
        self.batches = 0

    def prepare(self, req: Request):
        req.ints = int(self.index.lengths[req.lists].sum(dtype=np.int64))
        req.tiles = int(self.tiles[req.lists].sum())

    def _free_slot(self):
        for s in self.slots:
            if s.batch is None:
                return s
        return None

    def _launch(self, slot: _Slot, reqs, units):
        sel = np.concatenate([r.lists for r in reqs]).astype(np.uint32)
        n = len(sel)
        # the batch's requests sit back to back in the arena from reqs[0].out,
        # their lists in order: each list goes where the ones before it end
        lens = self.index.lengths[sel].astype(np.int64)
        outs = np.empty(n, np.int64)
        outs[0] = reqs[0].out
        np.cumsum(lens[:-1], out=outs[1:])
        outs[1:] += reqs[0].out
        # the slot's previous batch has completed (its event), so its copies
        # are done and the pinned buffers of this turn are free
        h_sel, h_out = slot.h_sel[slot.turn], slot.h_out[slot.turn]
        slot.turn = (slot.turn + 1) % slot.ring
        h_sel[:n].numpy()[:] = sel.view(np.int32)
        h_out[:n].numpy()[:] = outs
        ix = self.index
        with self.torch.cuda.stream(slot.stream):
            slot.d_sel[:n].copy_(h_sel[:n], non_blocking=True)
            slot.d_out[:n].copy_(h_out[:n], non_blocking=True)
            _gc.gc_plan_select(ix.codec, ix.lists, ix.nlists, slot.d_sel, slot.d_out, n, ix.tiles, ix.ctrl,
                               slot.work, slot.count, slot.status, slot.stream)
            launches = _gc.gc_last_launch_count()
            _gc.gc_decode_plan(ix.codec, slot.work, slot.count, ix.ctrl, ix.data, self.arena, self.restore,
                               self.launch, slot.scratch, slot.status, slot.stream)
            self.launches += launches + _gc.gc_last_launch_count()
            slot.event.record(slot.stream)
        slot.batch = (reqs, units)
        self.order.append(slot)
        self.batches += 1

    def poll(self, now: float, on_complete=None):
        """Mark the requests of every batch whose event has completed; give
        back arena space in batch order. Returns the requests completed."""
        done = []
        for s in self.slots:
            if s.batch is not None and s.batch[0] and s.batch[0][0].done < 0 and s.event.query():
                for r in s.batch[0]:
                    r.done = now
                done.extend(s.batch[0])
        while self.order and self.order[0].batch[0][0].done >= 0:
            s = self.order.popleft()
            if on_complete is not None:
                # (each slot's status is read once the run ends)
                for r in s.batch[0]:
                    on_complete(r, self.arena[r.out:r.out + r.ints])
            self.alloc.free_oldest()
            s.batch = None
        return done

    def run(self, requests, on_complete=None, time_limit: float = 60.0):
        """Serve `requests` (arrival times in seconds from now) to completion.
        Returns (wall seconds, requests)."""
        for r in requests:
            self.prepare(r)
        arrivals = deque(sorted(requests, key=lambda r: r.arrival))
        pending = deque()
        left = len(requests)
        t0 = time.perf_counter()
        while left:
            now = time.perf_counter() - t0
            if now > time_limit:
                raise RuntimeError(f"serving did not finish within {time_limit} s")
            while arrivals and arrivals[0].arrival <= now:
                pending.append(arrivals.popleft())
            left -= len(self.poll(now, on_complete))
            slot = self._free_slot() if pending else None
            if slot is not None:
                reqs, units = form_batch(pending, self.alloc, self.max_requests, self.max_lists, self.max_tiles)
                if reqs:
                    self._launch(slot, reqs, units)
        self.torch.cuda.synchronize(self.dev)
        for s in self.slots:
            _gc.check_status(s.status, "served batch")
        return time.perf_counter() - t0, requests


def serve_one_launch_per_list(index, requests, restore_docids: bool = True, time_limit: float = 60.0,
                              issue_limit: float | None = None):
    """The baseline: each list of each request decoded by its own gc_decode
    call (one launch of the decoder per list) as requests arrive, on one
    stream, into a reused output buffer. With issue_limit, no request is
    issued after that many seconds (a saturated baseline then serves only
    the requests issued by then). Returns (wall seconds, the requests
    served)."""
    import ctypes
    import torch
    dev = index.data.device
    lists = index.lists.cpu().numpy().view(_gc.LIST_DTYPE)
    nmax = int(max(int(index.lengths[r.lists].max()) for r in requests))
    scratch = torch.empty(_gc.gc_decode_scratch_size(index.codec, nmax, True), dtype=torch.uint8, device=dev)
    out = torch.empty(max(1, nmax), dtype=torch.int32, device=dev)
    st = torch.zeros(2, dtype=torch.int32, device=dev)
    lib = _gc.load()
    cp = ctypes.byref(index.codec)
    cbase, dbase, tbase = index.ctrl.data_ptr(), index.data.data_ptr(), index.tiles.data_ptr()
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream
    order = sorted(requests, key=lambda r: r.arrival)
    inflight = deque()
    left = len(order)
    t0 = time.perf_counter()
    i = 0
    while left:
        now = time.perf_counter() - t0
        if now > time_limit:
            raise RuntimeError(f"per-list serving did not finish within {time_limit} s")
        if issue_limit is not None and now > issue_limit and not inflight:
            break
        while inflight and inflight[0][1].query():
            inflight.popleft()[0].done = now
            left -= 1
        if i < len(order) and order[i].arrival <= now and (issue_limit is None or now <= issue_limit):
            r = order[i]
            i += 1
            for li in r.lists.tolist():
                d = lists[li]
                tp = tbase + (int(d["tile_off"]) - 1) * _gc.TILE_BYTES
                rc = lib.gc_decode(cp, cbase + int(d["ctrl_off"]), int(d["ctrl_bytes"]), dbase + 4 * int(d["data_off"]),
                                   int(d["data_words"]), int(d["n"]), tp, out.data_ptr(), int(restore_docids),
                                   scratch.data_ptr(), scratch.numel(), st.data_ptr(), s)
                if rc:
                    raise _gc.GcError(rc, "gc_decode")
            ev = torch.cuda.Event()
            ev.record(stream)
            inflight.append((r, ev))
    torch.cuda.synchronize(dev)
    _gc.check_status(st, "per-list decode")
    return time.perf_counter() - t0, [r for r in order if r.done >= 0]


def latency_summary(requests, wall: float, lengths: np.ndarray, offered: int | None = None):
    """p50/p99/max latency of the served requests, their ints per second,
    and how many of them waited for arena room (admission stalls); offered
    is how many requests the trace held (when fewer were served)."""
    served = [r for r in requests if r.done >= 0]
    lat = np.array([r.done - r.arrival for r in served]) if served else np.zeros(1)
    ints = int(sum(int(lengths[r.lists].sum(dtype=np.int64)) for r in served))
    return {"requests": len(requests) if offered is None else int(offered), "served": len(served),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "max_ms": float(lat.max() * 1e3), "ints": ints, "ints_per_s": ints / wall, "wall_s": wall,
            "admission_waits": int(sum(1 for r in served if r.waited))}
