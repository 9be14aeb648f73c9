"""GPU parity: the CUDA library against the CPU oracle, bit for bit.

Every test goes through the C ABI (via the ctypes binding). Decoding is
checked on streams the oracle encoded; encoding is checked byte for byte
against the oracle's streams; the batched decoder is checked on indexes the
GPU encoder built, list by list against the oracle. Integer work: no
tolerance anywhere.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

K_GSC = [(1, 0), (2, 0), (4, 0), (8, 0), (1, 1), (2, 1), (4, 1), (8, 1), (4, 2), (8, 2)]
CODECS = ([(O.SIMPLE, k, 0, 0, 0.1) for k in (4, 32)]
          + [(O.SCHEME, k, cg, ld, 0.1) for k in (4, 32) for cg, ld in K_GSC]
          + [(O.AFOR, k, 0, 0, 0.1) for k in (4, 32)]
          + [(O.PFD, k, 0, 0, z) for k in (4, 32) for z in (0.0, 0.01, 0.1, 0.3)])


def cid(c):
    kind, k, cg, ld, z = c
    return repr(O.Codec(kind, k, cg or 8, ld, z))


@pytest.fixture(scope="module")
def gc():
    from paper_1502_01916_gb300 import build
    build.build()
    import paper_1502_01916_gb300 as gc
    return gc


def pair(gc, c):
    kind, k, cg, ld, z = c
    return O.Codec(kind, k, cg or 8, ld, z), gc.make_codec(kind, k, cg or 8, ld, z)


def upload_u8(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint8).copy()).cuda()


def upload_u32(a):
    a = np.ascontiguousarray(a, np.uint32)
    if a.size == 0:
        a = np.zeros(4, np.uint32)
    return torch.from_numpy(a.view(np.int32).copy()).cuda()


def inputs(seed, n):
    """Values of every width (one case in four) or d-gap-like mixes."""
    if seed % 4 == 0:
        return synth.width_mix(seed, n, 0, 32)
    if seed % 4 == 1:
        return synth.width_mix(seed, n, 0, 9)
    if seed % 4 == 2:
        return synth.mixed_runs(seed, n, 256, 8.0, 0.1, 1 << 20)
    return synth.geometric_gaps(seed, n, 20.0)


SIZES = [1, 3, 31, 129, 1000, 1024, 1025, 4100, 33007]


# ------------------------------------------------------------------- decode

@pytest.mark.parametrize("c", CODECS, ids=cid)
def test_decode_matches_oracle(gc, c):
    """Oracle-encoded streams, decoded on the GPU with the oracle's tile index,
    with the GPU-built tile index and with none (built inside gc_decode)."""
    oc, gcc = pair(gc, c)
    for i, n in enumerate(SIZES):
        g = inputs(17 * i + c[1], n)
        ctrl, data = O.encode(oc, g)
        want_gaps = O.decode(oc, ctrl, data, n)
        assert (want_gaps == g).all()
        want_ids = O.prefix_sum(want_gaps)
        tiles_ref = O.tile_index(oc, ctrl, n)
        tiles_skip = O.tile_index(oc, ctrl, n, g)
        d_ctrl, d_data = upload_u8(ctrl), upload_u32(data)
        enc = gc.EncodedList(gcc, n, d_ctrl, d_data[:len(data)], upload_u8(tiles_ref.view(np.uint8)))
        got = gc.as_u32(gc.decode(enc, restore_docids=False))
        assert (got == want_gaps).all(), f"gaps n={n}"
        got = gc.as_u32(gc.decode(enc, restore_docids=True))
        assert (got == want_ids).all(), f"docids by look-back n={n}"
        enc_s = gc.EncodedList(gcc, n, d_ctrl, d_data[:len(data)], upload_u8(tiles_skip.view(np.uint8)))
        got = gc.as_u32(gc.decode(enc_s, restore_docids=True))
        assert (got == want_ids).all(), f"docids from skip entries n={n}"
        built = gc.build_tiles(gcc, d_ctrl, n).cpu().numpy()
        assert built.tobytes() == tiles_ref.tobytes(), f"tile index n={n}"
        got = gc.as_u32(gc.decode(enc, restore_docids=True, use_tiles=False))
        assert (got == want_ids).all(), f"docids without tiles n={n}"


@pytest.mark.parametrize("k", [4, 32])
def test_decode_paper_buffer(gc, k):
    """Section 4.3: the data-area offset is read from the buffer head."""
    oc, gcc = pair(gc, (O.SIMPLE, k, 0, 0, 0.1))
    g = synth.single_list_geometric(65536, 20.0, 0)
    ctrl, data = O.encode(oc, g)
    buf = O.paper_pack(ctrl, data)
    got = gc.as_u32(gc.decode_paper(gcc, upload_u8(buf), len(g)))
    assert (got == O.prefix_sum(g)).all()


def test_prefix_sum_wraps_mod_2_32(gc):
    """Gaps near 2^32: docIDs wrap modulo 2^32 on both sides."""
    oc, gcc = pair(gc, (O.PFD, 32, 0, 0, 0.1))
    g = synth.uniform_u32(5, 5000, 1 << 30, 0xFFFFFFFF)
    ctrl, data = O.encode(oc, g)
    enc = gc.EncodedList(gcc, len(g), upload_u8(ctrl), upload_u32(data), None)
    got = gc.as_u32(gc.decode(enc, restore_docids=True, use_tiles=False))
    assert (got == O.prefix_sum(g)).all()


@pytest.mark.parametrize("c", [(O.SIMPLE, 32, 0, 0, 0.1), (O.AFOR, 4, 0, 0, 0.1), (O.SCHEME, 4, 8, 2, 0.1),
                               (O.PFD, 32, 0, 0, 0.1)], ids=cid)
def test_corrupt_control_is_reported(gc, c):
    """A malformed control area ends in GC_ERR_CORRUPT, never in a fault."""
    oc, gcc = pair(gc, c)
    g = inputs(3, 5000)
    ctrl, data = O.encode(oc, g)
    bad = ctrl.copy()
    if c[0] == O.SIMPLE:
        bad[1] = 0xFF                      # selectors 2 and 3 become 15
    elif c[0] == O.AFOR:
        bad[0] = 0xFF                      # size code 3, b = 63
    elif c[0] == O.SCHEME:
        bad[:] = 0xFF                      # no closing zero anywhere
    else:
        bad[0] = (bad[0] & 0xC0) | 40      # b = 40
    enc = gc.EncodedList(gcc, len(g), upload_u8(bad), upload_u32(data), None)
    with pytest.raises(gc.GcError) as ei:
        gc.decode(enc, restore_docids=True, use_tiles=False)
    assert ei.value.code == 3


def test_truncated_data_is_reported(gc):
    oc, gcc = pair(gc, (O.SIMPLE, 32, 0, 0, 0.1))
    g = inputs(4, 5000)
    ctrl, data = O.encode(oc, g)
    enc = gc.EncodedList(gcc, len(g), upload_u8(ctrl), upload_u32(data)[:len(data) // 2], None)
    with pytest.raises(gc.GcError) as ei:
        gc.decode(enc, restore_docids=False, use_tiles=False)
    assert ei.value.code == 3


# ------------------------------------------------------------------- encode

@pytest.mark.parametrize("c", CODECS, ids=cid)
def test_encode_byte_identical(gc, c):
    """GPU streams and tile index equal the oracle's, byte for byte."""
    oc, gcc = pair(gc, c)
    for i, n in enumerate([1, 5, 1000, 1025, 4100, 33007]):
        g = inputs(31 * i + c[1] + 1, n)
        ctrl, data = O.encode(oc, g)
        enc = gc.encode(gcc, g)
        assert enc.ctrl.cpu().numpy().tobytes() == ctrl.tobytes(), f"control n={n}"
        assert (gc.as_u32(enc.data) == data).all(), f"data n={n}"
        assert enc.tiles.cpu().numpy().tobytes() == O.tile_index(oc, ctrl, n, g).tobytes(), f"tiles n={n}"


# ------------------------------------------------------------------- batch

def small_index(seed, nlists=300, universe=2_000_000):
    rng = np.random.default_rng(seed)
    lens = rng.integers(1, 3000, size=nlists).astype(np.uint32)
    lens[:12] = [0, 1, 2, 31, 32, 33, 1023, 1024, 1025, 2048, 70000, 0]
    rng.shuffle(lens)
    gaps, off = synth.uniform_index(seed, lens, universe)
    return lens, gaps, off


@pytest.mark.parametrize("c", CODECS, ids=cid)
def test_batch_encode_decode(gc, c):
    """gc_encode_batch lays out the oracle's per-list streams; gc_decode_batch
    restores every list's docIDs (and raw gaps) in one launch."""
    oc, gcc = pair(gc, c)
    lens, gaps, off = small_index(11 + c[1])
    idx = gc.encode_index(gcc, upload_u32(gaps), lens)
    lists = idx.lists.cpu().numpy().view(gc.LIST_DTYPE)
    ctrl_pool = idx.ctrl.cpu().numpy()
    data_pool = gc.as_u32(idx.data)
    tiles_pool = idx.tiles.cpu().numpy().view(O.TILE_DTYPE)
    want_ids = np.zeros(len(gaps), np.uint32)
    for i, n in enumerate(lens.tolist()):
        g = gaps[off[i]:off[i + 1]]
        ctrl, data = O.encode(oc, g)
        d = lists[i]
        assert int(d["n"]) == n and int(d["out_off"]) == int(off[i])
        assert int(d["ctrl_bytes"]) == len(ctrl) and int(d["data_words"]) == len(data), f"sizes list {i}"
        assert ctrl_pool[d["ctrl_off"]:d["ctrl_off"] + len(ctrl)].tobytes() == ctrl.tobytes(), f"list {i}"
        assert (data_pool[d["data_off"]:d["data_off"] + len(data)] == data).all(), f"list {i}"
        tref = O.tile_index(oc, ctrl, n, g)
        if len(tref) > 1:
            got_t = tiles_pool[d["tile_off"]:d["tile_off"] + len(tref) - 1]
            assert got_t.tobytes() == tref[1:].tobytes(), f"tiles list {i}"
        want_ids[off[i]:off[i + 1]] = O.prefix_sum(g)
    out = gc.decode_index(idx, restore_docids=True)
    assert (gc.as_u32(out)[:len(gaps)] == want_ids).all()
    out = gc.decode_index(idx, restore_docids=False)
    assert (gc.as_u32(out)[:len(gaps)] == gaps).all()


@pytest.mark.parametrize("n", [1024, 5000, 33007])
def test_pfd_exceptions_beyond_the_staging_room(gc, n):
    """Group-PFD at k = 32 with wide slots (b = 28) and every fourth row an
    exception row (8 of 32, under zeta = 0.3's limit of 9): a tile's 256
    exception values outnumber the 165 free words of the re-lay buffer, so
    the decoder reads them in place."""
    rng = np.random.default_rng(n)
    g = rng.integers(1 << 27, 1 << 28, size=n, dtype=np.uint64)
    wide = (np.arange(n) // 32) % 4 == 0
    g[wide] = rng.integers(1 << 30, 1 << 31, size=int(wide.sum()), dtype=np.uint64)
    g = g.astype(np.uint32)
    oc, gcc = pair(gc, (O.PFD, 32, 0, 0, 0.3))
    ctrl, data = O.encode(oc, g)
    assert (O.decode(oc, ctrl, data, n) == g).all()
    tiles = O.tile_index(oc, ctrl, n, g)
    d_data = upload_u32(data)
    enc = gc.EncodedList(gcc, n, upload_u8(ctrl), d_data[:len(data)], upload_u8(tiles.view(np.uint8)))
    for use_tiles in (True, False):
        for restore in (True, False):
            out = gc.decode(enc, restore_docids=restore, use_tiles=use_tiles)
            want = O.prefix_sum(g) if restore else g
            assert (gc.as_u32(out)[:n] == want).all(), (use_tiles, restore)


@pytest.mark.parametrize("kind", [O.SIMPLE, O.PFD, O.AFOR])
@pytest.mark.parametrize("k", [4, 32])
def test_batch_aligned_outputs(gc, kind, k):
    """Lists whose outputs start at 16-byte boundaries (gaps laid out with
    padding, output at the same offsets): whole tiles take 16-byte stores.
    Every list equals the oracle's docIDs and the padding stays untouched."""
    oc, gcc = pair(gc, (kind, k, 0, 0, 0.1))
    lens, gaps, off = small_index(23 + k)
    L = lens.astype(np.uint64)
    span = (L + 3) // 4 * 4 + 4 * (np.arange(len(L)) % 3 == 0)  # some gaps wider than the rounding
    outs = np.zeros(len(L), np.uint64)
    np.cumsum(span[:-1], out=outs[1:])
    total = int(outs[-1] + L[-1])
    padded = np.full(total, 0xDEADBEEF, np.uint32)
    for i in range(len(L)):
        padded[int(outs[i]):int(outs[i]) + int(L[i])] = gaps[off[i]:off[i + 1]]
    idx = gc.encode_index(gcc, upload_u32(padded), lens, out_offsets=outs)
    for restore in (True, False):
        out = torch.full((total,), -7, dtype=torch.int32, device="cuda")
        gc.decode_index(idx, out=out, restore_docids=restore)
        got = gc.as_u32(out)
        hole = np.ones(total, bool)
        for i in range(len(L)):
            a, n = int(outs[i]), int(L[i])
            g = gaps[off[i]:off[i + 1]]
            want = O.prefix_sum(g) if restore else g
            assert (got[a:a + n] == want).all(), (i, n, restore)
            hole[a:a + n] = False
        assert (got[hole] == np.uint32(0xFFFFFFF9)).all()


@pytest.mark.parametrize("warps,bps,claim,stage", [(1, 1, 1, 0), (4, 2, 2, 0), (8, 0, 0, 0), (15, 1, 7, 0),
                                                   (2, 1, 16, 12288), (11, 2, 32, 20480), (3, 4, 5, 0)])
@pytest.mark.parametrize("k", [4, 32])
def test_batch_launch_shapes(gc, warps, bps, claim, stage, k):
    """The result does not depend on the launch shape (decoding warps per
    block, blocks per SM, records per claim, ring bytes), with a plan built
    once and reused."""
    oc, gcc = pair(gc, (O.PFD, k, 0, 0, 0.1))
    lens, gaps, off = small_index(5)
    idx = gc.encode_index(gcc, upload_u32(gaps), lens)
    want = np.concatenate([O.prefix_sum(gaps[off[i]:off[i + 1]]) for i in range(len(lens))])
    out = gc.decode_index(idx, launch=gc.gc_launch(warps, bps, claim, stage))
    assert (gc.as_u32(out)[:len(gaps)] == want).all()
    plan = gc.plan_index(idx)
    assert int(plan.count[0].item()) == idx.max_tiles
    assert int(plan.count[1].item()) == 0  # every tile has its skip entry
    for _ in range(2):
        out = gc.decode_index(idx, launch=gc.gc_launch(warps, bps, claim, stage), plan=plan)
        assert (gc.as_u32(out)[:len(gaps)] == want).all()


@pytest.mark.parametrize("c", [(O.SIMPLE, 32, 0, 0, 0.1), (O.SCHEME, 32, 4, 1, 0.1), (O.AFOR, 32, 0, 0, 0.1)])
def test_batch_widest_block(gc, c):
    """k = 32 with the most decoding warps a block can have (23, one block
    per SM) and the smallest ring a shape may ask for."""
    _, gcc = pair(gc, c)
    lens, gaps, off = small_index(8)
    idx = gc.encode_index(gcc, upload_u32(gaps), lens)
    want = np.concatenate([O.prefix_sum(gaps[off[i]:off[i + 1]]) for i in range(len(lens))])
    for launch in (gc.gc_launch(23, 1, 32, 0), gc.gc_launch(23, 1, 32, 12288)):
        out = gc.decode_index(idx, launch=launch)
        assert (gc.as_u32(out)[:len(gaps)] == want).all()


def test_launch_shape_out_of_range_rejected(gc):
    """Claims of more than 32 records, more decoding warps than a block may
    have, more than 8 blocks per SM, and shapes that leave the ring less
    than 12 KB are refused on the host, before any launch."""
    for k, too_many in ((32, 24), (4, 16)):
        _, gcc = pair(gc, (O.SIMPLE, k, 0, 0, 0.1))
        lens, gaps, off = small_index(4, nlists=20)
        idx = gc.encode_index(gcc, upload_u32(gaps), lens)
        for bad in (gc.gc_launch(4, 0, 33), gc.gc_launch(too_many, 0, 1), gc.gc_launch(4, 9, 1),
                    gc.gc_launch(4, 1, 1, 4096), gc.gc_launch(too_many - 1, 4, 1)):
            with pytest.raises(gc.GcError) as ei:
                gc.decode_index(idx, launch=bad)
            assert ei.value.code == 1, (k, bad.warps_per_block, bad.blocks_per_sm, bad.stage_bytes)


def test_plan_records(gc):
    """Each plan record carries its list's areas, its tile's first unit and
    skip entry, and staging ranges inside the list; lists in order, a list's
    tiles at consecutive records."""
    for c in [(O.SIMPLE, 4, 0, 0, 0.1), (O.PFD, 32, 0, 0, 0.1), (O.AFOR, 32, 0, 0, 0.1)]:
        oc, gcc = pair(gc, c)
        k = c[1]
        lens, gaps, off = small_index(8, nlists=40)
        idx = gc.encode_index(gcc, upload_u32(gaps), lens)
        lists = idx.lists.cpu().numpy().view(gc.LIST_DTYPE)
        plan = gc.plan_index(idx)
        w = plan.work.cpu().numpy().view(gc.WORK_DTYPE)
        ntiles = [-(-(-(-int(n) // k)) // (1024 // k)) for n in lens]
        seen = {}
        recs = w[:int(plan.count[0].item())]
        for j, r in enumerate(recs):
            seen.setdefault(int(r["list"]), []).append(j)
        assert sorted(seen) == [i for i in range(len(lens)) if ntiles[i] > 0]
        for i, js in seen.items():
            assert js == list(range(js[0], js[0] + ntiles[i])), "a list's tiles are consecutive records"
            g = gaps[off[i]:off[i + 1]]
            ctrl, data = O.encode(oc, g)
            tref = O.tile_index(oc, ctrl, int(lens[i]), g)
            d = lists[i]
            for t, j in enumerate(js):
                r = recs[j]
                sh = int(r["shape"])
                assert int(r["tile"]) == t
                assert int(r["ctrl_at"]) == int(d["ctrl_off"]) and int(r["ctrl_bytes"]) == len(ctrl)
                assert int(r["out_at"]) == int(off[i]) + 1024 * t
                assert (sh & 1023) + 1 == min(1024, int(lens[i]) - 1024 * t)
                assert int(r["ctrl_bit"]) == int(tref[t]["ctrl_bit"])
                skip = int(tref[t]["row_skip"])
                first = int(tref[t]["lane_bit"])  # lane bit of the tile's first row
                if c[0] == O.AFOR and skip:
                    first += skip * (int(ctrl[int(tref[t]["ctrl_bit"]) >> 3]) & 63)
                assert (sh >> gc.WORK_BIT_SHIFT) & 31 == first & 31
                assert (sh >> gc.WORK_SKIP_SHIFT) & 31 == skip
                assert int(r["data_at"]) == int(d["data_off"]) + (first >> 5) * k
                vecs = (sh >> gc.WORK_VEC_SHIFT) & 511
                assert vecs <= 1024 // k + 1
                assert int(r["data_at"]) + vecs * k <= int(d["data_off"]) + len(data)
                assert sh & gc.WORK_HAS_BASE and int(r["base"]) == int(tref[t]["base"])
                assert (int(r["ctrl_at"]) + int(r["win_at"])) % 16 == 0 and int(r["win_len"]) % 16 == 0
                assert not sh & gc.WORK_PUBLISH


def test_batch_without_skip_entries_uses_look_back(gc):
    """An index whose tile records carry no bases (as gc_build_tiles would
    give): every tile after a list's first takes its prefix by look-back,
    claimed one at a time, and the docIDs are the same."""
    for c in [(O.SIMPLE, 32, 0, 0, 0.1), (O.PFD, 4, 0, 0, 0.1), (O.SCHEME, 32, 8, 2, 0.1)]:
        oc, gcc = pair(gc, c)
        lens, gaps, off = small_index(21 + c[1], nlists=120)
        idx = gc.encode_index(gcc, upload_u32(gaps), lens)
        t = idx.tiles.view(torch.int32).view(-1, 8)
        t[:, 6] = 0  # base
        t[:, 7] = 0  # flags
        plan = gc.plan_index(idx)
        assert int(plan.count[1].item()) == len(idx.tiles) // gc.TILE_BYTES
        want = np.concatenate([O.prefix_sum(gaps[off[i]:off[i + 1]]) for i in range(len(lens))])
        for launch in (None, gc.gc_launch(2, 1, 4)):
            out = gc.decode_index(idx, launch=launch, plan=plan)
            assert (gc.as_u32(out)[:len(gaps)] == want).all()
        out = gc.decode_index(idx)
        assert (gc.as_u32(out)[:len(gaps)] == want).all()


def test_batch_overflow_reports_nospace(gc):
    """A scratch sized for fewer tiles than the batch has: GC_ERR_NOSPACE."""
    _, gcc = pair(gc, (O.SIMPLE, 32, 0, 0, 0.1))
    lens, gaps, off = small_index(6, nlists=50)
    idx = gc.encode_index(gcc, upload_u32(gaps), lens)
    idx.max_tiles = max(1, idx.max_tiles // 2)
    with pytest.raises(gc.GcError) as ei:
        gc.decode_index(idx)
    assert ei.value.code == 2


# ------------------------------------------------------------ full sizes

CONFIG2 = [(O.SIMPLE, k, 0, 0, 0.1) for k in (4, 32)] + \
    [(O.SCHEME, k, cg, ld, 0.1) for k in (4, 32) for cg, ld in [(1, 0), (1, 1), (8, 0), (8, 2), (8, 1)]] + \
    [(O.AFOR, k, 0, 0, 0.1) for k in (4, 32)] + [(O.PFD, k, 0, 0, 0.1) for k in (4, 32)]


@pytest.mark.parametrize("c", CONFIG2, ids=cid)
def test_mixed_2_26_single_list(gc, c):
    """2^26 d-gaps (90% geometric mean 8, 10% uniform to 2^20, runs of 256):
    GPU encoding equals the oracle's; one-launch decode restores the gaps
    and the docIDs."""
    oc, gcc = pair(gc, c)
    g = synth.single_list_mixed(1 << 26, 0)
    enc = gc.encode(gcc, g)
    ctrl, data = O.encode(oc, g)
    assert enc.ctrl.cpu().numpy().tobytes() == ctrl.tobytes()
    assert (gc.as_u32(enc.data) == data).all()
    got = gc.as_u32(gc.decode(enc, restore_docids=False))
    assert (got == g).all()
    want = O.prefix_sum(g)
    got = gc.as_u32(gc.decode(enc, restore_docids=True))
    assert (got == want).all()
    got = gc.as_u32(gc.decode(enc, restore_docids=True, use_tiles=False))  # 2^16 tiles by look-back
    assert (got == want).all()


def _segmented_prefix(gaps, off, lengths):
    """docIDs of every list of an index from its gaps (uint32 wraparound)."""
    cs = np.cumsum(gaps, dtype=np.uint32)
    starts = off[:-1].astype(np.int64)
    before = np.where(starts > 0, cs[np.maximum(starts - 1, 0)], 0).astype(np.uint32)
    return cs - np.repeat(before, lengths.astype(np.int64))


@pytest.fixture(scope="module")
def clustered_index():
    """4,000,000 lists over 50M documents: log-normal lengths (median 12,
    sigma 1.5), docIDs in clustered runs (mean 16) separated by jumps (mean
    5000)."""
    gaps, off, lengths = synth.clustered_short_index(4_000_000, 50_000_000, 0)
    return gaps, off, lengths


@pytest.mark.parametrize("c", [(O.SCHEME, 32, 8, 2, 0.1), (O.SCHEME, 32, 8, 0, 0.1), (O.PFD, 32, 0, 0, 0.01),
                               (O.PFD, 32, 0, 0, 0.1), (O.PFD, 32, 0, 0, 0.3)], ids=cid)
def test_clustered_short_lists_4m(gc, clustered_index, c):
    """The clustered short-list index: every docID of one batched decode
    equals the host's prefix sums, and a sample of lists is encoded exactly
    as the oracle encodes it."""
    oc, gcc = pair(gc, c)
    gaps, off, lengths = clustered_index
    idx = gc.encode_index(gcc, upload_u32(gaps), lengths)
    out = gc.decode_index(idx, restore_docids=True)
    want = _segmented_prefix(gaps, off, lengths)
    assert (gc.as_u32(out)[:len(gaps)] == want).all()
    lists = idx.lists.cpu().numpy().view(gc.LIST_DTYPE)
    ctrl_pool, data_pool = idx.ctrl.cpu().numpy(), gc.as_u32(idx.data)
    rng = np.random.default_rng(1)
    for i in rng.choice(len(lengths), 300, replace=False).tolist():
        ctrl, data = O.encode(oc, gaps[off[i]:off[i + 1]])
        d = lists[i]
        assert ctrl_pool[d["ctrl_off"]:d["ctrl_off"] + len(ctrl)].tobytes() == ctrl.tobytes(), f"list {i}"
        assert (data_pool[d["data_off"]:d["data_off"] + len(data)] == data).all(), f"list {i}"
