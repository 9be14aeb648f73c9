"""Variable Byte for short lists (Sec 2.3, Sec 7.5) on the GPU against the
oracle: the batch encoder's bytes equal the oracle's, list by list; the
batch decoder restores gaps and docIDs; an index whose short lists are
Variable Byte decodes every list to its prefix sums and is smaller than the
same index with Group codecs alone in the short-list regime."""
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


def short_lists(seed, nlists=3000):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, 64, size=nlists).astype(np.uint32)
    lens[:4] = [0, 1, 63, 2]
    g = synth.width_mix(seed, int(lens.sum()), 0, 32)
    off = np.zeros(nlists + 1, np.uint64)
    np.cumsum(lens, out=off[1:])
    return lens, g, off


def test_vb_batch_matches_oracle(gc):
    lens, g, off = short_lists(3)
    dev = torch.device("cuda")
    d_gaps = torch.from_numpy(g.view(np.int32)).to(dev)
    d_lists = torch.empty(len(lens) * gc.VB_LIST_BYTES, dtype=torch.uint8, device=dev)
    d_bytes = torch.empty(5 * len(g), dtype=torch.uint8, device=dev)
    d_total = torch.zeros(1, dtype=torch.int64, device=dev)
    d_off = torch.from_numpy(off[:-1].view(np.int64)).to(dev)
    d_n = torch.from_numpy(lens.view(np.int32)).to(dev)
    gc.gc_vb_encode_batch(d_gaps, d_off, d_n, len(lens), d_lists, d_bytes, d_total)
    recs = d_lists.cpu().numpy().view(gc.VB_LIST_DTYPE)
    pool = d_bytes.cpu().numpy()
    total = int(d_total.item())
    want_total = 0
    for i in range(len(lens)):
        want = O.vb_encode(g[off[i]:off[i + 1]])
        r = recs[i]
        assert int(r["n"]) == lens[i] and int(r["out_off"]) == int(off[i]) and int(r["nbytes"]) == len(want)
        assert (pool[int(r["byte_off"]):int(r["byte_off"]) + len(want)] == want).all(), i
        want_total += len(want)
    assert total == want_total
    for restore in (False, True):
        out = torch.full((len(g) + 1,), -1, dtype=torch.int32, device=dev)
        st = gc.new_status(dev)
        gc.gc_vb_decode_batch(d_lists, len(lens), d_bytes[:total], out, restore, st)
        gc.check_status(st, "vb decode")
        got = gc.as_u32(out)
        for i in range(len(lens)):
            seg = g[off[i]:off[i + 1]]
            want = O.prefix_sum(seg) if restore else seg
            assert (got[int(off[i]):int(off[i + 1])] == want).all(), (i, restore)


@pytest.mark.parametrize("kind", [O.SIMPLE, O.PFD])
def test_mixed_index_short_lists(gc, kind):
    """Clustered short lists (config 4's recipe at 60,000 lists): lists under
    64 as Variable Byte, the rest with a Group codec at k = 32."""
    maxlen = synth.lognormal_lengths(9, 60_000, 12.0, 1.5, 1 << 16)
    gaps, off, lens = synth.clustered_index(10, maxlen, 50_000_000, 16.0, 5000.0)
    dev = torch.device("cuda")
    d_gaps = torch.from_numpy(gaps.view(np.int32)).to(dev)
    codec = gc.make_codec(kind, 32, zeta=0.1)
    mi = gc.encode_mixed_index(codec, d_gaps, lens, vb_below=64)
    assert mi.n_short == int((lens < 64).sum()) > 0
    out = gc.as_u32(gc.decode_mixed(mi))
    for i in range(len(lens)):
        a, b = int(off[i]), int(off[i + 1])
        assert (out[a:b] == O.prefix_sum(gaps[a:b])).all(), i
    whole = gc.encode_index(codec, d_gaps, lens)
    assert mi.compressed_bytes() < whole.compressed_bytes()


def test_vb_corrupt_list_reported(gc):
    lens, g, off = short_lists(5, 50)
    dev = torch.device("cuda")
    mi = gc.encode_mixed_index(gc.make_codec(O.SIMPLE, 32), torch.from_numpy(g.view(np.int32)).to(dev), lens)
    b = mi.vb_bytes.clone()
    b[:] = b & 0x7F  # no number ends: every list runs out of bytes
    mi.vb_bytes = b
    with pytest.raises(gc.GcError) as ei:
        gc.decode_mixed(mi)
    assert ei.value.code == 3


def vb_case_lists(seed, long_lists):
    """Byte strings of Variable Byte lists (oracle encodings of lists of 0 to
    70 numbers, with one of 300 to 3000 in every 50 when long_lists, else of
    0 to 40) and a few written by hand: leading zero groups that still fit
    32 bits (accepted), a number wider than 32 bits, a last number that runs
    on, a byte left over, bytes of an empty list."""
    rng = np.random.default_rng(seed)
    lists = []
    for i in range(700):
        if long_lists:
            n = int(rng.integers(0, 70)) if i % 50 else int(rng.integers(300, 3000))
        else:
            n = int(rng.integers(0, 40))
        hi = [8, 15, 22, 32][i % 4]
        g = synth.width_mix(seed + i, n, 0, hi)
        lists.append((bytes(O.vb_encode(g)) if n else b"", n))
    five = bytes(O.vb_encode(np.array([5], np.uint32)))
    lists[3] = (bytes([0x00, 0x00, 0x85]) + five, 2)                 # leading zero groups: 5, 5
    lists[9] = (bytes([0x10, 0x00, 0x00, 0x00, 0x80]), 1)           # 2^32: too wide
    lists[10] = (bytes([0x0f, 0x7f, 0x7f, 0x7f, 0xff]), 1)          # 2^32 - 1: fits
    lists[11] = (bytes([0x00] * 40 + [0x81]), 1)                     # 40 zero groups, then 1
    lists[20] = (lists[20][0][:-1] + bytes([lists[20][0][-1] & 0x7F]) if lists[20][0] else b"\x01", lists[20][1] or 1)
    lists[33] = (lists[33][0] + b"\x81", lists[33][1])               # a byte left over
    lists[34] = (b"\x81", 0)                                         # bytes of an empty list
    return lists


def oracle_vb(b, n):
    try:
        return O.vb_decode(np.frombuffer(b, np.uint8), n)
    except O.OracleError:
        return None


@pytest.mark.parametrize("long_lists", [False, True], ids=["short", "long"])
@pytest.mark.parametrize("back_to_back", [True, False], ids=["back_to_back", "scattered"])
def test_vb_decode_malformed_lists_stay_inside(gc, back_to_back, long_lists):
    """Every list decodes as the oracle's one-list decoder does: a batch with
    malformed lists reports GC_ERR_CORRUPT and every well-formed list still
    decodes exactly; the well-formed lists alone decode with no error. Short
    lists back to back take the block's staged path; blocks holding long
    lists, the warp's stream path (the group of each long list) and the
    one-thread path (the others); lists in reverse byte order, the one-thread
    path."""
    lists = vb_case_lists(11, long_lists)
    want = [oracle_vb(b, n) for b, n in lists]
    assert want[3] is not None and want[10] is not None and want[11] is not None
    assert want[9] is None and want[20] is None and want[33] is None and want[34] is None
    dev = torch.device("cuda")

    def run(sel, restore):
        order = sel if back_to_back else sel[::-1]
        pool, boff = bytearray(), {}
        for i in order:
            boff[i] = len(pool)
            pool += lists[i][0]
        recs = np.zeros(len(sel), gc.VB_LIST_DTYPE)
        out_off = np.zeros(len(sel) + 1, np.uint64)
        np.cumsum([lists[i][1] for i in sel], out=out_off[1:])
        for r, i in enumerate(sel):
            recs[r] = (boff[i], out_off[r], lists[i][1], len(lists[i][0]))
        d_lists = torch.from_numpy(recs.view(np.uint8)).to(dev)
        d_bytes = torch.from_numpy(np.frombuffer(bytes(pool) or b"\0", np.uint8).copy()).to(dev)
        out = torch.full((int(out_off[-1]) + 1,), -1, dtype=torch.int32, device=dev)
        st = gc.new_status(dev)
        gc.gc_vb_decode_batch(d_lists, len(sel), d_bytes[:len(pool)], out, restore, st)
        code = int(st.cpu()[0])
        got = gc.as_u32(out)
        for r, i in enumerate(sel):
            if want[i] is not None:
                w = O.prefix_sum(want[i]) if restore else want[i]
                assert (got[int(out_off[r]):int(out_off[r + 1])] == w).all(), (i, restore)
        return code

    every = list(range(len(lists)))
    good = [i for i in every if want[i] is not None]
    for restore in (False, True):
        assert run(every, restore) == 3
        assert run(good, restore) == 0
