"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: numbers
printed in the paper (tests/golden/), brute-force enumeration on tiny
inputs, closed forms, library routines, and invariants of the tables.
"""
import itertools
import os
from fractions import Fraction

import math

import numpy as np
import pytest

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out.setdefault(key, []).append([int(v) for v in vals])
    return out


def ebits(x):
    return int(x).bit_length()


# ----------------------------------------------------------------- Table III

def test_table3_invariants():
    """Table III: NUM*BW fits a 32-bit component, NUM decreases and BW
    increases strictly with SEL, BW reaches 32, and each NUM is the most
    BW-bit ints a component holds."""
    num, bw = O.table3()
    assert list(num) == [32, 16, 10, 8, 6, 5, 4, 3, 2, 1]
    assert list(bw) == [1, 2, 3, 4, 5, 6, 8, 10, 16, 32]
    assert all(int(a) * int(b) <= 32 for a, b in zip(num, bw))
    assert all(num[i] > num[i + 1] and bw[i] < bw[i + 1] for i in range(9))
    assert bw[9] == 32
    assert all(int(a) == 32 // int(b) for a, b in zip(num, bw))


def test_effective_bits_matches_bit_length():
    xs = [0, 1, 2, 3, 255, 256, 2**31 - 1, 2**31, 2**32 - 1] + list(synth.width_mix(1, 2000))
    for x in xs:
        assert O.effective_bits(int(x)) == ebits(x)


# --------------------------------------------------------------- Group-Simple

def test_gs_worked_example_sec42():
    g = read_golden("gs_worked_example.txt")
    ints = np.array(g["ints"][0], np.uint32)
    k = g["k"][0][0]
    c = O.Codec(O.SIMPLE, k)
    sel = O.gs_select(O.rowmax(ints, k))
    assert list(sel) == g["selectors"][0]
    ctrl, data = O.encode(c, ints)
    assert len(data) == g["vectors"][0][0] * k
    assert (O.decode(c, ctrl, data, len(ints)) == ints).all()
    ints64 = np.array(g["ints_with_64"][0], np.uint32)
    sel64 = O.gs_select(O.rowmax(ints64, k))
    assert sel64[0] == g["first_selector_with_64"][0][0]


def _valid_sequences(maxarr):
    """Every selector sequence that encodes maxarr: each selector takes
    min(NUM, rows left) rows and all of them fit in BW bits."""
    num, bw = O.table3()
    L = len(maxarr)

    def rec(j):
        if j == L:
            yield ()
            return
        for s in range(10):
            take = min(int(num[s]), L - j)
            if all(int(m) < (1 << int(bw[s])) for m in maxarr[j:j + take]):
                for rest in rec(j + take):
                    yield (s,) + rest

    return list(rec(0))


@pytest.mark.parametrize("seed", range(40))
def test_gs_algorithm1_is_lexicographically_first(seed):
    """Algorithm 1 tries SEL in ascending order and takes the first that
    fits; since any suffix can always be finished (SEL 9 fits anything), its
    output is the lexicographically smallest valid sequence. Brute force
    over every valid sequence on tiny inputs; every valid sequence must also
    decode back to the input."""
    rng = np.random.default_rng(seed)
    L = int(rng.integers(1, 7))
    widths = rng.integers(0, 7, size=L)
    widths[rng.random(L) < 0.15] = rng.integers(7, 33)
    maxarr = np.array([int(rng.integers(0, 1 << int(w))) if w else 0 for w in widths], np.uint32)
    # build a k = 4 list whose row maxima are exactly maxarr
    k = 4
    g = np.zeros(L * k, np.uint32)
    for r, m in enumerate(maxarr):
        g[r * k + int(rng.integers(0, k))] = m
        for j in range(k):
            if g[r * k + j] == 0 and m:
                g[r * k + j] = int(rng.integers(0, int(m) + 1))
    assert (O.rowmax(g, k) == maxarr).all()
    seqs = _valid_sequences(maxarr)
    assert seqs, "SEL 9 alone always encodes"
    greedy = tuple(int(s) for s in O.gs_select(maxarr))
    assert greedy == min(seqs)
    c = O.Codec(O.SIMPLE, k)
    for s in seqs[:64]:
        ctrl, data = O.gs_pack(g, k, np.array(s, np.uint8))
        assert (O.decode(c, ctrl, data, len(g)) == g).all()


def test_gs_pack_rejects_selector_that_does_not_fit():
    g = np.array([5, 0, 0, 0], np.uint32)
    with pytest.raises(O.OracleError):
        O.gs_pack(g, 4, np.array([1], np.uint8))  # BW 2 cannot hold 5


def test_gs_pseudo_quad_max_gives_same_selectors():
    """Section 4.4: OR of the quadruple has the effective width of its max,
    so Algorithm 1 (which only compares with 2^BW - 1) picks the same
    selectors."""
    for seed in range(10):
        g = synth.width_mix(seed, 4 * 500, 0, 32)
        true_max = O.rowmax(g, 4)
        pseudo = np.bitwise_or.reduce(g.reshape(-1, 4), axis=1).astype(np.uint32)
        assert (np.array([ebits(x) for x in pseudo]) == np.array([ebits(x) for x in true_max])).all()
        assert (O.gs_select(pseudo) == O.gs_select(true_max)).all()


def test_gs_layout_bits():
    """Row q of a selector sits at bits [q*BW, (q+1)*BW) of each component,
    component j of vector s is data word s*k + j, selector s is nibble s."""
    k = 4
    g = np.arange(1, 4 * 10 + 1, dtype=np.uint32) % 7  # widths <= 3 bits
    c = O.Codec(O.SIMPLE, k)
    ctrl, data = O.encode(c, g)
    sel = O.gs_select(O.rowmax(g, k))
    num, bw = O.table3()
    row = 0
    for s, sv in enumerate(sel):
        assert (ctrl[s // 2] >> (4 * (s % 2))) & 15 == sv
        for q in range(min(int(num[sv]), 10 - row)):
            for j in range(k):
                w = int(data[s * k + j])
                assert (w >> (q * int(bw[sv]))) & ((1 << int(bw[sv])) - 1) == g[(row + q) * k + j]
        row += int(num[sv])


# --------------------------------------------------------------- Group-Scheme

@pytest.mark.parametrize("cg", [1, 2, 4, 8])
def test_gsc_eq1_eq2_minimal_width(cg):
    """Eq. 1 then Eq. 2 give the smallest multiple of CG that holds the row
    max (a zero row still takes one unit, Table IV's unary range starts at 1)."""
    xs = [0, 1] + [v for b in range(1, 33) for v in ((1 << b) - 1, min((1 << b), 2**32 - 1))]
    xs += list(synth.width_mix(cg, 3000))
    for x in xs:
        u = O.gsc_units(int(x), cg)
        bwidth = cg * u
        need = max(1, ebits(x))
        assert bwidth >= need and bwidth - cg < need
        assert 1 <= u <= 32 // cg


def test_gsc_ld_example_sec51():
    g = read_golden("gsc_examples.txt")
    x, cg, units = g["ld_value"][0][0], g["ld_cg"][0][0], g["ld_units"][0][0]
    assert O.gsc_units(x, cg) == units
    # unary: the descriptor bits are the first bits of the control stream
    c = O.Codec(O.SCHEME, 4, cg=cg, ld=O.LD_CU)
    ctrl, data = O.encode(c, np.array([x, 0, 0, 0], np.uint32))
    bits = [(int(ctrl[0]) >> t) & 1 for t in range(units)]
    assert bits == g["ld_unary_bits"][0]
    # binary: Eq. 1 stores units - 1 in 5 - log2(CG) bits
    c = O.Codec(O.SCHEME, 4, cg=cg, ld=O.LD_BINARY)
    ctrl, data = O.encode(c, np.array([x, 0, 0, 0], np.uint32))
    assert int(ctrl[0]) & 0xF == units - 1


def test_gsc_cu_lut_example_sec531():
    g = read_golden("gsc_examples.txt")
    bits = g["cu_byte_bits"][0]
    byte = sum(b << t for t, b in enumerate(bits))
    # The dangling ones continue into the next byte, whose first bit (0) closes them.
    units, _ = O.gsc_parse(np.array([byte, 0x00], np.uint8), 1, O.LD_CU, 4)
    want = g["cu_descriptors"][0]
    assert list(units[:3]) == want
    assert units[3] == g["cu_dangling_ones"][0][0] + 1


def test_gsc_table4_widths_and_ranges():
    g = read_golden("gsc_examples.txt")
    for cg, nb, umax in zip(g["table4_cg"][0], g["table4_binary_bits"][0], g["table4_unary_max"][0]):
        assert O.gsc_units(2**32 - 1, cg) == umax
        # the largest binary value (umax - 1) needs exactly nb bits
        assert ebits(umax - 1) == nb


def test_gsc_ints_per_pattern_sequence():
    """Binary descriptors at k = 4: 12 ints per 16 bits (CG 1), 8 per byte
    (CG 2 and 4), 16 per byte (CG 8)."""
    g = read_golden("gsc_examples.txt")
    for cg, ints, bits in g["ints_per_pattern_bits"]:
        rows = ints // 4
        c = O.Codec(O.SCHEME, 4, cg=cg, ld=O.LD_BINARY)
        x = synth.width_mix(cg, 4 * rows * 50, 0, 32)
        ctrl, _ = O.encode(c, x)
        assert len(ctrl) * 8 == 50 * bits


def test_gsc_iu_packing_rule():
    """IU keeps each descriptor inside one byte and pads the rest with ones
    (Section 5.2.1(a)); CU lets it run on."""
    cg = 8
    rows_units = [3, 3, 2, 4, 1]
    vals = [(1 << (cg * u - 1)) for u in rows_units]
    g = np.array([v for v in vals for _ in range(4)], np.uint32)
    ctrl, _ = O.encode(O.Codec(O.SCHEME, 4, cg=cg, ld=O.LD_IU), g)
    bits = [(int(ctrl[t // 8]) >> (t % 8)) & 1 for t in range(8 * len(ctrl))]
    # byte 0: 110 110 10 ; byte 1: 1110 0 then padding 111
    assert bits[:8] == [1, 1, 0, 1, 1, 0, 1, 0]
    assert bits[8:16] == [1, 1, 1, 0, 0, 1, 1, 1]
    ctrl, _ = O.encode(O.Codec(O.SCHEME, 4, cg=cg, ld=O.LD_CU), g)
    bits = [(int(ctrl[t // 8]) >> (t % 8)) & 1 for t in range(8 * len(ctrl))]
    assert bits[:13] == [1, 1, 0, 1, 1, 0, 1, 0, 1, 1, 1, 0, 0]
    # IU with a descriptor that must move to the next byte
    rows_units = [4, 4, 4]
    vals = [(1 << (cg * u - 1)) for u in rows_units]
    g = np.array([v for v in vals for _ in range(4)], np.uint32)
    ctrl, _ = O.encode(O.Codec(O.SCHEME, 4, cg=cg, ld=O.LD_IU), g)
    assert list(ctrl) == [0b01110111, 0b11110111]


def test_gsc_1cu_k4_is_k_gamma_sized():
    """Section 5.1: with 1-bit granularity and complete unary descriptors at
    k = 4, Group-Scheme is k-Gamma: per quadruple, the width b in unary and
    four b-bit values."""
    for seed in range(5):
        g = synth.width_mix(seed, 4 * 300, 0, 32)
        c = O.Codec(O.SCHEME, 4, cg=1, ld=O.LD_CU)
        ctrl, data = O.encode(c, g)
        b = [max(1, ebits(max(g[4 * r:4 * r + 4]))) for r in range(300)]
        assert len(ctrl) == (sum(b) + 7) // 8
        assert len(data) == 4 * ((sum(b) + 31) // 32)


# ----------------------------------------------------------------- Group-AFOR

def _afor_cost(maxarr, k, parts):
    cost, row = 0, 0
    for F in parts:
        b = max((ebits(maxarr[r]) if r < len(maxarr) else 0) for r in range(row, row + F))
        cost += 8 + k * F * b
        row += F
    return cost


def _compositions(nblocks):
    if nblocks == 0:
        yield ()
        return
    for F in (8, 16, 32):
        if F // 8 <= nblocks:
            for rest in _compositions(nblocks - F // 8):
                yield (F,) + rest


@pytest.mark.parametrize("seed", range(30))
def test_afor_partition_is_optimal_by_enumeration(seed):
    """Section 6.1: the partition minimises 8 + k*F*b bits per frame. Check
    against every partition of <= 48 rows; among optimal partitions the
    oracle takes, at each frame, the largest size (lexicographically largest
    sequence)."""
    rng = np.random.default_rng(100 + seed)
    R = int(rng.integers(1, 49))
    k = [4, 32][seed % 2]
    widths = rng.integers(0, 12, size=R)
    widths[rng.random(R) < 0.2] = rng.integers(12, 33)
    maxarr = np.array([int(rng.integers(1 << (w - 1), 1 << w)) if w else 0 for w in widths],
                      np.uint64).astype(np.uint32)
    nb = (R + 7) // 8
    best = None
    for parts in _compositions(nb):
        c = _afor_cost(maxarr, k, parts)
        if best is None or c < best[0] or (c == best[0] and parts > best[1]):
            best = (c, parts)
    got = tuple(int(x) for x in O.afor_partition(maxarr, k))
    assert _afor_cost(maxarr, k, got) == best[0]
    assert got == best[1]


def test_afor_control_byte_layout():
    k = 4
    g = np.concatenate([np.full(8 * 4, 3, np.uint32), np.full(32 * 4, 1000, np.uint32)])
    c = O.Codec(O.AFOR, k)
    ctrl, data = O.encode(c, g)
    frames = [(8 << (int(x) >> 6), int(x) & 63) for x in ctrl]
    assert sum(F for F, _ in frames) == 40
    for F, b in frames:
        assert b in (2, 10)


# ------------------------------------------------------------------ Group-PFD

@pytest.mark.parametrize("zeta", [0.01, 0.05, 0.1, 0.125, 0.2, 0.3, 0.5, 0.99])
def test_pfd_rows_for_zeta_is_strictly_below(zeta):
    """Section 6.2 Step 2: the exception ratio must stay below zeta; the most
    exception rows c out of 32 with c/32 < zeta."""
    c = O.pfd_rows_for_zeta(zeta)
    z = Fraction(zeta).limit_denominator(10**9)
    assert Fraction(c, 32) < z
    assert c == 31 or Fraction(c + 1, 32) >= z


def _pfd_headers(ctrl, nf):
    h = ctrl[:4 * nf].view("<u4") if nf else np.zeros(0, np.uint32)
    return [(int(x) & 63, (int(x) >> 6) & 3, int(x) >> 8) for x in h]


@pytest.mark.parametrize("k,zeta,seed", [(4, 0.1, 0), (4, 0.3, 1), (4, 0.01, 2), (32, 0.1, 3),
                                         (32, 0.3, 4), (4, 0.1, 5)])
@pytest.mark.parametrize("tail_rows", [1, 5, 21, 31])
def test_pfd_b_minimal_and_exceptions(k, zeta, seed, tail_rows):
    """Section 6.2 Step 2: b is the minimum width whose exception rows keep
    the frame's exception ratio below zeta (b - 1 would break it). A whole
    frame's budget is the most rows c with c / 32 < zeta; a list's last frame
    of r < 32 rows has that budget times r / 32, rounded down (so its own
    ratio stays below zeta). Exceptions are exactly the ints above 2^b - 1;
    the exception width is the smallest of 8, 16, 32 bits that holds them."""
    n = 32 * k * 6 + (tail_rows - 1) * k + 3
    g = synth.mixed_runs(seed, n, 64, 8.0, 0.15, 1 << 20)
    c = O.Codec(O.PFD, k, zeta=zeta)
    ctrl, data = O.encode(c, g)
    R = (n + k - 1) // k
    assert R % 32 == tail_rows
    nf = (R + 31) // 32
    mx = O.rowmax(g, k)
    z = Fraction(zeta).limit_denominator(10**9)
    c32 = max(0, min(31, math.ceil(z * 32) - 1))  # the most rows c with c / 32 < zeta
    assert Fraction(c32, 32) < z and (c32 == 31 or not Fraction(c32 + 1, 32) < z)
    for f, (b, wcode, e) in enumerate(_pfd_headers(ctrl, nf)):
        fm = mx[32 * f:32 * f + 32]
        budget = c32 * len(fm) // 32
        cnt = lambda bb: sum(1 for m in fm if int(m) >= (1 << bb))
        assert cnt(b) <= budget and Fraction(cnt(b), len(fm)) < z
        assert b == 0 or cnt(b - 1) > budget
        vals = [int(v) for v in g[32 * k * f:32 * k * (f + 1)] if int(v) >= (1 << b)]
        assert e == len(vals)
        if e:
            w = 8 if max(vals) < 256 else 16 if max(vals) < 65536 else 32
            assert (1 << wcode) * 8 == w
    assert (O.decode(c, ctrl, data, n) == g).all()


def test_pfd_zero_ratio_is_bp128():
    """Section 6.3: with no exception rows allowed, Group-PFD at k = 4 is
    SIMD-BP128: 128-int frames packed at the width of the frame's maximum in
    the 4-way vertical layout. Compare with a numpy packer written from
    that definition."""
    k = 4
    g = synth.width_mix(7, 128 * 9, 0, 20)
    c = O.Codec(O.PFD, k, max_exc_rows=0)
    ctrl, data = O.encode(c, g)
    words = []
    for f in range(9):
        fr = g[128 * f:128 * (f + 1)].astype(np.uint64)
        b = ebits(int(fr.max()))
        lanes = fr.reshape(32, 4).T  # lane j holds ints 4r + j
        for j in range(4):
            acc = 0
            for r in range(32):
                acc |= int(lanes[j, r]) << (r * b)
            lane_words = [(acc >> (32 * w)) & 0xFFFFFFFF for w in range(b)]
            words.append(lane_words)
        # interleave: vector w holds word w of lanes 0..3
        block = np.array(words[-4:], np.uint64).T.reshape(-1) if b else np.zeros(0)
        words[-4:] = [list(block)]
    ref = np.array([x for blk in words for x in blk], np.uint32)
    assert (data == ref).all()
    hdr = _pfd_headers(ctrl, 9)
    assert all(e == 0 for _, _, e in hdr)


# ------------------------------------------------------------ common checks

CODECS = ([O.Codec(O.SIMPLE, k) for k in (4, 32)]
          + [O.Codec(O.SCHEME, k, cg, ld) for k in (4, 32)
             for cg, ld in [(1, 0), (2, 0), (4, 0), (8, 0), (1, 1), (2, 1), (4, 1), (8, 1),
                            (4, 2), (8, 2)]]
          + [O.Codec(O.AFOR, k) for k in (4, 32)]
          + [O.Codec(O.PFD, k, zeta=z) for k in (4, 32) for z in (0.0, 0.01, 0.1, 0.3)])


@pytest.mark.parametrize("codec", CODECS, ids=repr)
def test_round_trip(codec):
    rng = np.random.default_rng(codec.kind * 100 + codec.k + codec.cg + 7 * codec.ld)
    lens = [0, 1, 2, 3, 4, 5, 31, 32, 33, 127, 128, 129, 1023, 1024, 1025, 2000]
    lens += list(rng.integers(0, 3000, size=6))
    for i, n in enumerate(lens):
        hi = [32, 12, 6, 1][i % 4]
        g = synth.width_mix(1000 + i, int(n), 0, hi)
        ctrl, data = O.encode(codec, g)
        assert (O.decode(codec, ctrl, data, int(n)) == g).all()
        cc, dc = O.max_sizes(codec, int(n))
        assert len(ctrl) <= cc and len(data) <= dc


def test_prefix_sum_matches_cumsum_mod_2_32():
    g = synth.width_mix(3, 100000, 0, 32)
    ref = (np.cumsum(g.astype(np.uint64)) & 0xFFFFFFFF).astype(np.uint32)
    assert (O.prefix_sum(g) == ref).all()
    d = np.sort(synth.uniform_u32(4, 5000, 0, 10**6))
    assert (O.prefix_sum(O.dgaps(d)) == d).all()
    assert (O.dgaps(d)[0] == d[0])


def test_decode_rejects_corrupt_streams():
    g = synth.width_mix(9, 4000, 0, 10)
    c = O.Codec(O.SIMPLE, 4)
    ctrl, data = O.encode(c, g)
    bad = ctrl.copy()
    bad[0] = 0xFF  # selector 15 does not exist
    with pytest.raises(O.OracleError):
        O.decode(c, bad, data, 4000)
    with pytest.raises(O.OracleError):
        O.decode(c, ctrl, data[:len(data) // 2], 4000)


def test_paper_buffer_layout():
    g = synth.width_mix(11, 999, 0, 9)
    ctrl, data = O.encode(O.Codec(O.SIMPLE, 4), g)
    buf = O.paper_pack(ctrl, data)
    off = int(buf[:4].view("<u4")[0]) * 4
    assert off % 16 == 0 and off >= 4 + len(ctrl) and off - (4 + len(ctrl)) < 16
    assert (buf[4:4 + len(ctrl)] == ctrl).all()
    assert (buf[off:].view("<u4") == data).all()


# ------------------------------------------------------------- tile index

@pytest.mark.parametrize("codec", CODECS, ids=repr)
def test_tile_index_consistent_with_units(codec):
    """Each 1024-int tile record points at the unit that holds its first row;
    re-derived here from the unit sizes that the control area gives."""
    k = codec.k
    n = 1024 * 7 + 300
    g = synth.mixed_runs(5, n, 128, 6.0, 0.2, 1 << 18)
    ctrl, data = O.encode(codec, g)
    tiles = O.tile_index(codec, ctrl, n)
    R = (n + k - 1) // k
    tr = 1024 // k
    assert len(tiles) == (R + tr - 1) // tr
    # unit list: (rows, lane bits, ctrl start bit, exc bytes)
    units = []
    if codec.kind == O.SIMPLE:
        num, _ = O.table3()
        for s in range(2 * len(ctrl)):
            units.append((int(num[(int(ctrl[s // 2]) >> (4 * (s % 2))) & 15]), 32, 4 * s, 0))
    elif codec.kind == O.SCHEME:
        u, _ = O.gsc_parse(ctrl, codec.cg, codec.ld, R)
        cpos = []
        if codec.ld == O.LD_BINARY:
            per = {1: 3, 2: 2, 4: 2, 8: 4}[codec.cg]
            unit = 16 if codec.cg == 1 else 8
            w = 5 - {1: 0, 2: 1, 4: 2, 8: 3}[codec.cg]
            cpos = [(r // per) * unit + (r % per) * w for r in range(R)]
        else:
            p = 0
            for x in u:
                if codec.ld == O.LD_IU and p % 8 + int(x) > 8:
                    p = (p // 8 + 1) * 8
                cpos.append(p)
                p += int(x)
        units = [(1, codec.cg * int(x), cpos[r], 0) for r, x in enumerate(u)]
    elif codec.kind == O.AFOR:
        units = [(8 << (int(x) >> 6), (8 << (int(x) >> 6)) * (int(x) & 63), 8 * f, 0)
                 for f, x in enumerate(ctrl)]
    else:
        nf = (R + 31) // 32
        pb = 1 if 32 * k <= 256 else 2
        units = [(32, 32 * b, 32 * f, e * (pb + (1 << w))) for f, (b, w, e) in
                 enumerate(_pfd_headers(ctrl, nf))]
    row = lane = xoff = 0
    t = 0
    for rows, lb, cpos, xb in units:
        while t < len(tiles) and t * tr < row + rows:
            assert tiles[t]["lane_bit"] == lane
            assert tiles[t]["ctrl_bit"] == cpos
            assert tiles[t]["row_skip"] == t * tr - row
            assert tiles[t]["exc_off"] == xoff
            t += 1
        row += rows
        lane += lb
        xoff += xb
        if t == len(tiles):
            break
    assert t == len(tiles)


@pytest.mark.parametrize("k", [4, 32])
def test_tile_skip_entries_are_prefix_sums(k):
    """Sections 2.1.1 and 7.5: the skip entry of tile t is the docID just
    before it, the running sum of the gaps modulo 2^32 at int 1024*t - 1
    (numpy's cumulative sum in 64 bits, reduced), 0 for tile 0; the control
    area alone gives no entry but tile 0's."""
    codec = O.Codec(O.PFD, k)
    n = 1024 * 9 + 17
    g = synth.uniform_u32(3, n, 1 << 20, 1 << 30)  # sums pass 2^32: the wrap is exercised
    ctrl, _ = O.encode(codec, g)
    plain = O.tile_index(codec, ctrl, n)
    skip = O.tile_index(codec, ctrl, n, g)
    cum = np.cumsum(g.astype(np.uint64)) & 0xFFFFFFFF
    want = [0] + [int(cum[1024 * t - 1]) for t in range(1, len(skip))]
    assert [int(x) for x in skip["base"]] == want
    assert (skip["flags"] == 1).all()
    assert int(plain["flags"][0]) == 1 and not plain["flags"][1:].any() and not plain["base"].any()
    for f in ("lane_bit", "ctrl_bit", "exc_off", "row_skip"):
        assert (plain[f] == skip[f]).all()
    # a tile decoded on its own, plus its entry, gives the list's docIDs there
    ids = O.prefix_sum(g)
    for t in range(len(skip)):
        seg = g[1024 * t:1024 * (t + 1)]
        local = np.cumsum(seg.astype(np.uint64)) + int(skip["base"][t])
        assert (local.astype(np.uint64) & 0xFFFFFFFF == ids[1024 * t:1024 * t + len(seg)]).all()


# ------------------------------------------------------------- generators

def test_xoshiro_matches_published_definition():
    """The input generator: xoshiro256** seeded by splitmix64 (definitions
    by Blackman and Vigna), re-implemented here in Python."""
    M = (1 << 64) - 1

    def splitmix(s):
        s = (s + 0x9E3779B97F4A7C15) & M
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return s, z ^ (z >> 31)

    rotl = lambda x, r: ((x << r) | (x >> (64 - r))) & M
    seed = 12345
    st = []
    s = seed
    for _ in range(4):
        s, z = splitmix(s)
        st.append(z)
    want = []
    for _ in range(8):
        want.append((rotl((st[1] * 5) & M, 7) * 9) & M)
        t = (st[1] << 17) & M
        st[2] ^= st[0]
        st[3] ^= st[1]
        st[1] ^= st[2]
        st[0] ^= st[3]
        st[2] ^= t
        st[3] = rotl(st[3], 45)
    assert [int(x) for x in synth.raw_u64(seed, 8)] == want


def test_generators_shapes():
    g = synth.single_list_geometric(65536, 20.0, 0)
    assert len(g) == 65536 and g.min() >= 1 and 15 < g.mean() < 25
    lens = synth.zipf_lengths(0, 1000, 1e5, 1.1, 1 << 22)
    assert lens.min() >= 1 and lens.max() <= 1 << 22
    gaps, off, L = synth.clustered_index(1, synth.lognormal_lengths(0, 500), 50_000_000)
    docs = np.concatenate([O.prefix_sum(gaps[off[i]:off[i + 1]]) for i in range(500)])
    assert len(docs) == int(L.sum())
    for i in range(500):
        d = O.prefix_sum(gaps[off[i]:off[i + 1]])
        assert (np.diff(d.astype(np.int64)) > 0).all() and (len(d) == 0 or d[-1] < 50_000_000)


# ---------------------------------------------------------- Variable Byte

def test_vb_hand_worked_encodings():
    """Section 2.3, values worked by hand: 7-bit groups most significant
    first, the high bit set on the last byte."""
    cases = {
        0: [0x80],
        1: [0x81],
        127: [0xFF],
        128: [0x01, 0x80],
        300: [0x02, 0xAC],
        16383: [0x7F, 0xFF],
        16384: [0x01, 0x00, 0x80],
        2**21: [0x01, 0x00, 0x00, 0x80],
        2**28: [0x01, 0x00, 0x00, 0x00, 0x80],
        2**32 - 1: [0x0F, 0x7F, 0x7F, 0x7F, 0xFF],
    }
    for x, want in cases.items():
        assert list(O.vb_encode([x])) == want, x
        assert O.vb_size(x) == len(want)
        assert O.vb_decode(np.array(want, np.uint8), 1)[0] == x


def test_vb_stream_properties():
    """Every number has exactly one byte with the high bit set, its last;
    a number takes ceil(bits / 7) bytes (at least one); decoding restores
    the sequence."""
    g = synth.width_mix(5, 5000, 0, 32)
    b = O.vb_encode(g)
    last = (b & 0x80) != 0
    assert last.sum() == len(g) and last[-1]
    sizes = np.diff(np.concatenate(([-1], np.flatnonzero(last))))
    want = np.maximum(1, -(-np.array([int(x).bit_length() for x in g]) // 7))
    assert (sizes == want).all()
    assert (O.vb_decode(b, len(g)) == g).all()


def test_vb_rejects_malformed_streams():
    """Bytes that end inside a number, numbers wider than 32 bits and
    left-over bytes are reported."""
    b = O.vb_encode([5, 300])
    with pytest.raises(O.OracleError):
        O.vb_decode(b[:-1], 2)
    with pytest.raises(O.OracleError):
        O.vb_decode(np.array([0x10, 0x00, 0x00, 0x00, 0x80], np.uint8), 1)
    with pytest.raises(O.OracleError):
        O.vb_decode(np.concatenate((b, [0x81])).astype(np.uint8), 2)
