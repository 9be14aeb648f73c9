"""CPU oracle for the Group codecs of arXiv 1502.01916 (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It wraps ``gc_oracle.c``, a plain
single-threaded C implementation written from the paper's definitions
(Sections 2.1, 4, 5 and 6), compiled with gcc. It shares no code with the
CUDA library.

Every oracle function here is pinned by ``tests/test_oracle_*.py`` against
facts that the paper or the mathematics fix (Table III, Algorithm 1 by
brute force, Eq. 1/2 bounds, the worked examples of Sections 4.2, 5.1 and
5.3.1, exhaustive partitions for AFOR, minimality of the PFD width, Variable
Byte's encodings worked by hand).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gc_oracle.c")
_SO = os.path.join(_HERE, "_build", "libgc_oracle.so")
_lib = None
_lock = threading.Lock()

SIMPLE, SCHEME, AFOR, PFD = 0, 1, 2, 3
LD_BINARY, LD_CU, LD_IU = 0, 1, 2
OK, ERR_INVALID, ERR_NOSPACE, ERR_CORRUPT = 0, 1, 2, 3

TILE_DTYPE = np.dtype([("lane_bit", "<u8"), ("ctrl_bit", "<u8"), ("exc_off", "<u4"),
                       ("row_skip", "<u4"), ("base", "<u4"), ("flags", "<u4")])

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_U32, _U64 = ctypes.c_uint32, ctypes.c_uint64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no SIMD flags)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_effective_bits.argtypes = [_U32]
            lib.orc_effective_bits.restype = _U32
            lib.orc_table3.argtypes = [_u32p, _u32p]
            lib.orc_rowmax.argtypes = [_u32p, _U64, _U32, _u32p]
            lib.orc_prefix_sum.argtypes = [_u32p, _U64, _u32p]
            lib.orc_dgaps.argtypes = [_u32p, _U64, _u32p]
            lib.orc_gs_select.argtypes = [_u32p, _U64, _u8p]
            lib.orc_gs_select.restype = _U64
            lib.orc_gs_pack.argtypes = [_u32p, _U64, _U32, _u8p, _U64, _u8p, _u64p, _u32p, _u64p]
            lib.orc_gsc_units.argtypes = [_U32, _U32]
            lib.orc_gsc_units.restype = _U32
            lib.orc_gsc_parse.argtypes = [_u8p, _U64, _U32, _U32, _U64, _u32p]
            lib.orc_gsc_parse.restype = _U64
            lib.orc_afor_partition.argtypes = [_u32p, _U64, _U32, _u32p]
            lib.orc_afor_partition.restype = _U64
            lib.orc_pfd_rows_for_zeta.argtypes = [ctypes.c_double]
            lib.orc_pfd_rows_for_zeta.restype = _U32
            lib.orc_pfd_frame_b.argtypes = [_u32p, _U64, _U32]
            lib.orc_pfd_frame_b.restype = _U32
            lib.orc_max_sizes.argtypes = [_U32, _U32, _U32, _U32, _U32, _U64, _u64p, _u64p]
            lib.orc_encode.argtypes = [_U32, _U32, _U32, _U32, _U32, _u32p, _U64, _u8p, _U64, _u64p,
                                       _u32p, _U64, _u64p]
            lib.orc_decode.argtypes = [_U32, _U32, _U32, _U32, _u8p, _U64, _u32p, _U64, _U64, _u32p]
            lib.orc_paper_pack.argtypes = [_u8p, _U64, _u32p, _U64, _u8p]
            lib.orc_paper_pack.restype = _U64
            lib.orc_tile_count.argtypes = [_U64, _U32]
            lib.orc_tile_count.restype = _U64
            lib.orc_tile_index.argtypes = [_U32, _U32, _U32, _U32, _u8p, _U64, _U64, ctypes.c_void_p]
            lib.orc_tile_bases.argtypes = [_u32p, _U64, _U32, ctypes.c_void_p]
            lib.orc_tile_bases.restype = None
            lib.orc_vb_size.argtypes = [_U32]
            lib.orc_vb_size.restype = _U32
            lib.orc_vb_encode.argtypes = [_u32p, _U64, _u8p, _U64]
            lib.orc_vb_encode.restype = _U64
            lib.orc_vb_decode.argtypes = [_u8p, _U64, _U64, _u32p]
            _lib = lib
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


# --------------------------------------------------------------- primitives

def table3():
    """Table III as two arrays (NUM, BW), indexed by SEL."""
    num = np.zeros(10, np.uint32)
    bw = np.zeros(10, np.uint32)
    _load().orc_table3(_p(num, _u32p), _p(bw, _u32p))
    return num, bw


def effective_bits(x: int) -> int:
    return int(_load().orc_effective_bits(int(x)))


def rowmax(gaps, k: int) -> np.ndarray:
    g = _u32(gaps)
    R = (len(g) + k - 1) // k
    out = np.zeros(R, np.uint32)
    if R:
        _load().orc_rowmax(_p(g, _u32p), len(g), k, _p(out, _u32p))
    return out


def prefix_sum(gaps) -> np.ndarray:
    """docIDs from d-gaps (Section 2.1.1), modulo 2^32."""
    g = _u32(gaps)
    out = np.zeros(len(g), np.uint32)
    if len(g):
        _load().orc_prefix_sum(_p(g, _u32p), len(g), _p(out, _u32p))
    return out


def dgaps(docids) -> np.ndarray:
    d = _u32(docids)
    out = np.zeros(len(d), np.uint32)
    if len(d):
        _load().orc_dgaps(_p(d, _u32p), len(d), _p(out, _u32p))
    return out


def gs_select(maxarr) -> np.ndarray:
    """Algorithm 1 on a row (quad) max array: the selector sequence."""
    m = _u32(maxarr)
    sel = np.zeros(max(1, len(m)), np.uint8)
    S = _load().orc_gs_select(_p(m, _u32p), len(m), _p(sel, _u8p))
    return sel[:S].copy()


def gs_pack(gaps, k: int, sel):
    """Pack with a given selector sequence; returns (ctrl, data) or raises."""
    g = _u32(gaps)
    s = np.ascontiguousarray(sel, dtype=np.uint8)
    S = len(s)
    ctrl = np.zeros(max(1, (S + 1) // 2), np.uint8)
    data = np.zeros(max(1, S * k), np.uint32)
    cb, dw = ctypes.c_uint64(), ctypes.c_uint64()
    st = _load().orc_gs_pack(_p(g, _u32p), len(g), k, _p(s, _u8p), S, _p(ctrl, _u8p),
                             ctypes.byref(cb), _p(data, _u32p), ctypes.byref(dw))
    if st:
        raise OracleError(st, "gs_pack")
    return ctrl[:cb.value].copy(), data[:dw.value].copy()


def gsc_units(x: int, cg: int) -> int:
    """Eq. 1 unit count (unary descriptor value) for a row max x."""
    return int(_load().orc_gsc_units(int(x), cg))


def gsc_parse(ctrl, cg: int, ld: int, rows: int):
    """Read `rows` Group-Scheme descriptors; returns (units array, bits consumed)."""
    c = np.ascontiguousarray(ctrl, dtype=np.uint8)
    units = np.zeros(max(1, rows), np.uint32)
    used = _load().orc_gsc_parse(_p(c, _u8p), len(c), cg, ld, rows, _p(units, _u32p))
    if used == (1 << 64) - 1:
        raise OracleError(ERR_CORRUPT, "gsc_parse")
    return units[:rows].copy(), int(used)


def afor_partition(maxarr, k: int) -> np.ndarray:
    m = _u32(maxarr)
    R = len(m)
    out = np.zeros(max(1, (R + 7) // 8 + 1), np.uint32)
    nf = _load().orc_afor_partition(_p(m, _u32p), R, k, _p(out, _u32p))
    return out[:nf].copy()


def pfd_rows_for_zeta(zeta: float) -> int:
    """The ratio rule of Section 6.2 as an integer: the most exception rows
    (out of a frame's 32) whose ratio stays strictly below zeta. A list's
    last frame of r < 32 rows may have this many times r / 32, rounded down."""
    return int(_load().orc_pfd_rows_for_zeta(float(zeta)))


def pfd_frame_b(rowmax_frame, max_rows: int) -> int:
    m = _u32(rowmax_frame)
    return int(_load().orc_pfd_frame_b(_p(m, _u32p), len(m), max_rows))


# ---------------------------------------------------------------- codecs

class Codec:
    """Codec parameters: kind, k, Group-Scheme (cg, ld), Group-PFD exception
    rows per 32-row frame (from zeta)."""

    def __init__(self, kind: int, k: int = 4, cg: int = 8, ld: int = LD_BINARY,
                 zeta: float = 0.10, max_exc_rows: int | None = None):
        self.kind, self.k, self.cg, self.ld = kind, k, cg, ld
        self.max_exc_rows = pfd_rows_for_zeta(zeta) if max_exc_rows is None else max_exc_rows

    def args(self):
        return (self.kind, self.k, self.cg, self.ld, self.max_exc_rows)

    def __repr__(self):
        names = {SIMPLE: "GS", SCHEME: f"GSC-{self.cg}-{['B', 'CU', 'IU'][self.ld]}", AFOR: "AFOR",
                 PFD: f"PFD(x{self.max_exc_rows})"}
        return f"{names[self.kind]}/k{self.k}"


def max_sizes(codec: Codec, n: int):
    cc, dc = ctypes.c_uint64(), ctypes.c_uint64()
    st = _load().orc_max_sizes(*codec.args(), n, ctypes.byref(cc), ctypes.byref(dc))
    if st:
        raise OracleError(st, "max_sizes")
    return cc.value, dc.value


def encode(codec: Codec, gaps):
    """Encode a d-gap (or any uint32) sequence: returns (ctrl uint8, data uint32)."""
    g = _u32(gaps)
    cc, dc = max_sizes(codec, len(g))
    ctrl = np.zeros(max(1, cc), np.uint8)
    data = np.zeros(max(1, dc), np.uint32)
    cb, dw = ctypes.c_uint64(), ctypes.c_uint64()
    st = _load().orc_encode(*codec.args(), _p(g, _u32p), len(g), _p(ctrl, _u8p), len(ctrl),
                            ctypes.byref(cb), _p(data, _u32p), len(data), ctypes.byref(dw))
    if st:
        raise OracleError(st, "encode")
    return ctrl[:cb.value].copy(), data[:dw.value].copy()


def decode(codec: Codec, ctrl, data, n: int) -> np.ndarray:
    """Decode n ints (raw gaps, no prefix sum)."""
    c = np.ascontiguousarray(ctrl, dtype=np.uint8)
    d = _u32(data)
    c1 = c if len(c) else np.zeros(1, np.uint8)
    d1 = d if len(d) else np.zeros(1, np.uint32)
    out = np.zeros(max(1, n), np.uint32)
    st = _load().orc_decode(codec.kind, codec.k, codec.cg, codec.ld, _p(c1, _u8p), len(c),
                            _p(d1, _u32p), len(d), n, _p(out, _u32p))
    if st:
        raise OracleError(st, "decode")
    return out[:n].copy()


def vb_size(x: int) -> int:
    """Bytes Variable Byte takes for x (Section 2.3)."""
    return int(_load().orc_vb_size(int(x)))


def vb_encode(gaps) -> np.ndarray:
    """Variable Byte (Section 2.3; lists shorter than 64, Section 7.5):
    7-bit groups most significant first, the high bit set on each number's
    last byte. Returns the bytes (uint8)."""
    g = _u32(gaps)
    out = np.zeros(max(1, 5 * len(g)), np.uint8)
    g1 = g if len(g) else np.zeros(1, np.uint32)
    nb = _load().orc_vb_encode(_p(g1, _u32p), len(g), _p(out, _u8p), len(out))
    if nb == 2**64 - 1:
        raise OracleError(ERR_NOSPACE, "vb_encode")
    return out[:nb].copy()


def vb_decode(data, n: int) -> np.ndarray:
    """n ints from Variable Byte bytes (all of them used)."""
    b = np.ascontiguousarray(data, dtype=np.uint8)
    b1 = b if len(b) else np.zeros(1, np.uint8)
    out = np.zeros(max(1, n), np.uint32)
    st = _load().orc_vb_decode(_p(b1, _u8p), len(b), n, _p(out, _u32p))
    if st:
        raise OracleError(st, "vb_decode")
    return out[:n].copy()


def decode_docids(codec: Codec, ctrl, data, n: int) -> np.ndarray:
    return prefix_sum(decode(codec, ctrl, data, n))


def paper_pack(ctrl, data) -> np.ndarray:
    """The paper's single buffer: u32 data offset (words) | control | pad to
    16 B | data (Section 4.3, step 1)."""
    c = np.ascontiguousarray(ctrl, dtype=np.uint8)
    d = _u32(data)
    c1 = c if len(c) else np.zeros(1, np.uint8)
    d1 = d if len(d) else np.zeros(1, np.uint32)
    lib = _load()
    size = lib.orc_paper_pack(_p(c1, _u8p), len(c), _p(d1, _u32p), len(d), None)
    buf = np.zeros(size, np.uint8)
    lib.orc_paper_pack(_p(c1, _u8p), len(c), _p(d1, _u32p), len(d), _p(buf, _u8p))
    return buf


def tile_index(codec: Codec, ctrl, n: int, gaps=None) -> np.ndarray:
    """Per 1024-int tile: where its first unit starts (see gc_oracle.c). With
    the list's gaps, every record also gets its skip entry (the docID before
    the tile, Sections 2.1.1 and 7.5); without them only tile 0 has one."""
    lib = _load()
    nt = lib.orc_tile_count(n, codec.k)
    out = np.zeros(nt, TILE_DTYPE)
    c = np.ascontiguousarray(ctrl, dtype=np.uint8)
    c1 = c if len(c) else np.zeros(1, np.uint8)
    if nt:
        st = lib.orc_tile_index(codec.kind, codec.k, codec.cg, codec.ld, _p(c1, _u8p), len(c), n,
                                out.ctypes.data_as(ctypes.c_void_p))
        if st:
            raise OracleError(st, "tile_index")
        if gaps is not None:
            g = _u32(gaps)
            if len(g) != n:
                raise ValueError("gaps must hold the list's n ints")
            lib.orc_tile_bases(_p(g, _u32p), n, codec.k, out.ctypes.data_as(ctypes.c_void_p))
    return out


def bits_per_int(ctrl, data, n: int) -> float:
    return 8.0 * (len(ctrl) + 4 * len(data)) / max(1, n)
