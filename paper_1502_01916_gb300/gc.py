"""ctypes binding of the C ABI in ``include/gc.h``.

Each ``gc_*`` function here forwards to the C call of the same name: it
turns torch tensors into device pointers and sizes, passes the current CUDA
stream, and raises ``GcError`` on a non-zero status. Nothing is computed in
Python. A few helpers (``encode``, ``decode``, ``encode_index``,
``decode_index``) allocate the caller-owned buffers the C calls expect, with
torch, and then make exactly those calls.

Integer streams are held in torch tensors of dtype int32 (bit pattern of
the uint32 values) and uint8; ``as_u32`` views one as numpy uint32.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np
import torch

__all__ = [
    "SIMPLE", "SCHEME", "AFOR", "PFD", "LD_BINARY", "LD_CU", "LD_IU", "TILE_INTS", "TILE_BYTES", "LIST_BYTES",
    "TILE_BASE", "WORK_VEC_SHIFT", "WORK_BIT_SHIFT", "WORK_SKIP_SHIFT", "WORK_HAS_BASE", "WORK_PUBLISH",
    "TILE_DTYPE", "LIST_DTYPE", "WORK_DTYPE",
    "WORK_BYTES", "GcError", "gc_work", "gc_plan_batch", "gc_plan_select", "gc_decode_plan_scratch_size",
    "gc_decode_plan", "Plan", "gc_intersect_scratch_size", "gc_intersect", "intersect", "AndBatch", "and_batch",
    "run_and_batch", "and_batch_tiles", "VB_LIST_BYTES", "VB_LIST_DTYPE", "gc_vb_encode_batch",
    "gc_vb_decode_batch", "MixedIndex", "encode_mixed_index", "decode_mixed",
    "plan_index",
    "gc_codec", "gc_tile", "gc_list", "gc_launch", "library_path", "load", "make_codec",
    "gc_pfd_rows_for_zeta", "gc_max_encoded_size", "gc_encode_scratch_size", "gc_encode",
    "gc_encode_batch_scratch_size", "gc_encode_batch", "gc_decode_scratch_size", "gc_build_tiles",
    "gc_decode", "gc_decode_paper", "gc_decode_batch_scratch_size", "gc_decode_batch", "gc_decode_static",
    "DECODE_STATIC_MAX_INTS",
    "gc_last_launch_count", "gc_version", "EncodedList", "Index", "encode", "decode",
    "build_tiles", "decode_paper", "encode_index", "decode_index", "new_status", "check_status",
    "as_u32", "codec_name", "gc_paper_bytes", "gc_pack_paper", "gc_unpack_paper", "pack_paper", "unpack_paper",
    "gc_set_launch", "gc_get_launch", "gc_decode_plan_host_buffer_size", "gc_decode_plan_host", "gc_shutdown",
    "gc_plan_interleave", "RESTORE_PER_RECORD", "plan_interleave", "WORK_RAW", "tiles_of",
]

SIMPLE, SCHEME, AFOR, PFD = 0, 1, 2, 3
LD_BINARY, LD_CU, LD_IU = 0, 1, 2
TILE_INTS = 1024
_STATUS = {0: "GC_OK", 1: "GC_ERR_INVALID", 2: "GC_ERR_NOSPACE", 3: "GC_ERR_CORRUPT",
           4: "GC_ERR_CUDA", 5: "GC_ERR_TIMEOUT", 6: "GC_ERR_UNSUPPORTED"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "_build", "libgc.so")


class GcError(RuntimeError):
    def __init__(self, code: int, what: str, where: int | None = None):
        msg = f"{what}: {_STATUS.get(code, code)}"
        if where is not None:
            msg += f" (tile/list {where})"
        super().__init__(msg)
        self.code = code
        self.where = where


class gc_codec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("k", ctypes.c_uint32), ("cg", ctypes.c_uint32),
                ("ld", ctypes.c_uint32), ("pfd_exc_rows", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class gc_tile(ctypes.Structure):
    _fields_ = [("lane_bit", ctypes.c_uint64), ("ctrl_bit", ctypes.c_uint64),
                ("exc_off", ctypes.c_uint32), ("row_skip", ctypes.c_uint32),
                ("base", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class gc_list(ctypes.Structure):
    _fields_ = [("ctrl_off", ctypes.c_uint64), ("data_off", ctypes.c_uint64),
                ("out_off", ctypes.c_uint64), ("n", ctypes.c_uint32), ("tile_off", ctypes.c_uint32),
                ("ctrl_bytes", ctypes.c_uint32), ("data_words", ctypes.c_uint32)]


class gc_launch(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("items_per_claim", ctypes.c_uint32), ("stage_bytes", ctypes.c_uint32)]


class gc_work(ctypes.Structure):
    _fields_ = [("ctrl_at", ctypes.c_uint64), ("data_at", ctypes.c_uint64), ("out_at", ctypes.c_uint64),
                ("ctrl_bit", ctypes.c_uint64), ("ctrl_bytes", ctypes.c_uint32), ("tile", ctypes.c_uint32),
                ("list", ctypes.c_uint32), ("base", ctypes.c_uint32), ("exc_at", ctypes.c_uint32),
                ("win_at", ctypes.c_int32), ("shape", ctypes.c_uint32), ("win_len", ctypes.c_uint16),
                ("exc_len", ctypes.c_uint16)]


TILE_BASE = 1
WORK_VEC_SHIFT, WORK_BIT_SHIFT, WORK_SKIP_SHIFT = 10, 19, 24
WORK_HAS_BASE, WORK_PUBLISH, WORK_RAW = 1 << 29, 1 << 30, 1 << 31
TILE_DTYPE = np.dtype([("lane_bit", "<u8"), ("ctrl_bit", "<u8"), ("exc_off", "<u4"), ("row_skip", "<u4"),
                       ("base", "<u4"), ("flags", "<u4")])
LIST_DTYPE = np.dtype([("ctrl_off", "<u8"), ("data_off", "<u8"), ("out_off", "<u8"), ("n", "<u4"),
                       ("tile_off", "<u4"), ("ctrl_bytes", "<u4"), ("data_words", "<u4")])
WORK_DTYPE = np.dtype([("ctrl_at", "<u8"), ("data_at", "<u8"), ("out_at", "<u8"), ("ctrl_bit", "<u8"),
                       ("ctrl_bytes", "<u4"), ("tile", "<u4"), ("list", "<u4"), ("base", "<u4"),
                       ("exc_at", "<u4"), ("win_at", "<i4"), ("shape", "<u4"), ("win_len", "<u2"),
                       ("exc_len", "<u2")])


TILE_BYTES = ctypes.sizeof(gc_tile)
LIST_BYTES = ctypes.sizeof(gc_list)
WORK_BYTES = ctypes.sizeof(gc_work)

_lib = None
_lock = threading.Lock()
_V, _U32, _U64, _I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_CP = ctypes.POINTER(gc_codec)
_U64P = ctypes.POINTER(ctypes.c_uint64)


def library_path() -> str:
    return _LIB


def load():
    """Load libgc.so. Raises if it has not been built: there is no fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB):
            raise RuntimeError(f"{_LIB} is missing: build it with paper_1502_01916_gb300.build.build() "
                               "(nvcc, sm_103a); the decode path has no CPU fallback")
        lib = ctypes.CDLL(_LIB)
        sig = {
            "gc_pfd_rows_for_zeta": (_U32, [ctypes.c_double]),
            "gc_max_encoded_size": (_I, [_CP, _U64, _U64P, _U64P, _U64P]),
            "gc_encode_scratch_size": (_I, [_CP, _U64, _U64P]),
            "gc_encode": (_I, [_CP, _V, _U64, _V, _U64, _V, _U64, _V, _V, _V, _U64, _V]),
            "gc_encode_batch_scratch_size": (_I, [_CP, _V, _U64, _U64P]),
            "gc_encode_batch": (_I, [_CP, _V, _V, _V, _U64, _V, _V, _U64, _V, _U64, _V, _U64, _V, _V,
                                     _U64, _V]),
            "gc_decode_scratch_size": (_I, [_CP, _U64, _I, _U64P]),
            "gc_build_tiles": (_I, [_CP, _V, _U64, _U64, _V, _V, _U64, _V, _V]),
            "gc_decode": (_I, [_CP, _V, _U64, _V, _U64, _U64, _V, _V, _I, _V, _U64, _V, _V]),
            "gc_decode_paper": (_I, [_CP, _V, _U64, _U64, _V, _I, _V, _U64, _V, _V]),
            "gc_decode_static": (_I, [_CP, _V, _U64, _V, _U64, _U64, _V, _V, _I, _V, _V]),
            "gc_decode_batch_scratch_size": (_I, [_U64, _U64, _U64P]),
            "gc_decode_batch": (_I, [_CP, _V, _U64, _V, _U64, _V, _U64, _V, _U64, _V, _U64, _I, _U64,
                                     ctypes.POINTER(gc_launch), _V, _U64, _V, _V]),
            "gc_plan_batch": (_I, [_CP, _V, _U64, _V, _U64, _V, _U64, _V, _U64, _V, _V, _V]),
            "gc_plan_select": (_I, [_CP, _V, _U64, _V, _V, _U64, _V, _U64, _V, _U64, _V, _U64, _V, _V, _V]),
            "gc_plan_interleave": (_I, [_CP, _V, _U64, _V, _V, _U64, _V, _U64, _V, _U64, _V, _U64, _V, _V, _V]),
            "gc_decode_plan_scratch_size": (_I, [_U64, _U64P]),
            "gc_decode_plan": (_I, [_CP, _V, _V, _U64, _V, _U64, _V, _U64, _V, _U64, _I,
                                    ctypes.POINTER(gc_launch), _V, _U64, _V, _V]),
            "gc_vb_encode_batch_scratch_size": (_I, [_U64, _U64P]),
            "gc_vb_encode_batch": (_I, [_V, _V, _V, _U64, _V, _V, _U64, _V, _V, _U64, _V, _V]),
            "gc_vb_decode_batch": (_I, [_V, _U64, _V, _U64, _V, _U64, _I, _V, _V]),
            "gc_intersect_scratch_size": (_I, [_U64, _U64, _U64, _U64P]),
            "gc_intersect": (_I, [_CP, _V, _U64, _V, _U64, _V, _U64, _V, _U64, _V, _V, _V, _V, _U64, _U64, _U64,
                                  _U64, _V, _V, _V, _U64, _V, _V]),
            "gc_paper_bytes": (_U64, [_U64, _U64]),
            "gc_pack_paper": (_I, [_V, _U64, _V, _U64, _V, _U64, _V]),
            "gc_unpack_paper": (_I, [_V, _U64, _V, _U64, _V, _U64, _U64P, _U64P, _V]),
            "gc_set_launch": (_I, [_CP, _I, ctypes.POINTER(gc_launch)]),
            "gc_get_launch": (_I, [_CP, _I, ctypes.POINTER(gc_launch)]),
            "gc_decode_plan_host_buffer_size": (_I, [_U64, _U64, _U64, _U64, _U64P]),
            "gc_decode_plan_host": (_I, [_CP, _V, _U64, _V, _U64, _V, _U64, _V, _U64, _I,
                                         ctypes.POINTER(gc_launch), _V, _U64, _V, _V]),
            "gc_shutdown": (None, []),
            "gc_last_launch_count": (_U32, []),
            "gc_version": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(st: int, what: str):
    if st != 0:
        raise GcError(st, what)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _n(t, esize: int, what: str) -> int:
    """The element count of a device buffer whose size the C ABI takes in
    esize-byte units, after checking that it is a contiguous CUDA tensor of
    such elements (a wrong dtype would give the library a wrong size)."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous() or t.element_size() != esize:
        raise ValueError(f"{what}: expected a contiguous CUDA tensor of {esize}-byte elements")
    return t.numel()


def _restore(r) -> int:
    return RESTORE_PER_RECORD if (not isinstance(r, bool) and r == RESTORE_PER_RECORD) else int(bool(r))


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def make_codec(kind: int, k: int = 32, cg: int = 8, ld: int = LD_BINARY, zeta: float = 0.10,
               exc_rows: int | None = None) -> gc_codec:
    """A codec descriptor; Group-PFD's zeta becomes the row count of Step 2."""
    rows = gc_pfd_rows_for_zeta(zeta) if exc_rows is None else exc_rows
    return gc_codec(kind, k, cg if kind == SCHEME else 0, ld if kind == SCHEME else 0,
                    rows if kind == PFD else 0, 0)


def codec_name(c: gc_codec) -> str:
    base = {SIMPLE: "GS", AFOR: "AFOR"}.get(c.kind)
    if c.kind == SCHEME:
        base = f"GSC-{c.cg}-{['B', 'CU', 'IU'][c.ld]}"
    elif c.kind == PFD:
        base = f"PFD(x{c.pfd_exc_rows})"
    return f"{base}/k{c.k}"


# ------------------------------------------------------------------ raw ABI

def gc_pfd_rows_for_zeta(zeta: float) -> int:
    return int(load().gc_pfd_rows_for_zeta(float(zeta)))


def gc_max_encoded_size(codec: gc_codec, n: int):
    cc, dc, nt = _U64(), _U64(), _U64()
    _check(load().gc_max_encoded_size(ctypes.byref(codec), n, ctypes.byref(cc), ctypes.byref(dc),
                                      ctypes.byref(nt)), "gc_max_encoded_size")
    return cc.value, dc.value, nt.value


def gc_encode_scratch_size(codec: gc_codec, n: int) -> int:
    b = _U64()
    _check(load().gc_encode_scratch_size(ctypes.byref(codec), n, ctypes.byref(b)), "gc_encode_scratch_size")
    return b.value


def gc_encode(codec, d_gaps, n, d_ctrl, d_data, d_tiles, d_sizes, d_scratch, stream=None):
    lib = load()
    _check(lib.gc_encode(ctypes.byref(codec), _ptr(d_gaps), n, _ptr(d_ctrl), _n(d_ctrl, 1, "d_ctrl"), _ptr(d_data),
                         _n(d_data, 4, "d_data"), _ptr(d_tiles), _ptr(d_sizes), _ptr(d_scratch),
                         _n(d_scratch, 1, "d_scratch"), _stream(stream)), "gc_encode")


def gc_encode_batch_scratch_size(codec: gc_codec, h_n: np.ndarray) -> int:
    h_n = np.ascontiguousarray(h_n, dtype=np.uint32)
    b = _U64()
    _check(load().gc_encode_batch_scratch_size(ctypes.byref(codec), h_n.ctypes.data, len(h_n), ctypes.byref(b)),
           "gc_encode_batch_scratch_size")
    return b.value


def gc_encode_batch(codec, d_gaps, h_n, h_in_off, d_lists, d_ctrl, d_data, d_tiles, d_totals, d_scratch,
                    stream=None):
    h_n = np.ascontiguousarray(h_n, dtype=np.uint32)
    h_in_off = np.ascontiguousarray(h_in_off, dtype=np.uint64)
    _check(load().gc_encode_batch(ctypes.byref(codec), _ptr(d_gaps), h_n.ctypes.data, h_in_off.ctypes.data,
                                  len(h_n), _ptr(d_lists), _ptr(d_ctrl), _n(d_ctrl, 1, "d_ctrl"), _ptr(d_data),
                                  _n(d_data, 4, "d_data"), _ptr(d_tiles), _n(d_tiles, 1, "d_tiles") // TILE_BYTES,
                                  _ptr(d_totals), _ptr(d_scratch), _n(d_scratch, 1, "d_scratch"), _stream(stream)),
           "gc_encode_batch")


def gc_decode_scratch_size(codec: gc_codec, n: int, have_tiles: bool) -> int:
    b = _U64()
    _check(load().gc_decode_scratch_size(ctypes.byref(codec), n, int(bool(have_tiles)), ctypes.byref(b)),
           "gc_decode_scratch_size")
    return b.value


def gc_build_tiles(codec, d_ctrl, ctrl_bytes, n, d_tiles, d_scratch, d_status, stream=None):
    _check(load().gc_build_tiles(ctypes.byref(codec), _ptr(d_ctrl), ctrl_bytes, n, _ptr(d_tiles),
                                 _ptr(d_scratch), _n(d_scratch, 1, "d_scratch"), _ptr(d_status), _stream(stream)),
           "gc_build_tiles")


def gc_decode(codec, d_ctrl, ctrl_bytes, d_data, data_words, n, d_tiles, d_out, restore_docids, d_scratch,
              d_status, stream=None):
    _check(load().gc_decode(ctypes.byref(codec), _ptr(d_ctrl), ctrl_bytes, _ptr(d_data), data_words, n,
                            _ptr(d_tiles), _ptr(d_out), int(bool(restore_docids)), _ptr(d_scratch),
                            _n(d_scratch, 1, "d_scratch"), _ptr(d_status), _stream(stream)), "gc_decode")


DECODE_STATIC_MAX_INTS = 1 << 20


def gc_decode_static(codec, d_ctrl, ctrl_bytes, d_data, data_words, n, d_tiles, d_out, restore_docids, d_status,
                     stream=None):
    """gc_decode with the library's own fixed scratch (no allocation; n <= DECODE_STATIC_MAX_INTS)."""
    _check(load().gc_decode_static(ctypes.byref(codec), _ptr(d_ctrl), ctrl_bytes, _ptr(d_data), data_words, n,
                                   _ptr(d_tiles), _ptr(d_out), int(bool(restore_docids)), _ptr(d_status),
                                   _stream(stream)), "gc_decode_static")


def gc_decode_paper(codec, d_buf, n, d_out, restore_docids, d_scratch, d_status, stream=None):
    _check(load().gc_decode_paper(ctypes.byref(codec), _ptr(d_buf), _n(d_buf, 1, "d_buf"), n, _ptr(d_out),
                                  int(bool(restore_docids)), _ptr(d_scratch), _n(d_scratch, 1, "d_scratch"),
                                  _ptr(d_status), _stream(stream)), "gc_decode_paper")


def gc_decode_batch_scratch_size(nlists: int, max_tiles: int) -> int:
    b = _U64()
    _check(load().gc_decode_batch_scratch_size(nlists, max_tiles, ctypes.byref(b)), "gc_decode_batch_scratch_size")
    return b.value


def gc_decode_batch(codec, d_lists, nlists, d_ctrl_pool, d_data_pool, d_tile_pool, d_out_pool, restore_docids,
                    max_tiles, launch, d_scratch, d_status, stream=None):
    lp = ctypes.byref(launch) if launch is not None else None
    tile_len = _n(d_tile_pool, 1, "d_tile_pool") // TILE_BYTES if d_tile_pool is not None else 0
    _check(load().gc_decode_batch(ctypes.byref(codec), _ptr(d_lists), nlists, _ptr(d_ctrl_pool),
                                  _n(d_ctrl_pool, 1, "d_ctrl_pool"), _ptr(d_data_pool),
                                  _n(d_data_pool, 4, "d_data_pool"), _ptr(d_tile_pool), tile_len, _ptr(d_out_pool),
                                  _n(d_out_pool, 4, "d_out_pool"), int(bool(restore_docids)), max_tiles, lp,
                                  _ptr(d_scratch), _n(d_scratch, 1, "d_scratch"), _ptr(d_status), _stream(stream)),
           "gc_decode_batch")


def gc_plan_batch(codec, d_lists, nlists, d_tile_pool, d_ctrl_pool, d_work, d_count, d_status, stream=None):
    tile_len = _n(d_tile_pool, 1, "d_tile_pool") // TILE_BYTES if d_tile_pool is not None else 0
    _check(load().gc_plan_batch(ctypes.byref(codec), _ptr(d_lists), nlists, _ptr(d_tile_pool), tile_len,
                                _ptr(d_ctrl_pool), _n(d_ctrl_pool, 1, "d_ctrl_pool"), _ptr(d_work),
                                _n(d_work, 1, "d_work") // WORK_BYTES, _ptr(d_count), _ptr(d_status),
                                _stream(stream)), "gc_plan_batch")


def gc_plan_select(codec, d_lists, nlists, d_sel, d_out_offs, nsel, d_tile_pool, d_ctrl_pool, d_work, d_count,
                   d_status, stream=None):
    tile_len = _n(d_tile_pool, 1, "d_tile_pool") // TILE_BYTES if d_tile_pool is not None else 0
    _check(load().gc_plan_select(ctypes.byref(codec), _ptr(d_lists), nlists, _ptr(d_sel), _ptr(d_out_offs), nsel,
                                 _ptr(d_tile_pool), tile_len, _ptr(d_ctrl_pool), _n(d_ctrl_pool, 1, "d_ctrl_pool"),
                                 _ptr(d_work), _n(d_work, 1, "d_work") // WORK_BYTES, _ptr(d_count), _ptr(d_status),
                                 _stream(stream)),
           "gc_plan_select")


def gc_plan_interleave(codec, d_lists, nlists, d_sel_pairs, d_out_pairs, npairs, d_tile_pool, d_ctrl_pool, d_work,
                       d_count, d_status, stream=None):
    tile_len = _n(d_tile_pool, 1, "d_tile_pool") // TILE_BYTES if d_tile_pool is not None else 0
    if npairs and (_n(d_sel_pairs, 4, "d_sel_pairs") < 2 * npairs or _n(d_out_pairs, 8, "d_out_pairs") < 2 * npairs):
        raise ValueError("d_sel_pairs / d_out_pairs hold fewer than 2 * npairs entries")
    _check(load().gc_plan_interleave(ctypes.byref(codec), _ptr(d_lists), nlists, _ptr(d_sel_pairs),
                                     _ptr(d_out_pairs), npairs, _ptr(d_tile_pool), tile_len, _ptr(d_ctrl_pool),
                                     _n(d_ctrl_pool, 1, "d_ctrl_pool"), _ptr(d_work), _n(d_work, 1, "d_work") // WORK_BYTES,
                                     _ptr(d_count), _ptr(d_status), _stream(stream)), "gc_plan_interleave")


RESTORE_PER_RECORD = 2


def gc_decode_plan_scratch_size(work_cap: int) -> int:
    b = _U64()
    _check(load().gc_decode_plan_scratch_size(work_cap, ctypes.byref(b)), "gc_decode_plan_scratch_size")
    return b.value


def gc_decode_plan(codec, d_work, d_count, d_ctrl_pool, d_data_pool, d_out_pool, restore_docids, launch, d_scratch,
                   d_status, stream=None):
    """restore_docids: 0 values, 1 docIDs, RESTORE_PER_RECORD docIDs except raw (TF) records."""
    lp = ctypes.byref(launch) if launch is not None else None
    _check(load().gc_decode_plan(ctypes.byref(codec), _ptr(d_work), _ptr(d_count),
                                 _n(d_work, 1, "d_work") // WORK_BYTES, _ptr(d_ctrl_pool),
                                 _n(d_ctrl_pool, 1, "d_ctrl_pool"), _ptr(d_data_pool),
                                 _n(d_data_pool, 4, "d_data_pool"), _ptr(d_out_pool), _n(d_out_pool, 4, "d_out_pool"),
                                 _restore(restore_docids), lp, _ptr(d_scratch), _n(d_scratch, 1, "d_scratch"),
                                 _ptr(d_status), _stream(stream)),
           "gc_decode_plan")


def gc_paper_bytes(ctrl_bytes: int, data_words: int) -> int:
    return int(load().gc_paper_bytes(ctrl_bytes, data_words))


def gc_pack_paper(d_ctrl, ctrl_bytes, d_data, data_words, d_buf, stream=None):
    _check(load().gc_pack_paper(_ptr(d_ctrl), ctrl_bytes, _ptr(d_data), data_words, _ptr(d_buf),
                                _n(d_buf, 1, "d_buf"), _stream(stream)), "gc_pack_paper")


def gc_unpack_paper(d_buf, d_ctrl, d_data, stream=None):
    """Returns (ctrl_bytes, data_words) of the buffer's areas."""
    cb, dw = _U64(), _U64()
    st = load().gc_unpack_paper(_ptr(d_buf), _n(d_buf, 1, "d_buf"), _ptr(d_ctrl),
                                _n(d_ctrl, 1, "d_ctrl") if d_ctrl is not None else 0, _ptr(d_data),
                                _n(d_data, 4, "d_data") if d_data is not None else 0, ctypes.byref(cb),
                                ctypes.byref(dw), _stream(stream))
    _check(st, "gc_unpack_paper")
    return cb.value, dw.value


def gc_set_launch(codec, restore_docids, launch):
    lp = ctypes.byref(launch) if launch is not None else None
    _check(load().gc_set_launch(ctypes.byref(codec), int(bool(restore_docids)), lp), "gc_set_launch")


def gc_get_launch(codec, restore_docids) -> gc_launch:
    l = gc_launch()
    _check(load().gc_get_launch(ctypes.byref(codec), int(bool(restore_docids)), ctypes.byref(l)), "gc_get_launch")
    return l


def gc_decode_plan_host_buffer_size(nwork: int, ctrl_pool_bytes: int, data_pool_words: int,
                                    out_pool_len: int) -> int:
    b = _U64()
    _check(load().gc_decode_plan_host_buffer_size(nwork, ctrl_pool_bytes, data_pool_words, out_pool_len,
                                                  ctypes.byref(b)), "gc_decode_plan_host_buffer_size")
    return b.value


def _h(t, esize: int, what: str):
    """(pointer, element count) of a host buffer: a contiguous CPU tensor or
    numpy array of esize-byte elements."""
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"] or t.itemsize != esize:
            raise ValueError(f"{what}: expected a contiguous array of {esize}-byte elements")
        return t.ctypes.data, t.size
    if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_contiguous() or t.element_size() != esize:
        raise ValueError(f"{what}: expected a contiguous host tensor of {esize}-byte elements")
    return t.data_ptr(), t.numel()


def gc_decode_plan_host(codec, h_work, nwork, h_ctrl_pool, h_data_pool, h_out_pool, restore_docids, launch,
                        d_buffers, d_status, stream=None):
    """gc_decode_plan with the plan, pools and output in host memory (nwork
    records of h_work are decoded)."""
    wp, wb = _h(h_work, 1, "h_work")
    if nwork * WORK_BYTES > wb:
        raise ValueError("h_work holds fewer than nwork records")
    cp, cn = _h(h_ctrl_pool, 1, "h_ctrl_pool")
    dp, dn = _h(h_data_pool, 4, "h_data_pool")
    op, on = _h(h_out_pool, 4, "h_out_pool")
    lp = ctypes.byref(launch) if launch is not None else None
    _check(load().gc_decode_plan_host(ctypes.byref(codec), wp, nwork, cp, cn, dp, dn, op, on,
                                      _restore(restore_docids), lp, _ptr(d_buffers), _n(d_buffers, 1, "d_buffers"),
                                      _ptr(d_status), _stream(stream)), "gc_decode_plan_host")


def gc_shutdown():
    load().gc_shutdown()


def gc_last_launch_count() -> int:
    return int(load().gc_last_launch_count())


def gc_version() -> str:
    return load().gc_version().decode()


# ------------------------------------------------------------------ helpers

def _dev(device=None):
    return torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)


def new_status(device=None) -> torch.Tensor:
    """The two-word device status a decode call reports into (zeroed)."""
    return torch.zeros(2, dtype=torch.int32, device=_dev(device))


def check_status(status: torch.Tensor, what: str = "device status"):
    """Synchronise by reading the status words; raise if the GPU reported one."""
    code, where = (int(x) & 0xFFFFFFFF for x in status.cpu().tolist())
    if code:
        raise GcError(code, what, where)


def as_u32(t: torch.Tensor) -> np.ndarray:
    """A device or host int32 tensor's values as numpy uint32."""
    return t.detach().cpu().numpy().view(np.uint32)


def _i32(a, device) -> torch.Tensor:
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).to(device)


@dataclasses.dataclass
class EncodedList:
    """One encoded list on the device: control bytes, data words (int32
    holding uint32), and its tile index (gc_tile records as raw bytes)."""
    codec: gc_codec
    n: int
    ctrl: torch.Tensor
    data: torch.Tensor
    tiles: torch.Tensor | None

    @property
    def ctrl_bytes(self) -> int:
        return self.ctrl.numel()

    @property
    def data_words(self) -> int:
        return self.data.numel()

    def compressed_bytes(self) -> int:
        return self.ctrl.numel() + 4 * self.data.numel()


def _data_buffer(words: int, device) -> torch.Tensor:
    # 16-byte aligned by the torch caching allocator (512-byte blocks)
    return torch.empty(max(4, words), dtype=torch.int32, device=device)


def encode(codec: gc_codec, gaps, device=None, with_tiles: bool = True, stream=None) -> EncodedList:
    """Encode one list on the GPU (gc_encode). `gaps` is a uint32 array or an
    int32 CUDA tensor."""
    dev = _dev(device)
    d_gaps = gaps if isinstance(gaps, torch.Tensor) else _i32(gaps, dev)
    n = d_gaps.numel()
    cc, dc, nt = gc_max_encoded_size(codec, n)
    d_ctrl = torch.empty(max(4, cc), dtype=torch.uint8, device=dev)
    d_data = _data_buffer(dc, dev)
    d_tiles = torch.empty(max(1, nt) * TILE_BYTES, dtype=torch.uint8, device=dev) if with_tiles else None
    d_sizes = torch.zeros(2, dtype=torch.int64, device=dev)
    d_scratch = torch.empty(max(256, gc_encode_scratch_size(codec, n)), dtype=torch.uint8, device=dev)
    gc_encode(codec, d_gaps, n, d_ctrl, d_data, d_tiles, d_sizes, d_scratch, stream)
    cb, dw = (int(x) for x in d_sizes.cpu().tolist())
    return EncodedList(codec, n, d_ctrl[:cb], d_data[:dw], d_tiles[:nt * TILE_BYTES] if with_tiles else None)


def decode(enc: EncodedList, restore_docids: bool = True, use_tiles: bool = True, out=None,
           status=None, check: bool = True, stream=None) -> torch.Tensor:
    """Decode one list (gc_decode); docIDs when restore_docids, else gaps."""
    dev = enc.data.device
    out = torch.empty(max(1, enc.n), dtype=torch.int32, device=dev) if out is None else out
    tiles = enc.tiles if use_tiles else None
    scratch = torch.empty(max(256, gc_decode_scratch_size(enc.codec, enc.n, tiles is not None)),
                          dtype=torch.uint8, device=dev)
    st = new_status(dev) if status is None else status
    gc_decode(enc.codec, enc.ctrl, enc.ctrl_bytes, enc.data, enc.data_words, enc.n, tiles, out,
              restore_docids, scratch, st, stream)
    if check:
        check_status(st, "gc_decode")
    return out[:enc.n]


def build_tiles(codec: gc_codec, ctrl: torch.Tensor, n: int, status=None, stream=None) -> torch.Tensor:
    """The tile index of an encoded list from its control area (gc_build_tiles)."""
    dev = ctrl.device
    _, _, nt = gc_max_encoded_size(codec, n)
    tiles = torch.zeros(max(1, nt) * TILE_BYTES, dtype=torch.uint8, device=dev)
    scratch = torch.empty(max(256, gc_decode_scratch_size(codec, n, False)), dtype=torch.uint8, device=dev)
    st = new_status(dev) if status is None else status
    gc_build_tiles(codec, ctrl, ctrl.numel(), n, tiles, scratch, st, stream)
    check_status(st, "gc_build_tiles")
    return tiles[:nt * TILE_BYTES]


def decode_paper(codec: gc_codec, buf: torch.Tensor, n: int, restore_docids: bool = True,
                 stream=None) -> torch.Tensor:
    """Decode the paper's single buffer (gc_decode_paper)."""
    dev = buf.device
    out = torch.empty(max(1, n), dtype=torch.int32, device=dev)
    scratch = torch.empty(max(256, gc_decode_scratch_size(codec, n, False)), dtype=torch.uint8, device=dev)
    st = new_status(dev)
    gc_decode_paper(codec, buf, n, out, restore_docids, scratch, st, stream)
    check_status(st, "gc_decode_paper")
    return out[:n]


def pack_paper(enc: "EncodedList", stream=None) -> torch.Tensor:
    """The paper's single buffer of an encoded list (gc_pack_paper)."""
    dev = enc.data.device
    cb, dw = enc.ctrl_bytes, enc.data_words
    buf = torch.empty(gc_paper_bytes(cb, dw), dtype=torch.uint8, device=dev)
    gc_pack_paper(enc.ctrl, cb, enc.data, dw, buf, stream)
    return buf


def unpack_paper(buf: torch.Tensor, stream=None):
    """(control bytes, data words) tensors of the paper's single buffer
    (gc_unpack_paper); the control area includes its padding zeros."""
    dev = buf.device
    ctrl = torch.empty(max(16, buf.numel()), dtype=torch.uint8, device=dev)
    data = _data_buffer(max(4, buf.numel() // 4), dev)
    cb, dw = gc_unpack_paper(buf, ctrl, data, stream)
    return ctrl[:cb], data[:dw]


@dataclasses.dataclass
class Index:
    """Many encoded lists laid out back to back on the device (gc_encode_batch):
    descriptors (gc_list records), control pool, data pool, tile pool."""
    codec: gc_codec
    lengths: np.ndarray      # uint32 per list
    out_offsets: np.ndarray  # uint64 per list: first output int
    lists: torch.Tensor      # nlists * 40 bytes (gc_list)
    ctrl: torch.Tensor
    data: torch.Tensor
    tiles: torch.Tensor
    max_tiles: int           # tiles of all lists (the decode scratch bound)

    @property
    def nlists(self) -> int:
        return len(self.lengths)

    @property
    def total_ints(self) -> int:
        return int(self.lengths.sum(dtype=np.uint64))

    @property
    def out_ints(self) -> int:
        """Length of an output that holds every list at its offset."""
        if not len(self.lengths):
            return 0
        return int((self.out_offsets + self.lengths.astype(np.uint64)).max())

    def compressed_bytes(self) -> int:
        return self.ctrl.numel() + 4 * self.data.numel()

    def index_bytes(self) -> int:
        """Everything the batched decoder reads besides the streams."""
        return self.lists.numel() + self.tiles.numel()


def encode_index(codec: gc_codec, d_gaps: torch.Tensor, lengths, out_offsets=None, stream=None) -> Index:
    """Encode every list of `d_gaps` in one gc_encode_batch call. List i's
    `lengths[i]` gaps start at `out_offsets[i]` of `d_gaps` (default: back to
    back), and its docIDs decode to the same offsets of the output: padding
    between lists in `d_gaps` places each list's output, e.g. at 16-byte
    boundaries."""
    dev = d_gaps.device
    h_n = np.ascontiguousarray(lengths, dtype=np.uint32)
    if out_offsets is None:
        out_offsets = np.zeros(len(h_n), np.uint64)
        if len(h_n) > 1:
            np.cumsum(h_n[:-1], dtype=np.uint64, out=out_offsets[1:])
    out_offsets = np.ascontiguousarray(out_offsets, dtype=np.uint64)
    if out_offsets.shape != h_n.shape:
        raise ValueError("out_offsets needs one offset per list")
    # the library cannot see the length of d_gaps: check every list lies in it
    if len(h_n) and int((out_offsets + h_n.astype(np.uint64)).max()) > d_gaps.numel():
        raise ValueError("a list runs past the end of d_gaps")
    tr = TILE_INTS // codec.k
    rows = (h_n.astype(np.uint64) + codec.k - 1) // codec.k
    nt = (rows + tr - 1) // tr
    max_tiles = int(nt.sum())
    tile_recs = int(np.maximum(nt, 1).sum() - len(nt))
    cc = dc = 0
    # per-list bounds, summed on the host (the C call re-checks them)
    for kind_n in _bounds(codec, h_n):
        cc += kind_n[0]
        dc += kind_n[1]
    d_lists = torch.empty(max(1, len(h_n)) * LIST_BYTES, dtype=torch.uint8, device=dev)
    d_ctrl = torch.empty(max(4, cc), dtype=torch.uint8, device=dev)
    d_data = _data_buffer(dc, dev)
    d_tiles = torch.empty(max(1, tile_recs) * TILE_BYTES, dtype=torch.uint8, device=dev)
    d_totals = torch.zeros(3, dtype=torch.int64, device=dev)
    scratch = torch.empty(max(256, gc_encode_batch_scratch_size(codec, h_n)), dtype=torch.uint8, device=dev)
    gc_encode_batch(codec, d_gaps, h_n, out_offsets, d_lists, d_ctrl, d_data, d_tiles, d_totals, scratch, stream)
    cb, dw, tl = (int(x) for x in d_totals.cpu().tolist())
    del scratch
    return Index(codec, h_n, out_offsets, d_lists, d_ctrl[:cb], d_data[:dw], d_tiles[:tl * TILE_BYTES],
                 max_tiles)


def _bounds(codec: gc_codec, h_n: np.ndarray):
    """(ctrl, data) capacity of every distinct length, expanded per list."""
    uniq, counts = np.unique(h_n, return_counts=True)
    for n, c in zip(uniq.tolist(), counts.tolist()):
        cc, dc, _ = gc_max_encoded_size(codec, n)
        yield cc * c, dc * c


@dataclasses.dataclass
class Plan:
    """The work plan of an index (gc_plan_batch): one gc_work per tile."""
    work: torch.Tensor   # max_tiles * 64 bytes
    count: torch.Tensor  # two int64: tiles, tiles that take their prefix by look-back

    def nbytes(self) -> int:
        return self.work.numel()


def tiles_of(codec: gc_codec, lengths) -> np.ndarray:
    """Tiles (1024 ints, whole rows of k) of lists of these lengths."""
    rows = (np.asarray(lengths, np.int64) + codec.k - 1) // codec.k
    tr = TILE_INTS // codec.k
    return (rows + tr - 1) // tr


def plan_interleave(index: Index, pairs, out_pairs, status=None, stream=None) -> Plan:
    """The interleaved plan (gc_plan_interleave) of (d-gap list, TF list)
    pairs of `index`: pairs is (npairs, 2) list indexes, out_pairs (npairs,
    2) output offsets (docIDs, TFs). Decode it with decode_index(...,
    restore_docids=RESTORE_PER_RECORD, plan=...)."""
    dev = index.data.device
    pairs = np.ascontiguousarray(pairs, np.uint32).reshape(-1, 2)
    outs = np.ascontiguousarray(out_pairs, np.uint64).reshape(-1, 2)
    ntile = tiles_of(index.codec, index.lengths)
    cap = max(1, 2 * int(ntile[pairs[:, 0]].sum())) if len(pairs) else 1
    work = torch.empty(cap * WORK_BYTES, dtype=torch.uint8, device=dev)
    count = torch.zeros(2, dtype=torch.int64, device=dev)
    d_sel = torch.from_numpy(pairs.reshape(-1).view(np.int32).copy()).to(dev)
    d_out = torch.from_numpy(outs.reshape(-1).view(np.int64).copy()).to(dev)
    st = new_status(dev) if status is None else status
    gc_plan_interleave(index.codec, index.lists, index.nlists, d_sel, d_out, len(pairs), index.tiles, index.ctrl, work,
                       count, st, stream)
    check_status(st, "gc_plan_interleave")
    return Plan(work, count)


def plan_index(index: Index, status=None, stream=None) -> Plan:
    """Build the index's work plan on the device (gc_plan_batch)."""
    dev = index.data.device
    work = torch.empty(max(1, index.max_tiles) * WORK_BYTES, dtype=torch.uint8, device=dev)
    count = torch.zeros(2, dtype=torch.int64, device=dev)
    st = new_status(dev) if status is None else status
    gc_plan_batch(index.codec, index.lists, index.nlists, index.tiles, index.ctrl, work, count, st, stream)
    check_status(st, "gc_plan_batch")
    return Plan(work, count)


def decode_index(index: Index, out: torch.Tensor | None = None, restore_docids: bool = True,
                 launch: gc_launch | None = None, scratch: torch.Tensor | None = None, status=None,
                 check: bool = True, stream=None, plan: Plan | None = None) -> torch.Tensor:
    """Decode every list of an index in one call: gc_decode_plan when a plan
    is given, else gc_decode_batch (which plans into its scratch)."""
    dev = index.data.device
    out = torch.empty(max(1, index.out_ints), dtype=torch.int32, device=dev) if out is None else out
    if scratch is None:
        size = (gc_decode_plan_scratch_size(index.max_tiles) if plan is not None
                else gc_decode_batch_scratch_size(index.nlists, index.max_tiles))
        scratch = torch.empty(size, dtype=torch.uint8, device=dev)
    st = new_status(dev) if status is None else status
    if plan is not None:
        gc_decode_plan(index.codec, plan.work, plan.count, index.ctrl, index.data, out, restore_docids, launch,
                       scratch, st, stream)
    else:
        gc_decode_batch(index.codec, index.lists, index.nlists, index.ctrl, index.data, index.tiles, out,
                        restore_docids, index.max_tiles, launch, scratch, st, stream)
    if check:
        check_status(st, "gc_decode_plan" if plan is not None else "gc_decode_batch")
    return out


def gc_intersect_scratch_size(a_ints: int, a_tiles: int, b_tiles: int) -> int:
    b = _U64()
    _check(load().gc_intersect_scratch_size(a_ints, a_tiles, b_tiles, ctypes.byref(b)), "gc_intersect_scratch_size")
    return b.value


def gc_intersect(index, d_a, d_b, d_a_offs, d_b_tile_offs, nqueries, a_ints, a_tiles, b_tiles, d_out, d_counts,
                 d_scratch, d_status, stream=None):
    tile_len = _n(index.tiles, 1, "index.tiles") // TILE_BYTES
    if _n(d_out, 4, "d_out") < a_ints or _n(d_counts, 4, "d_counts") < nqueries:
        raise ValueError("gc_intersect: d_out must hold a_ints and d_counts nqueries uint32")
    _check(load().gc_intersect(ctypes.byref(index.codec), _ptr(index.lists), index.nlists, _ptr(index.tiles), tile_len,
                               _ptr(index.ctrl), _n(index.ctrl, 1, "index.ctrl"), _ptr(index.data),
                               _n(index.data, 4, "index.data"), _ptr(d_a), _ptr(d_b), _ptr(d_a_offs),
                               _ptr(d_b_tile_offs), nqueries, a_ints, a_tiles, b_tiles, _ptr(d_out), _ptr(d_counts),
                               _ptr(d_scratch), _n(d_scratch, 1, "d_scratch"), _ptr(d_status), _stream(stream)),
           "gc_intersect")


@dataclasses.dataclass
class AndBatch:
    """A batch of AND queries laid out for gc_intersect (device arrays and
    the totals that size its scratch)."""
    qa: np.ndarray         # per query: list decoded whole (the shorter)
    qb: np.ndarray         # per query: list decoded by tile
    aoff: np.ndarray       # per query: first int of its a docIDs and results
    d_a: torch.Tensor
    d_b: torch.Tensor
    d_aoff: torch.Tensor
    d_boff: torch.Tensor
    a_ints: int
    a_tiles: int
    b_tiles: int
    b_ints: int
    d_out: torch.Tensor
    d_counts: torch.Tensor
    scratch: torch.Tensor

    @property
    def nqueries(self) -> int:
        return len(self.qa)


def and_batch(index: Index, pairs) -> AndBatch:
    """Lay out the queries (i, j) of `pairs` for gc_intersect: each query's
    shorter list first, offsets, tile totals, output and scratch buffers."""
    dev = index.data.device
    P = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    nq = len(P)
    L = index.lengths.astype(np.int64)
    li, lj = P[:, 0], P[:, 1]
    swap = L[lj] < L[li]
    qa = np.where(swap, lj, li).astype(np.uint32)
    qb = np.where(swap, li, lj).astype(np.uint32)
    tr = TILE_INTS // index.codec.k

    def tiles(n):
        return ((n + index.codec.k - 1) // index.codec.k + tr - 1) // tr

    na = L[qa]
    tb = tiles(L[qb])
    aoff = np.zeros(nq, np.uint64)
    boff = np.zeros(nq, np.uint64)
    if nq > 1:
        np.cumsum(na[:-1], out=aoff[1:])
        np.cumsum(tb[:-1], out=boff[1:])
    a_ints, a_tiles, b_tiles = int(na.sum()), int(tiles(na).sum()), int(tb.sum())

    def up(x, dt):
        return torch.from_numpy(np.ascontiguousarray(x).view(dt)).to(dev)

    return AndBatch(qa, qb, aoff, up(qa, np.int32), up(qb, np.int32), up(aoff, np.int64), up(boff, np.int64),
                    a_ints, a_tiles, b_tiles, int(L[qb].sum()),
                    torch.empty(max(1, a_ints), dtype=torch.int32, device=dev),
                    torch.zeros(max(1, nq), dtype=torch.int32, device=dev),
                    torch.empty(gc_intersect_scratch_size(a_ints, a_tiles, b_tiles), dtype=torch.uint8, device=dev))


def run_and_batch(index: Index, b: AndBatch, status, stream=None):
    """gc_intersect on a prepared batch (asynchronous)."""
    gc_intersect(index, b.d_a, b.d_b, b.d_aoff, b.d_boff, b.nqueries, b.a_ints, b.a_tiles, b.b_tiles, b.d_out,
                 b.d_counts, b.scratch, status, stream)


def and_batch_tiles(b: AndBatch):
    """(a tiles decoded, b tiles decoded) of the last run (the scratch
    header gc_intersect fills)."""
    h = b.scratch[:32].view(torch.int64).cpu().numpy()
    return int(h[0]), int(h[2])


def intersect(index: Index, pairs, status=None, stream=None, check: bool = True):
    """AND queries over a resident index: for each (i, j) in `pairs`, the
    docIDs in both list i and list j (gc_intersect; each query's shorter list
    is decoded whole, the other only where its skip entries allow a match).
    Returns (results, counts, offsets): query q's docIDs are
    results[offsets[q]:offsets[q] + counts[q]] (uint32 numpy)."""
    b = and_batch(index, pairs)
    st = new_status(index.data.device) if status is None else status
    run_and_batch(index, b, st, stream)
    if check:
        check_status(st, "gc_intersect")
    return as_u32(b.d_out), as_u32(b.d_counts[:b.nqueries]), b.aoff


# ------------------------------------------------ Variable Byte short lists

VB_LIST_BYTES = 24
VB_LIST_DTYPE = np.dtype([("byte_off", "<u8"), ("out_off", "<u8"), ("n", "<u4"), ("nbytes", "<u4")])


def gc_vb_encode_batch(d_gaps, d_in_off, d_n, nlists, d_lists, d_bytes, d_total, stream=None, status=None):
    dev = d_gaps.device
    b = _U64()
    _check(load().gc_vb_encode_batch_scratch_size(nlists, ctypes.byref(b)), "gc_vb_encode_batch_scratch_size")
    scratch = torch.empty(max(256, b.value), dtype=torch.uint8, device=dev)
    st = new_status(dev) if status is None else status
    _check(load().gc_vb_encode_batch(_ptr(d_gaps), _ptr(d_in_off), _ptr(d_n), nlists, _ptr(d_lists), _ptr(d_bytes),
                                     _n(d_bytes, 1, "d_bytes"), _ptr(d_total), _ptr(scratch), scratch.numel(),
                                     _ptr(st), _stream(stream)),
           "gc_vb_encode_batch")
    if status is None:
        check_status(st, "gc_vb_encode_batch")


def gc_vb_decode_batch(d_lists, nlists, d_bytes, d_out, restore_docids, d_status, stream=None):
    if _n(d_lists, 1, "d_lists") < nlists * VB_LIST_BYTES:
        raise ValueError("d_lists: fewer than nlists records")
    _check(load().gc_vb_decode_batch(_ptr(d_lists), nlists, _ptr(d_bytes), _n(d_bytes, 1, "d_bytes"), _ptr(d_out),
                                     _n(d_out, 4, "d_out"), int(bool(restore_docids)), _ptr(d_status),
                                     _stream(stream)),
           "gc_vb_decode_batch")


@dataclasses.dataclass
class MixedIndex:
    """An index whose lists shorter than `vb_below` are Variable Byte (the
    paper's rule for short lists, Section 7.5) and the others a Group codec:
    `group` holds the long lists (None when there are none), the Variable
    Byte pools the short ones; every list decodes to its offset of one
    output."""
    lengths: np.ndarray       # all lists
    out_offsets: np.ndarray   # all lists
    vb_below: int
    group: Index | None
    vb_lists: torch.Tensor    # gc_vb_list records of the short lists
    vb_bytes: torch.Tensor
    n_short: int

    @property
    def out_ints(self) -> int:
        if not len(self.lengths):
            return 0
        return int((self.out_offsets + self.lengths.astype(np.uint64)).max())

    @property
    def total_ints(self) -> int:
        return int(self.lengths.sum(dtype=np.uint64))

    def compressed_bytes(self) -> int:
        g = self.group.compressed_bytes() if self.group is not None else 0
        return g + self.vb_bytes.numel()


def encode_mixed_index(codec: gc_codec, d_gaps: torch.Tensor, lengths, out_offsets=None, vb_below: int = 64,
                       stream=None) -> MixedIndex:
    """Encode lists shorter than vb_below with Variable Byte and the rest
    with `codec` (encode_index); offsets as for encode_index."""
    dev = d_gaps.device
    L = np.ascontiguousarray(lengths, dtype=np.uint32)
    if out_offsets is None:
        out_offsets = np.zeros(len(L), np.uint64)
        if len(L) > 1:
            np.cumsum(L[:-1], dtype=np.uint64, out=out_offsets[1:])
    offs = np.ascontiguousarray(out_offsets, dtype=np.uint64)
    if len(L) and int((offs + L.astype(np.uint64)).max()) > d_gaps.numel():
        raise ValueError("a list runs past the end of d_gaps")
    short = L < vb_below
    group = encode_index(codec, d_gaps, L[~short], out_offsets=offs[~short], stream=stream) if (~short).any() else None
    ns = int(short.sum())
    d_lists = torch.empty(max(1, ns) * VB_LIST_BYTES, dtype=torch.uint8, device=dev)
    cap = 5 * int(L[short].sum(dtype=np.uint64))
    d_bytes = torch.empty(max(16, cap), dtype=torch.uint8, device=dev)
    d_total = torch.zeros(1, dtype=torch.int64, device=dev)
    if ns:
        up = lambda x, dt: torch.from_numpy(np.ascontiguousarray(x).view(dt)).to(dev)
        gc_vb_encode_batch(d_gaps, up(offs[short], np.int64), up(L[short], np.int32), ns, d_lists, d_bytes, d_total,
                           stream)
    nb = int(d_total.item())
    return MixedIndex(L, offs, vb_below, group, d_lists, d_bytes[:max(1, nb)] if ns else d_bytes[:0], ns)


def decode_mixed(mi: MixedIndex, out: torch.Tensor | None = None, restore_docids: bool = True, plan=None,
                 status=None, check: bool = True, stream=None, launch=None) -> torch.Tensor:
    """Decode every list of a mixed index into one output (two launches
    after the plan: the Group decoder and the Variable Byte decoder)."""
    dev = mi.vb_bytes.device
    out = torch.empty(max(1, mi.out_ints), dtype=torch.int32, device=dev) if out is None else out
    st = new_status(dev) if status is None else status
    if mi.group is not None:
        decode_index(mi.group, out=out, restore_docids=restore_docids, status=st, check=False, stream=stream,
                     plan=plan, launch=launch)
    if mi.n_short:
        gc_vb_decode_batch(mi.vb_lists, mi.n_short, mi.vb_bytes, out, restore_docids, st, stream)
    if check:
        check_status(st, "decode_mixed")
    return out

