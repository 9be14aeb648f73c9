"""The C ABI without a GPU: the library builds, loads, exports every call that
include/gc.h declares, and validates arguments on the host (no kernel is
launched by any call made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gc():
    from paper_1502_01916_gb300 import build
    build.build()
    import paper_1502_01916_gb300 as gc
    return gc


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(gc_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gc_encode", "gc_decode", "gc_decode_batch", "gc_build_tiles", "gc_decode_paper",
                 "gc_max_encoded_size", "gc_paper_bytes", "gc_pack_paper", "gc_unpack_paper", "gc_set_launch",
                 "gc_get_launch", "gc_decode_plan_host", "gc_decode_plan_host_buffer_size", "gc_shutdown"):
        assert must in names


@pytest.mark.parametrize("cb,dw", [(0, 0), (1, 0), (11, 3), (12, 8), (13, 4), (100, 1000)])
def test_paper_buffer_size_agrees_with_oracle(gc, cb, dw):
    """The single buffer of Sec 4.3 step 1: head, control, padding, data."""
    rng = np.random.default_rng(cb * 1000 + dw)
    ctrl = rng.integers(0, 256, cb, dtype=np.uint8)
    data = rng.integers(0, 2**32, dw, dtype=np.uint64).astype(np.uint32)
    assert gc.gc_paper_bytes(cb, dw) == len(O.paper_pack(ctrl, data))


def test_shutdown_without_a_device_is_harmless(gc):
    gc.gc_shutdown()
    gc.gc_shutdown()


def test_library_exports_every_declared_symbol(gc):
    lib = ctypes.CDLL(gc.library_path())
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_struct_sizes_match_header(gc):
    assert ctypes.sizeof(gc.gc_codec) == 24
    assert ctypes.sizeof(gc.gc_tile) == 32
    assert ctypes.sizeof(gc.gc_list) == 40
    assert ctypes.sizeof(gc.gc_work) == 64
    assert ctypes.sizeof(gc.gc_launch) == 16
    assert O.TILE_DTYPE.itemsize == 32
    assert gc.TILE_DTYPE == O.TILE_DTYPE
    assert gc.LIST_DTYPE.itemsize == 40 and gc.WORK_DTYPE.itemsize == 64
    for name, _ in gc.gc_work._fields_:
        assert getattr(gc.gc_work, name).offset == gc.WORK_DTYPE.fields[name][1], name


@pytest.mark.parametrize("zeta", [0.0, 0.01, 0.05, 0.1, 0.125, 0.3, 0.5, 0.99, 1.0, 2.0])
def test_zeta_rule_agrees_with_oracle(gc, zeta):
    assert gc.gc_pfd_rows_for_zeta(zeta) == O.pfd_rows_for_zeta(zeta)


@pytest.mark.parametrize("kind,cg,ld", [(0, 8, 0), (1, 1, 0), (1, 2, 1), (1, 4, 2), (1, 8, 2), (2, 8, 0),
                                        (3, 8, 0)])
@pytest.mark.parametrize("k", [4, 32])
def test_size_bounds_cover_oracle(gc, kind, cg, ld, k):
    """The library's worst-case sizes are at least the oracle's."""
    c = gc.make_codec(kind, k, cg, ld, 0.3)
    oc = O.Codec(kind, k, cg, ld, 0.3)
    for n in [0, 1, 7, 1000, 1024, 1025, 123457]:
        cc, dc, nt = gc.gc_max_encoded_size(c, n)
        occ, odc = O.max_sizes(oc, n)
        assert cc >= occ and dc >= odc and cc % 4 == 0
        assert nt == -(-(-(-n // k)) // (1024 // k))


@pytest.mark.parametrize("bad", [dict(k=8), dict(kind=5), dict(kind=1, cg=3), dict(kind=1, cg=2, ld=2),
                                 dict(kind=1, cg=8, ld=3), dict(kind=3, pfd_exc_rows=32),
                                 dict(reserved=1)])
def test_bad_codec_rejected_on_host(gc, bad):
    c = gc.gc_codec(0, 32, 0, 0, 0, 0)
    for key, val in bad.items():
        setattr(c, key, val)
    with pytest.raises(gc.GcError) as ei:
        gc.gc_max_encoded_size(c, 100)
    assert ei.value.code == 1
    lib = gc.load()
    st = lib.gc_decode(ctypes.byref(c), None, 0, None, 0, 10, None, None, 1, None, 0, None, None)
    assert st == 1


def test_decode_rejects_missing_buffers_and_misaligned_data(gc):
    lib = gc.load()
    c = gc.make_codec(gc.SIMPLE, 32)
    buf = (ctypes.c_uint8 * 96)()
    base = (ctypes.addressof(buf) + 15) // 16 * 16
    # NULL output
    assert lib.gc_decode(ctypes.byref(c), base, 4, base, 4, 10, None, None, 1, base, 1 << 20, None, None) == 1
    # data not 16-byte aligned
    mis = base + 4
    assert lib.gc_decode(ctypes.byref(c), base, 4, mis, 4, 10, None, base, 1, base, 1 << 20, None, None) == 1
    # scratch too small
    assert lib.gc_decode(ctypes.byref(c), base, 4, base, 4, 10, None, base, 1, base, 0, None, None) == 2
    # n = 0 is a no-op
    assert lib.gc_decode(ctypes.byref(c), None, 0, None, 0, 0, None, None, 1, None, 0, None, None) == 0
    # the fixed-scratch decoder refuses a list above its limit before any CUDA call
    assert lib.gc_decode_static(ctypes.byref(c), base, 4, base, 4, gc.DECODE_STATIC_MAX_INTS + 1, None, base, 1,
                                None, None) == 2


def test_scratch_sizes(gc):
    c = gc.make_codec(gc.PFD, 32)
    assert gc.gc_decode_scratch_size(c, 1 << 20, True) < gc.gc_decode_scratch_size(c, 1 << 20, False)
    assert gc.gc_decode_batch_scratch_size(10, 1000) >= 2 * 8 * 1000
    lens = np.array([0, 1, 5000, 70000], np.uint32)
    assert gc.gc_encode_batch_scratch_size(c, lens) > 0
    assert gc.gc_version().startswith("gc ")


def test_encode_index_rejects_lists_past_the_gaps(gc):
    """List offsets are also where the encoder reads each list's gaps; a list
    that would run past the gaps buffer is refused before any device call."""
    import torch
    c = gc.make_codec(gc.SIMPLE, 32)
    gaps = torch.zeros(100, dtype=torch.int32)
    with pytest.raises(ValueError):
        gc.encode_index(c, gaps, [40, 40], out_offsets=np.array([0, 64], np.uint64))
    with pytest.raises(ValueError):
        gc.encode_index(c, gaps, [40, 40], out_offsets=np.array([0], np.uint64))


def test_intersect_validates_on_the_host(gc):
    """gc_intersect: no queries is a no-op, missing buffers are refused,
    scratch grows with the work, all before any device call."""
    lib = gc.load()
    c = gc.make_codec(gc.SIMPLE, 32)
    args = [None, 1, None, 0, None, 0, None, 0, None, None, None, None]
    assert lib.gc_intersect(ctypes.byref(c), *args, 0, 0, 0, 0, None, None, None, 0, None, None) == 0
    assert lib.gc_intersect(ctypes.byref(c), *args, 1, 0, 0, 0, None, None, None, 0, None, None) == 1
    s1 = gc.gc_intersect_scratch_size(1000, 2, 10)
    s2 = gc.gc_intersect_scratch_size(100000, 200, 1000)
    assert 0 < s1 < s2


def test_vb_batch_validates_on_the_host(gc):
    """gc_vb_decode_batch / gc_vb_encode_batch: empty batches are no-ops,
    missing buffers are refused, before any device call."""
    lib = gc.load()
    assert lib.gc_vb_decode_batch(None, 0, None, 0, None, 0, 1, None, None) == 0
    assert lib.gc_vb_decode_batch(None, 3, None, 0, None, 0, 1, None, None) == 1
    assert lib.gc_vb_encode_batch(None, None, None, 3, None, None, 0, None, None, 0, None, None) == 1
    buf = (ctypes.c_uint8 * 64)()
    p = ctypes.addressof(buf)
    assert lib.gc_vb_decode_batch(p, 1 << 32, p, 64, p, 16, 1, None, None) == 6  # more lists than uint32 indices
    b = ctypes.c_uint64()
    assert lib.gc_vb_encode_batch_scratch_size(5000, ctypes.byref(b)) == 0 and b.value >= 5000 * 8


def test_binding_refuses_buffers_of_the_wrong_kind(gc):
    """The binding passes buffer sizes in the units the C ABI takes (bytes
    for byte pools, uint32 for words): a buffer of another element size, or
    one not on the GPU, is refused before the library is called."""
    import torch
    c = gc.make_codec(gc.SIMPLE, 32)
    host = torch.zeros(64, dtype=torch.uint8)
    with pytest.raises(ValueError):
        gc.gc_vb_decode_batch(host, 1, host, host, True, None)
    with pytest.raises(ValueError):
        gc.gc_decode(c, host, 4, host, 4, 10, None, host, True, host, None)
    from paper_1502_01916_gb300 import gc as binding
    with pytest.raises(ValueError):
        binding._n(torch.zeros(4, dtype=torch.int64), 4, "d_out")


def test_service_calls_validate_on_the_host(gc):
    """The boundary's service calls refuse bad arguments before any device
    call: a launch shape out of range, a misaligned or short paper buffer, a
    head-less buffer, a misaligned host-decode buffer or one too small."""
    lib = gc.load()
    c = gc.make_codec(gc.PFD, 32)
    for bad in (gc.gc_launch(24, 1, 1), gc.gc_launch(1, 9, 1), gc.gc_launch(1, 1, 33)):
        assert lib.gc_set_launch(ctypes.byref(c), 1, ctypes.byref(bad)) == 1
    buf = (ctypes.c_uint8 * 256)()
    base = (ctypes.addressof(buf) + 15) // 16 * 16
    # paper buffer: misaligned, then too small for head + 20 control bytes + 8 words
    assert lib.gc_pack_paper(base, 20, base, 8, base + 4, 200, None) == 1
    assert lib.gc_pack_paper(base, 20, base, 8, base, gc.gc_paper_bytes(20, 8) - 1, None) == 2
    cb, dw = ctypes.c_uint64(), ctypes.c_uint64()
    assert lib.gc_unpack_paper(base, 3, base, 16, base, 4, ctypes.byref(cb), ctypes.byref(dw), None) == 1
    # host-buffer decode: NULL device buffer, misaligned one, one smaller than it needs
    need = gc.gc_decode_plan_host_buffer_size(10, 64, 64, 1000)
    assert need >= 10 * gc.WORK_BYTES + 64 + 4 * 64 + 4 * 1000
    args = (ctypes.byref(c), base, 10, base, 64, base, 64, base, 1000, 1, None)
    assert lib.gc_decode_plan_host(*args, None, need, None, None) == 1
    assert lib.gc_decode_plan_host(*args, base + 16, need, None, None) == 1
    assert lib.gc_decode_plan_host(*args, (base + 255) // 256 * 256, need - 1, None, None) == 2
    # nothing to decode is a no-op
    assert lib.gc_decode_plan_host(ctypes.byref(c), None, 0, None, 0, None, 0, None, 0, 1, None, None, 0, None,
                                   None) == 0


def test_interleaved_plan_validates_on_the_host(gc):
    lib = gc.load()
    c = gc.make_codec(gc.SIMPLE, 32)
    cnt = (ctypes.c_uint64 * 2)()
    # pairs without selection arrays
    assert lib.gc_plan_interleave(ctypes.byref(c), 1, 4, None, None, 2, None, 0, None, 0, 1, 8,
                                  ctypes.byref(cnt), None, None) == 1
    assert gc.RESTORE_PER_RECORD == 2 and gc.WORK_RAW == 1 << 31
