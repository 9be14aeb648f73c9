"""gc_decode_static: decoding for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: code that runs while a stream is being
captured into a CUDA graph (allocation is not allowed during capture), and
latency-critical code that cannot pay the device-wide synchronisation that
cudaMalloc and cudaFree imply. gc_decode_static serves them with a fixed
scratch array inside the library instead of caller scratch. These tests call
it through the C ABI and check that its docIDs (and raw gaps) equal those of
gc_decode, the entry point that takes caller scratch, bit for bit, on two
calls in a row on different lists (so that a call never sees what the
previous one left in the shared array), and that a list above its limit is
refused before anything runs.

The file sorts last so that a run which stops at the first failure has run
every other test first; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    from paper_1502_01916_gb300 import build
    build.build()
    import paper_1502_01916_gb300 as gc
    return gc


def decode_with_scratch(gc, enc, restore, use_tiles):
    return gc.as_u32(gc.decode(enc, restore_docids=restore, use_tiles=use_tiles))


def decode_static(gc, enc, restore, use_tiles):
    dev = enc.data.device
    out = torch.empty(max(1, enc.n), dtype=torch.int32, device=dev)
    st = gc.new_status(dev)
    gc.gc_decode_static(enc.codec, enc.ctrl, enc.ctrl_bytes, enc.data, enc.data_words, enc.n,
                        enc.tiles if use_tiles else None, out, restore, st)
    gc.check_status(st, "gc_decode_static")
    return gc.as_u32(out[:enc.n])


def test_static_scratch_matches_caller_scratch(gc):
    """Two lists of different codecs, layouts and lengths, decoded one after
    the other with the fixed scratch, equal gc_decode's results."""
    cases = [
        (gc.make_codec(gc.PFD, 32, zeta=0.1), synth.mixed_runs(41, 300_001, 256, 8.0, 0.1, 1 << 20)),
        (gc.make_codec(gc.SCHEME, 4, cg=1, ld=gc.LD_CU), synth.geometric_gaps(42, gc.DECODE_STATIC_MAX_INTS, 20.0)),
        (gc.make_codec(gc.SIMPLE, 32), synth.geometric_gaps(43, 70_000, 300.0)),
    ]
    for use_tiles in (True, False):
        for restore in (True, False):
            encs = [gc.encode(c, g) for c, g in cases]
            for enc, (_, g) in zip(encs, cases):
                want = decode_with_scratch(gc, enc, restore, use_tiles)
                got = decode_static(gc, enc, restore, use_tiles)
                assert (got == want).all(), (gc.codec_name(enc.codec), use_tiles, restore)
                if not restore:
                    assert (got == g).all()


def test_static_scratch_refuses_longer_lists(gc):
    """A list above the limit returns GC_ERR_NOSPACE before any work."""
    c = gc.make_codec(gc.SIMPLE, 32)
    dev = torch.device("cuda", 0)
    dummy = torch.zeros(16, dtype=torch.int32, device=dev)
    with pytest.raises(gc.GcError) as ei:
        gc.gc_decode_static(c, dummy, 4, dummy, 4, gc.DECODE_STATIC_MAX_INTS + 1, None, dummy, True, None)
    assert ei.value.code == 2
