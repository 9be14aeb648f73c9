"""gc_decode_static: decoding for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: a plug-in or service embedded in a host
application that owns all of the device's memory through its own allocator
(a search server that reserves the GPU's memory at start-up), and
latency-critical code that cannot pay the device-wide synchronisation that
cudaMalloc and cudaFree imply. gc_decode_static serves them with a fixed
scratch array inside the library instead of caller scratch. These tests call
it through the C ABI and check that its docIDs (and raw gaps) equal those of
gc_decode, the entry point that takes caller scratch, and the oracle's, bit
for bit, on two calls in a row on different lists (so that a call never sees
what the previous one left in the shared array); that a call allocates no
device memory; and that a list above its limit is refused before anything
runs.

The file sorts last so that a run which stops at the first failure has run
every other test first; it passes alone in a fresh process as well.
"""
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


def decode_with_scratch(gc, enc, restore, use_tiles):
    return gc.as_u32(gc.decode(enc, restore_docids=restore, use_tiles=use_tiles))


def decode_static(gc, enc, restore, use_tiles):
    """One gc_decode_static call; the output and status buffers are made
    first, and the call itself must leave the device's memory as it was."""
    dev = enc.data.device
    out = torch.empty(max(1, enc.n), dtype=torch.int32, device=dev)
    st = gc.new_status(dev)
    torch.cuda.synchronize(dev)
    held, free = torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0]
    gc.gc_decode_static(enc.codec, enc.ctrl, enc.ctrl_bytes, enc.data, enc.data_words, enc.n,
                        enc.tiles if use_tiles else None, out, restore, st)
    torch.cuda.synchronize(dev)
    assert torch.cuda.memory_allocated(dev) == held
    assert torch.cuda.mem_get_info(dev)[0] == free, "gc_decode_static allocated device memory"
    gc.check_status(st, "gc_decode_static")
    return gc.as_u32(out[:enc.n])


def test_static_scratch_matches_caller_scratch(gc):
    """Three lists of different codecs, layouts and lengths, decoded one
    after the other with the fixed scratch, equal gc_decode's results and the
    oracle's prefix sums (or the gaps themselves)."""
    cases = [
        (gc.make_codec(gc.PFD, 32, zeta=0.1), synth.mixed_runs(41, 300_001, 256, 8.0, 0.1, 1 << 20)),
        (gc.make_codec(gc.SCHEME, 4, cg=1, ld=gc.LD_CU), synth.geometric_gaps(42, gc.DECODE_STATIC_MAX_INTS, 20.0)),
        (gc.make_codec(gc.SIMPLE, 32), synth.geometric_gaps(43, 70_000, 300.0)),
    ]
    oracle_ids = [O.prefix_sum(g) for _, g in cases]
    encs = [gc.encode(c, g) for c, g in cases]
    # the first call on the device looks up the array's address (and may load
    # the library's device code); the memory checks start after it
    enc0 = encs[2]
    out0 = torch.empty(enc0.n, dtype=torch.int32, device=enc0.data.device)
    gc.gc_decode_static(enc0.codec, enc0.ctrl, enc0.ctrl_bytes, enc0.data, enc0.data_words, enc0.n, enc0.tiles,
                        out0, True, None)
    torch.cuda.synchronize()
    for use_tiles in (True, False):
        for restore in (True, False):
            for enc, (_, g), ids in zip(encs, cases, oracle_ids):
                want = decode_with_scratch(gc, enc, restore, use_tiles)
                got = decode_static(gc, enc, restore, use_tiles)
                assert (got == want).all(), (gc.codec_name(enc.codec), use_tiles, restore)
                assert (got == (ids if restore else g)).all(), (gc.codec_name(enc.codec), use_tiles, restore)


def test_static_scratch_refuses_longer_lists(gc):
    """A list above the limit returns GC_ERR_NOSPACE before any work."""
    c = gc.make_codec(gc.SIMPLE, 32)
    dev = torch.device("cuda", 0)
    dummy = torch.zeros(16, dtype=torch.int32, device=dev)
    with pytest.raises(gc.GcError) as ei:
        gc.gc_decode_static(c, dummy, 4, dummy, 4, gc.DECODE_STATIC_MAX_INTS + 1, None, dummy, True, None)
    assert ei.value.code == 2
