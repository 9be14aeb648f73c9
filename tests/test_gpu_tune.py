"""The autotuner on the GPU: it picks one of its candidate shapes, decoding
with that shape gives the oracle's docIDs, and a second call comes from the
cache."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def test_tune_picks_a_shape_that_decodes_right(tmp_path):
    from paper_1502_01916_gb300 import build
    build.build()
    import paper_1502_01916_gb300 as gc
    from paper_1502_01916_gb300.tune import candidates_for, tune
    lens = synth.zipf_index_lengths(3000, 4, 2e5)
    gaps, off = synth.uniform_index(4, lens, 3_000_000)
    idx = gc.encode_index(gc.make_codec(gc.PFD, 32), torch.from_numpy(gaps.view(np.int32).copy()).cuda(), lens)
    path = str(tmp_path / "tune.json")
    launch, info = tune(idx, cache_path=path, reps=2)
    shape = (launch.warps_per_block, launch.blocks_per_sm, launch.items_per_claim, launch.stage_bytes)
    assert not info["cached"] and shape in candidates_for(32)
    want = np.concatenate([O.prefix_sum(gaps[off[i]:off[i + 1]]) for i in range(len(lens))])
    out = gc.decode_index(idx, launch=launch)
    assert (gc.as_u32(out)[:len(gaps)] == want).all()
    launch2, info2 = tune(idx, cache_path=path)
    assert info2["cached"] and (launch2.warps_per_block, launch2.blocks_per_sm, launch2.items_per_claim,
                                launch2.stage_bytes) == shape
    # the pick is registered: a decode given no shape uses it
    got = gc.gc_get_launch(idx.codec, True)
    assert (got.warps_per_block, got.blocks_per_sm, got.items_per_claim, got.stage_bytes) == shape
    out = gc.decode_index(idx)
    assert (gc.as_u32(out)[:len(gaps)] == want).all()
    gc.gc_set_launch(idx.codec, True, None)


def test_choose_k_times_both_widths():
    """choose_k encodes the same lists at k = 4 and k = 32, tunes each and
    reports both; the pick decodes to the oracle's docIDs."""
    from paper_1502_01916_gb300 import build
    build.build()
    import paper_1502_01916_gb300 as gc
    from paper_1502_01916_gb300.tune import choose_k
    lens = synth.zipf_index_lengths(2000, 9, 1e5)
    gaps, off = synth.uniform_index(9, lens, 2_000_000)
    d = torch.from_numpy(gaps.view(np.int32).copy()).cuda()
    try:
        k, by_k = choose_k(gc.SIMPLE, d, lens, reps=1)
        assert k in (4, 32) and set(by_k) == {4, 32}
        for v in by_k.values():
            assert v["ms"] > 0 and 0 < v["bits_per_int"] < 40 and len(v["shape"]) == 4
        idx = gc.encode_index(gc.make_codec(gc.SIMPLE, k), d, lens)
        want = np.concatenate([O.prefix_sum(gaps[off[i]:off[i + 1]]) for i in range(len(lens))])
        assert (gc.as_u32(gc.decode_index(idx))[:len(gaps)] == want).all()
    finally:
        for k in (4, 32):
            gc.gc_set_launch(gc.make_codec(gc.SIMPLE, k), True, None)
