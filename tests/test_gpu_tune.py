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
