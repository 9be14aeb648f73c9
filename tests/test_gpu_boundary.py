"""The boundary's service calls on the GPU, through the C ABI.

- gc_pack_paper / gc_unpack_paper: the single buffer of Sec 4.3 step 1
  built on the device is byte for byte the oracle's, splits back into the
  same areas, and decodes (gc_decode_paper) to the oracle's docIDs.
- gc_set_launch / gc_get_launch / gc_shutdown: a registered shape is what a
  decode call with launch = NULL uses, and it still decodes bit-exact.
- gc_decode_plan_host: a plan and pools in host memory decode to the
  oracle's docIDs (with skip entries, and without them by look-back);
  output ints no record writes come back as 0.
- A look-back that nothing ever completes (a host-built plan whose
  predecessor record never publishes) runs out after its bounded wait and
  reports GC_ERR_TIMEOUT; the launch ends and the context stays usable.

Integer work: bit-exact, no tolerance."""
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


def upload_u32(a):
    a = np.ascontiguousarray(a, np.uint32)
    if a.size == 0:
        a = np.zeros(4, np.uint32)
    return torch.from_numpy(a.view(np.int32).copy()).cuda()


@pytest.mark.parametrize("kind,k", [(0, 4), (0, 32), (3, 4), (3, 32), (2, 32)])
@pytest.mark.parametrize("n", [1, 37, 1024, 65536])
def test_paper_buffer_round_trip(gc, kind, k, n):
    """Sec 4.3 step 1: head | control | zero pad to 16 B | data."""
    oc = O.Codec(kind, k, 8, 0, 0.1)
    gcc = gc.make_codec(kind, k, 8, 0, 0.1)
    g = synth.single_list_geometric(n, 20.0, n + k)
    enc = gc.encode(gcc, upload_u32(g))
    ctrl, data = O.encode(oc, g)
    want = O.paper_pack(ctrl, data)
    buf = gc.pack_paper(enc)
    assert buf.numel() == len(want) == gc.gc_paper_bytes(len(ctrl), len(data))
    assert (buf.cpu().numpy() == want).all()
    c2, d2 = gc.unpack_paper(buf)
    c2, d2 = c2.cpu().numpy(), gc.as_u32(d2)
    assert len(c2) >= len(ctrl) and (c2[:len(ctrl)] == ctrl).all() and not c2[len(ctrl):].any()
    assert len(d2) == len(data) and (d2 == data).all()
    got = gc.as_u32(gc.decode_paper(gcc, buf, n))
    assert (got == O.prefix_sum(g)).all()


def test_unpack_paper_rejects_a_bad_head(gc):
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    buf[0] = 3  # 12 bytes: not on a 16-byte boundary
    with pytest.raises(gc.GcError) as ei:
        gc.unpack_paper(buf)
    assert ei.value.code == 3
    buf[0] = 200  # 800 bytes: past the buffer's end
    with pytest.raises(gc.GcError) as ei:
        gc.unpack_paper(buf)
    assert ei.value.code == 3


def test_pack_paper_refuses_a_short_buffer(gc):
    gcc = gc.make_codec(0, 32)
    enc = gc.encode(gcc, upload_u32(synth.single_list_geometric(5000, 20.0, 1)))
    short = torch.empty(gc.gc_paper_bytes(enc.ctrl_bytes, enc.data_words) - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(gc.GcError) as ei:
        gc.gc_pack_paper(enc.ctrl, enc.ctrl_bytes, enc.data, enc.data_words, short)
    assert ei.value.code == 2


def small_index(gc, seed, kind=0, k=32, nlists=200):
    rng = np.random.default_rng(seed)
    lens = rng.integers(1, 5000, size=nlists).astype(np.uint32)
    lens[:6] = [1, 1023, 1024, 1025, 40000, 3]
    gaps, off = synth.uniform_index(seed, lens, 3_000_000)
    idx = gc.encode_index(gc.make_codec(kind, k, 8, 0, 0.1), upload_u32(gaps), lens)
    want = [O.prefix_sum(gaps[off[i]:off[i + 1]]) for i in range(len(lens))]
    return idx, off, want


def test_registered_launch_shape(gc):
    idx, off, want = small_index(gc, 3)
    c = idx.codec
    try:
        d = gc.gc_get_launch(c, True)
        assert (d.warps_per_block, d.blocks_per_sm, d.items_per_claim) == (7, 3, 32)
        gc.gc_set_launch(c, True, gc.gc_launch(3, 2, 8, 16384))
        r = gc.gc_get_launch(c, True)
        assert (r.warps_per_block, r.blocks_per_sm, r.items_per_claim, r.stage_bytes) == (3, 2, 8, 16384)
        # the other restore flag and the other k keep their defaults
        assert gc.gc_get_launch(c, False).warps_per_block == 7
        assert gc.gc_get_launch(gc.make_codec(0, 4), True).blocks_per_sm == 2
        out = gc.decode_index(idx, launch=None)
        got = gc.as_u32(out)
        for i, w in enumerate(want):
            assert (got[off[i]:off[i] + len(w)] == w).all(), f"list {i}"
        with pytest.raises(gc.GcError):
            gc.gc_set_launch(c, True, gc.gc_launch(99, 1, 1))
        gc.gc_set_launch(c, True, None)
        assert gc.gc_get_launch(c, True).warps_per_block == 7
        gc.gc_set_launch(c, True, gc.gc_launch(5, 2, 4))
        gc.gc_shutdown()  # forgets registered shapes
        assert gc.gc_get_launch(c, True).warps_per_block == 7
        out = gc.decode_index(idx)
        got = gc.as_u32(out)
        for i, w in enumerate(want):
            assert (got[off[i]:off[i] + len(w)] == w).all(), f"list {i} after shutdown"
    finally:
        gc.gc_set_launch(c, True, None)


def host_decode(gc, idx, plan, nwork, restore=True, launch=None):
    work = plan.work.cpu().pin_memory() if nwork else plan.work.cpu()
    ctrl = idx.ctrl.cpu().pin_memory()
    data = idx.data.cpu().pin_memory()
    out = torch.full((max(1, idx.out_ints),), -5, dtype=torch.int32).pin_memory()
    size = gc.gc_decode_plan_host_buffer_size(nwork, ctrl.numel(), data.numel(), out.numel())
    buf = torch.empty(size, dtype=torch.uint8, device="cuda")
    st = gc.new_status()
    gc.gc_decode_plan_host(idx.codec, work, nwork, ctrl, data, out, restore, launch, buf, st)
    torch.cuda.current_stream().synchronize()
    return out, st


@pytest.mark.parametrize("kind,k", [(0, 32), (3, 32), (3, 4), (1, 32)])
def test_decode_from_host_buffers(gc, kind, k):
    idx, off, want = small_index(gc, 11 + kind + k, kind, k)
    plan = gc.plan_index(idx)
    nwork = int(plan.count[0].item())
    out, st = host_decode(gc, idx, plan, nwork)
    gc.check_status(st, "gc_decode_plan_host")
    got = out.numpy().view(np.uint32)
    written = np.zeros(len(got), bool)
    for i, w in enumerate(want):
        assert (got[off[i]:off[i] + len(w)] == w).all(), f"list {i}"
        written[off[i]:off[i] + len(w)] = True
    assert not got[~written].any()
    # raw gaps too
    out, st = host_decode(gc, idx, plan, nwork, restore=False)
    gc.check_status(st, "gc_decode_plan_host (gaps)")
    got = out.numpy().view(np.uint32)
    for i, w in enumerate(want):
        assert (got[off[i]:off[i] + len(w)] == O.dgaps(w)).all(), f"list {i} gaps"


def test_decode_from_host_buffers_by_look_back(gc):
    """The same plan with every base dropped on the host: tiles after a
    list's first take their prefix by look-back (the call recounts them)."""
    idx, off, want = small_index(gc, 29)
    plan = gc.plan_index(idx)
    nwork = int(plan.count[0].item())
    w = plan.work.cpu().numpy().view(gc.WORK_DTYPE)[:nwork].copy()
    w["shape"] &= np.uint32(~(gc.WORK_HAS_BASE | gc.WORK_PUBLISH) & 0xFFFFFFFF)
    w["base"] = 0
    nxt = np.zeros(nwork, bool)
    nxt[:-1] = (w["list"][1:] == w["list"][:-1]) & (w["tile"][1:] > 0)
    w["shape"][nxt] |= np.uint32(gc.WORK_PUBLISH)
    w["shape"][w["tile"] == 0] |= np.uint32(gc.WORK_HAS_BASE)
    assert (w["tile"] > 0).sum() > 50
    plan.work[:nwork * gc.WORK_BYTES] = torch.from_numpy(w.view(np.uint8).reshape(-1)).cuda()
    out, st = host_decode(gc, idx, plan, nwork)
    gc.check_status(st, "gc_decode_plan_host (look-back)")
    got = out.numpy().view(np.uint32)
    for i, ww in enumerate(want):
        assert (got[off[i]:off[i] + len(ww)] == ww).all(), f"list {i}"


def test_look_back_that_never_completes_times_out(gc):
    """A record that waits for a predecessor which never publishes: the
    bounded wait (1 s) runs out, GC_ERR_TIMEOUT is reported, the launch
    ends, and the next decode on the same context is correct."""
    g = synth.single_list_geometric(3000, 20.0, 5)
    idx = gc.encode_index(gc.make_codec(0, 32), upload_u32(g), np.array([len(g)], np.uint32))
    plan = gc.plan_index(idx)
    nwork = int(plan.count[0].item())
    assert nwork == 3
    w = plan.work.cpu().numpy().view(gc.WORK_DTYPE)[:nwork].copy()
    # tile 0 publishes nothing; tile 1 has no base and waits for tile 0
    w["shape"][0] &= np.uint32(~gc.WORK_PUBLISH & 0xFFFFFFFF)
    w["shape"][1] &= np.uint32(~gc.WORK_HAS_BASE & 0xFFFFFFFF)
    bad = plan.work.clone()
    bad[:nwork * gc.WORK_BYTES] = torch.from_numpy(w.view(np.uint8).reshape(-1)).cuda()
    out, st = host_decode(gc, idx, gc.Plan(bad, plan.count), nwork)
    code, where = (int(x) & 0xFFFFFFFF for x in st.cpu().tolist())
    assert code == 5  # GC_ERR_TIMEOUT
    assert where == 0  # the list whose look-back ran out
    # the context is still usable
    out, st = host_decode(gc, idx, plan, nwork)
    gc.check_status(st, "gc_decode_plan_host after a timeout")
    assert (out.numpy().view(np.uint32)[:len(g)] == O.prefix_sum(g)).all()
