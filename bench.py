"""Benchmark of the batched Group-codec decode path on one GB300 (or N, as
independent replicas).

Workload (default): a synthetic inverted index of 1,000,000 posting lists
over a 25M-document universe, rank-law (Zipf s = 1.1) lengths clipped to
[1, 2^22] (1.5e9 docIDs), each list a sorted uniform sample. The index is
encoded on the GPU with Group-Simple and Group-PFD (zeta = 0.1), both with
the k = 32 vertical layout. Each list's docIDs go to a 16-byte aligned
offset of the output (at most 3 ints of padding per list). One step decodes the whole index once per codec
and restores docIDs (fused prefix sum): one CUDA-graph launch per codec.

Prints one JSON line: decoded ints/s (all codecs, all ranks), the roofline of
the decode kernel, the end-to-end rate through the C ABI with host buffers
(gc_decode_plan_host), the one-launch-per-list rate, the CPU oracle baseline
and the SM clocks. Beside the headline, after its timed region and each
checked against the host's prefix sums on its own: the single 65,536-docID
list (latency, with its tile index and as the paper's single buffer), the
2^26-gap list for every codec variant at k = 4 and k = 32, the headline
index decoded without skip entries (decoupled look-back on the timed path),
k = 4 against k = 32 on the headline lists, the clustered short-list index
(zeta sweep, Group-Scheme 8-IU and 8-B, with and without Variable Byte),
AND queries, TF streams and the serving loop at three request rates against
one launch per list.
`--impl reference` times the CPU oracle instead (the slow reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

UNIVERSE = 25_000_000
CODECS = {"simple": (0, "Group-Simple"), "pfd": (3, "Group-PFD")}
# DRAM traffic of one decode launch, measured by ncu (dram__bytes_read.sum,
# dram__bytes_write.sum) on the small Zipf index (100,000 lists,
# C = 3.0406e7, 1.8e8 docIDs), with the hash of the kernel sources it was
# taken on: the reads per algorithmic read (the compressed streams and the
# plan; the decoder reads each byte once, so reads grow in proportion), and
# the docID bytes the launch's writes fell short by (the docIDs still in L2
# when it ends: a fixed amount, about half of the L2). The full-size launch's
# traffic is reported as its algorithmic reads times that ratio plus its
# docID bytes less that shortfall; once the sources change, null.
# Multi-metric captures of the full-size workload are not taken.
NCU_TRAFFIC_RATIO = {
    "simple": {"read": 350758912 / 348266713, "write_short": 724566460 - 668499456, "hash": "b7fafb21786a88f5"},
    "pfd": {"read": 283119360 / 280634604, "write_short": 724566460 - 665709056, "hash": "b7fafb21786a88f5"},
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--nlists", type=int, default=1_000_000)
    p.add_argument("--zipf-c", type=float, default=0.0,
                   help="C of the rank law L_r = C r^-1.1 (0 = the 1.5e9-posting index); a smaller C makes "
                        "the small case that ncu captures")
    p.add_argument("--codecs", default="simple,pfd")
    p.add_argument("--k", type=int, default=32)
    p.add_argument("--zeta", type=float, default=0.10)
    p.add_argument("--warps", type=int, default=0, help="warps per block (0 = library default)")
    p.add_argument("--bps", type=int, default=0, help="blocks per SM (0 = as many as fit)")
    p.add_argument("--claim", type=int, default=0, help="plan records per claim (0 = library default)")
    p.add_argument("--stage", type=int, default=0, help="staging ring bytes per block (0 = all that fits)")
    p.add_argument("--no-tune", action="store_true", help="library default launch shape instead of the autotuner's")
    p.add_argument("--no-verify", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-per-list", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the TF-stream and zeta = 0 decodes")
    p.add_argument("--no-and", action="store_true", help="skip the AND-query measurement")
    p.add_argument("--no-short", action="store_true", help="skip the short-list (Variable Byte rule) measurement")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the single-list, 2^26-list and look-back measurements")
    p.add_argument("--no-k-choice", action="store_true", help="skip timing the index at k = 4 against k = 32")
    p.add_argument("--and-queries", type=int, default=4000, help="two-list AND queries in the timed batch")
    p.add_argument("--serve-seconds", type=float, default=2.0, help="trace length per request rate")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="seconds of oracle work per codec")
    return p.parse_args()


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("gc_decode.cu", "gc_device.cuh"):
        with open(os.path.join(ROOT, "paper_1502_01916_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def workload(nlists: int, zipf_c: float = 0.0):
    """(gaps, starts, lengths): list i is gaps[starts[i]:starts[i] + lengths[i]],
    every start a multiple of 4 ints, zeros between lists; starts[-1] is the
    layout's length."""
    import synth
    gaps, off, lengths = synth.zipf_index(nlists, UNIVERSE, 0, C=zipf_c or synth.ZIPF_C, align=4)
    return gaps, off, lengths


def workload_name(a) -> str:
    c = f", C={a.zipf_c:g}" if a.zipf_c else ""
    return (f"zipf-index: {a.nlists} lists, universe {UNIVERSE}, Zipf(1.1) lengths in [1, 2^22]{c}, "
            f"uniform docIDs; k={a.k}; batched persistent decode + docID prefix sum")


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return parse_clocks(out)


def parse_clocks(out: str):
    """The clocks object of the JSON line from nvidia-smi's CSV samples
    (ClockSampler.FIELDS, no header, no units): median SM clock, the largest
    maximum clock seen, and every throttle reason seen active. None without
    a sample."""
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx = max(mx, float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU baseline

def cpu_oracle_rate(lengths, kinds, k, zeta, seconds, seed=7):
    """The CPU oracle (single-threaded C, as it stands) decoding and
    restoring docIDs for a random sample of lists of the same workload.
    Returns (ints/s, sample description)."""
    import oracle as O
    import synth
    rng = np.random.default_rng(seed)
    # about seconds * 13e6 ints per codec: lists drawn uniformly at random
    work = int(seconds * 13e6)
    order = rng.permutation(len(lengths))
    cum = np.cumsum(lengths[order].astype(np.int64))
    m = int(np.searchsorted(cum, work)) + 1
    L = lengths[order[:m]]
    gaps, off = synth.uniform_index(seed, L, UNIVERSE)
    tot_ints, tot_s = 0, 0.0
    for kind in kinds:
        c = O.Codec(kind, k, zeta=zeta)
        encs = [O.encode(c, gaps[off[i]:off[i + 1]]) for i in range(m)]
        t0 = time.perf_counter()
        for i, (cc, dd) in enumerate(encs):
            O.prefix_sum(O.decode(c, cc, dd, int(L[i])))
        tot_s += time.perf_counter() - t0
        tot_ints += int(L.sum())
    desc = (f"{m} lists drawn at random from the workload's length distribution "
            f"({int(L.sum())} ints per codec, {len(kinds)} codec(s)), docIDs by the same recipe; "
            f"oracle decode + prefix sum, 1 thread")
    return tot_ints / tot_s, desc, tot_s


def _oracle_worker(seed, L, kinds, k, zeta):
    """One host process's share of the parallel oracle run: its lists' gaps,
    encoded by the oracle, then decoded with docIDs restored, timed.
    Returns (ints decoded, seconds)."""
    import oracle as O
    import synth
    gaps, off = synth.uniform_index(seed, L, UNIVERSE, threads=1)
    ints, secs = 0, 0.0
    for kind in kinds:
        c = O.Codec(kind, k, zeta=zeta)
        encs = [O.encode(c, gaps[off[i]:off[i + 1]]) for i in range(len(L))]
        t0 = time.perf_counter()
        for i, (cc, dd) in enumerate(encs):
            O.prefix_sum(O.decode(c, cc, dd, int(L[i])))
        secs += time.perf_counter() - t0
        ints += int(L.sum())
    return ints, secs


def cpu_oracle_rate_parallel(lengths, kinds, k, zeta, seconds, seed=9, workers=None):
    """The same oracle on every host core at once: a random sample of the
    workload's lists split over `workers` spawned processes (one per core),
    each decoding its share; the rate is all ints over the slowest share's
    time. Returns (ints/s, sample description, cores)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    workers = workers or os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    work = int(seconds * 13e6) * workers
    order = rng.permutation(len(lengths))
    cum = np.cumsum(lengths[order].astype(np.int64))
    m = int(np.searchsorted(cum, work)) + 1
    chunks = np.array_split(order[:m], workers)
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(_oracle_worker, seed * 1000 + w, lengths[ch], kinds, k, zeta)
                for w, ch in enumerate(chunks) if len(ch)]
        res = [f.result() for f in futs]
    ints = sum(r[0] for r in res)
    slowest = max(r[1] for r in res)
    desc = (f"{m} lists drawn at random from the workload's length distribution, split over {len(res)} "
            f"processes ({ints // len(kinds)} ints per codec, {len(kinds)} codec(s)); oracle decode + prefix sum, "
            f"rate = all ints / the slowest process's decode time")
    return ints / slowest, desc, len(res)


def reference_arm(a, rank, world):
    """--impl reference: the CPU oracle, timed on the host cores."""
    if rank != 0:
        return
    import synth
    lengths = synth.zipf_index_lengths(a.nlists, 0, a.zipf_c or synth.ZIPF_C)
    kinds = [CODECS[c][0] for c in a.codecs.split(",")]
    # decode seconds per step (each process also encodes its share first, a
    # few times longer): the default 10 + 3 steps end within about 3 minutes
    per_step = max(0.5, min(4.0, 40.0 / max(1, a.steps + a.warmup)))
    for _ in range(a.warmup):
        cpu_oracle_rate_parallel(lengths, kinds, a.k, a.zeta, per_step / len(kinds) / 4, seed=11)
    rates, secs = [], []
    desc, cores = "", 1
    for s in range(a.steps):
        t0 = time.perf_counter()
        r, desc, cores = cpu_oracle_rate_parallel(lengths, kinds, a.k, a.zeta, per_step / len(kinds), seed=100 + s)
        rates.append(r)
        secs.append(time.perf_counter() - t0)
    value = float(np.mean(rates))
    line = {
        "impl": "reference", "metric": "decoded uint32/s (batched index decode + docID prefix sum)",
        "value": value, "unit": "ints/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_name(a), "codecs": a.codecs, "k": a.k},
        "cpu_baseline": {"value": value, "unit": "ints/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "ints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return reference_arm(a, rank, world)

    import torch
    import torch.distributed as dist

    from paper_1502_01916_gb300 import build as gcbuild
    if local == 0:
        gcbuild.build()
    else:
        # the other ranks of this node load what local rank 0 builds (two
        # builds at once would write the same object files)
        deadline = time.time() + 900
        while not os.path.exists(gcbuild.LIB) and time.time() < deadline:
            time.sleep(1.0)
    import paper_1502_01916_gb300 as gc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    t0 = time.time()
    gaps, off, lengths = workload(a.nlists, a.zipf_c)
    t_gen = time.time() - t0
    total_ints = int(lengths.sum(dtype=np.uint64))  # decoded ints
    out_len = int(off[-1])                            # output ints, padding included
    d_gaps = torch.from_numpy(gaps.view(np.int32)).to(dev)
    kinds = [c for c in a.codecs.split(",")]
    idxs = {}
    t0 = time.time()
    for name in kinds:
        codec = gc.make_codec(CODECS[name][0], a.k, zeta=a.zeta)
        idxs[name] = gc.encode_index(codec, d_gaps, lengths, out_offsets=off[:-1])
    plans = {n: gc.plan_index(idx) for n, idx in idxs.items()}
    torch.cuda.synchronize()
    t_enc = time.time() - t0
    del d_gaps
    torch.cuda.empty_cache()

    out = torch.empty(out_len, dtype=torch.int32, device=dev)
    scratch = {n: torch.empty(gc.gc_decode_plan_scratch_size(i.max_tiles), dtype=torch.uint8, device=dev)
               for n, i in idxs.items()}
    status = {n: gc.new_status(dev) for n in idxs}
    # launch shape per codec: given on the command line, the library default,
    # or the autotuner's choice (timed on this index, before the timed region)
    launches_cfg, tuned = {}, {}
    for n, idx in idxs.items():
        if a.warps or a.bps or a.claim or a.stage:
            launches_cfg[n] = gc.gc_launch(a.warps, a.bps, a.claim, a.stage)
        elif a.no_tune:
            launches_cfg[n] = None
        else:
            from paper_1502_01916_gb300.tune import tune
            launches_cfg[n], info = tune(idx, plans[n], use_cache=False)
            tuned[n] = {"shape": [launches_cfg[n].warps_per_block, launches_cfg[n].blocks_per_sm,
                                  launches_cfg[n].items_per_claim, launches_cfg[n].stage_bytes], "ms": info["ms"]}

    # correctness at full size: every docID against the host's prefix sums
    # (the zeros between lists leave the running sum unchanged), and the
    # padding between lists untouched
    verified = None
    if not a.no_verify:
        cs = np.cumsum(gaps, dtype=np.uint32)
        base = np.where(off[:-1] > 0, cs[np.maximum(off[:-1].astype(np.int64) - 1, 0)], 0).astype(np.uint32)
        want = cs - np.repeat(base, np.diff(off).astype(np.int64))
        del cs
        npad = (off[1:] - off[:-1] - lengths).astype(np.int64)
        first = (off[:-1] + lengths).astype(np.int64)
        pad = np.repeat(first - (np.cumsum(npad) - npad), npad) + np.arange(int(npad.sum()), dtype=np.int64)
        sentinel = np.uint32(0x9E3779B9)
        want[pad] = sentinel
        verified = True
        for n, idx in idxs.items():
            out.fill_(int(sentinel.view(np.int32)))
            gc.decode_index(idx, out=out, scratch=scratch[n], status=status[n], launch=launches_cfg[n],
                            plan=plans[n])
            if not np.array_equal(gc.as_u32(out), want):
                verified = False
                print(f"VERIFY FAILED for {n}", file=sys.stderr)
        del want, pad
        if not verified:
            raise SystemExit("decoded docIDs differ from the input's prefix sums")

    # one CUDA graph per codec: zero the queue and the look-back words, decode
    stream = torch.cuda.Stream(device=dev)
    graphs, launches = {}, {}
    for n, idx in idxs.items():
        with torch.cuda.stream(stream):
            gc.decode_index(idx, out=out, scratch=scratch[n], status=status[n], launch=launches_cfg[n], check=False,
                            plan=plans[n])
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
            gc.decode_index(idx, out=out, scratch=scratch[n], status=status[n], launch=launches_cfg[n], check=False,
                            plan=plans[n])
        launches[n] = gc.gc_last_launch_count()
        graphs[n] = g
    torch.cuda.synchronize()

    def step():
        for n in idxs:
            graphs[n].replay()

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    cur = torch.cuda.current_stream()
    ev = {n: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(a.steps)] for n in idxs}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for s in range(a.steps):
        for n in idxs:
            ev[n][s][0].record(cur)
            graphs[n].replay()
            ev[n][s][1].record(cur)
    e1.record(cur)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    elapsed_ms = e0.elapsed_time(e1)
    for n in idxs:
        gc.check_status(status[n], f"decode {n}")
    if world > 1:
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    ints_per_step = total_ints * len(idxs)
    value = ints_per_step * a.steps * world / (elapsed_ms / 1e3)

    # roofline of each codec's decode launch (algorithmic bytes / duration)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    per_codec = {}
    for n, idx in idxs.items():
        ms = float(np.mean([s.elapsed_time(e) for s, e in ev[n]]))
        comp = idx.compressed_bytes()
        alg = comp + plans[n].nbytes() + 4 * total_ints
        per_codec[n] = {"ms_per_launch": ms, "ints_per_s": total_ints / (ms / 1e3),
                        "algorithmic_bytes": alg, "compressed_bytes": comp,
                        "bits_per_int": 8.0 * comp / total_ints, "plan_bytes": plans[n].nbytes(),
                        "tiles": idx.max_tiles, "achieved_gbs": alg / (ms / 1e3) / 1e9,
                        "frac": alg / (ms / 1e3) / 1e9 / peak, "launches_per_graph": launches[n]}
    dom = max(per_codec, key=lambda n: per_codec[n]["ms_per_launch"])
    kh = kernel_hash()
    ratio = NCU_TRAFFIC_RATIO.get(dom)
    traffic, traffic_source = None, "none: no ncu capture of these kernel sources"
    if ratio and ratio.get("hash") == kh and a.k == 32 and a.zeta == 0.10:
        wr = 4 * total_ints
        traffic = ratio["read"] * (per_codec[dom]["algorithmic_bytes"] - wr) + max(0, wr - ratio["write_short"])
        traffic_source = ("ncu dram__bytes_read.sum and dram__bytes_write.sum on the 1.8e8-docID Zipf index: "
                          f"reads {ratio['read']:.4f} of its algorithmic reads, scaled to this launch's; writes "
                          f"this launch's docIDs less the {ratio['write_short'] / 1e6:.0f} MB that launch still "
                          "held in L2 when it ended")
    roofline = {"bound": "hbm", "kernel": f"k_decode<{CODECS[dom][1]}, k={a.k}, batched>",
                "bytes_per_launch": per_codec[dom]["algorithmic_bytes"],
                "achieved": per_codec[dom]["achieved_gbs"], "peak": peak, "unit": "GB/s",
                "frac": per_codec[dom]["frac"], "traffic": traffic, "traffic_source": traffic_source,
                "peak_source": peak_src,
                "timed_as": "graph launch (memset of the queue counter and look-back words + decode kernel)"}

    def list_ids(i):
        return np.cumsum(gaps[int(off[i]):int(off[i]) + int(lengths[i])], dtype=np.uint32)

    rng_s = np.random.default_rng(23)
    sample = rng_s.choice(len(lengths), min(300, len(lengths)), replace=False).tolist()
    sample += np.argsort(lengths)[-3:].tolist()  # and the longest lists

    # end to end through the C ABI with host buffers: every step hands each
    # codec's plan, pools and output, all in page-locked host memory, to
    # gc_decode_plan_host, which copies them in, decodes and copies the
    # docIDs back out on its stream; the two codecs use two streams, so one
    # codec's copies overlap the other's decode.
    e2e = None
    if not a.no_e2e:
        hbuf, dbuf, sts = {}, {}, {}
        h2d = 0
        for n, idx in idxs.items():
            nwork = int(plans[n].count[0].item())
            hw = torch.empty(nwork * gc.WORK_BYTES, dtype=torch.uint8, pin_memory=True)
            hw.copy_(plans[n].work[:nwork * gc.WORK_BYTES])
            hc = torch.empty(idx.ctrl.shape, dtype=idx.ctrl.dtype, pin_memory=True)
            hc.copy_(idx.ctrl)
            hd = torch.empty(idx.data.shape, dtype=idx.data.dtype, pin_memory=True)
            hd.copy_(idx.data)
            ho = torch.empty(out_len, dtype=torch.int32, pin_memory=True)
            hbuf[n] = (hw, nwork, hc, hd, ho)
            h2d += hw.numel() + hc.numel() + 4 * hd.numel()
            size = gc.gc_decode_plan_host_buffer_size(nwork, hc.numel(), hd.numel(), out_len)
            dbuf[n] = torch.empty(size, dtype=torch.uint8, device=dev)
            sts[n] = torch.cuda.Stream(device=dev)
        d2h = 4 * out_len * len(idxs)
        torch.cuda.synchronize()

        def e2e_step():
            for n, idx in idxs.items():
                hw, nwork, hc, hd, ho = hbuf[n]
                gc.gc_decode_plan_host(idx.codec, hw, nwork, hc, hd, ho, True, launches_cfg[n], dbuf[n], status[n],
                                       sts[n])

        for _ in range(max(1, min(a.warmup, 2))):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(cur)
        for st_ in sts.values():
            st_.wait_event(f0)
        ksteps = max(1, min(a.steps, 5))
        for _ in range(ksteps):
            e2e_step()
        for st_ in sts.values():
            e = torch.cuda.Event()
            e.record(st_)
            cur.wait_event(e)
        f1.record(cur)
        torch.cuda.synchronize()
        barrier()
        ems = f0.elapsed_time(f1)
        if world > 1:
            t = torch.tensor([ems], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        ok = True
        for n in idxs:
            gc.check_status(status[n], f"e2e decode {n}")
            got = hbuf[n][4].numpy().view(np.uint32)
            ok = ok and all(np.array_equal(got[int(off[i]):int(off[i]) + int(lengths[i])], list_ids(i))
                            for i in sample)
        e2e = {"value": ints_per_step * ksteps * world / (ems / 1e3), "unit": "ints/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": ksteps,
               "api": "gc_decode_plan_host (plan, pools and output in page-locked host memory), one stream per codec",
               "sample_verified": bool(ok), "sample_lists": len(sample)}
        del hbuf, dbuf

    # one launch per list (gc_decode on each list of a sample)
    per_list = None
    if not a.no_per_list:
        per_list = per_list_rate(gc, idxs, lengths, dev)

    # the other workloads' single-list paths and the headline index without
    # skip entries (look-back on the timed path)
    configs = None
    if not a.no_configs:
        configs = {"single_list_65536": single_list_latency(gc, dev, peak),
                   "mixed_2_26": mixed_list_rates(gc, dev, peak),
                   "lookback": lookback_rate(gc, idxs[dom], plans[dom], out, peak, total_ints, off, lengths,
                                             list_ids, sample)}

    # k = 4 against k = 32 on the same lists (the autotuner's index-build choice)
    k_choice = None
    if not a.no_k_choice and a.k == 32:
        k_choice = k_choice_rates(gc, gaps, lengths, off, dev, [CODECS[n][0] for n in idxs])

    # serving: continuous batching over the resident index, Poisson arrivals
    serving = None
    if not a.no_serving:
        sn = "pfd" if "pfd" in idxs else next(iter(idxs))
        serving = serving_rates(gc, idxs[sn], list_ids, a.serve_seconds, launch=launches_cfg[sn])

    # AND queries over the resident index (skip entries bound what is decoded)
    and_q = None
    if not a.no_and:
        sn = "pfd" if "pfd" in idxs else next(iter(idxs))
        and_q = and_query_rates(gc, idxs[sn], lengths, off, gaps, dev, a.and_queries)

    # the clustered short-list index with and without Variable Byte for
    # lists shorter than 64
    short = None
    if not a.no_short:
        short = short_list_rates(gc, dev)

    # TF streams and Group-PFD without exceptions (BP128's fixed-width frames),
    # after the timed region
    extras = None
    if not a.no_extras:
        extras = extra_rates(gc, lengths, off, gaps, dev, peak,
                             ids_ms={n: per_codec[n]["ms_per_launch"] for n in per_codec})

    cpu = None
    if not a.no_cpu_baseline and rank == 0 and world == 1:
        kinds_id = [CODECS[n][0] for n in idxs]
        r1, desc1, _ = cpu_oracle_rate(lengths, kinds_id, a.k, a.zeta, a.cpu_seconds / 3 / len(kinds_id))
        rn, descn, cores = cpu_oracle_rate_parallel(lengths, kinds_id, a.k, a.zeta,
                                                    2 * a.cpu_seconds / 3 / len(kinds_id))
        cpu = {"value": rn, "unit": "ints/s", "cores": cores, "kind": "oracle", "sample": descn,
               "single_thread": {"value": r1, "unit": "ints/s", "cores": 1, "sample": desc1}}

    line = {
        "metric": "decoded uint32/s (batched index decode + docID prefix sum)",
        "value": value, "unit": "ints/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": elapsed_ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_name(a), "nlists": a.nlists, "ints": total_ints,
                   "codecs": [CODECS[n][1] + (f" zeta={a.zeta}" if n == "pfd" else "") for n in idxs],
                   "k": a.k, "l2": "inputs and outputs larger than L2 (no flush)",
                   "output": f"each list at a 16-byte aligned offset ({out_len - total_ints} padding ints)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "launch": ({n: {"warps_per_block": l.warps_per_block, "blocks_per_sm": l.blocks_per_sm,
                                   "items_per_claim": l.items_per_claim, "stage_bytes": l.stage_bytes}
                               if l is not None else "library default"
                               for n, l in launches_cfg.items()}),
                   "autotuned": tuned or None,
                   "plan": "work plan (64 B per tile) built once per resident index, outside the timed region"},
        "roofline": roofline, "per_codec": per_codec, "e2e": e2e, "per_list_launch": per_list, "serving": serving,
        "configs": configs, "k_choice": k_choice, "extras": extras, "and_queries": and_q, "short_lists": short,
        "cpu_baseline": cpu, "clocks": clk,
        "gpu_launches": int(sum(launches.values()) * a.steps),
        "verified_full_output": verified, "setup_s": {"generate": t_gen, "encode": t_enc},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def extra_rates(gc, lengths, off, gaps, dev, peak, ids_ms=None, reps=5, nsample=300, seed=5):
    """Decode rates beyond the main workload, each on the same lists and
    output layout, timed like the main decode (CUDA events, library default
    launch shape) and checked on a random sample of lists:
    - tf_<codec>: term-frequency streams (values >= 1, geometric with mean 2),
      decoded without the prefix sum (restore_docids = 0);
    - bp_k<k>: Group-PFD with no exception rows (zeta = 0), i.e. SIMD-BP128's
      fixed-width frames (Sec 6.3), on the d-gaps, docIDs restored; k = 4 is
      the paper's 128-int frame, k = 32 the GPU layout;
    - tf_interleaved_<codec>: each list's docIDs and TFs from one index
      (d-gap lists, then TF lists) in one launch, the two streams' tiles
      planned alternately (gc_plan_interleave, restore_docids =
      GC_RESTORE_PER_RECORD), against the two decodes apart (the headline's
      docID decode + the tf_<codec> decode)."""
    import torch
    import synth
    rng = np.random.default_rng(seed)
    ids = rng.choice(len(lengths), min(nsample, len(lengths)), replace=False)
    total = int(lengths.sum(dtype=np.uint64))

    def run(idx, restore, want):
        plan = gc.plan_index(idx)
        out = torch.empty(max(1, idx.out_ints), dtype=torch.int32, device=dev)
        scratch = torch.empty(gc.gc_decode_plan_scratch_size(idx.max_tiles), dtype=torch.uint8, device=dev)
        st = gc.new_status(dev)
        for _ in range(3):
            gc.decode_index(idx, out=out, restore_docids=restore, scratch=scratch, status=st, plan=plan, check=False)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gc.decode_index(idx, out=out, restore_docids=restore, scratch=scratch, status=st, plan=plan, check=False)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        gc.check_status(st, "extra decode")
        got = gc.as_u32(out)
        ok = all(np.array_equal(got[int(off[i]):int(off[i]) + int(lengths[i])], want(i)) for i in ids)
        ms = float(np.median(ts))
        alg = idx.compressed_bytes() + plan.nbytes() + 4 * total
        return {"ms_per_launch": ms, "ints_per_s": total / (ms / 1e3), "bits_per_int": 8.0 * idx.compressed_bytes() / total,
                "achieved_gbs": alg / (ms / 1e3) / 1e9, "frac": alg / (ms / 1e3) / 1e9 / peak, "sample_verified": ok}

    res = {"lists_verified": len(ids)}
    tfs, _ = synth.tf_index(21, lengths, 2.0, align=4)
    d = torch.from_numpy(tfs.view(np.int32)).to(dev)
    for name, kind in (("simple", CODECS["simple"][0]), ("pfd", CODECS["pfd"][0])):
        idx = gc.encode_index(gc.make_codec(kind, 32, zeta=0.10), d, lengths, out_offsets=off[:-1])
        res[f"tf_{name}"] = run(idx, False, lambda i: tfs[int(off[i]):int(off[i]) + int(lengths[i])])
        del idx
    # docIDs and TFs interleaved: one index of both streams, one launch
    L, N = int(off[-1]), len(lengths)
    both = torch.cat([torch.from_numpy(gaps.view(np.int32)).to(dev), d])
    del d
    starts = np.concatenate([off[:-1], L + off[:-1]]).astype(np.uint64)
    pairs = np.stack([np.arange(N), N + np.arange(N)], axis=1)
    out2 = torch.empty(2 * L, dtype=torch.int32, device=dev)
    for name, kind in (("simple", CODECS["simple"][0]), ("pfd", CODECS["pfd"][0])):
        idx = gc.encode_index(gc.make_codec(kind, 32, zeta=0.10), both, np.concatenate([lengths, lengths]),
                              out_offsets=starts)
        plan = gc.plan_interleave(idx, pairs, starts.reshape(2, N).T)
        scratch = torch.empty(gc.gc_decode_plan_scratch_size(int(plan.count[0].item())), dtype=torch.uint8,
                              device=dev)
        st = gc.new_status(dev)
        ms = _timed(lambda: gc.decode_index(idx, out=out2, restore_docids=gc.RESTORE_PER_RECORD, scratch=scratch,
                                            status=st, plan=plan, check=False), reps=reps)
        gc.check_status(st, "interleaved decode")
        got = gc.as_u32(out2)
        ok = all(np.array_equal(got[int(off[i]):int(off[i]) + int(lengths[i])],
                                np.cumsum(gaps[int(off[i]):int(off[i]) + int(lengths[i])], dtype=np.uint32)) and
                 np.array_equal(got[L + int(off[i]):L + int(off[i]) + int(lengths[i])],
                                tfs[int(off[i]):int(off[i]) + int(lengths[i])]) for i in ids)
        alg = idx.compressed_bytes() + plan.nbytes() + 8 * total
        sep = (ids_ms or {}).get(name)
        res[f"tf_interleaved_{name}"] = {
            "ms_per_launch": ms, "ints_per_s": 2 * total / (ms / 1e3), "achieved_gbs": alg / (ms / 1e3) / 1e9,
            "frac": alg / (ms / 1e3) / 1e9 / peak, "sample_verified": bool(ok),
            "apart_ms": (sep + res[f"tf_{name}"]["ms_per_launch"]) if sep else None}
        del idx, plan, scratch
    del both, out2, tfs
    d = torch.from_numpy(gaps.view(np.int32)).to(dev)
    for k in (4, 32):
        idx = gc.encode_index(gc.make_codec(CODECS["pfd"][0], k, zeta=0.0), d, lengths, out_offsets=off[:-1])
        res[f"bp_k{k}"] = run(idx, True, lambda i: np.cumsum(gaps[int(off[i]):int(off[i]) + int(lengths[i])],
                                                              dtype=np.uint32))
        del idx
    del d
    torch.cuda.empty_cache()
    return res


def short_list_rates(gc, dev, reps=5, nsample=300, seed=17):
    """The clustered short-list index (4M lists over 50M documents,
    log-normal lengths with median 12, clustered docIDs; 87% of the lists
    shorter than 64), encoded with Group-PFD at zeta 0.01, 0.1 and 0.3 and
    with Group-Scheme at byte granularity (incomplete unary and binary
    descriptors), each alone and with the paper's rule for short lists
    (Variable Byte below 64 postings, Sec 7.5): compressed bits per int and
    the decode time of the whole index (CUDA events; the plan of the Group
    part built beforehand), checked on a sample of lists."""
    import torch
    import synth
    gaps, off, lens = synth.clustered_short_index()
    total = int(lens.sum(dtype=np.uint64))
    d = torch.from_numpy(gaps.view(np.int32)).to(dev)
    rng = np.random.default_rng(seed)
    ids = rng.choice(len(lens), min(nsample, len(lens)), replace=False)
    out = torch.empty(max(1, total), dtype=torch.int32, device=dev)
    st = gc.new_status(dev)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        gc.check_status(st, "short lists")
        got = gc.as_u32(out)
        ok = all(np.array_equal(got[int(off[i]):int(off[i + 1])],
                                np.cumsum(gaps[int(off[i]):int(off[i + 1])], dtype=np.uint32)) for i in ids)
        return float(np.median(ts)), ok

    res = {"lists": int(len(lens)), "ints": total, "short_share": float((lens < 64).mean())}
    for name, kind, kw in (("pfd_z0.01", 3, {"zeta": 0.01}), ("pfd", 3, {"zeta": 0.10}), ("pfd_z0.3", 3, {"zeta": 0.30}),
                           ("scheme_iu_cg8", 1, {"cg": 8, "ld": gc.LD_IU}),
                           ("scheme_b_cg8", 1, {"cg": 8, "ld": gc.LD_BINARY})):
        codec = gc.make_codec(kind, 32, **kw)
        idx = gc.encode_index(codec, d, lens)
        plan = gc.plan_index(idx)
        scratch = torch.empty(gc.gc_decode_plan_scratch_size(idx.max_tiles), dtype=torch.uint8, device=dev)
        ms, ok = timed(lambda: gc.decode_index(idx, out=out, scratch=scratch, status=st, plan=plan, check=False))
        res[name] = {"bits_per_int": 8.0 * (idx.compressed_bytes() + idx.index_bytes()) / total, "ms": ms,
                     "ints_per_s": total / (ms / 1e3), "sample_verified": ok}
        if name == "pfd":
            # the autotuner's shapes on this index (not registered: the other
            # legs keep theirs), against the library default
            from paper_1502_01916_gb300.tune import tune
            best, info = tune(idx, plan, use_cache=False, register=False, reps=3)
            res[name]["autotuned"] = {
                "shape": [best.warps_per_block, best.blocks_per_sm, best.items_per_claim, best.stage_bytes],
                "ms": info["best_ms"], "library_default_ms": info["ms"].get("7x3x32x0"), "ms_by_shape": info["ms"]}
        del idx, plan, scratch
        mi = gc.encode_mixed_index(codec, d, lens, vb_below=64)
        mplan = gc.plan_index(mi.group)
        ms, ok = timed(lambda: gc.decode_mixed(mi, out=out, status=st, plan=mplan, check=False))
        gbytes = mi.group.compressed_bytes() + mi.group.index_bytes()
        res[name + "_vb_below_64"] = {
            "bits_per_int": 8.0 * (gbytes + mi.vb_bytes.numel() + 24 * mi.n_short) / total, "ms": ms,
            "ints_per_s": total / (ms / 1e3), "sample_verified": ok, "vb_lists": mi.n_short}
        del mi, mplan
        torch.cuda.empty_cache()
    del d, out
    torch.cuda.empty_cache()
    return res


def and_query_rates(gc, idx, lengths, off, gaps, dev, nq=4000, reps=5, nverify=200, seed=13):
    """Two-list AND queries over the resident index (gc_intersect), each
    list drawn with probability proportional to length^0.5 (as the serving
    trace draws them), answered as one batch: timed with CUDA events, checked
    on a sample of queries against numpy's intersection of the host's prefix
    sums. Reports how many tiles of the longer lists the skip entries let
    the call leave undecoded."""
    import torch
    rng = np.random.default_rng(seed)
    w = np.sqrt(lengths.astype(np.float64))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    pairs = np.minimum(np.searchsorted(cdf, rng.random((nq, 2)), side="right"), len(lengths) - 1)
    b = gc.and_batch(idx, pairs)
    st = gc.new_status(dev)
    for _ in range(3):
        gc.run_and_batch(idx, b, st)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gc.run_and_batch(idx, b, st)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    gc.check_status(st, "and queries")
    res, counts = gc.as_u32(b.d_out), gc.as_u32(b.d_counts[:nq])
    a_tiles, b_tiles_decoded = gc.and_batch_tiles(b)

    def ids(i):
        return np.cumsum(gaps[int(off[i]):int(off[i]) + int(lengths[i])], dtype=np.uint32)

    ok = True
    for q in rng.choice(nq, min(nverify, nq), replace=False):
        want = np.intersect1d(ids(b.qa[q]), ids(b.qb[q]))
        got = res[int(b.aoff[q]):int(b.aoff[q]) + int(counts[q])]
        ok = ok and np.array_equal(got, want)
    ms = float(np.median(ts))
    return {"queries": nq, "ms_per_batch": ms, "queries_per_s": nq / (ms / 1e3),
            "codec": gc.codec_name(idx.codec), "results": int(counts.sum()),
            "shorter_list_ints": b.a_ints, "longer_list_ints": b.b_ints,
            "longer_list_tiles": b.b_tiles, "longer_list_tiles_decoded": b_tiles_decoded,
            "decoded_ints_vs_both_whole": (b.a_ints + 1024 * b_tiles_decoded) / max(1, b.a_ints + b.b_ints),
            "sample_verified": bool(ok), "sample": int(min(nverify, nq)),
            "launches_per_batch": gc.gc_last_launch_count()}


def serving_rates(gc, idx, list_ids, seconds, rates=(1e4, 5e4, 2e5), launch=None, nverify=40, seed=31):
    """Requests of 2-8 lists (chosen with probability proportional to
    length^0.5) arriving as a Poisson process for `seconds`, served by
    continuous batching over the resident index (arena: half the free device
    memory, at most 4 GiB) and, on the same trace, by one decoder launch per
    list (which stops issuing when the trace ends: a saturated baseline
    serves fewer requests, and says so). Latency is arrival to completion of
    the request's last list. A random sample of the batched requests'
    docIDs is checked against the host's prefix sums."""
    from paper_1502_01916_gb300 import serve
    res = {"codec": gc.codec_name(idx.codec), "seconds": seconds, "rates": {}}
    rng = np.random.default_rng(seed)
    for rate in rates:
        reqs = serve.poisson_trace(idx.lengths, rate, seconds, seed=int(rate))
        check = set(rng.choice(len(reqs), min(nverify, len(reqs)), replace=False).tolist())
        got = {}

        def keep(r, view, check=check, got=got):
            if r.rid in check:
                got[r.rid] = gc.as_u32(view).copy()

        srv = serve.Server(idx, streams=3, launch=launch)
        wall, done = srv.run(reqs, on_complete=keep, time_limit=seconds + 120.0)
        summ = serve.latency_summary(done, wall, idx.lengths)
        ok = len(got) == len(check) and all(
            np.array_equal(got[r.rid], np.concatenate([list_ids(li) for li in r.lists.tolist()]))
            for r in reqs if r.rid in check)
        summ.update({"batches": srv.batches, "gpu_launches": srv.launches, "sample_verified": bool(ok),
                     "arena_ints": srv.alloc.size})
        del srv
        base = serve.poisson_trace(idx.lengths, rate, seconds, seed=int(rate))
        bwall, served = serve.serve_one_launch_per_list(idx, base, time_limit=seconds + 120.0, issue_limit=seconds)
        bsum = serve.latency_summary(served, bwall, idx.lengths, offered=len(base))
        bsum["saturated"] = len(served) < len(base) or bsum["p50_ms"] > 1e3 * seconds / 4
        res["rates"][f"{int(rate)}"] = {"batched": summ, "one_launch_per_list": bsum}
    return res


def _timed(fn, reps=5, warm=3):
    """Median milliseconds of fn() over reps runs (CUDA events on the current
    stream, after warm runs)."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def single_list_latency(gc, dev, peak, reps=50):
    """One list of 65,536 docIDs (d-gaps geometric, mean 20), Group-Simple
    at k = 4 (the paper's layout) and k = 32: the latency of one decode call
    with its tile index (gc_decode) and, at k = 4, of the paper's single
    buffer (gc_decode_paper: the tile index built from the control area, the
    tiles joined by look-back; the call reads the buffer's head on the host,
    so it synchronises once). Device time by CUDA events, host time by the
    wall clock around call + synchronise; the list fits in L2."""
    import torch
    import synth
    g = synth.single_list_geometric(65536, 20.0, 0)
    want = np.cumsum(g, dtype=np.uint32)
    n = len(g)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    st = gc.new_status(dev)
    res = {"ints": n, "codec": "Group-Simple", "bound": "latency (L2-resident)"}
    for k in (4, 32):
        codec = gc.make_codec(gc.SIMPLE, k)
        enc = gc.encode(codec, g)
        scratch = torch.empty(gc.gc_decode_scratch_size(codec, n, True), dtype=torch.uint8, device=dev)

        def call():
            gc.gc_decode(codec, enc.ctrl, enc.ctrl_bytes, enc.data, enc.data_words, n, enc.tiles, out, True, scratch,
                         st)

        paths = [("with_tile_index", call)]
        if k == 4:
            buf = gc.pack_paper(enc)
            pscratch = torch.empty(gc.gc_decode_scratch_size(codec, n, False), dtype=torch.uint8, device=dev)
            paths.append(("paper_buffer", lambda: gc.gc_decode_paper(codec, buf, n, out, True, pscratch, st)))
        for name, fn in paths:
            out.fill_(0)
            ms = _timed(fn, reps=reps)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
                torch.cuda.synchronize()
            host_us = (time.perf_counter() - t0) / reps * 1e6
            gc.check_status(st, f"single list {name}")
            alg = enc.compressed_bytes() + 4 * n
            res[f"k{k}_{name}"] = {"device_us": 1e3 * ms, "host_us": host_us, "ints_per_s": n / (ms / 1e3),
                                   "achieved_gbs": alg / (ms / 1e3) / 1e9, "frac": alg / (ms / 1e3) / 1e9 / peak,
                                   "bits_per_int": 8.0 * enc.compressed_bytes() / n,
                                   "verified": bool(np.array_equal(gc.as_u32(out), want))}
    return res


def mixed_list_rates(gc, dev, peak, reps=5):
    """One list of 2^26 d-gaps (runs of 256: 90% geometric mean 8, 10%
    uniform to 2^20), one decode call (plan + persistent decode, docIDs
    restored) for every codec variant at k = 4 and k = 32; algorithmic
    bytes = control + data + the tile index read (32 B per tile) + 4 B per
    docID written. Every docID checked against the host's prefix sums."""
    import torch
    import synth
    g = synth.single_list_mixed(1 << 26, 0)
    n = len(g)
    want = np.cumsum(g, dtype=np.uint32)
    d = torch.from_numpy(g.view(np.int32)).to(dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    st = gc.new_status(dev)
    variants = [("simple", gc.SIMPLE, {}), ("scheme_1B", gc.SCHEME, {"cg": 1, "ld": gc.LD_BINARY}),
                ("scheme_1CU", gc.SCHEME, {"cg": 1, "ld": gc.LD_CU}),
                ("scheme_8B", gc.SCHEME, {"cg": 8, "ld": gc.LD_BINARY}),
                ("scheme_8IU", gc.SCHEME, {"cg": 8, "ld": gc.LD_IU}), ("afor", gc.AFOR, {}),
                ("pfd", gc.PFD, {"zeta": 0.10})]
    res = {"ints": n}
    for k in (4, 32):
        for name, kind, kw in variants:
            codec = gc.make_codec(kind, k, **kw)
            enc = gc.encode(codec, d)
            scratch = torch.empty(gc.gc_decode_scratch_size(codec, n, True), dtype=torch.uint8, device=dev)
            ms = _timed(lambda: gc.gc_decode(codec, enc.ctrl, enc.ctrl_bytes, enc.data, enc.data_words, n, enc.tiles,
                                             out, True, scratch, st))
            gc.check_status(st, f"2^26 list {name} k={k}")
            alg = enc.compressed_bytes() + enc.tiles.numel() + 4 * n
            res[f"{name}_k{k}"] = {"ms": ms, "ints_per_s": n / (ms / 1e3), "bits_per_int": 8.0 * enc.compressed_bytes() / n,
                                   "achieved_gbs": alg / (ms / 1e3) / 1e9, "frac": alg / (ms / 1e3) / 1e9 / peak,
                                   "verified": bool(np.array_equal(gc.as_u32(out), want))}
            del enc, scratch
    del d, out
    torch.cuda.empty_cache()
    return res


def lookback_rate(gc, idx, plan, out, peak, total_ints, off, lengths, list_ids, sample, reps=5):
    """The headline index decoded without skip entries: the plan's records
    lose their bases (a list's first tile starts from 0), so every later
    tile takes its prefix from the tiles before it by decoupled look-back
    (claimed one record at a time). Timed like the headline, checked on a
    sample of lists and the longest ones."""
    import torch
    dev = out.device
    nwork = int(plan.count[0].item())
    w = plan.work[:nwork * gc.WORK_BYTES].cpu().numpy().view(gc.WORK_DTYPE).copy()
    w["shape"] &= np.uint32(~(gc.WORK_HAS_BASE | gc.WORK_PUBLISH) & 0xFFFFFFFF)
    w["base"] = 0
    first = w["tile"] == 0
    w["shape"][first] |= np.uint32(gc.WORK_HAS_BASE)
    nxt = np.zeros(nwork, bool)
    nxt[:-1] = (w["list"][1:] == w["list"][:-1]) & (w["tile"][1:] > 0)
    w["shape"][nxt & first] |= np.uint32(gc.WORK_PUBLISH)
    nlb = int((~first & (w["list"] != 0xFFFFFFFF)).sum())
    lplan = gc.Plan(torch.from_numpy(w.view(np.uint8).reshape(-1)).to(dev),
                    torch.tensor([nwork, nlb], dtype=torch.int64, device=dev))
    del w
    scratch = torch.empty(gc.gc_decode_plan_scratch_size(nwork), dtype=torch.uint8, device=dev)
    st = gc.new_status(dev)
    ms = _timed(lambda: gc.decode_index(idx, out=out, scratch=scratch, status=st, plan=lplan, check=False), reps=reps)
    gc.check_status(st, "look-back decode")
    got = gc.as_u32(out)
    ok = all(np.array_equal(got[int(off[i]):int(off[i]) + int(lengths[i])], list_ids(i)) for i in sample)
    alg = idx.compressed_bytes() + lplan.nbytes() + 4 * total_ints
    del lplan, scratch
    return {"codec": gc.codec_name(idx.codec), "ms_per_launch": ms, "ints_per_s": total_ints / (ms / 1e3),
            "look_back_tiles": nlb, "tiles": nwork, "achieved_gbs": alg / (ms / 1e3) / 1e9,
            "frac": alg / (ms / 1e3) / 1e9 / peak, "sample_verified": bool(ok), "sample_lists": len(sample)}


def k_choice_rates(gc, gaps, lengths, off, dev, kinds):
    """The headline lists encoded at k = 4 and at k = 32 per codec, each
    decode tuned and timed (tune.choose_k): bits per int beside the rate,
    and which k the autotuner would build the index with."""
    import torch
    from paper_1502_01916_gb300.tune import choose_k
    d = torch.from_numpy(gaps.view(np.int32)).to(dev)
    res = {}
    for kind in kinds:
        k, by_k = choose_k(kind, d, lengths, out_offsets=off[:-1], reps=2, register=False)
        total = int(lengths.sum(dtype=np.uint64))
        for v in by_k.values():
            v["ints_per_s"] = total / (v["ms"] / 1e3)
        res[gc.codec_name(gc.make_codec(kind, 32))] = {"chosen_k": k, "by_k": {str(kk): v for kk, v in by_k.items()}}
    del d
    torch.cuda.empty_cache()
    return res


def per_list_rate(gc, idxs, lengths, dev, nsample=2000, seed=3):
    """Decode a random sample of lists with one gc_decode call (one launch)
    per list, from the same resident pools."""
    import ctypes
    import torch
    rng = np.random.default_rng(seed)
    ids = rng.choice(len(lengths), min(nsample, len(lengths)), replace=False)
    res = {}
    lib = gc.load()
    for n, idx in idxs.items():
        lists = idx.lists.cpu().numpy().view(gc.LIST_DTYPE)
        nmax = int(lengths[ids].max())
        scratch = torch.empty(gc.gc_decode_scratch_size(idx.codec, nmax, True), dtype=torch.uint8, device=dev)
        out = torch.empty(nmax, dtype=torch.int32, device=dev)
        st = gc.new_status(dev)
        cbase, dbase, tbase = idx.ctrl.data_ptr(), idx.data.data_ptr(), idx.tiles.data_ptr()
        s = torch.cuda.current_stream().cuda_stream
        calls = []
        for i in ids.tolist():
            d = lists[i]
            # gc_decode indexes a single list's records from tile 0; the pool
            # holds them from tile 1 (tile 0's record is never read)
            tp = tbase + (int(d["tile_off"]) - 1) * gc.TILE_BYTES
            calls.append((cbase + int(d["ctrl_off"]), int(d["ctrl_bytes"]), dbase + 4 * int(d["data_off"]),
                          int(d["data_words"]), int(d["n"]), tp))
        cp = ctypes.byref(idx.codec)

        def run():
            for c in calls:
                rc = lib.gc_decode(cp, c[0], c[1], c[2], c[3], c[4], c[5], out.data_ptr(), 1, scratch.data_ptr(),
                                   scratch.numel(), st.data_ptr(), s)
                if rc:
                    raise gc.GcError(rc, "gc_decode")

        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        gc.check_status(st, "per-list decode")
        ints = int(lengths[ids].sum())
        res[n] = {"ints_per_s": ints / (ms / 1e3), "lists": len(ids), "ints": ints, "ms": ms}
    return res


if __name__ == "__main__":
    main()
