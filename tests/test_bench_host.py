"""bench.py's host logic (no GPU): the clocks object it reads from nvidia-smi
samples, the traffic it derives from the small-case counters, and the JSON
line of the reference arm (the CPU oracle on a tiny sample)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_samples_median_max_and_reasons():
    out = "\n".join([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    c = bench.parse_clocks(out)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.parse_clocks("") is None


def test_clock_samples_flag_slowdowns():
    out = "0, 1200, 2070, 1400, 0x8, Active, Not Active, Active, Not Active\n" * 3
    c = bench.parse_clocks(out)
    assert c["sm_mhz"] == 1200.0 and c["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_traffic_ratios_are_for_the_current_sources_or_absent():
    """The recorded counters name the kernel sources they were taken on; a
    stale hash makes the benchmark report traffic as null."""
    for name, r in bench.NCU_TRAFFIC_RATIO.items():
        assert name in bench.CODECS
        assert 0.99 < r["read"] < 1.05 and 0 <= r["write_short"] < 200e6
        assert len(r["hash"]) == 16
    assert len(bench.kernel_hash()) == 16


def test_reference_arm_prints_one_json_line():
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--nlists", "2000"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "ints/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["higher_is_better"] is True
