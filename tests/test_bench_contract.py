"""Host-only checks of bench.py: the reference arm's JSON line (the CPU
oracle timed on a bounded sample) and the kernel-source hash that guards
recorded DRAM traffic."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                        "--warmup", "3", "--ref-budget", "2"], cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GFLOP/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_traffic_record_is_tied_to_kernel_sources():
    sys.path.insert(0, ROOT)
    import bench
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h == bench.kernel_source_hash()
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    key = "grouped_s_1-16_N100000_nn_b0"
    got = bench.ncu_traffic(key)
    # the recorded DRAM bytes are returned only for the sources they were taken with
    assert got == (rec[key]["dram_bytes_per_launch"] if rec[key]["source_hash"] == h else None)
    assert bench.ncu_traffic("no such kernel") is None
