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


def test_measurement_arithmetic():
    """The numerators of every reported rate: flops 2mnk (real) or 8mnk
    (complex) per pair (Section 7), algorithmic bytes s*(mk + kn + mn*(1 +
    [beta != 0])) per pair; the bench's step is 3.70 GFLOP and 1.795 GB, and
    the paper's Table implies 128 GFLOP/s for the same step on its K20c."""
    sys.path.insert(0, ROOT)
    import bench
    import sweep
    r = sweep.row("c", "T", "N", 3, 9, 3, 1000, -0.5, 1.0)        # 1 ms
    assert r["gflops"] == round(8 * 3 * 9 * 3 * 1000 / 1e-3 / 1e9, 1)
    assert r["gbps"] == round(8 * 1000 * (9 + 27 + 27 * 2) / 1e-3 / 1e9, 1)
    r = sweep.row("s", "N", "N", 16, 16, 16, 100_000, 0.0, 1.0)
    assert r["gbps"] == round(4 * 100_000 * 3 * 256 / 1e-3 / 1e9, 1)
    assert r["gflops"] == round(2 * 4096 * 100_000 / 1e-3 / 1e9, 1)
    fl = sum(bench.flops_per_pair(m) * bench.N_PAIRS for m in bench.SIZES)
    by = sum(bench.bytes_per_pair(m) * bench.N_PAIRS for m in bench.SIZES)
    assert fl == 3_699_200_000 and by == 1_795_200_000
    assert 127.0 < bench.paper_aggregate_gflops() < 129.0


def test_gpus_without_launcher_starts_one_rank_per_gpu():
    """`bench.py --gpus 2` with no launcher in the environment starts two
    ranks itself (never a silent one-rank run); shown on the reference arm,
    which runs on the host cores."""
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    r = subprocess.run([sys.executable, "bench.py", "--gpus", "2", "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--ref-budget", "1"], cwd=ROOT,
                       capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    assert json.loads(lines[0])["n_gpus"] == 2


def test_gpus_disagreeing_with_launcher_is_an_error():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--gpus", "2", "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--ref-budget", "1"], cwd=ROOT,
                       capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode != 0 and "launcher started 1 ranks" in r.stderr
