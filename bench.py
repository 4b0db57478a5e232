"""Benchmark: batched small-matrix GEMM on GB300 (arXiv 1304.7053).

Workload (the paper's basic parameter set, Section 7): for every square size
m = 1..16, one batch of N = 100,000 independent pairs, fp32, op = N/N,
alpha = 1, beta = 0, minimal leading dimensions.  One step runs the 16
batches through the C ABI as one grouped call (one persistent launch); the
same step as 16 uniform calls is reported beside it.  Inputs are seeded
synthetic uniform[-1, 1] data resident in HBM.  The step touches 1.8 GB, far
more than the 129 MB L2, so every batch starts cold without an explicit
flush.

Reported (one JSON line on rank 0):
  value      GFLOP/s over the whole step (2 m^3 flops per pair, Section 7),
             summed over ranks (weak scaling: every rank runs the workload)
  gbps       algorithmic HBM GB/s of the step (12 m^2 bytes per pair)
  roofline   the kernel with the largest share of the step, its algorithmic
             bytes per launch / its mean CUDA-event duration, against the
             measured copy bandwidth
  e2e        the same metric with host buffers: pinned host -> device copies
             of A and B and the device -> host copy of C inside the timed
             region, every step
  cpu_baseline  the CPU oracle on the host cores on a bounded sample
--impl reference times the CPU oracle alone (the only other implementation
of this method that runs here).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SIZES = list(range(1, 17))
N_PAIRS = 100_000
METRIC = "batched GEMM GFLOP/s and HBM GB/s (% of ~8 TB/s) at N=1e5, sizes 1-16"
# Table "tab:gflop" (Section 7), single-precision real column, GFLOP/s on a
# Tesla K20c at N = 100,000, a1b0, sizes 1..16.
PAPER_S_GFLOPS = [1, 3, 12, 26, 48, 59, 83, 125, 102, 104, 126, 129, 124, 126, 150, 216]


def flops_per_pair(m):
    return 2 * m ** 3


def bytes_per_pair(m, es=4):
    return es * 3 * m * m


def paper_aggregate_gflops():
    """The same metric derived from the paper's per-size table: total flops of
    the step over the sum of the per-size times the table implies."""
    fl = sum(flops_per_pair(m) * N_PAIRS for m in SIZES)
    t = sum(flops_per_pair(m) * N_PAIRS / (g * 1e9) for m, g in zip(SIZES, PAPER_S_GFLOPS))
    return fl / t / 1e9


# the sources the fp32 grouped kernel and its launch are built from
GROUPED_SOURCES = ("grouped.cuh", "grouped_S.cu", "grouped_api.cu", "sbgemm_launch.cuh",
                   "sbgemm_device.cuh", "tile_table.h")


def kernel_source_hash():
    """Hash of the grouped kernel's source files: recorded DRAM traffic is
    reported only while it matches."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1304_7053_gb300", "csrc")
    for fn in GROUPED_SOURCES:
        with open(os.path.join(d, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel_key):
    """DRAM bytes per launch recorded from an ncu capture, if the kernel
    sources have not changed since (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_key)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0, period_ms=100):
        self.rows, self.proc, self.gpu, self.period = [], None, gpu_index, period_ms

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", f"-lms={self.period}"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ------------------------------------------------------------------ our arm

def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1304_7053_gb300 import sbgemm, shard

    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    sbgemm.lib()
    stream = torch.cuda.Stream(device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234 + rank)

    bufs = {}
    for m in SIZES:
        S = m * m
        A = (torch.rand(N_PAIRS * S, device=dev, generator=gen) * 2 - 1).contiguous()
        B = (torch.rand(N_PAIRS * S, device=dev, generator=gen) * 2 - 1).contiguous()
        C = torch.empty(N_PAIRS * S, device=dev)
        bufs[m] = (A, B, C)
    torch.cuda.synchronize()

    calls = {m: sbgemm.prepare_uniform("s", "N", "N", m, m, m, 1.0, bufs[m][0], m, m * m,
                                       bufs[m][1], m, m * m, 0.0, bufs[m][2], m, m * m,
                                       N_PAIRS, stream=stream) for m in SIZES}

    def launch(m):
        calls[m]()

    # the step as one grouped call (all 16 batches in one persistent launch)
    import ctypes
    groups = (sbgemm.Group * len(SIZES))()
    for gr, m in zip(groups, SIZES):
        A, B, C = bufs[m]
        gr.transa, gr.transb, gr.m, gr.n, gr.k = b"N", b"N", m, m, m
        gr.A, gr.lda, gr.lda2 = A.data_ptr(), m, m * m
        gr.B, gr.ldb, gr.ldb2 = B.data_ptr(), m, m * m
        gr.C, gr.ldc, gr.ldc2 = C.data_ptr(), m, m * m
        gr.batchCount = N_PAIRS
    g_one, g_zero = (ctypes.c_float * 1)(1.0), (ctypes.c_float * 1)(0.0)
    Lg = sbgemm.lib()
    g_args = (0, ctypes.addressof(g_one), ctypes.addressof(g_zero), ctypes.addressof(groups),
              len(SIZES), 0, stream.cuda_stream)

    def grouped_step():
        st = Lg.sbgemm_gemm_grouped(*g_args)
        if st != 0:
            raise sbgemm.SbgemmError(st, "gemm_grouped")

    def barrier():
        if world > 1:
            dist.barrier()

    # Timed region: K steps of 16 eager launches on one stream.  One pair of
    # CUDA events per step brackets one kernel, rotating over the sizes, so
    # every kernel is timed K/16 times inside the timed region while the
    # events add almost nothing to the step.
    K = args.steps
    nsz = len(SIZES)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            for m in SIZES:
                launch(m)
    torch.cuda.synchronize()
    # short runs (fewer steps than sizes) time every kernel of every step
    every = K < nsz
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(nsz if every else 1)] for _ in range(K)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)   # let the sampler start before the timed region
    with torch.cuda.stream(stream):
        t0.record(stream)
        for s in range(K):
            jt = s % nsz
            for j, m in enumerate(SIZES):
                if every or j == jt:
                    e = ev[s][j if every else 0]
                    e[0].record(stream)
                    launch(m)
                    e[1].record(stream)
                else:
                    launch(m)
        t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    # the timed region ends when the slowest rank does
    elapsed_ms = shard.max_over_ranks(t0.elapsed_time(t1), dev)
    ms_step = elapsed_ms / K
    per = {}
    for j, m in enumerate(SIZES):
        if every:
            d = [ev[s][j][0].elapsed_time(ev[s][j][1]) for s in range(K)]
        else:
            d = [ev[s][0][0].elapsed_time(ev[s][0][1]) for s in range(K) if s % nsz == j]
        if not d:
            continue
        mean_ms = sum(d) / len(d)
        per[m] = {"us": round(mean_ms * 1e3, 3), "samples": len(d),
                  "gflops": round(flops_per_pair(m) * N_PAIRS / (mean_ms * 1e-3) / 1e9, 1),
                  "gbps": round(bytes_per_pair(m) * N_PAIRS / (mean_ms * 1e-3) / 1e9, 1)}

    sep_ms_step, sep_per = ms_step, per

    # The headline: the same K steps, each step one grouped call (one
    # persistent launch for the 16 batches), events around every step's
    # launch on the stream it runs on.
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            grouped_step()
    torch.cuda.synchronize()
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    clocks = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        t0.record(stream)
        for s in range(K):
            gev[s][0].record(stream)
            grouped_step()
            gev[s][1].record(stream)
        t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms_step = shard.max_over_ranks(t0.elapsed_time(t1), dev) / K
    grouped_kernel_ms = sum(a.elapsed_time(b) for a, b in gev) / K

    # cross-check: the step replayed from a CUDA graph (no host launch cost)
    graph_ms = None
    try:
        cap = torch.cuda.Stream(device=dev)
        gcalls = {m: sbgemm.prepare_uniform("s", "N", "N", m, m, m, 1.0, bufs[m][0], m, m * m,
                                            bufs[m][1], m, m * m, 0.0, bufs[m][2], m, m * m,
                                            N_PAIRS, stream=cap) for m in SIZES}
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            for m in SIZES:
                gcalls[m]()
        with torch.cuda.stream(stream):
            for _ in range(3):
                g.replay()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = min(K, 200)
            e0.record(stream)
            for _ in range(reps):
                g.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        graph_ms = round(e0.elapsed_time(e1) / reps, 5)
    except Exception as ex:
        graph_ms = f"unavailable: {type(ex).__name__}"
    total_flops = sum(flops_per_pair(m) * N_PAIRS for m in SIZES)
    total_bytes = sum(bytes_per_pair(m) * N_PAIRS for m in SIZES)
    value = world * total_flops / (ms_step * 1e-3) / 1e9
    gbps = world * total_bytes / (ms_step * 1e-3) / 1e9

    # the grouped kernel is the only kernel of the step
    peak, peak_kind = measured_peaks()
    achieved = total_bytes / (grouped_kernel_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": ncu_traffic(f"grouped_s_1-16_N{N_PAIRS}_nn_b0"),
                "kernel": f"grouped_kernel fp32 m=1..16 N={N_PAIRS} each (one launch per step)",
                "peak_kind": peak_kind, "algorithmic_bytes": total_bytes,
                "kernel_us": round(grouped_kernel_ms * 1e3, 3)}
    dom = max(SIZES, key=lambda m: sep_per[m]["us"])
    sep_ach = bytes_per_pair(dom) * N_PAIRS / (sep_per[dom]["us"] * 1e-6) / 1e9
    separate = {"ms_per_step": round(sep_ms_step, 5),
                "gflops": round(world * total_flops / (sep_ms_step * 1e-3) / 1e9, 1),
                "dominant_kernel": f"pipe_kernel fp32 {dom}x{dom}x{dom}",
                "dominant_gbps": round(sep_ach, 1), "dominant_frac": round(sep_ach / peak, 4),
                "per_size": sep_per}

    e2e = run_e2e(args, bufs, launch, stream, barrier, world, dev) if not args.no_e2e else None
    vb = None
    if not args.no_vbatch and rank == 0:
        try:
            del bufs
            torch.cuda.empty_cache()
            vb = [run_vbatch_bench(d, dev, stream) for d in ("s", "d")]
        except Exception as ex:
            vb = f"failed: {type(ex).__name__}: {ex}"
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "GFLOP/s",
        "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(ms_step, 5), "ms_per_step_graph_replay": graph_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": (round(value / (world * paper_aggregate_gflops()), 2)
                        if SIZES == list(range(1, 17)) else None),
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "fp32 square m=1..16, N=100000 pairs each, op N/N, alpha=1, "
                               "beta=0, minimal leading dims" if SIZES == list(range(1, 17)) else
                               f"fp32 square m in {SIZES}, N=100000 pairs each, op N/N, alpha=1, beta=0",
                   "pairs_per_size": N_PAIRS, "sizes": ",".join(map(str, SIZES)),
                   "l2": "no flush: 1.8 GB touched per step >> 129 MB L2",
                   "parallelism": f"replicas x{world} (independent batches, no collective)"},
        "gbps": round(gbps, 1),
        "pct_of_8TBs": round(100 * gbps / world / 8000.0, 1),
        "pct_of_measured_hbm": round(100 * gbps / world / peak, 1),
        "separate_calls": separate,
        "roofline": roofline,
        "gpu_launches": K,
        "timing": "each step is one sbgemm_gemm_grouped call (16 batches, one persistent "
                  "launch), events around every launch; separate_calls: the 16 uniform calls per "
                  "step with one event pair per step rotating over the sizes",
        "clocks": clk,
        "e2e": e2e,
        "vbatch": vb,
    }
    return out


def run_e2e(args, bufs, launch, stream, barrier, world, dev):
    """Same workload with host buffers, through the C ABI's host-array entry
    point: every step streams A and B from pinned host memory to the device,
    computes, and copies C back (copies and kernels of consecutive chunks
    overlap inside the call)."""
    import ctypes
    import torch
    from paper_1304_7053_gb300 import sbgemm, shard
    host = {}
    for m in SIZES:
        A, B, C = bufs[m]
        host[m] = (A.cpu().pin_memory(), B.cpu().pin_memory(),
                   torch.empty(C.numel(), dtype=C.dtype).pin_memory())
    work = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    one = (ctypes.c_float * 1)(1.0)
    zero = (ctypes.c_float * 1)(0.0)
    L = sbgemm.lib()
    groups = (sbgemm.HostGroup * len(SIZES))()
    for g, m in zip(groups, SIZES):
        hA, hB, hC = host[m]
        g.transa, g.transb, g.m, g.n, g.k = b"N", b"N", m, m, m
        g.hA, g.lda, g.lda2 = hA.data_ptr(), m, m * m
        g.hB, g.ldb, g.ldb2 = hB.data_ptr(), m, m * m
        g.hC, g.ldc, g.ldc2 = hC.data_ptr(), m, m * m
        g.batchCount = N_PAIRS

    def step():
        # the 16 batches of a step as one grouped call: one copy pipeline
        st = L.sbgemm_gemm_grouped_host(0, ctypes.addressof(one), ctypes.addressof(zero),
                                        ctypes.addressof(groups), len(SIZES), work.data_ptr(),
                                        work.numel(), stream.cuda_stream)
        if st != 0:
            raise sbgemm.SbgemmError(st, "gemm_grouped_host")

    K = max(3, args.e2e_steps)
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = shard.max_over_ranks(e0.elapsed_time(e1) / K, dev)
    # the result read back equals the device path's (same kernels, same inputs)
    ok = all(torch.equal(host[m][2], bufs[m][2].cpu()) for m in SIZES[-2:])
    total_flops = sum(flops_per_pair(m) * N_PAIRS for m in SIZES)
    h2d = sum(2 * 4 * m * m * N_PAIRS for m in SIZES)
    d2h = sum(4 * m * m * N_PAIRS for m in SIZES)
    return {"value": round(world * total_flops / (ms * 1e-3) / 1e9, 1), "unit": "GFLOP/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": K,
            "ms_per_step": round(ms, 3), "link_gbps": round((h2d + d2h) / (ms * 1e-3) / 1e9, 1),
            "matches_device_result": bool(ok),
            "path": "sbgemm_gemm_grouped_host (16 groups per step), 512 MB device work buffer, "
                    "pinned host arrays"}


# ------------------------------------------------------------------ variable size

def run_vbatch_bench(dtype, dev, stream, reps=20, warm=3, N=1_000_000):
    """The variable-size batch: N problems, m = n = k = p + 1 with P(p)
    proportional to 1/p, beta per problem in {0, 1}, back to back in one
    arena; one plan run (memset + one persistent kernel) against the same
    problems partitioned by size and run as one fixed-size call per size."""
    import numpy as np
    import torch
    from paper_1304_7053_gb300 import inputs, sbgemm
    desc, la, lb, lc = inputs.vbatch_problems(N, seed=0)
    tdt = torch.float32 if dtype == "s" else torch.float64
    es = 4 if dtype == "s" else 8
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    A = torch.rand(la, device=dev, generator=gen, dtype=tdt) * 2 - 1
    B = torch.rand(lb, device=dev, generator=gen, dtype=tdt) * 2 - 1
    C = torch.rand(lc, device=dev, generator=gen, dtype=tdt) * 2 - 1
    # the plan's bucketing window, tuned on this batch by the autotuner
    from paper_1304_7053_gb300 import selector
    problems = sbgemm.vproblems_from_desc(desc)
    window, wtimes = selector.tune_vbatch(dtype, problems, A, B, C,
                                          windows=(selector.WHOLE_BATCH, 262144, 65536, 16384),
                                          reps=3, stream=stream)
    plan = sbgemm.VPlan(dtype, problems)
    sbgemm.lib().sbgemm_vbatch_config(0)
    sizes = desc[:, 0]
    bz = (desc[:, 3] >> 4) & 1
    alg_bytes = int(np.sum(es * sizes * sizes * (3 + (1 - bz))))
    flops = int(np.sum(2 * sizes ** 3))
    with torch.cuda.stream(stream):
        for _ in range(warm):
            plan.run(1.0, A, B, 1.0, C, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plan.run(1.0, A, B, 1.0, C, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    v_ms = e0.elapsed_time(e1) / reps
    info = plan.info()
    plan.close()
    # comparator: the paper's partition by size, one uniform call per size
    # (beta = 1 for every problem: the byte count below includes the C read)
    calls = []
    fbytes = 0
    for sz in range(2, 17):
        cnt = int(np.sum(sizes == sz))
        if cnt == 0:
            continue
        S = sz * sz
        a = torch.rand(cnt * S, device=dev, generator=gen, dtype=tdt)
        b = torch.rand(cnt * S, device=dev, generator=gen, dtype=tdt)
        c = torch.rand(cnt * S, device=dev, generator=gen, dtype=tdt)
        calls.append((sbgemm.prepare_uniform(dtype, "N", "N", sz, sz, sz, 1.0, a, sz, S, b, sz, S,
                                             1.0, c, sz, S, cnt, stream=stream), (a, b, c)))
        fbytes += es * cnt * S * 4
    with torch.cuda.stream(stream):
        for _ in range(warm):
            for f, _keep in calls:
                f()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(reps):
            for f, _keep in calls:
                f()
        f1.record(stream)
    torch.cuda.synchronize()
    f_ms = f0.elapsed_time(f1) / reps
    return {"dtype": dtype, "problems": N, "tiles": info["tiles"], "buckets": info["buckets"],
            "window": "whole batch" if window == selector.WHOLE_BATCH else window,
            "window_trials_ms": {("whole" if w == selector.WHOLE_BATCH else str(w)): round(t, 4)
                                 for w, t in wtimes.items()},
            "ms": round(v_ms, 4), "gflops": round(flops / (v_ms * 1e-3) / 1e9, 1),
            "gbps": round(alg_bytes / (v_ms * 1e-3) / 1e9, 1),
            "fixed_per_size_ms": round(f_ms, 4),
            "fixed_per_size_gbps": round(fbytes / (f_ms * 1e-3) / 1e9, 1),
            "note": "vbatch: mixed beta (C read for half the problems); per-size fixed calls: "
                    "beta = 1 for all, bytes counted accordingly"}


# ------------------------------------------------------------------ CPU oracle

def oracle_sample(budget_s, threads):
    """Time the CPU oracle on a bounded sample of the workload: the same
    sizes, fp32, NN, alpha 1, beta 0, with fewer pairs per size (chosen so
    each size takes a similar share of the budget).  Returns (GFLOP/s,
    description, threads, seconds)."""
    import numpy as np
    import oracle
    from paper_1304_7053_gb300 import inputs
    oracle.build()
    # calibrate on m = 8
    def run(m, n):
        b = inputs.UniformBatch("s", "N", "N", m, m, m, n, seed=m)
        t = time.perf_counter()
        oracle.gemm_uniform("s", "N", "N", m, m, m, 1.0, b.A, m, m * m, b.B, m, m * m, 0.0,
                            b.C, m, m * m, n, threads=threads)
        return time.perf_counter() - t
    cal_n = 2000
    cal = run(8, cal_n)
    per_pair_m8 = max(cal / cal_n, 1e-9)
    flops = 0
    secs = 0.0
    counts = {}
    for m in SIZES:
        est = per_pair_m8 * (m / 8) ** 3 + 2e-8
        n = int(min(N_PAIRS, max(64, budget_s / len(SIZES) / est)))
        dt = run(m, n)
        secs += dt
        flops += flops_per_pair(m) * n
        counts[m] = n
    # when the whole workload takes less than the budget, repeat it so the
    # timing covers about the budget (a steadier figure than one short pass)
    passes = 1
    if all(counts[m] == N_PAIRS for m in SIZES) and 0.0 < secs < budget_s:
        one = secs
        for _ in range(min(20, int(budget_s / one) - 1)):
            for m in SIZES:
                secs += run(m, N_PAIRS)
                flops += flops_per_pair(m) * N_PAIRS
            passes += 1
    desc = ("oracle (double-double triple loop), fp32 NN alpha=1 beta=0, sizes 1-16, pairs per "
            "size " + ",".join(f"{m}:{counts[m]}" for m in SIZES) + f", {passes} pass(es)")
    return flops / secs / 1e9, desc, threads, secs


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle is this method's only other
    implementation here; rank 0 times it, other ranks exit."""
    if rank != 0:
        return None
    import oracle
    threads = oracle.max_threads()
    vals = []
    t_all = time.perf_counter()
    desc = ""
    for _ in range(args.warmup):
        oracle_sample(max(0.5, args.ref_budget / 10), threads)
    for _ in range(args.steps):
        v, desc, threads, secs = oracle_sample(args.ref_budget / max(1, args.steps), threads)
        vals.append(v)
    value = statistics.median(vals)
    total_flops = sum(flops_per_pair(m) * N_PAIRS for m in SIZES)
    return {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_flops / (value * 1e9) * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "fp32 square m=1..16, N=100000 pairs each, op N/N, alpha=1, "
                                   "beta=0, minimal leading dims (timed on a bounded sample)"},
            "cpu_baseline": {"value": round(value, 3), "unit": "GFLOP/s", "cores": threads,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": round(value, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": round(time.perf_counter() - t_all, 1)}


def relaunch_command(gpus, argv, port=None):
    """The torch.distributed.run command that starts `gpus` ranks of this
    script on one node (loopback rendezvous on a free port)."""
    if port is None:
        import socket
        with socket.socket() as so:
            so.bind(("127.0.0.1", 0))
            port = so.getsockname()[1]
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
            f"--nproc-per-node={gpus}", "--master-addr", "127.0.0.1", "--master-port", str(port),
            os.path.abspath(__file__), *argv]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-vbatch", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle time")
    ap.add_argument("--ref-budget", type=float, default=60.0)
    ap.add_argument("--sizes", default="1-16",
                    help="square sizes in the step, e.g. 16 or 8,12,16 (default: the 1-16 workload)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    global SIZES
    if args.sizes != "1-16":
        SIZES = [int(x) for x in args.sizes.split(",")]

    if args.gpus < 1:
        sys.exit("bench.py: --gpus must be at least 1")
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # no launcher: start one rank per GPU through torch.distributed.run
        # and report its result (rank 0 prints the JSON line)
        sys.exit(subprocess.call(relaunch_command(args.gpus, sys.argv[1:])))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        sys.exit(f"bench.py: --gpus {args.gpus} but the launcher started {world} ranks")

    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local_rank}"))
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu:
            import oracle
            v, desc, threads, secs = oracle_sample(args.cpu_budget, oracle.max_threads())
            out["cpu_baseline"] = {"value": round(v, 3), "unit": "GFLOP/s", "cores": threads,
                                   "kind": "oracle", "sample": desc, "seconds": round(secs, 1)}
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
