"""Throughput sweeps on the current GPU (timings only; correctness is the
tests' job).

Every timing is the mean of `reps` calls (those within 2 us of the median;
event timestamps advance in steps of about 1 us, and the mean of calls that
start at varying phases resolves below a step), each preceded by a read of a
256 MB buffer (twice the L2): every call starts with a cold L2 that holds only
clean lines, so the previous call's results are written back outside the
timed interval.  Timed with CUDA events (the library's timing core for this
library's kernels).  The comparator is
cuBLAS strided-batched GEMM through torch.bmm on the same column-major data
(C = A B column-major is C^T = B^T A^T row-major).

    python sweep.py --out sweep.json [--quick]

Sections: the small configuration (fp32, m = 10, N = 1e4: cold and hot,
direct and CUDA-graph replay, cuBLAS beside it), the fixed-size sweep
(S/D/C/Z, m = 1..16, N = 1e3/1e5/1e6,
op N/N, alpha = 1.5, beta in {0, -0.5}), the op sweep (complex single, all 9
op pairs at N = 1e5), FEM-like rectangular shapes (S/D, N = 5e5, op(A) = T,
beta = 1), the interface comparison (3-D layout vs pointer arrays vs cuBLAS,
N = 1e5), one A shared by all pairs (lda2 = 0, N = 1e6; algorithmic bytes
count B and C only), and 16-bit storage (binary16/bfloat16, m in
{8, 12, 16}, N = 1e6).  ``grouped_config`` (only when named) sweeps the
launch configuration of the grouped call on the fp32 and fp64 sizes 1..16
workload; ``vbatch`` (only when named) compares the variable-size plan with
cublasSgemmGroupedBatched on the fp32 mixed-size batch; ``once`` (only when
named) makes one untimed call per type and
size (fp32, fp64 and complex128, m = 8..16, N = 1e5, op N/N, alpha = 1, beta = 0, L2
evicted before each): the launches a kernel-level profile reads.  ``fp64tc``
(only when named) times real and complex fp64 (``--fp64tc-types``) on the
fp64 FMA kernel (variant 0) and on the tensor-core kernel (variant 7).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1304_7053_gb300 import sbgemm  # noqa: E402

ES = {"s": 4, "d": 8, "c": 8, "z": 16, "h": 2, "b": 2}
CPLX = {"c", "z"}


class Pools:
    """Reusable device buffers filled once with uniform[-1, 1) values: fp32
    for the s, c and 16-bit types (which read the same bytes; their kernels'
    timing does not depend on the values) and fp64 for d and z, whose
    tensor-core kernel takes its fp64-FMA path for entries of very different
    sizes (fp32 bytes read as fp64 are such entries)."""

    def __init__(self, max_bytes, dev):
        import torch
        self.torch = torch
        n = (max_bytes + 3) // 4
        g = torch.Generator(device=dev)
        g.manual_seed(5)
        self.A = torch.rand(n, device=dev, generator=g) * 2 - 1
        self.B = torch.rand(n, device=dev, generator=g) * 2 - 1
        self.C = torch.rand(n, device=dev, generator=g) * 2 - 1
        n64 = (max_bytes + 7) // 8
        self.A64 = torch.rand(n64, device=dev, generator=g, dtype=torch.float64) * 2 - 1
        self.B64 = torch.rand(n64, device=dev, generator=g, dtype=torch.float64) * 2 - 1
        self.C64 = torch.rand(n64, device=dev, generator=g, dtype=torch.float64) * 2 - 1
        self.flush = torch.ones(256 << 20, dtype=torch.uint8, device=dev)
        self._sink = torch.empty((), dtype=torch.int64, device=dev)

    def for_type(self, dtype):
        """(A, B, C) buffers holding values of the type's precision."""
        if dtype in ("d", "z"):
            return self.A64, self.B64, self.C64
        return self.A, self.B, self.C

    def evict(self):
        """Read the 256 MB flush buffer (L2 ends cold and clean)."""
        torch = self.torch
        self._sink = torch.sum(self.flush.view(torch.int32), dtype=torch.int64)

    def as_dtype(self, buf, dtype):
        torch = self.torch
        t = {"s": torch.float32, "d": torch.float64, "c": torch.complex64,
             "z": torch.complex128, "h": torch.float16, "b": torch.bfloat16}[dtype]
        if dtype in ("h", "b"):
            return buf.view(torch.int16).view(t)
        return buf.view(t)


def time_ours(pools, dtype, ta, tb, m, n, k, N, alpha, beta, reps, variant=None,
              shared_a=False):
    """Median time of the uniform call; ``shared_a``: lda2 = 0 (one A for
    every pair)."""
    opa, opb = ta, tb
    ar, ac = (m, k) if opa == "N" else (k, m)
    br, bc = (k, n) if opb == "N" else (n, k)
    lda2 = 0 if shared_a else ar * ac
    L = sbgemm.lib()
    pA, pB, pC = pools.for_type(dtype)
    ab, bb = sbgemm._scalar_buf(dtype, alpha), sbgemm._scalar_buf(dtype, beta)
    if variant is None:
        variant = sbgemm.get_choice(dtype, m, n, k, opa != "N", opb != "N", complex(beta) == 0,
                                    size_class(N))
    ms = ctypes.c_float()
    s = pools.torch.cuda.current_stream().cuda_stream
    st = L.sbgemm_time_variant(sbgemm.TYPE_CODES[dtype], opa.encode(), opb.encode(), m, n, k,
                               ctypes.addressof(ab), pA.data_ptr(), max(1, ar), lda2,
                               pB.data_ptr(), max(1, br), br * bc, ctypes.addressof(bb),
                               pC.data_ptr(), max(1, m), m * n, N, variant, reps,
                               pools.flush.data_ptr(), pools.flush.numel(), s, ctypes.byref(ms))
    if st != 0:
        raise sbgemm.SbgemmError(st, "time_variant")
    return float(ms.value)


def robust_mean(ts):
    """Mean of the times within 2 us (0.002 ms) of their median: event
    timestamps can advance in steps of about 1 us and a call's start varies
    against them, so the mean resolves below a step; delayed calls drop out
    (the estimator of the native timing core)."""
    ts = sorted(ts)
    med = ts[len(ts) // 2]
    keep = [t for t in ts if abs(t - med) <= 0.002]
    return sum(keep) / len(keep)


def time_fn(pools, fn, reps):
    """CUDA-event time of fn() on the current stream (``robust_mean`` of
    `reps` calls after one untimed call), L2 evicted before every call."""
    torch = pools.torch
    ts = []
    for _ in range(reps + 1):
        pools.evict()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return robust_mean(ts[1:])


def time_nounif(pools, dtype, m, N, reps):
    """The pointer-array form on the same flat data (pointer p -> matrix p),
    op N/N, beta = 0; the pointer arrays are built outside the timing."""
    torch = pools.torch
    es = ES[dtype]
    S = m * m
    pA, pB, pC = pools.for_type(dtype)
    idx = torch.arange(N, device=pA.device, dtype=torch.int64) * (S * es)
    Ap, Bp, Cp = idx + pA.data_ptr(), idx + pB.data_ptr(), idx + pC.data_ptr()
    fn = lambda: sbgemm.gemm_multi_nounif(dtype, "N", "N", m, m, m, 1.0, Ap, m, Bp, m, 0.0, Cp,
                                          m, N)
    return time_fn(pools, fn, reps)


def grouped_config_sweep(dtype, dev, reps=200, N=100_000):
    """Wall time per ``sbgemm_gemm_grouped`` call over the square N/N batches
    m = 1..16 (N pairs each, alpha = 1, beta = 0) for every launch
    configuration (threads x stage bytes x depth) that fits; the batches
    (1.8 GB fp32) are far above L2, so calls run back to back."""
    import torch
    tdt = {"s": torch.float32, "d": torch.float64}[dtype]
    L = sbgemm.lib()
    gen = torch.Generator(device=dev)
    gen.manual_seed(1)
    sizes = list(range(1, 17))
    bufs = {m: tuple(torch.rand(N * m * m, device=dev, generator=gen, dtype=tdt) for _ in range(3))
            for m in sizes}
    groups = (sbgemm.Group * len(sizes))()
    for gr, m in zip(groups, sizes):
        A, B, C = bufs[m]
        gr.transa, gr.transb, gr.m, gr.n, gr.k = b"N", b"N", m, m, m
        gr.A, gr.lda, gr.lda2 = A.data_ptr(), m, m * m
        gr.B, gr.ldb, gr.ldb2 = B.data_ptr(), m, m * m
        gr.C, gr.ldc, gr.ldc2 = C.data_ptr(), m, m * m
        gr.batchCount = N
    one, zero = _scalar_pair(dtype)
    stream = torch.cuda.Stream(device=dev)
    flops = sum(2 * m ** 3 * N for m in sizes)

    def call():
        st = L.sbgemm_gemm_grouped(sbgemm.TYPE_CODES[dtype], ctypes.addressof(one),
                                   ctypes.addressof(zero), ctypes.addressof(groups), len(sizes),
                                   0, stream.cuda_stream)
        if st != 0:
            raise sbgemm.SbgemmError(st, "gemm_grouped")

    out = []
    try:
        for threads in (128, 256):
            for sb in (8192, 16384, 20480, 24576, 28672, 32768, 40960, 49152):
                for stg in (2, 3, 4):
                    if stg * sb + sb // 2 > 220 * 1024:
                        continue
                    sbgemm.grouped_config(dtype, threads, sb, stg)
                    with torch.cuda.stream(stream):
                        for _ in range(5):
                            call()
                        t0 = torch.cuda.Event(enable_timing=True)
                        t1 = torch.cuda.Event(enable_timing=True)
                        t0.record(stream)
                        for _ in range(reps):
                            call()
                        t1.record(stream)
                    torch.cuda.synchronize()
                    us = t0.elapsed_time(t1) / reps * 1e3
                    out.append({"dtype": dtype, "threads": threads, "stage_bytes": sb, "stages": stg,
                                "smem_bytes": stg * sb + sb // 2, "us_per_call": round(us, 1),
                                "gflops": round(flops / (us * 1e-6) / 1e9, 1)})
    finally:
        sbgemm.grouped_config(dtype)
    return out


def _scalar_pair(dtype):
    c = ctypes.c_float if dtype == "s" else ctypes.c_double
    return (c * 1)(1.0), (c * 1)(0.0)


def time_cublas(pools, dtype, m, n, k, N, reps):
    """cuBLAS strided batched (torch.bmm) on column-major N/N data, beta = 0."""
    torch = pools.torch
    pA, pB, pC = pools.for_type(dtype)
    A = pools.as_dtype(pA, dtype)[:N * m * k].view(N, k, m)   # row-major view of A^T
    B = pools.as_dtype(pB, dtype)[:N * k * n].view(N, n, k)   # row-major view of B^T
    C = pools.as_dtype(pC, dtype)[:N * m * n].view(N, n, m)   # row-major view of C^T
    ts = []
    for _ in range(reps + 1):
        pools.evict()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.bmm(B, A, out=C)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return robust_mean(ts[1:])


def small_case(pools, reps=41, m=10, N=10_000):
    """The small configuration: fp32, m = n = k = 10, N = 1e4, op N/N, alpha = 1,
    beta = 0 (12 MB, L2-resident, launch-bound: no roofline fraction).  Per
    call, cold (L2 evicted before each call) and hot (calls back to back),
    issued directly and replayed from a CUDA graph, with cuBLAS strided
    batched beside it: p10 / p50 / p90 and the robust mean of `reps` timed
    calls, in microseconds."""
    torch = pools.torch
    S = m * m
    s = torch.cuda.Stream(device=pools.A.device)
    call = sbgemm.prepare_uniform("s", "N", "N", m, m, m, 1.0, pools.A, m, S, pools.B, m, S, 0.0,
                                  pools.C, m, S, N, stream=s)
    A = pools.A[:N * S].view(N, m, m)
    B = pools.B[:N * S].view(N, m, m)
    C = pools.C[:N * S].view(N, m, m)
    ours = lambda: call()
    cublas = lambda: torch.bmm(B, A, out=C)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        call()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        call()
    replay = lambda: g.replay()

    def per_call(fn, cold):
        ts = []
        with torch.cuda.stream(s):
            for _ in range(3):
                fn()
            for _ in range(reps):
                if cold:
                    pools.evict()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                fn()
                e1.record(s)
                ts.append((e0, e1))
        torch.cuda.synchronize()
        us = sorted(a.elapsed_time(b) * 1e3 for a, b in ts)
        q = lambda f: us[min(len(us) - 1, int(f * len(us)))]
        return {"p10_us": round(q(0.1), 2), "p50_us": round(q(0.5), 2), "p90_us": round(q(0.9), 2),
                "mean_us": round(robust_mean([u * 1e-3 for u in us]) * 1e3, 2)}

    flops = 2 * m * m * m * N
    rows = []
    for name, fn in (("direct", ours), ("graph_replay", replay), ("cublas", cublas)):
        for cold in (True, False):
            r = {"dtype": "s", "op": "NN", "m": m, "n": m, "k": m, "N": N, "beta": "0.0",
                 "path": name, "l2": "cold" if cold else "hot"}
            r.update(per_call(fn, cold))
            r["gflops_p50"] = round(flops / (r["p50_us"] * 1e-6) / 1e9, 1)
            rows.append(r)
    return rows


def _cublas():
    """cuBLAS handle functions and cublasSgemmGroupedBatched through ctypes
    (the comparator only; nothing of this library calls cuBLAS)."""
    for name in ("libcublas.so.13", "libcublas.so"):
        try:
            lib = ctypes.CDLL(name)
            break
        except OSError:
            lib = None
    if lib is None or not hasattr(lib, "cublasSgemmGroupedBatched"):
        return None
    vp, i = ctypes.c_void_p, ctypes.c_int
    lib.cublasCreate_v2.argtypes = [ctypes.POINTER(vp)]
    lib.cublasSetStream_v2.argtypes = [vp, vp]
    lib.cublasDestroy_v2.argtypes = [vp]
    lib.cublasSgemmGroupedBatched.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                              vp, i, vp]
    for f in ("cublasCreate_v2", "cublasSetStream_v2", "cublasDestroy_v2",
              "cublasSgemmGroupedBatched"):
        getattr(lib, f).restype = i
    return lib


def vbatch_compare(dev, N=1_000_000, reps=20):
    """The variable-size batch (fp32, N problems, m = n = k = p + 1 with
    P(p) ~ 1/p, beta per problem in {0, 1}, back to back in one arena): this
    library's plan (one persistent launch) against cublasSgemmGroupedBatched
    on the same arena (problems grouped by size and beta, device arrays of
    pointers).  Both start from the same C once and their results are
    compared; then `reps` runs of each back to back (0.65 GB per run)."""
    import torch
    from paper_1304_7053_gb300 import inputs
    lib = _cublas()
    desc, la, lb, lc = inputs.vbatch_problems(N, seed=0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    A = torch.rand(la, device=dev, generator=gen) * 2 - 1
    B = torch.rand(lb, device=dev, generator=gen) * 2 - 1
    C0 = torch.rand(lc, device=dev, generator=gen) * 2 - 1
    sizes = desc[:, 0]
    bz = (desc[:, 3] >> 4) & 1
    alg_bytes = int(np.sum(4 * sizes * sizes * (3 + (1 - bz))))
    flops = int(np.sum(2 * sizes ** 3))
    s = torch.cuda.Stream(device=dev)
    plan = sbgemm.VPlan("s", sbgemm.vproblems_from_desc(desc))
    C1 = C0.clone()
    out = {"problems": N, "algorithmic_bytes": alg_bytes}

    def timed(fn):
        with torch.cuda.stream(s):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                fn()
            e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        return {"ms": round(ms, 4), "gbps": round(alg_bytes / (ms * 1e-3) / 1e9, 1),
                "gflops": round(flops / (ms * 1e-3) / 1e9, 1)}

    with torch.cuda.stream(s):
        plan.run(1.0, A, B, 1.0, C1, stream=s)
    torch.cuda.synchronize()
    if lib is None:
        out["sbgemm_vbatch"] = timed(lambda: plan.run(1.0, A, B, 1.0, C1, stream=s))
        plan.close()
        out["cublas_grouped"] = "unavailable: cublasSgemmGroupedBatched not found"
        return out
    # groups: (size, beta-zero); problems of a group in arena order
    keys = sizes * 2 + bz
    order = np.argsort(keys, kind="stable")
    gk, gsize = np.unique(keys[order], return_counts=True)
    G = len(gk)
    gm = (gk // 2).astype(np.int32)
    gbeta = np.where(gk % 2 == 1, 0.0, 1.0).astype(np.float32)
    ops = np.zeros(G, dtype=np.int32)                       # CUBLAS_OP_N
    alpha = np.ones(G, dtype=np.float32)
    gsize = gsize.astype(np.int32)
    C2 = C0.clone()
    offs = desc[order]
    ptrs = np.stack([A.data_ptr() + 4 * offs[:, 4], B.data_ptr() + 4 * offs[:, 5],
                     C2.data_ptr() + 4 * offs[:, 6]]).astype(np.int64)
    dptr = torch.from_numpy(ptrs).to(dev)
    h = ctypes.c_void_p()
    if lib.cublasCreate_v2(ctypes.byref(h)) != 0:
        out["sbgemm_vbatch"] = timed(lambda: plan.run(1.0, A, B, 1.0, C1, stream=s))
        plan.close()
        out["cublas_grouped"] = "unavailable: cublasCreate failed"
        return out
    lib.cublasSetStream_v2(h, ctypes.c_void_p(s.cuda_stream))
    ad = lambda x: ctypes.c_void_p(x.ctypes.data)
    keep = (ops, gm, alpha, gbeta, gsize)

    def cub():
        st = lib.cublasSgemmGroupedBatched(
            h, ad(ops), ad(ops), ad(gm), ad(gm), ad(gm), ad(alpha),
            ctypes.c_void_p(dptr[0].data_ptr()), ad(gm), ctypes.c_void_p(dptr[1].data_ptr()),
            ad(gm), ad(gbeta), ctypes.c_void_p(dptr[2].data_ptr()), ad(gm), G, ad(gsize))
        if st != 0:
            raise RuntimeError(f"cublasSgemmGroupedBatched status {st}")
    try:
        with torch.cuda.stream(s):
            cub()
        torch.cuda.synchronize()
        # one run of each from the same C: the same products up to rounding
        out["max_abs_diff_first_run"] = (C1 - C2).abs().max().item()
        out["sbgemm_vbatch"] = timed(lambda: plan.run(1.0, A, B, 1.0, C1, stream=s))
        out["cublas_grouped"] = timed(cub)
        out["cublas_groups"] = G
    finally:
        lib.cublasDestroy_v2(h)
        plan.close()
        del keep
    return out


def size_class(N):
    c = 0
    while N >= 10 and c < 7:
        N //= 10
        c += 1
    return c


def row(dtype, ta, tb, m, n, k, N, beta, ms, cublas_ms=None):
    es = ES[dtype]
    fl = (8 if dtype in CPLX else 2) * m * n * k * N
    by = es * N * (m * k + k * n + m * n * (1 + (complex(beta) != 0)))
    r = {"dtype": dtype, "op": ta + tb, "m": m, "n": n, "k": k, "N": N, "beta": str(beta),
         "ms": round(ms, 5), "gflops": round(fl / (ms * 1e-3) / 1e9, 1),
         "gbps": round(by / (ms * 1e-3) / 1e9, 1)}
    if cublas_ms is not None:
        r["cublas_ms"] = round(cublas_ms, 5)
        r["speedup_vs_cublas"] = round(cublas_ms / ms, 2)
    return r


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="sweep.json")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--fp64tc-types", default="d,z", type=lambda v: v.split(","),
                    help="types of the fp64tc section (d, z)")
    ap.add_argument("--fixed-types", default="s,d,c,z", type=lambda v: v.split(","),
                    help="types of the fixed section")
    ap.add_argument("--quick", action="store_true", help="N = 1e5 only, fewer sizes")
    ap.add_argument("--sections", default="small,fixed,ops,fem,interface,shared_a,16bit",
                    help="comma-separated subset of the sections to run "
                         "(grouped_config, vbatch, once and once16 run only when named)")
    args = ap.parse_args(argv)
    want = set(args.sections.split(","))
    import torch
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    rows = []
    Ns = [100_000] if args.quick else [1_000, 100_000, 1_000_000]
    sizes = [2, 4, 8, 10, 12, 16] if args.quick else list(range(1, 17))
    if "grouped_config" in want:
        for dtype in ("s", "d"):
            for r in grouped_config_sweep(dtype, dev):
                r["section"] = "grouped_config"
                rows.append(r)
                print(json.dumps(r), flush=True)
        want.discard("grouped_config")
        if not want:
            with open(args.out, "w") as f:
                json.dump(rows, f)
            return rows
    if "once" in want:
        pools = Pools(16 * 256 * 100_000 + 4096, dev)
        for dtype in ("s", "d", "z"):
            for m in range(8, 17):
                S = m * m
                pools.evict()
                pA, pB, pC = pools.for_type(dtype)
                sbgemm.gemm_multi_uniform(dtype, "N", "N", m, m, m, 1.0, pA.data_ptr(), m, S,
                                          pB.data_ptr(), m, S, 0.0, pC.data_ptr(), m, S,
                                          100_000)
        torch.cuda.synchronize()
        want.discard("once")
        if not want:
            with open(args.out, "w") as f:
                json.dump(rows, f)
            return rows
    if "once16" in want:
        # one call per 16-bit case at N = 1e6 (the tensor-core kernel at
        # m = 8, 12, 16), each after an L2 eviction: the launches a profiler
        # captures for the 16-bit table
        pools = Pools(256 * 1_000_000 * 2 + 4096, dev)
        for dtype in ("h", "b"):
            for m in (8, 12, 16):
                for beta in (0.0, -0.5):
                    S = m * m
                    pools.evict()
                    pA, pB, pC = pools.for_type(dtype)
                    sbgemm.gemm_multi_uniform(dtype, "N", "N", m, m, m, 1.5, pA.data_ptr(), m, S,
                                              pB.data_ptr(), m, S, beta, pC.data_ptr(), m, S,
                                              1_000_000)
        torch.cuda.synchronize()
        want.discard("once16")
        if not want:
            with open(args.out, "w") as f:
                json.dump(rows, f)
            return rows
    if "vbatch" in want:
        r = vbatch_compare(dev)
        r["section"] = "vbatch"
        rows.append(r)
        print(json.dumps(r), flush=True)
        want.discard("vbatch")
        if not want:
            with open(args.out, "w") as f:
                json.dump(rows, f)
            return rows
    pools = Pools(16 * 256 * 1_000_000 + 4096, dev)

    def emit(r, section):
        r["section"] = section
        rows.append(r)
        print(json.dumps(r), flush=True)

    # the small configuration (L2-resident, launch-bound)
    if "small" in want:
        for r in small_case(pools):
            emit(r, "small")
    # fixed-size sweep, op N/N
    if "fixed" in want:
        for dtype in args.fixed_types:
            for N in Ns:
                for m in sizes:
                    for beta in (0.0, -0.5):
                        alpha = 1.5
                        ms = time_ours(pools, dtype, "N", "N", m, m, m, N, alpha, beta, args.reps)
                        cb = time_cublas(pools, dtype, m, m, m, N, args.reps) if beta == 0.0 else None
                        emit(row(dtype, "N", "N", m, m, m, N, beta, ms, cb), "fixed")
    # op sweep: complex single, N = 1e5, general alpha/beta
    if "ops" in want:
        for m in sizes:
            for ta in "NTC":
                for tb in "NTC":
                    ms = time_ours(pools, "c", ta, tb, m, m, m, 100_000, 1.5 - 0.5j, -0.5 + 0.25j, args.reps)
                    emit(row("c", ta, tb, m, m, m, 100_000, -0.5, ms), "ops")
    # FEM-like rectangular shapes
    if "fem" in want:
        for dtype in ("s", "d"):
            for (m, n, k) in ((4, 16, 4), (9, 16, 9), (16, 8, 16), (3, 9, 3), (16, 16, 1)):
                ms = time_ours(pools, dtype, "T", "N", m, n, k, 500_000, 1.0, 1.0, args.reps)
                emit(row(dtype, "T", "N", m, n, k, 500_000, 1.0, ms), "fem")
    # interface comparison (Section 7's cuBLAS comparison): the 3-D layout,
    # the pointer-array form and cuBLAS strided batched, N = 1e5, beta = 0
    if "interface" in want:
        for dtype in ("s", "d", "c", "z"):
            for m in sizes:
                ms_u = time_ours(pools, dtype, "N", "N", m, m, m, 100_000, 1.0, 0.0, args.reps)
                ms_p = time_nounif(pools, dtype, m, 100_000, args.reps)
                cb = time_cublas(pools, dtype, m, m, m, 100_000, args.reps)
                r = row(dtype, "N", "N", m, m, m, 100_000, 0.0, ms_u, cb)
                r["nounif_ms"] = round(ms_p, 5)
                r["nounif_gflops"] = round((8 if dtype in CPLX else 2) * m ** 3 * 100_000 / (ms_p * 1e-3) / 1e9, 1)
                r["uniform_over_nounif"] = round(ms_p / ms_u, 2)
                emit(r, "interface")
    # one A shared by every pair (lda2 = 0) against a streamed A, N = 1e6
    if "shared_a" in want:
        for dtype in ("s", "d"):
            for m in sizes:
                ms_s = time_ours(pools, dtype, "N", "N", m, m, m, 1_000_000, 1.0, 0.0, args.reps,
                                 shared_a=True)
                ms_u = time_ours(pools, dtype, "N", "N", m, m, m, 1_000_000, 1.0, 0.0, args.reps)
                r = row(dtype, "N", "N", m, m, m, 1_000_000, 0.0, ms_s)
                r["gbps"] = round(ES[dtype] * 1_000_000 * 2 * m * m / (ms_s * 1e-3) / 1e9, 1)
                r["streamed_a_ms"] = round(ms_u, 5)
                r["speedup_vs_streamed_a"] = round(ms_u / ms_s, 2)
                emit(r, "shared_a")
    # real fp64: the fp64 FMA kernel (variant 0) against the tensor-core
    # kernel (variant 7), square N/N and the FEM shapes, alpha = 1.5
    if "fp64tc" in want:
        for dt in args.fp64tc_types:
            for N in (100_000, 1_000_000):
                for (m, n, k, ta, beta) in [(s_, s_, s_, "N", b_) for s_ in sizes for b_ in (0.0, -0.5)] + \
                        [(4, 16, 4, "T", 1.0), (9, 16, 9, "T", 1.0), (16, 8, 16, "T", 1.0),
                         (3, 9, 3, "T", 1.0), (16, 16, 1, "T", 1.0)]:
                    if N == 1_000_000 and (m != n or m not in (8, 12, 13, 14, 15, 16)):
                        continue
                    ms0 = time_ours(pools, dt, ta, "N", m, n, k, N, 1.5, beta, args.reps, variant=0)
                    ms7 = time_ours(pools, dt, ta, "N", m, n, k, N, 1.5, beta, args.reps, variant=7)
                    r = row(dt, ta, "N", m, n, k, N, beta, ms7)
                    r["fma_ms"] = round(ms0, 5)
                    r["tensor_over_fma_speedup"] = round(ms0 / ms7, 2)
                    emit(r, "fp64tc")
    # 16-bit storage
    if "16bit" in want:
        for dtype in ("h", "b"):
            for m in (8, 12, 16):
                for beta in (0.0, -0.5):
                    ms = time_ours(pools, dtype, "N", "N", m, m, m, 1_000_000, 1.5, beta, args.reps)
                    cb = time_cublas(pools, dtype, m, m, m, 1_000_000, args.reps) if beta == 0.0 else None
                    emit(row(dtype, "N", "N", m, m, m, 1_000_000, beta, ms, cb), "16bit")
    with open(args.out, "w") as f:
        json.dump(rows, f)
    return rows


if __name__ == "__main__":
    main(sys.argv[1:])
