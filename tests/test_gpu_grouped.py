"""GPU parity of the grouped call: square N/N flat groups share one
persistent launch, the other groups fall back to separate calls; every
group's result is compared with the oracle."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

from paper_1304_7053_gb300 import inputs, sbgemm
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def build(dtype, specs, int_valued):
    groups = (sbgemm.Group * len(specs))()
    keep = []
    for g, (ta, tb, m, n, k, N, pad) in zip(groups, specs):
        b = inputs.UniformBatch(dtype, ta, tb, m, n, k, N, seed=7 * m + n, int_valued=int_valued,
                                pad_ld=pad, pad_ld2=pad)
        tA, pA = H.to_dev(b.A)
        tB, pB = H.to_dev(b.B)
        tC, pC = H.to_dev(b.C)
        g.transa, g.transb, g.m, g.n, g.k = ta.encode(), tb.encode(), m, n, k
        g.A, g.lda, g.lda2 = pA, b.lda, b.lda2
        g.B, g.ldb, g.ldb2 = pB, b.ldb, b.ldb2
        g.C, g.ldc, g.ldc2 = pC, b.ldc, b.ldc2
        g.batchCount = N
        keep.append((b, tA, tB, tC))
    return groups, keep


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z", "h"])
@pytest.mark.parametrize("beta", [0.0, -0.5])
def test_grouped_matches_oracle(dtype, beta):
    int_valued = dtype in "sdcz"
    specs = [("N", "N", s, s, s, 997 + 31 * s, 0) for s in range(1, 17)]
    specs += [("T", "N", 5, 5, 5, 300, 0), ("N", "N", 4, 4, 4, 200, 1), ("N", "N", 3, 7, 2, 150, 0),
              ("N", "N", 8, 8, 8, 0, 0)]
    groups, keep = build(dtype, specs, int_valued)
    alpha = 1.5
    ab, bb = sbgemm._scalar_buf(dtype, alpha), sbgemm._scalar_buf(dtype, beta)
    s = torch.cuda.current_stream()
    st = sbgemm.lib().sbgemm_gemm_grouped(sbgemm.TYPE_CODES[dtype], ctypes.addressof(ab),
                                          ctypes.addressof(bb), ctypes.addressof(groups), len(specs),
                                          0, s.cuda_stream)
    assert st == 0, sbgemm.status_string(st)
    s.synchronize()
    for b, tA, tB, tC in keep:
        got, _ = H.from_dev(tC, b.C)
        H.assert_parity(b, got, H.oracle_ref(b, alpha, beta), alpha, beta,
                        exact=int_valued)


def test_grouped_device_scalars_and_errors():
    specs = [("N", "N", s, s, s, 500, 0) for s in (2, 9, 16)]
    groups, keep = build("s", specs, False)
    a = torch.tensor([1.5], device="cuda")
    bta = torch.tensor([-0.5], device="cuda")
    s = torch.cuda.current_stream()
    st = sbgemm.lib().sbgemm_gemm_grouped(0, a.data_ptr(), bta.data_ptr(), ctypes.addressof(groups),
                                          len(specs), 1, s.cuda_stream)
    assert st == 0
    s.synchronize()
    for b, tA, tB, tC in keep:
        H.assert_parity(b, H.from_dev(tC, b.C)[0], H.oracle_ref(b, 1.5, -0.5), 1.5, -0.5)
    # a bad group is rejected before anything runs
    groups[1].lda = 1
    ab = sbgemm._scalar_buf("s", 1.0)
    st = sbgemm.lib().sbgemm_gemm_grouped(0, ctypes.addressof(ab), ctypes.addressof(ab),
                                          ctypes.addressof(groups), len(specs), 0, s.cuda_stream)
    assert st == -3


@pytest.mark.parametrize("cfg", [(256, 16384, 4), (128, 8192, 2), (256, 65536, 2)])
def test_grouped_launch_configurations(cfg):
    """Every launch configuration gives the oracle's result (bit-exact on
    small integers)."""
    specs = [("N", "N", s, s, s, 700 + 13 * s, 0) for s in (1, 3, 4, 7, 8, 12, 13, 16)]
    groups, keep = build("s", specs, True)
    sbgemm.grouped_config("s", *cfg)
    try:
        ab, bb = sbgemm._scalar_buf("s", 1.5), sbgemm._scalar_buf("s", -0.5)
        s = torch.cuda.current_stream()
        st = sbgemm.lib().sbgemm_gemm_grouped(0, ctypes.addressof(ab), ctypes.addressof(bb),
                                              ctypes.addressof(groups), len(specs), 0,
                                              s.cuda_stream)
        assert st == 0, sbgemm.status_string(st)
        s.synchronize()
    finally:
        sbgemm.grouped_config("s")
    for b, tA, tB, tC in keep:
        H.assert_parity(b, H.from_dev(tC, b.C)[0], H.oracle_ref(b, 1.5, -0.5), 1.5, -0.5,
                        exact=True)


def test_grouped_full_size_sampled():
    """The benchmark's step at full size in its launch configuration: fp32,
    m = 1..16 with N = 100,000 pairs each, op N/N, alpha = 1, beta = 0, one
    grouped call (C starts as NaN, so a read of C would show), checked on a
    sample of pairs of every size that the oracle computes one by one."""
    N = 100_000
    sizes = list(range(1, 17))
    groups = (sbgemm.Group * len(sizes))()
    keep = {}
    for g, m in zip(groups, sizes):
        S = m * m
        A = inputs.draw("s", N * S, 1000 + m)
        B = inputs.draw("s", N * S, 2000 + m)
        tA, pA = H.to_dev(A)
        tB, pB = H.to_dev(B)
        tC = torch.full((N * S,), float("nan"), dtype=torch.float32, device=H.dev())
        g.transa, g.transb, g.m, g.n, g.k = b"N", b"N", m, m, m
        g.A, g.lda, g.lda2 = pA, m, S
        g.B, g.ldb, g.ldb2 = pB, m, S
        g.C, g.ldc, g.ldc2 = tC.data_ptr(), m, S
        g.batchCount = N
        keep[m] = (A, B, tA, tB, tC)
    ab, bb = sbgemm._scalar_buf("s", 1.0), sbgemm._scalar_buf("s", 0.0)
    s = torch.cuda.current_stream()
    st = sbgemm.lib().sbgemm_gemm_grouped(0, ctypes.addressof(ab), ctypes.addressof(bb),
                                          ctypes.addressof(groups), len(sizes), 0, s.cuda_stream)
    assert st == 0, sbgemm.status_string(st)
    s.synchronize()
    for m in sizes:
        A, B, tA, tB, tC = keep[m]
        S = m * m
        got = tC.cpu().numpy()
        pick = np.unique((inputs.splitmix64(3000 + m, 256) % np.uint64(N)).astype(np.int64))
        pick = np.concatenate([pick, [N - 1]])
        sub = inputs.UniformBatch("s", "N", "N", m, m, m, pick.size, seed=0)
        sub.A = A.reshape(N, S)[pick].ravel().copy()
        sub.B = B.reshape(N, S)[pick].ravel().copy()
        sub.C = np.full(pick.size * S, np.nan, dtype=np.float32)
        ref = H.oracle_ref(sub, 1.0, 0.0)
        H.assert_parity(sub, got.reshape(N, S)[pick].ravel().copy(), ref, 1.0, 0.0)
        assert np.all(np.isfinite(got)), f"m={m}: an entry of C was not written"


def test_tuned_grouped_config_installed_and_exact():
    """The autotuner times the grouped call under each candidate launch
    configuration, installs the fastest, and the call stays exact."""
    from paper_1304_7053_gb300 import selector
    specs = [("N", "N", s, s, s, 3000 + s, 0) for s in (2, 7, 12, 16)]
    groups, keep = build("s", specs, True)
    ab, bb = sbgemm._scalar_buf("s", 1.5), sbgemm._scalar_buf("s", -0.5)
    s = torch.cuda.current_stream()

    def call():
        st = sbgemm.lib().sbgemm_gemm_grouped(0, ctypes.addressof(ab), ctypes.addressof(bb),
                                              ctypes.addressof(groups), len(specs), 0,
                                              s.cuda_stream)
        assert st == 0

    try:
        cfgs = [(128, 16384, 2), (128, 28672, 2), (256, 32768, 2)]
        best, times = selector.tune_grouped("s", call, configs=cfgs, reps=3, stream=s)
        assert best in cfgs and times[best] == min(times.values())
        for b, tA, tB, tC in keep:          # fresh C, then one call with the tuned launch
            tC.copy_(torch.from_numpy(b.C.view(np.uint8)).cuda())
        call()
        s.synchronize()
        for b, tA, tB, tC in keep:
            H.assert_parity(b, H.from_dev(tC, b.C)[0], H.oracle_ref(b, 1.5, -0.5), 1.5, -0.5,
                            exact=True)
    finally:
        sbgemm.grouped_config("s")


@pytest.mark.parametrize("dtype", ["s", "d", "c", "b"])
@pytest.mark.parametrize("beta", [0.0, -0.5])
def test_grouped_sizes_off_the_16_byte_grid(dtype, beta):
    """Sizes whose matrices are not a whole number of 16-byte chunks (tiles
    a multiple of 2-8 pairs, a ragged last tile whose final chunk is
    partial): results match the oracle and the bytes around every C stay
    untouched."""
    int_valued = dtype in "sdc"
    sizes = list(range(1, 17, 2)) + [6, 10, 14]
    groups = (sbgemm.Group * len(sizes))()
    keep = []
    guard_front, guard_back = 32, 48
    for g, m in zip(groups, sizes):
        N = 1000 + 37 * m
        b = inputs.UniformBatch(dtype, "N", "N", m, m, m, N, seed=11 * m, int_valued=int_valued)
        tA, pA = H.to_dev(b.A)
        tB, pB = H.to_dev(b.B)
        tC, pC = H.to_dev(b.C, pad_front=guard_front, pad_back=guard_back)
        g.transa, g.transb, g.m, g.n, g.k = b"N", b"N", m, m, m
        g.A, g.lda, g.lda2 = pA, m, m * m
        g.B, g.ldb, g.ldb2 = pB, m, m * m
        g.C, g.ldc, g.ldc2 = pC, m, m * m
        g.batchCount = N
        keep.append((b, tA, tB, tC))
    ab, bb = sbgemm._scalar_buf(dtype, 1.5), sbgemm._scalar_buf(dtype, beta)
    s = torch.cuda.current_stream()
    st = sbgemm.lib().sbgemm_gemm_grouped(sbgemm.TYPE_CODES[dtype], ctypes.addressof(ab),
                                          ctypes.addressof(bb), ctypes.addressof(groups),
                                          len(sizes), 0, s.cuda_stream)
    assert st == 0, sbgemm.status_string(st)
    s.synchronize()
    for b, tA, tB, tC in keep:
        got, raw = H.from_dev(tC, b.C, pad_front=guard_front)
        assert np.all(raw[:guard_front] == 0x5A) and np.all(raw[guard_front + b.C.nbytes:] == 0x5A)
        H.assert_parity(b, got, H.oracle_ref(b, 1.5, beta), 1.5, beta, exact=int_valued)
