"""The allocation-free variable-size entry point (for callers that cannot
allocate device memory while they run) against the plan-based entry point.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test; it also passes on its own in a
fresh process."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

from paper_1304_7053_gb300 import inputs, sbgemm
from tests import gpu_helpers as H
from tests.test_gpu_vbatch import vbound

pytestmark = pytest.mark.gpu


def mixed_desc(count, seed):
    """Square sizes with weights 1/p, mixed beta, plus some rectangular and
    transposed problems (generic buckets) and some m = 0 problems."""
    desc, la, lb, lc = inputs.vbatch_problems(count, seed=seed)
    r = inputs.splitmix64(seed + 99, count)
    rect = (r % np.uint64(7)) == 0
    desc[rect, 1] = np.maximum(1, desc[rect, 1] - 1)          # n = m - 1
    desc[rect, 3] |= (((r[rect] >> np.uint64(8)) % np.uint64(3)).astype(np.int64))  # opA
    desc[(r % np.uint64(97)) == 5, 0] = 0                        # a few empty problems
    return desc, la, lb, lc


def run_plan(dtype, desc, A, B, C, alpha, beta):
    tA, pA = H.to_dev(A)
    tB, pB = H.to_dev(B)
    tC, pC = H.to_dev(C)
    plan = sbgemm.VPlan(dtype, sbgemm.vproblems_from_desc(desc))
    plan.run(alpha, pA, pB, beta, pC)
    torch.cuda.synchronize()
    plan.close()
    return H.from_dev(tC, C)[0]


def run_noalloc(dtype, dprob, count, pA, pB, tC, C0, alpha, beta):
    tC.copy_(C0)
    ab, bb = sbgemm._scalar_buf(dtype, alpha), sbgemm._scalar_buf(dtype, beta)
    s = torch.cuda.current_stream()
    st = sbgemm.lib().sbgemm_vbatch_run_noalloc(sbgemm.TYPE_CODES[dtype], dprob.data_ptr(), count,
                                                ctypes.addressof(ab), pA, pB, ctypes.addressof(bb),
                                                tC.data_ptr(), sbgemm.SCALARS_HOST, s.cuda_stream)
    assert st == 0, sbgemm.status_string(st)
    torch.cuda.synchronize()
    return tC.cpu().numpy().view(np.uint8)


@pytest.mark.parametrize("dtype", ["s", "d", "z"])
def test_noalloc_matches_plan_path_twice(dtype):
    count = 40000
    desc, la, lb, lc = mixed_desc(count, seed=5)
    # every problem keeps the s*s slots vbatch_problems laid out; the
    # rectangular ones (n = m - 1) use less of them
    A, B, C = inputs.draw(dtype, la, 1), inputs.draw(dtype, lb, 2), inputs.draw(dtype, lc, 3)
    alpha, beta = (1.5 - 0.5j, -0.5 + 0.25j) if dtype in "cz" else (1.5, -0.5)
    ref = run_plan(dtype, desc, A, B, C, alpha, beta)
    probs = sbgemm.vproblems_from_desc(desc)
    dprob = torch.from_numpy(probs.view(np.uint8).copy()).cuda()
    tA, pA = H.to_dev(A)
    tB, pB = H.to_dev(B)
    C0 = torch.from_numpy(C.view(np.uint8).copy()).cuda()
    tC = torch.empty_like(C0)
    bd = vbound(dtype, desc, A, B, C, alpha, beta)
    r = H.decode(ref, dtype)
    for _ in range(2):                     # two calls in a row share the static array
        got = H.decode(run_noalloc(dtype, dprob, count, pA, pB, tC, C0, alpha, beta).view(C.dtype), dtype)
        err = np.maximum(np.abs((got - r).real), np.abs((got - r).imag)) if dtype in "cz" else np.abs(got - r)
        assert np.all(err <= bd), float(np.max(err - bd))


def _noalloc_bound(dtype, desc, A, B, C, alpha, beta, ref):
    bd = vbound(dtype, desc, A, B, C, alpha, beta)
    if dtype in "hb":
        bd = H.U16[dtype] * np.abs(ref) + (1 + H.U16[dtype]) * bd + H.SUB16[dtype]
    return bd


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z", "h", "b"])
def test_noalloc_matches_oracle_twice(dtype):
    """Against the CPU oracle, element by element, on every storage type:
    square sizes with weights 1/p and mixed beta, rectangular and
    transposed or conjugated problems (generic buckets) and m = 0 problems,
    on two calls in a row (the second reuses the static array)."""
    import oracle
    count = 20000
    desc, la, lb, lc = mixed_desc(count, seed=11)
    A, B, C = inputs.draw(dtype, la, 21), inputs.draw(dtype, lb, 22), inputs.draw(dtype, lc, 23)
    alpha, beta = (1.5 - 0.5j, -0.5 + 0.25j) if dtype in "cz" else (1.5, -0.5)
    ref = oracle.gemm_vbatch(dtype, desc, alpha, A, B, beta, C, threads=8)
    bd = _noalloc_bound(dtype, desc, A, B, C, alpha, beta, ref)
    probs = sbgemm.vproblems_from_desc(desc)
    dprob = torch.from_numpy(probs.view(np.uint8).copy()).cuda()
    tA, pA = H.to_dev(A)
    tB, pB = H.to_dev(B)
    C0 = torch.from_numpy(C.view(np.uint8).copy()).cuda()
    tC = torch.empty_like(C0)
    for _ in range(2):
        got = H.decode(run_noalloc(dtype, dprob, count, pA, pB, tC, C0, alpha, beta).view(C.dtype),
                       dtype)
        err = (np.maximum(np.abs((got - ref).real), np.abs((got - ref).imag)) if dtype in "cz"
               else np.abs(got - ref))
        assert np.all(err <= bd), float(np.max(err - bd))


def test_noalloc_bad_problem_leaves_c_and_next_call_works():
    """A batch with one invalid problem (m = 17) is rejected with
    SBGEMM_ERR_INVALID_SIZE and no GEMM runs (C is unchanged); the next
    valid call on the same static array gives the plan path's result."""
    dtype, count = "s", 5000
    desc, la, lb, lc = mixed_desc(count, seed=13)
    A, B, C = inputs.draw(dtype, la, 31), inputs.draw(dtype, lb, 32), inputs.draw(dtype, lc, 33)
    tA, pA = H.to_dev(A)
    tB, pB = H.to_dev(B)
    C0 = torch.from_numpy(C.view(np.uint8).copy()).cuda()
    tC = C0.clone()
    bad = desc.copy()
    bad[count // 2, 0] = 17
    dbad = torch.from_numpy(sbgemm.vproblems_from_desc(bad).view(np.uint8).copy()).cuda()
    ab, bb = sbgemm._scalar_buf(dtype, 1.5), sbgemm._scalar_buf(dtype, -0.5)
    st = sbgemm.lib().sbgemm_vbatch_run_noalloc(0, dbad.data_ptr(), count, ctypes.addressof(ab), pA,
                                                pB, ctypes.addressof(bb), tC.data_ptr(),
                                                sbgemm.SCALARS_HOST, None)
    assert st == -2
    torch.cuda.synchronize()
    assert torch.equal(tC, C0)
    ref = run_plan(dtype, desc, A, B, C, 1.5, -0.5)
    dgood = torch.from_numpy(sbgemm.vproblems_from_desc(desc).view(np.uint8).copy()).cuda()
    got = run_noalloc(dtype, dgood, count, pA, pB, tC, C0, 1.5, -0.5)
    bd = vbound(dtype, desc, A, B, C, 1.5, -0.5)
    assert np.all(np.abs(got.view(np.float32).astype(np.float64) - ref.astype(np.float64)) <= 2 * bd)


def test_noalloc_call_allocates_no_device_memory():
    """After one warm-up call (which loads the kernels and looks up the
    static array), a call changes neither the driver's free device memory
    nor the bytes torch's allocator holds."""
    dtype, count = "d", 8000
    desc, la, lb, lc = mixed_desc(count, seed=17)
    A, B, C = inputs.draw(dtype, la, 41), inputs.draw(dtype, lb, 42), inputs.draw(dtype, lc, 43)
    tA, pA = H.to_dev(A)
    tB, pB = H.to_dev(B)
    C0 = torch.from_numpy(C.view(np.uint8).copy()).cuda()
    tC = torch.empty_like(C0)
    dprob = torch.from_numpy(sbgemm.vproblems_from_desc(desc).view(np.uint8).copy()).cuda()
    run_noalloc(dtype, dprob, count, pA, pB, tC, C0, 1.5, -0.5)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    held0 = torch.cuda.memory_allocated()
    ab, bb = sbgemm._scalar_buf(dtype, 1.5), sbgemm._scalar_buf(dtype, -0.5)
    st = sbgemm.lib().sbgemm_vbatch_run_noalloc(1, dprob.data_ptr(), count, ctypes.addressof(ab),
                                                pA, pB, ctypes.addressof(bb), tC.data_ptr(),
                                                sbgemm.SCALARS_HOST, None)
    assert st == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == held0


def test_noalloc_rejects_too_many_problems():
    one = sbgemm._scalar_buf("s", 1.0)
    st = sbgemm.lib().sbgemm_vbatch_run_noalloc(0, 16, 262145, ctypes.addressof(one), 16, 16,
                                                ctypes.addressof(one), 16, 0, None)
    assert st == -8
