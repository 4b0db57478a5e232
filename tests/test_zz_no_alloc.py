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


def test_noalloc_rejects_too_many_problems():
    one = sbgemm._scalar_buf("s", 1.0)
    st = sbgemm.lib().sbgemm_vbatch_run_noalloc(0, 16, 262145, ctypes.addressof(one), 16, 16,
                                                ctypes.addressof(one), 16, 0, None)
    assert st == -8
