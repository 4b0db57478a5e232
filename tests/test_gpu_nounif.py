"""GPU parity of the pointer-array form (Section 4's TGEMM_multi_nounif).

The matrices live in arenas of uniform slots; pair p uses A slot pa[p] and
B slot pb[p] (repeats allowed) and C slot pc[p] (all distinct).  The oracle
runs on the gathered uniform batch; the arena slots the call must not touch
keep their bytes."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_1304_7053_gb300 import inputs, sbgemm
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def gather(x, ld2, slots, idx):
    return np.ascontiguousarray(x.reshape(slots, ld2)[idx]).ravel()


def run_case(dtype, shape, pads, N, alpha, beta, seed, device_scalars=False):
    ta, tb, m, n, k = shape
    exact = dtype in "sdcz"
    slots = N + 37
    ar = inputs.UniformBatch(dtype, ta, tb, m, n, k, slots, seed=seed, int_valued=exact,
                             pad_ld=pads[0], pad_ld2=pads[1])
    rng = np.random.default_rng(seed)
    pa = rng.integers(0, slots, N)
    pb = rng.integers(0, slots, N)
    pc = rng.permutation(slots)[:N]
    es = ar.A.itemsize
    tA, pA = H.to_dev(ar.A)
    tB, pB = H.to_dev(ar.B)
    tC, pC = H.to_dev(ar.C)
    ptr = lambda base, ld2, idx: torch.tensor(base + idx.astype(np.int64) * ld2 * es,
                                              dtype=torch.int64, device=H.dev())
    Ap, Bp, Cp = ptr(pA, ar.lda2, pa), ptr(pB, ar.ldb2, pb), ptr(pC, ar.ldc2, pc)
    if device_scalars:
        sd = {"s": np.float32, "h": np.float32, "b": np.float32, "d": np.float64,
              "c": np.complex64, "z": np.complex128}[dtype]
        ta_, a_arg = H.to_dev(np.array([alpha], dtype=sd))
        tb_, b_arg = H.to_dev(np.array([beta], dtype=sd))
    else:
        a_arg, b_arg = alpha, beta
    sbgemm.gemm_multi_nounif(dtype, ta, tb, m, n, k, a_arg, Ap, ar.lda, Bp, ar.ldb, b_arg, Cp,
                             ar.ldc, N, device_scalars=device_scalars)
    torch.cuda.synchronize()
    got, _ = H.from_dev(tC, ar.C)
    # the gathered uniform batch the oracle sees
    g = inputs.UniformBatch(dtype, ta, tb, m, n, k, 1, seed=0, pad_ld=pads[0], pad_ld2=pads[1])
    g.batch = N
    g.A = gather(ar.A, ar.lda2, slots, pa)
    g.B = gather(ar.B, ar.ldb2, slots, pb)
    g.C = gather(ar.C, ar.ldc2, slots, pc)
    ref = H.oracle_ref(g, alpha, beta)
    H.assert_parity(g, gather(got, ar.ldc2, slots, pc), ref, alpha, beta, exact=exact)
    untouched = np.setdiff1d(np.arange(slots), pc)
    assert np.array_equal(gather(got, ar.ldc2, slots, untouched).view(np.uint8),
                          gather(ar.C, ar.ldc2, slots, untouched).view(np.uint8))


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z", "h", "b"])
@pytest.mark.parametrize("shape", [("N", "N", 16, 16, 16), ("T", "C", 5, 7, 3),
                                   ("N", "T", 8, 8, 8), ("N", "N", 7, 3, 11)])
@pytest.mark.parametrize("pads", [(0, 0), (1, 1), (0, 1)])
def test_nounif_matches_oracle(dtype, shape, pads):
    for beta in (0.0, -0.5):
        run_case(dtype, shape, pads, 1500, 1.5, beta, seed=3 + shape[2] + 5 * pads[1])


@pytest.mark.parametrize("dtype", ["s", "z"])
def test_nounif_device_scalars_and_scale_path(dtype):
    run_case(dtype, ("N", "N", 12, 12, 12), (0, 0), 900, 1.5, -0.5, seed=11, device_scalars=True)
    # alpha = 0: C = beta * C through the pointers, A and B unread
    run_case(dtype, ("N", "N", 4, 4, 4), (0, 1), 900, 0.0, -0.5, seed=12)
    # k = 0
    run_case(dtype, ("N", "N", 4, 4, 0), (0, 0), 300, 1.5, -0.5, seed=13)
