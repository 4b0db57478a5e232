"""16-bit storage with fp32 accumulation: error against the fp64 oracle.

For binary16 and bfloat16 at m = n = k in {8, 12, 16}, N = 1,000,000 pairs
(uniform[-1, 1] rounded to 16 bits), the GPU result is compared on a sample
of pairs with
  (a) the oracle on the 16-bit inputs: the arithmetic error, held to the
      bound of tests/gpu_helpers.py (fp32 accumulation plus the final
      rounding to 16 bits);
  (b) the oracle on the unrounded inputs: the total error of storing the
      operands in 16 bits, reported (it is dominated by input quantisation).
With SBGEMM_REPORT_DIR set, the statistics are written to
precision_16bit.json there."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1304_7053_gb300 import inputs, sbgemm
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

REPORT = {}


@pytest.mark.parametrize("dtype", ["h", "b"])
@pytest.mark.parametrize("m", [8, 12, 16])
def test_16bit_error_vs_fp64_oracle(dtype, m):
    N = 1_000_000
    S = m * m
    x_a = inputs.uniform(101, N * S)
    x_b = inputs.uniform(102, N * S)
    A16, B16 = inputs.to_storage(x_a, dtype), inputs.to_storage(x_b, dtype)
    C16 = np.zeros(N * S, dtype=np.uint16)
    tA, pA = H.to_dev(A16)
    tB, pB = H.to_dev(B16)
    tC, pC = H.to_dev(C16)
    sbgemm.gemm_multi_uniform(dtype, "N", "N", m, m, m, 1.0, pA, m, S, pB, m, S, 0.0, pC, m, S, N)
    torch.cuda.synchronize()
    got16 = H.from_dev(tC, C16)[0]
    pick = np.unique((inputs.splitmix64(103, 2000) % np.uint64(N)).astype(np.int64))
    n = pick.size
    sub = lambda x: x.reshape(N, S)[pick].ravel().copy()
    Az, Bz = sub(A16), sub(B16)
    got = oracle._decode16(sub(got16), dtype)
    ref16 = oracle.gemm_uniform(dtype, "N", "N", m, m, m, 1.0, Az, m, S, Bz, m, S, 0.0,
                                np.zeros(n * S, np.uint16), m, S, n, threads=8)
    # (a) arithmetic error on the 16-bit inputs, against the bound
    b = inputs.UniformBatch(dtype, "N", "N", m, m, m, n, seed=0)
    b.A, b.B, b.C = Az, Bz, np.zeros(n * S, np.uint16)
    H.assert_parity(b, sub(got16), ref16, 1.0, 0.0)
    # (b) total error against the unrounded fp32 inputs
    Af, Bf = sub(x_a.astype(np.float32)), sub(x_b.astype(np.float32))
    reff = oracle.gemm_uniform("s", "N", "N", m, m, m, 1.0, Af, m, S, Bf, m, S, 0.0,
                               np.zeros(n * S, np.float32), m, S, n, threads=8)
    scale = np.abs(reff) + 1e-30
    rec = {
        "pairs_checked": int(n),
        "arith_max_abs": float(np.max(np.abs(got - ref16))),
        "arith_max_rel_to_result": float(np.max(np.abs(got - ref16) / (np.abs(ref16) + 1e-30))),
        "arith_rms": float(np.sqrt(np.mean((got - ref16) ** 2))),
        "total_max_abs_vs_fp32_inputs": float(np.max(np.abs(got - reff))),
        "total_rms_vs_fp32_inputs": float(np.sqrt(np.mean((got - reff) ** 2))),
        "total_median_rel_vs_fp32_inputs": float(np.median(np.abs(got - reff) / scale)),
        "result_rms": float(np.sqrt(np.mean(reff ** 2))),
    }
    REPORT[f"{dtype}_m{m}"] = rec
    d = os.environ.get("SBGEMM_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "precision_16bit.json"), "w") as f:
            json.dump(REPORT, f, indent=1)
