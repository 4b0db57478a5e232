"""An expired bounded wait is reported, without any fault.

The library's kernels bound every barrier wait; on expiry they record
SBGEMM_ERR_TIMEOUT in a per-device error word and return.  Here the wait is
made to expire on purpose through ``sbgemm_wait_selftest`` (a barrier armed
for copies that are never issued, polled a bounded number of times), and
the test checks that the code is reported once, then cleared, and that the
context still computes exact results."""
from __future__ import annotations

import ctypes

import pytest
import torch

from paper_1304_7053_gb300 import inputs, sbgemm
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def read_error():
    code = ctypes.c_int(-1)
    st = sbgemm.lib().sbgemm_device_error(ctypes.byref(code), None)
    assert st == 0, sbgemm.status_string(st)
    return code.value


def test_expired_wait_is_reported_and_cleared():
    torch.cuda.synchronize()
    # no earlier kernel of this session hit a wait limit
    assert read_error() == 0
    assert sbgemm.lib().sbgemm_wait_selftest(0, None) == -5
    assert sbgemm.lib().sbgemm_wait_selftest((1 << 22) + 1, None) == -5
    for limit in (1, 1000):
        assert sbgemm.lib().sbgemm_wait_selftest(limit, None) == 0
        torch.cuda.synchronize()
        assert read_error() == -6            # SBGEMM_ERR_TIMEOUT, once
        assert read_error() == 0             # cleared by the read
    # the context is intact: a bulk-copy shape (fp32 m = 13) is exact
    b = inputs.UniformBatch("s", "N", "N", 13, 13, 13, 5003, seed=31, int_valued=True)
    got = H.run_gpu(b, 1.5, -0.5)
    H.assert_parity(b, got, H.oracle_ref(b, 1.5, -0.5), 1.5, -0.5, exact=True)
    assert read_error() == 0
