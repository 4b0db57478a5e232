"""Runs after the other GPU tests (file order): no kernel of the session hit
the limit of a bounded barrier wait (the device error word is clear)."""
from __future__ import annotations

import ctypes

import pytest
import torch

from paper_1304_7053_gb300 import sbgemm

pytestmark = pytest.mark.gpu


def test_no_expired_waits_in_session():
    torch.cuda.synchronize()
    code = ctypes.c_int(-1)
    st = sbgemm.lib().sbgemm_device_error(ctypes.byref(code), None)
    assert st == 0, sbgemm.status_string(st)
    assert code.value == 0, f"a bounded in-kernel wait expired: {sbgemm.status_string(code.value)}"
