"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/sbgemm.h declares, and rejects invalid arguments with
the documented status codes before touching the device."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

from paper_1304_7053_gb300 import sbgemm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(sbgemm_\w+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = sbgemm.lib()
    names = declared_symbols()
    assert len(names) >= 18
    for name in names:
        assert hasattr(L, name), f"{name} declared but not exported"
        assert name in sbgemm.SIGNATURES, f"{name} has no binding signature"


def test_binding_covers_only_declared_symbols():
    assert set(sbgemm.SIGNATURES) <= set(declared_symbols())


def call(dtype="s", ta="N", tb="N", m=2, n=2, k=2, lda=2, lda2=4, ldb=2, ldb2=4, ldc=2,
         ldc2=4, batch=1, A=16, B=16, C=16, mode=0, alpha=True, beta=True):
    a = sbgemm._scalar_buf(dtype, 1.0)
    b = sbgemm._scalar_buf(dtype, 0.0)
    L = sbgemm.lib()
    return L.sbgemm_gemm_multi_uniform_variant(
        sbgemm.TYPE_CODES[dtype], ta.encode(), tb.encode(), m, n, k,
        ctypes.addressof(a) if alpha else None, A, lda, lda2, B, ldb, ldb2,
        ctypes.addressof(b) if beta else None, C, ldc, ldc2, batch, mode, 0, None)


@pytest.mark.parametrize("kw,status", [
    (dict(ta="X"), -1), (dict(tb="q"), -1),
    (dict(m=17), -2), (dict(k=-1), -2), (dict(batch=-1), -2),
    (dict(lda=1), -3), (dict(ldc=1), -3), (dict(ldc2=3), -3), (dict(lda2=3), -3),
    (dict(ta="T", m=3, lda=2, ldc=3, ldc2=6), -3),
    (dict(C=0), -4), (dict(alpha=False), -4), (dict(A=0), -4),
    (dict(mode=7), -5), (dict(dtype="z", m=0), 0), (dict(batch=0), 0),
])
def test_argument_errors(kw, status):
    assert call(**kw) == status


def call_nounif(dtype="s", ta="N", tb="N", m=2, n=2, k=2, lda=2, ldb=2, ldc=2, batch=1,
                Ap=16, Bp=16, Cp=16, mode=0, alpha=True, beta=True):
    a = sbgemm._scalar_buf(dtype, 1.0)
    b = sbgemm._scalar_buf(dtype, 0.0)
    return sbgemm.lib().sbgemm_gemm_multi_nounif(
        sbgemm.TYPE_CODES[dtype], ta.encode(), tb.encode(), m, n, k,
        ctypes.addressof(a) if alpha else None, Ap, lda, Bp, ldb,
        ctypes.addressof(b) if beta else None, Cp, ldc, batch, mode, None)


@pytest.mark.parametrize("kw,status", [
    (dict(ta="X"), -1), (dict(m=17), -2), (dict(batch=-1), -2),
    (dict(lda=1), -3), (dict(ldc=1), -3), (dict(tb="T", n=3, ldb=2, ldc=2), -3),
    (dict(Cp=0), -4), (dict(beta=False), -4), (dict(Bp=0), -4),
    (dict(mode=3), -5), (dict(dtype="b", n=0), 0), (dict(batch=0), 0), (dict(dtype=None), -5),
])
def test_nounif_argument_errors(kw, status):
    """Pointer-array form: rejected before anything touches the device."""
    if kw.get("dtype", "s") is None:
        L = sbgemm.lib()
        a = sbgemm._scalar_buf("s", 1.0)
        assert L.sbgemm_gemm_multi_nounif(9, b"N", b"N", 2, 2, 2, ctypes.addressof(a), 16, 2, 16,
                                          2, ctypes.addressof(a), 16, 2, 1, 0, None) == status
        return
    assert call_nounif(**kw) == status


def test_status_strings_and_version():
    assert sbgemm.status_string(0) == "success"
    assert "trans" in sbgemm.status_string(-1)
    assert sbgemm.lib().sbgemm_version() >= 100


def test_variant_table_host_logic():
    assert sbgemm.num_variants("s", 16, 16, 16) == 7
    assert sbgemm.num_variants("s", 7, 3, 11) == 1 and sbgemm.num_variants("d", 7, 3, 11) == 2
    assert sbgemm.num_variants("s", 17, 3, 11) == 0
    assert "generic" in sbgemm.variant_name("s", 7, 3, 11, 0)
    # the 16-bit types at m = n = k = 8, 16 also have the tensor-core variant
    assert sbgemm.num_variants("b", 16, 16, 16) == 8 and sbgemm.num_variants("h", 8, 8, 8) == 8
    assert sbgemm.num_variants("b", 12, 12, 12) == 8 and sbgemm.num_variants("d", 16, 16, 16) == 8
    assert sbgemm.num_variants("z", 16, 16, 16) == 8 and sbgemm.num_variants("d", 9, 16, 9) == 8
    assert sbgemm.num_variants("z", 7, 3, 11) == 2 and sbgemm.num_variants("c", 7, 3, 11) == 1
    assert sbgemm.num_variants("h", 10, 10, 10) == 7
    assert "tensor-core" in sbgemm.variant_name("h", 16, 16, 16, 7)
    sbgemm.clear_choices()
    # defaults without a table entry: 32 KB two-stage tiles (variant 2) for
    # fp32 below 1e6 pairs and for complex64, the tensor cores for 16-bit
    # m = 8, 12, 16, variant 0 elsewhere, the generic kernel (0) off the table
    assert sbgemm.get_choice("s", 10, 10, 10, 0, 0, 1, 5) == 2
    assert sbgemm.get_choice("s", 10, 10, 10, 0, 0, 1, 6) == 0
    assert sbgemm.get_choice("c", 10, 10, 10, 0, 0, 1, 6) == 2
    assert sbgemm.get_choice("d", 10, 10, 10, 0, 0, 1, 5) == 0
    assert sbgemm.get_choice("d", 13, 13, 13, 1, 0, 1, 5) == 7
    # generic fp64 shapes: the tensor-core kernel (variant 1) from m n k = 1024
    # (beta == 0) or 1320 (beta != 0)
    assert sbgemm.get_choice("d", 16, 16, 15, 0, 0, 1, 5) == 1
    assert sbgemm.get_choice("d", 8, 8, 16, 0, 0, 1, 5) == 1
    assert sbgemm.get_choice("d", 8, 8, 16, 0, 0, 0, 5) == 0
    assert sbgemm.get_choice("d", 8, 11, 15, 0, 0, 0, 5) == 1
    assert sbgemm.get_choice("d", 7, 3, 11, 0, 0, 1, 5) == 0
    assert sbgemm.get_choice("s", 16, 16, 15, 0, 0, 1, 5) == 0
    # complex128: the tensor cores at m = n = k >= 12 and 16 x 8 x 16, on
    # generic shapes from m n k = 1024; real fp64 at m = n = k >= 13 and 12
    # with beta != 0
    assert sbgemm.get_choice("z", 13, 13, 13, 0, 0, 0, 5) == 7
    assert sbgemm.get_choice("z", 12, 12, 12, 0, 0, 1, 5) == 7
    assert sbgemm.get_choice("z", 12, 12, 12, 0, 0, 0, 5) == 7
    assert sbgemm.get_choice("z", 16, 8, 16, 1, 0, 0, 5) == 7
    assert sbgemm.get_choice("z", 11, 11, 11, 0, 0, 1, 5) == 0
    assert sbgemm.get_choice("z", 16, 16, 15, 0, 0, 1, 5) == 1
    assert sbgemm.get_choice("z", 8, 11, 13, 0, 0, 0, 5) == 1
    assert sbgemm.get_choice("z", 8, 8, 15, 0, 0, 1, 5) == 0
    assert sbgemm.get_choice("d", 13, 13, 13, 1, 0, 0, 5) == 7
    assert sbgemm.get_choice("d", 12, 12, 12, 0, 0, 1, 5) == 0
    assert sbgemm.get_choice("d", 12, 12, 12, 0, 0, 0, 5) == 7
    assert sbgemm.get_choice("d", 11, 11, 11, 0, 0, 0, 5) == 0
    assert sbgemm.get_choice("z", 16, 16, 16, 0, 0, 1, 5) == 7
    assert sbgemm.get_choice("h", 16, 16, 16, 0, 0, 1, 6) == 7
    assert sbgemm.get_choice("h", 12, 12, 12, 0, 0, 1, 6) == 7
    assert sbgemm.get_choice("s", 7, 3, 11, 0, 0, 1, 5) == 0
    sbgemm.set_choice("s", 10, 10, 10, 0, 0, 1, 5, 3)
    assert sbgemm.get_choice("s", 10, 10, 10, 0, 0, 1, 5) == 3
    sbgemm.set_choice("s", 10, 10, 10, 0, 0, 1, 5, -1)
    assert sbgemm.get_choice("s", 10, 10, 10, 0, 0, 1, 5) == 2
    with pytest.raises(sbgemm.SbgemmError):
        sbgemm.set_choice("s", 10, 10, 10, 0, 0, 1, 5, 99)
    sbgemm.clear_choices()


def test_vbatch_plan_rejects_bad_problems():
    import numpy as np
    p = np.zeros(2, dtype=sbgemm.vproblem_dtype())
    p["m"], p["n"], p["k"] = 3, 3, 3
    p[1]["m"] = 17
    with pytest.raises(sbgemm.SbgemmError) as e:
        sbgemm.VPlan("s", p)
    assert e.value.status == -2
    p[1]["m"] = 3
    p[1]["flags"] = 3          # op code 3 is not N, T or C
    with pytest.raises(sbgemm.SbgemmError) as e:
        sbgemm.VPlan("s", p)
    assert e.value.status == -1


def test_grouped_config_validation():
    """Host-only: the grouped launch configuration accepts the documented
    range and rejects the rest without changing the setting."""
    L = sbgemm.lib()
    assert L.sbgemm_grouped_config(0, 256, 16384, 4) == 0
    assert L.sbgemm_grouped_config(0, 0, 0, 0) == 0
    for bad in [(0, 64, 16384, 3), (0, 128, 2048, 3), (0, 128, 16384, 5), (0, 128, 16500, 3),
                (0, 128, 65536, 4), (9, 128, 16384, 3), (0, 128, 16384, 1)]:
        assert L.sbgemm_grouped_config(*bad) == -5, bad   # SBGEMM_ERR_INVALID_VALUE


def test_vbatch_window_config_validation():
    """Host-only: the plan's bucketing window accepts 0 (default) and any
    positive count, and rejects negative values."""
    L = sbgemm.lib()
    assert L.sbgemm_vbatch_config(-1) == -5   # SBGEMM_ERR_INVALID_VALUE
    assert L.sbgemm_vbatch_config(65536) == 0
    assert L.sbgemm_vbatch_config(0) == 0


def test_mlp_adam_argument_errors():
    """Host-only: the Adam step rejects a negative or non-finite L2 penalty
    and a step number below 1 before touching the device."""
    L = sbgemm.lib()
    args = dict(lr=1e-3, b1=0.9, b2=0.999, eps=1e-8)
    call = lambda t, l2, ptr: L.sbgemm_mlp_adam(4, ptr, ptr, ptr, ptr, t, args["lr"], args["b1"],
                                                 args["b2"], args["eps"], l2, None)
    assert call(1, -1.0, None) == -5
    assert call(1, float("nan"), None) == -5
    assert call(1, float("inf"), None) == -5
    assert call(0, 0.0, None) == -5
    assert call(1, 0.0, None) == -4       # valid penalty, missing buffers
    assert L.sbgemm_mlp_adam(0, None, None, None, None, 1, 1e-3, 0.9, 0.999, 1e-8, 5e-3, None) == 0
