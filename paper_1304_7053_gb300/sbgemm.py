"""Thin ctypes binding over ``libsbgemm.so`` (the C ABI in ``include/sbgemm.h``).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  Functions named ``sbgemm_*`` are the C entry points
themselves (raw integers for pointers); ``gemm_multi_uniform`` is a
convenience wrapper that takes torch tensors for the device buffers.

Loading fails loudly when the library has not been built; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsbgemm.so")

TYPE_CODES = {"s": 0, "d": 1, "c": 2, "z": 3, "h": 4, "b": 5}
SCALARS_HOST, SCALARS_DEVICE = 0, 1

STATUS = {0: "SUCCESS", -1: "ERR_INVALID_TRANS", -2: "ERR_INVALID_SIZE", -3: "ERR_INVALID_LD",
          -4: "ERR_NULL_POINTER", -5: "ERR_INVALID_VALUE", -6: "ERR_TIMEOUT",
          -7: "ERR_NOT_SUPPORTED", -8: "ERR_CAPACITY", -9: "ERR_IO"}

# Every symbol include/sbgemm.h declares, with its ctypes signature.
_c, _i, _ll, _vp = ctypes.c_char, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p
_UNIFORM = [_c, _c, _i, _i, _i, _vp, _vp, _i, _ll, _vp, _i, _ll, _vp, _vp, _i, _ll, _i]
SIGNATURES = {
    "sbgemm_Sgemm_multi_uniform": (_i, _UNIFORM),
    "sbgemm_Dgemm_multi_uniform": (_i, _UNIFORM),
    "sbgemm_Cgemm_multi_uniform": (_i, _UNIFORM),
    "sbgemm_Zgemm_multi_uniform": (_i, _UNIFORM),
    "sbgemm_Sgemm_multi_uniform_async": (_i, _UNIFORM + [_i, _vp]),
    "sbgemm_Dgemm_multi_uniform_async": (_i, _UNIFORM + [_i, _vp]),
    "sbgemm_Cgemm_multi_uniform_async": (_i, _UNIFORM + [_i, _vp]),
    "sbgemm_Zgemm_multi_uniform_async": (_i, _UNIFORM + [_i, _vp]),
    "sbgemm_Hgemm_multi_uniform_async": (_i, _UNIFORM + [_i, _vp]),
    "sbgemm_Bgemm_multi_uniform_async": (_i, _UNIFORM + [_i, _vp]),
    "sbgemm_gemm_multi_uniform_host": (_i, [_i] + _UNIFORM + [_vp, ctypes.c_size_t, _vp]),
    "sbgemm_gemm_grouped_host": (_i, [_i, _vp, _vp, _vp, _i, _vp, ctypes.c_size_t, _vp]),
    "sbgemm_gemm_grouped": (_i, [_i, _vp, _vp, _vp, _i, _i, _vp]),
    "sbgemm_grouped_config": (_i, [_i, _i, _i, _i]),
    "sbgemm_vbatch_config": (_i, [_i]),
    "sbgemm_device_error": (_i, [_vp, _vp]),
    "sbgemm_wait_selftest": (_i, [_ll, _vp]),
    "sbgemm_Sgemm_multi_nounif": (_i, [_c, _c, _i, _i, _i, _vp, _vp, _i, _vp, _i, _vp, _vp, _i, _i]),
    "sbgemm_Dgemm_multi_nounif": (_i, [_c, _c, _i, _i, _i, _vp, _vp, _i, _vp, _i, _vp, _vp, _i, _i]),
    "sbgemm_Cgemm_multi_nounif": (_i, [_c, _c, _i, _i, _i, _vp, _vp, _i, _vp, _i, _vp, _vp, _i, _i]),
    "sbgemm_Zgemm_multi_nounif": (_i, [_c, _c, _i, _i, _i, _vp, _vp, _i, _vp, _i, _vp, _vp, _i, _i]),
    "sbgemm_gemm_multi_nounif": (_i, [_i, _c, _c, _i, _i, _i, _vp, _vp, _i, _vp, _i, _vp, _vp, _i,
                                      _i, _i, _vp]),
    "sbgemm_num_variants": (_i, [_i, _i, _i, _i]),
    "sbgemm_variant_name": (ctypes.c_char_p, [_i, _i, _i, _i, _i]),
    "sbgemm_gemm_multi_uniform_variant": (_i, [_i] + _UNIFORM + [_i, _i, _vp]),
    "sbgemm_set_choice": (_i, [_i] * 9),
    "sbgemm_get_choice": (_i, [_i] * 8),
    "sbgemm_clear_choices": (None, []),
    "sbgemm_default_variant": (_i, [_i] * 6),
    "sbgemm_last_variant": (_i, []),
    "sbgemm_save_table": (_i, [ctypes.c_char_p]),
    "sbgemm_load_table": (_i, [ctypes.c_char_p]),
    "sbgemm_set_selector": (_i, [_i]),
    "sbgemm_get_selector": (_i, [ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "sbgemm_set_cost_model": (_i, [_i, _i, _i, _vp, ctypes.c_double, ctypes.c_double, _vp]),
    "sbgemm_save_cost_model": (_i, [ctypes.c_char_p]),
    "sbgemm_load_cost_model": (_i, [ctypes.c_char_p]),
    "sbgemm_tune": (_i, [_i] + _UNIFORM + [_i, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_i),
                                           _vp]),
    "sbgemm_vbatch_plan_create": (_i, [ctypes.POINTER(_vp), _i, _vp, _i]),
    "sbgemm_vbatch_plan_destroy": (_i, [_vp]),
    "sbgemm_vbatch_run": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i, _vp]),
    "sbgemm_vbatch_plan_info": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i),
                                     ctypes.POINTER(_ll)]),
    "sbgemm_vbatch_run_noalloc": (_i, [_i, _vp, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp]),
    "sbgemm_timer_create": (_i, [ctypes.POINTER(_vp), _i]),
    "sbgemm_timer_mark": (_i, [_vp, _i, _vp]),
    "sbgemm_timer_elapsed": (_i, [_vp, _i, _i, ctypes.POINTER(ctypes.c_float)]),
    "sbgemm_timer_destroy": (_i, [_vp]),
    "sbgemm_time_variant": (_i, [_i] + _UNIFORM + [_i, _i, _vp, ctypes.c_size_t, _vp,
                                                   ctypes.POINTER(ctypes.c_float)]),
    "sbgemm_mlp_param_count": (_ll, [_i, _i, _i]),
    "sbgemm_mlp_forward": (_i, [_i, _i, _i, _vp, _vp, _i, _vp, _vp, _vp]),
    "sbgemm_mlp_backward": (_i, [_i, _i, _i, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                 _vp]),
    "sbgemm_mlp_adam": (_i, [_ll, _vp, _vp, _vp, _vp, _i, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, ctypes.c_float, ctypes.c_float, _vp]),
    "sbgemm_status_string": (ctypes.c_char_p, [_i]),
    "sbgemm_version": (_i, []),
}

_lock = threading.Lock()
_lib = None


class SbgemmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: status {status} ({status_string(status)})")


def lib():
    """Load the library (once).  Raises if it is missing: no fallback."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().sbgemm_status_string(status).decode()
    except Exception:
        return STATUS.get(status, str(status))


def __getattr__(name):
    # the C entry points under their own names
    if name in SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)


# ---------------------------------------------------------------- helpers

def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _scalar_buf(dtype: str, value):
    """Host scalar for alpha/beta in the storage arithmetic type."""
    if dtype == "s" or dtype in "hb":
        return (ctypes.c_float * 1)(float(complex(value).real))
    if dtype == "d":
        return (ctypes.c_double * 1)(float(complex(value).real))
    v = complex(value)
    if dtype == "c":
        return (ctypes.c_float * 2)(v.real, v.imag)
    return (ctypes.c_double * 2)(v.real, v.imag)


def gemm_multi_uniform(dtype: str, transa: str, transb: str, m: int, n: int, k: int,
                       alpha, A, lda: int, lda2: int, B, ldb: int, ldb2: int,
                       beta, C, ldc: int, ldc2: int, batch: int, stream=None,
                       variant: int | None = None, device_scalars: bool = False,
                       check: bool = True) -> int:
    """Eq. (1) on the Section 4 layout.  A, B, C are torch CUDA tensors (or
    raw device addresses as int).  alpha/beta are Python numbers (host
    scalars) or, with ``device_scalars``, device tensors holding one scalar.
    Returns the status; raises ``SbgemmError`` on a nonzero status when
    ``check``."""
    L = lib()
    t = TYPE_CODES[dtype]
    if device_scalars:
        pa, pb, mode = _ptr(alpha), _ptr(beta), SCALARS_DEVICE
        keep = None
    else:
        ab, bb = _scalar_buf(dtype, alpha), _scalar_buf(dtype, beta)
        keep = (ab, bb)
        pa, pb, mode = ctypes.addressof(ab), ctypes.addressof(bb), SCALARS_HOST
    s = _stream_ptr(stream)
    args = (transa.encode(), transb.encode(), m, n, k, pa, _ptr(A), lda, lda2, _ptr(B), ldb, ldb2,
            pb, _ptr(C), ldc, ldc2, batch)
    if variant is None:
        fn = {"s": L.sbgemm_Sgemm_multi_uniform_async, "d": L.sbgemm_Dgemm_multi_uniform_async,
              "c": L.sbgemm_Cgemm_multi_uniform_async, "z": L.sbgemm_Zgemm_multi_uniform_async,
              "h": L.sbgemm_Hgemm_multi_uniform_async, "b": L.sbgemm_Bgemm_multi_uniform_async}[dtype]
        st = fn(*args, mode, s)
    else:
        st = L.sbgemm_gemm_multi_uniform_variant(t, *args, mode, variant, s)
    del keep
    if check and st != 0:
        raise SbgemmError(st, "gemm_multi_uniform")
    return st


def gemm_multi_nounif(dtype: str, transa: str, transb: str, m: int, n: int, k: int,
                      alpha, Aarray, lda: int, Barray, ldb: int, beta, Carray, ldc: int,
                      batch: int, stream=None, device_scalars: bool = False,
                      check: bool = True) -> int:
    """Eq. (1) in the pointer-array form: Aarray, Barray, Carray are device
    arrays (torch int64 CUDA tensors or raw addresses) of per-pair matrix
    pointers.  Scalars as for ``gemm_multi_uniform``."""
    if device_scalars:
        pa, pb, mode, keep = _ptr(alpha), _ptr(beta), SCALARS_DEVICE, None
    else:
        ab, bb = _scalar_buf(dtype, alpha), _scalar_buf(dtype, beta)
        pa, pb, mode, keep = ctypes.addressof(ab), ctypes.addressof(bb), SCALARS_HOST, (ab, bb)
    st = lib().sbgemm_gemm_multi_nounif(TYPE_CODES[dtype], transa.encode(), transb.encode(), m, n,
                                        k, pa, _ptr(Aarray), lda, _ptr(Barray), ldb, pb,
                                        _ptr(Carray), ldc, batch, mode, _stream_ptr(stream))
    del keep
    if check and st != 0:
        raise SbgemmError(st, "gemm_multi_nounif")
    return st


def prepare_uniform(dtype: str, transa: str, transb: str, m: int, n: int, k: int,
                    alpha, A, lda: int, lda2: int, B, ldb: int, ldb2: int,
                    beta, C, ldc: int, ldc2: int, batch: int, stream=None,
                    variant: int | None = None):
    """Bind every argument once and return a no-argument callable that issues
    the call (host scalars); for timing loops where per-call marshalling
    would otherwise cost more host time than a small kernel takes."""
    L = lib()
    ab, bb = _scalar_buf(dtype, alpha), _scalar_buf(dtype, beta)
    args = (transa.encode(), transb.encode(), m, n, k, ctypes.addressof(ab), _ptr(A), lda, lda2,
            _ptr(B), ldb, ldb2, ctypes.addressof(bb), _ptr(C), ldc, ldc2, batch)
    s = _stream_ptr(stream)
    if variant is None:
        fn = {"s": L.sbgemm_Sgemm_multi_uniform_async, "d": L.sbgemm_Dgemm_multi_uniform_async,
              "c": L.sbgemm_Cgemm_multi_uniform_async, "z": L.sbgemm_Zgemm_multi_uniform_async,
              "h": L.sbgemm_Hgemm_multi_uniform_async, "b": L.sbgemm_Bgemm_multi_uniform_async}[dtype]
        full = args + (SCALARS_HOST, s)
    else:
        fn = L.sbgemm_gemm_multi_uniform_variant
        full = (TYPE_CODES[dtype],) + args + (SCALARS_HOST, variant, s)

    def call(_fn=fn, _a=full, _keep=(ab, bb)):
        st = _fn(*_a)
        if st != 0:
            raise SbgemmError(st, "gemm_multi_uniform")
    return call


def num_variants(dtype: str, m: int, n: int, k: int) -> int:
    return lib().sbgemm_num_variants(TYPE_CODES[dtype], m, n, k)


def variant_name(dtype: str, m: int, n: int, k: int, v: int) -> str:
    return lib().sbgemm_variant_name(TYPE_CODES[dtype], m, n, k, v).decode()


def set_choice(dtype, m, n, k, ta, tb, beta_zero, size_class, variant) -> None:
    st = lib().sbgemm_set_choice(TYPE_CODES[dtype], m, n, k, int(ta), int(tb), int(beta_zero),
                                 size_class, variant)
    if st != 0:
        raise SbgemmError(st, "set_choice")


def get_choice(dtype, m, n, k, ta, tb, beta_zero, size_class) -> int:
    return lib().sbgemm_get_choice(TYPE_CODES[dtype], m, n, k, int(ta), int(tb), int(beta_zero),
                                   size_class)


def clear_choices() -> None:
    lib().sbgemm_clear_choices()


def default_variant(dtype, m, n, k, beta_zero, size_class) -> int:
    return lib().sbgemm_default_variant(TYPE_CODES[dtype], m, n, k, int(beta_zero), size_class)


def last_variant() -> int:
    return lib().sbgemm_last_variant()


SELECTOR_DEFAULT, SELECTOR_TABLE, SELECTOR_MODEL = 0, 1, 2


def set_selector(mode: int) -> None:
    st = lib().sbgemm_set_selector(mode)
    if st != 0:
        raise SbgemmError(st, "set_selector")


def get_selector():
    """(mode, first error of the environment settings)."""
    mode, env = ctypes.c_int(), ctypes.c_int()
    st = lib().sbgemm_get_selector(ctypes.byref(mode), ctypes.byref(env))
    if st != 0:
        raise SbgemmError(st, "get_selector")
    return mode.value, env.value


def save_table(path: str) -> None:
    st = lib().sbgemm_save_table(os.fsencode(path))
    if st != 0:
        raise SbgemmError(st, "save_table")


def load_table(path: str) -> None:
    st = lib().sbgemm_load_table(os.fsencode(path))
    if st != 0:
        raise SbgemmError(st, "load_table")


def margin_array(margins):
    """Per-storage-type trust margins in type-code order: a number (every
    type), a mapping from dtype letter to margin (missing types: 0), or a
    sequence of six."""
    if isinstance(margins, dict):
        return [float(margins.get(d, 0.0)) for d in "sdczhb"]
    if isinstance(margins, (int, float)):
        return [float(margins)] * 6
    out = [float(x) for x in margins]
    if len(out) != 6:
        raise ValueError("six margins expected, one per storage type")
    return out


def set_cost_model(F: int, H: int, V: int, params, log_time_mean: float, log_time_std: float,
                   margins) -> None:
    """Install a cost model from a host float32 numpy array of parameters;
    ``margins`` as ``margin_array`` takes them."""
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    mg = np.ascontiguousarray(margin_array(margins), dtype=np.float64)
    st = lib().sbgemm_set_cost_model(F, H, V, p.ctypes.data, float(log_time_mean),
                                     float(log_time_std), mg.ctypes.data)
    if st != 0:
        raise SbgemmError(st, "set_cost_model")


def save_cost_model(path: str) -> None:
    st = lib().sbgemm_save_cost_model(os.fsencode(path))
    if st != 0:
        raise SbgemmError(st, "save_cost_model")


def load_cost_model(path: str) -> None:
    st = lib().sbgemm_load_cost_model(os.fsencode(path))
    if st != 0:
        raise SbgemmError(st, "load_cost_model")


# ---------------------------------------------------------------- variable size

def vproblem_dtype():
    """numpy layout of ``sbgemm_vproblem`` (32 bytes)."""
    import numpy as np
    return np.dtype([("m", "<i4"), ("n", "<i4"), ("k", "<i4"), ("flags", "<i4"),
                     ("a", "<i8"), ("b", "<i8"), ("c", "<i8")])


def vproblems_from_desc(desc):
    """Convert an (count, 8) int64 table (m, n, k, flags, offA, offB, offC, 0)
    into an array of ``sbgemm_vproblem`` records."""
    import numpy as np
    desc = np.asarray(desc, dtype=np.int64)
    out = np.zeros(desc.shape[0], dtype=vproblem_dtype())
    for i, f in enumerate(("m", "n", "k", "flags")):
        out[f] = desc[:, i].astype(np.int32)
    out["a"], out["b"], out["c"] = desc[:, 4], desc[:, 5], desc[:, 6]
    return out


class HostGroup(ctypes.Structure):
    """``sbgemm_host_group``: one uniform batch on host arrays."""
    _fields_ = [("transa", ctypes.c_char), ("transb", ctypes.c_char),
                ("m", ctypes.c_int), ("n", ctypes.c_int), ("k", ctypes.c_int),
                ("hA", ctypes.c_void_p), ("lda", ctypes.c_int), ("lda2", ctypes.c_longlong),
                ("hB", ctypes.c_void_p), ("ldb", ctypes.c_int), ("ldb2", ctypes.c_longlong),
                ("hC", ctypes.c_void_p), ("ldc", ctypes.c_int), ("ldc2", ctypes.c_longlong),
                ("batchCount", ctypes.c_int)]


class Group(ctypes.Structure):
    """``sbgemm_group``: one uniform batch on device arrays."""
    _fields_ = [("transa", ctypes.c_char), ("transb", ctypes.c_char),
                ("m", ctypes.c_int), ("n", ctypes.c_int), ("k", ctypes.c_int),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int), ("lda2", ctypes.c_longlong),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int), ("ldb2", ctypes.c_longlong),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int), ("ldc2", ctypes.c_longlong),
                ("batchCount", ctypes.c_int)]


def grouped_config(dtype: str, threads: int = 0, stage_bytes: int = 0, stages: int = 0) -> None:
    """Launch configuration of the grouped persistent launch for one storage
    type (all zero: the default)."""
    st = lib().sbgemm_grouped_config(TYPE_CODES[dtype], threads, stage_bytes, stages)
    if st != 0:
        raise SbgemmError(st, "grouped_config")


class VPlan:
    """A variable-size batch plan (``sbgemm_vbatch_plan_create``)."""

    def __init__(self, dtype: str, problems):
        import numpy as np
        self.dtype = dtype
        problems = np.ascontiguousarray(problems, dtype=vproblem_dtype())
        self._h = ctypes.c_void_p()
        st = lib().sbgemm_vbatch_plan_create(ctypes.byref(self._h), TYPE_CODES[dtype],
                                             problems.ctypes.data if problems.size else None,
                                             int(problems.size))
        if st != 0:
            self._h = None
            raise SbgemmError(st, "vbatch_plan_create")

    def info(self):
        nt, nb, by = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        st = lib().sbgemm_vbatch_plan_info(self._h, ctypes.byref(nt), ctypes.byref(nb),
                                           ctypes.byref(by))
        if st != 0:
            raise SbgemmError(st, "vbatch_plan_info")
        return {"tiles": nt.value, "buckets": nb.value, "device_bytes": by.value}

    def run(self, alpha, A, B, beta, C, stream=None, device_scalars=False, check=True):
        if device_scalars:
            pa, pb, mode, keep = _ptr(alpha), _ptr(beta), SCALARS_DEVICE, None
        else:
            ab, bb = _scalar_buf(self.dtype, alpha), _scalar_buf(self.dtype, beta)
            pa, pb, mode, keep = ctypes.addressof(ab), ctypes.addressof(bb), SCALARS_HOST, (ab, bb)
        st = lib().sbgemm_vbatch_run(self._h, pa, _ptr(A), _ptr(B), pb, _ptr(C), mode,
                                     _stream_ptr(stream))
        del keep
        if check and st != 0:
            raise SbgemmError(st, "vbatch_run")
        return st

    def close(self):
        if self._h:
            lib().sbgemm_vbatch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Timer:
    """CUDA-event marks (``sbgemm_timer_*``); marks issued on a capturing
    stream become event nodes of the graph and time every replay."""

    def __init__(self, n_marks: int):
        self._h = ctypes.c_void_p()
        st = lib().sbgemm_timer_create(ctypes.byref(self._h), int(n_marks))
        if st != 0:
            self._h = None
            raise SbgemmError(st, "timer_create")

    def mark(self, i: int, stream=None) -> None:
        st = lib().sbgemm_timer_mark(self._h, int(i), _stream_ptr(stream))
        if st != 0:
            raise SbgemmError(st, "timer_mark")

    def elapsed(self, i: int, j: int) -> float:
        ms = ctypes.c_float()
        st = lib().sbgemm_timer_elapsed(self._h, int(i), int(j), ctypes.byref(ms))
        if st != 0:
            raise SbgemmError(st, "timer_elapsed")
        return float(ms.value)

    def close(self):
        if self._h:
            lib().sbgemm_timer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
