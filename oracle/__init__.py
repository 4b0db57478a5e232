"""CPU oracle for batched small-matrix GEMM (arXiv 1304.7053, Section 2, Eq. 1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never loads it, and it shares no code with the
CUDA path.

``gemm_uniform`` wraps the C oracle in ``sbgemm_oracle.c`` (double-double
accumulation of the plain triple loop, inputs converted exactly to double).
``gemm_vbatch`` applies the same definition problem by problem.
``mlp`` holds the fp64 reference of the cost-model network.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
# A test may point the loader at a deliberately mutated build of the oracle
# to show that the pins catch planted mistakes.
_LIB_OVERRIDE = os.environ.get("SBGEMM_ORACLE_LIB")
_SRC = os.path.join(_HERE, "sbgemm_oracle.c")

# storage type codes shared with sbgemm_oracle.c
TYPES = {"s": 0, "d": 1, "c": 2, "z": 3, "h": 4, "b": 5}
ERRORS = {0: "ok", -1: "bad trans", -2: "bad dim", -3: "bad ld", -4: "bad type"}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` with gcc.

    Portable flags only (the same source builds on x86-64 and aarch64):
    -O3, no -march=native, no fast-math, and no floating-point contraction so
    the double-double steps round each operation separately (-O3 without
    fast-math keeps every IEEE operation as written).
    """
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wextra",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if _LIB_OVERRIDE:
                L = ctypes.CDLL(_LIB_OVERRIDE)
            else:
                build()
                L = ctypes.CDLL(_LIB_PATH)
            vp, ll, i, c = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_char
            L.oracle_gemm_uniform.argtypes = [i, c, c, i, i, i, vp, vp, ll, ll, vp, ll, ll,
                                              vp, vp, ll, ll, ll, vp, vp, i]
            L.oracle_gemm_uniform.restype = i
            L.oracle_gemm_vbatch.argtypes = [i, vp, ll, vp, vp, vp, vp, vp, vp, vp, i]
            L.oracle_gemm_vbatch.restype = i
            L.oracle_check_args.argtypes = [c, c, i, i, i, ll, ll, ll, ll, ll, ll, ll]
            L.oracle_check_args.restype = i
            L.oracle_max_threads.argtypes = []
            L.oracle_max_threads.restype = i
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _scalar2(x) -> np.ndarray:
    x = complex(x)
    return np.array([x.real, x.imag], dtype=np.float64)


def _flat(x):
    x = np.ascontiguousarray(x)
    return x


def check_args(transa, transb, m, n, k, lda, lda2, ldb, ldb2, ldc, ldc2, batch) -> int:
    return lib().oracle_check_args(transa.encode(), transb.encode(), m, n, k,
                                   lda, lda2, ldb, ldb2, ldc, ldc2, batch)


def gemm_uniform(dtype: str, transa: str, transb: str, m: int, n: int, k: int,
                 alpha, A: np.ndarray, lda: int, lda2: int,
                 B: np.ndarray, ldb: int, ldb2: int,
                 beta, C: np.ndarray, ldc: int, ldc2: int, batch: int,
                 threads: int = 1, return_lo: bool = False):
    """Eq. (1) over the batch on the Section 4 layout; returns the exact-ish
    result in C's layout as float64 (complex128 for c/z), unrounded.

    ``A``, ``B``, ``C`` are flat numpy arrays in storage type (float32,
    float64, complex64, complex128, or uint16 bit patterns for h/b).  Entries
    of the output outside the m x n blocks keep C's values.  With
    ``return_lo`` the low parts of the double-double result are returned too.
    """
    t = TYPES[dtype]
    A, B, C = _flat(A), _flat(B), _flat(C)
    cplx = dtype in "cz"
    nC = C.size
    if cplx:
        hi = np.ascontiguousarray(C.astype(np.complex128)).view(np.float64).copy()
    elif dtype in "hb":
        hi = np.zeros(nC, dtype=np.float64)
        hi[:] = _decode16(C, dtype)
    else:
        hi = C.astype(np.float64)
    lo = np.zeros_like(hi)
    st = lib().oracle_gemm_uniform(t, transa.encode(), transb.encode(), m, n, k,
                                   _ptr(_scalar2(alpha)), _ptr(A), lda, lda2,
                                   _ptr(B), ldb, ldb2,
                                   _ptr(_scalar2(beta)), _ptr(C), ldc, ldc2, batch,
                                   _ptr(hi), _ptr(lo), int(threads))
    if st != 0:
        raise ValueError(f"oracle_gemm_uniform: {ERRORS.get(st, st)}")
    if cplx:
        hi, lo = hi.view(np.complex128), lo.view(np.complex128)
    return (hi, lo) if return_lo else hi


def gemm_vbatch(dtype: str, desc: np.ndarray, alpha, A, B, beta, C, threads: int = 1,
                return_lo: bool = False):
    """Variable-size batch: ``desc`` is an int64 array of shape (count, 8)
    = (m, n, k, flags, offA, offB, offC, 0); see ``oracle_gemm_vbatch``."""
    t = TYPES[dtype]
    desc = np.ascontiguousarray(desc, dtype=np.int64)
    A, B, C = _flat(A), _flat(B), _flat(C)
    cplx = dtype in "cz"
    if cplx:
        hi = np.ascontiguousarray(C.astype(np.complex128)).view(np.float64).copy()
    elif dtype in "hb":
        hi = _decode16(C, dtype).astype(np.float64)
    else:
        hi = C.astype(np.float64)
    lo = np.zeros_like(hi)
    st = lib().oracle_gemm_vbatch(t, _ptr(desc), desc.shape[0], _ptr(_scalar2(alpha)),
                                  _ptr(A), _ptr(B), _ptr(_scalar2(beta)), _ptr(C),
                                  _ptr(hi), _ptr(lo), int(threads))
    if st != 0:
        raise ValueError(f"oracle_gemm_vbatch: {ERRORS.get(st, st)}")
    if cplx:
        hi, lo = hi.view(np.complex128), lo.view(np.complex128)
    return (hi, lo) if return_lo else hi


def _decode16(bits: np.ndarray, dtype: str) -> np.ndarray:
    """Exact decode of binary16 / bfloat16 bit patterns to float64."""
    bits = np.asarray(bits, dtype=np.uint16)
    if dtype == "h":
        return bits.view(np.float16).astype(np.float64)
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def max_threads() -> int:
    return int(lib().oracle_max_threads())
