"""Independent references used to pin the oracle (tests only).

Nothing here re-types the oracle's loop: each matrix of the batch is taken
as a strided numpy view of the flat buffer (numpy's own striding implements
the Section 4 index map X[i + ld*j + ld2*p]), op() is numpy's transpose /
conjugate, and the product is numpy's matmul.  Exact rational arithmetic
(``fractions``) gives ground truth for the double-double accuracy pins.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def views(flat: np.ndarray, rows: int, cols: int, ld: int, ld2: int, batch: int) -> np.ndarray:
    """(batch, rows, cols) strided view: element (p, i, j) = flat[i + ld*j + ld2*p]."""
    s = flat.itemsize
    return np.lib.stride_tricks.as_strided(flat, shape=(batch, rows, cols),
                                           strides=(ld2 * s, s, ld * s), writeable=False)


def apply_op(X: np.ndarray, op: str, cplx: bool) -> np.ndarray:
    if op in "nN":
        return X
    Xt = np.swapaxes(X, 1, 2)
    if op in "cC" and cplx:
        return np.conj(Xt)
    return Xt


def numpy_gemm(dtype, transa, transb, m, n, k, alpha, A, lda, lda2, B, ldb, ldb2,
               beta, C, ldc, ldc2, batch):
    """Eq. (1) by numpy matmul on strided views, in complex128 / float64."""
    cplx = dtype in "cz"
    wide = np.complex128 if cplx else np.float64
    ar, ac = (m, k) if transa in "nN" else (k, m)
    br, bc = (k, n) if transb in "nN" else (n, k)
    Av = views(A, ar, ac, lda, lda2, batch).astype(wide)
    Bv = views(B, br, bc, ldb, ldb2, batch).astype(wide)
    Cv = views(C, m, n, ldc, ldc2, batch).astype(wide)
    prod = np.matmul(apply_op(Av, transa, cplx), apply_op(Bv, transb, cplx))
    out = alpha * prod
    if beta != 0:
        out = out + beta * Cv
    return out


def gather_c(flat_out: np.ndarray, m, n, ldc, ldc2, batch) -> np.ndarray:
    return views(np.ascontiguousarray(flat_out), m, n, ldc, ldc2, batch)


def exact_dot(a_list, b_list) -> Fraction:
    s = Fraction(0)
    for a, b in zip(a_list, b_list):
        s += Fraction(float(a)) * Fraction(float(b))
    return s
