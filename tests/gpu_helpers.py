"""Shared helpers for the GPU parity tests: device round trips through the C
ABI binding, and the elementwise error bound the results are held to.

Error bound (Eq. 1 evaluated with fused multiply-adds in the storage
precision, unit roundoff u = 2^-24 for fp32 arithmetic, 2^-53 for fp64):
  scale_ij = |alpha| (|op(A)| |op(B)|)_ij + |beta| |C_ij|   (moduli for complex)
  real:    |C - C_ref| <= max(2k, k + 3) u scale
  complex: |Re/Im (C - C_ref)| <= (2k + 5) u scale
The k-term chain of FMAs contributes k roundings (2k per component for
complex, whose real and imaginary parts are dot products of length 2k).
Real epilogue: alpha * v (1 rounding), then fma(beta, C, .) (1), so at most
k + 2 in all; max(2k, k+3) equals the literal 2ku for k >= 3 and covers
k = 1, 2.  Complex epilogue, per component: alpha * v = fma(ar, vr, -ai vi)
(2 roundings: the product ai vi and the fma), beta * C likewise (2), and the
sum of the two (1): 2k + 5 in all, the bound used.  16-bit storage adds the final rounding
of the fp32 result to the 16-bit format: u16 |C_ref| + (1 + u16) * bound32
+ s16, u16 = 2^-11 (binary16) or 2^-8 (bfloat16), s16 half the subnormal
spacing (2^-25, 2^-134) for results below the normal range.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_1304_7053_gb300 import inputs, sbgemm
from tests import refmath

U = {"s": 2.0 ** -24, "c": 2.0 ** -24, "d": 2.0 ** -53, "z": 2.0 ** -53,
     "h": 2.0 ** -24, "b": 2.0 ** -24}
U16 = {"h": 2.0 ** -11, "b": 2.0 ** -8}
# half the spacing of the 16-bit subnormals: the absolute rounding error of a
# result below the normal range
SUB16 = {"h": 2.0 ** -25, "b": 2.0 ** -134}


def dev():
    return torch.device("cuda:0")


def to_dev(x: np.ndarray, pad_front: int = 0, pad_back: int = 0, fill: int = 0x5A):
    """Copy a flat numpy array to the GPU inside a byte buffer with guard
    bytes before and after; returns (buffer, address of the array)."""
    raw = np.ascontiguousarray(x).view(np.uint8)
    buf = np.full(raw.size + pad_front + pad_back, fill, dtype=np.uint8)
    buf[pad_front:pad_front + raw.size] = raw
    t = torch.from_numpy(buf).to(dev())
    return t, int(t.data_ptr()) + pad_front


def from_dev(t: torch.Tensor, like: np.ndarray, pad_front: int = 0):
    raw = t.cpu().numpy()
    return raw[pad_front:pad_front + like.nbytes].view(like.dtype).copy(), raw


def decode(x: np.ndarray, dtype: str) -> np.ndarray:
    if dtype in "hb":
        return oracle._decode16(x, dtype)
    return x.astype(np.complex128 if dtype in "cz" else np.float64)


def run_gpu(b: inputs.UniformBatch, alpha, beta, variant=None, device_scalars=False,
            guard: int = 64, A=None, B=None, C=None, stream=None):
    """Run the batch through the C ABI; returns the C array read back.
    Guard bytes around C must come back untouched (checked here)."""
    A = b.A if A is None else A
    B = b.B if B is None else B
    C = b.C if C is None else C
    tA, pA = to_dev(A)
    tB, pB = to_dev(B)
    tC, pC = to_dev(C, guard, guard)
    keep = []
    if device_scalars:
        sd = {"s": np.float32, "h": np.float32, "b": np.float32, "d": np.float64,
              "c": np.complex64, "z": np.complex128}[b.dtype]
        ta_, pa = to_dev(np.array([alpha], dtype=sd))
        tb_, pb = to_dev(np.array([beta], dtype=sd))
        keep += [ta_, tb_]
        a_arg, b_arg = pa, pb
    else:
        a_arg, b_arg = alpha, beta
    sbgemm.gemm_multi_uniform(b.dtype, b.transa, b.transb, b.m, b.n, b.k, a_arg, pA, b.lda,
                              b.lda2, pB, b.ldb, b.ldb2, b_arg, pC, b.ldc, b.ldc2, b.batch,
                              stream=stream, variant=variant, device_scalars=device_scalars)
    torch.cuda.synchronize()
    got, raw = from_dev(tC, C, guard)
    assert np.all(raw[:guard] == 0x5A) and np.all(raw[guard + C.nbytes:] == 0x5A), \
        "write outside C"
    del keep
    return got


def oracle_ref(b: inputs.UniformBatch, alpha, beta, A=None, B=None, C=None, threads=8):
    A = b.A if A is None else A
    B = b.B if B is None else B
    C = b.C if C is None else C
    return oracle.gemm_uniform(b.dtype, b.transa, b.transb, b.m, b.n, b.k, alpha, A, b.lda,
                               b.lda2, B, b.ldb, b.ldb2, beta, C, b.ldc, b.ldc2, b.batch,
                               threads=threads)


def scale_of(b: inputs.UniformBatch, alpha, beta, A=None, B=None, C=None) -> np.ndarray:
    """|alpha| |op(A)||op(B)| + |beta| |C| per entry, shape (batch, m, n)."""
    A = b.A if A is None else A
    B = b.B if B is None else B
    C = b.C if C is None else C
    ar, ac = inputs.stored_shape(b.transa, b.m, b.k)
    br, bc = inputs.stored_shape(b.transb, b.k, b.n)
    Av = np.abs(decode(np.ascontiguousarray(A), b.dtype))
    Bv = np.abs(decode(np.ascontiguousarray(B), b.dtype))
    Cv = np.abs(decode(np.ascontiguousarray(C), b.dtype))
    Aa = refmath.apply_op(refmath.views(Av, ar, ac, b.lda, b.lda2, b.batch), b.transa, False)
    Ba = refmath.apply_op(refmath.views(Bv, br, bc, b.ldb, b.ldb2, b.batch), b.transb, False)
    if complex(alpha) != 0:
        s = abs(complex(alpha)) * np.matmul(Aa, Ba)
    else:
        s = np.zeros((b.batch, b.m, b.n))
    if complex(beta) != 0:
        s = s + abs(complex(beta)) * refmath.views(Cv, b.m, b.n, b.ldc, b.ldc2, b.batch)
    return s


def bound(b: inputs.UniformBatch, alpha, beta, ref_blocks: np.ndarray, **kw) -> np.ndarray:
    k = b.k
    u = U[b.dtype]
    s = scale_of(b, alpha, beta, **kw)
    c = (2 * k + 5) if b.dtype in "cz" else max(2 * k, k + 3)
    bd = c * u * s
    if b.dtype in "hb":
        bd = U16[b.dtype] * np.abs(ref_blocks) + (1 + U16[b.dtype]) * bd + SUB16[b.dtype]
    return bd


def blocks(b, flat):
    return refmath.gather_c(flat, b.m, b.n, b.ldc, b.ldc2, b.batch)


def assert_parity(b, got, ref, alpha, beta, exact=False, **kw):
    """Elementwise comparison of the m x n blocks, plus untouched padding."""
    g = blocks(b, decode(got, b.dtype))
    r = blocks(b, ref)
    if exact:
        bad = np.argwhere(g != r)
        assert bad.size == 0, f"not bit-exact at {bad[:5].tolist()}: {g[tuple(bad[0])]} vs {r[tuple(bad[0])]}"
    elif r.size:
        bd = bound(b, alpha, beta, r, **kw)
        if b.dtype in "cz":
            err = np.maximum(np.abs((g - r).real), np.abs((g - r).imag))
        else:
            err = np.abs(g - r)
        ratio = np.where(bd > 0, err / np.where(bd > 0, bd, 1), np.where(err > 0, np.inf, 0))
        worst = np.unravel_index(np.argmax(ratio), ratio.shape)
        assert ratio.max() <= 1.0, (f"error {err[worst]} > bound {bd[worst]} at {worst} "
                                    f"(ratio {ratio.max():.3g})")
    # entries outside the m x n blocks keep C's old contents
    mask = np.zeros(got.shape[0], dtype=bool)
    idx = (np.arange(b.batch)[:, None, None] * b.ldc2 + np.arange(b.m)[None, :, None]
           + np.arange(b.n)[None, None, :] * b.ldc)
    mask[idx.ravel()] = True
    C0 = kw.get("C", b.C)
    assert np.array_equal(got[~mask].view(np.uint8), np.ascontiguousarray(C0)[~mask].view(np.uint8))
