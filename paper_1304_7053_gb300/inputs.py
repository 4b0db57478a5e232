"""Seeded synthetic inputs for batched small-matrix GEMM.

This module only draws numbers and lays them out; it holds none of the
GEMM arithmetic.  Both the CUDA-path tests and the CPU oracle take their
inputs from here, so the two sides see identical buffers.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), a counter-based generator: the
i-th draw of stream ``seed`` is a pure function of (seed, i), so every
platform and numpy version reproduces the same bytes.

Workload recipes follow the paper's experiments (Section 7: N = 100,000
square pairs of sizes 1-16, minimal leading dimensions, alpha = 1, beta = 0)
and the extra shapes this library is exercised on (rectangular FEM-like
shapes, variable-size batches with size weights proportional to 1/p, 16-bit
storage).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

NP_DTYPES = {"s": np.float32, "d": np.float64, "c": np.complex64, "z": np.complex128,
             "h": np.uint16, "b": np.uint16}
ELEM_BYTES = {"s": 4, "d": 8, "c": 8, "z": 16, "h": 2, "b": 2}


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Draws start .. start+count-1 of SplitMix64 stream ``seed`` as uint64."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, lo: float = -1.0, hi: float = 1.0, start: int = 0) -> np.ndarray:
    """Draws start .. start+count-1 as float64, uniform on [lo, hi), from
    53-bit mantissas."""
    u = (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def small_ints(seed: int, count: int, lo: int = -4, hi: int = 4) -> np.ndarray:
    """``count`` integers uniform on [lo, hi] as float64 (exact in any type)."""
    span = np.uint64(hi - lo + 1)
    return (splitmix64(seed, count) % span).astype(np.int64).astype(np.float64) + lo


def to_storage(x: np.ndarray, dtype: str) -> np.ndarray:
    """Round float64 draws to a storage type.

    Complex types take two consecutive draws per element (re, im), so ``x``
    must hold twice as many values.  The 16-bit types return raw bit patterns
    (uint16): binary16 via numpy's round-to-nearest-even conversion, bfloat16
    by round-to-nearest-even on the upper half of the binary32 pattern.
    """
    if dtype in ("s", "d"):
        return x.astype(NP_DTYPES[dtype])
    if dtype in ("c", "z"):
        pair = x.reshape(-1, 2)
        real = np.float32 if dtype == "c" else np.float64
        out = np.empty(pair.shape[0], dtype=NP_DTYPES[dtype])
        out.real = pair[:, 0].astype(real)
        out.imag = pair[:, 1].astype(real)
        return out
    if dtype == "h":
        return x.astype(np.float16).view(np.uint16)
    if dtype == "b":
        f = x.astype(np.float32).view(np.uint32).astype(np.uint64)
        lsb = (f >> np.uint64(16)) & np.uint64(1)
        r = (f + np.uint64(0x7FFF) + lsb) >> np.uint64(16)
        return r.astype(np.uint16)
    raise ValueError(dtype)


def draw(dtype: str, count: int, seed: int, int_valued: bool = False) -> np.ndarray:
    """``count`` elements of storage type ``dtype`` (complex: independent parts)."""
    n = count * (2 if dtype in ("c", "z") else 1)
    x = small_ints(seed, n) if int_valued else uniform(seed, n)
    return to_storage(x, dtype)


# ---------------------------------------------------------------- large batches
#
# Batches of 1e5-1e6 pairs are drawn on the device (torch elementwise ops)
# from the same counter-based streams, so a full-size case costs no host
# generation or transfer; the host functions below give any element range of
# the same stream, and the tests check that the two agree on the pairs they
# sample.  Draws: uniform[-1, 1) exactly as ``uniform`` (float64, rounded to
# the storage type) for s, d, c, z and bfloat16; for binary16 a grid of
# 2^-10 steps on [-1, 1), exact in the format, so no conversion rounding is
# involved on either side.

GRID16_BITS = 11          # binary16 grid: k * 2^-10, k uniform in [-1024, 1024)


def draw_range(dtype: str, seed: int, start: int, count: int) -> np.ndarray:
    """Elements start .. start+count-1 of the large-batch stream ``seed`` of
    storage type ``dtype`` (host side of ``device_draw``)."""
    w = 2 if dtype in ("c", "z") else 1
    if dtype == "h":
        z = splitmix64(seed, count, start)
        k = (z >> np.uint64(64 - GRID16_BITS)).astype(np.int64) - (1 << (GRID16_BITS - 1))
        return (k.astype(np.float64) * 2.0 ** -(GRID16_BITS - 1)).astype(np.float16).view(np.uint16)
    return to_storage(uniform(seed, count * w, start=start * w), dtype)


def device_draw(dtype: str, count: int, seed: int, device, chunk: int = 1 << 26):
    """``count`` elements of the large-batch stream ``seed`` as a flat torch
    tensor on ``device`` (complex types as float pairs, 16-bit types as
    int16 bit patterns); element e equals ``draw_range(dtype, seed, e, 1)``."""
    import torch

    w = 2 if dtype in ("c", "z") else 1
    n = count * w
    real = {"s": torch.float32, "c": torch.float32, "d": torch.float64, "z": torch.float64,
            "b": torch.bfloat16, "h": torch.float16}[dtype]
    out = torch.empty(n, dtype=real, device=device)

    def as_i64(v):
        return v - (1 << 64) if v >= (1 << 63) else v

    gold, m1, m2 = as_i64(int(_GOLDEN)), as_i64(int(_M1)), as_i64(int(_M2))
    s64 = as_i64(seed & 0xFFFFFFFFFFFFFFFF)

    def lsr(z, r):           # logical shift right of int64 bit patterns
        return (z >> r) & ((1 << (64 - r)) - 1)

    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        # int64 arithmetic wraps modulo 2^64: the uint64 recurrence bit for bit
        z = torch.arange(c0 + 1, c1 + 1, dtype=torch.int64, device=device) * gold + s64
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        z = z ^ lsr(z, 31)
        if dtype == "h":
            k = lsr(z, 64 - GRID16_BITS) - (1 << (GRID16_BITS - 1))
            out[c0:c1] = (k.to(torch.float64) * 2.0 ** -(GRID16_BITS - 1)).to(torch.float16)
        else:
            u = lsr(z, 11).to(torch.float64) * (2.0 ** -53)
            x = -1.0 + 2.0 * u
            if dtype == "b":
                x = x.to(torch.float32)
            out[c0:c1] = x.to(real)
    if dtype in ("h", "b"):
        return out.view(torch.int16)
    return out


def stored_shape(op: str, rows: int, cols: int):
    """(rows, cols) of the stored matrix whose op() is rows x cols."""
    return (rows, cols) if op in "nN" else (cols, rows)


class UniformBatch:
    """A, B, C of one uniform-layout batch (Section 4) as flat host arrays.

    ``pad_ld`` adds that many elements to each leading dimension and
    ``pad_ld2`` to each matrix stride, so non-minimal layouts can be tested.
    """

    def __init__(self, dtype, transa, transb, m, n, k, batch, seed=0, int_valued=False,
                 pad_ld=0, pad_ld2=0, c_fill=None):
        self.dtype, self.transa, self.transb = dtype, transa, transb
        self.m, self.n, self.k, self.batch = m, n, k, batch
        ar, ac = stored_shape(transa, m, k)
        br, bc = stored_shape(transb, k, n)
        self.lda = max(1, ar) + pad_ld
        self.ldb = max(1, br) + pad_ld
        self.ldc = max(1, m) + pad_ld
        self.lda2 = self.lda * ac + pad_ld2
        self.ldb2 = self.ldb * bc + pad_ld2
        self.ldc2 = self.ldc * n + pad_ld2
        na = self.lda2 * batch
        nb = self.ldb2 * batch
        nc = self.ldc2 * batch
        self.A = draw(dtype, na, seed * 3 + 1, int_valued)
        self.B = draw(dtype, nb, seed * 3 + 2, int_valued)
        if c_fill is None:
            self.C = draw(dtype, nc, seed * 3 + 3, int_valued)
        else:
            self.C = np.full(nc, c_fill, dtype=NP_DTYPES[dtype]) if dtype not in "hb" \
                else np.full(nc, c_fill, dtype=np.uint16)

    def args(self):
        return (self.lda, self.lda2, self.ldb, self.ldb2, self.ldc, self.ldc2)

    @property
    def algorithmic_bytes(self):
        """s * (mk + kn + mn * (1 + [beta != 0])) per pair, beta == 0 form."""
        s = ELEM_BYTES[self.dtype]
        return s * self.batch * (self.m * self.k + self.k * self.n + self.m * self.n)


def vbatch_sizes(count: int, seed: int = 0, pmax: int = 15) -> np.ndarray:
    """Sizes p + 1 with p drawn from {1..pmax} with weights proportional to
    1/p, by inverse-CDF sampling of uniform draws."""
    w = 1.0 / np.arange(1, pmax + 1)
    cdf = np.cumsum(w) / w.sum()
    u = uniform(seed, count, 0.0, 1.0)
    p = np.searchsorted(cdf, u, side="right") + 1
    return np.minimum(p, pmax) + 1


VDESC_FIELDS = ("m", "n", "k", "flags", "offA", "offB", "offC", "reserved")


def vbatch_problems(count: int, seed: int = 0, beta_mixed: bool = True,
                    sizes: np.ndarray | None = None, flags_op: int = 0):
    """Descriptor table (count x 8 int64) for square problems stored back to
    back in three arenas: m = n = k = size, flags = op bits | beta-zero bit.
    Returns (desc, lenA, lenB, lenC) with arena lengths in elements."""
    if sizes is None:
        sizes = vbatch_sizes(count, seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    sq = sizes * sizes
    off = np.concatenate([[0], np.cumsum(sq)[:-1]]).astype(np.int64)
    desc = np.zeros((count, 8), dtype=np.int64)
    desc[:, 0] = sizes
    desc[:, 1] = sizes
    desc[:, 2] = sizes
    flags = np.full(count, flags_op, dtype=np.int64)
    if beta_mixed:
        bz = (splitmix64(seed + 7919, count) >> np.uint64(63)).astype(np.int64)
        flags |= bz << 4
    desc[:, 3] = flags
    desc[:, 4] = off
    desc[:, 5] = off
    desc[:, 6] = off
    total = int(sq.sum())
    return desc, total, total, total
