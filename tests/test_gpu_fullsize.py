"""Parity at the sizes the throughput figures are quoted at.

Every configuration of the fixed-size sweep (S/D/C/Z, square m = 1..16,
N = 100,000 and 1,000,000, op N/N and transposed/conjugated, alpha = 1.5,
beta in {0, -0.5}), 16-bit storage with beta != 0 at N = 1,000,000 on both
the tensor-core and the CUDA-core kernels, the grouped call at N = 100,000
per size, and the pointer-array form at N = 100,000 run at full size in the
default launch configuration.  The inputs are drawn on the device from the
counter-based streams of ``inputs`` (``device_draw``); a sample of pairs,
always including the first and the last, is read back, checked against the
host generator (``draw_range``), and compared element by element with the
oracle run on exactly those pairs, within the bound of ``gpu_helpers``.
Guard elements after C must come back untouched."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

from paper_1304_7053_gb300 import inputs, sbgemm
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

GUARD = 64          # elements after C that no call may write
NP = {"s": np.float32, "d": np.float64, "c": np.complex64, "z": np.complex128,
      "h": np.uint16, "b": np.uint16}


def _np_view(t: torch.Tensor, dtype: str) -> np.ndarray:
    return t.cpu().numpy().view(NP[dtype])


class DevBatch:
    """A uniform-layout batch with minimal leading dimensions, drawn on the
    device; matrix p of X occupies elements [p*SX, (p+1)*SX)."""

    def __init__(self, dtype, ta, tb, m, n, k, N, seed):
        self.dtype, self.ta, self.tb, self.m, self.n, self.k, self.N = dtype, ta, tb, m, n, k, N
        ar, ac = inputs.stored_shape(ta, m, k)
        br, bc = inputs.stored_shape(tb, k, n)
        self.lda, self.ldb, self.ldc = max(1, ar), max(1, br), max(1, m)
        self.SA, self.SB, self.SC = ar * ac, br * bc, m * n
        self.seeds = (seed * 3 + 1, seed * 3 + 2, seed * 3 + 3)
        dev = H.dev()
        self.w = 2 if dtype in "cz" else 1
        self.A = inputs.device_draw(dtype, N * self.SA, self.seeds[0], dev)
        self.B = inputs.device_draw(dtype, N * self.SB, self.seeds[1], dev)
        self.C = inputs.device_draw(dtype, N * self.SC + GUARD, self.seeds[2], dev)
        self.guard = self.C[N * self.SC * self.w:].clone()

    def pick(self, seed, count=400):
        N = self.N
        p = (inputs.splitmix64(seed, count) % np.uint64(N)).astype(np.int64)
        return np.unique(np.concatenate([p, [0, N - 1]]))

    def rows(self, t, S, pick):
        """Matrices `pick` of a flat device operand, as a flat host array."""
        idx = torch.from_numpy(pick).to(t.device)
        return _np_view(t[: self.N * S * self.w].view(self.N, S * self.w)[idx].reshape(-1), self.dtype)

    def sample(self, pick, C_before):
        """Host UniformBatch of the picked pairs (inputs from the host
        generator, checked equal to the device draws)."""
        d = self.dtype
        sub = inputs.UniformBatch(d, self.ta, self.tb, self.m, self.n, self.k, pick.size, seed=0)
        parts = []
        for seed, S, t in zip(self.seeds, (self.SA, self.SB, self.SC), (self.A, self.B, C_before)):
            host = np.concatenate([inputs.draw_range(d, seed, int(p) * S, S) for p in pick])
            devv = self.rows(t, S, pick)
            assert np.array_equal(host.view(np.uint8), devv.view(np.uint8)), \
                "device inputs differ from the host generator"
            parts.append(host)
        sub.A, sub.B, sub.C = parts
        return sub

    def check(self, got_C, C_before, alpha, beta, pick_seed):
        pick = self.pick(pick_seed)
        sub = self.sample(pick, C_before)
        got = self.rows(got_C, self.SC, pick)
        H.assert_parity(sub, got, H.oracle_ref(sub, alpha, beta), alpha, beta)
        assert torch.equal(got_C[self.N * self.SC * self.w:], self.guard), "write past the last C"

    def run(self, alpha, beta, variant=None):
        C0 = self.C.clone()
        sbgemm.gemm_multi_uniform(self.dtype, self.ta, self.tb, self.m, self.n, self.k, alpha,
                                  self.A, self.lda, self.SA, self.B, self.ldb, self.SB, beta, self.C,
                                  self.ldc, self.SC, self.N, variant=variant)
        torch.cuda.synchronize()
        return C0


def _scalars(dtype, beta):
    if dtype in "cz":
        return 1.5 + 0.0j, complex(beta)
    return 1.5, beta


def _release():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


CASES_1E5 = [("N", "N", 0.0), ("N", "N", -0.5), ("T", "C", -0.5)]
CASES_1E6 = [("N", "N", 0.0), ("C", "T", -0.5)]


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z"])
@pytest.mark.parametrize("m", list(range(1, 17)))
def test_fixed_size_n1e5_sampled(dtype, m):
    """N = 100,000: the paper's batch size (Section 7)."""
    for i, (ta, tb, beta) in enumerate(CASES_1E5):
        b = DevBatch(dtype, ta, tb, m, m, m, 100_000, seed=1000 + 10 * m + i)
        alpha, beta = _scalars(dtype, beta)
        C0 = b.run(alpha, beta)
        b.check(b.C, C0, alpha, beta, pick_seed=7 * m + i)
        del b, C0
    _release()


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z"])
@pytest.mark.parametrize("m", list(range(1, 17)))
def test_fixed_size_n1e6_sampled(dtype, m):
    """N = 1,000,000: the largest batch of the sweep (complex128 at m = 16
    holds 12 GB of operands)."""
    for i, (ta, tb, beta) in enumerate(CASES_1E6):
        b = DevBatch(dtype, ta, tb, m, m, m, 1_000_000, seed=2000 + 10 * m + i)
        alpha, beta = _scalars(dtype, beta)
        C0 = b.run(alpha, beta)
        b.check(b.C, C0, alpha, beta, pick_seed=11 * m + i)
        del b, C0
    _release()


@pytest.mark.parametrize("dtype", ["h", "b"])
@pytest.mark.parametrize("m", [8, 12, 16])
@pytest.mark.parametrize("variant", [0, 7])
def test_16bit_beta_nonzero_n1e6_sampled(dtype, m, variant):
    """16-bit storage with beta != 0 (C read and rounded back to 16 bits) at
    N = 1,000,000, on the CUDA-core kernel (variant 0) and the tensor-core
    kernel (variant 7)."""
    b = DevBatch(dtype, "N", "N", m, m, m, 1_000_000, seed=3000 + m)
    C0 = b.run(1.5, -0.5, variant=variant)
    b.check(b.C, C0, 1.5, -0.5, pick_seed=13 * m + variant)
    del b, C0
    _release()


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z", "h"])
@pytest.mark.parametrize("beta", [0.0, -0.5])
def test_grouped_n1e5_per_size_sampled(dtype, beta):
    """The grouped call at the benchmark's size: sizes 1..16, N = 100,000
    pairs each, one persistent launch."""
    N = 100_000
    alpha, beta = _scalars(dtype, beta)
    batches = [DevBatch(dtype, "N", "N", m, m, m, N, seed=4000 + m + (beta != 0) * 50)
               for m in range(1, 17)]
    groups = (sbgemm.Group * 16)()
    for g, b in zip(groups, batches):
        g.transa, g.transb, g.m, g.n, g.k = b"N", b"N", b.m, b.m, b.m
        g.A, g.lda, g.lda2 = b.A.data_ptr(), b.m, b.SA
        g.B, g.ldb, g.ldb2 = b.B.data_ptr(), b.m, b.SB
        g.C, g.ldc, g.ldc2 = b.C.data_ptr(), b.m, b.SC
        g.batchCount = N
    C0s = [b.C.clone() for b in batches]
    ab, bb = sbgemm._scalar_buf(dtype, alpha), sbgemm._scalar_buf(dtype, beta)
    s = torch.cuda.current_stream()
    st = sbgemm.lib().sbgemm_gemm_grouped(sbgemm.TYPE_CODES[dtype], ctypes.addressof(ab),
                                          ctypes.addressof(bb), ctypes.addressof(groups), 16, 0,
                                          s.cuda_stream)
    assert st == 0, sbgemm.status_string(st)
    s.synchronize()
    for b, C0 in zip(batches, C0s):
        b.check(b.C, C0, alpha, beta, pick_seed=17 * b.m)
    del batches, C0s
    _release()


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z"])
@pytest.mark.parametrize("m", [4, 9, 16])
@pytest.mark.parametrize("ops", [("N", "N", 0.0), ("T", "C", -0.5)])
def test_pointer_arrays_n1e5_sampled(dtype, m, ops):
    """The pointer-array form at N = 100,000: pair p's matrices are those of
    a pseudo-random permutation of the 3-D batch, so consecutive pointers
    are far apart; the result of pair p lands in matrix perm[p] of C."""
    ta, tb, beta = ops
    N = 100_000
    alpha, beta = _scalars(dtype, beta)
    b = DevBatch(dtype, ta, tb, m, m, m, N, seed=5000 + m)
    perm = np.argsort(inputs.splitmix64(5100 + m, N)).astype(np.int64)
    es = inputs.ELEM_BYTES[dtype]
    tp = torch.from_numpy(perm).to(H.dev())
    Ap = b.A.data_ptr() + tp * (b.SA * es)
    Bp = b.B.data_ptr() + tp * (b.SB * es)
    Cp = b.C.data_ptr() + tp * (b.SC * es)
    C0 = b.C.clone()
    sbgemm.gemm_multi_nounif(dtype, ta, tb, m, m, m, alpha, Ap, b.lda, Bp, b.ldb, beta, Cp, b.ldc, N)
    torch.cuda.synchronize()
    # pair p used matrix perm[p] of every operand: C matrix q holds its own product
    b.check(b.C, C0, alpha, beta, pick_seed=19 * m)
    del b, C0
    _release()
