"""GPU parity of the fixed-size uniform-layout path against the CPU oracle.

Every case goes through the C ABI (ctypes binding) and is compared element
by element with ``oracle.gemm_uniform`` on the same seeded inputs:
bit-exact on small-integer inputs (every product and partial sum is exact),
within the bound documented in ``tests/gpu_helpers.py`` on uniform[-1, 1]
inputs.  Batch sizes span several tiles plus a ragged tail."""
from __future__ import annotations

import itertools

import numpy as np
import pytest
import torch

from paper_1304_7053_gb300 import inputs, sbgemm
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

SIZES = list(range(1, 17))
OPS4 = [("N", "N"), ("T", "N"), ("N", "T"), ("C", "C")]
OPS9 = list(itertools.product("NTC", "NTC"))


def scalars(dtype):
    if dtype in "cz":
        return 1.5 + 0.0j, -0.5 + 0.0j
    return 1.5, -0.5


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z"])
@pytest.mark.parametrize("m", SIZES)
def test_integer_inputs_bit_exact(dtype, m):
    """Small integers in [-4, 4], alpha = 1.5, beta in {0, -0.5}: exact."""
    for (ta, tb), beta0 in itertools.product(OPS4, (True, False)):
        alpha, beta = scalars(dtype)
        if beta0:
            beta = 0.0
        b = inputs.UniformBatch(dtype, ta, tb, m, m, m, 1237, seed=m, int_valued=True)
        got = H.run_gpu(b, alpha, beta)
        H.assert_parity(b, got, H.oracle_ref(b, alpha, beta), alpha, beta, exact=True)


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z"])
@pytest.mark.parametrize("m", SIZES)
def test_uniform_inputs_within_bound(dtype, m):
    for (ta, tb), beta0 in itertools.product(OPS4, (True, False)):
        alpha, beta = scalars(dtype)
        if beta0:
            beta = 0.0
        b = inputs.UniformBatch(dtype, ta, tb, m, m, m, 1031, seed=100 + m)
        got = H.run_gpu(b, alpha, beta)
        H.assert_parity(b, got, H.oracle_ref(b, alpha, beta), alpha, beta)


@pytest.mark.parametrize("dtype", ["s", "c", "d"])
@pytest.mark.parametrize("m", [11, 13, 14, 15])
def test_bulk_copy_ragged_tails(dtype, m):
    """Shapes staged by one bulk copy per operand and tile (large unpadded
    matrices): batch sizes that end in a tile whose bytes are not a multiple
    of 16 (the ragged end is copied with plain loads and stores), tiny
    batches, C read (beta != 0) and not; bit-exact on small integers."""
    alpha = 1.5
    for N in (1, 2, 3, 5, 17, 257, 1001):
        for beta in (0.0, -0.5):
            b = inputs.UniformBatch(dtype, "N", "N", m, m, m, N, seed=7 * N + m, int_valued=True)
            got = H.run_gpu(b, alpha, beta)
            H.assert_parity(b, got, H.oracle_ref(b, alpha, beta), alpha, beta, exact=True)


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z"])
@pytest.mark.parametrize("m", [5, 16])
def test_all_nine_op_pairs_complex_scalars(dtype, m):
    """All 9 op combinations (Section 2), genuinely complex alpha and beta."""
    alpha, beta = (1.5 - 0.5j, -0.5 + 0.25j) if dtype in "cz" else (1.5, -0.5)
    for ta, tb in OPS9:
        b = inputs.UniformBatch(dtype, ta, tb, m, m, m, 517, seed=7)
        got = H.run_gpu(b, alpha, beta)
        H.assert_parity(b, got, H.oracle_ref(b, alpha, beta), alpha, beta)


@pytest.mark.parametrize("dtype", ["s", "d"])
@pytest.mark.parametrize("shape", [(4, 16, 4), (9, 16, 9), (16, 8, 16), (3, 9, 3), (16, 16, 1)])
def test_rectangular_fem_shapes(dtype, shape):
    """FEM-like rectangular shapes, op(A) = T, op(B) = N, beta = 1."""
    m, n, k = shape
    b = inputs.UniformBatch(dtype, "T", "N", m, n, k, 5003, seed=11)
    got = H.run_gpu(b, 1.0, 1.0)
    H.assert_parity(b, got, H.oracle_ref(b, 1.0, 1.0), 1.0, 1.0)
    bi = inputs.UniformBatch(dtype, "T", "N", m, n, k, 2001, seed=12, int_valued=True)
    H.assert_parity(bi, H.run_gpu(bi, 1.0, 1.0), H.oracle_ref(bi, 1.0, 1.0), 1.0, 1.0, exact=True)


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z", "h", "b"])
@pytest.mark.parametrize("shape", [(7, 3, 11), (1, 16, 16), (16, 1, 16), (2, 13, 5), (16, 16, 15)])
def test_generic_runtime_shapes(dtype, shape):
    """Shapes without a specialised kernel run on the generic kernel."""
    m, n, k = shape
    alpha, beta = scalars(dtype)
    for ta, tb in (("N", "N"), ("C", "T")):
        b = inputs.UniformBatch(dtype, ta, tb, m, n, k, 777, seed=13)
        got = H.run_gpu(b, alpha, beta)
        H.assert_parity(b, got, H.oracle_ref(b, alpha, beta), alpha, beta)


@pytest.mark.parametrize("dtype", ["s", "z"])
@pytest.mark.parametrize("m", [3, 8, 16])
def test_non_minimal_leading_dimensions(dtype, m):
    """Padded ld and ld2 take the element-gather staging path; the gaps in
    C are left untouched."""
    alpha, beta = scalars(dtype)
    for ta, tb in (("N", "N"), ("T", "C")):
        b = inputs.UniformBatch(dtype, ta, tb, m, m, m, 613, seed=17, pad_ld=1, pad_ld2=3)
        got = H.run_gpu(b, alpha, beta)
        H.assert_parity(b, got, H.oracle_ref(b, alpha, beta), alpha, beta)


@pytest.mark.parametrize("dtype", ["s", "c"])
def test_unaligned_base_pointers(dtype):
    """Operands starting off a 16-byte boundary still give the exact result."""
    m = 8
    b = inputs.UniformBatch(dtype, "N", "N", m, m, m, 999, seed=19, int_valued=True)
    es = b.A.itemsize
    tA, pA = H.to_dev(b.A, pad_front=es)
    tB, pB = H.to_dev(b.B, pad_front=es)
    tC, pC = H.to_dev(b.C, pad_front=es)
    sbgemm.gemm_multi_uniform(dtype, "N", "N", m, m, m, 1.5, pA, m, m * m, pB, m, m * m, -0.5,
                              pC, m, m * m, b.batch)
    torch.cuda.synchronize()
    got, _ = H.from_dev(tC, b.C, es)
    H.assert_parity(b, got, H.oracle_ref(b, 1.5, -0.5), 1.5, -0.5, exact=True)


def test_shared_a_matrix_ld2_zero():
    """lda2 = 0: every pair uses the same A (C_p = A B_p)."""
    m, N = 6, 400
    b = inputs.UniformBatch("d", "N", "N", m, m, m, N, seed=23, int_valued=True)
    A1 = b.A[:m * m].copy()
    tA, pA = H.to_dev(A1)
    tB, pB = H.to_dev(b.B)
    tC, pC = H.to_dev(b.C)
    sbgemm.gemm_multi_uniform("d", "N", "N", m, m, m, 1.0, pA, m, 0, pB, m, m * m, 0.0, pC, m,
                              m * m, N)
    torch.cuda.synchronize()
    got, _ = H.from_dev(tC, b.C)
    import oracle
    ref = oracle.gemm_uniform("d", "N", "N", m, m, m, 1.0, A1, m, 0, b.B, m, m * m, 0.0, b.C, m,
                              m * m, N)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z", "h", "b"])
@pytest.mark.parametrize("shared", ["A", "B", "AB"])
@pytest.mark.parametrize("shape", [("N", "N", 16, 16, 16), ("T", "C", 5, 7, 3),
                                   ("N", "T", 8, 8, 8), ("N", "N", 1, 1, 1)])
def test_shared_matrix_staged_once(dtype, shared, shape):
    """ld2 = 0 for A and/or B: one matrix for every pair, staged once per
    block; many tiles and a ragged last tile, beta zero and nonzero."""
    ta, tb, m, n, k = shape
    N = 2999
    exact = dtype in "sdcz"
    b = inputs.UniformBatch(dtype, ta, tb, m, n, k, N, seed=31 + m, int_valued=exact)
    if "A" in shared:
        b.A = b.A[:b.lda2].copy()
        b.lda2 = 0
    if "B" in shared:
        b.B = b.B[:b.ldb2].copy()
        b.ldb2 = 0
    for beta in (0.0, -0.5):
        got = H.run_gpu(b, 1.5, beta)
        H.assert_parity(b, got, H.oracle_ref(b, 1.5, beta), 1.5, beta, exact=exact)


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z", "h", "b"])
def test_beta_zero_never_reads_c(dtype):
    """beta = 0: C filled with NaN must not reach the result."""
    m = 9
    nan_bits = {"h": 0x7E00, "b": 0x7FC0}
    b = inputs.UniformBatch(dtype, "N", "T", m, m, m, 800, seed=29)
    C = b.C.copy()
    C[:] = nan_bits[dtype] if dtype in "hb" else np.nan
    got = H.run_gpu(b, 1.5, 0.0, C=C)
    ref = H.oracle_ref(b, 1.5, 0.0, C=C)
    assert np.all(np.isfinite(H.blocks(b, H.decode(got, dtype))))
    H.assert_parity(b, got, ref, 1.5, 0.0, C=C)


@pytest.mark.parametrize("dtype", ["s", "z"])
def test_alpha_zero_and_k_zero(dtype):
    """alpha = 0 or k = 0: C = beta*C without reading A or B (NaN there)."""
    m = 5
    b = inputs.UniformBatch(dtype, "N", "N", m, m, m, 300, seed=31)
    A = b.A.copy(); A[:] = np.nan
    B = b.B.copy(); B[:] = np.nan
    got = H.run_gpu(b, 0.0, -0.5, A=A, B=B)
    H.assert_parity(b, got, H.oracle_ref(b, 0.0, -0.5, A=A, B=B), 0.0, -0.5, exact=True, A=A, B=B)
    b0 = inputs.UniformBatch(dtype, "N", "N", m, m, 0, 300, seed=32)
    got0 = H.run_gpu(b0, 1.5, -0.5)
    H.assert_parity(b0, got0, H.oracle_ref(b0, 1.5, -0.5), 1.5, -0.5, exact=True)


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z"])
def test_device_scalars(dtype):
    """alpha and beta read by the kernel from device memory, including a
    device beta of 0 (C must not be read) and a device alpha of 0."""
    m = 12
    alpha, beta = (1.5 - 0.5j, -0.5 + 0.25j) if dtype in "cz" else (1.5, -0.5)
    b = inputs.UniformBatch(dtype, "T", "N", m, m, m, 700, seed=37)
    got = H.run_gpu(b, alpha, beta, device_scalars=True)
    H.assert_parity(b, got, H.oracle_ref(b, alpha, beta), alpha, beta)
    C = b.C.copy(); C[:] = np.nan
    got = H.run_gpu(b, alpha, 0.0, device_scalars=True, C=C)
    H.assert_parity(b, got, H.oracle_ref(b, alpha, 0.0, C=C), alpha, 0.0, C=C)
    A = b.A.copy(); A[:] = np.nan
    got = H.run_gpu(b, 0.0, beta, device_scalars=True, A=A)
    H.assert_parity(b, got, H.oracle_ref(b, 0.0, beta, A=A), 0.0, beta, A=A)


@pytest.mark.parametrize("dtype", ["s", "z"])
@pytest.mark.parametrize("m", [3, 10, 16])
def test_every_variant(dtype, m):
    nv = sbgemm.num_variants(dtype, m, m, m)
    assert nv >= 2
    alpha, beta = scalars(dtype)
    b = inputs.UniformBatch(dtype, "N", "C", m, m, m, 2111, seed=41, int_valued=True)
    ref = H.oracle_ref(b, alpha, beta)
    for v in range(nv):
        got = H.run_gpu(b, alpha, beta, variant=v)
        H.assert_parity(b, got, ref, alpha, beta, exact=True)


@pytest.mark.parametrize("dtype", ["h", "b"])
@pytest.mark.parametrize("m", [8, 12, 16])
def test_16bit_storage(dtype, m):
    """16-bit storage, fp32 accumulation, result rounded to 16 bits."""
    for (ta, tb), beta in itertools.product((("N", "N"), ("T", "N")), (0.0, -0.5)):
        b = inputs.UniformBatch(dtype, ta, tb, m, m, m, 1500, seed=43)
        got = H.run_gpu(b, 1.5, beta)
        H.assert_parity(b, got, H.oracle_ref(b, 1.5, beta), 1.5, beta)


@pytest.mark.parametrize("dtype", ["h", "b"])
@pytest.mark.parametrize("m", [8, 12, 16])
def test_tensor_core_variant(dtype, m):
    """The mma.sync path of the 16-bit types (variant 7; the default for N/N
    flat m = 8, 12, 16)
    against the pipelined kernel's variant 0 and the oracle: ragged and tiny
    batches (odd counts leave m = 8 with a half-used MMA), beta zero and not,
    device scalars, and alpha = 0 with NaN in A and B (not read)."""
    for N in (1, 2, 3, 31, 1001, 4099):
        for beta in (0.0, -0.5):
            b = inputs.UniformBatch(dtype, "N", "N", m, m, m, N, seed=3 * N + m)
            ref = H.oracle_ref(b, 1.5, beta)
            got7 = H.run_gpu(b, 1.5, beta, variant=7)
            H.assert_parity(b, got7, ref, 1.5, beta)
            assert np.array_equal(H.run_gpu(b, 1.5, beta), got7)   # the default: same kernel
    b = inputs.UniformBatch(dtype, "N", "N", m, m, m, 777, seed=5)
    H.assert_parity(b, H.run_gpu(b, 1.5, -0.5, device_scalars=True), H.oracle_ref(b, 1.5, -0.5),
                    1.5, -0.5)
    nan = {"h": 0x7E00, "b": 0x7FC0}[dtype]
    A = np.full_like(b.A, nan)
    B = np.full_like(b.B, nan)
    got = H.run_gpu(b, 0.0, -0.5, A=A, B=B, device_scalars=True)
    H.assert_parity(b, got, H.oracle_ref(b, 0.0, -0.5), 0.0, -0.5)
    # a request the tensor-core kernel does not take runs variant 0
    bt = inputs.UniformBatch(dtype, "T", "N", m, m, m, 500, seed=6)
    H.assert_parity(bt, H.run_gpu(bt, 1.5, -0.5, variant=7), H.oracle_ref(bt, 1.5, -0.5), 1.5, -0.5)


def test_quick_returns_leave_c_untouched():
    b = inputs.UniformBatch("s", "N", "N", 4, 4, 4, 10, seed=47)
    for (m, n, N) in ((0, 4, 10), (4, 0, 10), (4, 4, 0)):
        tC, pC = H.to_dev(b.C)
        st = sbgemm.gemm_multi_uniform("s", "N", "N", m, n, 4, 1.0, 0, 4, 16, 0, 4, 16, 0.0, pC,
                                       4, 16, N)
        torch.cuda.synchronize()
        assert st == 0
        got, _ = H.from_dev(tC, b.C)
        assert np.array_equal(got, b.C)


def test_nondefault_stream_and_paper_entry_point():
    """The _async entry point on a side stream, and the paper-shaped
    synchronous-signature entry point on the default stream."""
    m = 10
    b = inputs.UniformBatch("s", "N", "N", m, m, m, 3000, seed=53, int_valued=True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        got = H.run_gpu(b, 1.0, 0.0, stream=s)
    H.assert_parity(b, got, H.oracle_ref(b, 1.0, 0.0), 1.0, 0.0, exact=True)
    import ctypes
    tA, pA = H.to_dev(b.A)
    tB, pB = H.to_dev(b.B)
    tC, pC = H.to_dev(b.C)
    one, zero = (ctypes.c_float * 1)(1.0), (ctypes.c_float * 1)(0.0)
    st = sbgemm.lib().sbgemm_Sgemm_multi_uniform(b"N", b"N", m, m, m, ctypes.addressof(one), pA,
                                                 m, m * m, pB, m, m * m, ctypes.addressof(zero),
                                                 pC, m, m * m, b.batch)
    assert st == 0
    torch.cuda.synchronize()
    got2, _ = H.from_dev(tC, b.C)
    assert np.array_equal(got2, got)


@pytest.mark.parametrize("m", SIZES)
def test_full_size_sampled(m):
    """The paper's basic workload (N = 100,000, NN, alpha = 1, beta = 0,
    Section 7) at full size in the benchmark's launch configuration,
    checked on a sample of pairs the oracle computes one by one."""
    N = 100_000
    b = inputs.UniformBatch("s", "N", "N", m, m, m, N, seed=59)
    got = H.run_gpu(b, 1.0, 0.0)
    rng = inputs.splitmix64(61, 512) % np.uint64(N)
    pick = np.unique(rng.astype(np.int64))
    sub = inputs.UniformBatch("s", "N", "N", m, m, m, pick.size, seed=0)
    S = m * m
    sub.A = b.A.reshape(N, S)[pick].ravel().copy()
    sub.B = b.B.reshape(N, S)[pick].ravel().copy()
    sub.C = b.C.reshape(N, S)[pick].ravel().copy()
    ref = H.oracle_ref(sub, 1.0, 0.0)
    gsub = got.reshape(N, S)[pick].ravel().copy()
    H.assert_parity(sub, gsub, ref, 1.0, 0.0)


@pytest.mark.parametrize("dtype", ["s", "d"])
@pytest.mark.parametrize("shape", [(4, 16, 4), (9, 16, 9), (16, 8, 16), (3, 9, 3), (16, 16, 1)])
def test_fem_shapes_full_size_sampled(dtype, shape):
    """The FEM-shaped batches at their benchmarked size (N = 500,000,
    op(A) = T, op(B) = N, alpha = 1, beta = 1) in the default launch
    configuration, checked on a sample of pairs (and the last pair) that the
    oracle computes one by one."""
    m, n, k = shape
    N = 500_000
    b = inputs.UniformBatch(dtype, "T", "N", m, n, k, N, seed=73)
    got = H.run_gpu(b, 1.0, 1.0)
    pick = np.unique((inputs.splitmix64(79, 300) % np.uint64(N)).astype(np.int64))
    pick = np.concatenate([pick, [N - 1]])
    sub = inputs.UniformBatch(dtype, "T", "N", m, n, k, pick.size, seed=0)
    sub.A = b.A.reshape(N, k * m)[pick].ravel().copy()
    sub.B = b.B.reshape(N, k * n)[pick].ravel().copy()
    sub.C = b.C.reshape(N, m * n)[pick].ravel().copy()
    H.assert_parity(sub, got.reshape(N, m * n)[pick].ravel().copy(), H.oracle_ref(sub, 1.0, 1.0),
                    1.0, 1.0)


def test_million_pairs_size16_sampled():
    N, m = 1_000_000, 16
    b = inputs.UniformBatch("s", "T", "N", m, m, m, N, seed=67)
    got = H.run_gpu(b, 1.5, -0.5)
    pick = np.unique((inputs.splitmix64(71, 400) % np.uint64(N)).astype(np.int64))
    pick = np.concatenate([pick, [N - 1]])
    S = m * m
    sub = inputs.UniformBatch("s", "T", "N", m, m, m, pick.size, seed=0)
    sub.A = b.A.reshape(N, S)[pick].ravel().copy()
    sub.B = b.B.reshape(N, S)[pick].ravel().copy()
    sub.C = b.C.reshape(N, S)[pick].ravel().copy()
    H.assert_parity(sub, got.reshape(N, S)[pick].ravel().copy(), H.oracle_ref(sub, 1.5, -0.5),
                    1.5, -0.5)


@pytest.mark.parametrize("dtype,pad", [("s", 0), ("d", 0), ("c", 1), ("z", 2), ("b", 0)])
def test_host_array_entry_point(dtype, pad):
    """Host arrays streamed through a small device work buffer (many chunks,
    double-buffered): same result as the oracle, gaps of a padded C intact."""
    import ctypes
    m, N = 9, 3001
    alpha, beta = (1.5 - 0.5j, -0.5 + 0.25j) if dtype in "cz" else (1.5, -0.5)
    b = inputs.UniformBatch(dtype, "T", "N", m, m, m, N, seed=71, pad_ld=pad, pad_ld2=pad)
    hA = torch.from_numpy(b.A.view(np.uint8).copy()).pin_memory()
    hB = torch.from_numpy(b.B.view(np.uint8).copy()).pin_memory()
    hC = torch.from_numpy(b.C.view(np.uint8).copy()).pin_memory()
    work = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    ab, bb = sbgemm._scalar_buf(dtype, alpha), sbgemm._scalar_buf(dtype, beta)
    s = torch.cuda.current_stream()
    st = sbgemm.lib().sbgemm_gemm_multi_uniform_host(
        sbgemm.TYPE_CODES[dtype], b"T", b"N", m, m, m, ctypes.addressof(ab), hA.data_ptr(), b.lda,
        b.lda2, hB.data_ptr(), b.ldb, b.ldb2, ctypes.addressof(bb), hC.data_ptr(), b.ldc, b.ldc2, N,
        work.data_ptr(), work.numel(), s.cuda_stream)
    assert st == 0
    s.synchronize()
    got = hC.numpy().view(b.C.dtype).copy()
    H.assert_parity(b, got, H.oracle_ref(b, alpha, beta), alpha, beta)
    # beta = 0 with a flat C: C is not copied in (NaN there must not matter)
    b0 = inputs.UniformBatch(dtype, "N", "N", m, m, m, N, seed=72)
    hC0 = torch.full((b0.C.nbytes,), 0xFF, dtype=torch.uint8).pin_memory()
    hA0 = torch.from_numpy(b0.A.view(np.uint8).copy()).pin_memory()
    hB0 = torch.from_numpy(b0.B.view(np.uint8).copy()).pin_memory()
    zb = sbgemm._scalar_buf(dtype, 0.0)
    st = sbgemm.lib().sbgemm_gemm_multi_uniform_host(
        sbgemm.TYPE_CODES[dtype], b"N", b"N", m, m, m, ctypes.addressof(ab), hA0.data_ptr(), m,
        m * m, hB0.data_ptr(), m, m * m, ctypes.addressof(zb), hC0.data_ptr(), m, m * m, N,
        work.data_ptr(), work.numel(), s.cuda_stream)
    assert st == 0
    s.synchronize()
    got0 = hC0.numpy().view(b0.C.dtype).copy()
    H.assert_parity(b0, got0, H.oracle_ref(b0, alpha, 0.0), alpha, 0.0)


def test_host_array_entry_point_errors():
    import ctypes
    L = sbgemm.lib()
    one = sbgemm._scalar_buf("s", 1.0)
    work = torch.empty(64, dtype=torch.uint8, device="cuda")
    h = torch.zeros(16 * 100, dtype=torch.float32).pin_memory()
    # a 64-byte work buffer cannot hold two 4x4 pairs
    st = L.sbgemm_gemm_multi_uniform_host(0, b"N", b"N", 4, 4, 4, ctypes.addressof(one), h.data_ptr(),
                                          4, 16, h.data_ptr(), 4, 16, ctypes.addressof(one),
                                          h.data_ptr(), 4, 16, 100, work.data_ptr(), 64, None)
    assert st == -8
    st = L.sbgemm_gemm_multi_uniform_host(0, b"N", b"N", 4, 4, 4, ctypes.addressof(one), h.data_ptr(),
                                          3, 16, h.data_ptr(), 4, 16, ctypes.addressof(one),
                                          h.data_ptr(), 4, 16, 100, work.data_ptr(), 64, None)
    assert st == -3


def test_grouped_host_entry_point():
    """Several uniform batches (different shapes and ops) as one grouped
    host-array call through a small work buffer."""
    import ctypes
    specs = [("N", "N", 3, 3, 3, 5001), ("T", "N", 16, 16, 16, 2000), ("N", "T", 7, 5, 9, 3333),
             ("C", "N", 1, 1, 1, 10)]
    batches, groups, keep = [], (sbgemm.HostGroup * len(specs))(), []
    for g, (ta, tb, m, n, k, N) in zip(groups, specs):
        b = inputs.UniformBatch("s", ta, tb, m, n, k, N, seed=m + n)
        hA = torch.from_numpy(b.A.copy()).pin_memory()
        hB = torch.from_numpy(b.B.copy()).pin_memory()
        hC = torch.from_numpy(b.C.copy()).pin_memory()
        keep += [hA, hB, hC]
        g.transa, g.transb, g.m, g.n, g.k = ta.encode(), tb.encode(), m, n, k
        g.hA, g.lda, g.lda2 = hA.data_ptr(), b.lda, b.lda2
        g.hB, g.ldb, g.ldb2 = hB.data_ptr(), b.ldb, b.ldb2
        g.hC, g.ldc, g.ldc2 = hC.data_ptr(), b.ldc, b.ldc2
        g.batchCount = N
        batches.append((b, hC))
    work = torch.empty(2 << 20, dtype=torch.uint8, device="cuda")
    ab, bb = sbgemm._scalar_buf("s", 1.5), sbgemm._scalar_buf("s", -0.5)
    s = torch.cuda.current_stream()
    st = sbgemm.lib().sbgemm_gemm_grouped_host(0, ctypes.addressof(ab), ctypes.addressof(bb),
                                               ctypes.addressof(groups), len(specs), work.data_ptr(),
                                               work.numel(), s.cuda_stream)
    assert st == 0
    s.synchronize()
    for b, hC in batches:
        H.assert_parity(b, hC.numpy().copy(), H.oracle_ref(b, 1.5, -0.5), 1.5, -0.5)
