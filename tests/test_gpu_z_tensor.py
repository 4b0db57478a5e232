"""Complex fp64 on the tensor cores (variant 7 of the z shapes with
specialised kernels, variant 1 of the others): real and imaginary parts
split into exact 8-bit digits, the four real products on the fp16 MMA path,
recombined exactly in integers.  Held to the oracle checks of the complex
FMA kernels: bit-exact on small-integer inputs, within the elementwise bound
of gpu_helpers on uniform inputs, on parts spanning many binades (the
entries the emulation cannot bound fall back to fp64 FMAs), and on special
values, for every op pair including conjugation."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

from paper_1304_7053_gb300 import inputs, sbgemm
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

TC = 7
OPS = [("N", "N"), ("T", "N"), ("N", "C"), ("C", "C"), ("C", "T")]
ALPHA = 1.5 - 0.5j
BETAS = (0.0 + 0.0j, -0.5 + 0.25j)


@pytest.mark.parametrize("m", list(range(1, 17)))
def test_integer_inputs_bit_exact(m):
    for (ta, tb), beta in itertools.product(OPS, BETAS):
        b = inputs.UniformBatch("z", ta, tb, m, m, m, 613, seed=300 + m, int_valued=True)
        got = H.run_gpu(b, ALPHA, beta, variant=TC)
        H.assert_parity(b, got, H.oracle_ref(b, ALPHA, beta), ALPHA, beta, exact=True)


@pytest.mark.parametrize("m", list(range(1, 17)))
def test_uniform_inputs_within_bound(m):
    for (ta, tb), beta in itertools.product(OPS, BETAS):
        b = inputs.UniformBatch("z", ta, tb, m, m, m, 517, seed=400 + m)
        got = H.run_gpu(b, ALPHA, beta, variant=TC)
        H.assert_parity(b, got, H.oracle_ref(b, ALPHA, beta), ALPHA, beta)
    # alpha = 1, beta = 0 (the epilogue that writes the product as is)
    b = inputs.UniformBatch("z", "N", "N", m, m, m, 517, seed=450 + m)
    H.assert_parity(b, H.run_gpu(b, 1.0 + 0j, 0j, variant=TC), H.oracle_ref(b, 1.0 + 0j, 0j),
                    1.0 + 0j, 0j)


@pytest.mark.parametrize("shape", [(4, 16, 4), (9, 16, 9), (16, 8, 16), (3, 9, 3), (16, 16, 1)])
def test_fem_shapes_and_padded_layout(shape):
    m, n, k = shape
    b = inputs.UniformBatch("z", "T", "N", m, n, k, 1003, seed=17)
    H.assert_parity(b, H.run_gpu(b, 1.0 + 0j, 1.0 + 0j, variant=TC),
                    H.oracle_ref(b, 1.0 + 0j, 1.0 + 0j), 1.0 + 0j, 1.0 + 0j)
    bp = inputs.UniformBatch("z", "N", "C", m, n, k, 499, seed=18, pad_ld=2, pad_ld2=5)
    H.assert_parity(bp, H.run_gpu(bp, ALPHA, BETAS[1], variant=TC),
                    H.oracle_ref(bp, ALPHA, BETAS[1]), ALPHA, BETAS[1])


def _scale_parts(x, seed, lo=-60):
    """Scale the real and the imaginary part of every entry by independent
    powers 2^e, e uniform in lo..0."""
    v = x.view(np.float64)
    e = (inputs.splitmix64(seed, v.size) % np.uint64(1 - lo)).astype(np.int64) + lo
    v[:] = np.ldexp(v, e)


@pytest.mark.parametrize("m", [4, 9, 16])
def test_wide_dynamic_range_within_bound(m):
    """Parts spanning 60 binades: many outputs fail the emulation's own
    accuracy test and take the fp64 FMA path; every output meets the bound."""
    for ta, tb in (("N", "N"), ("C", "T")):
        b = inputs.UniformBatch("z", ta, tb, m, m, m, 1001, seed=500 + m)
        _scale_parts(b.A, 700 + m)
        _scale_parts(b.B, 800 + m)
        got = H.run_gpu(b, ALPHA, BETAS[1], variant=TC)
        H.assert_parity(b, got, H.oracle_ref(b, ALPHA, BETAS[1]), ALPHA, BETAS[1])


def test_real_or_imaginary_operands():
    """One part of an operand zero (purely real or purely imaginary
    matrices): the emulation's scale comes from the other part."""
    m, N = 12, 301
    for which in range(4):
        b = inputs.UniformBatch("z", "N", "T", m, m, m, N, seed=550 + which)
        (b.A if which < 2 else b.B).view(np.float64)[which % 2::2] = 0.0
        got = H.run_gpu(b, ALPHA, BETAS[1], variant=TC)
        H.assert_parity(b, got, H.oracle_ref(b, ALPHA, BETAS[1]), ALPHA, BETAS[1])


def test_extreme_exponents_and_special_values():
    """Pairs scaled near the top and bottom of the fp64 range, zero rows and
    columns, a subnormal row, and pairs with NaN or Inf in one part: finite
    results within the bound, non-finite positions as the FMA kernel gives
    them."""
    m, N = 8, 64
    b = inputs.UniformBatch("z", "N", "N", m, m, m, N, seed=601)
    A = b.A.reshape(N, m * m)
    B = b.B.reshape(N, m * m)
    A[0] *= 2.0 ** 500
    B[0] *= 2.0 ** 500
    A[1] *= 2.0 ** -540
    B[1] *= 2.0 ** -540
    A[2, :m] = 0.0                                  # column 0 of pair 2's A
    A[3, 5] = complex(1.0, np.nan)
    B[4, 7] = complex(np.inf, 0.5)
    A[5, 0::m] = 0.0                                # row 0 of pair 5's A
    B[6, :m] = 0.0                                  # column 0 of pair 6's B
    A[7] = 0.0                                      # all of pair 7's A
    A[8, 1::m] = np.ldexp(np.arange(1, m + 1), -1070) * (1 + 1j)   # a subnormal row,
    B[8] *= 2.0 ** 60                                               # products normal
    got = H.run_gpu(b, 1.0 + 0j, 0j, variant=TC)
    ref_fma = H.run_gpu(b, 1.0 + 0j, 0j, variant=0)
    g, r = got.reshape(N, -1), ref_fma.reshape(N, -1)
    for part in (np.real, np.imag):
        assert np.array_equal(np.isnan(part(g)), np.isnan(part(r)))
        assert np.array_equal(np.isinf(part(g)), np.isinf(part(r)))
    fin = np.ones(N, dtype=bool)
    fin[[3, 4]] = False
    sub = inputs.UniformBatch("z", "N", "N", m, m, m, int(fin.sum()), seed=0)
    sub.A = A[fin].ravel().copy()
    sub.B = B[fin].ravel().copy()
    sub.C = b.C.reshape(N, -1)[fin].ravel().copy()
    H.assert_parity(sub, g[fin].ravel().copy(), H.oracle_ref(sub, 1.0 + 0j, 0j), 1.0 + 0j, 0j)


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 12, 12), (16, 16, 15)])
def test_device_scalars(shape):
    """alpha and beta read from device memory: the general case, a device
    beta of 0 (NaN-filled C is not read), a device alpha of 0 (C = beta C,
    NaN-filled A is not read), on the tensor-core variant and the default."""
    m, n, k = shape
    tc = TC if m == n == k else 1
    b = inputs.UniformBatch("z", "C", "N", m, n, k, 1501, seed=77)
    for variant in (tc, None):
        got = H.run_gpu(b, ALPHA, BETAS[1], variant=variant, device_scalars=True)
        H.assert_parity(b, got, H.oracle_ref(b, ALPHA, BETAS[1]), ALPHA, BETAS[1])
        C = b.C.copy(); C[:] = np.nan
        got = H.run_gpu(b, ALPHA, 0j, variant=variant, device_scalars=True, C=C)
        H.assert_parity(b, got, H.oracle_ref(b, ALPHA, 0j, C=C), ALPHA, 0j, C=C)
        A = b.A.copy(); A[:] = np.nan
        got = H.run_gpu(b, 0j, BETAS[1], variant=variant, device_scalars=True, A=A)
        H.assert_parity(b, got, H.oracle_ref(b, 0j, BETAS[1], A=A), 0j, BETAS[1], A=A)
        got = H.run_gpu(b, 0j, 0j, variant=variant, device_scalars=True, A=A, C=C)
        assert np.all(H.blocks(b, got) == 0)


GENERIC_SHAPES = [(16, 16, 15), (15, 16, 16), (14, 16, 12), (16, 9, 13), (13, 7, 16),
                  (1, 16, 16), (16, 1, 16), (7, 3, 11), (5, 16, 2)]


@pytest.mark.parametrize("shape", GENERIC_SHAPES)
def test_generic_shapes_variant1(shape):
    m, n, k = shape
    assert sbgemm.num_variants("z", m, n, k) == 2
    assert "tensor-core" in sbgemm.variant_name("z", m, n, k, 1)
    for i, ((ta, tb), beta) in enumerate(itertools.product(OPS, BETAS)):
        bi = inputs.UniformBatch("z", ta, tb, m, n, k, 301, seed=800 + i, int_valued=True)
        H.assert_parity(bi, H.run_gpu(bi, ALPHA, beta, variant=1), H.oracle_ref(bi, ALPHA, beta),
                        ALPHA, beta, exact=True)
        bu = inputs.UniformBatch("z", ta, tb, m, n, k, 401, seed=900 + i, pad_ld=i % 3,
                                 pad_ld2=(3 * i) % 7)
        H.assert_parity(bu, H.run_gpu(bu, ALPHA, beta, variant=1), H.oracle_ref(bu, ALPHA, beta),
                        ALPHA, beta)
