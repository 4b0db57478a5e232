"""Real fp64 on the tensor cores (variant 7 of the d shapes with specialised
kernels): operands split into exact 8-bit digits, digit products on the fp16
MMA path, recombined exactly in integers.  Held to the same oracle checks as
the fp64 FMA kernels: bit-exact on small-integer inputs, within the
elementwise bound of gpu_helpers on uniform[-1, 1] inputs, and within the
bound on inputs whose rows and columns span many binades (the entries the
emulation cannot bound fall back to fp64 FMAs inside the kernel)."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

from paper_1304_7053_gb300 import inputs
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

TC = 7
OPS = [("N", "N"), ("T", "N"), ("N", "T"), ("C", "C")]


@pytest.mark.parametrize("m", list(range(1, 17)))
def test_integer_inputs_bit_exact(m):
    for (ta, tb), beta in itertools.product(OPS, (0.0, -0.5)):
        b = inputs.UniformBatch("d", ta, tb, m, m, m, 1237, seed=300 + m, int_valued=True)
        got = H.run_gpu(b, 1.5, beta, variant=TC)
        H.assert_parity(b, got, H.oracle_ref(b, 1.5, beta), 1.5, beta, exact=True)


@pytest.mark.parametrize("m", list(range(1, 17)))
def test_uniform_inputs_within_bound(m):
    for (ta, tb), beta in itertools.product(OPS, (0.0, -0.5)):
        b = inputs.UniformBatch("d", ta, tb, m, m, m, 1031, seed=400 + m)
        got = H.run_gpu(b, 1.5, beta, variant=TC)
        H.assert_parity(b, got, H.oracle_ref(b, 1.5, beta), 1.5, beta)


@pytest.mark.parametrize("shape", [(4, 16, 4), (9, 16, 9), (16, 8, 16), (3, 9, 3), (16, 16, 1)])
def test_fem_shapes_and_padded_layout(shape):
    m, n, k = shape
    b = inputs.UniformBatch("d", "T", "N", m, n, k, 2003, seed=17)
    H.assert_parity(b, H.run_gpu(b, 1.0, 1.0, variant=TC), H.oracle_ref(b, 1.0, 1.0), 1.0, 1.0)
    bp = inputs.UniformBatch("d", "N", "T", m, n, k, 999, seed=18, pad_ld=2, pad_ld2=5)
    H.assert_parity(bp, H.run_gpu(bp, 1.5, -0.5, variant=TC), H.oracle_ref(bp, 1.5, -0.5), 1.5, -0.5)


def _wide_range(b, seed):
    """Scale every entry of A and B by 2^e, e uniform in -60..0, so rows and
    columns mix entries of very different sizes."""
    for name, s in (("A", seed), ("B", seed + 1)):
        x = getattr(b, name)
        e = (inputs.splitmix64(s, x.size) % np.uint64(61)).astype(np.int64)
        setattr(b, name, np.ldexp(x, -e))


@pytest.mark.parametrize("m", [4, 9, 16])
def test_wide_dynamic_range_within_bound(m):
    """Entries spanning 60 binades: many outputs fail the emulation's own
    accuracy test and take the fp64 FMA path; every output meets the bound."""
    for ta, tb in (("N", "N"), ("T", "T")):
        b = inputs.UniformBatch("d", ta, tb, m, m, m, 2001, seed=500 + m)
        _wide_range(b, 700 + m)
        got = H.run_gpu(b, 1.5, -0.5, variant=TC)
        H.assert_parity(b, got, H.oracle_ref(b, 1.5, -0.5), 1.5, -0.5)


def test_extreme_exponents_and_special_values():
    """Rows scaled near the top and bottom of the fp64 range (subnormal
    products), a zero row, and pairs with NaN or Inf: finite results within
    the bound, non-finite positions as the FMA kernel gives them."""
    m, N = 8, 64
    b = inputs.UniformBatch("d", "N", "N", m, m, m, N, seed=601)
    A = b.A.reshape(N, m * m)
    B = b.B.reshape(N, m * m)
    A[0] *= 2.0 ** 500
    B[0] *= 2.0 ** 500
    A[1] *= 2.0 ** -540
    B[1] *= 2.0 ** -540
    A[2, :m] = 0.0               # column 0 of pair 2's A
    A[3, 5] = np.nan
    B[4, 7] = np.inf
    A[5, 0::m] = 0.0             # row 0 of pair 5's A
    B[6, :m] = 0.0               # column 0 of pair 6's B
    A[7] = 0.0                   # all of pair 7's A
    A[8, 1::m] = np.ldexp(np.arange(1, m + 1), -1070)   # a subnormal row,
    B[8] *= 2.0 ** 60                                    # products in the normal range
    got = H.run_gpu(b, 1.0, 0.0, variant=TC)
    ref_fma = H.run_gpu(b, 1.0, 0.0, variant=0)
    g, r = got.reshape(N, -1), ref_fma.reshape(N, -1)
    assert np.array_equal(np.isnan(g), np.isnan(r)) and np.array_equal(np.isinf(g), np.isinf(r))
    fin = np.ones(N, dtype=bool)
    fin[[3, 4]] = False
    sub = inputs.UniformBatch("d", "N", "N", m, m, m, int(fin.sum()), seed=0)
    sub.A = A[fin].ravel().copy()
    sub.B = B[fin].ravel().copy()
    sub.C = b.C.reshape(N, -1)[fin].ravel().copy()
    H.assert_parity(sub, g[fin].ravel().copy(), H.oracle_ref(sub, 1.0, 0.0), 1.0, 0.0)


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 12, 12), (16, 16, 15)])
def test_device_scalars_and_default_selection(shape):
    """alpha and beta read from device memory: the general case, a device
    beta of 0 (C is not read: NaN-filled C), a device alpha of 0 (C = beta C,
    A and B are not read: NaN-filled A), on the tensor-core variant (7, or 1
    for a shape without specialised kernels) and on the default choice."""
    m, n, k = shape
    tc = TC if m == n == k else 1
    b = inputs.UniformBatch("d", "N", "N", m, n, k, 3001, seed=77)
    for variant in (tc, None):
        got = H.run_gpu(b, 1.5, -0.5, variant=variant, device_scalars=True)
        H.assert_parity(b, got, H.oracle_ref(b, 1.5, -0.5), 1.5, -0.5)
        C = b.C.copy(); C[:] = np.nan
        got = H.run_gpu(b, 1.5, 0.0, variant=variant, device_scalars=True, C=C)
        H.assert_parity(b, got, H.oracle_ref(b, 1.5, 0.0, C=C), 1.5, 0.0, C=C)
        A = b.A.copy(); A[:] = np.nan
        got = H.run_gpu(b, 0.0, -0.5, variant=variant, device_scalars=True, A=A)
        H.assert_parity(b, got, H.oracle_ref(b, 0.0, -0.5, A=A), 0.0, -0.5, A=A)
        got = H.run_gpu(b, 0.0, 0.0, variant=variant, device_scalars=True, A=A, C=C)
        assert np.all(H.blocks(b, got) == 0.0)


# shapes without specialised kernels: the tensor-core kernel is public
# variant 1 there (variant 0 is the generic kernel)
GENERIC_SHAPES = [(16, 16, 15), (15, 16, 16), (16, 15, 16), (14, 16, 12), (16, 9, 13),
                  (13, 7, 16), (1, 16, 16), (16, 1, 16), (7, 3, 11), (5, 16, 2), (12, 10, 14)]


@pytest.mark.parametrize("shape", GENERIC_SHAPES)
def test_generic_shapes_variant1(shape):
    m, n, k = shape
    from paper_1304_7053_gb300 import sbgemm
    assert sbgemm.num_variants("d", m, n, k) == 2
    assert "tensor-core" in sbgemm.variant_name("d", m, n, k, 1)
    for i, ((ta, tb), beta) in enumerate(itertools.product(OPS, (0.0, -0.5))):
        bi = inputs.UniformBatch("d", ta, tb, m, n, k, 777, seed=800 + i, int_valued=True)
        H.assert_parity(bi, H.run_gpu(bi, 1.5, beta, variant=1), H.oracle_ref(bi, 1.5, beta),
                        1.5, beta, exact=True)
        bu = inputs.UniformBatch("d", ta, tb, m, n, k, 901, seed=900 + i, pad_ld=i % 3,
                                 pad_ld2=(3 * i) % 7)
        H.assert_parity(bu, H.run_gpu(bu, 1.5, beta, variant=1), H.oracle_ref(bu, 1.5, beta),
                        1.5, beta)


@pytest.mark.parametrize("shape", [(16, 16, 15), (14, 16, 12), (7, 3, 11)])
def test_generic_shapes_default_and_pointer_arrays(shape):
    """Whatever the default rule picks for a generic fp64 shape (the
    tensor-core kernel or the generic one), the uniform call and the
    pointer-array call (which has no tensor-core form and runs the generic
    kernel) both meet the bound."""
    m, n, k = shape
    b = inputs.UniformBatch("d", "N", "T", m, n, k, 1501, seed=950 + m)
    H.assert_parity(b, H.run_gpu(b, 1.5, -0.5), H.oracle_ref(b, 1.5, -0.5), 1.5, -0.5)
    H.assert_parity(b, H.run_gpu(b, 1.0, 0.0), H.oracle_ref(b, 1.0, 0.0), 1.0, 0.0)
    from tests.test_gpu_nounif import run_case
    for beta in (0.0, -0.5):
        run_case("d", ("N", "T", m, n, k), (1, 1), 1500, 1.5, beta, seed=970 + m)
