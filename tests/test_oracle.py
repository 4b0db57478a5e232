"""Pins for the CPU oracle (no GPU).  Each test checks the oracle against
something other than itself: numpy's strided views and matmul, exact
rational arithmetic, hand-expanded 2 x 2 / 3 x 3 products, closed forms,
and invariants that hold exactly on small-integer inputs."""
from __future__ import annotations

import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1304_7053_gb300 import inputs
from tests import refmath

OPS = ["N", "T", "C"]
HERE = os.path.dirname(os.path.abspath(__file__))


def run_oracle(b: inputs.UniformBatch, alpha, beta, **kw):
    return oracle.gemm_uniform(b.dtype, b.transa, b.transb, b.m, b.n, b.k, alpha,
                               b.A, b.lda, b.lda2, b.B, b.ldb, b.ldb2, beta,
                               b.C, b.ldc, b.ldc2, b.batch, **kw)


def blocks(b, flat):
    return refmath.gather_c(flat, b.m, b.n, b.ldc, b.ldc2, b.batch)


# ---------------------------------------------------------------- brute force

def test_hand_expanded_2x2_all_ops():
    """C = alpha op(A) op(B) + beta C for one 2x2 pair, every op pair, with
    each entry written out by hand (Eq. 1 and the op definitions of Sec. 2)."""
    a = {(0, 0): 1 + 2j, (1, 0): 3 - 1j, (0, 1): -2 + 0.5j, (1, 1): 4 + 1j}
    b = {(0, 0): 0.5 - 1j, (1, 0): 2 + 2j, (0, 1): -1 + 3j, (1, 1): 1 - 0.25j}
    c = {(0, 0): 1 + 1j, (1, 0): -1 + 0j, (0, 1): 0 + 2j, (1, 1): 3 - 3j}
    alpha, beta = 1.5 - 0.5j, -0.5 + 0.25j

    def opx(x, op, i, j):
        if op == "N":
            return x[(i, j)]
        if op == "T":
            return x[(j, i)]
        return np.conj(x[(j, i)])

    A = np.array([a[(0, 0)], a[(1, 0)], a[(0, 1)], a[(1, 1)]], dtype=np.complex128)
    B = np.array([b[(0, 0)], b[(1, 0)], b[(0, 1)], b[(1, 1)]], dtype=np.complex128)
    C = np.array([c[(0, 0)], c[(1, 0)], c[(0, 1)], c[(1, 1)]], dtype=np.complex128)
    for ta, tb in itertools.product(OPS, OPS):
        out = oracle.gemm_uniform("z", ta, tb, 2, 2, 2, alpha, A, 2, 4, B, 2, 4,
                                  beta, C, 2, 4, 1)
        for i in range(2):
            for j in range(2):
                want = alpha * (opx(a, ta, i, 0) * opx(b, tb, 0, j)
                                + opx(a, ta, i, 1) * opx(b, tb, 1, j)) + beta * c[(i, j)]
                assert out[i + 2 * j] == pytest.approx(want, abs=1e-14), (ta, tb, i, j)


def test_hand_expanded_real_3x3_transposes():
    """3x3 real entries written out: (A^T B)_ij = sum_l A_li B_lj."""
    A = np.arange(1, 10, dtype=np.float64)            # column-major: A(i,j) = A[i+3j]
    B = np.array([2, -1, 0, 1, 3, -2, 0, 1, 1], dtype=np.float64)
    C = np.zeros(9)
    out_nn = oracle.gemm_uniform("d", "N", "N", 3, 3, 3, 1.0, A, 3, 9, B, 3, 9, 0.0, C, 3, 9, 1)
    out_tn = oracle.gemm_uniform("d", "T", "N", 3, 3, 3, 1.0, A, 3, 9, B, 3, 9, 0.0, C, 3, 9, 1)
    out_nt = oracle.gemm_uniform("d", "N", "T", 3, 3, 3, 1.0, A, 3, 9, B, 3, 9, 0.0, C, 3, 9, 1)
    Aij = lambda i, j: A[i + 3 * j]
    Bij = lambda i, j: B[i + 3 * j]
    for i in range(3):
        for j in range(3):
            nn = Aij(i, 0) * Bij(0, j) + Aij(i, 1) * Bij(1, j) + Aij(i, 2) * Bij(2, j)
            tn = Aij(0, i) * Bij(0, j) + Aij(1, i) * Bij(1, j) + Aij(2, i) * Bij(2, j)
            nt = Aij(i, 0) * Bij(j, 0) + Aij(i, 1) * Bij(j, 1) + Aij(i, 2) * Bij(j, 2)
            assert out_nn[i + 3 * j] == nn
            assert out_tn[i + 3 * j] == tn
            assert out_nt[i + 3 * j] == nt


def test_1x1_is_scalar_fma():
    A = np.array([3.0, -2.0], dtype=np.float32)
    B = np.array([0.5, 4.0], dtype=np.float32)
    C = np.array([1.0, 1.0], dtype=np.float32)
    out = oracle.gemm_uniform("s", "N", "N", 1, 1, 1, 2.0, A, 1, 1, B, 1, 1, -3.0, C, 1, 1, 2)
    assert list(out) == [2.0 * 1.5 - 3.0, 2.0 * -8.0 - 3.0]


# ------------------------------------------------- numpy strided-view matmul

@pytest.mark.parametrize("dtype", ["s", "d", "c", "z"])
@pytest.mark.parametrize("ta,tb", list(itertools.product(OPS, OPS)))
def test_matches_numpy_strided_matmul(dtype, ta, tb):
    """Every op pair, rectangular sizes, padded ld and ld2 (Section 4 layout)."""
    m, n, k, N = 5, 3, 4, 7
    b = inputs.UniformBatch(dtype, ta, tb, m, n, k, N, seed=11, pad_ld=2, pad_ld2=3)
    alpha, beta = (1.5, -0.5) if dtype in "sd" else (1.5 - 0.5j, -0.5 + 0.25j)
    out = run_oracle(b, alpha, beta)
    want = refmath.numpy_gemm(dtype, ta, tb, m, n, k, alpha, b.A, b.lda, b.lda2, b.B,
                              b.ldb, b.ldb2, beta, b.C, b.ldc, b.ldc2, N)
    got = blocks(b, out)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (16, 16, 16), (4, 16, 4), (9, 16, 9),
                                   (16, 8, 16), (3, 9, 3), (16, 16, 1), (2, 7, 13)])
def test_shapes_match_numpy(m, n, k):
    b = inputs.UniformBatch("s", "T", "N", m, n, k, 5, seed=3)
    out = run_oracle(b, 1.0, 1.0)
    want = refmath.numpy_gemm("s", "T", "N", m, n, k, 1.0, b.A, b.lda, b.lda2, b.B, b.ldb,
                              b.ldb2, 1.0, b.C, b.ldc, b.ldc2, 5)
    np.testing.assert_allclose(blocks(b, out), want, rtol=1e-14, atol=1e-14)


def test_padding_untouched():
    """Entries outside the m x n blocks (ld and ld2 gaps) keep C's values."""
    b = inputs.UniformBatch("d", "N", "N", 3, 2, 4, 4, seed=5, pad_ld=3, pad_ld2=5)
    out = run_oracle(b, 1.0, 0.0)
    mask = np.zeros(b.C.size, dtype=bool)
    for p in range(b.batch):
        for j in range(b.n):
            for i in range(b.m):
                mask[i + b.ldc * j + b.ldc2 * p] = True
    assert np.array_equal(out[~mask], b.C[~mask])


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("dtype", ["s", "d", "c", "z"])
def test_all_ones_closed_form(dtype):
    """A = J (m x k), B = J (k x n)  =>  C = alpha k J + beta C."""
    m, n, k, N = 6, 5, 7, 3
    b = inputs.UniformBatch(dtype, "N", "N", m, n, k, N, seed=9)
    b.A[:] = 1
    b.B[:] = 1
    alpha, beta = 1.5, -0.5
    out = blocks(b, run_oracle(b, alpha, beta))
    Cv = refmath.views(b.C, m, n, b.ldc, b.ldc2, N)
    np.testing.assert_array_equal(out, alpha * k * np.ones((N, m, n)) + beta * Cv.astype(out.dtype))


@pytest.mark.parametrize("tb", OPS)
def test_identity_closed_form(tb):
    """A = I  =>  C = alpha op(B) + beta C (exact)."""
    m = n = k = 5
    N = 4
    b = inputs.UniformBatch("z", "N", tb, m, n, k, N, seed=2)
    b.A[:] = 0
    for p in range(N):
        for i in range(m):
            b.A[i + b.lda * i + b.lda2 * p] = 1
    alpha, beta = 2.0 - 1.0j, 0.5
    out = blocks(b, run_oracle(b, alpha, beta))
    br, bc = (k, n) if tb == "N" else (n, k)
    Bv = refmath.views(b.B, br, bc, b.ldb, b.ldb2, N)
    opB = refmath.apply_op(Bv, tb, True).astype(np.complex128)
    Cv = refmath.views(b.C, m, n, b.ldc, b.ldc2, N).astype(np.complex128)
    np.testing.assert_allclose(out, alpha * opB + beta * Cv, rtol=0, atol=1e-15)


def test_permutation_and_diagonal():
    """A permutation on the left permutes rows exactly; a diagonal scales rows."""
    m = n = k = 4
    b = inputs.UniformBatch("d", "N", "N", m, n, k, 1, seed=4)
    perm = [2, 0, 3, 1]
    b.A[:] = 0
    for i, pi in enumerate(perm):
        b.A[i + 4 * pi] = 1.0             # row i of P A picks row perm[i]
    out = blocks(b, run_oracle(b, 1.0, 0.0))[0]
    Bm = refmath.views(b.B, k, n, b.ldb, b.ldb2, 1)[0]
    np.testing.assert_array_equal(out, Bm[perm, :])
    d = np.array([2.0, -0.5, 4.0, 0.25])
    b.A[:] = 0
    for i in range(4):
        b.A[i + 4 * i] = d[i]
    out = blocks(b, run_oracle(b, 1.0, 0.0))[0]
    np.testing.assert_array_equal(out, d[:, None] * Bm)


# ----------------------------------------- beta == 0 / alpha == 0 semantics

@pytest.mark.parametrize("dtype", ["s", "d", "c", "z", "h", "b"])
def test_beta_zero_never_reads_c(dtype):
    """beta = 0: C is write-only, so NaN in C must not reach the result
    (the a1b0 functor of Section 5 never reads y)."""
    b = inputs.UniformBatch(dtype, "N", "N", 3, 3, 3, 4, seed=1)
    if dtype in "hb":
        b.C[:] = 0x7E00 if dtype == "h" else 0x7FC0
    else:
        b.C[:] = np.nan
    out = run_oracle(b, 1.0, 0.0)
    assert np.all(np.isfinite(blocks(b, out)))


@pytest.mark.parametrize("dtype", ["s", "z"])
def test_alpha_zero_or_k_zero_is_beta_c(dtype):
    b = inputs.UniformBatch(dtype, "N", "N", 3, 4, 5, 3, seed=6)
    b.A[:] = np.nan
    b.B[:] = np.nan
    out = blocks(b, run_oracle(b, 0.0, -0.5))
    Cv = refmath.views(b.C, 3, 4, b.ldc, b.ldc2, 3).astype(out.dtype)
    np.testing.assert_array_equal(out, -0.5 * Cv)
    b2 = inputs.UniformBatch(dtype, "N", "N", 3, 4, 0, 3, seed=6)
    out2 = blocks(b2, run_oracle(b2, 1.5, 2.0))
    Cv2 = refmath.views(b2.C, 3, 4, b2.ldc, b2.ldc2, 3).astype(out2.dtype)
    np.testing.assert_array_equal(out2, 2.0 * Cv2)


def test_real_c_is_t():
    b = inputs.UniformBatch("d", "C", "C", 4, 3, 5, 3, seed=8)
    out_c = run_oracle(b, 1.5, -0.5)
    out_t = oracle.gemm_uniform("d", "T", "T", 4, 3, 5, 1.5, b.A, b.lda, b.lda2, b.B, b.ldb,
                                b.ldb2, -0.5, b.C, b.ldc, b.ldc2, 3)
    assert np.array_equal(out_c, out_t)


def test_lowercase_trans():
    b = inputs.UniformBatch("c", "T", "C", 3, 3, 3, 2, seed=8)
    up = run_oracle(b, 1.0, 0.0)
    lo = oracle.gemm_uniform("c", "t", "c", 3, 3, 3, 1.0, b.A, b.lda, b.lda2, b.B, b.ldb,
                             b.ldb2, 0.0, b.C, b.ldc, b.ldc2, 2)
    assert np.array_equal(up, lo)


def test_argument_errors():
    # bad trans char, negative size, ld below rows, ldc2 below ldc*n (Fig. LD2)
    assert oracle.check_args("X", "N", 2, 2, 2, 2, 4, 2, 4, 2, 4, 1) == -1
    assert oracle.check_args("N", "N", -1, 2, 2, 2, 4, 2, 4, 2, 4, 1) == -2
    assert oracle.check_args("N", "N", 3, 2, 2, 2, 6, 2, 4, 3, 6, 1) == -3
    assert oracle.check_args("T", "N", 3, 2, 2, 1, 6, 2, 4, 3, 6, 1) == -3
    assert oracle.check_args("N", "N", 3, 2, 2, 3, 6, 2, 4, 3, 5, 1) == -3
    assert oracle.check_args("N", "N", 3, 2, 2, 3, 6, 2, 4, 3, 6, 1) == 0
    with pytest.raises(ValueError):
        oracle.gemm_uniform("s", "Q", "N", 1, 1, 1, 1.0, np.ones(1, np.float32), 1, 1,
                            np.ones(1, np.float32), 1, 1, 0.0, np.ones(1, np.float32), 1, 1, 1)


# ------------------------------------------- exact invariants on small ints

def test_associativity_on_integers():
    """(A B) x = A (B x) exactly on small-integer inputs (Eq. 1 applied twice)."""
    m = k = 6
    N = 5
    A = inputs.draw("d", m * k * N, 21, int_valued=True)
    Bm = inputs.draw("d", k * k * N, 22, int_valued=True)
    x = inputs.draw("d", k * N, 23, int_valued=True)
    z = np.zeros(m * k * N)
    AB = oracle.gemm_uniform("d", "N", "N", m, k, k, 1.0, A, m, m * k, Bm, k, k * k,
                             0.0, z, m, m * k, N)
    ABx = oracle.gemm_uniform("d", "N", "N", m, 1, k, 1.0, AB, m, m * k, x, k, k,
                              0.0, np.zeros(m * N), m, m, N)
    Bx = oracle.gemm_uniform("d", "N", "N", k, 1, k, 1.0, Bm, k, k * k, x, k, k,
                             0.0, np.zeros(k * N), k, k, N)
    ABx2 = oracle.gemm_uniform("d", "N", "N", m, 1, k, 1.0, A, m, m * k, Bx, k, k,
                               0.0, np.zeros(m * N), m, m, N)
    assert np.array_equal(ABx, ABx2)


def test_transpose_identity():
    """gemm(T, T, B, A) = (gemm(N, N, A, B))^T, exact on integers."""
    m, n, k, N = 4, 6, 5, 3
    A = inputs.draw("s", m * k * N, 31, int_valued=True)
    B = inputs.draw("s", k * n * N, 32, int_valued=True)
    ab = oracle.gemm_uniform("s", "N", "N", m, n, k, 1.0, A, m, m * k, B, k, k * n, 0.0,
                             np.zeros(m * n * N, np.float32), m, m * n, N)
    ba = oracle.gemm_uniform("s", "T", "T", n, m, k, 1.0, B, k, k * n, A, m, m * k, 0.0,
                             np.zeros(m * n * N, np.float32), n, m * n, N)
    v1 = refmath.views(ab, m, n, m, m * n, N)
    v2 = refmath.views(ba, n, m, n, m * n, N)
    assert np.array_equal(v1, np.swapaxes(v2, 1, 2))


def test_conjugate_identity():
    """gemm(C, C, B, A) = conj(gemm(N, N, A, B))^T, exact on integer parts."""
    m, n, k, N = 3, 5, 4, 3
    A = inputs.draw("c", m * k * N, 41, int_valued=True)
    B = inputs.draw("c", k * n * N, 42, int_valued=True)
    ab = oracle.gemm_uniform("c", "N", "N", m, n, k, 1.0, A, m, m * k, B, k, k * n, 0.0,
                             np.zeros(m * n * N, np.complex64), m, m * n, N)
    ba = oracle.gemm_uniform("c", "C", "C", n, m, k, 1.0, B, k, k * n, A, m, m * k, 0.0,
                             np.zeros(m * n * N, np.complex64), n, m * n, N)
    v1 = refmath.views(ab, m, n, m, m * n, N)
    v2 = refmath.views(ba, n, m, n, m * n, N)
    assert np.array_equal(np.conj(v1), np.swapaxes(v2, 1, 2))


def test_complex_from_real_decomposition():
    """Re(AB) = Ar Br - Ai Bi, Im(AB) = Ar Bi + Ai Br, with four real calls."""
    m, n, k, N = 5, 4, 6, 4
    A = inputs.draw("z", m * k * N, 51, int_valued=True)
    B = inputs.draw("z", k * n * N, 52, int_valued=True)
    z = np.zeros(m * n * N)

    def real(X, Y):
        return oracle.gemm_uniform("d", "N", "N", m, n, k, 1.0, np.ascontiguousarray(X), m,
                                   m * k, np.ascontiguousarray(Y), k, k * n, 0.0, z, m, m * n, N)

    ab = oracle.gemm_uniform("z", "N", "N", m, n, k, 1.0, A, m, m * k, B, k, k * n, 0.0,
                             np.zeros(m * n * N, np.complex128), m, m * n, N)
    re = real(A.real, B.real) - real(A.imag, B.imag)
    im = real(A.real, B.imag) + real(A.imag, B.real)
    assert np.array_equal(ab.real, re)
    assert np.array_equal(ab.imag, im)


def test_zero_imaginary_reproduces_real():
    m, n, k, N = 4, 4, 4, 3
    Ar = inputs.draw("s", m * k * N, 61)
    Br = inputs.draw("s", k * n * N, 62)
    Cr = inputs.draw("s", m * n * N, 63)
    real = oracle.gemm_uniform("s", "T", "N", m, n, k, 1.5, Ar, k, m * k, Br, k, k * n,
                               -0.5, Cr, m, m * n, N)
    cplx = oracle.gemm_uniform("c", "T", "N", m, n, k, 1.5, Ar.astype(np.complex64), k, m * k,
                               Br.astype(np.complex64), k, k * n, -0.5,
                               Cr.astype(np.complex64), m, m * n, N)
    assert np.array_equal(cplx.real, real)
    assert np.all(cplx.imag == 0)


def test_linearity_in_alpha_beta():
    b = inputs.UniformBatch("d", "N", "T", 5, 5, 5, 3, seed=71, int_valued=True)
    f = lambda a, be: run_oracle(b, a, be)
    assert np.array_equal(f(3.0, 0.0), 3.0 * f(1.0, 0.0))
    assert np.array_equal(f(1.0, 2.0) - f(1.0, 0.0), 2.0 * b.C)


def test_batch_independence_and_permutation():
    """Pair p's result does not depend on N or on the other pairs."""
    m, n, k, N = 4, 3, 5, 6
    b = inputs.UniformBatch("s", "N", "N", m, n, k, N, seed=81)
    full = blocks(b, run_oracle(b, 1.5, -0.5))
    perm = np.array([3, 0, 5, 1, 4, 2])
    Ap = b.A.reshape(N, -1)[perm].ravel()
    Bp = b.B.reshape(N, -1)[perm].ravel()
    Cp = b.C.reshape(N, -1)[perm].ravel()
    outp = oracle.gemm_uniform("s", "N", "N", m, n, k, 1.5, Ap, b.lda, b.lda2, Bp, b.ldb,
                               b.ldb2, -0.5, Cp, b.ldc, b.ldc2, N)
    assert np.array_equal(refmath.views(outp, m, n, b.ldc, b.ldc2, N), full[perm])
    one = oracle.gemm_uniform("s", "N", "N", m, n, k, 1.5, b.A[b.lda2 * 2:], b.lda, b.lda2,
                              b.B[b.ldb2 * 2:], b.ldb, b.ldb2, -0.5, b.C[b.ldc2 * 2:],
                              b.ldc, b.ldc2, 1)
    assert np.array_equal(refmath.views(one, m, n, b.ldc, b.ldc2, 1)[0], full[2])


def test_threads_do_not_change_result():
    b = inputs.UniformBatch("z", "C", "N", 7, 7, 7, 64, seed=91)
    assert np.array_equal(run_oracle(b, 1.5, -0.5, threads=1),
                          run_oracle(b, 1.5, -0.5, threads=4))


# --------------------------------------- double-double accuracy (exact ground truth)

def test_double_double_against_exact_rationals():
    """fp64 inputs: hi + lo equals the exact rational result to ~2^-100."""
    m, n, k, N = 3, 3, 16, 3
    b = inputs.UniformBatch("d", "N", "N", m, n, k, N, seed=101)
    alpha, beta = 1.5, -0.5
    hi, lo = run_oracle(b, alpha, beta, return_lo=True)
    for p in range(N):
        for i in range(m):
            for j in range(n):
                arow = [b.A[i + b.lda * l + b.lda2 * p] for l in range(k)]
                bcol = [b.B[l + b.ldb * j + b.ldb2 * p] for l in range(k)]
                exact = Fraction(alpha) * refmath.exact_dot(arow, bcol) \
                    + Fraction(beta) * Fraction(float(b.C[i + b.ldc * j + b.ldc2 * p]))
                idx = i + b.ldc * j + b.ldc2 * p
                got = Fraction(float(hi[idx])) + Fraction(float(lo[idx]))
                scale = sum(abs(Fraction(float(x)) * Fraction(float(y)))
                            for x, y in zip(arow, bcol)) + 1
                assert abs(got - exact) <= scale * Fraction(1, 2 ** 100)
                # and a plain-double sum would not be this close in general:
                assert abs(Fraction(float(hi[idx])) - exact) <= scale * Fraction(1, 2 ** 52)


def test_complex_double_double_against_exact():
    m = n = 2
    k, N = 9, 2
    b = inputs.UniformBatch("z", "C", "T", m, n, k, N, seed=103)
    alpha, beta = 1.5 - 0.5j, -0.5 + 0.25j
    hi, lo = run_oracle(b, alpha, beta, return_lo=True)
    F = lambda x: Fraction(float(x))
    for p in range(N):
        for i in range(m):
            for j in range(n):
                re, im = Fraction(0), Fraction(0)
                for l in range(k):
                    a = b.A[l + b.lda * i + b.lda2 * p]
                    bb = b.B[j + b.ldb * l + b.ldb2 * p]
                    ar, ai = F(a.real), -F(a.imag)       # conjugate transpose
                    br, bi = F(bb.real), F(bb.imag)      # transpose
                    re += ar * br - ai * bi
                    im += ar * bi + ai * br
                c = b.C[i + b.ldc * j + b.ldc2 * p]
                er = F(alpha.real) * re - F(alpha.imag) * im + F(beta.real) * F(c.real) - F(beta.imag) * F(c.imag)
                ei = F(alpha.real) * im + F(alpha.imag) * re + F(beta.real) * F(c.imag) + F(beta.imag) * F(c.real)
                idx = i + b.ldc * j + b.ldc2 * p
                gr = F(hi[idx].real) + F(lo[idx].real)
                gi = F(hi[idx].imag) + F(lo[idx].imag)
                assert abs(gr - er) <= Fraction(1, 2 ** 95)
                assert abs(gi - ei) <= Fraction(1, 2 ** 95)


# --------------------------------------------------------- 16-bit storage

@pytest.mark.parametrize("dtype", ["h", "b"])
def test_16bit_decode_exhaustive(dtype):
    """C = 1 * A * 1 with m = n = k = 1 reproduces every finite 16-bit value
    exactly (decoders written from the binary16 / bfloat16 definitions)."""
    bits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    one = np.uint16(0x3C00 if dtype == "h" else 0x3F80)
    B = np.full(bits.size, one, dtype=np.uint16)
    C = np.zeros(bits.size, dtype=np.uint16)
    out = oracle.gemm_uniform(dtype, "N", "N", 1, 1, 1, 1.0, bits, 1, 1, B, 1, 1, 0.0,
                              C, 1, 1, bits.size)
    if dtype == "h":
        ref = bits.view(np.float16).astype(np.float64)
    else:
        with np.errstate(invalid="ignore"):          # signalling NaN patterns
            ref = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    fin = np.isfinite(ref)
    assert np.array_equal(out[fin], ref[fin])
    assert np.all(np.isnan(out[np.isnan(ref)]))


def test_16bit_storage_matches_numpy():
    for dtype in "hb":
        b = inputs.UniformBatch(dtype, "T", "N", 8, 8, 8, 6, seed=111)
        out = run_oracle(b, 1.5, -0.5)
        dec = lambda x: oracle._decode16(x, dtype)
        want = refmath.numpy_gemm("d", "T", "N", 8, 8, 8, 1.5, dec(b.A), b.lda, b.lda2,
                                  dec(b.B), b.ldb, b.ldb2, -0.5, dec(b.C), b.ldc, b.ldc2, 6)
        np.testing.assert_allclose(blocks(b, out), want, rtol=1e-14, atol=1e-14)


# -------------------------------------------------------- variable size

def test_vbatch_matches_numpy_per_problem():
    desc, la, lb, lc = inputs.vbatch_problems(200, seed=5)
    desc[::3, 3] |= 1          # some opA = T
    desc[1::4, 3] |= 2 << 2    # some opB = C
    A = inputs.draw("c", la, 1)
    B = inputs.draw("c", lb, 2)
    C = inputs.draw("c", lc, 3)
    alpha, beta = 1.5 - 0.5j, 1.0
    out = oracle.gemm_vbatch("c", desc, alpha, A, B, beta, C)
    for q in range(desc.shape[0]):
        m, n, k, fl, oa, ob, oc, _ = (int(v) for v in desc[q])
        ta = "NTC"[fl & 3]
        tb = "NTC"[(fl >> 2) & 3]
        be = 0.0 if (fl >> 4) & 1 else beta
        ar, ac = (m, k) if ta == "N" else (k, m)
        br, bc = (k, n) if tb == "N" else (n, k)
        want = refmath.numpy_gemm("c", ta, tb, m, n, k, alpha, A[oa:], ar, ar * ac, B[ob:], br,
                                  br * bc, be, C[oc:], m, m * n, 1)[0]
        got = refmath.views(out[oc:], m, n, m, m * n, 1)[0]
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dtype", ["s", "d", "c", "z", "h", "b"])
def test_vbatch_every_storage_type_matches_numpy(dtype):
    """The per-type element size and decode of the variable-size oracle:
    problems at nonzero, unequal offsets in the three arenas (the arenas
    have different lengths, so a wrong element size moves every later
    problem's operands), mixed ops and beta, against numpy problem by
    problem on the decoded inputs."""
    rng = inputs.splitmix64(901, 64)
    count = 60
    shapes = [(1 + int(r % np.uint64(16)), 1 + int((r >> np.uint64(8)) % np.uint64(16)),
               1 + int((r >> np.uint64(16)) % np.uint64(16))) for r in rng[:count]]
    desc = np.zeros((count, 8), dtype=np.int64)
    oa = ob = oc = 0
    for q, (m, n, k) in enumerate(shapes):
        fl = int(rng[q] >> np.uint64(24)) % 3 | ((int(rng[q] >> np.uint64(28)) % 3) << 2)
        fl |= (q % 3 == 0) << 4
        desc[q] = (m, n, k, fl, oa + 1, ob + 2, oc + 3, 0)
        oa, ob, oc = oa + m * k + 5, ob + k * n + 7, oc + m * n + 3
    A = inputs.draw(dtype, oa + 8, 1)
    B = inputs.draw(dtype, ob + 8, 2)
    C = inputs.draw(dtype, oc + 8, 3)
    alpha, beta = ((1.5 - 0.5j, -0.5 + 0.25j) if dtype in "cz" else (1.5, -0.5))
    out = oracle.gemm_vbatch(dtype, desc, alpha, A, B, beta, C)
    dec = (lambda x: oracle._decode16(x, dtype)) if dtype in "hb" else (lambda x: x)
    Ad, Bd, Cd = dec(A), dec(B), dec(C)
    ref_t = "z" if dtype in "cz" else "d"
    covered = np.zeros(C.size, dtype=bool)
    for q in range(count):
        m, n, k, fl, pa, pb, pc, _ = (int(v) for v in desc[q])
        ta, tb = "NTC"[fl & 3], "NTC"[(fl >> 2) & 3]
        if dtype not in "cz":
            ta, tb = ta.replace("C", "T"), tb.replace("C", "T")
        be = 0.0 if (fl >> 4) & 1 else beta
        ar, ac = (m, k) if ta == "N" else (k, m)
        br, bc = (k, n) if tb == "N" else (n, k)
        Cq = Cd[pc:pc + m * n].astype(np.complex128 if dtype in "cz" else np.float64)
        if be == 0.0:
            Cq = np.full_like(Cq, np.nan)          # beta = 0: C is never read
        want = refmath.numpy_gemm(ref_t, ta, tb, m, n, k, alpha, Ad[pa:], ar, ar * ac, Bd[pb:],
                                  br, br * bc, be if be != 0.0 else 0.0,
                                  np.nan_to_num(Cq), m, m * n, 1)[0]
        got = refmath.views(out[pc:], m, n, m, m * n, 1)[0]
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
        covered[pc:pc + m * n] = True
    # entries of C no problem owns keep their old (decoded) values
    np.testing.assert_array_equal(out[~covered], Cd[~covered])


def test_vbatch_size_distribution():
    """Sizes p + 1, p in 1..15 with P(p) proportional to 1/p."""
    s = inputs.vbatch_sizes(200000, seed=0)
    assert s.min() >= 2 and s.max() <= 16
    w = 1.0 / np.arange(1, 16)
    expect = w / w.sum()
    freq = np.bincount(s - 1, minlength=16)[1:16] / s.size
    np.testing.assert_allclose(freq, expect, atol=0.004)
    assert abs(expect[0] - 0.301) < 0.001 and abs(expect[14] - 0.020) < 0.001


# ------------------------------------------------------------- footprint

def test_footprint_matches_paper():
    path = os.path.join(HERE, "golden", "footprint_sec7.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for dtype, m, n, k, N, approx, tol in rows:
        m, n, k, N = int(m), int(n), int(k), int(N)
        nbytes = inputs.ELEM_BYTES[dtype] * N * (m * k + k * n + m * n)
        assert abs(nbytes - float(approx)) <= float(tol) * float(approx)


def test_generator_is_deterministic():
    a = inputs.uniform(7, 1000)
    b = inputs.uniform(7, 1000)
    assert np.array_equal(a, b)
    assert a.min() >= -1 and a.max() < 1
    # a known SplitMix64 value (seed 0, first draw) from the published algorithm
    assert int(inputs.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF
