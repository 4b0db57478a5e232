/*
 * CPU oracle for the batched small-matrix GEMM of Jhurani & Mullowney,
 * "A GEMM interface and implementation on NVIDIA GPUs for multiple small
 * matrices" (arXiv 1304.7053).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * What it computes (Section 2, Eq. 1):
 *     C^p <- alpha * op(A^p) * op(B^p) + beta * C^p,   p = 0 .. N-1,
 * with op(X) in {X, X^T, X^*} chosen separately for A and B, C m x n,
 * op(A) m x k, op(B) k x n.  Storage follows the second-level leading
 * dimension layout of Section 4: entry (i, j) of the p-th matrix is
 * X[i + ldx*j + ldx2*p], counted in scalar elements, column-major.
 *
 * It is the plain definition: a loop over p, then i, then j, then l
 * ascending.  Every input is first converted exactly to double.  Products
 * are accumulated in double-double (error-free TwoProd via fma, TwoSum), so
 * the oracle's own rounding error is of order 2^-104 relative to
 * sum |op(A)||op(B)| and is negligible against the fp64 bound the CUDA path
 * is tested to.  The result is returned unrounded as a (hi, lo) pair of
 * doubles per real component.
 *
 * Readings of points the paper leaves open:
 *   - beta == 0 means C is never read (the a1b0 functor of Section 5 never
 *     reads y); NaN or Inf in C then cannot reach the result.
 *   - alpha == 0 or k == 0 gives C = beta*C and A, B are not read.
 *   - 'C' (conjugate transpose) on a real type is the same as 'T'.
 *   - trans characters are case-insensitive: [nN], [tT], [cC] (Section 4).
 *
 * Build with -ffp-contract=off: the double-double steps rely on every + and
 * * being rounded separately; only the explicit fma() is fused.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Scalar storage types understood by the oracle.  The 16-bit formats hold
 * raw IEEE binary16 / bfloat16 bit patterns. */
enum {
    OR_S = 0,   /* float */
    OR_D = 1,   /* double */
    OR_C = 2,   /* complex float, interleaved (re, im) */
    OR_Z = 3,   /* complex double, interleaved (re, im) */
    OR_H = 4,   /* IEEE binary16 bits */
    OR_B = 5    /* bfloat16 bits (upper half of a binary32) */
};

enum { OR_OK = 0, OR_BAD_TRANS = -1, OR_BAD_DIM = -2, OR_BAD_LD = -3, OR_BAD_TYPE = -4 };

/* ---------------- double-double arithmetic (Dekker / Knuth) ---------------- */

typedef struct { double hi, lo; } dd;

static dd two_sum(double a, double b)
{
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    dd r = { s, e };
    return r;
}

static dd quick_two_sum(double a, double b)
{
    double s = a + b;
    double e = b - (s - a);
    dd r = { s, e };
    return r;
}

static dd two_prod(double a, double b)
{
    double p = a * b;
    double e = fma(a, b, -p);
    dd r = { p, e };
    return r;
}

static dd dd_add(dd x, dd y)
{
    dd s = two_sum(x.hi, y.hi);
    dd t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

static dd dd_neg(dd x) { dd r = { -x.hi, -x.lo }; return r; }

/* dd times a plain double */
static dd dd_mul_d(dd x, double y)
{
    dd p = two_prod(x.hi, y);
    p.lo += x.lo * y;
    return quick_two_sum(p.hi, p.lo);
}

static dd dd_from(double a) { dd r = { a, 0.0 }; return r; }

/* ---------------- exact decoding of the 16-bit storage formats ---------------- */

/* IEEE 754 binary16: 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits. */
static double decode_binary16(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int e = (h >> 10) & 0x1f;
    int f = h & 0x3ff;
    double v;
    if (e == 0)
        v = ldexp((double)f, -24);                 /* subnormal: f * 2^-24 */
    else if (e == 31)
        v = f ? NAN : INFINITY;
    else
        v = ldexp((double)(1024 + f), e - 25);     /* (1 + f/2^10) * 2^(e-15) */
    return sign ? -v : v;
}

/* bfloat16: the upper 16 bits of an IEEE binary32. */
static double decode_bfloat16(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, sizeof f);
    return (double)f;
}

/* Read element `idx` (in scalar units) of a real-typed buffer as a double. */
static double load_real(int type, const void* base, long long idx)
{
    switch (type) {
    case OR_S: return (double)((const float*)base)[idx];
    case OR_D: return ((const double*)base)[idx];
    case OR_H: return decode_binary16(((const uint16_t*)base)[idx]);
    case OR_B: return decode_bfloat16(((const uint16_t*)base)[idx]);
    default:   return NAN;
    }
}

/* Read complex element `idx` (in complex-scalar units). */
static void load_cplx(int type, const void* base, long long idx, double* re, double* im)
{
    if (type == OR_C) {
        const float* p = (const float*)base + 2 * idx;
        *re = (double)p[0];
        *im = (double)p[1];
    } else {
        const double* p = (const double*)base + 2 * idx;
        *re = p[0];
        *im = p[1];
    }
}

static int is_complex(int type) { return type == OR_C || type == OR_Z; }

/* op code: 0 = N, 1 = T, 2 = C (conjugate transpose); -1 = invalid. */
static int op_code(char t)
{
    switch (t) {
    case 'n': case 'N': return 0;
    case 't': case 'T': return 1;
    case 'c': case 'C': return 2;
    default: return -1;
    }
}

/* Offset (scalar units) of op(X)(r, c) of matrix p, for X stored column-major
 * with leading dimensions ld, ld2 (Section 4 layout, Section 2 op). */
static long long op_index(int op, long long r, long long c, long long ld, long long ld2, long long p)
{
    return op == 0 ? r + ld * c + ld2 * p    /* op(X) = X:  X(r, c)          */
                   : c + ld * r + ld2 * p;   /* op(X) = X^T or X^*: X(c, r)  */
}

/*
 * Argument checks, stated by the layout of Section 4 (Fig. "LD2": ldc >= m,
 * ldc2 >= ldc*n) and the dimensions of Section 2.  Returns OR_OK or a code.
 */
int oracle_check_args(char transa, char transb, int m, int n, int k,
                      long long lda, long long lda2, long long ldb, long long ldb2,
                      long long ldc, long long ldc2, long long batch)
{
    int opa = op_code(transa), opb = op_code(transb);
    if (opa < 0 || opb < 0) return OR_BAD_TRANS;
    if (m < 0 || n < 0 || k < 0 || batch < 0) return OR_BAD_DIM;
    long long ar = opa == 0 ? m : k, ac = opa == 0 ? k : m;   /* stored A rows, cols */
    long long br = opb == 0 ? k : n, bc = opb == 0 ? n : k;   /* stored B rows, cols */
    if (lda < (ar > 1 ? ar : 1) || ldb < (br > 1 ? br : 1) || ldc < (m > 1 ? m : 1))
        return OR_BAD_LD;
    if (lda2 != 0 && lda2 < lda * ac) return OR_BAD_LD;
    if (ldb2 != 0 && ldb2 < ldb * bc) return OR_BAD_LD;
    if (ldc2 < ldc * n) return OR_BAD_LD;
    return OR_OK;
}

/*
 * Eq. (1) for one pair p.  alpha, beta are (re, im) doubles; for real types
 * only [0] is used.  out_hi / out_lo have C's layout (for complex: two
 * doubles per element, interleaved re, im); only the m x n entries of
 * matrix p are written.
 */
static void gemm_one(int type, int opa, int opb, int m, int n, int k,
                     const double* alpha, const void* A, long long lda, long long lda2,
                     const void* B, long long ldb, long long ldb2,
                     const double* beta, const void* C, long long ldc, long long ldc2,
                     long long p, double* out_hi, double* out_lo)
{
    const int cplx = is_complex(type);
    const int skip_ab = (k == 0) || (alpha[0] == 0.0 && (!cplx || alpha[1] == 0.0));
    const int read_c = !(beta[0] == 0.0 && (!cplx || beta[1] == 0.0));

    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < n; ++j) {
            long long ci = i + ldc * j + ldc2 * p;
            if (!cplx) {
                dd acc = dd_from(0.0);
                if (!skip_ab) {
                    for (int l = 0; l < k; ++l) {
                        double a = load_real(type, A, op_index(opa, i, l, lda, lda2, p));
                        double b = load_real(type, B, op_index(opb, l, j, ldb, ldb2, p));
                        acc = dd_add(acc, two_prod(a, b));
                    }
                }
                dd r = dd_mul_d(acc, alpha[0]);
                if (skip_ab) r = dd_from(0.0);
                if (read_c)
                    r = dd_add(r, two_prod(beta[0], load_real(type, C, ci)));
                out_hi[ci] = r.hi;
                out_lo[ci] = r.lo;
            } else {
                dd re = dd_from(0.0), im = dd_from(0.0);
                if (!skip_ab) {
                    for (int l = 0; l < k; ++l) {
                        double ar, ai, br, bi;
                        load_cplx(type, A, op_index(opa, i, l, lda, lda2, p), &ar, &ai);
                        load_cplx(type, B, op_index(opb, l, j, ldb, ldb2, p), &br, &bi);
                        if (opa == 2) ai = -ai;   /* conjugate: {a.x, -a.y} (Section 5) */
                        if (opb == 2) bi = -bi;
                        /* (ar + i ai)(br + i bi) = (ar br - ai bi) + i (ar bi + ai br) */
                        re = dd_add(re, two_prod(ar, br));
                        re = dd_add(re, dd_neg(two_prod(ai, bi)));
                        im = dd_add(im, two_prod(ar, bi));
                        im = dd_add(im, two_prod(ai, br));
                    }
                }
                /* alpha * acc */
                dd rr = dd_add(dd_mul_d(re, alpha[0]), dd_neg(dd_mul_d(im, alpha[1])));
                dd ri = dd_add(dd_mul_d(im, alpha[0]), dd_mul_d(re, alpha[1]));
                if (skip_ab) { rr = dd_from(0.0); ri = dd_from(0.0); }
                if (read_c) {
                    double cr, cim;
                    load_cplx(type, C, ci, &cr, &cim);
                    rr = dd_add(rr, two_prod(beta[0], cr));
                    rr = dd_add(rr, dd_neg(two_prod(beta[1], cim)));
                    ri = dd_add(ri, two_prod(beta[0], cim));
                    ri = dd_add(ri, two_prod(beta[1], cr));
                }
                out_hi[2 * ci] = rr.hi;
                out_lo[2 * ci] = rr.lo;
                out_hi[2 * ci + 1] = ri.hi;
                out_lo[2 * ci + 1] = ri.lo;
            }
        }
    }
}

/*
 * The whole batch, Eq. (1) for p = 0 .. batch-1, on the uniform 3-D layout
 * of Section 4.  `type` is one of OR_S .. OR_B; C has the same storage type
 * as A and B.  Returns OR_OK or an argument error; on error nothing is
 * written.  `threads` > 1 runs independent pairs on OpenMP threads (the
 * pairs are independent, Section 2); the result does not depend on it.
 */
int oracle_gemm_uniform(int type, char transa, char transb, int m, int n, int k,
                        const double* alpha, const void* A, long long lda, long long lda2,
                        const void* B, long long ldb, long long ldb2,
                        const double* beta, const void* C, long long ldc, long long ldc2,
                        long long batch, double* out_hi, double* out_lo, int threads)
{
    if (type < OR_S || type > OR_B) return OR_BAD_TYPE;
    int st = oracle_check_args(transa, transb, m, n, k, lda, lda2, ldb, ldb2, ldc, ldc2, batch);
    if (st != OR_OK) return st;
    int opa = op_code(transa), opb = op_code(transb);
    if (!is_complex(type)) {            /* 'C' on a real type is 'T' */
        if (opa == 2) opa = 1;
        if (opb == 2) opb = 1;
    }
#ifdef _OPENMP
    if (threads < 1) threads = 1;
    #pragma omp parallel for schedule(static) num_threads(threads)
#endif
    for (long long p = 0; p < batch; ++p)
        gemm_one(type, opa, opb, m, n, k, alpha, A, lda, lda2, B, ldb, ldb2,
                 beta, C, ldc, ldc2, p, out_hi, out_lo);
    (void)threads;
    return OR_OK;
}

/*
 * Variable-size batch: problem q has its own (m, n, k, opA, opB) and its own
 * offsets into three arenas, minimal leading dimensions (rows of the stored
 * matrix), and uses beta_q = 0 when its beta-zero flag is set, else the
 * call's beta.  This is Eq. (1) applied problem by problem; the paper's
 * remark that differently sized matrices can be partitioned into sets of
 * identical size (Section 1) is what the GPU path does with it.
 *
 * desc is an array of `count` records of 8 int64 each:
 *   m, n, k, flags, offA, offB, offC, reserved
 * flags: bits 0-1 opA (0 N, 1 T, 2 C), bits 2-3 opB, bit 4 beta-zero.
 * Output arrays have the C arena's layout.
 */
int oracle_gemm_vbatch(int type, const long long* desc, long long count,
                       const double* alpha, const void* A, const void* B,
                       const double* beta, const void* C,
                       double* out_hi, double* out_lo, int threads)
{
    if (type < OR_S || type > OR_B) return OR_BAD_TYPE;
    for (long long q = 0; q < count; ++q) {
        const long long* d = desc + 8 * q;
        if (d[0] < 0 || d[1] < 0 || d[2] < 0 || d[0] > 16 || d[1] > 16 || d[2] > 16) return OR_BAD_DIM;
        if ((d[3] & 3) == 3 || ((d[3] >> 2) & 3) == 3) return OR_BAD_TRANS;
    }
    const double zero[2] = { 0.0, 0.0 };
#ifdef _OPENMP
    if (threads < 1) threads = 1;
    #pragma omp parallel for schedule(dynamic, 256) num_threads(threads)
#endif
    for (long long q = 0; q < count; ++q) {
        const long long* d = desc + 8 * q;
        int m = (int)d[0], n = (int)d[1], k = (int)d[2];
        int opa = (int)(d[3] & 3), opb = (int)((d[3] >> 2) & 3);
        int beta_zero = (int)((d[3] >> 4) & 1);
        if (!is_complex(type)) {
            if (opa == 2) opa = 1;
            if (opb == 2) opb = 1;
        }
        long long lda = opa == 0 ? m : k, ldb = opb == 0 ? k : n, ldc = m;
        if (lda < 1) lda = 1;
        if (ldb < 1) ldb = 1;
        if (ldc < 1) ldc = 1;
        /* offsets in scalar units; for complex types, in complex units */
        size_t es = (type == OR_S) ? 4 : (type == OR_D || type == OR_C) ? 8 : (type == OR_Z) ? 16 : 2;
        const char* a = (const char*)A + es * (size_t)d[4];
        const char* b = (const char*)B + es * (size_t)d[5];
        const char* c = (const char*)C + es * (size_t)d[6];
        size_t oc = (size_t)d[6] * (is_complex(type) ? 2 : 1);
        gemm_one(type, opa, opb, m, n, k, alpha, a, lda, 0, b, ldb, 0,
                 beta_zero ? zero : beta, c, ldc, 0, 0, out_hi + oc, out_lo + oc);
    }
    (void)threads;
    return OR_OK;
}

/* Number of OpenMP threads the oracle would use by default (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
