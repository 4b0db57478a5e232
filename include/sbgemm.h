/*
 * sbgemm — batched GEMM for many small matrices on NVIDIA GB300 (sm_103a).
 *
 * Computes, for p = 0 .. batchCount-1 independently (arXiv 1304.7053,
 * Section 2, Eq. 1):
 *
 *     C_p <- alpha * op(A_p) * op(B_p) + beta * C_p
 *
 * with op(X) one of X, X^T, X^* selected by a trans character, C_p m x n,
 * op(A_p) m x k, op(B_p) k x n, and 0 <= m, n, k <= 16.
 *
 * Storage (Section 4): every operand is one 3-D array addressed through a
 * second-level leading dimension.  Entry (i, j) of the p-th matrix X is
 * X[i + ldx*j + ldx2*p]; all leading dimensions are counted in scalar
 * elements (complex elements for the complex types), column-major.
 *
 * Conventions shared by every entry point:
 *   - transa / transb: 'N'/'n' (op(X) = X), 'T'/'t' (X^T), 'C'/'c' (X^*).
 *     For real types 'C' is the same as 'T'.
 *   - Stored A is m x k for 'N' and k x m otherwise; stored B is k x n for
 *     'N' and n x k otherwise.  lda >= max(1, rows of stored A),
 *     ldb >= max(1, rows of stored B), ldc >= max(1, m).
 *     lda2 >= lda * cols(stored A) or lda2 == 0 (every pair uses the same A);
 *     ldb2 likewise; ldc2 >= ldc * n so the C matrices never overlap
 *     (Section 4, Fig. LD2).
 *   - beta == 0: C is only written, never read, so NaN or Inf in C does not
 *     reach the result (the a1b0 functor of Section 5 never reads y).
 *     alpha == 0 or k == 0: C = beta * C and A, B are not read.
 *     batchCount == 0, m == 0 or n == 0: nothing is done.
 *   - Ownership: all matrix pointers are device memory owned by the caller;
 *     these calls allocate nothing.  Calls are asynchronous with respect to
 *     the host and ordered on the given stream.
 *   - Return value: SBGEMM_SUCCESS (0); a negative SBGEMM_ERR_* code for a
 *     rejected argument (nothing is launched); or a positive cudaError_t
 *     value reported by the CUDA runtime at launch.  No C++ exception
 *     crosses this interface.
 *   - Results: rounded to the storage type once at the end; products are
 *     accumulated in the storage precision (fp32 for S/C and the 16-bit
 *     types, fp64 for D/Z) with fused multiply-adds.
 */
#ifndef SBGEMM_H
#define SBGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int sbgemm_status;

enum {
    SBGEMM_SUCCESS = 0,
    SBGEMM_ERR_INVALID_TRANS = -1,  /* trans character not in [nNtTcC] */
    SBGEMM_ERR_INVALID_SIZE = -2,   /* m, n or k outside 0..16, or batchCount < 0 */
    SBGEMM_ERR_INVALID_LD = -3,     /* a leading dimension below its minimum */
    SBGEMM_ERR_NULL_POINTER = -4,   /* a required pointer is NULL */
    SBGEMM_ERR_INVALID_VALUE = -5,  /* other invalid argument (mode, variant, plan) */
    SBGEMM_ERR_TIMEOUT = -6,        /* a bounded in-kernel wait gave up */
    SBGEMM_ERR_NOT_SUPPORTED = -7,  /* valid request this build cannot serve */
    SBGEMM_ERR_CAPACITY = -8        /* request exceeds a fixed capacity */
};

/* Where alpha and beta live (Section 4: "host or device pointer"). */
enum {
    SBGEMM_SCALARS_HOST = 0,    /* read on the host at call time */
    SBGEMM_SCALARS_DEVICE = 1   /* read by the kernel from device memory */
};

typedef struct { float x, y; } sbgemm_c32;   /* same layout as cuComplex */
typedef struct { double x, y; } sbgemm_c64;  /* same layout as cuDoubleComplex */

/* ------------------------------------------------------------------ */
/* Fixed-size batches on the uniform 3-D layout (Section 4 interface). */
/* ------------------------------------------------------------------ */

/*
 * The paper's interface, TGEMM_multi_uniform of Section 4, one per type
 * T = S (float), D (double), C (complex float), Z (complex double).
 * alpha and beta are host pointers; the work is queued on the legacy
 * default stream and the call returns without waiting for it.
 */
sbgemm_status sbgemm_Sgemm_multi_uniform(char transa, char transb, int m, int n, int k,
    const float* alpha, const float* A, int lda, long long lda2,
    const float* B, int ldb, long long ldb2,
    const float* beta, float* C, int ldc, long long ldc2, int batchCount);
sbgemm_status sbgemm_Dgemm_multi_uniform(char transa, char transb, int m, int n, int k,
    const double* alpha, const double* A, int lda, long long lda2,
    const double* B, int ldb, long long ldb2,
    const double* beta, double* C, int ldc, long long ldc2, int batchCount);
sbgemm_status sbgemm_Cgemm_multi_uniform(char transa, char transb, int m, int n, int k,
    const sbgemm_c32* alpha, const sbgemm_c32* A, int lda, long long lda2,
    const sbgemm_c32* B, int ldb, long long ldb2,
    const sbgemm_c32* beta, sbgemm_c32* C, int ldc, long long ldc2, int batchCount);
sbgemm_status sbgemm_Zgemm_multi_uniform(char transa, char transb, int m, int n, int k,
    const sbgemm_c64* alpha, const sbgemm_c64* A, int lda, long long lda2,
    const sbgemm_c64* B, int ldb, long long ldb2,
    const sbgemm_c64* beta, sbgemm_c64* C, int ldc, long long ldc2, int batchCount);

/*
 * Same operation on an explicit stream (a cudaStream_t passed as void*;
 * NULL is the legacy default stream).  scalar_mode says whether alpha and
 * beta are host or device pointers (SBGEMM_SCALARS_*).  With device
 * scalars the kernel itself tests beta == 0 and then does not read C.
 */
sbgemm_status sbgemm_Sgemm_multi_uniform_async(char transa, char transb, int m, int n, int k,
    const float* alpha, const float* A, int lda, long long lda2,
    const float* B, int ldb, long long ldb2,
    const float* beta, float* C, int ldc, long long ldc2, int batchCount,
    int scalar_mode, void* stream);
sbgemm_status sbgemm_Dgemm_multi_uniform_async(char transa, char transb, int m, int n, int k,
    const double* alpha, const double* A, int lda, long long lda2,
    const double* B, int ldb, long long ldb2,
    const double* beta, double* C, int ldc, long long ldc2, int batchCount,
    int scalar_mode, void* stream);
sbgemm_status sbgemm_Cgemm_multi_uniform_async(char transa, char transb, int m, int n, int k,
    const sbgemm_c32* alpha, const sbgemm_c32* A, int lda, long long lda2,
    const sbgemm_c32* B, int ldb, long long ldb2,
    const sbgemm_c32* beta, sbgemm_c32* C, int ldc, long long ldc2, int batchCount,
    int scalar_mode, void* stream);
sbgemm_status sbgemm_Zgemm_multi_uniform_async(char transa, char transb, int m, int n, int k,
    const sbgemm_c64* alpha, const sbgemm_c64* A, int lda, long long lda2,
    const sbgemm_c64* B, int ldb, long long ldb2,
    const sbgemm_c64* beta, sbgemm_c64* C, int ldc, long long ldc2, int batchCount,
    int scalar_mode, void* stream);

/*
 * 16-bit storage with fp32 arithmetic: A, B and C hold IEEE binary16 (H) or
 * bfloat16 (B) bit patterns; alpha and beta are fp32; products accumulate
 * in fp32 and the result is rounded to the 16-bit format (nearest-even) on
 * store.  Eq. (1) with the storage precision of the operands halved.
 */
sbgemm_status sbgemm_Hgemm_multi_uniform_async(char transa, char transb, int m, int n, int k,
    const float* alpha, const uint16_t* A, int lda, long long lda2,
    const uint16_t* B, int ldb, long long ldb2,
    const float* beta, uint16_t* C, int ldc, long long ldc2, int batchCount,
    int scalar_mode, void* stream);
sbgemm_status sbgemm_Bgemm_multi_uniform_async(char transa, char transb, int m, int n, int k,
    const float* alpha, const uint16_t* A, int lda, long long lda2,
    const uint16_t* B, int ldb, long long ldb2,
    const float* beta, uint16_t* C, int ldc, long long ldc2, int batchCount,
    int scalar_mode, void* stream);

/* ------------------------------------------------------------------ */
/* Kernel variants (used by the autotuner and the learned selector).   */
/* ------------------------------------------------------------------ */

/*
 * Type codes for the variant, tuning and planning calls below.
 */
enum { SBGEMM_TYPE_S = 0, SBGEMM_TYPE_D = 1, SBGEMM_TYPE_C = 2, SBGEMM_TYPE_Z = 3,
       SBGEMM_TYPE_H = 4, SBGEMM_TYPE_B = 5 };

/* Number of kernel variants a (type, m, n, k) problem can run with; variant
 * 0 is always the default choice.  Returns 0 for an invalid request. */
int sbgemm_num_variants(int type, int m, int n, int k);

/* Human-readable description of a variant (static storage, never NULL). */
const char* sbgemm_variant_name(int type, int m, int n, int k, int variant);

/*
 * Eq. (1) with an explicitly chosen kernel variant (0 .. num_variants-1);
 * otherwise identical to the _async entry points (type-erased pointers:
 * alpha/beta point to one scalar of the type; fp32 for H and B).
 * A variant index out of range gives SBGEMM_ERR_INVALID_VALUE.
 */
sbgemm_status sbgemm_gemm_multi_uniform_variant(int type, char transa, char transb,
    int m, int n, int k, const void* alpha, const void* A, int lda, long long lda2,
    const void* B, int ldb, long long ldb2, const void* beta, void* C, int ldc,
    long long ldc2, int batchCount, int scalar_mode, int variant, void* stream);

/*
 * Selection table: the variant the _async entry points use for
 * (type, m, n, k, opA-transposed, opB-transposed, beta == 0, batch-size
 * class).  sbgemm_set_choice installs one entry (variant < 0 removes it);
 * sbgemm_get_choice returns the installed or default variant.  The table is
 * process-wide host state; set it before issuing work, not concurrently with
 * calls that read it.  size_class = floor(log10(batchCount)) clamped to 0..7.
 */
sbgemm_status sbgemm_set_choice(int type, int m, int n, int k, int ta, int tb,
                                int beta_zero, int size_class, int variant);
int sbgemm_get_choice(int type, int m, int n, int k, int ta, int tb,
                      int beta_zero, int size_class);
void sbgemm_clear_choices(void);

/* ------------------------------------------------------------------ */
/* Status and device fault word.                                        */
/* ------------------------------------------------------------------ */

/* Static description of a status code (never NULL). */
const char* sbgemm_status_string(sbgemm_status status);

/* Library version as major*10000 + minor*100 + patch. */
int sbgemm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SBGEMM_H */
