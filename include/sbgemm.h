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
    SBGEMM_ERR_CAPACITY = -8,       /* request exceeds a fixed capacity */
    SBGEMM_ERR_IO = -9              /* a file cannot be read or written, or has a bad format */
};

/* Where alpha and beta live (Section 4: "host or device pointer"). */
enum {
    SBGEMM_SCALARS_HOST = 0,    /* read on the host at call time */
    SBGEMM_SCALARS_DEVICE = 1   /* read by the kernel from device memory */
};

/* Type codes for the type-erased calls (variants, host arrays, plans). */
enum { SBGEMM_TYPE_S = 0, SBGEMM_TYPE_D = 1, SBGEMM_TYPE_C = 2, SBGEMM_TYPE_Z = 3,
       SBGEMM_TYPE_H = 4, SBGEMM_TYPE_B = 5 };

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

/*
 * Eq. (1) on HOST arrays (pinned memory gives overlapped copies; pageable
 * memory works but serialises).  The batch streams through the caller's
 * device work buffer `dwork` (dwork_bytes, at least two pairs' worth of A,
 * B and C) in chunks, double-buffered: host->device copies, kernels (on
 * `stream`) and device->host copies of consecutive chunks overlap on two
 * internal streams.  The call is ordered after earlier work on `stream` and
 * later work on `stream` waits for the last copy back; it returns before the
 * copies finish (synchronise the stream before reading hC).  Host scalars
 * only; lda2 and ldb2 must be nonzero.  C is copied in when beta != 0 or
 * when its layout has gaps.  Allocates nothing; SBGEMM_ERR_CAPACITY when
 * half of dwork cannot hold one pair.  Calls that share dwork must be
 * ordered.
 */
sbgemm_status sbgemm_gemm_multi_uniform_host(int type, char transa, char transb,
    int m, int n, int k, const void* alpha, const void* hA, int lda, long long lda2,
    const void* hB, int ldb, long long ldb2, const void* beta, void* hC, int ldc,
    long long ldc2, int batchCount, void* dwork, size_t dwork_bytes, void* stream);

/* One uniform batch on host arrays, for sbgemm_gemm_grouped_host. */
typedef struct {
    char transa, transb;
    int m, n, k;
    const void* hA; int lda; long long lda2;
    const void* hB; int ldb; long long ldb2;
    void* hC; int ldc; long long ldc2;
    int batchCount;
} sbgemm_host_group;

/*
 * Several uniform batches on host arrays (same type, alpha and beta) as one
 * continuous pipeline through `dwork`: the copy-back of one group overlaps
 * the copy-in of the next, which separate sbgemm_gemm_multi_uniform_host
 * calls cannot do (each is ordered after the previous one's last copy).
 * Same rules as sbgemm_gemm_multi_uniform_host; every group is checked
 * before anything is queued; SBGEMM_ERR_CAPACITY when half of dwork cannot
 * hold one pair of some group.
 */
sbgemm_status sbgemm_gemm_grouped_host(int type, const void* alpha, const void* beta,
    const sbgemm_host_group* groups, int ngroups, void* dwork, size_t dwork_bytes, void* stream);

/* One uniform batch on device arrays, for sbgemm_gemm_grouped. */
typedef struct {
    char transa, transb;
    int m, n, k;
    const void* A; int lda; long long lda2;
    const void* B; int ldb; long long ldb2;
    void* C; int ldc; long long ldc2;
    int batchCount;
} sbgemm_group;

/*
 * Several independent uniform batches (same type, alpha and beta) in one
 * call.  Groups that are square (m = n = k <= 16), op N/N, stored with
 * minimal leading dimensions and 16-byte aligned share ONE persistent
 * launch (up to 32 per launch): their tiles interleave, so small groups cost
 * no launch of their own.  Other groups, and fp64 / complex128 groups whose
 * class the selector sends to the tensor-core variant (large sizes), run as
 * separate uniform calls on the same stream.  No group may read another
 * group's C (they run
 * concurrently).  Every group is checked before anything is queued; the
 * return value is that of the first failing check or launch.
 */
sbgemm_status sbgemm_gemm_grouped(int type, const void* alpha, const void* beta,
                                  const sbgemm_group* groups, int ngroups,
                                  int scalar_mode, void* stream);

/*
 * Launch configuration of the shared persistent launch of
 * sbgemm_gemm_grouped for one storage type: threads per block (128 or 256),
 * bytes of one pipeline stage (4096..65536, a multiple of 1024) and pipeline
 * depth (2..4); the block's shared memory is stages*stage_bytes +
 * stage_bytes/2 and must stay within 220 KB.  All three zero restores the
 * default (128, 28672, 2).  Process-wide; not synchronised with calls
 * running concurrently on other host threads.  Invalid values give
 * SBGEMM_ERR_INVALID_VALUE and leave the configuration unchanged.
 */
sbgemm_status sbgemm_grouped_config(int type, int threads, int stage_bytes, int stages);

/* ------------------------------------------------------------------ */
/* Pointer-array form (Section 4, TGEMM_multi_nounif).                 */
/* ------------------------------------------------------------------ */

/*
 * The same product with the batch given as arrays of matrix pointers, the
 * cuBLAS batched interface the paper compares against (Section 4 and the
 * cuBLAS comparison of Section 7): matrix p of A is Aarray[p], with entry
 * (i, j) at Aarray[p][i + lda*j]; likewise B and C.  Aarray, Barray and
 * Carray are DEVICE arrays of batchCount device pointers, owned by the
 * caller and read by the kernel.  A and B pointers may repeat; the C
 * matrices must not overlap one another or any A or B.  Every matrix
 * pointer is aligned to the element size (16 bytes for complex double);
 * a matrix with ld equal to its row count that starts 16-byte aligned is
 * moved in 16-byte chunks, anything else element by element.  Leading
 * dimensions, trans characters, degenerate cases, scalars and return
 * values as for the uniform calls (ld2 does not exist here).  The typed
 * calls take host scalars and use the legacy default stream; the
 * type-erased call takes a scalar mode and a stream (fp32 scalars for the
 * 16-bit types).
 */
sbgemm_status sbgemm_Sgemm_multi_nounif(char transa, char transb, int m, int n, int k,
    const float* alpha, const float* const* Aarray, int lda, const float* const* Barray, int ldb,
    const float* beta, float* const* Carray, int ldc, int batchCount);
sbgemm_status sbgemm_Dgemm_multi_nounif(char transa, char transb, int m, int n, int k,
    const double* alpha, const double* const* Aarray, int lda, const double* const* Barray,
    int ldb, const double* beta, double* const* Carray, int ldc, int batchCount);
sbgemm_status sbgemm_Cgemm_multi_nounif(char transa, char transb, int m, int n, int k,
    const sbgemm_c32* alpha, const sbgemm_c32* const* Aarray, int lda,
    const sbgemm_c32* const* Barray, int ldb, const sbgemm_c32* beta,
    sbgemm_c32* const* Carray, int ldc, int batchCount);
sbgemm_status sbgemm_Zgemm_multi_nounif(char transa, char transb, int m, int n, int k,
    const sbgemm_c64* alpha, const sbgemm_c64* const* Aarray, int lda,
    const sbgemm_c64* const* Barray, int ldb, const sbgemm_c64* beta,
    sbgemm_c64* const* Carray, int ldc, int batchCount);
sbgemm_status sbgemm_gemm_multi_nounif(int type, char transa, char transb, int m, int n, int k,
    const void* alpha, const void* const* Aarray, int lda, const void* const* Barray, int ldb,
    const void* beta, void* const* Carray, int ldc, int batchCount, int scalar_mode,
    void* stream);

/* ------------------------------------------------------------------ */
/* Kernel variants (used by the autotuner and the learned selector).   */
/* ------------------------------------------------------------------ */

/* Number of kernel variants a (type, m, n, k) problem can run with (0 for
 * an invalid request).  Shapes with specialised kernels have six settings of
 * the pipelined kernel (0..5) and the generic kernel (6); the 16-bit types at
 * m = n = k = 8, 12, 16 and real and complex fp64 add variant 7, the
 * tensor-core kernel (for fp64 and complex128: operands split into exact
 * 8-bit digits whose products run on the binary16 MMA path, recombined
 * exactly; entries whose accuracy the split cannot guarantee are recomputed
 * with fp64 FMAs).  Other shapes have the generic kernel as variant 0 and,
 * for real and complex fp64 only, the same tensor-core kernel as
 * variant 1. */
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
 * Variant selection (the tunable launch configuration and specialised
 * kernels of Section 6).  Every fixed-size call (uniform and pointer-array
 * forms) runs the variant chosen for its class (type, m, n, k,
 * opA-transposed, opB-transposed, beta == 0, batch-size class), where
 * size_class = floor(log10(batchCount)) clamped to 0..7 and beta == 0 is
 * known only for host scalars (device scalars count as beta != 0).  The
 * choice depends on the selector mode:
 *   SBGEMM_SELECTOR_DEFAULT: the built-in rule only;
 *   SBGEMM_SELECTOR_TABLE (initial mode): the selection table's entry for
 *     the class, else the built-in rule;
 *   SBGEMM_SELECTOR_MODEL: the table's entry, else the installed cost
 *     model's choice, else the built-in rule.
 * Built-in rule: the tensor-core variant (7) for the 16-bit types at
 * m = n = k = 8, 12 and 16, for real fp64 at m = n = k >= 13, at 12 with
 * beta != 0 and at 16 x 8 x 16, and for complex128 at m = n = k >= 12 and
 * at 16 x 8 x 16; on real and complex fp64 shapes without specialised
 * kernels the tensor-core variant (1) from m n k = 1024 (real fp64 with
 * beta != 0: 1320); variant 2 for complex64, and for fp32 with
 * size_class <= 5; variant 0 otherwise.
 * All of this is process-wide host state: set it before issuing work, not
 * concurrently with calls that read it.
 *
 * Environment, read once before the first selection or selector call:
 * SBGEMM_TABLE (a table file to load), SBGEMM_COST_MODEL (a cost-model
 * file to load) and SBGEMM_SELECTOR (default, table or model).  A failure
 * is not fatal: the affected setting keeps its initial value and
 * sbgemm_get_selector reports the first error.
 */
enum { SBGEMM_SELECTOR_DEFAULT = 0, SBGEMM_SELECTOR_TABLE = 1, SBGEMM_SELECTOR_MODEL = 2 };

/* Install one table entry (variant < 0 removes it). */
sbgemm_status sbgemm_set_choice(int type, int m, int n, int k, int ta, int tb,
                                int beta_zero, int size_class, int variant);
/* The variant a call of this class would run under the current mode
 * (-1 for an invalid class). */
int sbgemm_get_choice(int type, int m, int n, int k, int ta, int tb,
                      int beta_zero, int size_class);
/* The built-in rule's variant for the class (-1 for an invalid class). */
int sbgemm_default_variant(int type, int m, int n, int k, int beta_zero, int size_class);
void sbgemm_clear_choices(void);
/* The public variant index the calling thread's most recent fixed-size
 * call ran (-1 before any); for checking which kernel a selection reached. */
int sbgemm_last_variant(void);

/*
 * Table files (text): a line "sbgemm-table 1", a line "device <name>"
 * (the GPU the table was measured on, informational), then one line per
 * entry "type m n k ta tb beta_zero size_class variant"; '#' starts a
 * comment line.  Saving writes the whole table (through a temporary file
 * renamed into place).  Loading validates every line first and then adds
 * the entries to the table (an entry for a class already present replaces
 * it); on any error nothing is added.  SBGEMM_ERR_IO for an unreadable,
 * unwritable or malformed file.
 */
sbgemm_status sbgemm_save_table(const char* path);
sbgemm_status sbgemm_load_table(const char* path);

/* Selector mode (SBGEMM_SELECTOR_*).  MODEL needs an installed cost model
 * (else SBGEMM_ERR_INVALID_VALUE) and evaluates it first if needed (see
 * sbgemm_set_cost_model); the mode is unchanged on any error. */
sbgemm_status sbgemm_set_selector(int mode);
/* Current mode, and the first error met while applying the environment
 * settings (0 when none; env_status may be NULL). */
sbgemm_status sbgemm_get_selector(int* mode, int* env_status);

/*
 * Cost model of the selector: a network of the sbgemm_mlp_* layout with
 * F = 16 inputs (the class features: m, n, k / 16; (log10 N - 4.5) / 1.5
 * at the middle of the size class; the storage-type one-hot in type-code
 * order; opA and opB transposed; conjugation (0); beta == 0; a flag for
 * shapes with specialised kernels; (mnk)^(1/3) / 16), H hidden units and
 * V outputs, output v the standardised log-time of variant v: predicted
 * time = exp(y_v * log_time_std + log_time_mean) (only ratios between the
 * variants of one class are used, so the outputs may be log-times relative
 * to any per-class reference).  For each class with more than one variant
 * the model's choice is the valid variant with the smallest prediction if
 * that is below (1 - margins[type]) times the prediction of the built-in
 * rule's variant, else the built-in rule's variant: `margins` holds one
 * trust margin per storage type, indexed by type code (SBGEMM_TYPE_S ..
 * SBGEMM_TYPE_B), each in [0, 1]; 1 keeps the built-in rule for that type.
 * sbgemm_set_cost_model copies `params` (host array of
 * sbgemm_mlp_param_count(F, H, V) floats) and replaces any installed model.
 * The choices of every class are evaluated at once, on the current GPU,
 * with sbgemm_mlp_forward (device memory allocated and freed for it, the
 * call synchronises): right away when the mode is MODEL, else when the
 * mode becomes MODEL, or at the first call that needs them when the model
 * and mode come from the environment; make that first call outside any
 * stream capture.  F must be 16, 1 <= H <= 4096, 1 <= V <= 64,
 * log_time_std > 0, every margin in [0, 1] (else SBGEMM_ERR_INVALID_VALUE);
 * params or margins NULL: SBGEMM_ERR_NULL_POINTER.
 */
sbgemm_status sbgemm_set_cost_model(int F, int H, int V, const float* params,
                                    double log_time_mean, double log_time_std,
                                    const double* margins);
/*
 * Cost-model files (text, version 2): "sbgemm-cost-model 2", "device
 * <name>" (the GPU it was trained on), "features F hidden H outputs V",
 * "log_time_mean mu log_time_std sd", "margins m_S m_D m_C m_Z m_H m_B",
 * "params n", then the n parameters (9 significant digits, exact for
 * fp32).  Version 1 files (one "margin m" for every type after the
 * log-time line) still load.  Loading installs the
 * model as sbgemm_set_cost_model does; SBGEMM_ERR_IO for an unreadable or
 * malformed file; SBGEMM_ERR_INVALID_VALUE from sbgemm_save_cost_model when
 * no model is installed.
 */
sbgemm_status sbgemm_save_cost_model(const char* path);
sbgemm_status sbgemm_load_cost_model(const char* path);

/*
 * The autotuner's exhaustive step for one class, natively: times every
 * variant of the request with sbgemm_time_variant (host scalars; `reps`,
 * `flush`, `flush_bytes` and `stream` as there), writes the times to ms[v]
 * when ms is not NULL (sbgemm_num_variants entries), the fastest variant to
 * *best, and installs it in the selection table for the request's class.
 * C is overwritten by the timed calls.  Synchronises the stream.
 */
sbgemm_status sbgemm_tune(int type, char transa, char transb, int m, int n, int k,
    const void* alpha, const void* A, int lda, long long lda2,
    const void* B, int ldb, long long ldb2, const void* beta, void* C, int ldc,
    long long ldc2, int batchCount, int reps, void* flush, size_t flush_bytes, void* stream,
    int* best, float* ms);

/* ------------------------------------------------------------------ */
/* Variable-size batches (Section 1: matrices of different sizes are     */
/* partitioned into sets of identical size; here one persistent launch). */
/* ------------------------------------------------------------------ */

/*
 * One problem of a variable-size batch: Eq. (1) for C_q = alpha op(A_q)
 * op(B_q) + beta_q C_q with 0 <= m, n, k <= 16, each matrix stored
 * column-major with minimal leading dimension (rows of the stored matrix)
 * at element offset a, b, c of three arenas.  flags: bits 0-1 opA (0 N,
 * 1 T, 2 C), bits 2-3 opB, bit 4 set = beta_q is 0 for this problem (C_q
 * is then not read), else beta_q is the call's beta.  32 bytes.
 */
typedef struct {
    int m, n, k;
    int flags;
    long long a, b, c;
} sbgemm_vproblem;

typedef struct sbgemm_vplan_s* sbgemm_vplan;

/*
 * Build a plan for `count` problems (host array, copied): problems are
 * bucketed by (m, n, k, opA transposed, opB transposed), each bucket is cut
 * into tiles, and the tile list and per-problem records are uploaded to
 * device memory owned by the plan (allocated here, on the current device).
 * For real and complex fp64, the buckets whose class the selector sends to
 * the tensor-core kernel (as for a uniform batch of the bucket's size, beta
 * taken as nonzero; large sizes under the built-in rule) are not tiled:
 * their problems form a record list that the same run computes with that
 * kernel, in a second launch.  The selection applies when the plan is
 * built.  The C_q must not overlap.  Returns SBGEMM_ERR_INVALID_SIZE /
 * SBGEMM_ERR_INVALID_TRANS for a bad problem (nothing allocated).
 */
sbgemm_status sbgemm_vbatch_plan_create(sbgemm_vplan* plan, int type,
                                        const sbgemm_vproblem* problems, int count);
sbgemm_status sbgemm_vbatch_plan_destroy(sbgemm_vplan plan);

/*
 * Bucketing window of the plans created after this call: problems are
 * bucketed within windows of `window` consecutive problems and the tiles
 * are queued window by window, so neighbours in the arenas (which may share
 * memory sectors) are processed close in time and those sectors are read
 * from DRAM once.  0 restores the default, 65,536 problems; a window of at
 * least the problem count buckets the whole batch at once.  Process-wide;
 * negative values give SBGEMM_ERR_INVALID_VALUE.
 */
sbgemm_status sbgemm_vbatch_config(int window);

/*
 * Run a plan: one persistent kernel launch whose blocks take tiles from a
 * device work queue (an atomic counter reset by a memset node first), so
 * the whole batch is a memset plus one kernel on `stream` and can be
 * captured into a CUDA graph.  alpha/beta as for the uniform entry points
 * (scalar_mode; fp32 scalars for the 16-bit types).  A, B, C are the
 * arenas, each aligned to the element size (16 bytes for complex double).
 * A matrix is moved in 16-byte chunks wherever its start and its size
 * allow; for sizes whose matrices are not a whole number of 16-byte chunks
 * (odd sizes of the 4- and 8-byte types, for example), the middle of the
 * matrix moves in chunks at any start address and only the ragged head and
 * tail move element by element.  Concurrent runs of the same plan race on
 * its queue counter.
 */
sbgemm_status sbgemm_vbatch_run(sbgemm_vplan plan, const void* alpha, const void* A,
                                const void* B, const void* beta, void* C,
                                int scalar_mode, void* stream);

/* Plan statistics: number of tiles, of buckets, and device bytes owned. */
sbgemm_status sbgemm_vbatch_plan_info(sbgemm_vplan plan, int* n_tiles, int* n_buckets,
                                      long long* device_bytes);

/* Largest problem count sbgemm_vbatch_run_noalloc accepts. */
#define SBGEMM_NOALLOC_MAX_PROBLEMS 262144

/*
 * The variable-size run without any memory allocation.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * while they run, such as a plug-in inside a host application that owns all
 * device memory, or a latency-critical loop that must keep a fixed footprint
 * and cannot take the device-wide synchronisation cudaMalloc may imply.
 *
 * `problems` is a DEVICE array of `count` records (same meaning as for
 * sbgemm_vbatch_plan_create).  The tile list, the per-problem records, the
 * bucketing counters and the work-queue counter live in one fixed-size
 * static device array of this library (about 13 MB, held by every GPU that
 * loads the library until the process exits); the bucketing runs on the
 * device, then the same persistent kernel as sbgemm_vbatch_run computes.
 * No cudaMalloc, cudaFree or other allocating routine is called.
 *
 *  - count above SBGEMM_NOALLOC_MAX_PROBLEMS returns SBGEMM_ERR_CAPACITY
 *    before anything is queued.
 *  - The first call on a device looks up the device address of the static
 *    array (set-up, once per device, with that device current).
 *  - Every call uses the same array: it clears the counters it needs, but
 *    two calls whose work overlaps on the GPU (other streams, other host
 *    threads) race on it and give wrong results.
 *  - The tile count is read back to the host before the GEMM kernel is
 *    launched, so the call returns after the earlier work on `stream` and
 *    the bucketing kernels have finished.  For the same reason this call
 *    cannot be captured into a CUDA graph (use a plan and sbgemm_vbatch_run
 *    for that).
 *  - Every problem stays on the CUDA-core kernels (no tensor-core record
 *    list as in a plan).
 *  - A problem with m, n or k outside 0..16, an op code of 3 or a negative
 *    offset gives SBGEMM_ERR_INVALID_SIZE (no GEMM is launched).
 */
sbgemm_status sbgemm_vbatch_run_noalloc(int type, const sbgemm_vproblem* problems, int count,
                                        const void* alpha, const void* A, const void* B,
                                        const void* beta, void* C, int scalar_mode, void* stream);

/* ------------------------------------------------------------------ */
/* Timing core (autotuner).                                             */
/* ------------------------------------------------------------------ */

typedef struct sbgemm_timer_s* sbgemm_timer;

/* A set of n_marks CUDA events.  A mark is an external event record, so
 * marks issued while a stream is being captured become event nodes of the
 * graph and time every replay. */
sbgemm_status sbgemm_timer_create(sbgemm_timer* timer, int n_marks);
sbgemm_status sbgemm_timer_mark(sbgemm_timer timer, int mark, void* stream);
/* Milliseconds between two marks; waits for mark `to` to complete. */
sbgemm_status sbgemm_timer_elapsed(sbgemm_timer timer, int from, int to, float* ms);
sbgemm_status sbgemm_timer_destroy(sbgemm_timer timer);

/*
 * Time (ms) of one call of a kernel variant (host scalars): the mean over
 * `reps` calls, each timed alone with CUDA events, of those within 2 us of
 * the median (event timestamps can advance in steps of about 1 us; the mean
 * of many calls resolves below a step).
 * When `flush` is not NULL, flush_bytes of that device buffer (choose more
 * than the L2 size) are read before each call, outside the timed interval:
 * every call then starts with a cold L2 holding only clean lines (the
 * previous call's results are written back before the timing starts).
 * Synchronises the stream.
 */
sbgemm_status sbgemm_time_variant(int type, char transa, char transb, int m, int n, int k,
    const void* alpha, const void* A, int lda, long long lda2,
    const void* B, int ldb, long long ldb2, const void* beta, void* C, int ldc,
    long long ldc2, int batchCount, int variant, int reps, void* flush, size_t flush_bytes,
    void* stream, float* ms);

/* ------------------------------------------------------------------ */
/* Learned variant selector: a 3-layer perceptron cost model.           */
/* ------------------------------------------------------------------ */

/*
 * Network with F inputs, H hidden units (two hidden layers) and V outputs
 * (one predicted log-time per kernel variant), fp32:
 *   Z1 = X W1^T + b1, H1 = relu(Z1); Z2 = H1 W2^T + b2, H2 = relu(Z2);
 *   Y = H2 W3^T + b3.
 * Parameters are one device buffer, row-major: W1 (H x F), b1 (H),
 * W2 (H x H), b2 (H), W3 (V x H), b3 (V); sbgemm_mlp_param_count gives its
 * length in floats (0 for invalid sizes).  X is batch x F, Y batch x V,
 * row-major, device memory owned by the caller.  The paper has no
 * counterpart: this selects among this library's kernel variants.
 */
long long sbgemm_mlp_param_count(int F, int H, int V);

/* Forward pass.  work: 4*batch*H floats (keeps Z1, H1, Z2, H2 for the
 * backward pass). */
sbgemm_status sbgemm_mlp_forward(int F, int H, int V, const float* params, const float* X,
                                 int batch, float* Y, float* work, void* stream);

/*
 * Masked mean-squared-error loss and its gradient:
 *   L = sum mask (Y - T)^2 / (2 M), M = sum mask (L = 0 when M = 0),
 * back-propagated through the network (relu'(0) = 0).  Y and work come from
 * sbgemm_mlp_forward with the same X.  grads has the parameter layout;
 * work2: batch*(V + 2H) floats; loss: 2 floats on the device (L, M).
 * Reductions run in a fixed order: results are reproducible.
 */
sbgemm_status sbgemm_mlp_backward(int F, int H, int V, const float* params, const float* X,
                                  int batch, const float* Y, const float* T, const float* mask,
                                  const float* work, float* grads, float* work2, float* loss,
                                  void* stream);

/* One Adam step (Kingma & Ba 2015, Algorithm 1) on n parameters; t >= 1 is
 * the step number used in the bias corrections; m, v are the moment
 * buffers (zero before the first step).  l2 >= 0 adds an L2 penalty
 * (l2 / 2) |params|^2 to the loss: the step uses g = grads + l2 * params in
 * place of grads (0 gives plain Adam; negative or non-finite l2 is
 * SBGEMM_ERR_INVALID_VALUE). */
sbgemm_status sbgemm_mlp_adam(long long n, float* params, const float* grads, float* m, float* v,
                              int t, float lr, float beta1, float beta2, float eps, float l2,
                              void* stream);

/* ------------------------------------------------------------------ */
/* Status.                                                              */
/* ------------------------------------------------------------------ */

/* Static description of a status code (never NULL). */
/*
 * Kernels that wait on hardware barriers (bulk copies) bound every wait; a
 * wait that expires records SBGEMM_ERR_TIMEOUT in a per-device error word
 * and the kernel stops early (its results are then incomplete).  This call
 * waits for `stream`, returns the word in *code (0: no expired wait since
 * the last call) and clears it.
 */
sbgemm_status sbgemm_device_error(int* code, void* stream);

/*
 * Self-test of the failure detection above (no counterpart in the paper):
 * one thread arms a barrier for copies that are never issued and waits on
 * it with the same bounded wait the kernels use, giving up after
 * `spin_limit` polls (1 .. 4194304, else SBGEMM_ERR_INVALID_VALUE).  The
 * expired wait records SBGEMM_ERR_TIMEOUT in the device error word, which
 * the next sbgemm_device_error reports and clears; the kernel then returns
 * with nothing in flight, so the context stays usable.  Queued on `stream`.
 */
sbgemm_status sbgemm_wait_selftest(long long spin_limit, void* stream);

const char* sbgemm_status_string(sbgemm_status status);

/* Library version as major*10000 + minor*100 + patch. */
int sbgemm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SBGEMM_H */
