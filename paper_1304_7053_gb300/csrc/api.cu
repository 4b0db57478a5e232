// C ABI of the batched small-matrix GEMM library (declarations and the
// argument conventions are in include/sbgemm.h).
//
// Each call validates its arguments (dimensions and trans characters of
// Section 2, leading dimensions of the Section 4 layout), classifies alpha
// and beta when they are host scalars (the functor choice of Section 5:
// beta == 0 never reads C; alpha == 0 or k == 0 reduces to C = beta*C),
// picks a kernel variant from the selection table, and launches.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "sbgemm_launch.cuh"
#include "sbgemm_shapes.h"
#include "selection.h"

namespace sbg {

int num_sms() {
    static std::atomic<int> cache[kMaxDevices];
    const int dev = current_device();
    if (dev < 0) return 1;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

// Error word written by kernels whose bounded waits expire (one per
// device, in this module; kernels of other modules get its address).
__device__ int g_device_error;

int* device_error_ptr() {
    static std::atomic<int*> cache[kMaxDevices];
    const int dev = current_device();
    if (dev < 0) return nullptr;
    int* p = cache[dev].load(std::memory_order_acquire);
    if (!p) {
        void* a = nullptr;
        if (cudaGetSymbolAddress(&a, g_device_error) != cudaSuccess) return nullptr;
        p = static_cast<int*>(a);
        cache[dev].store(p, std::memory_order_release);
    }
    return p;
}

// Failure-detection self-test: thread 0 arms a barrier for 16 bytes of
// copies that are never issued and waits on it with the kernels' bounded
// wait (at most `limit` polls); the expired wait is recorded like any other.
// No copy is in flight when the kernel returns.
__global__ void wait_selftest_kernel(long long limit, int* err) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_fence_init();
    mbar_arrive_expect_tx(&bar, 16);
    if (!mbar_wait(&bar, 0, limit) && err) atomicExch(err, (int)SBGEMM_ERR_TIMEOUT);
}

namespace {

int op_code(char t) {
    switch (t) {
    case 'n': case 'N': return 0;
    case 't': case 'T': return 1;
    case 'c': case 'C': return 2;
    default: return -1;
    }
}

bool is_complex_type(int type) { return type == SBGEMM_TYPE_C || type == SBGEMM_TYPE_Z; }

bool host_scalar_zero(int type, const void* p) {
    switch (type) {
    case SBGEMM_TYPE_D: return *static_cast<const double*>(p) == 0.0;
    case SBGEMM_TYPE_C: { const float* f = static_cast<const float*>(p); return f[0] == 0.f && f[1] == 0.f; }
    case SBGEMM_TYPE_Z: { const double* d = static_cast<const double*>(p); return d[0] == 0.0 && d[1] == 0.0; }
    default: return *static_cast<const float*>(p) == 0.f;
    }
}

// Map a public variant index to the internal one.  Shapes with specialised
// kernels use the internal index as is; the other shapes have the generic
// kernel (internal kNumPipeVariants) as variant 0 and, for real and complex
// fp64, the tensor-core kernel (internal kMmaVariant) as variant 1.
int internal_variant(int type, int m, int n, int k, int v) {
    if (has_specialized(0, m, n, k)) return v;
    return (type == SBGEMM_TYPE_D || type == SBGEMM_TYPE_Z) && v == 1 ? kMmaVariant
                                                                       : kNumPipeVariants;
}

sbgemm_status run_typed(const Req& r) {
    switch (r.type) {
    case SBGEMM_TYPE_S: return run_S(r);
    case SBGEMM_TYPE_D: return run_D(r);
    case SBGEMM_TYPE_C: return run_C(r);
    case SBGEMM_TYPE_Z: return run_Z(r);
    case SBGEMM_TYPE_H: return run_H(r);
    case SBGEMM_TYPE_B: return run_B(r);
    default: return SBGEMM_ERR_INVALID_VALUE;
    }
}

sbgemm_status scale_typed(const Req& r) {
    switch (r.type) {
    case SBGEMM_TYPE_S: return launch_scale<TyS>(r);
    case SBGEMM_TYPE_D: return launch_scale<TyD>(r);
    case SBGEMM_TYPE_C: return launch_scale<TyC>(r);
    case SBGEMM_TYPE_Z: return launch_scale<TyZ>(r);
    case SBGEMM_TYPE_H: return launch_scale<TyH>(r);
    case SBGEMM_TYPE_B: return launch_scale<TyB>(r);
    default: return SBGEMM_ERR_INVALID_VALUE;
    }
}

}  // namespace

// Shared by every uniform-layout entry point.  variant < 0: use the table.
sbgemm_status gemm_uniform(int type, char transa, char transb, int m, int n, int k,
                           const void* alpha, const void* A, int lda, long long lda2,
                           const void* B, int ldb, long long ldb2,
                           const void* beta, void* C, int ldc, long long ldc2, int batch,
                           int scalar_mode, int variant, cudaStream_t stream)
{
    if (type < SBGEMM_TYPE_S || type > SBGEMM_TYPE_B) return SBGEMM_ERR_INVALID_VALUE;
    int opa = op_code(transa), opb = op_code(transb);
    if (opa < 0 || opb < 0) return SBGEMM_ERR_INVALID_TRANS;
    if (m < 0 || n < 0 || k < 0 || m > 16 || n > 16 || k > 16 || batch < 0)
        return SBGEMM_ERR_INVALID_SIZE;
    if (scalar_mode != SBGEMM_SCALARS_HOST && scalar_mode != SBGEMM_SCALARS_DEVICE)
        return SBGEMM_ERR_INVALID_VALUE;
    const long long ar = opa == 0 ? m : k, ac = opa == 0 ? k : m;
    const long long br = opb == 0 ? k : n, bc = opb == 0 ? n : k;
    auto max1 = [](long long v) { return v > 1 ? v : 1LL; };
    if (lda < max1(ar) || ldb < max1(br) || ldc < max1(m)) return SBGEMM_ERR_INVALID_LD;
    if (lda2 != 0 && lda2 < (long long)lda * ac) return SBGEMM_ERR_INVALID_LD;
    if (ldb2 != 0 && ldb2 < (long long)ldb * bc) return SBGEMM_ERR_INVALID_LD;
    if (lda2 < 0 || ldb2 < 0 || ldc2 < (long long)ldc * n) return SBGEMM_ERR_INVALID_LD;
    if (batch == 0 || m == 0 || n == 0) return SBGEMM_SUCCESS;   // quick return
    if (!alpha || !beta || !C) return SBGEMM_ERR_NULL_POINTER;

    Req r;
    std::memset(&r, 0, sizeof r);
    r.type = type; r.m = m; r.n = n; r.k = k;
    const bool cplx = is_complex_type(type);
    r.ta = opa != 0; r.tb = opb != 0;
    r.conja = cplx && opa == 2; r.conjb = cplx && opb == 2;
    r.A = A; r.B = B; r.C = C;
    r.lda = lda; r.ldb = ldb; r.ldc = ldc;
    r.lda2 = lda2; r.ldb2 = ldb2; r.ldc2 = ldc2;
    r.batch = batch;
    r.scalar_mode = scalar_mode;
    r.alpha = alpha; r.beta = beta;
    r.stream = stream;
    if (scalar_mode == SBGEMM_SCALARS_HOST) {
        r.alpha_zero = host_scalar_zero(type, alpha);
        r.beta_zero = host_scalar_zero(type, beta);
    }
    if (k == 0 || r.alpha_zero) return scale_typed(r);   // C = beta*C, A and B unread
    if (!A || !B) return SBGEMM_ERR_NULL_POINTER;

    const int nv = variants_for(type, m, n, k);
    if (variant >= 0) {
        if (variant >= nv) return SBGEMM_ERR_INVALID_VALUE;
    } else {
        variant = select_variant(type, m, n, k, r.ta, r.tb,
                                 scalar_mode == SBGEMM_SCALARS_HOST ? r.beta_zero : 0,
                                 size_class(batch));
    }
    note_variant(variant);
    r.variant = internal_variant(type, m, n, k, variant);
    return run_typed(r);
}

// The pointer-array form (Section 4's TGEMM_multi_nounif): the same
// checks and kernels as the 3-D layout, matrix p of each operand at the
// p-th pointer of a device array.
sbgemm_status gemm_nounif(int type, char transa, char transb, int m, int n, int k,
                          const void* alpha, const void* const* Ap, int lda,
                          const void* const* Bp, int ldb, const void* beta, void* const* Cp,
                          int ldc, int batch, int scalar_mode, cudaStream_t stream)
{
    if (type < SBGEMM_TYPE_S || type > SBGEMM_TYPE_B) return SBGEMM_ERR_INVALID_VALUE;
    int opa = op_code(transa), opb = op_code(transb);
    if (opa < 0 || opb < 0) return SBGEMM_ERR_INVALID_TRANS;
    if (m < 0 || n < 0 || k < 0 || m > 16 || n > 16 || k > 16 || batch < 0)
        return SBGEMM_ERR_INVALID_SIZE;
    if (scalar_mode != SBGEMM_SCALARS_HOST && scalar_mode != SBGEMM_SCALARS_DEVICE)
        return SBGEMM_ERR_INVALID_VALUE;
    const long long ar = opa == 0 ? m : k;
    const long long br = opb == 0 ? k : n;
    auto max1 = [](long long v) { return v > 1 ? v : 1LL; };
    if (lda < max1(ar) || ldb < max1(br) || ldc < max1(m)) return SBGEMM_ERR_INVALID_LD;
    if (batch == 0 || m == 0 || n == 0) return SBGEMM_SUCCESS;
    if (!alpha || !beta || !Cp) return SBGEMM_ERR_NULL_POINTER;

    Req r;
    std::memset(&r, 0, sizeof r);
    r.type = type; r.m = m; r.n = n; r.k = k;
    const bool cplx = is_complex_type(type);
    r.ta = opa != 0; r.tb = opb != 0;
    r.conja = cplx && opa == 2; r.conjb = cplx && opb == 2;
    r.Ap = Ap; r.Bp = Bp; r.Cp = Cp;
    r.lda = lda; r.ldb = ldb; r.ldc = ldc;
    r.lda2 = r.ldb2 = r.ldc2 = -1;     // unused in the pointer-array form
    r.batch = batch;
    r.scalar_mode = scalar_mode;
    r.alpha = alpha; r.beta = beta;
    r.stream = stream;
    if (scalar_mode == SBGEMM_SCALARS_HOST) {
        r.alpha_zero = host_scalar_zero(type, alpha);
        r.beta_zero = host_scalar_zero(type, beta);
    }
    if (k == 0 || r.alpha_zero) return scale_typed(r);
    if (!Ap || !Bp) return SBGEMM_ERR_NULL_POINTER;
    const int variant = select_variant(type, m, n, k, r.ta, r.tb,
                                       scalar_mode == SBGEMM_SCALARS_HOST ? r.beta_zero : 0,
                                       size_class(batch));
    note_variant(variant);
    r.variant = internal_variant(type, m, n, k, variant);
    return run_typed(r);
}

}  // namespace sbg

using sbg::gemm_uniform;
using sbg::gemm_nounif;

extern "C" {

#define SBG_PAPER_ENTRY(L, T, CODE)                                                         \
    sbgemm_status sbgemm_##L##gemm_multi_uniform(char transa, char transb, int m, int n, int k, \
        const T* alpha, const T* A, int lda, long long lda2, const T* B, int ldb,           \
        long long ldb2, const T* beta, T* C, int ldc, long long ldc2, int batchCount) {     \
        return gemm_uniform(CODE, transa, transb, m, n, k, alpha, A, lda, lda2, B, ldb,     \
                            ldb2, beta, C, ldc, ldc2, batchCount, SBGEMM_SCALARS_HOST, -1,  \
                            (cudaStream_t)0);                                               \
    }                                                                                       \
    sbgemm_status sbgemm_##L##gemm_multi_uniform_async(char transa, char transb, int m,     \
        int n, int k, const T* alpha, const T* A, int lda, long long lda2, const T* B,      \
        int ldb, long long ldb2, const T* beta, T* C, int ldc, long long ldc2,              \
        int batchCount, int scalar_mode, void* stream) {                                    \
        return gemm_uniform(CODE, transa, transb, m, n, k, alpha, A, lda, lda2, B, ldb,     \
                            ldb2, beta, C, ldc, ldc2, batchCount, scalar_mode, -1,          \
                            (cudaStream_t)stream);                                          \
    }

#define SBG_NOUNIF_ENTRY(L, T, CODE)                                                        \
    sbgemm_status sbgemm_##L##gemm_multi_nounif(char transa, char transb, int m, int n, int k,  \
        const T* alpha, const T* const* Aarray, int lda, const T* const* Barray, int ldb,   \
        const T* beta, T* const* Carray, int ldc, int batchCount) {                         \
        return gemm_nounif(CODE, transa, transb, m, n, k, alpha,                            \
                           reinterpret_cast<const void* const*>(Aarray), lda,               \
                           reinterpret_cast<const void* const*>(Barray), ldb, beta,         \
                           reinterpret_cast<void* const*>(Carray), ldc, batchCount,         \
                           SBGEMM_SCALARS_HOST, (cudaStream_t)0);                           \
    }

SBG_NOUNIF_ENTRY(S, float, SBGEMM_TYPE_S)
SBG_NOUNIF_ENTRY(D, double, SBGEMM_TYPE_D)
SBG_NOUNIF_ENTRY(C, sbgemm_c32, SBGEMM_TYPE_C)
SBG_NOUNIF_ENTRY(Z, sbgemm_c64, SBGEMM_TYPE_Z)
#undef SBG_NOUNIF_ENTRY

sbgemm_status sbgemm_gemm_multi_nounif(int type, char transa, char transb, int m, int n, int k,
    const void* alpha, const void* const* Aarray, int lda, const void* const* Barray, int ldb,
    const void* beta, void* const* Carray, int ldc, int batchCount, int scalar_mode,
    void* stream) {
    return gemm_nounif(type, transa, transb, m, n, k, alpha, Aarray, lda, Barray, ldb, beta,
                       Carray, ldc, batchCount, scalar_mode, (cudaStream_t)stream);
}

SBG_PAPER_ENTRY(S, float, SBGEMM_TYPE_S)
SBG_PAPER_ENTRY(D, double, SBGEMM_TYPE_D)
SBG_PAPER_ENTRY(C, sbgemm_c32, SBGEMM_TYPE_C)
SBG_PAPER_ENTRY(Z, sbgemm_c64, SBGEMM_TYPE_Z)
#undef SBG_PAPER_ENTRY

sbgemm_status sbgemm_Hgemm_multi_uniform_async(char transa, char transb, int m, int n, int k,
    const float* alpha, const uint16_t* A, int lda, long long lda2,
    const uint16_t* B, int ldb, long long ldb2,
    const float* beta, uint16_t* C, int ldc, long long ldc2, int batchCount,
    int scalar_mode, void* stream) {
    return gemm_uniform(SBGEMM_TYPE_H, transa, transb, m, n, k, alpha, A, lda, lda2, B, ldb,
                        ldb2, beta, C, ldc, ldc2, batchCount, scalar_mode, -1, (cudaStream_t)stream);
}

sbgemm_status sbgemm_Bgemm_multi_uniform_async(char transa, char transb, int m, int n, int k,
    const float* alpha, const uint16_t* A, int lda, long long lda2,
    const uint16_t* B, int ldb, long long ldb2,
    const float* beta, uint16_t* C, int ldc, long long ldc2, int batchCount,
    int scalar_mode, void* stream) {
    return gemm_uniform(SBGEMM_TYPE_B, transa, transb, m, n, k, alpha, A, lda, lda2, B, ldb,
                        ldb2, beta, C, ldc, ldc2, batchCount, scalar_mode, -1, (cudaStream_t)stream);
}

int sbgemm_num_variants(int type, int m, int n, int k) {
    if (type < SBGEMM_TYPE_S || type > SBGEMM_TYPE_B) return 0;
    return sbg::variants_for(type, m, n, k);
}

const char* sbgemm_variant_name(int type, int m, int n, int k, int variant) {
    static const char* names[] = {
        "pipe tile16K st3 occ-max (st2 for fp64)", "pipe tile8K st4 occ-max",
        "pipe tile32K st2 occ-max", "pipe tile16K st3 1cta/sm (st2 for fp64)",
        "pipe tile4K st4 occ-max", "pipe tile24K st3 2cta/sm",
        "generic thread-per-entry",
        "tensor-core: mma.sync for 16-bit N/N flat; 8-bit digit products for fp64 and complex128; else variant 0"};
    const int nv = sbgemm_num_variants(type, m, n, k);
    if (variant < 0 || variant >= nv) return "invalid";
    return names[sbg::internal_variant(type, m, n, k, variant)];
}

sbgemm_status sbgemm_gemm_multi_uniform_variant(int type, char transa, char transb,
    int m, int n, int k, const void* alpha, const void* A, int lda, long long lda2,
    const void* B, int ldb, long long ldb2, const void* beta, void* C, int ldc,
    long long ldc2, int batchCount, int scalar_mode, int variant, void* stream) {
    if (variant < 0) return SBGEMM_ERR_INVALID_VALUE;
    return gemm_uniform(type, transa, transb, m, n, k, alpha, A, lda, lda2, B, ldb, ldb2,
                        beta, C, ldc, ldc2, batchCount, scalar_mode, variant, (cudaStream_t)stream);
}

const char* sbgemm_status_string(sbgemm_status s) {
    switch (s) {
    case SBGEMM_SUCCESS: return "success";
    case SBGEMM_ERR_INVALID_TRANS: return "invalid trans character";
    case SBGEMM_ERR_INVALID_SIZE: return "m, n, k outside 0..16 or negative batch count";
    case SBGEMM_ERR_INVALID_LD: return "leading dimension below its minimum";
    case SBGEMM_ERR_NULL_POINTER: return "null pointer";
    case SBGEMM_ERR_INVALID_VALUE: return "invalid argument";
    case SBGEMM_ERR_TIMEOUT: return "bounded in-kernel wait expired";
    case SBGEMM_ERR_NOT_SUPPORTED: return "not supported";
    case SBGEMM_ERR_CAPACITY: return "request exceeds a fixed capacity";
    case SBGEMM_ERR_IO: return "file cannot be read or written, or has a bad format";
    default: return s > 0 ? cudaGetErrorString((cudaError_t)s) : "unknown status";
    }
}

sbgemm_status sbgemm_device_error(int* code, void* stream) {
    if (!code) return SBGEMM_ERR_NULL_POINTER;
    *code = 0;
    int* p = sbg::device_error_ptr();
    if (!p) return SBGEMM_ERR_NOT_SUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, p, sizeof v, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && v != 0) e = cudaMemsetAsync(p, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return (sbgemm_status)e;
    *code = v;
    return SBGEMM_SUCCESS;
}

sbgemm_status sbgemm_wait_selftest(long long spin_limit, void* stream) {
    if (spin_limit < 1 || spin_limit > sbg::kSpinLimit) return SBGEMM_ERR_INVALID_VALUE;
    int* err = sbg::device_error_ptr();
    if (!err) return SBGEMM_ERR_NOT_SUPPORTED;
    sbg::wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(spin_limit, err);
    return (sbgemm_status)cudaGetLastError();
}

int sbgemm_version(void) { return 100; }

}  // extern "C"
