// Eq. (1) on host-resident arrays: the batch streams through a caller-owned
// device work buffer in chunks, double-buffered, with host->device copies,
// kernels and device->host copies of consecutive chunks overlapping on three
// streams (copy-in, the caller's stream for compute, copy-out).
#include <mutex>

#include "sbgemm_launch.cuh"

namespace sbg {
sbgemm_status gemm_uniform(int type, char transa, char transb, int m, int n, int k,
                           const void* alpha, const void* A, int lda, long long lda2,
                           const void* B, int ldb, long long ldb2,
                           const void* beta, void* C, int ldc, long long ldc2, int batch,
                           int scalar_mode, int variant, cudaStream_t stream);

namespace {

struct StreamSet {
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t h2d[2] = {}, comp[2] = {}, d2h[2] = {}, start = nullptr;
    bool ready = false;
};

std::mutex g_mu;
StreamSet g_sets[64];

sbgemm_status stream_set(StreamSet** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (sbgemm_status)e;
    if (dev < 0 || dev >= 64) return SBGEMM_ERR_NOT_SUPPORTED;
    StreamSet& s = g_sets[dev];
    if (!s.ready) {
        if ((e = cudaStreamCreateWithFlags(&s.in, cudaStreamNonBlocking)) != cudaSuccess) return (sbgemm_status)e;
        if ((e = cudaStreamCreateWithFlags(&s.out, cudaStreamNonBlocking)) != cudaSuccess) return (sbgemm_status)e;
        for (int b = 0; b < 2; ++b) {
            if ((e = cudaEventCreateWithFlags(&s.h2d[b], cudaEventDisableTiming)) != cudaSuccess) return (sbgemm_status)e;
            if ((e = cudaEventCreateWithFlags(&s.comp[b], cudaEventDisableTiming)) != cudaSuccess) return (sbgemm_status)e;
            if ((e = cudaEventCreateWithFlags(&s.d2h[b], cudaEventDisableTiming)) != cudaSuccess) return (sbgemm_status)e;
        }
        if ((e = cudaEventCreateWithFlags(&s.start, cudaEventDisableTiming)) != cudaSuccess) return (sbgemm_status)e;
        s.ready = true;
    }
    *out = &s;
    return SBGEMM_SUCCESS;
}

size_t elem_bytes(int type) {
    switch (type) {
    case SBGEMM_TYPE_S: return 4;
    case SBGEMM_TYPE_D: return 8;
    case SBGEMM_TYPE_C: return 8;
    case SBGEMM_TYPE_Z: return 16;
    default: return 2;
    }
}

bool scalar_is_zero(int type, const void* p) {
    switch (type) {
    case SBGEMM_TYPE_D: return *static_cast<const double*>(p) == 0.0;
    case SBGEMM_TYPE_C: { const float* f = static_cast<const float*>(p); return f[0] == 0.f && f[1] == 0.f; }
    case SBGEMM_TYPE_Z: { const double* d = static_cast<const double*>(p); return d[0] == 0.0 && d[1] == 0.0; }
    default: return *static_cast<const float*>(p) == 0.f;
    }
}

}  // namespace
}  // namespace sbg

extern "C" sbgemm_status sbgemm_gemm_multi_uniform_host(int type, char transa, char transb,
    int m, int n, int k, const void* alpha, const void* hA, int lda, long long lda2,
    const void* hB, int ldb, long long ldb2, const void* beta, void* hC, int ldc,
    long long ldc2, int batchCount, void* dwork, size_t dwork_bytes, void* stream) {
    using namespace sbg;
    if (type < SBGEMM_TYPE_S || type > SBGEMM_TYPE_B) return SBGEMM_ERR_INVALID_VALUE;
    if (m < 0 || n < 0 || k < 0 || m > 16 || n > 16 || k > 16 || batchCount < 0)
        return SBGEMM_ERR_INVALID_SIZE;
    if (batchCount == 0 || m == 0 || n == 0) return SBGEMM_SUCCESS;
    if (!alpha || !beta || !hC || !dwork) return SBGEMM_ERR_NULL_POINTER;
    if (lda2 == 0 || ldb2 == 0) return SBGEMM_ERR_NOT_SUPPORTED;   // shared A/B: use the device entry
    {   // full argument check before anything is queued (a zero-pair call)
        const sbgemm_status chk = gemm_uniform(type, transa, transb, m, n, k, alpha, hA, lda, lda2,
                                               hB, ldb, ldb2, beta, hC, ldc, ldc2, 0,
                                               SBGEMM_SCALARS_HOST, -1, (cudaStream_t)stream);
        if (chk != SBGEMM_SUCCESS) return chk;
    }
    const size_t es = elem_bytes(type);
    const bool beta0 = scalar_is_zero(type, beta);
    // C is copied in when beta != 0, and also when its layout has gaps, so the
    // copy back returns the gaps unchanged
    const bool c_in = !beta0 || ldc != m || ldc2 != (long long)ldc * n;
    const bool ab_in = k > 0 && !scalar_is_zero(type, alpha);
    const size_t per = es * ((ab_in ? (size_t)(lda2 + ldb2) : 0) + (size_t)ldc2);
    // two buffers, each with chunk * per bytes, 256-byte aligned sections
    long long chunk = (long long)((dwork_bytes / 2) / (per + 1));
    while (chunk > 0 && 2 * (((size_t)chunk * es * lda2 + 255) / 256 * 256 * (ab_in ? 1 : 0)
                             + ((size_t)chunk * es * ldb2 + 255) / 256 * 256 * (ab_in ? 1 : 0)
                             + ((size_t)chunk * es * ldc2 + 255) / 256 * 256) > dwork_bytes)
        --chunk;
    if (chunk < 1) return SBGEMM_ERR_CAPACITY;
    // at least four chunks so the copies overlap, when the batch allows it
    if (chunk > (batchCount + 3) / 4 && batchCount >= 4) chunk = (batchCount + 3) / 4;
    const size_t secA = ab_in ? ((size_t)chunk * es * lda2 + 255) / 256 * 256 : 0;
    const size_t secB = ab_in ? ((size_t)chunk * es * ldb2 + 255) / 256 * 256 : 0;
    const size_t secC = ((size_t)chunk * es * ldc2 + 255) / 256 * 256;
    const size_t bufsz = secA + secB + secC;

    std::lock_guard<std::mutex> lk(g_mu);
    StreamSet* ss = nullptr;
    sbgemm_status st = stream_set(&ss);
    if (st != SBGEMM_SUCCESS) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e;
    // everything earlier on the caller's stream comes first
    if ((e = cudaEventRecord(ss->start, cs)) != cudaSuccess) return (sbgemm_status)e;
    if ((e = cudaStreamWaitEvent(ss->in, ss->start, 0)) != cudaSuccess) return (sbgemm_status)e;
    const char* a8 = static_cast<const char*>(hA);
    const char* b8 = static_cast<const char*>(hB);
    char* c8 = static_cast<char*>(hC);
    int last = 0;
    for (long long p0 = 0, i = 0; p0 < batchCount; p0 += chunk, ++i) {
        const int b = (int)(i & 1);
        last = b;
        const long long cnt = (batchCount - p0) < chunk ? (batchCount - p0) : chunk;
        char* base = static_cast<char*>(dwork) + b * bufsz;
        char* dA = base;
        char* dB = base + secA;
        char* dC = base + secA + secB;
        // spans: the last matrix of a chunk ends at its own last element
        const size_t spanA = es * ((size_t)(cnt - 1) * lda2 + (size_t)lda * (transa == 'N' || transa == 'n' ? k : m));
        const size_t spanB = es * ((size_t)(cnt - 1) * ldb2 + (size_t)ldb * (transb == 'N' || transb == 'n' ? n : k));
        const size_t spanC = es * ((size_t)(cnt - 1) * ldc2 + (size_t)ldc * n);
        if ((e = cudaStreamWaitEvent(ss->in, ss->d2h[b], 0)) != cudaSuccess) return (sbgemm_status)e;
        if (ab_in) {
            if ((e = cudaMemcpyAsync(dA, a8 + es * (size_t)p0 * lda2, spanA, cudaMemcpyHostToDevice, ss->in)) != cudaSuccess) return (sbgemm_status)e;
            if ((e = cudaMemcpyAsync(dB, b8 + es * (size_t)p0 * ldb2, spanB, cudaMemcpyHostToDevice, ss->in)) != cudaSuccess) return (sbgemm_status)e;
        }
        if (c_in && (e = cudaMemcpyAsync(dC, c8 + es * (size_t)p0 * ldc2, spanC, cudaMemcpyHostToDevice, ss->in)) != cudaSuccess)
            return (sbgemm_status)e;
        if ((e = cudaEventRecord(ss->h2d[b], ss->in)) != cudaSuccess) return (sbgemm_status)e;
        if ((e = cudaStreamWaitEvent(cs, ss->h2d[b], 0)) != cudaSuccess) return (sbgemm_status)e;
        st = gemm_uniform(type, transa, transb, m, n, k, alpha, dA, lda, lda2, dB, ldb, ldb2, beta,
                          dC, ldc, ldc2, (int)cnt, SBGEMM_SCALARS_HOST, -1, cs);
        if (st != SBGEMM_SUCCESS) return st;
        if ((e = cudaEventRecord(ss->comp[b], cs)) != cudaSuccess) return (sbgemm_status)e;
        if ((e = cudaStreamWaitEvent(ss->out, ss->comp[b], 0)) != cudaSuccess) return (sbgemm_status)e;
        if ((e = cudaMemcpyAsync(c8 + es * (size_t)p0 * ldc2, dC, spanC, cudaMemcpyDeviceToHost, ss->out)) != cudaSuccess)
            return (sbgemm_status)e;
        if ((e = cudaEventRecord(ss->d2h[b], ss->out)) != cudaSuccess) return (sbgemm_status)e;
    }
    // the caller's stream continues after the last copy back
    if ((e = cudaStreamWaitEvent(cs, ss->d2h[last], 0)) != cudaSuccess) return (sbgemm_status)e;
    if ((e = cudaStreamWaitEvent(cs, ss->d2h[last ^ 1], 0)) != cudaSuccess) return (sbgemm_status)e;
    return SBGEMM_SUCCESS;
}
