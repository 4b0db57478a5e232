// Eq. (1) on host-resident arrays: one or more uniform batches stream through
// a caller-owned device work buffer in chunks, double-buffered, with
// host->device copies, kernels and device->host copies of consecutive chunks
// overlapping on three streams (copy-in, the caller's stream for compute,
// copy-out).  Several groups form one continuous pipeline, so the copy-back
// tail of one group overlaps the copy-in of the next.
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
constexpr size_t kChunkBytes = 48u << 20;

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

// One continuous double-buffered pipeline over the chunks of every group.
static sbgemm_status stream_groups(int type, const void* alpha, const void* beta,
                                   const sbgemm_host_group* groups, int ngroups, void* dwork,
                                   size_t dwork_bytes, cudaStream_t cs) {
    using namespace sbg;
    if (type < SBGEMM_TYPE_S || type > SBGEMM_TYPE_B) return SBGEMM_ERR_INVALID_VALUE;
    if (ngroups < 0) return SBGEMM_ERR_INVALID_SIZE;
    if (ngroups > 0 && !groups) return SBGEMM_ERR_NULL_POINTER;
    if (!alpha || !beta || !dwork) return SBGEMM_ERR_NULL_POINTER;
    const size_t es = elem_bytes(type);
    const bool beta0 = scalar_is_zero(type, beta);
    const bool alpha0 = scalar_is_zero(type, alpha);
    const size_t half = dwork_bytes / 2 / 256 * 256;
    // full argument checks and capacity before anything is queued
    for (int g = 0; g < ngroups; ++g) {
        const sbgemm_host_group& G = groups[g];
        if (G.m < 0 || G.n < 0 || G.k < 0 || G.m > 16 || G.n > 16 || G.k > 16 || G.batchCount < 0)
            return SBGEMM_ERR_INVALID_SIZE;
        if (G.batchCount == 0 || G.m == 0 || G.n == 0) continue;
        if (!G.hC) return SBGEMM_ERR_NULL_POINTER;
        if (G.lda2 == 0 || G.ldb2 == 0) return SBGEMM_ERR_NOT_SUPPORTED;
        const sbgemm_status chk = gemm_uniform(type, G.transa, G.transb, G.m, G.n, G.k, alpha,
                                               G.hA, G.lda, G.lda2, G.hB, G.ldb, G.ldb2, beta,
                                               G.hC, G.ldc, G.ldc2, 0, SBGEMM_SCALARS_HOST, -1, cs);
        if (chk != SBGEMM_SUCCESS) return chk;
        const bool ab_in = G.k > 0 && !alpha0;
        const size_t perA = ab_in ? es * (size_t)G.lda2 : 0, perB = ab_in ? es * (size_t)G.ldb2 : 0;
        const size_t perC = es * (size_t)G.ldc2;
        if (3 * 256 + perA + perB + perC > half) return SBGEMM_ERR_CAPACITY;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    StreamSet* ss = nullptr;
    sbgemm_status st = stream_set(&ss);
    if (st != SBGEMM_SUCCESS) return st;
    cudaError_t e;
    // everything earlier on the caller's stream comes first
    if ((e = cudaEventRecord(ss->start, cs)) != cudaSuccess) return (sbgemm_status)e;
    if ((e = cudaStreamWaitEvent(ss->in, ss->start, 0)) != cudaSuccess) return (sbgemm_status)e;
    long long i = 0;           // chunk counter across all groups
    for (int g = 0; g < ngroups; ++g) {
        const sbgemm_host_group& G = groups[g];
        if (G.batchCount == 0 || G.m == 0 || G.n == 0) continue;
        const int m = G.m, n = G.n, k = G.k;
        const bool ab_in = k > 0 && !alpha0;
        // C is copied in when beta != 0, and also when its layout has gaps,
        // so the copy back returns the gaps unchanged
        const bool c_in = !beta0 || G.ldc != m || G.ldc2 != (long long)G.ldc * n;
        const size_t perA = ab_in ? es * (size_t)G.lda2 : 0, perB = ab_in ? es * (size_t)G.ldb2 : 0;
        const size_t perC = es * (size_t)G.ldc2;
        // chunks of about kChunkBytes: large enough that a copy's fixed cost
        // is small, small enough that copies of consecutive chunks overlap
        // (a small group is one chunk; the pipeline runs across groups)
        const size_t limit = half - 3 * 256 < kChunkBytes ? half - 3 * 256 : kChunkBytes;
        long long chunk = (long long)(limit / (perA + perB + perC));
        if (chunk < 1) chunk = 1;
        if (chunk > G.batchCount) chunk = G.batchCount;
        const size_t secA = (chunk * perA + 255) / 256 * 256;
        const size_t secB = (chunk * perB + 255) / 256 * 256;
        const char* a8 = static_cast<const char*>(G.hA);
        const char* b8 = static_cast<const char*>(G.hB);
        char* c8 = static_cast<char*>(G.hC);
        const bool na = G.transa == 'N' || G.transa == 'n', nbt = G.transb == 'N' || G.transb == 'n';
        for (long long p0 = 0; p0 < G.batchCount; p0 += chunk, ++i) {
            const int b = (int)(i & 1);
            const long long cnt = (G.batchCount - p0) < chunk ? (G.batchCount - p0) : chunk;
            char* base = static_cast<char*>(dwork) + b * half;
            char* dA = base;
            char* dB = base + secA;
            char* dC = base + secA + secB;
            // spans: the last matrix of a chunk ends at its own last element
            const size_t spanA = es * ((size_t)(cnt - 1) * G.lda2 + (size_t)G.lda * (na ? k : m));
            const size_t spanB = es * ((size_t)(cnt - 1) * G.ldb2 + (size_t)G.ldb * (nbt ? n : k));
            const size_t spanC = es * ((size_t)(cnt - 1) * G.ldc2 + (size_t)G.ldc * n);
            if ((e = cudaStreamWaitEvent(ss->in, ss->d2h[b], 0)) != cudaSuccess) return (sbgemm_status)e;
            if (ab_in) {
                if ((e = cudaMemcpyAsync(dA, a8 + es * (size_t)p0 * G.lda2, spanA, cudaMemcpyHostToDevice, ss->in)) != cudaSuccess) return (sbgemm_status)e;
                if ((e = cudaMemcpyAsync(dB, b8 + es * (size_t)p0 * G.ldb2, spanB, cudaMemcpyHostToDevice, ss->in)) != cudaSuccess) return (sbgemm_status)e;
            }
            if (c_in && (e = cudaMemcpyAsync(dC, c8 + es * (size_t)p0 * G.ldc2, spanC, cudaMemcpyHostToDevice, ss->in)) != cudaSuccess)
                return (sbgemm_status)e;
            if ((e = cudaEventRecord(ss->h2d[b], ss->in)) != cudaSuccess) return (sbgemm_status)e;
            if ((e = cudaStreamWaitEvent(cs, ss->h2d[b], 0)) != cudaSuccess) return (sbgemm_status)e;
            st = gemm_uniform(type, G.transa, G.transb, m, n, k, alpha, dA, G.lda, G.lda2, dB, G.ldb,
                              G.ldb2, beta, dC, G.ldc, G.ldc2, (int)cnt, SBGEMM_SCALARS_HOST, -1, cs);
            if (st != SBGEMM_SUCCESS) return st;
            if ((e = cudaEventRecord(ss->comp[b], cs)) != cudaSuccess) return (sbgemm_status)e;
            if ((e = cudaStreamWaitEvent(ss->out, ss->comp[b], 0)) != cudaSuccess) return (sbgemm_status)e;
            if ((e = cudaMemcpyAsync(c8 + es * (size_t)p0 * G.ldc2, dC, spanC, cudaMemcpyDeviceToHost, ss->out)) != cudaSuccess)
                return (sbgemm_status)e;
            if ((e = cudaEventRecord(ss->d2h[b], ss->out)) != cudaSuccess) return (sbgemm_status)e;
        }
    }
    // the caller's stream continues after the last copies back
    if ((e = cudaStreamWaitEvent(cs, ss->d2h[0], 0)) != cudaSuccess) return (sbgemm_status)e;
    if ((e = cudaStreamWaitEvent(cs, ss->d2h[1], 0)) != cudaSuccess) return (sbgemm_status)e;
    return SBGEMM_SUCCESS;
}

extern "C" sbgemm_status sbgemm_gemm_multi_uniform_host(int type, char transa, char transb,
    int m, int n, int k, const void* alpha, const void* hA, int lda, long long lda2,
    const void* hB, int ldb, long long ldb2, const void* beta, void* hC, int ldc,
    long long ldc2, int batchCount, void* dwork, size_t dwork_bytes, void* stream) {
    sbgemm_host_group g;
    g.transa = transa; g.transb = transb; g.m = m; g.n = n; g.k = k;
    g.hA = hA; g.lda = lda; g.lda2 = lda2;
    g.hB = hB; g.ldb = ldb; g.ldb2 = ldb2;
    g.hC = hC; g.ldc = ldc; g.ldc2 = ldc2;
    g.batchCount = batchCount;
    if (type < SBGEMM_TYPE_S || type > SBGEMM_TYPE_B) return SBGEMM_ERR_INVALID_VALUE;
    if (m < 0 || n < 0 || k < 0 || m > 16 || n > 16 || k > 16 || batchCount < 0)
        return SBGEMM_ERR_INVALID_SIZE;
    if (batchCount == 0 || m == 0 || n == 0) return SBGEMM_SUCCESS;
    return stream_groups(type, alpha, beta, &g, 1, dwork, dwork_bytes, (cudaStream_t)stream);
}

extern "C" sbgemm_status sbgemm_gemm_grouped_host(int type, const void* alpha, const void* beta,
    const sbgemm_host_group* groups, int ngroups, void* dwork, size_t dwork_bytes, void* stream) {
    return stream_groups(type, alpha, beta, groups, ngroups, dwork, dwork_bytes, (cudaStream_t)stream);
}
