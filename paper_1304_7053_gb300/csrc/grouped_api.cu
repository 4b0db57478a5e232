// C entry point for several uniform batches in one call: qualifying groups
// share one persistent launch (grouped.cuh), the rest (and the fp64 /
// complex128 groups that take the tensor-core kernel) run as separate
// uniform calls on the same stream.
#include "grouped.cuh"
#include "selection.h"

namespace sbg {

sbgemm_status gemm_uniform(int type, char transa, char transb, int m, int n, int k,
                           const void* alpha, const void* A, int lda, long long lda2,
                           const void* B, int ldb, long long ldb2,
                           const void* beta, void* C, int ldc, long long ldc2, int batch,
                           int scalar_mode, int variant, cudaStream_t stream);

#define SBG_GDECL(T)                                                                        \
    void gkinds_##T(int threads, GKindInfo* out);                                           \
    sbgemm_status grun_##T(const GIn*, int, const void*, const void*, int, int, int,        \
                           const GConfig&, cudaStream_t);
SBG_GDECL(S) SBG_GDECL(D) SBG_GDECL(C) SBG_GDECL(Z) SBG_GDECL(H) SBG_GDECL(B)
#undef SBG_GDECL

namespace {

// launch configuration per storage type (sbgemm_grouped_config)
GConfig g_config[6] = {kGDefault, kGDefault, kGDefault, kGDefault, kGDefault, kGDefault};

bool gkinds(int type, int threads, GKindInfo* k) {
    switch (type) {
    case SBGEMM_TYPE_S: gkinds_S(threads, k); return true;
    case SBGEMM_TYPE_D: gkinds_D(threads, k); return true;
    case SBGEMM_TYPE_C: gkinds_C(threads, k); return true;
    case SBGEMM_TYPE_Z: gkinds_Z(threads, k); return true;
    case SBGEMM_TYPE_H: gkinds_H(threads, k); return true;
    case SBGEMM_TYPE_B: gkinds_B(threads, k); return true;
    default: return false;
    }
}

sbgemm_status grun(int type, const GIn* in, int n, const void* alpha, const void* beta, int mode,
                   int bz, int az, const GConfig& c, cudaStream_t s) {
    switch (type) {
    case SBGEMM_TYPE_S: return grun_S(in, n, alpha, beta, mode, bz, az, c, s);
    case SBGEMM_TYPE_D: return grun_D(in, n, alpha, beta, mode, bz, az, c, s);
    case SBGEMM_TYPE_C: return grun_C(in, n, alpha, beta, mode, bz, az, c, s);
    case SBGEMM_TYPE_Z: return grun_Z(in, n, alpha, beta, mode, bz, az, c, s);
    case SBGEMM_TYPE_H: return grun_H(in, n, alpha, beta, mode, bz, az, c, s);
    case SBGEMM_TYPE_B: return grun_B(in, n, alpha, beta, mode, bz, az, c, s);
    default: return SBGEMM_ERR_INVALID_VALUE;
    }
}

bool host_zero(int type, const void* p) {
    switch (type) {
    case SBGEMM_TYPE_D: return *static_cast<const double*>(p) == 0.0;
    case SBGEMM_TYPE_C: { const float* f = static_cast<const float*>(p); return f[0] == 0.f && f[1] == 0.f; }
    case SBGEMM_TYPE_Z: { const double* d = static_cast<const double*>(p); return d[0] == 0.0 && d[1] == 0.0; }
    default: return *static_cast<const float*>(p) == 0.f;
    }
}

bool is_n(char t) { return t == 'N' || t == 'n'; }
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace
}  // namespace sbg

extern "C" sbgemm_status sbgemm_gemm_grouped(int type, const void* alpha, const void* beta,
                                             const sbgemm_group* groups, int ngroups,
                                             int scalar_mode, void* stream) {
    using namespace sbg;
    GKindInfo kinfo[16];
    if (type < SBGEMM_TYPE_S || type > SBGEMM_TYPE_B) return SBGEMM_ERR_INVALID_VALUE;
    const GConfig cfg = g_config[type];
    if (!gkinds(type, cfg.threads, kinfo)) return SBGEMM_ERR_INVALID_VALUE;
    if (scalar_mode != SBGEMM_SCALARS_HOST && scalar_mode != SBGEMM_SCALARS_DEVICE)
        return SBGEMM_ERR_INVALID_VALUE;
    if (ngroups < 0) return SBGEMM_ERR_INVALID_SIZE;
    if (ngroups == 0) return SBGEMM_SUCCESS;
    if (!groups || !alpha || !beta) return SBGEMM_ERR_NULL_POINTER;
    cudaStream_t s = (cudaStream_t)stream;
    // every group's arguments are checked before anything is queued
    for (int i = 0; i < ngroups; ++i) {
        const sbgemm_group& G = groups[i];
        const sbgemm_status st = gemm_uniform(type, G.transa, G.transb, G.m, G.n, G.k, alpha, G.A,
                                              G.lda, G.lda2, G.B, G.ldb, G.ldb2, beta, G.C, G.ldc,
                                              G.ldc2, 0, scalar_mode, -1, s);
        if (st != SBGEMM_SUCCESS) return st;
        if (G.batchCount < 0) return SBGEMM_ERR_INVALID_SIZE;
        if (G.batchCount > 0 && G.m > 0 && G.n > 0 && !G.C) return SBGEMM_ERR_NULL_POINTER;
    }
    int bz = 0, az = 0;
    if (scalar_mode == SBGEMM_SCALARS_HOST) {
        bz = host_zero(type, beta);
        az = host_zero(type, alpha);
    }
    GIn fused[kGMaxGroups];
    int nf = 0;
    auto flush = [&]() -> sbgemm_status {
        if (nf == 0) return SBGEMM_SUCCESS;
        const sbgemm_status st = grun(type, fused, nf, alpha, beta, scalar_mode, bz, az, cfg, s);
        nf = 0;
        return st;
    };
    for (int i = 0; i < ngroups; ++i) {
        const sbgemm_group& G = groups[i];
        if (G.batchCount == 0 || G.m == 0 || G.n == 0) continue;
        const int m = G.m;
        bool fuse = !az && is_n(G.transa) && is_n(G.transb) && G.n == m && G.k == m && m >= 1 &&
                    G.lda == m && G.ldb == m && G.ldc == m && G.lda2 == (long long)m * m &&
                    G.ldb2 == (long long)m * m && G.ldc2 == (long long)m * m && G.A && G.B &&
                    aligned16(G.A) && aligned16(G.B) && aligned16(G.C);
        if (fuse) {
            const GKindInfo& k = kinfo[m - 1];
            fuse = k.ok && gtile_pairs(k, bz != 0, cfg) > 0;
        }
        // fp64 and complex128 classes that the selector sends to the
        // tensor-core kernel (large sizes: up to 2.1x / 2.6x the fp64 FMA
        // pipe) run as their own uniform call, which takes that kernel
        if (fuse && (type == SBGEMM_TYPE_D || type == SBGEMM_TYPE_Z) &&
            select_variant(type, m, m, m, 0, 0, bz, size_class(G.batchCount)) == kMmaVariant)
            fuse = false;
        if (fuse) {
            fused[nf++] = GIn{G.A, G.B, G.C, m, (long long)G.batchCount};
            if (nf == kGMaxGroups) {
                const sbgemm_status st = flush();
                if (st != SBGEMM_SUCCESS) return st;
            }
        } else {
            const sbgemm_status st = gemm_uniform(type, G.transa, G.transb, G.m, G.n, G.k, alpha,
                                                  G.A, G.lda, G.lda2, G.B, G.ldb, G.ldb2, beta,
                                                  G.C, G.ldc, G.ldc2, G.batchCount, scalar_mode,
                                                  -1, s);
            if (st != SBGEMM_SUCCESS) return st;
        }
    }
    return flush();
}

extern "C" sbgemm_status sbgemm_grouped_config(int type, int threads, int stage_bytes, int stages) {
    using namespace sbg;
    if (type < SBGEMM_TYPE_S || type > SBGEMM_TYPE_B) return SBGEMM_ERR_INVALID_VALUE;
    if (threads == 0 && stage_bytes == 0 && stages == 0) {
        g_config[type] = kGDefault;
        return SBGEMM_SUCCESS;
    }
    const GConfig c = {threads, stage_bytes, stages};
    if ((threads != 128 && threads != 256) || stage_bytes < 4096 || stage_bytes > 65536 ||
        stage_bytes % 1024 != 0 || stages < 2 || stages > 4 || gsmem_bytes(c) > 220 * 1024)
        return SBGEMM_ERR_INVALID_VALUE;
    g_config[type] = c;
    return SBGEMM_SUCCESS;
}
