// Launcher of the fp64 tensor-core kernel (csrc/ozaki.cuh): public variant 7
// of the real fp64 shapes with specialised kernels.
#include "ozaki.cuh"

namespace sbg {

bool ozaki_ok(const Req& r) {
    return r.type == SBGEMM_TYPE_D && !r.Cp && r.m >= 1 && r.n >= 1 && r.k >= 1;
}

sbgemm_status run_ozaki(const Req& r) {
    if (!ozaki_ok(r)) return SBGEMM_ERR_NOT_SUPPORTED;
    constexpr int NT = 128;
    OzArgs g;
    g.A = static_cast<const double*>(r.A);
    g.B = static_cast<const double*>(r.B);
    g.C = static_cast<double*>(r.C);
    g.lda2 = r.lda2; g.ldb2 = r.ldb2; g.ldc2 = r.ldc2;
    g.lda = r.lda; g.ldb = r.ldb; g.ldc = r.ldc;
    g.m = r.m; g.n = r.n; g.k = r.k;
    g.ta = r.ta; g.tb = r.tb;
    g.batch = r.batch;
    if (r.scalar_mode == SBGEMM_SCALARS_DEVICE) {
        g.alpha_ptr = static_cast<const double*>(r.alpha);
        g.beta_ptr = static_cast<const double*>(r.beta);
        g.alpha = 0.0; g.beta = 0.0; g.beta_zero = 0;
    } else {
        g.alpha_ptr = nullptr; g.beta_ptr = nullptr;
        g.alpha = *static_cast<const double*>(r.alpha);
        g.beta = *static_cast<const double*>(r.beta);
        g.beta_zero = r.beta_zero;
    }
    // epilogue: C = v, C = alpha v, or the general form (device scalars)
    const int em = r.scalar_mode == SBGEMM_SCALARS_DEVICE ? 2
                 : !r.beta_zero ? 2 : (g.alpha == 1.0 ? 0 : 1);
    auto kern = em == 0 ? ozaki_kernel<NT, 0> : em == 1 ? ozaki_kernel<NT, 1> : ozaki_kernel<NT, 2>;
    const size_t smem = 0;
    static thread_local OccCache occ[3];
    int per_sm = 0;
    cudaError_t e = blocks_per_sm(kern, NT, smem, occ[em], &per_sm);
    if (e != cudaSuccess) return (sbgemm_status)e;
    if (per_sm < 1) return SBGEMM_ERR_NOT_SUPPORTED;
    // one warp per pair at a time
    long long grid = (long long)num_sms() * per_sm;
    const long long need = ((long long)r.batch + NT / 32 - 1) / (NT / 32);
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(NT);
    lc.dynamicSmemBytes = smem;
    lc.stream = r.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    e = cudaLaunchKernelEx(&lc, kern, g);
    if (e != cudaSuccess) return (sbgemm_status)e;
    return (sbgemm_status)cudaGetLastError();
}

}  // namespace sbg
