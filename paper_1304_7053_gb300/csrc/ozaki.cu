// Launchers of the fp64 tensor-core kernels (csrc/ozaki.cuh for real fp64,
// csrc/ozaki_z.cuh for complex fp64): variant 7 of the shapes with
// specialised kernels, variant 1 of the others.
#include <cstring>

#include "ozaki_z.cuh"

namespace sbg {

bool ozaki_ok(const Req& r) {
    return (r.type == SBGEMM_TYPE_D || r.type == SBGEMM_TYPE_Z) && r.m >= 1 &&
           r.n >= 1 && r.k >= 1;
}

namespace {

// Persistent grid of one warp per pair at a time, programmatic dependent
// launch.
template <class Kern, class Args>
sbgemm_status launch_oz(Kern kern, const Args& g, int NT, size_t smem, long long batch,
                        OccCache& occ, cudaStream_t stream) {
    int per_sm = 0;
    cudaError_t e = blocks_per_sm(kern, NT, smem, occ, &per_sm);
    if (e != cudaSuccess) return (sbgemm_status)e;
    if (per_sm < 1) return SBGEMM_ERR_NOT_SUPPORTED;
    long long grid = (long long)num_sms() * per_sm;
    const long long need = (batch + NT / 32 - 1) / (NT / 32);
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(NT);
    lc.dynamicSmemBytes = smem;
    lc.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    e = cudaLaunchKernelEx(&lc, kern, g);
    if (e != cudaSuccess) return (sbgemm_status)e;
    return (sbgemm_status)cudaGetLastError();
}

sbgemm_status run_ozaki_z(const Req& r) {
    constexpr int NT = 128;
    OzZArgs g;
    std::memset(&g, 0, sizeof g);
    g.A = static_cast<const double2*>(r.A);
    g.B = static_cast<const double2*>(r.B);
    g.C = static_cast<double2*>(r.C);
    g.lda2 = r.lda2; g.ldb2 = r.ldb2; g.ldc2 = r.ldc2;
    g.lda = r.lda; g.ldb = r.ldb; g.ldc = r.ldc;
    g.m = r.m; g.n = r.n; g.k = r.k;
    g.ta = r.ta; g.tb = r.tb;
    g.ca = r.conja; g.cb = r.conjb;
    g.batch = r.batch;
    if (r.scalar_mode == SBGEMM_SCALARS_DEVICE) {
        g.alpha_ptr = static_cast<const double2*>(r.alpha);
        g.beta_ptr = static_cast<const double2*>(r.beta);
        g.alpha = make_double2(0.0, 0.0); g.beta = make_double2(0.0, 0.0); g.beta_zero = 0;
    } else {
        g.alpha_ptr = nullptr; g.beta_ptr = nullptr;
        g.alpha = *static_cast<const double2*>(r.alpha);
        g.beta = *static_cast<const double2*>(r.beta);
        g.beta_zero = r.beta_zero;
    }
    const bool alpha_one = g.alpha.x == 1.0 && g.alpha.y == 0.0;
    const int em = r.scalar_mode == SBGEMM_SCALARS_DEVICE ? 2
                 : !r.beta_zero ? 2 : (alpha_one ? 0 : 1);
    // per kernel instantiation: epilogue x (3-D layout, pointer arrays)
    static thread_local OccCache occ[6];
    static DeviceFlags attr[6];
    // the pointer-array form reads pair p's matrices through the arrays
    const bool ptrs = r.Cp != nullptr;
    const int ki = em + (ptrs ? 3 : 0);
    if (ptrs) {
        g.Ap = reinterpret_cast<const double2* const*>(r.Ap);
        g.Bp = reinterpret_cast<const double2* const*>(r.Bp);
        g.Cp = reinterpret_cast<double2* const*>(r.Cp);
    }
    auto kern = ptrs ? (em == 0 ? ozaki_z_kernel<NT, 0, 2> : em == 1 ? ozaki_z_kernel<NT, 1, 2>
                                                                     : ozaki_z_kernel<NT, 2, 2>)
                     : (em == 0 ? ozaki_z_kernel<NT, 0> : em == 1 ? ozaki_z_kernel<NT, 1>
                                                                  : ozaki_z_kernel<NT, 2>);
    const size_t smem = oz_z_smem_bytes(NT);
    cudaError_t e = ensure_smem_limit(kern, (int)smem, attr[ki]);
    if (e != cudaSuccess) return (sbgemm_status)e;
    return launch_oz(kern, g, NT, smem, r.batch, occ[ki], r.stream);
}

}  // namespace

static_assert(sizeof(OzRec) == 32, "OzRec mirrors the variable-size path's record layout");

// The problems of a record list (element offsets from the arena bases A, B,
// C; flags and shape per problem) on the tensor-core kernel of real or
// complex fp64: the variable-size path's problems whose class takes it.
sbgemm_status run_ozaki_records(int type, const void* recs, long long count, const void* A,
                                const void* B, void* C, const void* alpha, const void* beta,
                                int scalar_mode, int beta_zero, cudaStream_t stream) {
    constexpr int NT = 128;
    if (count <= 0) return SBGEMM_SUCCESS;
    const bool dev = scalar_mode == SBGEMM_SCALARS_DEVICE;
    if (type == SBGEMM_TYPE_D) {
        OzArgs g;
        std::memset(&g, 0, sizeof g);
        g.recs = static_cast<const OzRec*>(recs);
        g.A = static_cast<const double*>(A);
        g.B = static_cast<const double*>(B);
        g.C = static_cast<double*>(C);
        g.batch = count;
        if (dev) {
            g.alpha_ptr = static_cast<const double*>(alpha);
            g.beta_ptr = static_cast<const double*>(beta);
        } else {
            g.alpha = *static_cast<const double*>(alpha);
            g.beta = *static_cast<const double*>(beta);
            g.beta_zero = beta_zero;
        }
        // a host alpha of 0 takes the general epilogue, which scales C
        const int em = dev || !beta_zero || g.alpha == 0.0 ? 2 : (g.alpha == 1.0 ? 0 : 1);
        auto kern = em == 0 ? ozaki_kernel<NT, 0, 1>
                  : em == 1 ? ozaki_kernel<NT, 1, 1> : ozaki_kernel<NT, 2, 1>;
        static thread_local OccCache occ[3];
        return launch_oz(kern, g, NT, 0, count, occ[em], stream);
    }
    if (type == SBGEMM_TYPE_Z) {
        OzZArgs g;
        std::memset(&g, 0, sizeof g);
        g.recs = static_cast<const OzRec*>(recs);
        g.A = static_cast<const double2*>(A);
        g.B = static_cast<const double2*>(B);
        g.C = static_cast<double2*>(C);
        g.batch = count;
        if (dev) {
            g.alpha_ptr = static_cast<const double2*>(alpha);
            g.beta_ptr = static_cast<const double2*>(beta);
        } else {
            g.alpha = *static_cast<const double2*>(alpha);
            g.beta = *static_cast<const double2*>(beta);
            g.beta_zero = beta_zero;
        }
        const bool a0 = g.alpha.x == 0.0 && g.alpha.y == 0.0;
        const bool a1 = g.alpha.x == 1.0 && g.alpha.y == 0.0;
        const int em = dev || !beta_zero || a0 ? 2 : (a1 ? 0 : 1);
        auto kern = em == 0 ? ozaki_z_kernel<NT, 0, 1>
                  : em == 1 ? ozaki_z_kernel<NT, 1, 1> : ozaki_z_kernel<NT, 2, 1>;
        static thread_local OccCache occ[3];
        static DeviceFlags attr[3];
        const size_t smem = oz_z_smem_bytes(NT);
        cudaError_t e = ensure_smem_limit(kern, (int)smem, attr[em]);
        if (e != cudaSuccess) return (sbgemm_status)e;
        return launch_oz(kern, g, NT, smem, count, occ[em], stream);
    }
    return SBGEMM_ERR_NOT_SUPPORTED;
}

sbgemm_status run_ozaki(const Req& r) {
    if (!ozaki_ok(r)) return SBGEMM_ERR_NOT_SUPPORTED;
    if (r.type == SBGEMM_TYPE_Z) return run_ozaki_z(r);
    constexpr int NT = 128;
    OzArgs g;
    std::memset(&g, 0, sizeof g);
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
    const bool ptrs = r.Cp != nullptr;
    if (ptrs) {
        g.Ap = reinterpret_cast<const double* const*>(r.Ap);
        g.Bp = reinterpret_cast<const double* const*>(r.Bp);
        g.Cp = reinterpret_cast<double* const*>(r.Cp);
    }
    auto kern = ptrs ? (em == 0 ? ozaki_kernel<NT, 0, 2> : em == 1 ? ozaki_kernel<NT, 1, 2>
                                                                   : ozaki_kernel<NT, 2, 2>)
                     : (em == 0 ? ozaki_kernel<NT, 0> : em == 1 ? ozaki_kernel<NT, 1>
                                                                : ozaki_kernel<NT, 2>);
    static thread_local OccCache occ[6];       // epilogue x (3-D layout, pointer arrays)
    return launch_oz(kern, g, NT, 0, r.batch, occ[em + (ptrs ? 3 : 0)], r.stream);
}

}  // namespace sbg
