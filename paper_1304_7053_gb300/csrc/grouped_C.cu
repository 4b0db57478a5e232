// Grouped persistent kernel, storage type C.
#include "grouped.cuh"

namespace sbg {

void gkinds_C(int threads, GKindInfo* out) { gkind_table<TyC>(threads, out); }

sbgemm_status grun_C(const GIn* in, int n, const void* alpha, const void* beta, int scalar_mode,
                        int beta_zero, int alpha_zero, const GConfig& cfg, cudaStream_t stream) {
    return grouped_launch<TyC>(in, n, alpha, beta, scalar_mode, beta_zero, alpha_zero, cfg, stream);
}

}  // namespace sbg
