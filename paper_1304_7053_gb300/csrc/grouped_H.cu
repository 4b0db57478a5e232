// Grouped persistent kernel, storage type H.
#include "grouped.cuh"

namespace sbg {

void gkinds_H(int threads, GKindInfo* out) { gkind_table<TyH>(threads, out); }

sbgemm_status grun_H(const GIn* in, int n, const void* alpha, const void* beta, int scalar_mode,
                        int beta_zero, int alpha_zero, const GConfig& cfg, cudaStream_t stream) {
    return grouped_launch<TyH>(in, n, alpha, beta, scalar_mode, beta_zero, alpha_zero, cfg, stream);
}

}  // namespace sbg
