// Variable-size persistent kernel, storage type D.
#include "vbatch.cuh"

namespace sbg {

void vkinds_D(VKindInfo* out) { vkind_table<TyD>(out); }

sbgemm_status vrun_D(const VItem* items, int n_items, const VRec* recs, int* counter,
                        const void* A, const void* B, void* C, const void* alpha,
                        const void* beta, int scalar_mode, int beta_zero, int alpha_zero,
                        cudaStream_t stream) {
    return vbatch_launch<TyD>(items, n_items, recs, counter, A, B, C, alpha, beta, scalar_mode,
                                 beta_zero, alpha_zero, stream);
}

}  // namespace sbg
