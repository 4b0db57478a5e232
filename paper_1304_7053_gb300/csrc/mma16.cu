// Tensor-core path of the 16-bit storage types (binary16, bfloat16).
#include "mma16.cuh"

namespace sbg {

sbgemm_status run_mma16(const Req& r) {
    if (!mma16_eligible(r)) return SBGEMM_ERR_NOT_SUPPORTED;
    const bool b = r.type == SBGEMM_TYPE_B;
    if (r.m == 16) return b ? launch_mma16<TyB, 16>(r) : launch_mma16<TyH, 16>(r);
    if (r.m == 12) return b ? launch_mma16<TyB, 12>(r) : launch_mma16<TyH, 12>(r);
    return b ? launch_mma16<TyB, 8>(r) : launch_mma16<TyH, 8>(r);
}

}  // namespace sbg

namespace sbg {
bool mma16_ok(const Req& r) { return mma16_eligible(r); }
}  // namespace sbg
