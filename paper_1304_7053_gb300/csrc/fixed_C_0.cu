// Specialised fixed-size kernels: storage type C, shape group 0.
#include "sbgemm_launch.cuh"
#include "sbgemm_shapes.h"

namespace sbg {

bool run_C_part0(const Req& r, sbgemm_status* st) {
#define SBG_CASE(M, N, K) \
    if (r.m == M && r.n == N && r.k == K) { *st = launch_shape<TyC, M, N, K>(r); return true; }
    SBG_SHAPES_PART0(SBG_CASE)
#undef SBG_CASE
    return false;
}

}  // namespace sbg
