// Specialised fixed-size kernels: storage type Z, shape group 1.
#include "sbgemm_launch.cuh"
#include "sbgemm_shapes.h"

namespace sbg {

bool run_Z_part1(const Req& r, sbgemm_status* st) {
#define SBG_CASE(M, N, K) \
    if (r.m == M && r.n == N && r.k == K) { *st = launch_shape<TyZ, M, N, K>(r); return true; }
    SBG_SHAPES_PART1(SBG_CASE)
#undef SBG_CASE
    return false;
}

}  // namespace sbg
