// Per-type entry: specialised shape if there is one, else the generic kernel.
#include "sbgemm_launch.cuh"
#include "sbgemm_shapes.h"

namespace sbg {

#define SBG_DECL(T) bool run_##T##_part0(const Req&, sbgemm_status*); \
                    bool run_##T##_part1(const Req&, sbgemm_status*);
SBG_DECL(S) SBG_DECL(D) SBG_DECL(C) SBG_DECL(Z) SBG_DECL(H) SBG_DECL(B)
#undef SBG_DECL

#define SBG_RUN(T)                                                         \
    sbgemm_status run_##T(const Req& r) {                                  \
        sbgemm_status st;                                                  \
        if (r.variant == kMmaVariant) {                                    \
            if (mma16_ok(r)) return run_mma16(r);                          \
            if (ozaki_ok(r)) return run_ozaki(r);                          \
            Req r0 = r;                                                    \
            r0.variant = 0;                                                \
            return run_##T(r0);                                            \
        }                                                                  \
        if (r.variant < kNumPipeVariants) {                                \
            if (run_##T##_part0(r, &st)) return st;                        \
            if (run_##T##_part1(r, &st)) return st;                        \
        }                                                                  \
        return launch_generic<Ty##T>(r);                                   \
    }
SBG_RUN(S) SBG_RUN(D) SBG_RUN(C) SBG_RUN(Z) SBG_RUN(H) SBG_RUN(B)
#undef SBG_RUN

bool has_specialized(int /*type*/, int m, int n, int k) {
#define SBG_CASE(M, N, K) if (m == M && n == N && k == K) return true;
    SBG_SHAPES(SBG_CASE)
#undef SBG_CASE
    return false;
}

}  // namespace sbg
