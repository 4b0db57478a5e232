// Shapes with compile-time specialised kernels.  Every other (m, n, k) with
// m, n, k <= 16 runs on the generic run-time-size kernel.
//   - square sizes 1..16 (the paper's experiments, Section 7);
//   - rectangular shapes typical of high-order finite elements, the
//     application the paper targets (Section 1), built natively instead of
//     from square sub-blocks (Section 6).
#pragma once

#define SBG_SHAPES_PART0(X) \
    X(1, 1, 1) X(2, 2, 2) X(3, 3, 3) X(4, 4, 4) X(5, 5, 5) X(6, 6, 6) X(7, 7, 7) \
    X(8, 8, 8) X(9, 9, 9) X(10, 10, 10) X(3, 9, 3) X(4, 16, 4) X(16, 16, 1)
#define SBG_SHAPES_PART1(X) \
    X(11, 11, 11) X(12, 12, 12) X(13, 13, 13) X(14, 14, 14) X(15, 15, 15) X(16, 16, 16) \
    X(9, 16, 9) X(16, 8, 16)
#define SBG_SHAPES(X) SBG_SHAPES_PART0(X) SBG_SHAPES_PART1(X)
