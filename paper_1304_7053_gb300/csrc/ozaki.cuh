// fp64 batched GEMM on the tensor cores by exact integer splitting (an
// Ozaki-type scheme: Ozaki, Ogita, Oishi & Rump, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication
// and its applications", Numer. Algorithms 59, 2012).
//
// Eq. (1) of the paper for real fp64 (the d entry points), m, n, k <= 16.
// GB300's fp64 FMA pipe (about 1.26 TFLOP/s) bounds the direct kernels far
// below the HBM roofline; this kernel moves the products to the fp16 tensor
// cores instead:
//   1. Row i of op(A) is scaled by 2^(63 - e_i) and column j of op(B) by
//      2^(63 - f_j), where 2^e_i > max_l |a_il| and 2^f_j > max_l |b_lj|, and
//      truncated to 64-bit integers X (exact for every entry within 2^-11 of
//      its row or column maximum).
//   2. Each |X| is split into eight unsigned 8-bit digits,
//      |X| = sum_s U_s 2^(56 - 8s), U_0 < 128; with the sign of the entry
//      every digit is an integer of magnitude at most 255, exact in binary16.
//   3. For every digit pair (s, t) with s + t <= 7 (36 of the 64), one
//      m16n8k16 MMA per 8 columns adds the exact integer product
//      D^A_s D^B_t (k terms of at most 2^16) into the fp32 accumulator of
//      diagonal d = s + t; no fp32 accumulator sums more than four such
//      products (diagonals 4..7 use two), so every value stays below 2^22
//      and every accumulation is exact.
//   4. The eight diagonal sums are combined exactly in 64-bit integers (two
//      partial sums of under 2^48) and converted to fp64 with one rounding:
//      (AB)_ij ~ 2^(e_i + f_j - 38) (S_hi + 2^-32 S_lo).
// Error: the truncation in step 1 and the dropped digit products (s + t >= 8)
// together stay below k 2^(e_i + f_j - 59).  The kernel also forms
// T_ij = sum_l |top digit of |X_a||_il |top digit of |X_b||_lj (one more MMA),
// a lower bound of (|A||B|)_ij 2^(14 - e_i - f_j); T_ij >= 512 guarantees
// that the emulation error is at most (k/2) u (|A||B|)_ij (u = 2^-53), so the
// result meets the elementwise bound (k/2 + 3) u (|alpha||A||B| + |beta||C|)
// including the final roundings.  Entries that fail the test (an output whose
// row and column are dominated by entries of very different sizes, or whose
// row of op(A) or column of op(B) is zero or subnormal), and every pair with
// a non-finite input, are recomputed with fp64 FMAs: always correct, at the
// fp64 pipe's speed for those entries.
//
// One warp computes one pair (a 16 x 16 x 16 product; smaller shapes read
// zeros outside m x k and k x n); a persistent grid of warps walks the batch.
#pragma once

#include "sbgemm_launch.cuh"

namespace sbg {

// One problem of a record list (the variable-size path): element offsets of
// its A, B and C from the arena bases, flags (bits 0-1 op(A), 2-3 op(B):
// 0 N, 1 T, 2 C; bit 4: C not read, as if beta were 0) and shape
// (m | n << 8 | k << 16); matrices stored with minimal leading dimensions.
struct OzRec {
    long long a, b, c;
    int flags;
    int shape;
};

struct OzArgs {
    const OzRec* recs;      // record list (source 1): g.batch records
    const double* const* Ap; const double* const* Bp;   // pointer arrays (source 2)
    double* const* Cp;
    const double* A; const double* B; double* C;
    long long lda2, ldb2, ldc2;
    int lda, ldb, ldc;
    int m, n, k;
    int ta, tb;             // stored transposed (op = T, or C on a real type)
    long long batch;
    double alpha, beta;     // host scalars (when the pointers are null)
    const double* alpha_ptr;
    const double* beta_ptr;
    int beta_zero;          // host mode: beta == 0 known on the host
};

__device__ __forceinline__ void oz_mma(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
                 "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// biased exponent field of x (0 for zero and subnormals, 0x7FF for Inf/NaN)
__device__ __forceinline__ int oz_expf(double x) {
    return (__double2hiint(x) >> 20) & 0x7FF;
}

// |x| 2^(63 - e) truncated toward zero, for |x| < 2^e (e = field - 1022 of
// the largest exponent field of the row or column), and the sign of x:
// integer operations only.
__device__ __forceinline__ unsigned long long oz_mag(double x, int e, bool* neg) {
    const long long bits = __double_as_longlong(x);
    *neg = bits < 0;
    const int E = (int)((bits >> 52) & 0x7FF);
    const unsigned long long frac = (unsigned long long)bits & 0xFFFFFFFFFFFFFull;
    // |x| = mant 2^(E - 1075);  |X| = mant 2^(E - 1075 + 63 - e), shift <= 10
    const int sh = E - 1012 - e;
    if (E != 0 && sh >= 0) return (frac | (1ull << 52)) << sh;      // the common case
    const unsigned long long mant = E ? (frac | (1ull << 52)) : frac;
    const int s2 = E ? sh : sh + 1;                                  // subnormals: exponent 1 - 1075
    if (s2 >= 0) return mant << s2;
    return s2 > -64 ? mant >> (-s2) : 0ull;
}

// Byte 7 - s of two magnitudes (digit s, 0 = top) as the binary16 halves
// 1024 + byte of one register (first value in the low half).
template <int s>
__device__ __forceinline__ unsigned oz_bytes(unsigned long long x0, unsigned long long x1) {
    constexpr int b = 7 - s;
    const unsigned w0 = b >= 4 ? (unsigned)(x0 >> 32) : (unsigned)x0;
    const unsigned w1 = b >= 4 ? (unsigned)(x1 >> 32) : (unsigned)x1;
    constexpr unsigned sel = (unsigned)(b & 3) | ((unsigned)(4 + (b & 3)) << 8);
    return (__byte_perm(w0, w1, sel) & 0x00FF00FFu) | 0x64006400u;
}

// signed digit pair: sgn * (h - 1024) = h sgn + nb with nb = -1024 sgn, exact
__device__ __forceinline__ unsigned oz_signed(unsigned v, __half2 sgn, __half2 nb) {
    const __half2 r = __hfma2(*reinterpret_cast<const __half2*>(&v), sgn, nb);
    return *reinterpret_cast<const unsigned*>(&r);
}

// per-register sign factors (+-1 for each half) and their -1024 multiples
__device__ __forceinline__ void oz_signs(bool n0, bool n1, __half2* sgn, __half2* nb) {
    const unsigned short p1 = 0x3C00, m1 = 0xBC00, p1024 = 0x6400, m1024 = 0xE400;
    *sgn = __halves2half2(__ushort_as_half(n0 ? m1 : p1), __ushort_as_half(n1 ? m1 : p1));
    *nb = __halves2half2(__ushort_as_half(n0 ? p1024 : m1024), __ushort_as_half(n1 ? p1024 : m1024));
}

// fp32 holding an integer of magnitude below 2^22 -> that integer
__device__ __forceinline__ int oz_int(float f) {
    return __float_as_int(f + 12582912.0f) - 0x4B400000;
}

// An accumulator that starts at kOzBias = 1.5 * 2^23 holds bias + v for the
// integer v it has summed (|v| < 2^22): every value lies in [2^23, 2^24),
// where fp32 represents each integer exactly, so the MMAs stay exact and v
// is the bit pattern minus that of the bias (no add needed to read it back).
constexpr float kOzBias = 12582912.0f;
__device__ __forceinline__ int oz_unbias(float f) {
    return __float_as_int(f) - 0x4B400000;
}

// The double nearest to (S_hi 2^32 + S_lo) 2^(sc - 32) (|S_hi|, |S_lo| <
// 2^48), assembled with integer operations (round to nearest even); results
// outside the normal range go through ldexp.
__device__ __forceinline__ double oz_assemble(long long shi, long long slo, int sc) {
    // V = S_hi 2^32 + S_lo as a 128-bit two's-complement value (vh:vl)
    const unsigned long long sl = (unsigned long long)shi << 32;
    unsigned long long vl = sl + (unsigned long long)slo;
    long long vh = (shi >> 32) + (vl < sl ? 1 : 0) + (slo < 0 ? -1 : 0);
    const bool neg = vh < 0;
    unsigned long long mh = (unsigned long long)vh, ml = vl;
    if (neg) {                                     // magnitude
        ml = ~ml + 1ull;
        mh = ~mh + (ml == 0 ? 1ull : 0ull);
    }
    if ((mh | ml) == 0) return 0.0;
    int P;                                         // position of the leading bit
    unsigned long long mant;
    bool rnd = false, sticky = false;
    if (mh) {
        P = 127 - __clzll((long long)mh);          // 64..81
        const int sh = P - 52;                     // 12..29
        mant = (mh << (64 - sh)) | (ml >> sh);
        rnd = (ml >> (sh - 1)) & 1ull;
        sticky = (ml & ((1ull << (sh - 1)) - 1ull)) != 0;
    } else {
        P = 63 - __clzll((long long)ml);
        if (P > 52) {
            const int sh = P - 52;
            mant = ml >> sh;
            rnd = (ml >> (sh - 1)) & 1ull;
            sticky = (ml & ((1ull << (sh - 1)) - 1ull)) != 0;
        } else {
            mant = ml << (52 - P);
        }
    }
    if (rnd && (sticky || (mant & 1ull))) {
        ++mant;
        if (mant >> 53) { mant >>= 1; ++P; }
    }
    const int biased = P + sc - 32 + 1023;         // value = 1.f 2^(P + sc - 32)
    if (biased >= 1 && biased <= 2046)
        return __longlong_as_double((long long)(((unsigned long long)neg << 63) |
                                                ((unsigned long long)biased << 52) |
                                                (mant & 0xFFFFFFFFFFFFFull)));
    const double v = ldexp((double)mant, P - 52 + sc - 32);
    return neg ? -v : v;
}

// EM: the epilogue, fixed per launch (a run-time select made the compiler
// evaluate alpha * v for every entry on the slow fp64 pipe):
// 0 C = v (alpha = 1, beta = 0), 1 C = alpha v (beta = 0), 2 the general case.
// SRC: where pair p's matrices are: 0 the uniform 3-D batch (base + p * ld2),
// 1 a record list (per-problem offsets, shape, ops and beta flag), 2 device
// arrays of per-pair pointers (the pointer-array form; uniform shape).
template <int NT, int EM, int SRC = 0>
__global__ void __launch_bounds__(NT, 3) ozaki_kernel(OzArgs g)
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    double alpha = g.alpha_ptr ? *g.alpha_ptr : g.alpha;
    double beta = g.beta_ptr ? *g.beta_ptr : g.beta;
    const bool beta_zero = g.beta_ptr ? beta == 0.0 : g.beta_zero != 0;
    const int lane = threadIdx.x & 31;
    const int gq = lane >> 2, tq = lane & 3;
    const long long warp = (blockIdx.x * (long long)NT + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * NT) >> 5;
    // the current pair's shape, ops, leading dimensions and beta flag
    int m = g.m, n = g.n, k = g.k;
    int ta = g.ta, tb = g.tb, lda = g.lda, ldb = g.ldb, ldc = g.ldc;
    bool bzp = beta_zero;                 // this pair's C is not read
    auto pair = [&](long long p, const double*& Ap, const double*& Bp, double*& Cp) {
        if constexpr (SRC == 1) {
            const OzRec r = g.recs[p];
            Ap = g.A + r.a; Bp = g.B + r.b; Cp = g.C + r.c;
            m = r.shape & 255; n = (r.shape >> 8) & 255; k = (r.shape >> 16) & 255;
            ta = (r.flags & 3) != 0; tb = ((r.flags >> 2) & 3) != 0;
            lda = ta ? k : m; ldb = tb ? n : k; ldc = m;
            bzp = beta_zero || (r.flags & 16) != 0;
        } else if constexpr (SRC == 2) {
            Ap = g.Ap[p]; Bp = g.Bp[p]; Cp = g.Cp[p];
        } else {
            Ap = g.A + p * g.lda2; Bp = g.B + p * g.ldb2; Cp = g.C + p * g.ldc2;
        }
    };
    if constexpr (EM == 2) {
        // an alpha of 0 read from the device (or, for a record list, given
        // on the host): C = beta C (0 when beta == 0), A and B unread
        if (alpha == 0.0) {
            for (long long p = warp; p < g.batch; p += nwarps) {
                const double *Ap, *Bp;
                double* Cp;
                pair(p, Ap, Bp, Cp);
                for (int e = lane; e < m * n; e += 32) {
                    double* c = Cp + e % m + (long long)ldc * (e / m);
                    *c = bzp ? 0.0 : beta * *c;
                }
            }
            return;
        }
    }

    // op(A)(i, l) and op(B)(l, j) of pair p, zero outside the shape
    auto ldA = [&](const double* Ap, int i, int l) -> double {
        if (i >= m || l >= k) return 0.0;
        return ta ? Ap[l + (long long)lda * i] : Ap[i + (long long)lda * l];
    };
    auto ldB = [&](const double* Bp, int l, int j) -> double {
        if (l >= k || j >= n) return 0.0;
        return tb ? Bp[j + (long long)ldb * l] : Bp[l + (long long)ldb * j];
    };

    for (long long p = warp; p < g.batch; p += nwarps) {
        const double *Ap, *Bp;
        double* Cp;
        pair(p, Ap, Bp, Cp);
        // this lane's operand entries (the m16n8k16 fragment positions):
        // A rows gq, gq+8, columns 2tq, 2tq+1, 2tq+8, 2tq+9;
        // B rows 2tq, 2tq+1, 2tq+8, 2tq+9, columns gq (nh = 0), gq+8 (nh = 1)
        double a[8], b[2][4];
        a[0] = ldA(Ap, gq, 2 * tq);         a[1] = ldA(Ap, gq, 2 * tq + 1);
        a[2] = ldA(Ap, gq + 8, 2 * tq);     a[3] = ldA(Ap, gq + 8, 2 * tq + 1);
        a[4] = ldA(Ap, gq, 2 * tq + 8);     a[5] = ldA(Ap, gq, 2 * tq + 9);
        a[6] = ldA(Ap, gq + 8, 2 * tq + 8); a[7] = ldA(Ap, gq + 8, 2 * tq + 9);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = gq + 8 * h;
            b[h][0] = ldB(Bp, 2 * tq, j);     b[h][1] = ldB(Bp, 2 * tq + 1, j);
            b[h][2] = ldB(Bp, 2 * tq + 8, j); b[h][3] = ldB(Bp, 2 * tq + 9, j);
        }
        // row exponents (rows gq, gq + 8) and column exponents (columns gq,
        // gq + 8): the largest exponent field over the quad of lanes that
        // holds the row or column
        int ra0 = max(max(oz_expf(a[0]), oz_expf(a[1])), max(oz_expf(a[4]), oz_expf(a[5])));
        int ra1 = max(max(oz_expf(a[2]), oz_expf(a[3])), max(oz_expf(a[6]), oz_expf(a[7])));
        int cb0 = max(max(oz_expf(b[0][0]), oz_expf(b[0][1])), max(oz_expf(b[0][2]), oz_expf(b[0][3])));
        int cb1 = max(max(oz_expf(b[1][0]), oz_expf(b[1][1])), max(oz_expf(b[1][2]), oz_expf(b[1][3])));
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            ra0 = max(ra0, __shfl_xor_sync(0xffffffffu, ra0, o));
            ra1 = max(ra1, __shfl_xor_sync(0xffffffffu, ra1, o));
            cb0 = max(cb0, __shfl_xor_sync(0xffffffffu, cb0, o));
            cb1 = max(cb1, __shfl_xor_sync(0xffffffffu, cb1, o));
        }
        const bool nonfinite = __any_sync(0xffffffffu, ra0 == 0x7FF || ra1 == 0x7FF ||
                                                       cb0 == 0x7FF || cb1 == 0x7FF);
        // e = field - 1022: 2^e exceeds every entry of the row or column
        const int ea0 = ra0 - 1022, ea1 = ra1 - 1022, eb0 = cb0 - 1022, eb1 = cb1 - 1022;

        // the column exponents of this lane's outputs live in the lanes whose
        // gq is that column (mod 8)
        int ecol[2][2];
#pragma unroll
        for (int x = 0; x < 2; ++x) {
            const int src = (2 * tq + x) * 4;
            ecol[0][x] = __shfl_sync(0xffffffffu, eb0, src);
            ecol[1][x] = __shfl_sync(0xffffffffu, eb1, src);
        }
        unsigned fa[8][4];          // A digit fragments of every slice
        unsigned fta[4];            // top digits of |X| of A (the accuracy test)
        if (!nonfinite) {
            unsigned long long xa[8];
            bool na[8];
            xa[0] = oz_mag(a[0], ea0, &na[0]); xa[1] = oz_mag(a[1], ea0, &na[1]);
            xa[2] = oz_mag(a[2], ea1, &na[2]); xa[3] = oz_mag(a[3], ea1, &na[3]);
            xa[4] = oz_mag(a[4], ea0, &na[4]); xa[5] = oz_mag(a[5], ea0, &na[5]);
            xa[6] = oz_mag(a[6], ea1, &na[6]); xa[7] = oz_mag(a[7], ea1, &na[7]);
            __half2 sg[4], nb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) oz_signs(na[2 * q], na[2 * q + 1], &sg[q], &nb[q]);
            const __half2 c1024 = __half2half2(__ushort_as_half((unsigned short)0x6400));
#define OZ_AFRAG(S)                                                                      \
            _Pragma("unroll") for (int q = 0; q < 4; ++q)                                \
                fa[S][q] = oz_signed(oz_bytes<S>(xa[2 * q], xa[2 * q + 1]), sg[q], nb[q]);
            OZ_AFRAG(0) OZ_AFRAG(1) OZ_AFRAG(2) OZ_AFRAG(3)
            OZ_AFRAG(4) OZ_AFRAG(5) OZ_AFRAG(6) OZ_AFRAG(7)
#undef OZ_AFRAG
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const unsigned v = oz_bytes<0>(xa[2 * q], xa[2 * q + 1]);
                const __half2 r = __hsub2(*reinterpret_cast<const __half2*>(&v), c1024);
                fta[q] = *reinterpret_cast<const unsigned*>(&r);
            }
        }
        // column halves h = 0 (columns 0..7) and 1 (8..15) one after the other
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (8 * h >= n) break;
            long long shi[4], slo[4];
            unsigned use = 0;
            // the old C of this half's outputs, loaded before the products so
            // the load latency is hidden behind them (general epilogue only)
            double cold[4] = {0.0, 0.0, 0.0, 0.0};
            if constexpr (EM == 2) {
                if (!bzp) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int i = gq + 8 * (r >> 1), j = 2 * tq + (r & 1) + 8 * h;
                        if (i < m && j < n) cold[r] = Cp[i + (long long)ldc * j];
                    }
                }
            }
            if (!nonfinite) {
                const int eb = h ? eb1 : eb0;
                unsigned long long xb[4];
                bool nbq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) xb[q] = oz_mag(b[h][q], eb, &nbq[q]);
                __half2 sg[2], nb[2];
                oz_signs(nbq[0], nbq[1], &sg[0], &nb[0]);
                oz_signs(nbq[2], nbq[3], &sg[1], &nb[1]);
                const __half2 c1024 = __half2half2(__ushort_as_half((unsigned short)0x6400));
                {
                    float tacc[4] = {0.f, 0.f, 0.f, 0.f};
                    const unsigned v0 = oz_bytes<0>(xb[0], xb[1]), v1 = oz_bytes<0>(xb[2], xb[3]);
                    const __half2 r0 = __hsub2(*reinterpret_cast<const __half2*>(&v0), c1024);
                    const __half2 r1 = __hsub2(*reinterpret_cast<const __half2*>(&v1), c1024);
                    oz_mma(tacc, fta, *reinterpret_cast<const unsigned*>(&r0),
                           *reinterpret_cast<const unsigned*>(&r1));
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (tacc[r] >= 512.f) use |= 1u << r;
                }
                unsigned fb[8][2];
#define OZ_BFRAG(T)                                                               \
                fb[T][0] = oz_signed(oz_bytes<T>(xb[0], xb[1]), sg[0], nb[0]);    \
                fb[T][1] = oz_signed(oz_bytes<T>(xb[2], xb[3]), sg[1], nb[1]);
                OZ_BFRAG(0) OZ_BFRAG(1) OZ_BFRAG(2) OZ_BFRAG(3)
                OZ_BFRAG(4) OZ_BFRAG(5) OZ_BFRAG(6) OZ_BFRAG(7)
#undef OZ_BFRAG
                // 12 fp32 accumulators: diagonals d = s + t = 0..3 one each, 4..7
                // two each (products with s < 4 and with s >= 4), so none sums
                // more than four digit products (every value stays below 2^22).
                // The 36 MMAs go out in four rounds over the 12 accumulators,
                // so dependent MMAs are 12 apart.
                float acc[12][4];
#pragma unroll
                for (int x = 0; x < 12; ++x)
#pragma unroll
                    for (int r = 0; r < 4; ++r) acc[x][r] = kOzBias;
#pragma unroll
                for (int round = 0; round < 4; ++round)
#pragma unroll
                    for (int x = 0; x < 12; ++x) {
                        // accumulator x: diagonal d (and, from d = 4, the half
                        // s < 4 or s >= 4); its round-th product is (s, d - s)
                        const int d = x < 4 ? x : 4 + (x - 4) / 2;
                        const bool upper = x >= 4 && ((x - 4) & 1);
                        const int s_ = upper ? 4 + round : round;
                        const int t = d - s_;
                        const bool ok = x < 4 ? round <= d : (upper ? s_ <= d : t <= 7);
                        if (ok && t >= 0) oz_mma(acc[x], fa[s_], fb[t][0], fb[t][1]);
                    }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    // 32-bit inner sums, then one 64-bit shift-add per partial
                    // sum: an accumulator holds at most 4 * 16 * 255^2 =
                    // 4,161,600 in magnitude, a two-accumulator sum 8,323,200,
                    // and 257 times that is below 2^31
                    const int h01 = oz_unbias(acc[0][r]) * 256 + oz_unbias(acc[1][r]);
                    const int h23 = oz_unbias(acc[2][r]) * 256 + oz_unbias(acc[3][r]);
                    const int l01 = (oz_unbias(acc[4][r]) + oz_unbias(acc[5][r])) * 256 +
                                    (oz_unbias(acc[6][r]) + oz_unbias(acc[7][r]));
                    const int l23 = (oz_unbias(acc[8][r]) + oz_unbias(acc[9][r])) * 256 +
                                    (oz_unbias(acc[10][r]) + oz_unbias(acc[11][r]));
                    shi[r] = (long long)h01 * 65536 + h23;
                    slo[r] = (long long)l01 * 65536 + l23;
                }
            }
            // outputs: rows gq (r = 0, 1) and gq + 8 (r = 2, 3), columns
            // 2tq + (r & 1) + 8h
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i = gq + 8 * (r >> 1);
                const int j = 2 * tq + (r & 1) + 8 * h;
                if (i >= m || j >= n) continue;
                double v;
                const int er = r >> 1 ? ea1 : ea0, ec = ecol[h][r & 1];
                if (!nonfinite && ((use >> r) & 1u)) {
                    v = oz_assemble(shi[r], slo[r], er + ec - 38);
                } else {
                    // fp64 FMAs for this entry (inputs out of the emulation's range)
                    v = 0.0;
                    for (int l = 0; l < k; ++l) v = fma(ldA(Ap, i, l), ldB(Bp, l, j), v);
                }
                double* c = Cp + i + (long long)ldc * j;
                if constexpr (EM == 0) *c = v;
                else if constexpr (EM == 1) *c = alpha * v;
                else *c = bzp ? alpha * v : fma(beta, cold[r], alpha * v);
            }
        }
    }
}

}  // namespace sbg
