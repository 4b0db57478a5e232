// Complex fp64 batched GEMM on the tensor cores by exact integer splitting,
// the complex counterpart of csrc/ozaki.cuh (Ozaki, Ogita, Oishi & Rump,
// Numer. Algorithms 59, 2012, applied to the four real products of a
// complex product).
//
// Eq. (1) of the paper for complex fp64 (the z entry points), m, n, k <= 16.
// With op(A) = Ar + i Ai and op(B) = Br + i Bi (conjugation folded into the
// sign of the imaginary parts),
//     op(A) op(B) = (Ar Br - Ai Bi) + i (Ar Bi + Ai Br).
//   1. Row i of op(A) (real and imaginary parts together) is scaled by
//      2^(63 - e_i) with 2^e_i above every |Re| and |Im| of the row, column
//      j of op(B) by 2^(63 - f_j), and truncated to 64-bit integers.
//   2. Each magnitude splits into eight 8-bit digits, signed by its entry
//      (exact in binary16), as in the real kernel.
//   3. Each of the four real products runs as the real kernel does: 36
//      m16n8k16 MMAs (digit pairs s + t <= 7) into 12 fp32 accumulators of at
//      most four exact products each (values below 2^22), read back as
//      integers and combined into two 64-bit partial sums.  The two products
//      of a component are added (or subtracted) exactly in 64-bit integers.
//   4. Each component is converted to fp64 with one rounding.
// Error: per real product the truncation and the dropped digit products stay
// below k 2^(e_i + f_j - 59), so each component is within 2k 2^(e_i + f_j -
// 59) of the exact one.  With the top digits U of step 2, |z| >= (|Re z| +
// |Im z|) / sqrt 2 gives (|op(A)| |op(B)|)_ij >= 2^(e_i + f_j - 15) T_ij,
// T_ij = sum_l (U(Ar_il) + U(Ai_il)) (U(Br_lj) + U(Bi_lj)), formed by one
// more MMA (operands up to 254, exact).  T_ij >= 1024 bounds the emulation
// error of each component by k u (|op(A)| |op(B)|)_ij (u = 2^-53), so the
// result meets the elementwise bound (2k + 5) u (|alpha||A||B| + |beta||C|)
// of the FMA kernels with room for the final roundings.  Entries that fail
// the test, and every pair with a non-finite input, are recomputed with
// fp64 FMAs.
//
// One warp computes one pair (a 16 x 16 x 16 complex product; smaller shapes
// read zeros outside m x k and k x n); a persistent grid walks the batch.
#pragma once

#include "ozaki.cuh"

namespace sbg {

// shared-memory slots per lane and stage of the complex kernel: 8 entries of
// op(A), 8 of op(B) and (general epilogue) the 8 old C entries of the lane's
// outputs, 16 bytes each
constexpr int kZSlots = 24;
inline constexpr size_t oz_z_smem_bytes(int threads) {
    return (size_t)(threads / 32) * 2 * kZSlots * 32 * sizeof(double2);
}

struct OzZArgs {
    const OzRec* recs;      // record list (source 1): g.batch records
    const double2* const* Ap; const double2* const* Bp;  // pointer arrays (source 2)
    double2* const* Cp;
    const double2* A; const double2* B; double2* C;
    long long lda2, ldb2, ldc2;
    int lda, ldb, ldc;
    int m, n, k;
    int ta, tb;             // stored transposed (op = T or C)
    int ca, cb;             // conjugated (op = C)
    long long batch;
    double2 alpha, beta;    // host scalars (when the pointers are null)
    const double2* alpha_ptr;
    const double2* beta_ptr;
    int beta_zero;          // host mode: beta == 0 known on the host
};

// One real digit-split product of the warp's 16 x 16 x 8 block: the 36 MMAs
// of the digit pairs s + t <= 7 into 12 accumulators (diagonals 0..3 one
// each, 4..7 two each: no accumulator sums more than four products), read
// back as integers (the accumulators start at kOzBias) and added to (neg:
// subtracted from) the two partial sums
// hi = sum_{d<4} 256^(3-d) D_d and lo = sum_{d>=4} 256^(7-d) D_d of every
// output r of the lane.
__device__ __forceinline__ void oz_product(const unsigned (&fa)[8][4], const unsigned (&fb)[8][2],
                                           long long (&hi)[4], long long (&lo)[4], bool neg) {
    float acc[12][4];
#pragma unroll
    for (int x = 0; x < 12; ++x)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[x][r] = kOzBias;
#pragma unroll
    for (int round = 0; round < 4; ++round)
#pragma unroll
        for (int x = 0; x < 12; ++x) {
            // accumulator x: diagonal d (and, from d = 4, the half s < 4 or
            // s >= 4); its round-th product is (s, d - s)
            const int d = x < 4 ? x : 4 + (x - 4) / 2;
            const bool upper = x >= 4 && ((x - 4) & 1);
            const int s_ = upper ? 4 + round : round;
            const int t = d - s_;
            const bool ok = x < 4 ? round <= d : (upper ? s_ <= d : t <= 7);
            if (ok && t >= 0) oz_mma(acc[x], fa[s_], fb[t][0], fb[t][1]);
        }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        // 32-bit inner sums, then one 64-bit shift-add per partial sum: an
        // accumulator holds at most 4 * 16 * 255^2 = 4,161,600 in magnitude,
        // a two-accumulator sum 8,323,200, and 257 times that is below 2^31
        const int h01 = oz_unbias(acc[0][r]) * 256 + oz_unbias(acc[1][r]);
        const int h23 = oz_unbias(acc[2][r]) * 256 + oz_unbias(acc[3][r]);
        const int l01 = (oz_unbias(acc[4][r]) + oz_unbias(acc[5][r])) * 256 +
                        (oz_unbias(acc[6][r]) + oz_unbias(acc[7][r]));
        const int l23 = (oz_unbias(acc[8][r]) + oz_unbias(acc[9][r])) * 256 +
                        (oz_unbias(acc[10][r]) + oz_unbias(acc[11][r]));
        const long long vh = (long long)h01 * 65536 + h23;
        const long long vl = (long long)l01 * 65536 + l23;
        hi[r] += neg ? -vh : vh;
        lo[r] += neg ? -vl : vl;
    }
}

// Signed digit fragments (all eight slices) of the lane's eight A magnitudes.
#define OZZ_FRAG8(DST, X, SG, NB)                                                  \
    _Pragma("unroll") for (int q = 0; q < 4; ++q) {                                \
        DST[0][q] = oz_signed(oz_bytes<0>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[1][q] = oz_signed(oz_bytes<1>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[2][q] = oz_signed(oz_bytes<2>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[3][q] = oz_signed(oz_bytes<3>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[4][q] = oz_signed(oz_bytes<4>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[5][q] = oz_signed(oz_bytes<5>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[6][q] = oz_signed(oz_bytes<6>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[7][q] = oz_signed(oz_bytes<7>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
    }

// Signed digit fragments (all eight slices) of the lane's four B magnitudes
// of one column half.
#define OZZ_FRAG4(DST, X, SG, NB)                                                  \
    _Pragma("unroll") for (int q = 0; q < 2; ++q) {                                \
        DST[0][q] = oz_signed(oz_bytes<0>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[1][q] = oz_signed(oz_bytes<1>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[2][q] = oz_signed(oz_bytes<2>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[3][q] = oz_signed(oz_bytes<3>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[4][q] = oz_signed(oz_bytes<4>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[5][q] = oz_signed(oz_bytes<5>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[6][q] = oz_signed(oz_bytes<6>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
        DST[7][q] = oz_signed(oz_bytes<7>(X[2 * q], X[2 * q + 1]), SG[q], NB[q]);  \
    }

// top digits of two magnitude pairs: (U(x0) + U(y0), U(x1) + U(y1)) as
// binary16 (at most 254, exact)
__device__ __forceinline__ unsigned oz_top_sum(unsigned long long x0, unsigned long long x1,
                                               unsigned long long y0, unsigned long long y1) {
    const __half2 c1024 = __half2half2(__ushort_as_half((unsigned short)0x6400));
    const unsigned vx = oz_bytes<0>(x0, x1), vy = oz_bytes<0>(y0, y1);
    const __half2 r = __hadd2(__hsub2(*reinterpret_cast<const __half2*>(&vx), c1024),
                              __hsub2(*reinterpret_cast<const __half2*>(&vy), c1024));
    return *reinterpret_cast<const unsigned*>(&r);
}

// larger of the exponent fields of the two parts of a complex entry
__device__ __forceinline__ int oz_expz(double2 z) {
    return max(oz_expf(z.x), oz_expf(z.y));
}

// EM: the epilogue, fixed per launch: 0 C = v (alpha = 1, beta = 0),
// 1 C = alpha v (beta = 0), 2 the general case.  Two blocks per SM: the
// fragments of both parts of op(A) and op(B) stay live (about 200 registers).
// SRC: where pair p's matrices are: 0 the uniform 3-D batch (base + p * ld2),
// 1 a record list (per-problem offsets, shape, ops and beta flag), 2 device
// arrays of per-pair pointers (the pointer-array form; uniform shape).
template <int NT, int EM, int SRC = 0>
__global__ void __launch_bounds__(NT, 2) ozaki_z_kernel(OzZArgs g)
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const double2 alpha = g.alpha_ptr ? *g.alpha_ptr : g.alpha;
    const double2 beta = g.beta_ptr ? *g.beta_ptr : g.beta;
    const bool beta_zero = g.beta_ptr ? (beta.x == 0.0 && beta.y == 0.0) : g.beta_zero != 0;
    const int lane = threadIdx.x & 31;
    const int gq = lane >> 2, tq = lane & 3;
    const long long warp = (blockIdx.x * (long long)NT + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * NT) >> 5;
    // one pair's operands, shape, ops, leading dimensions and beta flag
    struct Pair {
        const double2* A; const double2* B; double2* C;
        int m, n, k, ta, tb, ca, cb, lda, ldb, ldc;
        bool bz;                              // C is not read
    };
    auto pair = [&](long long p) -> Pair {
        Pair q;
        if constexpr (SRC == 1) {
            const OzRec r = g.recs[p];
            q.A = g.A + r.a; q.B = g.B + r.b; q.C = g.C + r.c;
            q.m = r.shape & 255; q.n = (r.shape >> 8) & 255; q.k = (r.shape >> 16) & 255;
            const int oa = r.flags & 3, ob = (r.flags >> 2) & 3;
            q.ta = oa != 0; q.tb = ob != 0; q.ca = oa == 2; q.cb = ob == 2;
            q.lda = q.ta ? q.k : q.m; q.ldb = q.tb ? q.n : q.k; q.ldc = q.m;
            q.bz = beta_zero || (r.flags & 16) != 0;
        } else {
            if constexpr (SRC == 2) {
                q.A = g.Ap[p]; q.B = g.Bp[p]; q.C = g.Cp[p];
            } else {
                q.A = g.A + p * g.lda2; q.B = g.B + p * g.ldb2; q.C = g.C + p * g.ldc2;
            }
            q.m = g.m; q.n = g.n; q.k = g.k;
            q.ta = g.ta; q.tb = g.tb; q.ca = g.ca; q.cb = g.cb;
            q.lda = g.lda; q.ldb = g.ldb; q.ldc = g.ldc;
            q.bz = beta_zero;
        }
        return q;
    };
    Pair cur;                                 // the pair being computed
    cur.m = cur.n = cur.k = 0;

    // op(A)(i, l) and op(B)(l, j) of the current pair (conjugated for op = C),
    // zero outside the shape
    auto ldA = [&](int i, int l) -> double2 {
        if (i >= cur.m || l >= cur.k) return make_double2(0.0, 0.0);
        double2 v = cur.ta ? cur.A[l + (long long)cur.lda * i] : cur.A[i + (long long)cur.lda * l];
        if (cur.ca) v.y = -v.y;
        return v;
    };
    auto ldB = [&](int l, int j) -> double2 {
        if (l >= cur.k || j >= cur.n) return make_double2(0.0, 0.0);
        double2 v = cur.tb ? cur.B[j + (long long)cur.ldb * l] : cur.B[l + (long long)cur.ldb * j];
        if (cur.cb) v.y = -v.y;
        return v;
    };

    // Operands of the warp's next pair are prefetched into shared memory
    // (two stages per warp, 16-byte cp.async with zero fill outside the
    // shape) while the current pair computes: slot e of lane L at
    // stage * kZSlots * 32 + e * 32 + L holds the lane's A entry e (e < 8), B
    // entry e - 8 (column half (e - 8) / 4) or, when the epilogue reads C, the
    // old C of output e - 16 (column half (e - 16) / 4); consecutive lanes
    // read consecutive 16-byte words.
    extern __shared__ __align__(16) unsigned char oz_smem[];
    double2* wbuf = reinterpret_cast<double2*>(oz_smem) + (threadIdx.x >> 5) * (2 * kZSlots * 32);
    auto prefetch = [&](long long p, int stage) {
        const Pair q = pair(p);
        double2* d = wbuf + stage * kZSlots * 32 + lane;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int i = gq + 8 * ((e >> 1) & 1), l = 2 * tq + (e & 1) + 8 * (e >> 2);
            const bool in = i < q.m && l < q.k;
            const double2* src = q.ta ? q.A + l + (long long)q.lda * i : q.A + i + (long long)q.lda * l;
            cp_async16(d + e * 32, in ? src : q.A, in ? 16 : 0);
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int l = 2 * tq + (e & 1) + 8 * ((e >> 1) & 1), j = gq + 8 * (e >> 2);
            const bool in = l < q.k && j < q.n;
            const double2* src = q.tb ? q.B + j + (long long)q.ldb * l : q.B + l + (long long)q.ldb * j;
            cp_async16(d + (8 + e) * 32, in ? src : q.B, in ? 16 : 0);
        }
        if constexpr (EM == 2) {
            if (!q.bz) {                      // the old C of the lane's outputs
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int i = gq + 8 * ((e >> 1) & 1), j = 2 * tq + (e & 1) + 8 * (e >> 2);
                    const bool in = i < q.m && j < q.n;
                    cp_async16(d + (16 + e) * 32, in ? q.C + i + (long long)q.ldc * j : q.C,
                               in ? 16 : 0);
                }
            }
        }
    };

    if constexpr (EM == 2) {
        // an alpha of 0 read from the device (or, for a record list, given
        // on the host): C = beta C (0 when beta == 0), A and B unread
        if (alpha.x == 0.0 && alpha.y == 0.0) {
            for (long long p = warp; p < g.batch; p += nwarps) {
                const Pair q = pair(p);
                for (int e = lane; e < q.m * q.n; e += 32) {
                    double2* c = q.C + e % q.m + (long long)q.ldc * (e / q.m);
                    if (q.bz) {
                        *c = make_double2(0.0, 0.0);
                    } else {
                        const double2 c0 = *c;
                        *c = make_double2(fma(beta.x, c0.x, -beta.y * c0.y),
                                          fma(beta.x, c0.y, beta.y * c0.x));
                    }
                }
            }
            return;
        }
    }
    if (warp < g.batch) prefetch(warp, 0);
    cp_async_commit();
    int stage = 0;
    for (long long p = warp; p < g.batch; p += nwarps, stage ^= 1) {
        cur = pair(p);
        const int m = cur.m, n = cur.n, k = cur.k;
        double2* Cp = cur.C;
        if (p + nwarps < g.batch) prefetch(p + nwarps, stage ^ 1);
        cp_async_commit();
        cp_async_wait_dyn(1);                 // this pair's operands have landed
        const double2* sl = wbuf + stage * kZSlots * 32 + lane;
        // the lane's fragment positions, as in the real kernel: A rows gq,
        // gq+8, columns 2tq, 2tq+1, 2tq+8, 2tq+9; B rows 2tq, 2tq+1, 2tq+8,
        // 2tq+9, columns gq (h = 0) and gq+8 (h = 1)
        double2 a[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            a[e] = sl[e * 32];
            if (cur.ca) a[e].y = -a[e].y;
        }
        auto loadB = [&](int h, double2 (&b)[4]) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                b[q] = sl[(8 + 4 * h + q) * 32];
                if (cur.cb) b[q].y = -b[q].y;
            }
        };
        // row and column exponents over both parts, reduced over the quad
        int ra0 = max(max(oz_expz(a[0]), oz_expz(a[1])), max(oz_expz(a[4]), oz_expz(a[5])));
        int ra1 = max(max(oz_expz(a[2]), oz_expz(a[3])), max(oz_expz(a[6]), oz_expz(a[7])));
        int cb0, cb1;
        {
            double2 b0[4], b1[4];
            loadB(0, b0);
            loadB(1, b1);
            cb0 = max(max(oz_expz(b0[0]), oz_expz(b0[1])), max(oz_expz(b0[2]), oz_expz(b0[3])));
            cb1 = max(max(oz_expz(b1[0]), oz_expz(b1[1])), max(oz_expz(b1[2]), oz_expz(b1[3])));
        }
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            ra0 = max(ra0, __shfl_xor_sync(0xffffffffu, ra0, o));
            ra1 = max(ra1, __shfl_xor_sync(0xffffffffu, ra1, o));
            cb0 = max(cb0, __shfl_xor_sync(0xffffffffu, cb0, o));
            cb1 = max(cb1, __shfl_xor_sync(0xffffffffu, cb1, o));
        }
        const bool nonfinite = __any_sync(0xffffffffu, ra0 == 0x7FF || ra1 == 0x7FF ||
                                                       cb0 == 0x7FF || cb1 == 0x7FF);
        const int ea0 = ra0 - 1022, ea1 = ra1 - 1022, eb0 = cb0 - 1022, eb1 = cb1 - 1022;
        unsigned fa_re[8][4], fa_im[8][4];   // digit fragments of Re and Im of op(A)
        unsigned fta[4];                 // top digits U(Re) + U(Im) of op(A)
        if (!nonfinite) {
            unsigned long long xr[8], xi[8];
            bool nr[8], ni[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = (q == 2 || q == 3 || q == 6 || q == 7) ? ea1 : ea0;
                xr[q] = oz_mag(a[q].x, e, &nr[q]);
                xi[q] = oz_mag(a[q].y, e, &ni[q]);
            }
            __half2 sgr[4], nbr[4], sgi[4], nbi[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                oz_signs(nr[2 * q], nr[2 * q + 1], &sgr[q], &nbr[q]);
                oz_signs(ni[2 * q], ni[2 * q + 1], &sgi[q], &nbi[q]);
            }
            OZZ_FRAG8(fa_re, xr, sgr, nbr)
            OZZ_FRAG8(fa_im, xi, sgi, nbi)
#pragma unroll
            for (int q = 0; q < 4; ++q) fta[q] = oz_top_sum(xr[2 * q], xr[2 * q + 1], xi[2 * q], xi[2 * q + 1]);
        }
        // the two column halves in a loop that is not unrolled: one copy of
        // the four products' code (the unrolled body overflowed the
        // instruction cache)
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            if (8 * h >= n) break;
            long long rhi[4] = {0, 0, 0, 0}, rlo[4] = {0, 0, 0, 0};   // real part
            long long ihi[4] = {0, 0, 0, 0}, ilo[4] = {0, 0, 0, 0};   // imaginary part
            unsigned use = 0;
            const int eb = h ? eb1 : eb0;
            // the column exponents of this lane's outputs live in the lanes
            // whose gq is that column (mod 8)
            int ecol[2];
#pragma unroll
            for (int x = 0; x < 2; ++x) ecol[x] = __shfl_sync(0xffffffffu, eb, (2 * tq + x) * 4);
            if (!nonfinite) {
                double2 b[4];
                loadB(h, b);
                unsigned long long yr[4], yi[4];
                bool mr[4], mi[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    yr[q] = oz_mag(b[q].x, eb, &mr[q]);
                    yi[q] = oz_mag(b[q].y, eb, &mi[q]);
                }
                {
                    float tacc[4] = {0.f, 0.f, 0.f, 0.f};
                    oz_mma(tacc, fta, oz_top_sum(yr[0], yr[1], yi[0], yi[1]),
                           oz_top_sum(yr[2], yr[3], yi[2], yi[3]));
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (tacc[r] >= 1024.f) use |= 1u << r;
                }
                __half2 sgr[2], nbr[2], sgi[2], nbi[2];
                oz_signs(mr[0], mr[1], &sgr[0], &nbr[0]);
                oz_signs(mr[2], mr[3], &sgr[1], &nbr[1]);
                oz_signs(mi[0], mi[1], &sgi[0], &nbi[0]);
                oz_signs(mi[2], mi[3], &sgi[1], &nbi[1]);
                unsigned fbr[8][2], fbi[8][2];
                OZZ_FRAG4(fbr, yr, sgr, nbr)
                OZZ_FRAG4(fbi, yi, sgi, nbi)
                oz_product(fa_re, fbr, rhi, rlo, false);    // Re: Ar Br
                oz_product(fa_im, fbi, rhi, rlo, true);     //     - Ai Bi
                oz_product(fa_re, fbi, ihi, ilo, false);    // Im: Ar Bi
                oz_product(fa_im, fbr, ihi, ilo, false);    //     + Ai Br
            }
            // outputs: rows gq (r = 0, 1) and gq + 8 (r = 2, 3), columns
            // 2tq + (r & 1) + 8h
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i = gq + 8 * (r >> 1);
                const int j = 2 * tq + (r & 1) + 8 * h;
                if (i >= m || j >= n) continue;
                double2 v;
                const int er = r >> 1 ? ea1 : ea0, ec = ecol[r & 1];
                if (!nonfinite && ((use >> r) & 1u)) {
                    v.x = oz_assemble(rhi[r], rlo[r], er + ec - 38);
                    v.y = oz_assemble(ihi[r], ilo[r], er + ec - 38);
                } else {
                    // fp64 FMAs for this entry (inputs out of the emulation's range)
                    v = make_double2(0.0, 0.0);
                    for (int l = 0; l < k; ++l) {
                        const double2 x = ldA(i, l), y = ldB(l, j);
                        v.x = fma(x.x, y.x, v.x);
                        v.x = fma(-x.y, y.y, v.x);
                        v.y = fma(x.x, y.y, v.y);
                        v.y = fma(x.y, y.x, v.y);
                    }
                }
                double2* c = Cp + i + (long long)cur.ldc * j;
                if constexpr (EM == 0) {
                    *c = v;
                } else {
                    double2 w;                        // alpha v
                    w.x = fma(alpha.x, v.x, -alpha.y * v.y);
                    w.y = fma(alpha.x, v.y, alpha.y * v.x);
                    if constexpr (EM == 2) {
                        if (!cur.bz) {                // + beta C
                            const double2 c0 = sl[(16 + 4 * h + r) * 32];
                            w.x = fma(beta.x, c0.x, fma(-beta.y, c0.y, w.x));
                            w.y = fma(beta.x, c0.y, fma(beta.y, c0.x, w.y));
                        }
                    }
                    *c = w;
                }
            }
        }
    }
    cp_async_wait_dyn(0);
}

#undef OZZ_FRAG8
#undef OZZ_FRAG4

}  // namespace sbg
