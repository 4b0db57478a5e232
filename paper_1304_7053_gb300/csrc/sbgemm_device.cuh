// Device code for batched small-matrix GEMM on sm_103a.
//
// Operation (arXiv 1304.7053, Section 2, Eq. 1), for every pair p:
//     C_p <- alpha * op(A_p) * op(B_p) + beta * C_p
// on the uniform 3-D layout of Section 4: X_p(i, j) = X[i + ldx*j + ldx2*p].
//
// Kernel structure (the design is ours; the paper's Kepler kernels are prior
// art only):
//   * A persistent grid walks tiles of P consecutive pairs (grid-stride).
//   * Each tile's A, B (and old C when beta != 0) are staged into shared
//     memory by a STAGES-deep cp.async pipeline.  When an operand is a flat
//     stream (minimal leading dimensions, 16-byte aligned), the tile is one
//     contiguous span copied in coalesced 16-byte chunks; matrices whose
//     byte size is an even number of 16-byte chunks get a one-chunk pad per
//     matrix slot so neighbouring matrices start in different bank groups.
//     Other layouts are gathered element by element (still asynchronous).
//   * Each thread owns a TM x TN block of one C_p and keeps it in
//     registers; op() is applied by the index map used to read shared
//     memory (Section 2), conjugation by a sign on the imaginary part
//     (Section 5 "conjugate" functor).
//   * The epilogue is alpha*acc when beta == 0, where C is never read
//     (Section 5 "axpby_a1b0"), else alpha*acc + beta*C_old (Section 5
//     "axpby").  Results go to a shared-memory tile and leave in coalesced
//     16-byte stores.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace sbg {

// ------------------------------------------------------------ scalar types

// Storage type S, arithmetic type A (fp32 for the 16-bit storage types).
struct TyS { using S = float;   using A = float;   using R = float;  static constexpr bool cplx = false; static constexpr int code = 0; };
struct TyD { using S = double;  using A = double;  using R = double; static constexpr bool cplx = false; static constexpr int code = 1; };
struct TyC { using S = float2;  using A = float2;  using R = float;  static constexpr bool cplx = true;  static constexpr int code = 2; };
struct TyZ { using S = double2; using A = double2; using R = double; static constexpr bool cplx = true;  static constexpr int code = 3; };
struct TyH { using S = __half;        using A = float; using R = float; static constexpr bool cplx = false; static constexpr int code = 4; };
struct TyB { using S = __nv_bfloat16; using A = float; using R = float; static constexpr bool cplx = false; static constexpr int code = 5; };

__device__ __forceinline__ float  to_a(float x)  { return x; }
__device__ __forceinline__ double to_a(double x) { return x; }
__device__ __forceinline__ float2 to_a(float2 x) { return x; }
__device__ __forceinline__ double2 to_a(double2 x) { return x; }
__device__ __forceinline__ float  to_a(__half x) { return __half2float(x); }
__device__ __forceinline__ float  to_a(__nv_bfloat16 x) { return __bfloat162float(x); }

template <class Ty> __device__ __forceinline__ typename Ty::S to_s(typename Ty::A x);
template <> __device__ __forceinline__ float   to_s<TyS>(float x)   { return x; }
template <> __device__ __forceinline__ double  to_s<TyD>(double x)  { return x; }
template <> __device__ __forceinline__ float2  to_s<TyC>(float2 x)  { return x; }
template <> __device__ __forceinline__ double2 to_s<TyZ>(double2 x) { return x; }
template <> __device__ __forceinline__ __half  to_s<TyH>(float x)   { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 to_s<TyB>(float x) { return __float2bfloat16_rn(x); }

template <class A> __device__ __forceinline__ A zero_a();
template <> __device__ __forceinline__ float   zero_a<float>()   { return 0.f; }
template <> __device__ __forceinline__ double  zero_a<double>()  { return 0.0; }
template <> __device__ __forceinline__ float2  zero_a<float2>()  { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 zero_a<double2>() { return make_double2(0.0, 0.0); }

// acc += a * b  (fused; complex uses the 4-multiply form, no 3M method,
// matching the flop convention of Section 7)
__device__ __forceinline__ void mac(float& c, float a, float b)   { c = fmaf(a, b, c); }
__device__ __forceinline__ void mac(double& c, double a, double b) { c = fma(a, b, c); }
__device__ __forceinline__ void mac(float2& c, float2 a, float2 b) {
    c.x = fmaf(a.x, b.x, c.x); c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y); c.y = fmaf(a.y, b.x, c.y);
}
__device__ __forceinline__ void mac(double2& c, double2 a, double2 b) {
    c.x = fma(a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y); c.y = fma(a.y, b.x, c.y);
}

// Conjugation (Section 5 "conjugate" functor): the imaginary part's sign
// bit is flipped when s is -1.  The flip is an integer XOR, so it costs no
// floating-point pipe slot (the fp64 pipe is the bound for complex double).
// Identity for real types.
__device__ __forceinline__ float   conj_s(float a, float)     { return a; }
__device__ __forceinline__ double  conj_s(double a, double)   { return a; }
__device__ __forceinline__ float2  conj_s(float2 a, float s) {
    const unsigned m = __float_as_uint(s) & 0x80000000u;
    return make_float2(a.x, __uint_as_float(__float_as_uint(a.y) ^ m));
}
__device__ __forceinline__ double2 conj_s(double2 a, double s) {
    const unsigned long long m = (unsigned long long)__double_as_longlong(s) & 0x8000000000000000ull;
    return make_double2(a.x, __longlong_as_double((long long)((unsigned long long)__double_as_longlong(a.y) ^ m)));
}

// alpha * x
__device__ __forceinline__ float   mul(float a, float x)     { return a * x; }
__device__ __forceinline__ double  mul(double a, double x)   { return a * x; }
__device__ __forceinline__ float2  mul(float2 a, float2 x)   { return make_float2(fmaf(a.x, x.x, -a.y * x.y), fmaf(a.x, x.y, a.y * x.x)); }
__device__ __forceinline__ double2 mul(double2 a, double2 x) { return make_double2(fma(a.x, x.x, -a.y * x.y), fma(a.x, x.y, a.y * x.x)); }
// v + b * c
__device__ __forceinline__ float   axpy(float b, float c, float v)       { return fmaf(b, c, v); }
__device__ __forceinline__ double  axpy(double b, double c, double v)    { return fma(b, c, v); }
__device__ __forceinline__ float2  axpy(float2 b, float2 c, float2 v) {
    v.x = fmaf(b.x, c.x, v.x); v.x = fmaf(-b.y, c.y, v.x);
    v.y = fmaf(b.x, c.y, v.y); v.y = fmaf(b.y, c.x, v.y);
    return v;
}
__device__ __forceinline__ double2 axpy(double2 b, double2 c, double2 v) {
    v.x = fma(b.x, c.x, v.x); v.x = fma(-b.y, c.y, v.x);
    v.y = fma(b.x, c.y, v.y); v.y = fma(b.y, c.x, v.y);
    return v;
}
__device__ __forceinline__ bool is_zero(float a)   { return a == 0.f; }
__device__ __forceinline__ bool is_zero(double a)  { return a == 0.0; }
__device__ __forceinline__ bool is_zero(float2 a)  { return a.x == 0.f && a.y == 0.f; }
__device__ __forceinline__ bool is_zero(double2 a) { return a.x == 0.0 && a.y == 0.0; }
__device__ __forceinline__ bool is_one(float a)    { return a == 1.f; }
__device__ __forceinline__ bool is_one(double a)   { return a == 1.0; }
__device__ __forceinline__ bool is_one(float2 a)   { return a.x == 1.f && a.y == 0.f; }
__device__ __forceinline__ bool is_one(double2 a)  { return a.x == 1.0 && a.y == 0.0; }

// ------------------------------------------------------------ async copies

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// 16-byte global -> shared copy; bytes beyond src_bytes are zero-filled and
// not read from global memory.
__device__ __forceinline__ void cp_async16(void* s, const void* g, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n"
                 :: "r"(smem_u32(s)), "l"(g), "r"(src_bytes) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* s, const void* g) {
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n"
                 :: "r"(smem_u32(s)), "l"(g), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_dyn(int pending) {
    // pending = number of most recent groups allowed to stay in flight
    if (pending <= 0)      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    else if (pending == 1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else if (pending == 2) asm volatile("cp.async.wait_group 2;\n" ::: "memory");
    else                   asm volatile("cp.async.wait_group 3;\n" ::: "memory");
}

// ------------------------------------------------------------ bulk copies (TMA, 1-D)

// Spin limit of every mbarrier wait: each try_wait may itself suspend the
// thread for a while, so this bounds a wait to well under a second of a
// healthy copy's latency many times over; on expiry the kernel records
// SBGEMM_ERR_TIMEOUT in the caller's error word and stops.
constexpr long long kSpinLimit = 1ll << 22;

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}
// make initialised barriers visible to the asynchronous (copy) proxy
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// one arrival that also announces `bytes` of copies completing on the barrier
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                 :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// wait for the phase with the given parity to complete; false when `limit`
// polls have not seen it
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit = kSpinLimit) {
    const unsigned a = smem_u32(bar);
    for (long long i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
// global -> shared bulk copy completing on `bar` (16-byte aligned addresses,
// size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* sdst, const void* gsrc, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 :: "r"(smem_u32(sdst)), "l"(gsrc), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// shared -> global bulk copy in the issuing thread's bulk group
__device__ __forceinline__ void bulk_s2g(void* gdst, const void* ssrc, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n"
                 :: "l"(gdst), "r"(smem_u32(ssrc)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// the issuing thread's bulk stores have read their shared-memory source
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// the issuing thread's bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// order this thread's shared-memory writes before later copy-proxy reads
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Stage `cnt` consecutive matrices of a flat operand (SE elements each,
// matrix p0 at g + p0*SE, 16-byte aligned) into slots of SP elements with
// bulk copies on `bar`: one copy of the whole span when the slots are
// unpadded (a ragged end of under 16 bytes is copied by thread 0 with plain
// loads), one copy per matrix when they are padded.  Returns the bytes that
// complete on the barrier (the same on every thread).
template <class S, int SE, int SP, int NT>
__device__ __forceinline__ unsigned stage_bulk(S* sdst, const S* g, long long p0, int cnt, uint64_t* bar) {
    constexpr int ES = sizeof(S);
    const S* src = g + p0 * (long long)SE;
    // (the callers' tile geometry makes both ends 16-byte aligned; should
    // that ever fail, the tile is copied with plain loads instead)
    if (((reinterpret_cast<uintptr_t>(src) | smem_u32(sdst)) & 15) != 0) {
        for (int e = threadIdx.x; e < cnt * SE; e += NT) sdst[(e / SE) * SP + e % SE] = src[e];
        return 0;
    }
    if constexpr (SP == SE) {
        const unsigned nbytes = (unsigned)(cnt * SE * ES);
        const unsigned body = nbytes & ~15u;
        if (threadIdx.x == 0) {
            if (body) bulk_g2s(sdst, src, body, bar);
            for (unsigned e = body / ES; e < nbytes / ES; ++e) sdst[e] = src[e];
        }
        return body;
    } else {
        static_assert((SE * ES) % 16 == 0, "padded slots hold whole 16-byte chunks");
        for (int q = threadIdx.x; q < cnt; q += NT) bulk_g2s(sdst + q * SP, src + q * SE, SE * ES, bar);
        return (unsigned)(cnt * SE * ES);
    }
}

// Write `cnt` result matrices from slots of SP elements to a flat C with
// bulk stores (the issuing threads commit a bulk group each); a ragged end
// of under 16 bytes is written by thread 0 directly.  The slots must have
// been written before a fence_proxy_async and a block barrier.
template <class S, int SE, int SP, int NT>
__device__ __forceinline__ void store_bulk(S* g, const S* ssrc, long long p0, int cnt) {
    constexpr int ES = sizeof(S);
    S* dst = g + p0 * (long long)SE;
    if (((reinterpret_cast<uintptr_t>(dst) | smem_u32(ssrc)) & 15) != 0) {
        for (int e = threadIdx.x; e < cnt * SE; e += NT) dst[e] = ssrc[(e / SE) * SP + e % SE];
        return;
    }
    if constexpr (SP == SE) {
        const unsigned nbytes = (unsigned)(cnt * SE * ES);
        const unsigned body = nbytes & ~15u;
        if (threadIdx.x == 0) {
            if (body) { bulk_s2g(dst, ssrc, body); bulk_commit(); }
            for (unsigned e = body / ES; e < nbytes / ES; ++e) dst[e] = ssrc[e];
        }
    } else {
        static_assert((SE * ES) % 16 == 0, "padded slots hold whole 16-byte chunks");
        if ((int)threadIdx.x < cnt) {
            for (int q = threadIdx.x; q < cnt; q += NT) bulk_s2g(dst + q * SE, ssrc + q * SP, SE * ES);
            bulk_commit();
        }
    }
}

// ------------------------------------------------------------ launch args

template <class Ty>
struct Args {
    using S = typename Ty::S;
    using A = typename Ty::A;
    const S* A_; const S* B_; S* C_;
    long long lda2, ldb2, ldc2;
    int lda, ldb, ldc;
    int batch;
    A alpha, beta;               // host scalars (used when the pointers are null)
    const A* alpha_ptr;          // device scalars (SBGEMM_SCALARS_DEVICE)
    const A* beta_ptr;
    typename Ty::R conja, conjb; // +1 or -1: sign applied to imaginary parts
    int flat;                    // bit 0: A flat, bit 1: B flat, bit 2: C flat
    int shared;                  // bit 0: one A for every pair (lda2 == 0), bit 1: one B (ldb2 == 0)
    // pointer-array form (Section 4's TGEMM_multi_nounif): matrix p of X at
    // Xp[p] with leading dimension ldx; null for the uniform 3-D layout
    const S* const* Ap; const S* const* Bp; S* const* Cp;
    int beta_zero;               // host mode: beta == 0 known on the host
    int alpha_zero;              // host mode: alpha == 0 known on the host
    int P;                       // pairs per tile
    int stages;                  // pipeline depth (2..4)
    int* err;                    // device error word (SBGEMM_ERR_TIMEOUT on an expired wait)
};

// Pad a matrix slot by one 16-byte chunk when its byte size is an even number
// of chunks, so consecutive matrices begin in different shared-memory bank
// groups.  Odd-chunk and non-chunk-multiple sizes stay unpadded.
__host__ __device__ constexpr int padded_elems(int elems, int es) {
    return ((elems * es) % 16 == 0 && ((elems * es) / 16) % 2 == 0) ? elems + 16 / es : elems;
}

__host__ __device__ constexpr int gcd_c(int a, int b) { return b ? gcd_c(b, a % b) : a; }
__host__ __device__ constexpr int lcm_c(int a, int b) { return a / gcd_c(a, b) * b; }

// Largest vector (elements, at most 16 bytes) dividing a, b and c.
__host__ __device__ constexpr int pick_vec(int es, int a, int b, int c) {
    for (int v = 16 / es; v >= 1; v /= 2)
        if (v * es <= 16 && a % v == 0 && b % v == 0 && c % v == 0) return v;
    return 1;
}

// Compile-time kernel configuration.  TM x TN: the block of C one thread
// owns; SI / SJ: rows / columns assigned to threads strided (i = ti + TI*r)
// instead of in contiguous blocks (i = ti*TM + r); NT: threads per block.
// The tile of each (type, shape, op) comes from the cost model in
// gen_tiles.py (tile_table.h); the vector widths below follow the same rules.
template <class Ty_, int M_, int N_, int K_, bool TA_, bool TB_, int TM_, int TN_,
          bool SI_, bool SJ_, int NT_, int UL_ = 0>
struct Cfg {
    using Ty = Ty_;
    using S = typename Ty::S;
    using A = typename Ty::A;
    using R = typename Ty::R;
    static constexpr int M = M_, N = N_, K = K_, TM = TM_, TN = TN_, NT = NT_;
    static constexpr bool TA = TA_, TB = TB_, SI = SI_, SJ = SJ_;
    static constexpr int TI = (M + TM - 1) / TM, TJ = (N + TN - 1) / TN, TPM = TI * TJ;
    static constexpr bool RAG_I = TI * TM != M, RAG_J = TJ * TN != N;
    static constexpr int MPR = NT / TPM;   // matrices per compute round
    static constexpr int ES = sizeof(S);
    static constexpr int SA = M * K, SB = K * N, SC = M * N;
    static constexpr int SA_P = padded_elems(SA, ES);
    static constexpr int SB_P = padded_elems(SB, ES);
    static constexpr int SC_P = padded_elems(SC, ES);
    static constexpr int RA = TA ? K : M;  // rows of stored A
    static constexpr int RB = TB ? N : K;  // rows of stored B
    // l-chunk: vectors along l for operands stored contiguous in l
    static constexpr int VL = (TA || !TB) ? pick_vec(ES, K, TA ? SA_P : K, !TB ? SB_P : K) : 1;
    // vectors along rows of A (stored m x k) / columns of B (stored n x k)
    static constexpr int VI = (!TA && !SI && !RAG_I) ? pick_vec(ES, TM, M, SA_P) : 1;
    static constexpr int VJ = (TB && !SJ && !RAG_J) ? pick_vec(ES, TN, N, SB_P) : 1;
    // direct 16-byte stores of contiguous row blocks of C (0: through a
    // shared tile and coalesced copy-out; narrower direct stores scatter
    // partial sectors across matrices and cost more L2 requests than the
    // shared-memory round trip)
    static constexpr int VS = (SI || RAG_I) ? 0
        : (TM % (16 / ES) == 0 && M % (16 / ES) == 0 && SC % (16 / ES) == 0) ? 16 / ES : 0;
    static_assert(MPR >= 1, "threads per matrix exceeds block size");
    static_assert(K % VL == 0, "l-chunk must divide k");
    // l-chunks per unrolled body of the product loop: about 128 FMAs per
    // body, so the large shapes keep a short loop instead of one fully
    // unrolled body (smaller code, fewer instruction-cache misses when
    // several shapes share one kernel); UL_ > 0 sets it explicitly
    static constexpr int UL = UL_ > 0 ? UL_ : (TM * TN * VL >= 128) ? 1 : (128 / (TM * TN * VL));
};

// ------------------------------------------------------------ staging

// Stage `cnt` consecutive matrices of one operand (first pair index `p0`)
// into a shared-memory slot array of stride SP elements.
template <class S, int SE, int SP, int ROWS, int NT>
__device__ __forceinline__ void stage_operand(S* sdst, const S* g, long long ld2, int ld,
                                              long long p0, int cnt, bool flat)
{
    constexpr int ES = sizeof(S);
    const int tid = threadIdx.x;
    if (flat) {
        // contiguous span of cnt*SE elements starting 16-byte aligned
        const char* src = reinterpret_cast<const char*>(g + p0 * (long long)SE);
        char* dst = reinterpret_cast<char*>(sdst);
        const int nbytes = cnt * SE * ES;
        const int nfull = nbytes >> 4;
        if constexpr (SP == SE) {
#pragma unroll 4
            for (int c = tid; c < nfull; c += NT) cp_async16(dst + 16 * c, src + 16 * c, 16);
        } else {
            // padded slots: chunks never straddle matrices
            constexpr int CPM = SE * ES / 16;            // chunks per matrix
#pragma unroll 4
            for (int c = tid; c < nfull; c += NT) {
                const int q = c / CPM;
                cp_async16(dst + 16 * c + q * (SP - SE) * ES, src + 16 * c, 16);
            }
        }
        if ((nbytes & 15) && tid == 0)                  // ragged last chunk, zero-filled
            cp_async16(dst + 16 * nfull, src + 16 * nfull, nbytes & 15);
    } else {
        const int n = cnt * SE;
        for (int e = tid; e < n; e += NT) {
            const int q = e / SE;
            const int r = e - q * SE;
            const int row = r % ROWS, col = r / ROWS;
            const S* src = g + (p0 + q) * ld2 + row + (long long)col * ld;
            S* dst = sdst + q * SP + r;
            if constexpr (ES == 4 || ES == 8 || ES == 16) cp_async_elem<ES>(dst, src);
            else *dst = *src;     // 16-bit storage: plain load
        }
    }
}

// Write `cnt` result matrices from shared memory (stride SP) to global C.
template <class S, int SE, int SP, int ROWS, int NT>
__device__ __forceinline__ void store_operand(S* g, const S* ssrc, long long ld2, int ld,
                                              long long p0, int cnt, bool flat)
{
    constexpr int ES = sizeof(S);
    const int tid = threadIdx.x;
    if (flat) {
        char* dst = reinterpret_cast<char*>(g + p0 * (long long)SE);
        const char* src = reinterpret_cast<const char*>(ssrc);
        const int nbytes = cnt * SE * ES;
        const int nfull = nbytes >> 4;
        if constexpr (SP == SE) {
#pragma unroll 4
            for (int c = tid; c < nfull; c += NT)
                *reinterpret_cast<uint4*>(dst + 16 * c) = *reinterpret_cast<const uint4*>(src + 16 * c);
        } else {
            constexpr int CPM = SE * ES / 16;
#pragma unroll 4
            for (int c = tid; c < nfull; c += NT) {
                const int q = c / CPM;
                *reinterpret_cast<uint4*>(dst + 16 * c) =
                    *reinterpret_cast<const uint4*>(src + 16 * c + q * (SP - SE) * ES);
            }
        }
        // ragged tail (< 16 bytes): element stores; slots are unpadded here
        // because a padded slot size is a multiple of 16 bytes
        const int e0 = (nfull << 4) / ES;
        const int e1 = nbytes / ES;
        for (int e = e0 + tid; e < e1; e += NT) {
            const int q = e / SE;
            const int r = e - q * SE;
            reinterpret_cast<S*>(dst)[e] = ssrc[q * SP + r];
        }
    } else {
        const int n = cnt * SE;
        for (int e = tid; e < n; e += NT) {
            const int q = e / SE;
            const int r = e - q * SE;
            const int row = r % ROWS, col = r / ROWS;
            g[(p0 + q) * ld2 + row + (long long)col * ld] = ssrc[q * SP + r];
        }
    }
}

// Stage a flat operand tile: with BULK and unpadded slots, one bulk copy of
// the whole span on `bar`; else 16-byte cp.async chunks (one bulk copy per
// matrix into padded slots measured slower: many small copies of 0.25-1 KB
// for fp32 m = 8, 12, 16).  Returns the bytes that complete on the barrier.
template <class S, int SE, int SP, int ROWS, int NT, bool BULK>
__device__ __forceinline__ unsigned stage_flat(S* sdst, const S* g, long long p0, int cnt, uint64_t* bar) {
    if constexpr (BULK && SP == SE) {
        return stage_bulk<S, SE, SP, NT>(sdst, g, p0, cnt, bar);
    } else {
        stage_operand<S, SE, SP, ROWS, NT>(sdst, g, SE, ROWS, p0, cnt, true);
        return 0;
    }
}

// Write a tile of results to a flat C: with BULK and unpadded slots one bulk
// store of the span, else 16-byte stores.  The caller has fenced its
// shared-memory writes (fence_proxy_async) and passed a block barrier.
template <class S, int SE, int SP, int ROWS, int NT, bool BULK>
__device__ __forceinline__ void store_flat(S* g, const S* ssrc, long long p0, int cnt) {
    if constexpr (BULK && SP == SE) store_bulk<S, SE, SP, NT>(g, ssrc, p0, cnt);
    else store_operand<S, SE, SP, ROWS, NT>(g, ssrc, SE, ROWS, p0, cnt, true);
}

// One pointer from a read-only device array, through the non-coherent
// (read-only) cache path.
template <class P>
__device__ __forceinline__ P ldg_ptr(const P* a) {
    return reinterpret_cast<P>(__ldg(reinterpret_cast<const unsigned long long*>(a)));
}

// Pointer-array staging: matrix q of the tile at sptr[q] (the tile's
// pointers, already in shared memory) with leading dimension ld.  A matrix
// stored contiguously (ld == ROWS) whose start is 16-byte aligned moves in
// 16-byte chunks; anything else moves element by element.
template <class S, int SE, int SP, int ROWS, int NT>
__device__ __forceinline__ void stage_ptrs(S* sdst, const S* const* sptr, int ld, int cnt)
{
    constexpr int ES = sizeof(S);
    const int tid = threadIdx.x;
    if constexpr ((SE * ES) % 16 == 0) {
        if (ld == ROWS) {
            constexpr int CPM = SE * ES / 16;
            constexpr int EPC = 16 / ES;
            for (int c = tid; c < cnt * CPM; c += NT) {
                const int q = c / CPM, r = c - q * CPM;
                const S* src = sptr[q] + r * EPC;
                S* dst = sdst + q * SP + r * EPC;
                if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
                    cp_async16(dst, src, 16);
                } else {
#pragma unroll
                    for (int v = 0; v < EPC; ++v) {
                        if constexpr (ES == 4 || ES == 8 || ES == 16) cp_async_elem<ES>(dst + v, src + v);
                        else dst[v] = src[v];
                    }
                }
            }
            return;
        }
    }
    for (int e = tid; e < cnt * SE; e += NT) {
        const int q = e / SE, r = e - q * SE;
        const int row = r % ROWS, col = r / ROWS;
        const S* src = sptr[q] + row + (long long)col * ld;
        S* dst = sdst + q * SP + r;
        if constexpr (ES == 4 || ES == 8 || ES == 16) cp_async_elem<ES>(dst, src);
        else *dst = *src;
    }
}

// Write cnt result matrices (slot stride SP) to the matrices at sptr[q].
template <class S, int SE, int SP, int ROWS, int NT>
__device__ __forceinline__ void store_ptrs(S* const* sptr, const S* ssrc, int ld, int cnt)
{
    constexpr int ES = sizeof(S);
    const int tid = threadIdx.x;
    if constexpr ((SE * ES) % 16 == 0) {
        if (ld == ROWS) {
            constexpr int CPM = SE * ES / 16;
            constexpr int EPC = 16 / ES;
            for (int c = tid; c < cnt * CPM; c += NT) {
                const int q = c / CPM, r = c - q * CPM;
                S* dst = sptr[q] + r * EPC;
                const S* src = ssrc + q * SP + r * EPC;
                if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
                    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
                } else {
#pragma unroll
                    for (int v = 0; v < EPC; ++v) dst[v] = src[v];
                }
            }
            return;
        }
    }
    for (int e = tid; e < cnt * SE; e += NT) {
        const int q = e / SE, r = e - q * SE;
        const int row = r % ROWS, col = r / ROWS;
        sptr[q][row + (long long)col * ld] = ssrc[q * SP + r];
    }
}

// ------------------------------------------------------------ compute

// V consecutive storage elements from 16/8/4-byte aligned shared memory in
// one vector load, converted to the arithmetic type.
template <int V, class S, class A>
__device__ __forceinline__ void ldvec(const S* p, A* out) {
    constexpr int BYTES = V * (int)sizeof(S);
    if constexpr (V > 1 && BYTES == 16) {
        union { uint4 u; S e[V]; } x;
        x.u = *reinterpret_cast<const uint4*>(p);
#pragma unroll
        for (int v = 0; v < V; ++v) out[v] = to_a(x.e[v]);
    } else if constexpr (V > 1 && BYTES == 8) {
        union { uint2 u; S e[V]; } x;
        x.u = *reinterpret_cast<const uint2*>(p);
#pragma unroll
        for (int v = 0; v < V; ++v) out[v] = to_a(x.e[v]);
    } else if constexpr (V > 1 && BYTES == 4) {
        union { uint32_t u; S e[V]; } x;
        x.u = *reinterpret_cast<const uint32_t*>(p);
#pragma unroll
        for (int v = 0; v < V; ++v) out[v] = to_a(x.e[v]);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) out[v] = to_a(p[v]);
    }
}

// V consecutive storage elements to 16/8/4-byte aligned memory in one store.
template <int V, class S>
__device__ __forceinline__ void stvec(S* p, const S* in) {
    constexpr int BYTES = V * (int)sizeof(S);
    if constexpr (V > 1 && BYTES == 16) {
        union { uint4 u; S e[V]; } x;
#pragma unroll
        for (int v = 0; v < V; ++v) x.e[v] = in[v];
        *reinterpret_cast<uint4*>(p) = x.u;
    } else if constexpr (V > 1 && BYTES == 8) {
        union { uint2 u; S e[V]; } x;
#pragma unroll
        for (int v = 0; v < V; ++v) x.e[v] = in[v];
        *reinterpret_cast<uint2*>(p) = x.u;
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) p[v] = in[v];
    }
}

// One thread: its TM x TN block (ti, tj) of matrix q of the staged tile.
// op(A)(i, l) = TA ? A[l + K i] : A[i + M l];  op(B)(l, j) = TB ? B[j + N l] : B[l + K j]
// (Section 2 op, Section 4 layout with minimal leading dimensions).
// direct: write C straight to gC (matrix q at gC + q*SC) with vector stores,
// else to the shared tile sOut.  sh bit 0 / bit 1: every pair reads the one
// A / B slot at sA / sB (a matrix shared by the whole batch).
template <class Cf>
__device__ __forceinline__ void compute_block(const typename Cf::S* __restrict__ sA,
                                              const typename Cf::S* __restrict__ sB,
                                              const typename Cf::S* __restrict__ sCold,
                                              typename Cf::S* __restrict__ sOut,
                                              typename Cf::S* __restrict__ gC, bool direct,
                                              int q, int ti, int tj,
                                              typename Cf::A alpha, typename Cf::A beta,
                                              bool beta_zero, bool alpha_one, bool skip_ab,
                                              typename Cf::R conja, typename Cf::R conjb,
                                              int sh = 0)
{
    using S = typename Cf::S;
    using A = typename Cf::A;
    constexpr int M = Cf::M, N = Cf::N, K = Cf::K, TM = Cf::TM, TN = Cf::TN;
    constexpr int TI = Cf::TI, TJ = Cf::TJ, VL = Cf::VL, VI = Cf::VI, VJ = Cf::VJ;
    const S* a = sA + ((sh & 1) ? 0 : q * Cf::SA_P);
    const S* b = sB + ((sh & 2) ? 0 : q * Cf::SB_P);

    int ri[TM], cj[TN];   // clamped row / column of each block entry
#pragma unroll
    for (int r = 0; r < TM; ++r) {
        const int i = Cf::SI ? ti + TI * r : ti * TM + r;
        ri[r] = i < M ? i : M - 1;
    }
#pragma unroll
    for (int c = 0; c < TN; ++c) {
        const int j = Cf::SJ ? tj + TJ * c : tj * TN + c;
        cj[c] = j < N ? j : N - 1;
    }

    A acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = zero_a<A>();

    if (!skip_ab) {
#pragma unroll Cf::UL
        for (int l0 = 0; l0 < K; l0 += VL) {
            A av[TM][VL], bv[TN][VL];
            if constexpr (Cf::TA) {
#pragma unroll
                for (int r = 0; r < TM; ++r) ldvec<VL>(a + K * ri[r] + l0, av[r]);
            } else {
#pragma unroll
                for (int dl = 0; dl < VL; ++dl)
#pragma unroll
                    for (int rg = 0; rg < TM; rg += VI) {
                        A t[VI];
                        ldvec<VI>(a + ri[rg] + M * (l0 + dl), t);
#pragma unroll
                        for (int v = 0; v < VI; ++v) av[rg + v][dl] = t[v];
                    }
            }
            if constexpr (!Cf::TB) {
#pragma unroll
                for (int c = 0; c < TN; ++c) ldvec<VL>(b + K * cj[c] + l0, bv[c]);
            } else {
#pragma unroll
                for (int dl = 0; dl < VL; ++dl)
#pragma unroll
                    for (int cg = 0; cg < TN; cg += VJ) {
                        A t[VJ];
                        ldvec<VJ>(b + cj[cg] + N * (l0 + dl), t);
#pragma unroll
                        for (int v = 0; v < VJ; ++v) bv[cg + v][dl] = t[v];
                    }
            }
#pragma unroll
            for (int dl = 0; dl < VL; ++dl) {
#pragma unroll
                for (int r = 0; r < TM; ++r) av[r][dl] = conj_s(av[r][dl], conja);
#pragma unroll
                for (int c = 0; c < TN; ++c) bv[c][dl] = conj_s(bv[c][dl], conjb);
#pragma unroll
                for (int r = 0; r < TM; ++r)
#pragma unroll
                    for (int c = 0; c < TN; ++c) mac(acc[r][c], av[r][dl], bv[c][dl]);
            }
        }
    }

    // epilogue: alpha*acc, plus beta*C_old unless beta == 0 (C then unread).
    // The three cases are separate loops so no per-element select remains.
    if (skip_ab) {
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
            for (int c = 0; c < TN; ++c) acc[r][c] = zero_a<A>();
    } else if (!alpha_one) {
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
            for (int c = 0; c < TN; ++c) acc[r][c] = mul(alpha, acc[r][c]);
    }
    const S* co = sCold + q * Cf::SC_P;
    if constexpr (Cf::VS > 0) {
        if (direct) {
            constexpr int VS = Cf::VS;
            S* g = gC + (long long)q * Cf::SC;
#pragma unroll
            for (int c = 0; c < TN; ++c) {
                const int j = Cf::SJ ? tj + TJ * c : tj * TN + c;
                if (Cf::RAG_J && j >= N) continue;
#pragma unroll
                for (int rg = 0; rg < TM; rg += VS) {
                    const int i0 = ti * TM + rg;
                    S out[VS];
                    if (beta_zero) {
#pragma unroll
                        for (int v = 0; v < VS; ++v) out[v] = to_s<typename Cf::Ty>(acc[rg + v][c]);
                    } else {
                        A cold[VS];
                        ldvec<VS>(co + i0 + M * j, cold);
#pragma unroll
                        for (int v = 0; v < VS; ++v)
                            out[v] = to_s<typename Cf::Ty>(axpy(beta, cold[v], acc[rg + v][c]));
                    }
                    stvec<VS>(g + i0 + M * j, out);
                }
            }
            return;
        }
    }
    S* o = sOut + q * Cf::SC_P;
    if (beta_zero) {
#pragma unroll
        for (int r = 0; r < TM; ++r) {
            const int i = Cf::SI ? ti + TI * r : ti * TM + r;
#pragma unroll
            for (int c = 0; c < TN; ++c) {
                const int j = Cf::SJ ? tj + TJ * c : tj * TN + c;
                if ((Cf::RAG_I && i >= M) || (Cf::RAG_J && j >= N)) continue;
                o[i + M * j] = to_s<typename Cf::Ty>(acc[r][c]);
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < TM; ++r) {
            const int i = Cf::SI ? ti + TI * r : ti * TM + r;
#pragma unroll
            for (int c = 0; c < TN; ++c) {
                const int j = Cf::SJ ? tj + TJ * c : tj * TN + c;
                if ((Cf::RAG_I && i >= M) || (Cf::RAG_J && j >= N)) continue;
                o[i + M * j] = to_s<typename Cf::Ty>(axpy(beta, to_a(co[i + M * j]), acc[r][c]));
            }
        }
    }
}

}  // namespace sbg
