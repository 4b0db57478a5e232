// Tensor-core kernel for 16-bit storage (binary16 / bfloat16 with fp32
// accumulation), square m = n = k = 8, 12 or 16, op N/N, flat batches.
//
// Every pair's product is one or two warp-level mma.sync m16n8k16
// operations (fp32 accumulators).  With column-major storage (Section 4),
// C^T = B^T A^T: the memory of B read row by row is B^T in the row-major
// layout the MMA's A operand takes, and A's memory is A^T; the MMA's result
// rows are columns of C, so each thread ends with pairs of C entries that
// are adjacent in memory (one 32-bit store each).
//   m = 16: per pair, A operand = B^T (16 x 16), two n8 tiles of A^T,
//           fragments loaded with ldmatrix (A^T with .trans).
//   m = 12: as m = 16 with zero fragments for rows and columns 12..15; the
//           fragments come from 32-bit and 16-bit shared loads (24-byte
//           columns give no 16-byte rows for ldmatrix) at per-lane offsets
//           and masks fixed before the loop, so the loads are branch-free;
//           each warp takes two pairs per iteration, their loads and MMAs
//           issued before either pair's stores.
//   m = 8:  two pairs per MMA, packed block-diagonally: A operand =
//           diag(B0^T, B1^T) (16 x 16), B operand = [A0^T; A1^T] (16 x 8),
//           result [C0^T; C1^T] (the off-diagonal fragment registers are 0).
// The tiles of pairs move through a cp.async pipeline; m = 16 operand slots
// are stored with their two 16-byte halves of rows 4..7 and 12..15 swapped
// (an XOR swizzle), which makes every 8 x 8 ldmatrix conflict-free.
#pragma once

#include "sbgemm_launch.cuh"

namespace sbg {

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], unsigned addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], unsigned addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(unsigned (&r)[2], unsigned addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n"
                 : "=r"(r[0]), "=r"(r[1]) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned (&r)[2], unsigned addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];\n"
                 : "=r"(r[0]), "=r"(r[1]) : "r"(addr));
}

// d += a b on the tensor cores, m16n8k16, fp32 accumulators
template <class Ty>
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    if constexpr (Ty::code == 5) {
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                     "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
                     : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
                     "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
                     : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// two fp32 values -> one 32-bit word of two 16-bit values (first in the low half)
template <class Ty> __device__ __forceinline__ unsigned pack2(float x, float y);
template <> __device__ __forceinline__ unsigned pack2<TyB>(float x, float y) {
    __nv_bfloat162 v = __floats2bfloat162_rn(x, y);
    return *reinterpret_cast<unsigned*>(&v);
}
template <> __device__ __forceinline__ unsigned pack2<TyH>(float x, float y) {
    __half2 v = __floats2half2_rn(x, y);
    return *reinterpret_cast<unsigned*>(&v);
}
template <class Ty> __device__ __forceinline__ float2 unpack2(unsigned w);
template <> __device__ __forceinline__ float2 unpack2<TyB>(unsigned w) {
    return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&w));
}
template <> __device__ __forceinline__ float2 unpack2<TyH>(unsigned w) {
    return __half22float2(*reinterpret_cast<__half2*>(&w));
}

// 16-byte chunk position of memory row u, half h of a 16 x 16 slot
__device__ __forceinline__ int mma_chunk16(int u, int h) { return 2 * u + (h ^ ((u >> 2) & 1)); }

struct MmaArgs {
    const void* A; const void* B; void* C;
    long long batch;
    int P;                     // pairs per tile (even)
    int stages;
    float alpha, beta;
    const float* alpha_ptr; const float* beta_ptr;
    int beta_zero;             // host scalars: C not read
};

// shared-memory bytes of one matrix slot (a matrix is stored contiguously)
__host__ __device__ constexpr int mma_slot_bytes(int m) { return 2 * m * m; }

template <class Ty, int M>
__global__ void __launch_bounds__(128) mma16_kernel(MmaArgs g)
{
    static_assert(M == 8 || M == 12 || M == 16, "tensor-core path for m = 8, 12 and 16");
    using S = typename Ty::S;
    constexpr int SE = M * M;                  // elements per matrix
    constexpr int CPM = SE * 2 / 16;           // 16-byte chunks per matrix
    extern __shared__ __align__(16) unsigned char smem_raw[];
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");

    float alpha = g.alpha, beta = g.beta;
    bool beta_zero = g.beta_zero != 0;
    const bool has_cold = !beta_zero;          // smem layout fixed by the host
    if (g.alpha_ptr) alpha = *g.alpha_ptr;
    if (g.beta_ptr) { beta = *g.beta_ptr; beta_zero = beta == 0.f; }
    const bool alpha_one = alpha == 1.f;
    const bool skip_ab = alpha == 0.f;         // C = beta C; A and B are not read

    const int P = g.P, stages = g.stages;
    const long long batch = g.batch;
    const int ntiles = (int)((batch + P - 1) / P);
    const int slot = mma_slot_bytes(M);        // bytes per matrix slot
    const int stage_bytes = P * slot * (has_cold ? 3 : 2);
    const S* gA = static_cast<const S*>(g.A);
    const S* gB = static_cast<const S*>(g.B);
    S* gC = static_cast<S*>(g.C);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // stage `cnt` pairs of one operand: 16-byte chunks (a tile is one
    // contiguous span); m = 16 slots swizzled
    auto stage_op = [&](unsigned char* dst, const S* src, int cnt) {
        const char* s8 = reinterpret_cast<const char*>(src);
        for (int c = tid; c < cnt * CPM; c += 128) {
            int pos = c;
            if constexpr (M == 16) {
                const int q = c / CPM, lc = c - q * CPM;
                pos = q * CPM + mma_chunk16(lc >> 1, lc & 1);
            }
            cp_async16(dst + pos * 16, s8 + 16 * (long long)c, 16);
        }
    };
    auto issue = [&](int t, int s) {
        unsigned char* st = smem_raw + s * stage_bytes;
        const long long p0 = (long long)t * P;
        const int cnt = (int)min((long long)P, batch - p0);
        if (!skip_ab) {
            stage_op(st, gA + p0 * SE, cnt);
            stage_op(st + P * slot, gB + p0 * SE, cnt);
        }
        if (!beta_zero) stage_op(st + 2 * P * slot, gC + p0 * SE, cnt);
    };

    for (int s = 0; s < stages - 1; ++s) {
        const int t = blockIdx.x + s * gridDim.x;
        if (t < ntiles) issue(t, s);
        cp_async_commit();
    }
    const int gq = lane >> 2, tq = lane & 3;   // fragment row group / thread in group
    const int mi = lane >> 3, rr = lane & 7;   // ldmatrix matrix / row of this lane

    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int tn = t + (stages - 1) * gridDim.x;
        if (tn < ntiles) issue(tn, (it + stages - 1) % stages);
        cp_async_commit();
        cp_async_wait_dyn(stages - 1);
        __syncthreads();

        const unsigned char* st = smem_raw + (it % stages) * stage_bytes;
        const unsigned sA = smem_u32(st), sB = smem_u32(st + P * slot);
        const unsigned char* sC = st + 2 * P * slot;
        const long long p0 = (long long)t * P;
        const int cnt = (int)min((long long)P, batch - p0);

        if constexpr (M == 12) {
            // 12 x 12 pairs computed as 16 x 16 with zero fragments outside:
            // the 24-byte columns leave no 16-byte rows for ldmatrix, so the
            // fragments are read as 32-bit pairs (B^T rows are contiguous)
            // and 16-bit entries (A^T: two columns of A per register).  Which
            // fragment entries lie inside the matrix depends on the lane
            // only: the offsets and masks are fixed per lane, invalid
            // entries load from offset 0 and are masked (no branches), and
            // two pairs are handled per iteration for independent loads.
            const bool r1 = gq < 4;                    // row / column gq + 8 < 12
            const bool c1 = tq < 2;                    // k index 2tq + 8 < 12
            const int oB[4] = {2 * tq + 12 * gq, r1 ? 2 * tq + 12 * (gq + 8) : 0,
                               c1 ? 2 * tq + 8 + 12 * gq : 0, (r1 && c1) ? 2 * tq + 8 + 12 * (gq + 8) : 0};
            const unsigned mB[4] = {~0u, r1 ? ~0u : 0u, c1 ? ~0u : 0u, (r1 && c1) ? ~0u : 0u};
            // A^T(l, i), A^T(l + 1, i) at As[i + 12 l], As[i + 12 (l + 1)] for
            // (nt, kh): i = 8 nt + gq, l = 2tq + 8 kh
            int oA[2][2];
            unsigned mA[2][2];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int kh = 0; kh < 2; ++kh) {
                    const bool ok = (nt == 0 || r1) && (kh == 0 || c1);
                    oA[nt][kh] = ok ? 8 * nt + gq + 12 * (2 * tq + 8 * kh) : 0;
                    mA[nt][kh] = ok ? ~0u : 0u;
                }
            auto pair_product = [&](int q, float (&d)[2][4]) {
                const unsigned short* Bs = reinterpret_cast<const unsigned short*>(st + P * slot + q * slot);
                const unsigned short* As = reinterpret_cast<const unsigned short*>(st + q * slot);
                unsigned a[4];
#pragma unroll
                for (int x = 0; x < 4; ++x) a[x] = *reinterpret_cast<const unsigned*>(Bs + oB[x]) & mB[x];
                unsigned b[2][2];
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int kh = 0; kh < 2; ++kh)
                        b[nt][kh] = ((unsigned)As[oA[nt][kh]] | ((unsigned)As[oA[nt][kh] + 12] << 16)) &
                                    mA[nt][kh];
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) mma16816<Ty>(d[nt], a, b[nt][0], b[nt][1]);
            };
            auto pair_store = [&](int q, const float (&d)[2][4]) {
                S* cp = gC + (p0 + q) * SE;
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    if (nt == 1 && tq >= 2) continue;       // i = 12..15: outside the matrix
#pragma unroll
                    for (int hr = 0; hr < 2; ++hr) {
                        const int j = gq + 8 * hr;
                        if (hr == 1 && !r1) continue;        // j = 12..15
                        const int i = 8 * nt + 2 * tq;
                        float x = d[nt][2 * hr], y = d[nt][2 * hr + 1];
                        if (!alpha_one) { x *= alpha; y *= alpha; }
                        if (!beta_zero) {
                            const float2 o = unpack2<Ty>(*reinterpret_cast<const unsigned*>(
                                sC + q * slot + 2 * (i + 12 * j)));
                            x = fmaf(beta, o.x, x);
                            y = fmaf(beta, o.y, y);
                        }
                        *reinterpret_cast<unsigned*>(cp + i + 12 * j) = pack2<Ty>(x, y);
                    }
                }
            };
            for (int q = warp; q < cnt; q += 8) {
                const bool two = q + 4 < cnt;
                float d0[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
                float d1[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
                if (!skip_ab) {
                    pair_product(q, d0);
                    if (two) pair_product(q + 4, d1);
                }
                pair_store(q, d0);
                if (two) pair_store(q + 4, d1);
            }
        } else if constexpr (M == 16) {
            for (int q = warp; q < cnt; q += 4) {
                float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
                if (!skip_ab) {
                    unsigned a[4], b[4];
                    // A operand: B^T; this lane's row: memory row u of B, half h
                    ldsm_x4(a, sB + q * slot + 16 * mma_chunk16(rr + 8 * (mi & 1), mi >> 1));
                    // B operands of both n8 tiles: A^T (.trans); k half = mi & 1, n tile = mi >> 1
                    ldsm_x4_t(b, sA + q * slot + 16 * mma_chunk16(rr + 8 * (mi & 1), mi >> 1));
                    mma16816<Ty>(d[0], a, b[0], b[1]);
                    mma16816<Ty>(d[1], a, b[2], b[3]);
                }
                S* cp = gC + (p0 + q) * SE;
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
                    for (int hr = 0; hr < 2; ++hr) {       // rows gq and gq + 8 (columns j of C)
                        const int j = gq + 8 * hr;
                        float x = d[nt][2 * hr], y = d[nt][2 * hr + 1];
                        if (!alpha_one) { x *= alpha; y *= alpha; }
                        if (!beta_zero) {
                            const float2 o = unpack2<Ty>(*reinterpret_cast<const unsigned*>(
                                sC + q * slot + 16 * mma_chunk16(j, nt) + 4 * tq));
                            x = fmaf(beta, o.x, x);
                            y = fmaf(beta, o.y, y);
                        }
                        *reinterpret_cast<unsigned*>(cp + 8 * nt + 2 * tq + 16 * j) = pack2<Ty>(x, y);
                    }
                }
            }
        } else {
            // two pairs per MMA: q0 = 2w, q1 = 2w + 1 (q1 repeats q0 at an odd end)
            for (int w = warp; 2 * w < cnt; w += 4) {
                const int q0 = 2 * w, q1 = (2 * w + 1 < cnt) ? 2 * w + 1 : 2 * w;
                const int qq = (mi & 1) ? q1 : q0;           // lanes 8..15 address pair q1
                float d[4] = {0.f, 0.f, 0.f, 0.f};
                if (!skip_ab) {
                    unsigned a2[2], b2[2];
                    ldsm_x2(a2, sB + qq * slot + 16 * rr);       // B0^T, B1^T
                    ldsm_x2_t(b2, sA + qq * slot + 16 * rr);     // A0^T, A1^T
                    const unsigned a[4] = {a2[0], 0u, 0u, a2[1]};
                    mma16816<Ty>(d, a, b2[0], b2[1]);
                }
#pragma unroll
                for (int hr = 0; hr < 2; ++hr) {             // rows gq: pair q0, gq + 8: pair q1
                    if (hr == 1 && q1 == q0) break;
                    const int q = hr ? q1 : q0;
                    float x = d[2 * hr], y = d[2 * hr + 1];
                    if (!alpha_one) { x *= alpha; y *= alpha; }
                    if (!beta_zero) {
                        const float2 o = unpack2<Ty>(*reinterpret_cast<const unsigned*>(
                            sC + q * slot + 16 * gq + 4 * tq));
                        x = fmaf(beta, o.x, x);
                        y = fmaf(beta, o.y, y);
                    }
                    *reinterpret_cast<unsigned*>(gC + (p0 + q) * SE + 2 * tq + 8 * gq) = pack2<Ty>(x, y);
                }
            }
        }
        // every thread is done with this stage before it is refilled
        __syncthreads();
    }
    cp_async_wait_dyn(0);
}

// Host side: the request qualifies when the shape, ops and layout match.
template <class Ty, int M>
sbgemm_status launch_mma16(const Req& r) {
    MmaArgs g;
    g.A = r.A; g.B = r.B; g.C = r.C;
    g.batch = r.batch;
    g.stages = 3;
    if (r.scalar_mode == SBGEMM_SCALARS_DEVICE) {
        g.alpha_ptr = static_cast<const float*>(r.alpha);
        g.beta_ptr = static_cast<const float*>(r.beta);
        g.alpha = 0.f; g.beta = 0.f; g.beta_zero = 0;
    } else {
        g.alpha_ptr = nullptr; g.beta_ptr = nullptr;
        g.alpha = *static_cast<const float*>(r.alpha);
        g.beta = *static_cast<const float*>(r.beta);
        g.beta_zero = r.beta_zero;
    }
    const int per_pair = mma_slot_bytes(M) * (g.beta_zero ? 2 : 3);
    // Stage bytes: 24 KB at m = 16 (three resident blocks of 128 threads);
    // 14 KB at m = 8 and 12 (five blocks), where more resident warps hide the
    // latency of the fragment loads.  Measured, binary16, N = 1e6, beta = 0 /
    // beta != 0: m = 12 153.5 / 207.8 us against 177.2 / 254.2 us with 24 KB
    // (stages of 10-20 KB: 150.7-180.6 / 207.8-235.9 us); m = 8 56.1 / 79.1
    // against 57.7 / 80.0 us; m = 16 slower with any smaller stage.
    constexpr int kStageBytes = (M == 16 ? 24 : 14) * 1024;
    constexpr int kResident = M == 16 ? 3 : 5;
    int P = kStageBytes / per_pair;
    P &= ~1;
    // at least two tiles per resident block when the batch is short
    const long long want = 2LL * num_sms() * kResident;
    if ((r.batch + P - 1) / P < want) {
        long long p2 = (r.batch + want - 1) / want;
        p2 = (p2 + 1) & ~1LL;
        if (p2 < 2) p2 = 2;
        if (p2 < P) P = (int)p2;
    }
    g.P = P;
    const size_t smem = (size_t)g.stages * P * per_pair;
    auto kern = mma16_kernel<Ty, M>;
    // per instantiation and device
    static DeviceFlags attr;
    static thread_local OccCache occ;
    cudaError_t ae = ensure_smem_limit(kern, 220 * 1024, attr);
    if (ae != cudaSuccess) return (sbgemm_status)ae;
    int occ_val = 0;
    ae = blocks_per_sm(kern, 128, smem, occ, &occ_val);
    if (ae != cudaSuccess) return (sbgemm_status)ae;
    if (occ_val < 1) return SBGEMM_ERR_NOT_SUPPORTED;
    const long long ntiles = (r.batch + P - 1) / P;
    long long grid = (long long)num_sms() * occ_val;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(128);
    lc.dynamicSmemBytes = smem;
    lc.stream = r.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&lc, kern, g);
    if (e != cudaSuccess) return (sbgemm_status)e;
    return (sbgemm_status)cudaGetLastError();
}

// true when the tensor-core kernel can run the request: 16-bit storage,
// m = n = k = 8, 12 or 16, op N/N, flat operands with 16-byte aligned bases
inline bool mma16_eligible(const Req& r) {
    if (r.type != SBGEMM_TYPE_H && r.type != SBGEMM_TYPE_B) return false;
    if (r.Cp || r.ta || r.tb) return false;
    const int m = r.m;
    if (!(m == 8 || m == 12 || m == 16) || r.n != m || r.k != m) return false;
    const long long S = (long long)m * m;
    if (r.lda != m || r.ldb != m || r.ldc != m || r.lda2 != S || r.ldb2 != S || r.ldc2 != S) return false;
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    return al(r.A) && al(r.B) && al(r.C);
}

}  // namespace sbg
