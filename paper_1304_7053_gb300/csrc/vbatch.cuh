// Variable-size batches: one persistent launch over a device work queue.
//
// The paper notes (Section 1) that matrices of different sizes can be
// partitioned into sets of identical size.  Here the partition is a host
// plan: problems are bucketed by (m, n, k, op), buckets are cut into tiles,
// and one persistent kernel takes tiles from an atomic counter, runs the
// size-specialised compute of the tile's bucket (the same register-blocked
// code as the fixed-size path), and double-buffers the next tile's staging
// behind the current tile's compute.  Each problem's matrices are contiguous
// (minimal leading dimensions) at arbitrary arena offsets; staging copies
// them asynchronously, in 16-byte chunks where the chunk boundaries of the
// arena and of the matrix's slot line up (see the shifted slots below).
#pragma once

#include "sbgemm_launch.cuh"

namespace sbg {

// per-problem record in bucket order (32 bytes)
struct VRec {
    long long a, b, c;
    int flags;     // bits 0-1 opA, 2-3 opB, bit 4 beta-zero
    int pad;
};

// one tile of one bucket
struct VItem {
    int kind;      // 0..15: square size kind+1 with op N/N; 16: generic
    int first;     // first record
    int count;     // records in the tile
    int shape;     // m | n << 8 | k << 16 | ta << 24 | tb << 25
};

constexpr int kVKinds = 17;
constexpr int kVGeneric = 16;
constexpr int kVThreads = 128;
constexpr int kVMaxTile = 128;
// Problems per bucketing window of a plan.  Arena neighbours share 32-byte
// memory sectors at their boundaries; bucketing the whole batch at once put
// neighbours of different sizes far apart in time, and DRAM read those
// sectors twice (1.40x the algorithmic bytes on the fp32 mix).  Windows of
// 65,536 problems (about 42 MB of fp32 operands, well inside the 129 MB L2)
// keep them close: 0.99x, and the fastest window of a sweep over
// whole / 262,144 / 65,536 / 16,384 / 4,096 for fp32 and fp64.
constexpr int kVDefaultWindow = 1 << 16;

// Pipeline shape per storage type: two stages (one tile in flight while
// another computes).  Memory-bound types take 28 KB stages and three blocks
// of 128 threads per SM (a cap of 168 registers); fp64 and complex128, bound
// by the fp64 pipe, 48 KB stages (more matrices per compute round) and two
// blocks.  Three stages of 24 KB with two blocks per SM measured 0.259 ms on
// the fp32 mix against 0.213 ms for this shape, four blocks of 20 KB stages
// 0.241 ms.  Shared memory: stages x stage bytes + (2 stages - 1) record
// buffers of kVMaxTile records + the tile descriptors.
__host__ __device__ constexpr bool vfp64(int type) { return type == SBGEMM_TYPE_D || type == SBGEMM_TYPE_Z; }
__host__ __device__ constexpr int vstages_of(int) { return 2; }
__host__ __device__ constexpr int vstage_bytes_of(int type) { return vfp64(type) ? 48 * 1024 : 28 * 1024; }
__host__ __device__ constexpr int vblocks_of(int type) { return vfp64(type) ? 2 : 3; }
__host__ __device__ constexpr int vrec_slots_of(int type) { return 2 * vstages_of(type) - 1; }
__host__ __device__ constexpr int vitem_slots_of(int type) { return 3 * vstages_of(type) - 2; }

template <class Ty>
struct VArgs {
    using S = typename Ty::S;
    using A = typename Ty::A;
    const VItem* items;
    int n_items;
    const VRec* recs;
    int* counter;
    const S* A_; const S* B_; S* C_;
    A alpha, beta;
    const A* alpha_ptr; const A* beta_ptr;
    int beta_zero, alpha_zero;   // host scalars only
    int max_tile;                // largest record count of any tile
};

// The specialised configuration of square size s (op N/N); kinds whose
// tile needs another block size fall back to the generic kind.  The product
// loop is not unrolled (one l-chunk per iteration) and neither are the
// staging copy loops: a block switches between the 16 size-specialised
// bodies from tile to tile, and with fully unrolled bodies (about 3x the
// code) instruction fetch bounded the kernel whenever neighbouring tiles had
// different sizes; with the short bodies, bucketing windows that keep arena
// neighbours close in time cost nothing (fp32 mix: windows of 4096 problems
// 0.438 -> 0.241 ms).  The C write-back loops stay unrolled (rolling them
// measured 6% slower).
template <class Ty, int s>
struct VKindCfg {
    static constexpr TileEntry te = tile_for(Ty::code, s, s, s, 0, 0);
    using Cf = Cfg<Ty, s, s, s, false, false, te.tm, te.tn, te.si != 0, te.sj != 0, te.nt, 1>;
    static constexpr bool ok = te.nt == kVThreads;
};

// Region offsets inside a stage are multiples of the tile's slot count
// rounded up to this quantum, so every region starts 16-byte aligned for the
// vector loads of the specialised compute.
template <class Cf>
__host__ __device__ constexpr int slot_quantum() {
    return lcm_c(lcm_c(16 / gcd_c(Cf::SA_P * Cf::ES, 16), 16 / gcd_c(Cf::SB_P * Cf::ES, 16)),
                 16 / gcd_c(Cf::SC_P * Cf::ES, 16));
}

// Shifted slots.  A square kind whose matrices are not a whole number of
// 16-byte chunks (odd sizes of the 4- and 8-byte types, and 16-bit sizes
// that are not multiples of 8) and whose compute reads shared memory one
// element at a time keeps each matrix in its slot at the element offset
// that the matrix's global start has within its 16-byte chunk (its phase).
// The chunk-aligned middle of every matrix then moves in 16-byte copies in
// both directions, and only the ragged head and tail move element by
// element.  In the packed arena of a variable-size batch most matrices start
// off a 16-byte boundary, and these kinds could otherwise only copy
// element by element.  A slot holds the matrix at any phase: its byte size
// is the matrix's plus 16 - ES, rounded up to 16.
template <class Cf>
__host__ __device__ constexpr bool vshifted() {
    return (Cf::SA * Cf::ES) % 16 != 0 && Cf::VL == 1 && Cf::VI == 1 && Cf::VJ == 1;
}
template <class Cf>
__host__ __device__ constexpr int vslot_elems() {
    return vshifted<Cf>() ? (Cf::SA * Cf::ES + 16 - Cf::ES + 15) / 16 * 16 / Cf::ES : Cf::SA_P;
}
template <class Cf>
__host__ __device__ constexpr int vquantum() { return vshifted<Cf>() ? 1 : slot_quantum<Cf>(); }

// Host view of a kind: matrices per compute round, staged bytes per pair
// (A, B and old C slots), slot quantum.
struct VKindInfo { int mpr; int bytes_per_pair; int quantum; };

template <class Ty, int s>
constexpr VKindInfo vkind_info_one() {
    using K = VKindCfg<Ty, s>;
    using Cf = typename K::Cf;
    static_assert(Cf::SA_P == Cf::SB_P && Cf::SB_P == Cf::SC_P, "square kinds share one slot size");
    return K::ok ? VKindInfo{Cf::MPR, 3 * vslot_elems<Cf>() * Cf::ES, vquantum<Cf>()}
                 : VKindInfo{0, 0, 1};
}

// ------------------------------------------------------------ device side

template <class S, int ES>
__device__ __forceinline__ void vcopy_elem(S* dst, const S* src) {
    if constexpr (ES == 4 || ES == 8 || ES == 16) cp_async_elem<ES>(dst, src);
    else *dst = *src;
}

// Copy one matrix of `n` elements (contiguous in global memory) into a
// shared-memory slot: the lanes of a warp take consecutive elements.
template <class S, int ES>
__device__ __forceinline__ void vcopy_matrix(S* dst, const S* src, int n, int lane) {
    for (int e = lane; e < n; e += 32) vcopy_elem<S, ES>(dst + e, src + e);
}

// Copy one contiguous matrix of SE elements into its slot: in 16-byte
// chunks when its byte size is a multiple of 16 and its start is 16-byte
// aligned (lanes l0, l0+LPP, ... take the chunks), element by element
// otherwise.
template <class S, int SE, int LPP>
__device__ __forceinline__ void vcopy_square(S* dst, const S* src, int l0) {
    constexpr int ES = sizeof(S);
    if constexpr ((SE * ES) % 16 == 0) {
        constexpr int CPM = SE * ES / 16, EPC = 16 / ES;
        if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
#pragma unroll 1
            for (int c = l0; c < CPM; c += LPP) cp_async16(dst + c * EPC, src + c * EPC, 16);
            return;
        }
    }
#pragma unroll 1
    for (int e = l0; e < SE; e += LPP) vcopy_elem<S, ES>(dst + e, src + e);
}

// Stage the A, B (and old C) matrices of a tile of a square specialised
// kind.  A group of LPP lanes takes one problem: it reads the problem's
// record once and copies its three matrices; a warp takes 32 / LPP problems
// per pass (LPP = the chunk or element count of one matrix, at most 32).
template <class S, int SE, int SP, int NT>
__device__ __forceinline__ void vstage_square(S* sA, S* sB, S* sC, const VRec* rec, int cnt,
                                              const S* gA, const S* gB, const S* gC, bool ab,
                                              bool any_c) {
    constexpr int ES = sizeof(S);
    constexpr int UNITS = (SE * ES) % 16 == 0 ? SE * ES / 16 : SE;   // chunks or elements
    constexpr int LPP = UNITS >= 32 ? 32 : UNITS;
    constexpr int PPW = 32 / LPP;
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / LPP, l0 = lane - sub * LPP;
    if (sub >= PPW) return;                             // lanes left over when LPP does not divide 32
    for (int q = warp * PPW + sub; q < cnt; q += NW * PPW) {
        const VRec r = rec[q];
        if (ab) {
            vcopy_square<S, SE, LPP>(sA + q * SP, gA + r.a, l0);
            vcopy_square<S, SE, LPP>(sB + q * SP, gB + r.b, l0);
        }
        if (any_c && !(r.flags & 16)) vcopy_square<S, SE, LPP>(sC + q * SP, gC + r.c, l0);
    }
}

// Stage a generic tile (run-time sizes): one warp per problem.
template <class S, int NT>
__device__ __forceinline__ void vstage(S* st, const VRec* rec, int cnt, const S* gA, const S* gB,
                                       const S* gC, int SA, int SB, int SC, int SA_P, int SB_P,
                                       int SC_P, int P, bool skip_ab, bool all_beta_zero) {
    constexpr int ES = sizeof(S);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    S* sB = st + P * SA_P;
    S* sC = st + P * (SA_P + SB_P);
    for (int q = warp; q < cnt; q += NW) {
        const VRec& r = rec[q];
        if (!skip_ab) {
            vcopy_matrix<S, ES>(st + q * SA_P, gA + r.a, SA, lane);
            vcopy_matrix<S, ES>(sB + q * SB_P, gB + r.b, SB, lane);
        }
        if (!all_beta_zero && !(r.flags & 16)) vcopy_matrix<S, ES>(sC + q * SC_P, gC + r.c, SC, lane);
    }
}

// Write the C slots of a square specialised tile back to each problem's C,
// with the lane mapping of vstage_square (16-byte stores where size and
// alignment allow).
template <class S, int SE, int SP, int NT>
__device__ __forceinline__ void vstore_fixed(S* gC, const S* sC, const VRec* rec, int cnt) {
    constexpr int ES = sizeof(S);
    constexpr int UNITS = (SE * ES) % 16 == 0 ? SE * ES / 16 : SE;
    constexpr int LPP = UNITS >= 32 ? 32 : UNITS;
    constexpr int PPW = 32 / LPP;
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / LPP, l0 = lane - sub * LPP;
    if (sub >= PPW) return;
    for (int q = warp * PPW + sub; q < cnt; q += NW * PPW) {
        S* dst = gC + rec[q].c;
        const S* src = sC + q * SP;
        if constexpr ((SE * ES) % 16 == 0) {
            constexpr int CPM = SE * ES / 16, EPC = 16 / ES;
            if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
                for (int c = l0; c < CPM; c += LPP)
                    *reinterpret_cast<uint4*>(dst + c * EPC) = *reinterpret_cast<const uint4*>(src + c * EPC);
                continue;
            }
        }
#pragma unroll
        for (int e = l0; e < SE; e += LPP) dst[e] = src[e];
    }
}

// Phase of a global address: its element offset within its 16-byte chunk
// (addresses are aligned to the element size).
template <class S>
__device__ __forceinline__ int vphase(const S* p) {
    return (int)((reinterpret_cast<uintptr_t>(p) & 15) / sizeof(S));
}

// A matrix of SE elements whose global start has phase h, in copy units:
// nh head elements up to the first 16-byte boundary, nc 16-byte chunks,
// nt tail elements.
template <class S, int SE>
struct VSplit {
    int nh, nc, nt;
    __device__ __forceinline__ explicit VSplit(int h) {
        constexpr int EPC = 16 / sizeof(S);
        nh = h ? min(EPC - h, SE) : 0;
        nc = (SE - nh) / EPC;
        nt = SE - nh - nc * EPC;
    }
};

// Lanes per problem of the shifted copies: the chunk count of a matrix,
// at least the ragged elements (at most 2 (16 / ES - 1)), at most a warp.
template <class S, int SE>
__host__ __device__ constexpr int vshift_lanes() {
    constexpr int es = (int)sizeof(S);
    constexpr int chunks = SE * es / 16, ragged = 2 * (16 / es - 1);
    return (chunks > ragged ? chunks : ragged) >= 32 ? 32 : (chunks > ragged ? chunks : ragged);
}

// Copy one matrix into its shifted slot (dst = slot start + phase of src).
// Lanes l0, l0 + LPP, ... take the 16-byte chunks (a loop of fixed trip
// count, unrolled, predicated on the matrix's own chunk count); then lane
// l0 < nh + nt takes one head or tail element.  dst + nh is 16-byte aligned
// because the slot start is.
template <class S, int SE, int LPP>
__device__ __forceinline__ void vcopy_shifted(S* dst, const S* src, int l0) {
    constexpr int ES = sizeof(S), EPC = 16 / ES;
    constexpr int ITER = (SE / EPC + LPP - 1) / LPP;
    const VSplit<S, SE> p(vphase(src));
#pragma unroll
    for (int i = 0; i < ITER; ++i) {
        const int c = l0 + i * LPP;
        if (c < p.nc) cp_async16(dst + p.nh + c * EPC, src + p.nh + c * EPC, 16);
    }
    if (l0 < p.nh + p.nt) {
        const int e = l0 < p.nh ? l0 : l0 + p.nc * EPC;
        vcopy_elem<S, ES>(dst + e, src + e);
    }
}

// Stage the A, B (and old C) matrices of a tile of a shifted kind (slots of
// SV elements), with the lane grouping of vstage_square.
template <class S, int SE, int SV, int NT>
__device__ __forceinline__ void vstage_shifted(S* sA, S* sB, S* sC, const VRec* rec, int cnt,
                                               const S* gA, const S* gB, const S* gC, bool ab,
                                               bool any_c) {
    constexpr int LPP = vshift_lanes<S, SE>();
    constexpr int PPW = 32 / LPP;
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / LPP, l0 = lane - sub * LPP;
    if (sub >= PPW) return;
    for (int q = warp * PPW + sub; q < cnt; q += NW * PPW) {
        const VRec r = rec[q];
        if (ab) {
            const S* a = gA + r.a;
            const S* b = gB + r.b;
            vcopy_shifted<S, SE, LPP>(sA + q * SV + vphase(a), a, l0);
            vcopy_shifted<S, SE, LPP>(sB + q * SV + vphase(b), b, l0);
        }
        if (any_c && !(r.flags & 16)) {
            const S* c = gC + r.c;
            vcopy_shifted<S, SE, LPP>(sC + q * SV + vphase(c), c, l0);
        }
    }
}

// Write the shifted C slots of a tile back to each problem's C: 16-byte
// stores for the chunk-aligned middle, element stores for head and tail
// (the lane mapping of vcopy_shifted).
template <class S, int SE, int SV, int NT>
__device__ __forceinline__ void vstore_shifted(S* gC, const S* sC, const VRec* rec, int cnt) {
    constexpr int EPC = 16 / (int)sizeof(S);
    constexpr int LPP = vshift_lanes<S, SE>();
    constexpr int ITER = (SE / EPC + LPP - 1) / LPP;
    constexpr int PPW = 32 / LPP;
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / LPP, l0 = lane - sub * LPP;
    if (sub >= PPW) return;
    for (int q = warp * PPW + sub; q < cnt; q += NW * PPW) {
        S* dst = gC + rec[q].c;
        const int h = vphase(dst);
        const S* src = sC + q * SV + h;
        const VSplit<S, SE> p(h);
#pragma unroll
        for (int i = 0; i < ITER; ++i) {
            const int c = l0 + i * LPP;
            if (c < p.nc)
                *reinterpret_cast<uint4*>(dst + p.nh + c * EPC) =
                    *reinterpret_cast<const uint4*>(src + p.nh + c * EPC);
        }
        if (l0 < p.nh + p.nt) {
            const int e = l0 < p.nh ? l0 : l0 + p.nc * EPC;
            dst[e] = src[e];
        }
    }
}

// Compute a tile of a shifted kind in place in its C slots: each matrix is
// read at its slot start plus its phase (compute_block with per-matrix
// pointers: q = 0 and both operand offsets switched off).
template <class Cf>
__device__ __forceinline__ void vcompute_shifted(const typename Cf::S* sA, const typename Cf::S* sB,
                                                 typename Cf::S* sC, const VRec* rec, int cnt,
                                                 const typename Cf::S* gA, const typename Cf::S* gB,
                                                 const typename Cf::S* gC, typename Cf::A alpha,
                                                 typename Cf::A beta, bool beta_zero,
                                                 bool alpha_one, bool skip_ab) {
    using R = typename Cf::R;
    constexpr int SV = vslot_elems<Cf>();
    const int tid = threadIdx.x;
    const int ql = tid / Cf::TPM;
    const int u = tid - ql * Cf::TPM;
    const int ti = u % Cf::TI, tj = u / Cf::TI;
    if (ql >= Cf::MPR) return;
    for (int q = ql; q < cnt; q += Cf::MPR) {
        const VRec r = rec[q];
        const R ca = ((r.flags & 3) == 2) ? R(-1) : R(1);
        const R cb = (((r.flags >> 2) & 3) == 2) ? R(-1) : R(1);
        typename Cf::S* c = sC + q * SV + vphase(gC + r.c);
        compute_block<Cf>(sA + q * SV + vphase(gA + r.a), sB + q * SV + vphase(gB + r.b), c, c,
                          nullptr, false, 0, ti, tj, alpha, beta, beta_zero || (r.flags & 16),
                          alpha_one, skip_ab, ca, cb, 3);
    }
}

// Write the C slots of a tile back to each problem's C (one warp per problem).
template <class S, int NT>
__device__ __forceinline__ void vstore(S* gC, const S* sC, const VRec* rec, int cnt, int SC,
                                       int SC_P) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    for (int q = warp; q < cnt; q += NW) {
        S* dst = gC + rec[q].c;
        const S* src = sC + q * SC_P;
        for (int e = lane; e < SC; e += 32) dst[e] = src[e];
    }
}

// Compute a tile of a specialised kind into the shared output tile.
template <class Cf>
__device__ __forceinline__ void vcompute_kind(const typename Cf::S* st, const VRec* rec, int cnt, int P,
                                              typename Cf::S* sOut, typename Cf::A alpha,
                                              typename Cf::A beta, bool beta_zero, bool alpha_one,
                                              bool skip_ab) {
    using R = typename Cf::R;
    const int tid = threadIdx.x;
    const int ql = tid / Cf::TPM;
    const int u = tid - ql * Cf::TPM;
    const int ti = u % Cf::TI, tj = u / Cf::TI;
    if (ql >= Cf::MPR) return;
    for (int q = ql; q < cnt; q += Cf::MPR) {
        const int fl = rec[q].flags;
        const R ca = ((fl & 3) == 2) ? R(-1) : R(1);
        const R cb = (((fl >> 2) & 3) == 2) ? R(-1) : R(1);
        compute_block<Cf>(st, st + P * Cf::SA_P, st + P * (Cf::SA_P + Cf::SB_P), sOut, nullptr,
                          false, q, ti, tj, alpha, beta, beta_zero || (fl & 16), alpha_one,
                          skip_ab, ca, cb);
    }
}

// Generic kind: run-time sizes and ops; the tile's (problem, entry) pairs
// are spread over the block, one entry of C per thread at a time.
template <class Ty>
__device__ __forceinline__ void vcompute_generic(const typename Ty::S* st, const VRec* rec, int cnt,
                                                 int P, typename Ty::S* sOut, int m, int n, int k,
                                                 int ta, int tb, typename Ty::A alpha,
                                                 typename Ty::A beta, bool beta_zero, bool skip_ab) {
    using S = typename Ty::S;
    using A = typename Ty::A;
    using R = typename Ty::R;
    const int sa = m * k, sb = k * n, sc = m * n;
    const S* sA = st;
    const S* sB = st + P * sa;
    const S* sC = st + P * (sa + sb);
    for (int w = threadIdx.x; w < cnt * sc; w += kVThreads) {
        const int q = w / sc, r = w - q * sc;
        const int i = r % m, j = r / m;
        const int fl = rec[q].flags;
        const R ca = ((fl & 3) == 2) ? R(-1) : R(1);
        const R cb = (((fl >> 2) & 3) == 2) ? R(-1) : R(1);
        A acc = zero_a<A>();
        if (!skip_ab) {
            const S* a = sA + q * sa;
            const S* b = sB + q * sb;
            for (int l = 0; l < k; ++l)
                mac(acc, conj_s(to_a(a[ta ? l + k * i : i + m * l]), ca),
                    conj_s(to_a(b[tb ? j + n * l : l + k * j]), cb));
        }
        A v = skip_ab ? zero_a<A>() : mul(alpha, acc);
        if (!(beta_zero || (fl & 16))) v = axpy(beta, to_a(sC[q * sc + i + m * j]), v);
        sOut[q * sc + i + m * j] = to_s<Ty>(v);     // sOut is this tile's C slots: in place
    }
}

// Stage / compute one tile, dispatching on its kind (uniform in the block).
template <class Ty, int s = 1>
__device__ __forceinline__ void vstage_kind(int kind, typename Ty::S* st, const VRec* rec, int cnt,
                                            const VArgs<Ty>& g, bool skip_ab, bool all_bz) {
    if constexpr (s <= 16) {
        if (kind == s - 1) {
            using K = VKindCfg<Ty, s>;
            if constexpr (K::ok) {
                using Cf = typename K::Cf;
                using S = typename Ty::S;
                static_assert(Cf::SA == Cf::SB && Cf::SB == Cf::SC && Cf::SA_P == Cf::SC_P,
                              "square kinds share one slot size");
                if constexpr (vshifted<Cf>()) {
                    constexpr int SV = vslot_elems<Cf>();
                    vstage_shifted<S, Cf::SA, SV, kVThreads>(st, st + cnt * SV, st + 2 * cnt * SV,
                                                             rec, cnt, g.A_, g.B_, g.C_, !skip_ab,
                                                             !all_bz);
                } else {
                    constexpr int Q = slot_quantum<Cf>();
                    const int P = (cnt + Q - 1) / Q * Q;
                    vstage_square<S, Cf::SA, Cf::SA_P, kVThreads>(
                        st, st + P * Cf::SA_P, st + P * (Cf::SA_P + Cf::SB_P), rec, cnt, g.A_,
                        g.B_, g.C_, !skip_ab, !all_bz);
                }
            }
            return;
        }
        vstage_kind<Ty, s + 1>(kind, st, rec, cnt, g, skip_ab, all_bz);
    }
}

template <class Ty, int s = 1>
__device__ __forceinline__ void vcompute_store_kind(int kind, typename Ty::S* st,
                                                    const VRec* rec, int cnt,
                                                    const VArgs<Ty>& g, typename Ty::A alpha,
                                                    typename Ty::A beta, bool all_bz,
                                                    bool alpha_one, bool skip_ab) {
    if constexpr (s <= 16) {
        if (kind == s - 1) {
            using K = VKindCfg<Ty, s>;
            if constexpr (K::ok) {
                using Cf = typename K::Cf;
                // every entry of C has one owning thread, which reads its old
                // value and writes the result in the same slot: C in place
                if constexpr (vshifted<Cf>()) {
                    constexpr int SV = vslot_elems<Cf>();
                    typename Ty::S* sC = st + 2 * cnt * SV;
                    vcompute_shifted<Cf>(st, st + cnt * SV, sC, rec, cnt, g.A_, g.B_, g.C_, alpha,
                                         beta, all_bz, alpha_one, skip_ab);
                    __syncthreads();
                    vstore_shifted<typename Ty::S, Cf::SC, SV, kVThreads>(g.C_, sC, rec, cnt);
                } else {
                    constexpr int Q = slot_quantum<Cf>();
                    const int P = (cnt + Q - 1) / Q * Q;
                    typename Ty::S* sC = st + P * (Cf::SA_P + Cf::SB_P);
                    vcompute_kind<Cf>(st, rec, cnt, P, sC, alpha, beta, all_bz, alpha_one, skip_ab);
                    __syncthreads();
                    vstore_fixed<typename Ty::S, Cf::SC, Cf::SC_P, kVThreads>(g.C_, sC, rec, cnt);
                }
            }
            return;
        }
        vcompute_store_kind<Ty, s + 1>(kind, st, rec, cnt, g, alpha, beta, all_bz, alpha_one,
                                       skip_ab);
    }
}

template <class Ty>
__global__ void __launch_bounds__(kVThreads, vblocks_of(Ty::code)) vbatch_kernel(VArgs<Ty> g)
{
    // Software pipeline of one block over the tiles it takes from the queue
    // (its j-th tile is "tile j"; D = pipeline stages).  Every tile needs, in order:
    // its queue index, its descriptor (VItem), its records, its data.  Each
    // is fetched asynchronously D - 1 iterations before the next step needs
    // it, all in the one cp.async group an iteration commits:
    //   iteration j waits for group j - D + 1, then issues
    //     data of tile j + D - 1      (records arrived with group j - D + 1)
    //     records of tile j + 2D - 2  (descriptor arrived with group j - D + 1)
    //     descriptor of tile j + 3D - 3 (index popped during iteration j - 1)
    //   and computes tile j while D - 1 tiles of data are in flight.
    // Queue indices of one block increase, so the first empty descriptor
    // (an index past the end) ends the block's work.
    using S = typename Ty::S;
    using A = typename Ty::A;
    constexpr int D = vstages_of(Ty::code);
    constexpr int kStageBytes = vstage_bytes_of(Ty::code);
    constexpr int kRecSlots = vrec_slots_of(Ty::code);
    constexpr int kItemSlots = vitem_slots_of(Ty::code);
    constexpr int kLead = 3 * D - 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_base;

    VRec* recbase = reinterpret_cast<VRec*>(smem_raw + D * kStageBytes);
    VItem* sitem = reinterpret_cast<VItem*>(smem_raw + D * kStageBytes +
                                            kRecSlots * kVMaxTile * sizeof(VRec));
    auto stage_of = [&](int t) { return reinterpret_cast<S*>(smem_raw + (t % D) * kStageBytes); };
    auto recs_of = [&](int t) { return recbase + (t % kRecSlots) * kVMaxTile; };
    auto item_of = [&](int t) -> VItem& { return sitem[t % kItemSlots]; };

    A alpha = g.alpha, beta = g.beta;
    bool all_bz = g.beta_zero != 0, az = g.alpha_zero != 0;
    if (g.alpha_ptr) { alpha = *g.alpha_ptr; az = is_zero(alpha); }
    if (g.beta_ptr)  { beta = *g.beta_ptr;   all_bz = is_zero(beta); }
    const bool alpha_one = is_one(alpha);
    const bool skip_ab = az;
    const int tid = threadIdx.x;
    const int n_items = g.n_items;

    // records of tile t (its descriptor is in shared memory)
    auto issue_recs = [&](int t) {
        const VItem it = item_of(t);
        if (it.count == 0) return;
        const char* src = reinterpret_cast<const char*>(g.recs + it.first);
        char* dst = reinterpret_cast<char*>(recs_of(t));
        for (int c = tid; c < it.count * 2; c += kVThreads)     // 16-byte halves of 32-byte records
            cp_async16(dst + 16 * c, src + 16 * c, 16);
    };
    // data of tile t (its records are in shared memory)
    auto issue_data = [&](int t) {
        const VItem it = item_of(t);
        if (it.count == 0) return;
        S* st = stage_of(t);
        const VRec* rb = recs_of(t);
        if (it.kind == kVGeneric) {
            const int m = it.shape & 255, n = (it.shape >> 8) & 255, k = (it.shape >> 16) & 255;
            vstage<S, kVThreads>(st, rb, it.count, g.A_, g.B_, g.C_, m * k, k * n, m * n, m * k,
                                 k * n, m * n, it.count, skip_ab, all_bz);
        } else {
            vstage_kind<Ty>(it.kind, st, rb, it.count, g, skip_ab, all_bz);
        }
    };

    // prologue: queue indices of tiles 0 .. kLead-1 in one pop, descriptors
    // by plain loads, records of tiles 0 .. 2D-3, then data of tiles
    // 0 .. D-2 (one group each)
    if (tid == 0) s_base = atomicAdd(g.counter, kLead);
    __syncthreads();
    const int base = s_base;
    if (base >= n_items) return;
    int pend = n_items;
    if (tid == 0) pend = atomicAdd(g.counter, 1);                 // tile kLead
    for (int t = tid; t < kLead; t += kVThreads) {
        VItem v = {0, 0, 0, 0};
        if (base + t < n_items) v = g.items[base + t];
        item_of(t) = v;
    }
    __syncthreads();
    for (int t = 0; t < 2 * D - 2; ++t) issue_recs(t);
    cp_async_commit();
    cp_async_wait_dyn(0);
    __syncthreads();
    for (int t = 0; t < D - 1; ++t) {
        issue_data(t);
        cp_async_commit();
    }

    for (int j = 0;; ++j) {
        cp_async_wait_dyn(D - 2);      // data of tile j, records of j+D-1, descriptor of j+2D-2
        __syncthreads();
        const VItem ci = item_of(j);
        if (ci.count == 0) break;
        issue_data(j + D - 1);
        issue_recs(j + 2 * D - 2);
        if (tid == 0) {
            VItem* dst = &item_of(j + kLead);
            if (pend < n_items) {
                cp_async16(dst, g.items + pend, 16);
                pend = atomicAdd(g.counter, 1);    // tile j + kLead + 1; read next iteration
            } else {
                *dst = VItem{0, 0, 0, 0};
            }
        }
        cp_async_commit();

        const VRec* rc = recs_of(j);
        S* st = stage_of(j);
        if (ci.kind == kVGeneric) {
            const int m = ci.shape & 255, n = (ci.shape >> 8) & 255, k = (ci.shape >> 16) & 255;
            const int ta = (ci.shape >> 24) & 1, tb = (ci.shape >> 25) & 1;
            S* sC = st + ci.count * (m * k + k * n);      // C slots: results in place
            vcompute_generic<Ty>(st, rc, ci.count, ci.count, sC, m, n, k, ta, tb,
                                 alpha, beta, all_bz, skip_ab);
            __syncthreads();
            vstore<S, kVThreads>(g.C_, sC, rc, ci.count, m * n, m * n);
        } else {
            vcompute_store_kind<Ty>(ci.kind, st, rc, ci.count, g, alpha, beta,
                                    all_bz, alpha_one, skip_ab);
        }
        // every thread is past this tile's stage, records and descriptor
        // before the next iteration refills them
        __syncthreads();
    }
    cp_async_wait_dyn(0);
}

constexpr size_t vbatch_smem_bytes(int type) {
    return (size_t)vstages_of(type) * vstage_bytes_of(type) +
           (size_t)vrec_slots_of(type) * kVMaxTile * sizeof(VRec) +
           (size_t)vitem_slots_of(type) * sizeof(VItem);
}

// Host: kind table of one type, and the launcher.
template <class Ty>
void vkind_table(VKindInfo* out) {
    constexpr VKindInfo t[16] = {
        vkind_info_one<Ty, 1>(), vkind_info_one<Ty, 2>(), vkind_info_one<Ty, 3>(), vkind_info_one<Ty, 4>(),
        vkind_info_one<Ty, 5>(), vkind_info_one<Ty, 6>(), vkind_info_one<Ty, 7>(), vkind_info_one<Ty, 8>(),
        vkind_info_one<Ty, 9>(), vkind_info_one<Ty, 10>(), vkind_info_one<Ty, 11>(), vkind_info_one<Ty, 12>(),
        vkind_info_one<Ty, 13>(), vkind_info_one<Ty, 14>(), vkind_info_one<Ty, 15>(), vkind_info_one<Ty, 16>()};
    for (int i = 0; i < 16; ++i) out[i] = t[i];
}

template <class Ty>
sbgemm_status vbatch_launch(const VItem* items, int n_items, const VRec* recs, int* counter,
                            const void* A, const void* B, void* C, const void* alpha,
                            const void* beta, int scalar_mode, int beta_zero, int alpha_zero,
                            cudaStream_t stream) {
    using S = typename Ty::S;
    using Asc = typename Ty::A;
    VArgs<Ty> g;
    g.items = items; g.n_items = n_items; g.recs = recs; g.counter = counter;
    g.A_ = static_cast<const S*>(A); g.B_ = static_cast<const S*>(B); g.C_ = static_cast<S*>(C);
    if (scalar_mode == SBGEMM_SCALARS_DEVICE) {
        g.alpha_ptr = static_cast<const Asc*>(alpha); g.beta_ptr = static_cast<const Asc*>(beta);
        g.alpha = Asc(); g.beta = Asc(); g.beta_zero = 0; g.alpha_zero = 0;
    } else {
        g.alpha_ptr = nullptr; g.beta_ptr = nullptr;
        g.alpha = *static_cast<const Asc*>(alpha); g.beta = *static_cast<const Asc*>(beta);
        g.beta_zero = beta_zero; g.alpha_zero = alpha_zero;
    }
    g.max_tile = kVMaxTile;
    const size_t smem = vbatch_smem_bytes(Ty::code);
    // per instantiation and device
    static DeviceFlags attr;
    static thread_local OccCache occ;
    cudaError_t ae = ensure_smem_limit(vbatch_kernel<Ty>, (int)smem, attr);
    if (ae != cudaSuccess) return (sbgemm_status)ae;
    int per_sm = 0;
    ae = blocks_per_sm(vbatch_kernel<Ty>, kVThreads, smem, occ, &per_sm);
    if (ae != cudaSuccess) return (sbgemm_status)ae;
    if (per_sm < 1) return SBGEMM_ERR_NOT_SUPPORTED;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
    if (e != cudaSuccess) return (sbgemm_status)e;
    long long grid = (long long)num_sms() * per_sm;
    if (grid > n_items) grid = n_items;
    if (grid < 1) grid = 1;
    vbatch_kernel<Ty><<<(unsigned)grid, kVThreads, smem, stream>>>(g);
    return (sbgemm_status)cudaGetLastError();
}

}  // namespace sbg
