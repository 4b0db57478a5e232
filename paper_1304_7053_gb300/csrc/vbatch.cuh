// Variable-size batches: one persistent launch over a device work queue.
//
// The paper notes (Section 1) that matrices of different sizes can be
// partitioned into sets of identical size.  Here the partition is a host
// plan: problems are bucketed by (m, n, k, op), buckets are cut into tiles,
// and one persistent kernel takes tiles from an atomic counter, runs the
// size-specialised compute of the tile's bucket (the same register-blocked
// code as the fixed-size path), and double-buffers the next tile's staging
// behind the current tile's compute.  Each problem's matrices are contiguous
// (minimal leading dimensions) at arbitrary arena offsets, so staging gathers
// element-wise with asynchronous copies.
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
constexpr int kVStageBytes = 48 * 1024;
constexpr int kVMaxTile = 128;

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
// tile needs another block size fall back to the generic kind.
template <class Ty, int s>
struct VKindCfg {
    static constexpr TileEntry te = tile_for(Ty::code, s, s, s, 0, 0);
    using Cf = Cfg<Ty, s, s, s, false, false, te.tm, te.tn, te.si != 0, te.sj != 0, te.nt>;
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

// Host view of a kind: matrices per compute round, staged bytes per pair
// (A, B and old C slots), slot quantum.
struct VKindInfo { int mpr; int bytes_per_pair; int quantum; };

template <class Ty, int s>
constexpr VKindInfo vkind_info_one() {
    using K = VKindCfg<Ty, s>;
    using Cf = typename K::Cf;
    return K::ok ? VKindInfo{Cf::MPR, (Cf::SA_P + Cf::SB_P + Cf::SC_P) * Cf::ES, slot_quantum<Cf>()}
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

// Stage a tile of a specialised kind (square size, compile-time slot sizes):
// each warp takes whole problems; when a matrix is shorter than a warp, the
// warp's lanes split into groups of SE lanes, one problem per group.
template <class S, int SE, int SP, int NT>
__device__ __forceinline__ void vstage_fixed(S* st, int which, const VRec* rec, int cnt,
                                             const S* g, bool need_all) {
    constexpr int ES = sizeof(S);
    constexpr int PPW = SE >= 32 ? 1 : 32 / SE;         // problems per warp pass
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    const int sub = PPW > 1 ? lane / SE : 0;
    const int l2 = PPW > 1 ? lane - sub * SE : lane;
    if (PPW > 1 && sub >= PPW) return;
    for (int q0 = warp * PPW; q0 < cnt; q0 += NW * PPW) {
        const int q = q0 + sub;
        if (q >= cnt) break;
        const VRec& r = rec[q];
        if (!need_all && (r.flags & 16)) continue;      // old C not needed (beta_q = 0)
        const long long off = which == 0 ? r.a : which == 1 ? r.b : r.c;
        const S* src = g + off;
        S* dst = st + q * SP;
        if (PPW > 1) vcopy_elem<S, ES>(dst + l2, src + l2);
        else vcopy_matrix<S, ES>(dst, src, SE, lane);
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
                constexpr int Q = slot_quantum<Cf>();
                const int P = (cnt + Q - 1) / Q * Q;
                if (!skip_ab) {
                    vstage_fixed<S, Cf::SA, Cf::SA_P, kVThreads>(st, 0, rec, cnt, g.A_, true);
                    vstage_fixed<S, Cf::SB, Cf::SB_P, kVThreads>(st + P * Cf::SA_P, 1, rec, cnt, g.B_, true);
                }
                if (!all_bz)
                    vstage_fixed<S, Cf::SC, Cf::SC_P, kVThreads>(st + P * (Cf::SA_P + Cf::SB_P), 2, rec,
                                                                 cnt, g.C_, false);
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
                constexpr int Q = slot_quantum<Cf>();
                const int P = (cnt + Q - 1) / Q * Q;
                // every entry of C has one owning thread, which reads its old
                // value and writes the result in the same slot: C in place
                typename Ty::S* sC = st + P * (Cf::SA_P + Cf::SB_P);
                vcompute_kind<Cf>(st, rec, cnt, P, sC, alpha, beta, all_bz, alpha_one, skip_ab);
                __syncthreads();
                vstore<typename Ty::S, kVThreads>(g.C_, sC, rec, cnt, Cf::SC, Cf::SC_P);
            }
            return;
        }
        vcompute_store_kind<Ty, s + 1>(kind, st, rec, cnt, g, alpha, beta, all_bz, alpha_one,
                                       skip_ab);
    }
}

template <class Ty>
__global__ void __launch_bounds__(kVThreads) vbatch_kernel(VArgs<Ty> g)
{
    // Pipeline per block, iteration i:
    //   wait for group i-1 (data of tile i, records of tile i+1);
    //   issue group i: data of tile i+1, records of tile i+2 (its index was
    //   popped from the queue during iteration i-1);
    //   pop the index of tile i+3 (its latency overlaps the compute);
    //   compute tile i and write its C.
    using S = typename Ty::S;
    using A = typename Ty::A;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item[4];

    S* stage[2] = {reinterpret_cast<S*>(smem_raw), reinterpret_cast<S*>(smem_raw + kVStageBytes)};
    VRec* recbase = reinterpret_cast<VRec*>(smem_raw + 2 * kVStageBytes);

    A alpha = g.alpha, beta = g.beta;
    bool all_bz = g.beta_zero != 0, az = g.alpha_zero != 0;
    if (g.alpha_ptr) { alpha = *g.alpha_ptr; az = is_zero(alpha); }
    if (g.beta_ptr)  { beta = *g.beta_ptr;   all_bz = is_zero(beta); }
    const bool alpha_one = is_one(alpha);
    const bool skip_ab = az;
    const int tid = threadIdx.x;
    const int n_items = g.n_items;

    // asynchronous copy of a tile's records into record buffer slot rb
    auto issue_recs = [&](int item, int rb) {
        if (item >= n_items) return;
        const VItem it = g.items[item];
        const char* src = reinterpret_cast<const char*>(g.recs + it.first);
        char* dst = reinterpret_cast<char*>(recbase + rb * kVMaxTile);
        for (int c = tid; c < it.count * 2; c += kVThreads)     // 16-byte halves of 32-byte records
            cp_async16(dst + 16 * c, src + 16 * c, 16);
    };
    auto issue_data = [&](int item, S* st, const VRec* rb) {
        if (item >= n_items) return;
        const VItem it = g.items[item];
        if (it.kind == kVGeneric) {
            const int m = it.shape & 255, n = (it.shape >> 8) & 255, k = (it.shape >> 16) & 255;
            vstage<S, kVThreads>(st, rb, it.count, g.A_, g.B_, g.C_, m * k, k * n, m * n, m * k,
                                 k * n, m * n, it.count, skip_ab, all_bz);
        } else {
            vstage_kind<Ty>(it.kind, st, rb, it.count, g, skip_ab, all_bz);
        }
    };

    // prologue: tiles 0, 1 and 2 of this block
    if (tid < 3) s_item[tid] = atomicAdd(g.counter, 1);
    __syncthreads();
    int item0 = s_item[0], item1 = s_item[1], item2 = s_item[2];
    if (item0 >= n_items) return;
    issue_recs(item0, 0);
    cp_async_commit();
    cp_async_wait_dyn(0);
    __syncthreads();
    issue_data(item0, stage[0], recbase);
    issue_recs(item1, 1);
    cp_async_commit();
    int pend = 0;
    if (tid == 0) pend = atomicAdd(g.counter, 1);   // tile 3

    int cur = item0, nxt = item1, nxt2 = item2;
    for (int it = 0;; ++it) {
        const int b = it & 1;
        const int rcur = it % 3, rnxt = (it + 1) % 3, rnxt2 = (it + 2) % 3;
        cp_async_wait_dyn(0);          // data of cur, records of nxt
        if (tid == 0) s_item[3] = pend;
        __syncthreads();
        const int nxt3 = s_item[3];
        issue_data(nxt, stage[b ^ 1], recbase + rnxt * kVMaxTile);
        issue_recs(nxt2, rnxt2);
        cp_async_commit();
        if (tid == 0 && nxt3 < n_items) pend = atomicAdd(g.counter, 1);
        else if (tid == 0) pend = n_items;

        const VItem ci = g.items[cur];
        const VRec* rc = recbase + rcur * kVMaxTile;
        if (ci.kind == kVGeneric) {
            const int m = ci.shape & 255, n = (ci.shape >> 8) & 255, k = (ci.shape >> 16) & 255;
            const int ta = (ci.shape >> 24) & 1, tb = (ci.shape >> 25) & 1;
            S* sC = stage[b] + ci.count * (m * k + k * n);      // C slots: results in place
            vcompute_generic<Ty>(stage[b], rc, ci.count, ci.count, sC, m, n, k, ta, tb,
                                 alpha, beta, all_bz, skip_ab);
            __syncthreads();
            vstore<S, kVThreads>(g.C_, sC, rc, ci.count, m * n, m * n);
        } else {
            vcompute_store_kind<Ty>(ci.kind, stage[b], rc, ci.count, g, alpha, beta,
                                    all_bz, alpha_one, skip_ab);
        }
        if (nxt >= n_items) break;
        // the copy-out above reads sOut and the record buffer of cur: every
        // thread is past it before they are refilled
        __syncthreads();
        cur = nxt;
        nxt = nxt2;
        nxt2 = nxt3;
    }
    cp_async_wait_dyn(0);
}

constexpr size_t vbatch_smem_bytes() {
    return 2 * (size_t)kVStageBytes + 3 * (size_t)kVMaxTile * sizeof(VRec);
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
    const size_t smem = vbatch_smem_bytes();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(vbatch_kernel<Ty>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return (sbgemm_status)e;
        attr = true;
    }
    static thread_local int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vbatch_kernel<Ty>,
                                                                      kVThreads, smem);
        if (e != cudaSuccess) return (sbgemm_status)e;
        if (per_sm < 1) return SBGEMM_ERR_NOT_SUPPORTED;
    }
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
    if (e != cudaSuccess) return (sbgemm_status)e;
    long long grid = (long long)num_sms() * per_sm;
    if (grid > n_items) grid = n_items;
    if (grid < 1) grid = 1;
    vbatch_kernel<Ty><<<(unsigned)grid, kVThreads, smem, stream>>>(g);
    return (sbgemm_status)cudaGetLastError();
}

}  // namespace sbg
