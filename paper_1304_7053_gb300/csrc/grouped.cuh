// Several uniform batches in one persistent launch.
//
// Each group is one batch of Eq. (1) on the Section 4 layout: square
// m = n = k, op N/N, flat 16-byte-aligned storage.  The tiles of every group
// form one index space (groups ordered by tile cost, largest first); the
// blocks walk it grid-stride through one cp.async pipeline whose stages hold
// a tile of any group, and each tile runs the register-blocked compute of its
// group's size.  One launch instead of one per group removes the per-launch
// ramp and tail of every small kernel.  Staging uses 16-byte cp.async
// chunks: one bulk copy per operand and tile (the fixed-size kernels' path
// for large unpadded matrices) measured 3-5% slower here, where a block has
// one tile in flight.
#pragma once

#include <algorithm>
#include <cstring>

#include "sbgemm_launch.cuh"

namespace sbg {

constexpr int kGMaxGroups = 32;

// Launch configuration of the grouped kernel: threads per block (128 or 256),
// bytes of one pipeline stage and the pipeline depth.  The output tile (for
// shapes without direct stores) is half a stage.
struct GConfig { int threads, stage_bytes, stages; };
// (the default is the fastest of a sweep over threads x stage bytes x depth
// on the fp32 and fp64 sizes 1..16 workloads: 70 KB of shared memory, three
// blocks of 128 threads per SM)
constexpr GConfig kGDefault = {128, 28 * 1024, 2};

inline size_t gsmem_bytes(const GConfig& c) {
    return (size_t)c.stages * c.stage_bytes + (size_t)c.stage_bytes / 2;
}

template <class Ty>
struct GGroup {
    const typename Ty::S* A;
    const typename Ty::S* B;
    typename Ty::S* C;
    long long batch;
    int kind;        // square size - 1
    int P;           // pairs per tile
    int tile0;       // first global tile index of the group
    int tiles;
};

template <class Ty>
struct GArgs {
    using A = typename Ty::A;
    GGroup<Ty> grp[kGMaxGroups];
    int ngroups;
    int total_tiles;
    int stage_elems;   // elements of one stage
    int stages;
    A alpha, beta;
    const A* alpha_ptr;
    const A* beta_ptr;
    int beta_zero, alpha_zero;
};

// Register tile of size s from the table, run with NT threads per block
// (a shape whose threads per matrix exceed NT is not fused).
template <class Ty, int s, int NT>
struct GKindCfg {
    static constexpr TileEntry te = tile_for(Ty::code, s, s, s, 0, 0);
    static constexpr int tpm = ((s + te.tm - 1) / te.tm) * ((s + te.tn - 1) / te.tn);
    static constexpr bool ok = tpm <= NT;
    using Cf = Cfg<Ty, s, s, s, false, false, te.tm, te.tn, te.si != 0, te.sj != 0, ok ? NT : te.nt>;
};

struct GKindInfo { int ok, mpr, sa_p, sb_p, sc_p, es, quantum, vs; };

template <class Ty, int s, int NT>
constexpr GKindInfo gkind_info_one() {
    using K = GKindCfg<Ty, s, NT>;
    using Cf = typename K::Cf;
    constexpr int q = lcm_c(lcm_c(16 / gcd_c(Cf::SA * Cf::ES, 16), 16 / gcd_c(Cf::SB * Cf::ES, 16)),
                             16 / gcd_c(Cf::SC * Cf::ES, 16));
    return GKindInfo{K::ok ? 1 : 0, Cf::MPR, Cf::SA_P, Cf::SB_P, Cf::SC_P, Cf::ES, q, Cf::VS};
}

// Stage one tile of a group (the kind is uniform in the block).
template <class Ty, int NT, int s = 1>
__device__ __forceinline__ void gstage(int kind, typename Ty::S* st, const GGroup<Ty>& G,
                                       long long p0, int cnt, int P, bool skip_ab, bool beta_zero) {
    if constexpr (s <= 16) {
        if (kind == s - 1) {
            using K = GKindCfg<Ty, s, NT>;
            if constexpr (K::ok) {
                using Cf = typename K::Cf;
                using S = typename Ty::S;
                if (!skip_ab) {
                    stage_operand<S, Cf::SA, Cf::SA_P, Cf::RA, Cf::NT>(st, G.A, Cf::SA, Cf::RA, p0, cnt, true);
                    stage_operand<S, Cf::SB, Cf::SB_P, Cf::RB, Cf::NT>(st + P * Cf::SA_P, G.B, Cf::SB, Cf::RB,
                                                                       p0, cnt, true);
                }
                if (!beta_zero)
                    stage_operand<S, Cf::SC, Cf::SC_P, Cf::M, Cf::NT>(st + P * (Cf::SA_P + Cf::SB_P), G.C,
                                                                      Cf::SC, Cf::M, p0, cnt, true);
            }
            return;
        }
        gstage<Ty, NT, s + 1>(kind, st, G, p0, cnt, P, skip_ab, beta_zero);
    }
}

// Compute one tile and write its C (direct 16-byte stores when the shape
// allows them, else through the shared output tile).
template <class Ty, int NT, int s = 1>
__device__ __forceinline__ void gcompute(int kind, const typename Ty::S* st, typename Ty::S* sOut,
                                         const GGroup<Ty>& G, long long p0, int cnt, int P,
                                         typename Ty::A alpha, typename Ty::A beta, bool beta_zero,
                                         bool alpha_one, bool skip_ab) {
    if constexpr (s <= 16) {
        if (kind == s - 1) {
            using K = GKindCfg<Ty, s, NT>;
            if constexpr (K::ok) {
                using Cf = typename K::Cf;
                using S = typename Ty::S;
                const int tid = threadIdx.x;
                const int ql = tid / Cf::TPM;
                const int u = tid - ql * Cf::TPM;
                const int ti = u % Cf::TI, tj = u / Cf::TI;
                constexpr bool direct = Cf::VS > 0;
                S* gC = G.C + p0 * Cf::SC;
                if (ql < Cf::MPR) {
                    for (int q = ql; q < cnt; q += Cf::MPR)
                        compute_block<Cf>(st, st + P * Cf::SA_P, st + P * (Cf::SA_P + Cf::SB_P), sOut,
                                          gC, direct, q, ti, tj, alpha, beta, beta_zero, alpha_one,
                                          skip_ab, typename Cf::R(1), typename Cf::R(1));
                }
                if constexpr (!direct) {
                    __syncthreads();
                    store_operand<S, Cf::SC, Cf::SC_P, Cf::M, Cf::NT>(G.C, sOut, Cf::SC, Cf::M, p0, cnt, true);
                }
            }
            return;
        }
        gcompute<Ty, NT, s + 1>(kind, st, sOut, G, p0, cnt, P, alpha, beta, beta_zero, alpha_one, skip_ab);
    }
}

// Minimum resident blocks: three of 128 threads (the default configuration;
// the compiler may then use up to 168 registers, and took 168 where it chose
// 148 without the bound, 2% faster per step: 324.6 against 331.8 us), two
// of 256.
template <class Ty, int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 3) grouped_kernel(GArgs<Ty> g)
{
    using S = typename Ty::S;
    using A = typename Ty::A;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");

    A alpha = g.alpha, beta = g.beta;
    bool beta_zero = g.beta_zero != 0, alpha_zero = g.alpha_zero != 0;
    if (g.alpha_ptr) { alpha = *g.alpha_ptr; alpha_zero = is_zero(alpha); }
    if (g.beta_ptr)  { beta = *g.beta_ptr;   beta_zero = is_zero(beta); }
    const bool alpha_one = is_one(alpha);
    const bool skip_ab = alpha_zero;
    const int stages = g.stages;
    const int stage_elems = g.stage_elems;
    S* stage_base = reinterpret_cast<S*>(smem_raw);
    S* sOut = stage_base + stages * stage_elems;
    const int T = g.total_tiles;

    // A block's tiles come in increasing order, so the group of the next
    // tile is found by moving forward from the previous one (one index for
    // the tiles issued, one for the tiles computed).  Searching from the
    // first group for every tile cost 12 us of the 323 us fp32 sizes 1..16
    // step (the group records are kernel parameters, read per field).
    int gi_issue = 0, gi_comp = 0;
    auto group_from = [&](int t, int& gi) {
        while (gi + 1 < g.ngroups && t >= g.grp[gi + 1].tile0) ++gi;
        return gi;
    };
    auto issue = [&](int t, int s) {
        const GGroup<Ty>& G = g.grp[group_from(t, gi_issue)];
        const long long p0 = (long long)(t - G.tile0) * G.P;
        const int cnt = (int)min((long long)G.P, G.batch - p0);
        gstage<Ty, NT>(G.kind, stage_base + s * stage_elems, G, p0, cnt, G.P, skip_ab, beta_zero);
    };

    for (int s = 0; s < stages - 1; ++s) {
        const int t = blockIdx.x + s * gridDim.x;
        if (t < T) issue(t, s);
        cp_async_commit();
    }
    int it = 0;
    for (int t = blockIdx.x; t < T; t += gridDim.x, ++it) {
        const int tn = t + (stages - 1) * gridDim.x;
        if (tn < T) issue(tn, (it + stages - 1) % stages);
        cp_async_commit();
        cp_async_wait_dyn(stages - 1);
        __syncthreads();
        const GGroup<Ty>& G = g.grp[group_from(t, gi_comp)];
        const long long p0 = (long long)(t - G.tile0) * G.P;
        const int cnt = (int)min((long long)G.P, G.batch - p0);
        gcompute<Ty, NT>(G.kind, stage_base + (it % stages) * stage_elems, sOut, G, p0, cnt, G.P,
                         alpha, beta, beta_zero, alpha_one, skip_ab);
        // every thread is done with this stage (and the output tile) before reuse
        __syncthreads();
    }
    cp_async_wait_dyn(0);
}

// Host: kind table of one type and the launcher for up to kGMaxGroups groups.
struct GIn { const void* A; const void* B; void* C; int m; long long batch; };

template <class Ty, int NT>
void gkind_table_nt(GKindInfo* out) {
    constexpr GKindInfo t[16] = {
        gkind_info_one<Ty, 1, NT>(), gkind_info_one<Ty, 2, NT>(), gkind_info_one<Ty, 3, NT>(),
        gkind_info_one<Ty, 4, NT>(), gkind_info_one<Ty, 5, NT>(), gkind_info_one<Ty, 6, NT>(),
        gkind_info_one<Ty, 7, NT>(), gkind_info_one<Ty, 8, NT>(), gkind_info_one<Ty, 9, NT>(),
        gkind_info_one<Ty, 10, NT>(), gkind_info_one<Ty, 11, NT>(), gkind_info_one<Ty, 12, NT>(),
        gkind_info_one<Ty, 13, NT>(), gkind_info_one<Ty, 14, NT>(), gkind_info_one<Ty, 15, NT>(),
        gkind_info_one<Ty, 16, NT>()};
    for (int i = 0; i < 16; ++i) out[i] = t[i];
}

template <class Ty>
void gkind_table(int threads, GKindInfo* out) {
    if (threads == 256) gkind_table_nt<Ty, 256>(out);
    else gkind_table_nt<Ty, 128>(out);
}

// Pairs per tile of a group: whole compute rounds that fit one stage (and,
// without direct stores, the output tile), rounded down to the group's
// 16-byte quantum.  0 when not even one quantum fits.
inline int gtile_pairs(const GKindInfo& k, bool beta_zero, const GConfig& c) {
    const int bpp = (k.sa_p + k.sb_p + (beta_zero ? 0 : k.sc_p)) * k.es;
    int P = c.stage_bytes / bpp;
    if (k.vs == 0) P = std::min(P, (c.stage_bytes / 2) / (k.sc_p * k.es));
    if (P >= k.mpr) P = P / k.mpr * k.mpr;
    P = P / k.quantum * k.quantum;
    return P;
}

template <class Ty, int NT>
sbgemm_status grouped_launch_nt(const GIn* in, int n, const void* alpha, const void* beta,
                                int scalar_mode, int beta_zero, int alpha_zero,
                                const GConfig& cfg, cudaStream_t stream) {
    using S = typename Ty::S;
    using Asc = typename Ty::A;
    GKindInfo kinfo[16];
    gkind_table_nt<Ty, NT>(kinfo);
    GArgs<Ty> g;
    std::memset(&g, 0, sizeof g);
    // order: largest per-tile cost first
    int order[kGMaxGroups];
    for (int i = 0; i < n; ++i) order[i] = i;
    std::sort(order, order + n, [&](int a, int b) { return in[a].m > in[b].m; });
    int tile0 = 0;
    for (int j = 0; j < n; ++j) {
        const GIn& x = in[order[j]];
        const GKindInfo& k = kinfo[x.m - 1];
        const int P = gtile_pairs(k, beta_zero != 0, cfg);
        if (!k.ok || P < 1) return SBGEMM_ERR_NOT_SUPPORTED;
        GGroup<Ty>& G = g.grp[j];
        G.A = static_cast<const S*>(x.A);
        G.B = static_cast<const S*>(x.B);
        G.C = static_cast<S*>(x.C);
        G.batch = x.batch;
        G.kind = x.m - 1;
        G.P = P;
        G.tile0 = tile0;
        G.tiles = (int)((x.batch + P - 1) / P);
        tile0 += G.tiles;
    }
    g.ngroups = n;
    g.total_tiles = tile0;
    g.stage_elems = cfg.stage_bytes / (int)sizeof(S);
    g.stages = cfg.stages;
    if (scalar_mode == SBGEMM_SCALARS_DEVICE) {
        g.alpha_ptr = static_cast<const Asc*>(alpha); g.beta_ptr = static_cast<const Asc*>(beta);
        g.alpha = Asc(); g.beta = Asc(); g.beta_zero = 0; g.alpha_zero = 0;
    } else {
        g.alpha_ptr = nullptr; g.beta_ptr = nullptr;
        g.alpha = *static_cast<const Asc*>(alpha); g.beta = *static_cast<const Asc*>(beta);
        g.beta_zero = beta_zero; g.alpha_zero = alpha_zero;
    }
    auto kern = grouped_kernel<Ty, NT>;
    const size_t smem = gsmem_bytes(cfg);
    // per instantiation and device
    static DeviceFlags attr;
    static thread_local OccCache occ;
    cudaError_t ae = ensure_smem_limit(kern, 220 * 1024, attr);
    if (ae != cudaSuccess) return (sbgemm_status)ae;
    int occ_val = 0;
    ae = blocks_per_sm(kern, NT, smem, occ, &occ_val);
    if (ae != cudaSuccess) return (sbgemm_status)ae;
    if (occ_val < 1) return SBGEMM_ERR_NOT_SUPPORTED;
    long long grid = (long long)num_sms() * occ_val;
    if (grid > g.total_tiles) grid = g.total_tiles;
    if (grid < 1) return SBGEMM_SUCCESS;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(NT);
    lc.dynamicSmemBytes = smem;
    lc.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&lc, kern, g);
    if (e != cudaSuccess) return (sbgemm_status)e;
    return (sbgemm_status)cudaGetLastError();
}

template <class Ty>
sbgemm_status grouped_launch(const GIn* in, int n, const void* alpha, const void* beta,
                             int scalar_mode, int beta_zero, int alpha_zero, const GConfig& cfg,
                             cudaStream_t stream) {
    if (cfg.threads == 256)
        return grouped_launch_nt<Ty, 256>(in, n, alpha, beta, scalar_mode, beta_zero, alpha_zero,
                                          cfg, stream);
    return grouped_launch_nt<Ty, 128>(in, n, alpha, beta, scalar_mode, beta_zero, alpha_zero, cfg,
                                      stream);
}

}  // namespace sbg
