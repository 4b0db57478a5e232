// Kernels and host-side launchers for the fixed-size uniform-layout path.
#pragma once

#include "device_setup.h"
#include "sbgemm_device.cuh"
#include "tile_table.h"
#include "../../include/sbgemm.h"

namespace sbg {

// Host request after argument checks (one per call).
struct Req {
    int type;
    int m, n, k;
    int ta, tb;            // stored-transposed flags (op = T or C)
    int conja, conjb;      // conjugation flags (complex types, op = C)
    const void* A; const void* B; void* C;
    int lda, ldb, ldc;
    long long lda2, ldb2, ldc2;
    int batch;
    int scalar_mode;
    const void* alpha;     // host or device pointer to one scalar
    const void* beta;
    int beta_zero;         // host scalars only
    int alpha_zero;
    int variant;
    cudaStream_t stream;
    // pointer-array form: device arrays of per-pair matrix pointers (the
    // 3-D layout fields A, B, C and the ld2 strides are then unused)
    const void* const* Ap; const void* const* Bp; void* const* Cp;
};

// Run-time launch options that do not change the kernel binary.
struct LaunchOpts {
    int tile_bytes;    // target staged input bytes per tile
    int stages;        // pipeline depth, 2..4
    int ctas_per_sm;   // 0 = as many as fit
};

// The variant table for the pipelined kernel; the last variant of every
// shape is the generic runtime-size kernel (one thread per C entry, the
// mapping of the paper's first method in Section 6).
constexpr int kNumPipeVariants = 6;
// Variant after the generic kernel: the tensor-core kernel of the 16-bit
// types (csrc/mma16.cuh), for m = n = k = 8, 12 or 16, op N/N, flat layouts,
// and of real and complex fp64 (csrc/ozaki.cuh, csrc/ozaki_z.cuh, any op
// and layout of the uniform form, and the pointer-array form); any other
// request given this variant runs variant 0.
constexpr int kMmaVariant = kNumPipeVariants + 1;
sbgemm_status run_mma16(const Req& r);   // mma16.cu
bool mma16_ok(const Req& r);
// The same variant index for real and complex fp64 runs the tensor-core
// kernels that split fp64 operands into exact 8-bit digits.
sbgemm_status run_ozaki(const Req& r);   // ozaki.cu
bool ozaki_ok(const Req& r);
inline LaunchOpts pipe_variant(int v, int type_code = 0) {
    // fp64 types are bound by the fp64 pipe, not by memory: two stages are
    // enough and leave room for more computing warps
    const bool fp64 = type_code == 1 || type_code == 3;
    switch (v) {
    case 1:  return {8192, 4, 0};
    case 2:  return {32768, 2, 0};
    case 3:  return {16384, fp64 ? 2 : 3, 1};
    case 4:  return {4096, 4, 0};
    case 5:  return {24576, 3, 2};
    default: return {16384, fp64 ? 2 : 3, 0};
    }
}

int num_sms();            // cached device attribute (api.cu)
int* device_error_ptr();  // the current device's error word (api.cu)

template <class Ty>
inline void fill_args(Args<Ty>& a, const Req& r) {
    using S = typename Ty::S;
    using A = typename Ty::A;
    a.A_ = static_cast<const S*>(r.A);
    a.B_ = static_cast<const S*>(r.B);
    a.C_ = static_cast<S*>(r.C);
    a.lda = r.lda; a.ldb = r.ldb; a.ldc = r.ldc;
    a.lda2 = r.lda2; a.ldb2 = r.ldb2; a.ldc2 = r.ldc2;
    a.batch = r.batch;
    if (r.scalar_mode == SBGEMM_SCALARS_DEVICE) {
        a.alpha_ptr = static_cast<const A*>(r.alpha);
        a.beta_ptr = static_cast<const A*>(r.beta);
        a.alpha = A(); a.beta = A();
        a.beta_zero = 0; a.alpha_zero = 0;
    } else {
        a.alpha_ptr = nullptr; a.beta_ptr = nullptr;
        a.alpha = *static_cast<const A*>(r.alpha);
        a.beta = *static_cast<const A*>(r.beta);
        a.beta_zero = r.beta_zero; a.alpha_zero = r.alpha_zero;
    }
    a.conja = r.conja ? typename Ty::R(-1) : typename Ty::R(1);
    a.conjb = r.conjb ? typename Ty::R(-1) : typename Ty::R(1);
    a.Ap = reinterpret_cast<const S* const*>(r.Ap);
    a.Bp = reinterpret_cast<const S* const*>(r.Bp);
    a.Cp = reinterpret_cast<S* const*>(r.Cp);
    a.shared = r.Cp ? 0 : (r.lda2 == 0 ? 1 : 0) | (r.ldb2 == 0 ? 2 : 0);
    a.flat = 0;
    a.err = device_error_ptr();
}

// Base of matrix p of an operand: pointer-array form or 3-D layout.
template <class S>
__device__ __forceinline__ const S* mat_of(const S* base, const S* const* ptrs, long long ld2,
                                           long long p) {
    return ptrs ? ldg_ptr(ptrs + p) : base + p * ld2;
}
template <class S>
__device__ __forceinline__ S* mat_of(S* base, S* const* ptrs, long long ld2, long long p) {
    return ptrs ? ldg_ptr(ptrs + p) : base + p * ld2;
}

// Shared-memory elements reserved for one shared (broadcast) matrix slot,
// rounded up to 16 bytes so the slot after it stays vector-aligned.
template <class S>
__host__ __device__ constexpr int shared_slot_elems(int slot_elems) {
    return (int)(((size_t)slot_elems * sizeof(S) + 15) / 16 * 16 / sizeof(S));
}

// ------------------------------------------------------------ pipelined kernel

// PF: the pointer-array form (a separate instantiation, so the 3-D layout
// kernels carry none of its code or registers).
template <class Cf, bool PF>
__global__ void __launch_bounds__(Cf::NT)
pipe_kernel(Args<typename Cf::Ty> g)
{
    using S = typename Cf::S;
    using A = typename Cf::A;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    // Launched with programmatic stream serialisation: this grid may start
    // while the previous kernel on the stream drains, so it waits for that
    // grid's completion (and memory) before touching global memory, then
    // lets the next launch begin its own set-up.
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");

    A alpha = g.alpha, beta = g.beta;
    bool beta_zero = g.beta_zero != 0, alpha_zero = g.alpha_zero != 0;
    const bool has_cold = !beta_zero;          // smem layout fixed by the host
    if (g.alpha_ptr) { alpha = *g.alpha_ptr; alpha_zero = is_zero(alpha); }
    if (g.beta_ptr)  { beta = *g.beta_ptr;   beta_zero = is_zero(beta); }
    const bool alpha_one = is_one(alpha);
    const bool skip_ab = alpha_zero;

    const int P = g.P;
    const int stages = g.stages;
    const long long batch = g.batch;
    const int ntiles = (int)((batch + P - 1) / P);
    const bool fa = g.flat & 1, fb = g.flat & 2, fc = g.flat & 4;
    const bool direct = (Cf::VS > 0) && fc;
    // A matrix shared by every pair (leading dimension 2 of zero) is staged
    // once per block into its own slot and left out of the tiles.
    const int sh = g.shared;
    const bool shA = sh & 1, shB = sh & 2;
    const int offB = shA ? 0 : P * Cf::SA_P;
    const int offC = offB + (shB ? 0 : P * Cf::SB_P);
    const int stage_elems = offC + (has_cold ? P * Cf::SC_P : 0);
    S* stage_base = reinterpret_cast<S*>(smem_raw);
    S* sOut = stage_base + stages * stage_elems;    // unused when C is stored directly
    S* sShA = sOut + (direct ? 0 : P * Cf::SC_P);
    S* sShB = sShA + (shA ? shared_slot_elems<S>(Cf::SA_P) : 0);
    // Pointer-array form: a ring of 2*stages + 1 slots, each with one tile's
    // A, B and C pointers.  The pointers of this block's tile j are fetched
    // (cp.async) with the group of iteration j - 2*stages + 1, so they have
    // arrived when the data of tile j is issued (iteration j - stages + 1),
    // and they stay until tile j's C has been written (end of iteration j).
    const S** sPtr = reinterpret_cast<const S**>(sShB + (shB ? shared_slot_elems<S>(Cf::SB_P) : 0));
    constexpr bool ptr_form = PF;
    const int ring = 2 * stages + 1;
    auto ptr_slot = [&](int j) { return sPtr + (j % ring) * 3 * P; };
    auto fetch_ptrs = [&](int j, bool async) {
        const long long t = blockIdx.x + (long long)j * gridDim.x;
        if (t >= ntiles) return;
        const long long p0 = t * P;
        const int cnt = (int)min((long long)P, batch - p0);
        const S** d = ptr_slot(j);
        for (int i = threadIdx.x; i < cnt; i += Cf::NT) {
            if (async) {
                cp_async_elem<8>(d + i, g.Ap + p0 + i);
                cp_async_elem<8>(d + P + i, g.Bp + p0 + i);
                cp_async_elem<8>(d + 2 * P + i, g.Cp + p0 + i);
            } else {
                d[i] = ldg_ptr(g.Ap + p0 + i);
                d[P + i] = ldg_ptr(g.Bp + p0 + i);
                d[2 * P + i] = ldg_ptr(g.Cp + p0 + i);
            }
        }
    };

    // Flat operands with unpadded slots of at least 480 bytes per matrix move
    // by one bulk copy per tile (measured faster for fp32 m = 11..15, slower
    // for smaller matrices, whose tiles are better served by many parallel
    // 16-byte cp.async requests).  Shapes with such an operand keep one
    // barrier per stage: the k-th use of stage s completes phase k once its
    // bulk copies have landed.
    constexpr int kBulkMin = 480;
    constexpr bool bulkA = !PF && Cf::SA_P == Cf::SA && Cf::SA * Cf::ES >= kBulkMin;
    constexpr bool bulkB = !PF && Cf::SB_P == Cf::SB && Cf::SB * Cf::ES >= kBulkMin;
    constexpr bool bulkC = !PF && Cf::SC_P == Cf::SC && Cf::SC * Cf::ES >= kBulkMin;
    constexpr bool kBulk = bulkA || bulkB || bulkC;
    __shared__ uint64_t s_bar[4];
    __shared__ int s_fail;
    if constexpr (kBulk) {
        if (threadIdx.x == 0) {
            for (int s = 0; s < stages; ++s) mbar_init(&s_bar[s], 1);
            mbar_fence_init();
            s_fail = 0;
        }
        __syncthreads();
    }

    auto issue = [&](int t, int s) {
        S* st = stage_base + s * stage_elems;
        const long long p0 = (long long)t * P;
        const int cnt = (int)min((long long)P, batch - p0);
        if constexpr (ptr_form) {
            const S** pa = ptr_slot((t - (int)blockIdx.x) / (int)gridDim.x);
            const S** pb = pa + P;
            const S** pc = pb + P;
            if (!skip_ab) {
                stage_ptrs<S, Cf::SA, Cf::SA_P, Cf::RA, Cf::NT>(st, pa, g.lda, cnt);
                stage_ptrs<S, Cf::SB, Cf::SB_P, Cf::RB, Cf::NT>(st + offB, pb, g.ldb, cnt);
            }
            if (!beta_zero)
                stage_ptrs<S, Cf::SC, Cf::SC_P, Cf::M, Cf::NT>(st + offC, pc, g.ldc, cnt);
            return;
        }
        // flat operands move by bulk copies on the stage's barrier where
        // they pay (stage_flat); strided ones element by element (cp.async)
        uint64_t* bar = &s_bar[s];
        unsigned bytes = 0;
        if (!skip_ab) {
            if (!shA) {
                if (fa) bytes += stage_flat<S, Cf::SA, Cf::SA_P, Cf::RA, Cf::NT, bulkA>(st, g.A_, p0, cnt, bar);
                else stage_operand<S, Cf::SA, Cf::SA_P, Cf::RA, Cf::NT>(st, g.A_, g.lda2, g.lda, p0, cnt, false);
            }
            if (!shB) {
                if (fb) bytes += stage_flat<S, Cf::SB, Cf::SB_P, Cf::RB, Cf::NT, bulkB>(st + offB, g.B_, p0, cnt, bar);
                else stage_operand<S, Cf::SB, Cf::SB_P, Cf::RB, Cf::NT>(st + offB, g.B_, g.ldb2, g.ldb, p0, cnt,
                                                                        false);
            }
        }
        if (!beta_zero) {
            if (fc) bytes += stage_flat<S, Cf::SC, Cf::SC_P, Cf::M, Cf::NT, bulkC>(st + offC, g.C_, p0, cnt, bar);
            else stage_operand<S, Cf::SC, Cf::SC_P, Cf::M, Cf::NT>(st + offC, g.C_, g.ldc2, g.ldc, p0, cnt, false);
        }
        if constexpr (kBulk) {
            if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, bytes);
        }
    };

    // the shared matrices join the first commit group
    if (!skip_ab && (int)blockIdx.x < ntiles) {
        if (shA) stage_operand<S, Cf::SA, Cf::SA_P, Cf::RA, Cf::NT>(sShA, g.A_, 0, g.lda, 0, 1, false);
        if (shB) stage_operand<S, Cf::SB, Cf::SB_P, Cf::RB, Cf::NT>(sShB, g.B_, 0, g.ldb, 0, 1, false);
    }

    if constexpr (ptr_form) {
        for (int j = 0; j < stages; ++j) fetch_ptrs(j, false);
        __syncthreads();
    }
    for (int s = 0; s < stages - 1; ++s) {
        const int t = blockIdx.x + s * gridDim.x;
        if (t < ntiles) issue(t, s);
        if constexpr (ptr_form) fetch_ptrs(s + stages, true);
        cp_async_commit();
    }

    const int tid = threadIdx.x;
    const int ql = tid / Cf::TPM;
    const int u = tid - ql * Cf::TPM;
    const int ti = u % Cf::TI, tj = u / Cf::TI;
    const bool active = ql < Cf::MPR;

    int it = 0;
    bool failed = false;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int tn = t + (stages - 1) * gridDim.x;
        if (tn < ntiles) issue(tn, (it + stages - 1) % stages);
        if constexpr (ptr_form) fetch_ptrs(it + 2 * stages - 1, true);
        cp_async_commit();
        cp_async_wait_dyn(stages - 1);
        if constexpr (kBulk) {
            // thread 0 waits for the stage's bulk copies (the block barrier
            // then orders its observation before every thread's reads) and
            // for its previous bulk stores to have read the output tile
            if (threadIdx.x == 0) {
                if (!mbar_wait(&s_bar[it % stages], (it / stages) & 1)) {
                    s_fail = 1;
                    if (g.err) atomicExch(g.err, (int)SBGEMM_ERR_TIMEOUT);
                }
                bulk_wait_read();
            }
            __syncthreads();
            if (s_fail) {
                failed = true;
                break;
            }
        } else {
            __syncthreads();
        }

        const S* st = stage_base + (it % stages) * stage_elems;
        const long long p0 = (long long)t * P;
        const int cnt = (int)min((long long)P, batch - p0);
        S* gC = g.C_ + p0 * Cf::SC;
        if (active) {
            const S* sA = shA ? sShA : st;
            const S* sB = shB ? sShB : st + offB;
            for (int q = ql; q < cnt; q += Cf::MPR)
                compute_block<Cf>(sA, sB, st + offC, sOut, gC, direct, q, ti, tj, alpha, beta,
                                  beta_zero, alpha_one, skip_ab, g.conja, g.conjb, sh);
        }
        // every thread is done reading this stage before it is refilled
        // (and has ordered its output-tile writes before the bulk stores)
        if constexpr (bulkC) {
            if (!direct && fc) fence_proxy_async();
        }
        __syncthreads();
        if constexpr (ptr_form) {
            store_ptrs<S, Cf::SC, Cf::SC_P, Cf::M, Cf::NT>(
                const_cast<S* const*>(ptr_slot(it) + 2 * P), sOut, g.ldc, cnt);
        } else if (!direct) {
            if (fc) store_flat<S, Cf::SC, Cf::SC_P, Cf::M, Cf::NT, bulkC>(g.C_, sOut, p0, cnt);
            else store_operand<S, Cf::SC, Cf::SC_P, Cf::M, Cf::NT>(g.C_, sOut, g.ldc2, g.ldc, p0, cnt, false);
        }
    }
    if constexpr (kBulk) {
        if (failed) {
            // let the copies already issued into this block's stages land (bounded)
            for (int k = 0; k < stages; ++k) {
                const long long tk = blockIdx.x + (long long)(it + k) * gridDim.x;
                if (tk < ntiles) mbar_wait(&s_bar[(it + k) % stages], ((it + k) / stages) & 1);
            }
        }
    }
    cp_async_wait_dyn(0);
    if constexpr (kBulk) bulk_wait_all();
}

// ------------------------------------------------------------ host launcher

inline int gcd_i(int a, int b) { while (b) { int t = a % b; a = b; b = t; } return a; }
inline int lcm_i(int a, int b) { return a / gcd_i(a, b) * b; }

// Tile geometry.  P (pairs per tile) is a whole number of compute rounds
// (MPR pairs each) near the byte target, a multiple of every operand's
// 16-byte quantum (so every tile of a flat stream starts 16-byte aligned),
// within the shared-memory budget, and small enough that the grid has work
// for every SM when the batch is short.
struct Geom { int P; size_t smem; };

template <class Cf>
inline Geom tile_geom(long long batch, const LaunchOpts& o, bool has_cold, bool direct,
                      int shared = 0, bool ptr_form = false) {
    using S = typename Cf::S;
    constexpr int ES = Cf::ES;
    const bool shA = shared & 1, shB = shared & 2;
    int quantum = 1;
    if (!shA) quantum = lcm_i(quantum, 16 / gcd_i(Cf::SA * ES, 16));
    if (!shB) quantum = lcm_i(quantum, 16 / gcd_i(Cf::SB * ES, 16));
    quantum = lcm_i(quantum, 16 / gcd_i(Cf::SC * ES, 16));
    const size_t in_bpp =
        (size_t)((shA ? 0 : Cf::SA_P) + (shB ? 0 : Cf::SB_P) + (has_cold ? Cf::SC_P : 0)) * ES;
    const size_t out_bpp = direct ? 0 : (size_t)Cf::SC_P * ES;
    // the pointer-array form keeps three pointers per pair in each of
    // 2*stages + 1 ring slots
    const size_t per_pair = in_bpp * o.stages + out_bpp +
                            (ptr_form ? 3 * sizeof(void*) * (2 * o.stages + 1) : 0);
    const size_t fixed = (size_t)((shA ? shared_slot_elems<S>(Cf::SA_P) : 0) +
                                  (shB ? shared_slot_elems<S>(Cf::SB_P) : 0)) * ES;
    const size_t cap = 200 * 1024 - fixed;
    auto round_up = [&](int p) { return (p + quantum - 1) / quantum * quantum; };
    // R whole compute rounds, rounded down to the quantum (a few idle threads
    // in the last round) rather than up (a nearly empty extra round)
    auto rounds_to_P = [&](int R) {
        const int want = Cf::MPR * R;
        const int down = want / quantum * quantum;
        return down >= quantum ? down : round_up(want);
    };
    // (with both A and B shared and beta == 0 nothing is staged per pair)
    const size_t in_eff = in_bpp ? in_bpp : (size_t)Cf::SC_P * ES;
    int R = (int)(o.tile_bytes / ((size_t)Cf::MPR * in_eff));
    if (R < 1) R = 1;
    int P = rounds_to_P(R);
    while (P > quantum && (size_t)P * per_pair > cap) {
        if (R > 1) { --R; P = rounds_to_P(R); }
        else P = (P - 1) / quantum * quantum;
    }
    if (P < quantum) P = quantum;
    // fill the GPU: at least two tiles per resident block when possible
    int per_sm = (int)((227 * 1024) / ((size_t)P * per_pair + fixed + 1024));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 2048 / Cf::NT) per_sm = 2048 / Cf::NT;
    if (o.ctas_per_sm > 0 && per_sm > o.ctas_per_sm) per_sm = o.ctas_per_sm;
    const long long want_tiles = 2LL * num_sms() * per_sm;
    if ((batch + P - 1) / P < want_tiles) {
        long long p2 = (batch + want_tiles - 1) / want_tiles;
        int pn = round_up((int)(p2 < 1 ? 1 : p2));
        if (pn < P) P = pn;
    }
    return Geom{P, (size_t)P * per_pair + fixed};
}

template <class Cf, bool PF>
sbgemm_status launch_pipe_k(const Req& r, const LaunchOpts& o) {
    using Ty = typename Cf::Ty;
    Args<Ty> a;
    fill_args(a, r);
    const bool has_cold = !a.beta_zero;
    // flat-stream test per operand: minimal leading dimensions and 16-byte alignment
    auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    int flat = 0;
    if (!r.Cp) {
        if (r.lda == Cf::RA && r.lda2 == (long long)Cf::SA && aligned(r.A)) flat |= 1;
        if (r.ldb == Cf::RB && r.ldb2 == (long long)Cf::SB && aligned(r.B)) flat |= 2;
        if (r.ldc == Cf::M && r.ldc2 == (long long)Cf::SC && aligned(r.C)) flat |= 4;
    }
    a.flat = flat;
    const bool direct = Cf::VS > 0 && (flat & 4);
    const Geom gm = tile_geom<Cf>(r.batch, o, has_cold, direct, a.shared, PF);
    a.P = gm.P;
    a.stages = o.stages;
    auto kern = pipe_kernel<Cf, PF>;
    // per instantiation and device
    static DeviceFlags attr_set;
    static thread_local OccCache occ;
    cudaError_t ae = ensure_smem_limit(kern, 220 * 1024, attr_set);
    if (ae != cudaSuccess) return (sbgemm_status)ae;
    int per_sm = 0;
    ae = blocks_per_sm(kern, Cf::NT, gm.smem, occ, &per_sm);
    if (ae != cudaSuccess) return (sbgemm_status)ae;
    if (per_sm < 1) return SBGEMM_ERR_NOT_SUPPORTED;
    if (o.ctas_per_sm > 0 && per_sm > o.ctas_per_sm) per_sm = o.ctas_per_sm;
    const long long ntiles = ((long long)r.batch + gm.P - 1) / gm.P;
    long long grid = (long long)num_sms() * per_sm;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(Cf::NT);
    lc.dynamicSmemBytes = gm.smem;
    lc.stream = r.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    cudaError_t le = cudaLaunchKernelEx(&lc, kern, a);
    if (le != cudaSuccess) return (sbgemm_status)le;
    return (sbgemm_status)cudaGetLastError();
}

template <class Cf>
sbgemm_status launch_pipe(const Req& r, const LaunchOpts& o) {
    return r.Cp ? launch_pipe_k<Cf, true>(r, o) : launch_pipe_k<Cf, false>(r, o);
}

// ------------------------------------------------------------ generic kernel

// Any (m, n, k) <= 16 and any op: one thread per entry of C (the mapping of
// the paper's first method, Section 6), run-time sizes, element gathers.
template <class Ty>
__global__ void __launch_bounds__(256)
generic_kernel(Args<Ty> g, int m, int n, int k, int ta, int tb)
{
    using S = typename Ty::S;
    using A = typename Ty::A;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A alpha = g.alpha, beta = g.beta;
    bool beta_zero = g.beta_zero != 0, alpha_zero = g.alpha_zero != 0;
    if (g.alpha_ptr) { alpha = *g.alpha_ptr; alpha_zero = is_zero(alpha); }
    if (g.beta_ptr)  { beta = *g.beta_ptr;   beta_zero = is_zero(beta); }
    const int P = g.P;
    const int sa = m * k, sb = k * n, sc = m * n;
    const int ra = ta ? k : m, rb = tb ? n : k;
    S* sA = reinterpret_cast<S*>(smem_raw);
    S* sB = sA + P * sa;
    S* sC = sB + P * sb;
    const long long batch = g.batch;
    const int ntiles = (int)((batch + P - 1) / P);
    const int tid = threadIdx.x;
    const int mpr = blockDim.x / sc;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long p0 = (long long)t * P;
        const int cnt = (int)min((long long)P, batch - p0);
        if (!alpha_zero) {
            for (int e = tid; e < cnt * sa; e += blockDim.x) {
                const int q = e / sa, r = e - q * sa;
                sA[e] = mat_of(g.A_, g.Ap, g.lda2, p0 + q)[r % ra + (long long)(r / ra) * g.lda];
            }
            for (int e = tid; e < cnt * sb; e += blockDim.x) {
                const int q = e / sb, r = e - q * sb;
                sB[e] = mat_of(g.B_, g.Bp, g.ldb2, p0 + q)[r % rb + (long long)(r / rb) * g.ldb];
            }
        }
        if (!beta_zero) {
            for (int e = tid; e < cnt * sc; e += blockDim.x) {
                const int q = e / sc, r = e - q * sc;
                sC[e] = mat_of(g.C_, g.Cp, g.ldc2, p0 + q)[r % m + (long long)(r / m) * g.ldc];
            }
        }
        __syncthreads();
        const int ql = tid / sc, r = tid - ql * sc;
        const int i = r % m, j = r / m;
        if (ql < mpr) {
            for (int q = ql; q < cnt; q += mpr) {
                A acc = zero_a<A>();
                if (!alpha_zero) {
                    const S* a = sA + q * sa;
                    const S* b = sB + q * sb;
                    for (int l = 0; l < k; ++l) {
                        A av = conj_s(to_a(a[ta ? l + k * i : i + m * l]), g.conja);
                        A bv = conj_s(to_a(b[tb ? j + n * l : l + k * j]), g.conjb);
                        mac(acc, av, bv);
                    }
                }
                A v = alpha_zero ? zero_a<A>() : mul(alpha, acc);
                if (!beta_zero) v = axpy(beta, to_a(sC[q * sc + i + m * j]), v);
                mat_of(g.C_, g.Cp, g.ldc2, p0 + q)[i + (long long)j * g.ldc] = to_s<Ty>(v);
            }
        }
        __syncthreads();
    }
}

template <class Ty>
sbgemm_status launch_generic(const Req& r) {
    Args<Ty> a;
    fill_args(a, r);
    using S = typename Ty::S;
    const int sc = r.m * r.n;
    const int mpr = 256 / sc;
    const size_t per = sizeof(S) * (size_t)(r.m * r.k + r.k * r.n + sc);
    // pairs per tile: up to four compute rounds, within 40 KB of shared memory
    int P = mpr * 4;
    if ((size_t)P * per > 40 * 1024) P = (int)((40 * 1024) / per);
    if (P < 1) P = 1;
    a.P = P;
    a.stages = 1;
    a.flat = 0;
    const size_t smem = per * P;
    const long long ntiles = ((long long)r.batch + P - 1) / P;
    long long grid = (long long)num_sms() * 8;
    if (grid > ntiles) grid = ntiles;
    generic_kernel<Ty><<<(unsigned)grid, 256, smem, r.stream>>>(a, r.m, r.n, r.k, r.ta, r.tb);
    return (sbgemm_status)cudaGetLastError();
}

// C = beta * C over the m x n blocks (alpha == 0 or k == 0); C is not read
// when beta == 0.
template <class Ty>
__global__ void scale_kernel(Args<Ty> g, int m, int n)
{
    using A = typename Ty::A;
    A beta = g.beta_ptr ? *g.beta_ptr : g.beta;
    const bool bz = is_zero(beta);
    const long long total = (long long)g.batch * m * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long p = e / (m * n);
        const int r = (int)(e - p * m * n);
        const int i = r % m, j = r / m;
        typename Ty::S* c = mat_of(g.C_, g.Cp, g.ldc2, p) + i + (long long)j * g.ldc;
        *c = to_s<Ty>(bz ? zero_a<A>() : mul(beta, to_a(*c)));
    }
}

template <class Ty>
sbgemm_status launch_scale(const Req& r) {
    Args<Ty> a;
    fill_args(a, r);
    const long long total = (long long)r.batch * r.m * r.n;
    long long grid = (total + 255) / 256;
    if (grid > (long long)num_sms() * 16) grid = (long long)num_sms() * 16;
    if (grid < 1) grid = 1;
    scale_kernel<Ty><<<(unsigned)grid, 256, 0, r.stream>>>(a, r.m, r.n);
    return (sbgemm_status)cudaGetLastError();
}

// ------------------------------------------------------------ shape dispatch

template <class Ty, int M, int N, int K, bool TA, bool TB>
sbgemm_status launch_shape_op(const Req& r, const LaunchOpts& o) {
    constexpr TileEntry te = tile_for(Ty::code, M, N, K, TA ? 1 : 0, TB ? 1 : 0);
    using Cf = Cfg<Ty, M, N, K, TA, TB, te.tm, te.tn, te.si != 0, te.sj != 0, te.nt>;
    return launch_pipe<Cf>(r, o);
}

template <class Ty, int M, int N, int K>
sbgemm_status launch_shape(const Req& r) {
    if (r.variant >= kNumPipeVariants) return launch_generic<Ty>(r);
    const LaunchOpts o = pipe_variant(r.variant, Ty::code);
    if (!r.ta && !r.tb) return launch_shape_op<Ty, M, N, K, false, false>(r, o);
    if (r.ta && !r.tb)  return launch_shape_op<Ty, M, N, K, true, false>(r, o);
    if (!r.ta && r.tb)  return launch_shape_op<Ty, M, N, K, false, true>(r, o);
    return launch_shape_op<Ty, M, N, K, true, true>(r, o);
}

// Per-type entry used by the C ABI; defined in one translation unit per type.
sbgemm_status run_S(const Req& r);
sbgemm_status run_D(const Req& r);
sbgemm_status run_C(const Req& r);
sbgemm_status run_Z(const Req& r);
sbgemm_status run_H(const Req& r);
sbgemm_status run_B(const Req& r);
bool has_specialized(int type, int m, int n, int k);

}  // namespace sbg
