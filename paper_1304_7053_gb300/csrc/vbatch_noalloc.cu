// Variable-size batch run that allocates nothing.
//
// Some callers cannot allocate device memory once they are running: a
// plug-in inside a host application that owns the device memory, or a
// latency-critical loop that must keep a fixed footprint and cannot afford
// the implicit device-wide synchronisation cudaMalloc may cause.  The plan
// path needs device memory for its tile list and records; this entry point
// keeps them, plus the bucketing counters and the work-queue counter, in one
// file-scope static device array of fixed size, and builds them on the
// device from a device-resident problem array.  The GEMM kernel itself is the
// plan path's persistent kernel, unchanged.
#include <mutex>

#include "vbatch.cuh"

namespace sbg {

#define SBG_VDECL(T)                                                                            \
    void vkinds_##T(VKindInfo* out);                                                            \
    sbgemm_status vrun_##T(const VItem*, int, const VRec*, int*, const void*, const void*,     \
                           void*, const void*, const void*, int, int, int, cudaStream_t);
SBG_VDECL(S) SBG_VDECL(D) SBG_VDECL(C) SBG_VDECL(Z) SBG_VDECL(H) SBG_VDECL(B)
#undef SBG_VDECL

namespace {

constexpr int kMaxProblems = SBGEMM_NOALLOC_MAX_PROBLEMS;
constexpr int kKeys = 17 * 17 * 17 * 4;            // (m, n, k, opA transposed, opB transposed)
constexpr size_t kCountersBytes = 4 * (size_t)kKeys * sizeof(int) + 256;
constexpr size_t kRecsOff = (kCountersBytes + 255) / 256 * 256;
constexpr size_t kItemsOff = kRecsOff + (size_t)kMaxProblems * sizeof(VRec);
constexpr size_t kScratchBytes = kItemsOff + (size_t)kMaxProblems * sizeof(VItem);

// hist | cursor | recoff | itemoff (kKeys ints each) | misc (64 ints) | records | tiles
// misc[0] tile count, misc[1] work-queue counter, misc[2] invalid problems
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct TileRule {
    int T[16];     // tile size of square N/N kind s+1, 0 when the kind is not specialised
    int es;        // storage element bytes
    int stage;     // bytes of one pipeline stage of the type
};

__device__ __forceinline__ int key_of(const sbgemm_vproblem& p, bool* valid) {
    const int opa = p.flags & 3, opb = (p.flags >> 2) & 3;
    *valid = p.m >= 0 && p.n >= 0 && p.k >= 0 && p.m <= 16 && p.n <= 16 && p.k <= 16 &&
             opa != 3 && opb != 3 && p.a >= 0 && p.b >= 0 && p.c >= 0;
    return ((p.m * 17 + p.n) * 17 + p.k) * 4 + (opa != 0) * 2 + (opb != 0);
}

__device__ __forceinline__ void key_shape(int key, int* m, int* n, int* k, int* ta, int* tb) {
    *tb = key & 1;
    *ta = (key >> 1) & 1;
    int r = key >> 2;
    *k = r % 17; r /= 17;
    *n = r % 17;
    *m = r / 17;
}

__device__ __forceinline__ int tile_of(int key, const TileRule& rule, int* kind) {
    int m, n, k, ta, tb;
    key_shape(key, &m, &n, &k, &ta, &tb);
    if (m == n && n == k && m >= 1 && !ta && !tb && rule.T[m - 1] > 0) {
        *kind = m - 1;
        return rule.T[m - 1];
    }
    *kind = kVGeneric;
    const int per = rule.es * (m * k + k * n + m * n);
    int T = per > 0 ? rule.stage / per : kVMaxTile;
    if (T > kVMaxTile) T = kVMaxTile;
    return T < 1 ? 1 : T;
}

__global__ void na_count(const sbgemm_vproblem* __restrict__ p, int count, int* hist, int* misc) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    const sbgemm_vproblem pq = p[q];
    bool valid;
    const int key = key_of(pq, &valid);
    if (!valid) { atomicAdd(&misc[2], 1); return; }
    if (pq.m == 0 || pq.n == 0) return;
    atomicAdd(&hist[key], 1);
}

// One block: exclusive scans of problem and tile counts over the keys, taken
// in descending key order so the largest shapes come first in the queue.
__global__ void __launch_bounds__(1024) na_scan(const int* __restrict__ hist, int* recoff,
                                                int* itemoff, int* misc, TileRule rule) {
    __shared__ int s_r[1024], s_t[1024];
    constexpr int PER = (kKeys + 1023) / 1024;
    const int tid = threadIdx.x;
    int r = 0, t = 0;
    for (int e = 0; e < PER; ++e) {
        const int o = tid * PER + e;              // position in processing order
        if (o >= kKeys) break;
        const int key = kKeys - 1 - o;
        const int h = hist[key];
        int kind;
        const int T = tile_of(key, rule, &kind);
        r += h;
        t += (h + T - 1) / T;
    }
    s_r[tid] = r;
    s_t[tid] = t;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {          // inclusive scan (Hillis-Steele)
        const int ar = tid >= d ? s_r[tid - d] : 0;
        const int at = tid >= d ? s_t[tid - d] : 0;
        __syncthreads();
        s_r[tid] += ar;
        s_t[tid] += at;
        __syncthreads();
    }
    int rb = s_r[tid] - r, tb = s_t[tid] - t;     // exclusive
    for (int e = 0; e < PER; ++e) {
        const int o = tid * PER + e;
        if (o >= kKeys) break;
        const int key = kKeys - 1 - o;
        const int h = hist[key];
        int kind;
        const int T = tile_of(key, rule, &kind);
        recoff[key] = rb;
        itemoff[key] = tb;
        rb += h;
        tb += (h + T - 1) / T;
    }
    if (tid == 1023) misc[0] = s_t[1023];
}

__global__ void na_scatter(const sbgemm_vproblem* __restrict__ p, int count,
                           const int* __restrict__ recoff, int* cursor, VRec* recs) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    const sbgemm_vproblem pq = p[q];
    bool valid;
    const int key = key_of(pq, &valid);
    if (!valid || pq.m == 0 || pq.n == 0) return;
    const int pos = recoff[key] + atomicAdd(&cursor[key], 1);
    VRec r;
    r.a = pq.a; r.b = pq.b; r.c = pq.c; r.flags = pq.flags & 31; r.pad = 0;
    recs[pos] = r;
}

__global__ void na_items(const int* __restrict__ hist, const int* __restrict__ recoff,
                         const int* __restrict__ itemoff, VItem* items, TileRule rule) {
    const int key = blockIdx.x * blockDim.x + threadIdx.x;
    if (key >= kKeys) return;
    const int h = hist[key];
    if (h == 0) return;
    int kind;
    const int T = tile_of(key, rule, &kind);
    int m, n, k, ta, tb;
    key_shape(key, &m, &n, &k, &ta, &tb);
    for (int t = 0, f = 0; f < h; ++t, f += T) {
        VItem it;
        it.kind = kind;
        it.first = recoff[key] + f;
        it.count = (h - f) < T ? (h - f) : T;
        it.shape = m | (n << 8) | (k << 16) | (ta << 24) | (tb << 25);
        items[itemoff[key] + t] = it;
    }
}

// Device address of the scratch array, looked up once per device (the
// array's name is only a host-side stand-in in host code).
std::mutex g_mu;
unsigned char* g_ptr[64] = {nullptr};

sbgemm_status scratch_ptr(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (sbgemm_status)e;
    if (dev < 0 || dev >= 64) return SBGEMM_ERR_NOT_SUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return (sbgemm_status)e;
        g_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_ptr[dev];
    return SBGEMM_SUCCESS;
}

bool kinds_of(int type, VKindInfo* k, int* es) {
    switch (type) {
    case SBGEMM_TYPE_S: vkinds_S(k); *es = 4; return true;
    case SBGEMM_TYPE_D: vkinds_D(k); *es = 8; return true;
    case SBGEMM_TYPE_C: vkinds_C(k); *es = 8; return true;
    case SBGEMM_TYPE_Z: vkinds_Z(k); *es = 16; return true;
    case SBGEMM_TYPE_H: vkinds_H(k); *es = 2; return true;
    case SBGEMM_TYPE_B: vkinds_B(k); *es = 2; return true;
    default: return false;
    }
}

bool host_zero(int type, const void* p) {
    switch (type) {
    case SBGEMM_TYPE_D: return *static_cast<const double*>(p) == 0.0;
    case SBGEMM_TYPE_C: { const float* f = static_cast<const float*>(p); return f[0] == 0.f && f[1] == 0.f; }
    case SBGEMM_TYPE_Z: { const double* d = static_cast<const double*>(p); return d[0] == 0.0 && d[1] == 0.0; }
    default: return *static_cast<const float*>(p) == 0.f;
    }
}

}  // namespace
}  // namespace sbg

extern "C" sbgemm_status sbgemm_vbatch_run_noalloc(int type, const sbgemm_vproblem* problems,
                                                   int count, const void* alpha, const void* A,
                                                   const void* B, const void* beta, void* C,
                                                   int scalar_mode, void* stream) {
    using namespace sbg;
    VKindInfo kinfo[16];
    int es = 0;
    if (!kinds_of(type, kinfo, &es)) return SBGEMM_ERR_INVALID_VALUE;
    if (count < 0) return SBGEMM_ERR_INVALID_SIZE;
    if (count > kMaxProblems) return SBGEMM_ERR_CAPACITY;
    if (scalar_mode != SBGEMM_SCALARS_HOST && scalar_mode != SBGEMM_SCALARS_DEVICE)
        return SBGEMM_ERR_INVALID_VALUE;
    if (count == 0) return SBGEMM_SUCCESS;
    if (!problems || !alpha || !beta || !C) return SBGEMM_ERR_NULL_POINTER;
    int bz = 0, az = 0;
    if (scalar_mode == SBGEMM_SCALARS_HOST) {
        bz = host_zero(type, beta);
        az = host_zero(type, alpha);
    }
    if (!az && (!A || !B)) return SBGEMM_ERR_NULL_POINTER;

    // tile sizes: the plan's rule (largest whole number of compute rounds
    // whose quantum-rounded slots fit one stage)
    TileRule rule;
    rule.es = es;
    rule.stage = vstage_bytes_of(type);
    for (int s = 0; s < 16; ++s) {
        const VKindInfo& ki = kinfo[s];
        if (ki.mpr <= 0) { rule.T[s] = 0; continue; }
        int T = kVMaxTile;
        while (T > 1 && (size_t)((T + ki.quantum - 1) / ki.quantum * ki.quantum) * ki.bytes_per_pair
                            > (size_t)rule.stage)
            --T;
        if (T >= ki.mpr) T = T / ki.mpr * ki.mpr;
        rule.T[s] = T;
    }

    unsigned char* base = nullptr;
    sbgemm_status st = scratch_ptr(&base);
    if (st != SBGEMM_SUCCESS) return st;
    int* hist = reinterpret_cast<int*>(base);
    int* cursor = hist + kKeys;
    int* recoff = cursor + kKeys;
    int* itemoff = recoff + kKeys;
    int* misc = itemoff + kKeys;
    VRec* recs = reinterpret_cast<VRec*>(base + kRecsOff);
    VItem* items = reinterpret_cast<VItem*>(base + kItemsOff);
    cudaStream_t s = (cudaStream_t)stream;

    // the array keeps the previous call's contents: clear the counters
    cudaError_t e = cudaMemsetAsync(base, 0, kCountersBytes, s);
    if (e != cudaSuccess) return (sbgemm_status)e;
    const unsigned nb = (unsigned)((count + 255) / 256);
    na_count<<<nb, 256, 0, s>>>(problems, count, hist, misc);
    na_scan<<<1, 1024, 0, s>>>(hist, recoff, itemoff, misc, rule);
    na_scatter<<<nb, 256, 0, s>>>(problems, count, recoff, cursor, recs);
    na_items<<<(kKeys + 255) / 256, 256, 0, s>>>(hist, recoff, itemoff, items, rule);
    if ((e = cudaGetLastError()) != cudaSuccess) return (sbgemm_status)e;
    // the tile count decides the launch: read it back
    int h[3] = {0, 0, 0};
    if ((e = cudaMemcpyAsync(h, misc, sizeof h, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return (sbgemm_status)e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return (sbgemm_status)e;
    if (h[2] > 0) return SBGEMM_ERR_INVALID_SIZE;
    if (h[0] == 0) return SBGEMM_SUCCESS;
#define SBG_VRUN(T, CODE)                                                                  \
    case CODE:                                                                             \
        return vrun_##T(items, h[0], recs, misc + 1, A, B, C, alpha, beta, scalar_mode, bz, \
                        az, s);
    switch (type) {
        SBG_VRUN(S, SBGEMM_TYPE_S) SBG_VRUN(D, SBGEMM_TYPE_D) SBG_VRUN(C, SBGEMM_TYPE_C)
        SBG_VRUN(Z, SBGEMM_TYPE_Z) SBG_VRUN(H, SBGEMM_TYPE_H) SBG_VRUN(B, SBGEMM_TYPE_B)
    default: return SBGEMM_ERR_INVALID_VALUE;
    }
#undef SBG_VRUN
}
