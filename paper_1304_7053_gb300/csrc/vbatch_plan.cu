// Host side of the variable-size path: bucketing into a tile list (the
// plan) and the C entry points.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "selection.h"
#include "vbatch.cuh"

struct sbgemm_vplan_s {
    int type;
    int device;
    int n_items;
    int n_buckets;
    void* dmem;
    size_t bytes;
    sbg::VItem* items;
    sbg::VRec* recs;
    int* counter;
    long long n_tc;        // problems on the fp64 / complex128 tensor-core kernel
    sbg::VRec* tc_recs;    // their records (pad = m | n << 8 | k << 16)
};

namespace sbg {

#define SBG_VDECL(T)                                                                            \
    void vkinds_##T(VKindInfo* out);                                                            \
    sbgemm_status vrun_##T(const VItem*, int, const VRec*, int*, const void*, const void*,     \
                           void*, const void*, const void*, int, int, int, cudaStream_t);
SBG_VDECL(S) SBG_VDECL(D) SBG_VDECL(C) SBG_VDECL(Z) SBG_VDECL(H) SBG_VDECL(B)
#undef SBG_VDECL
bool has_specialized(int type, int m, int n, int k);
sbgemm_status run_ozaki_records(int type, const void* recs, long long count, const void* A,
                                const void* B, void* C, const void* alpha, const void* beta,
                                int scalar_mode, int beta_zero, cudaStream_t stream);

namespace {

size_t elem_bytes(int type) {
    switch (type) {
    case SBGEMM_TYPE_S: return 4;
    case SBGEMM_TYPE_D: return 8;
    case SBGEMM_TYPE_C: return 8;
    case SBGEMM_TYPE_Z: return 16;
    default: return 2;
    }
}

bool kinds_of(int type, VKindInfo* k) {
    switch (type) {
    case SBGEMM_TYPE_S: vkinds_S(k); return true;
    case SBGEMM_TYPE_D: vkinds_D(k); return true;
    case SBGEMM_TYPE_C: vkinds_C(k); return true;
    case SBGEMM_TYPE_Z: vkinds_Z(k); return true;
    case SBGEMM_TYPE_H: vkinds_H(k); return true;
    case SBGEMM_TYPE_B: vkinds_B(k); return true;
    default: return false;
    }
}

// Real and complex fp64 problems whose class the selector sends to the
// tensor-core kernel (large sizes; the table, the cost model or the
// built-in rule as for a uniform batch of the bucket's size, beta taken
// as nonzero) run on it, from a record list, instead of in the tiles.
bool takes_tensor_cores(int type, int m, int n, int k, int ta, int tb, int count) {
    if (type != SBGEMM_TYPE_D && type != SBGEMM_TYPE_Z) return false;
    const int v = select_variant(type, m, n, k, ta, tb, 0, size_class(count));
    return has_specialized(0, m, n, k) ? v == kMmaVariant : v == 1;
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

// problems per bucketing window of a plan (sbgemm_vbatch_config)
int g_window = kVDefaultWindow;

}  // namespace sbg

extern "C" {

sbgemm_status sbgemm_vbatch_config(int window) {
    if (window < 0) return SBGEMM_ERR_INVALID_VALUE;
    sbg::g_window = window == 0 ? sbg::kVDefaultWindow : window;
    return SBGEMM_SUCCESS;
}

sbgemm_status sbgemm_vbatch_plan_create(sbgemm_vplan* plan, int type,
                                        const sbgemm_vproblem* problems, int count) {
    using namespace sbg;
    if (!plan) return SBGEMM_ERR_NULL_POINTER;
    *plan = nullptr;
    VKindInfo kinfo[16];
    if (!kinds_of(type, kinfo)) return SBGEMM_ERR_INVALID_VALUE;
    if (count < 0) return SBGEMM_ERR_INVALID_SIZE;
    if (count > 0 && !problems) return SBGEMM_ERR_NULL_POINTER;
    const size_t es = elem_bytes(type);

    // validate every problem first (nothing is allocated on error)
    for (int q = 0; q < count; ++q) {
        const sbgemm_vproblem& p = problems[q];
        if (p.m < 0 || p.n < 0 || p.k < 0 || p.m > 16 || p.n > 16 || p.k > 16)
            return SBGEMM_ERR_INVALID_SIZE;
        const int opa = p.flags & 3, opb = (p.flags >> 2) & 3;
        if (opa == 3 || opb == 3) return SBGEMM_ERR_INVALID_TRANS;
        if (p.a < 0 || p.b < 0 || p.c < 0) return SBGEMM_ERR_INVALID_VALUE;
    }

    // Bucket by (m, n, k, ta, tb) within windows of consecutive problems and
    // queue the tiles window by window: problems that are neighbours in the
    // arenas (and may share memory sectors) are then processed close in
    // time, while their data is still in L2.  Problems with m == 0 or n == 0
    // do nothing.
    using Key = std::tuple<int, int, int, int, int>;
    const int kWindow = g_window;
    struct Tile { VItem it; double cost; };
    std::vector<Tile> tiles;
    std::vector<VRec> recs, tc_recs;
    recs.reserve(count);
    std::map<Key, int> all_keys;
    for (int w0 = 0; w0 < count; w0 += kWindow) {
        const int w1 = std::min(count, w0 + kWindow);
        std::map<Key, std::vector<int>> buckets;
        for (int q = w0; q < w1; ++q) {
            const sbgemm_vproblem& p = problems[q];
            if (p.m == 0 || p.n == 0) continue;
            const int opa = p.flags & 3, opb = (p.flags >> 2) & 3;
            buckets[Key(p.m, p.n, p.k, opa != 0, opb != 0)].push_back(q);
        }
        std::vector<Tile> wtiles;
        for (auto& kv : buckets) {
            all_keys[kv.first] = 1;
            int m, n, k, ta, tb;
            std::tie(m, n, k, ta, tb) = kv.first;
            const std::vector<int>& ids = kv.second;
            if (takes_tensor_cores(type, m, n, k, ta, tb, (int)ids.size())) {
                for (int q : ids) {
                    const sbgemm_vproblem& p = problems[q];
                    VRec r;
                    r.a = p.a; r.b = p.b; r.c = p.c; r.flags = p.flags & 31;
                    r.pad = m | (n << 8) | (k << 16);
                    tc_recs.push_back(r);
                }
                continue;
            }
            int kind = kVGeneric;
            if (m == n && n == k && !ta && !tb && kinfo[m - 1].mpr > 0) kind = m - 1;
            int T;
            if (kind != kVGeneric) {
                const VKindInfo& ki = kinfo[kind];
                // largest tile whose quantum-rounded slots fit one stage
                T = kVMaxTile;
                while (T > 1 && (size_t)((T + ki.quantum - 1) / ki.quantum * ki.quantum) * ki.bytes_per_pair
                                    > (size_t)vstage_bytes_of(type))
                    --T;
                if (T >= ki.mpr) T = T / ki.mpr * ki.mpr;   // whole compute rounds
            } else {
                const size_t per = es * (size_t)(m * k + k * n + m * n);
                T = (int)std::min<size_t>(kVMaxTile, per ? vstage_bytes_of(type) / per : kVMaxTile);
                if (T < 1) T = 1;
            }
            const int base = (int)recs.size();
            for (int q : ids) {
                const sbgemm_vproblem& p = problems[q];
                VRec r;
                r.a = p.a; r.b = p.b; r.c = p.c; r.flags = p.flags & 31; r.pad = 0;
                recs.push_back(r);
            }
            const double unit = (double)es * (m * k + k * n + 2.0 * m * n) + 64.0;
            for (int f = 0; f < (int)ids.size(); f += T) {
                Tile t;
                t.it.kind = kind;
                t.it.first = base + f;
                t.it.count = std::min(T, (int)ids.size() - f);
                t.it.shape = m | (n << 8) | (k << 16) | (ta << 24) | (tb << 25);
                t.cost = unit * t.it.count;
                wtiles.push_back(t);
            }
        }
        // within a window, the most expensive tiles first
        std::stable_sort(wtiles.begin(), wtiles.end(),
                         [](const Tile& x, const Tile& y) { return x.cost > y.cost; });
        tiles.insert(tiles.end(), wtiles.begin(), wtiles.end());
    }

    sbgemm_vplan pl = new (std::nothrow) sbgemm_vplan_s;
    if (!pl) return SBGEMM_ERR_CAPACITY;
    std::memset(pl, 0, sizeof *pl);
    pl->type = type;
    cudaGetDevice(&pl->device);
    pl->n_items = (int)tiles.size();
    pl->n_buckets = (int)all_keys.size();
    const size_t items_b = sizeof(VItem) * std::max<size_t>(1, tiles.size());
    const size_t recs_b = sizeof(VRec) * std::max<size_t>(1, recs.size());
    const size_t off_recs = (items_b + 255) / 256 * 256;
    const size_t off_ctr = off_recs + (recs_b + 255) / 256 * 256;
    const size_t off_tc = off_ctr + 256;
    const size_t tc_b = sizeof(VRec) * std::max<size_t>(1, tc_recs.size());
    pl->bytes = off_tc + (tc_b + 255) / 256 * 256;
    pl->n_tc = (long long)tc_recs.size();
    cudaError_t e = cudaMalloc(&pl->dmem, pl->bytes);
    if (e != cudaSuccess) { delete pl; return (sbgemm_status)e; }
    char* base = static_cast<char*>(pl->dmem);
    pl->items = reinterpret_cast<VItem*>(base);
    pl->recs = reinterpret_cast<VRec*>(base + off_recs);
    pl->counter = reinterpret_cast<int*>(base + off_ctr);
    pl->tc_recs = reinterpret_cast<VRec*>(base + off_tc);
    std::vector<VItem> hitems(tiles.size());
    for (size_t i = 0; i < tiles.size(); ++i) hitems[i] = tiles[i].it;
    if (!hitems.empty())
        e = cudaMemcpy(pl->items, hitems.data(), sizeof(VItem) * hitems.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !recs.empty())
        e = cudaMemcpy(pl->recs, recs.data(), sizeof(VRec) * recs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !tc_recs.empty())
        e = cudaMemcpy(pl->tc_recs, tc_recs.data(), sizeof(VRec) * tc_recs.size(),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(pl->dmem); delete pl; return (sbgemm_status)e; }
    *plan = pl;
    return SBGEMM_SUCCESS;
}

sbgemm_status sbgemm_vbatch_plan_destroy(sbgemm_vplan plan) {
    if (!plan) return SBGEMM_ERR_INVALID_VALUE;
    cudaError_t e = cudaFree(plan->dmem);
    delete plan;
    return (sbgemm_status)e;
}

sbgemm_status sbgemm_vbatch_plan_info(sbgemm_vplan plan, int* n_tiles, int* n_buckets,
                                      long long* device_bytes) {
    if (!plan) return SBGEMM_ERR_INVALID_VALUE;
    if (n_tiles) *n_tiles = plan->n_items;
    if (n_buckets) *n_buckets = plan->n_buckets;
    if (device_bytes) *device_bytes = (long long)plan->bytes;
    return SBGEMM_SUCCESS;
}

sbgemm_status sbgemm_vbatch_run(sbgemm_vplan plan, const void* alpha, const void* A,
                                const void* B, const void* beta, void* C,
                                int scalar_mode, void* stream) {
    using namespace sbg;
    if (!plan) return SBGEMM_ERR_INVALID_VALUE;
    if (scalar_mode != SBGEMM_SCALARS_HOST && scalar_mode != SBGEMM_SCALARS_DEVICE)
        return SBGEMM_ERR_INVALID_VALUE;
    if (plan->n_items == 0 && plan->n_tc == 0) return SBGEMM_SUCCESS;
    if (!alpha || !beta || !C) return SBGEMM_ERR_NULL_POINTER;
    int bz = 0, az = 0;
    if (scalar_mode == SBGEMM_SCALARS_HOST) {
        bz = host_zero(plan->type, beta);
        az = host_zero(plan->type, alpha);
    }
    if (!az && (!A || !B)) return SBGEMM_ERR_NULL_POINTER;
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->n_tc > 0) {
        const sbgemm_status st = run_ozaki_records(plan->type, plan->tc_recs, plan->n_tc, A, B, C,
                                                   alpha, beta, scalar_mode, bz, s);
        if (st != SBGEMM_SUCCESS) return st;
    }
    if (plan->n_items == 0) return SBGEMM_SUCCESS;
#define SBG_VRUN(T, CODE)                                                                      \
    case CODE:                                                                                 \
        return vrun_##T(plan->items, plan->n_items, plan->recs, plan->counter, A, B, C, alpha, \
                        beta, scalar_mode, bz, az, s);
    switch (plan->type) {
        SBG_VRUN(S, SBGEMM_TYPE_S) SBG_VRUN(D, SBGEMM_TYPE_D) SBG_VRUN(C, SBGEMM_TYPE_C)
        SBG_VRUN(Z, SBGEMM_TYPE_Z) SBG_VRUN(H, SBGEMM_TYPE_H) SBG_VRUN(B, SBGEMM_TYPE_B)
    default: return SBGEMM_ERR_INVALID_VALUE;
    }
#undef SBG_VRUN
}

}  // extern "C"
