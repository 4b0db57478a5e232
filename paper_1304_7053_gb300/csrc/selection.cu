// Variant selection: the selection table, the selector mode, the cost
// model's per-class choices, their files, and the native autotuner loop.
//
// The paper (Section 6) leaves the launch configuration "tunable for minor
// gains" and suggests more specialised kernels; this library has several
// kernel variants per shape and picks one per problem class.  Order of
// consultation under the default mode: a table entry, else the built-in
// default rule; under the model mode a table entry, else the cost model's
// choice, else the default rule.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "sbgemm_launch.cuh"
#include "sbgemm_shapes.h"
#include "selection.h"

namespace sbg {

bool has_specialized(int type, int m, int n, int k);

namespace {

using Key = std::tuple<int, int, int, int, int, int, int, int>;   // type m n k ta tb bz sc

std::mutex g_choice_mu;
std::map<Key, int> g_choice;
std::atomic<int> g_mode{SBGEMM_SELECTOR_TABLE};
thread_local int t_last_variant = -1;

// cost model (host copy of the network; choices evaluated on the GPU)
struct CostModel {
    bool present = false;
    int F = 0, H = 0, V = 0;
    std::vector<float> params;
    double mu = 0.0, sd = 1.0;
    double margin[6] = {0, 0, 0, 0, 0, 0};   // trust margin per storage type
    std::string device;
    bool evaluated = false;        // choices below are current
    int eval_status = 0;           // error of the last evaluation (0: none)
    std::map<Key, int> choice;
};
std::mutex g_model_mu;
CostModel g_model;

std::once_flag g_env_once;
std::atomic<int> g_env_status{0};

// the tensor-core variant: 16-bit storage at m = n = k = 8, 12, 16, and real
// and complex fp64 (digit-split products) on every shape with specialised
// kernels
bool has_mma_variant(int type, int m, int n, int k) {
    if (type == SBGEMM_TYPE_D || type == SBGEMM_TYPE_Z) return has_specialized(0, m, n, k);
    return (type == SBGEMM_TYPE_H || type == SBGEMM_TYPE_B) && m == n && n == k &&
           (m == 8 || m == 12 || m == 16);
}

int lookup_choice(int type, int m, int n, int k, int ta, int tb, int bz, int sc) {
    std::lock_guard<std::mutex> lk(g_choice_mu);
    auto it = g_choice.find(Key(type, m, n, k, ta, tb, bz, sc));
    return it == g_choice.end() ? -1 : it->second;
}

bool valid_entry(int type, int m, int n, int k, int ta, int tb, int bz, int sc, int v) {
    if (type < SBGEMM_TYPE_S || type > SBGEMM_TYPE_B) return false;
    const int nv = variants_for(type, m, n, k);
    return nv > 0 && v >= 0 && v < nv && sc >= 0 && sc <= 7 && (ta == 0 || ta == 1) &&
           (tb == 0 || tb == 1) && (bz == 0 || bz == 1);
}

std::string device_name() {
    int dev = 0;
    cudaDeviceProp p;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    return std::string(p.name);
}

// Features of a class, as the trainer computes them (selector.features):
// m, n, k / 16; (log10 N - 4.5) / 1.5 with log10 N at the middle of the size
// class; storage-type one-hot; transposed flags, conjugation (0: the table
// key does not tell T from C), beta == 0; specialised-shape flag; (mnk)^(1/3)
// / 16.
void class_features(int type, int m, int n, int k, int ta, int tb, int bz, int sc, float* f) {
    for (int i = 0; i < 16; ++i) f[i] = 0.f;
    f[0] = (float)(m / 16.0); f[1] = (float)(n / 16.0); f[2] = (float)(k / 16.0);
    f[3] = (float)((sc + 0.5 - 4.5) / 1.5);
    f[4 + type] = 1.f;
    f[10] = (float)ta; f[11] = (float)tb; f[12] = 0.f; f[13] = (float)bz;
    f[14] = variants_for(type, m, n, k) > 3 ? 1.f : 0.f;
    f[15] = (float)(std::pow((double)(m * n * k), 1.0 / 3.0) / 16.0);
}

// Evaluate the network once for every class that has a choice (the shapes
// with specialised kernels, and every real fp64 shape), on the GPU with this
// library's forward kernel, and keep the chosen variant per class.  Caller holds g_model_mu.
int evaluate_model_locked() {
    CostModel& M = g_model;
    M.choice.clear();
    M.evaluated = false;
    std::vector<Key> keys;
    std::vector<float> X;
    for (int type = 0; type <= SBGEMM_TYPE_B; ++type)
        for (int m = 1; m <= 16; ++m)
            for (int n = 1; n <= 16; ++n)
                for (int k = 1; k <= 16; ++k) {
                    if (variants_for(type, m, n, k) < 2) continue;
                    for (int ta = 0; ta < 2; ++ta)
                        for (int tb = 0; tb < 2; ++tb)
                            for (int bz = 0; bz < 2; ++bz)
                                for (int sc = 0; sc <= 7; ++sc) {
                                    keys.emplace_back(type, m, n, k, ta, tb, bz, sc);
                                    X.resize(X.size() + 16);
                                    class_features(type, m, n, k, ta, tb, bz, sc, &X[X.size() - 16]);
                                }
                }
    // forward in chunks of rows, so the work buffer stays small (about 16 MB)
    // whatever the number of classes
    const int rows = (int)keys.size();
    const int chunk = 16384;
    const size_t np = M.params.size();
    std::vector<float> Y((size_t)rows * M.V);
    float *dp = nullptr, *dx = nullptr, *dy = nullptr, *dw = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&dp, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dx, (size_t)chunk * 16 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dy, (size_t)chunk * M.V * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dw, (size_t)4 * chunk * M.H * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dp, M.params.data(), np * sizeof(float), cudaMemcpyHostToDevice, s);
    int st = e == cudaSuccess ? 0 : (int)e;
    for (int r0 = 0; st == 0 && r0 < rows; r0 += chunk) {
        const int nr = std::min(chunk, rows - r0);
        e = cudaMemcpyAsync(dx, &X[(size_t)r0 * 16], (size_t)nr * 16 * sizeof(float),
                            cudaMemcpyHostToDevice, s);
        st = e == cudaSuccess ? 0 : (int)e;
        if (st == 0) st = sbgemm_mlp_forward(M.F, M.H, M.V, dp, dx, nr, dy, dw, s);
        if (st == 0) {
            e = cudaMemcpyAsync(&Y[(size_t)r0 * M.V], dy, (size_t)nr * M.V * sizeof(float),
                                cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            st = e == cudaSuccess ? 0 : (int)e;
        }
    }
    if (dp) cudaFree(dp);
    if (dx) cudaFree(dx);
    if (dy) cudaFree(dy);
    if (dw) cudaFree(dw);
    if (s) cudaStreamDestroy(s);
    if (st != 0) {
        cudaGetLastError();
        M.eval_status = st;
        return st;
    }
    for (int r = 0; r < rows; ++r) {
        const Key& key = keys[r];
        const int type = std::get<0>(key), m = std::get<1>(key), n = std::get<2>(key),
                  k = std::get<3>(key), sc = std::get<7>(key);
        const int nv = std::min(variants_for(type, m, n, k), M.V);
        const float* y = &Y[(size_t)r * M.V];
        int best = 0;
        for (int v = 1; v < nv; ++v) if (y[v] < y[best]) best = v;
        int dflt = default_variant(type, m, n, k, std::get<6>(key), sc);
        if (dflt >= nv) dflt = 0;
        // predicted times exp(y sd + mu): keep the default unless the best
        // is predicted faster by more than the trust margin
        const double tb_ = std::exp((double)y[best] * M.sd + M.mu);
        const double td_ = std::exp((double)y[dflt] * M.sd + M.mu);
        M.choice[key] = tb_ < td_ * (1.0 - M.margin[type]) ? best : dflt;
    }
    M.evaluated = true;
    M.eval_status = 0;
    return 0;
}

int model_choice(int type, int m, int n, int k, int ta, int tb, int bz, int sc) {
    std::lock_guard<std::mutex> lk(g_model_mu);
    if (!g_model.present) return -1;
    if (!g_model.evaluated) {
        if (g_model.eval_status != 0) return -1;       // failed before: do not retry per call
        if (evaluate_model_locked() != 0) return -1;
    }
    auto it = g_model.choice.find(Key(type, m, n, k, ta, tb, bz, sc));
    return it == g_model.choice.end() ? -1 : it->second;
}

// ---------------------------------------------------------------- files

int read_table_file(const char* path, std::map<Key, int>* out) {
    FILE* f = std::fopen(path, "r");
    if (!f) return SBGEMM_ERR_IO;
    char line[512];
    int st = SBGEMM_SUCCESS, lineno = 0;
    bool header = false;
    while (std::fgets(line, sizeof line, f)) {
        ++lineno;
        if (lineno == 1) {
            int ver = 0;
            if (std::sscanf(line, "sbgemm-table %d", &ver) != 1 || ver != 1) { st = SBGEMM_ERR_IO; break; }
            header = true;
            continue;
        }
        if (line[0] == '#' || line[0] == '\n' || std::strncmp(line, "device ", 7) == 0) continue;
        int t, m, n, k, ta, tb, bz, sc, v;
        char extra;
        if (std::sscanf(line, "%d %d %d %d %d %d %d %d %d %c", &t, &m, &n, &k, &ta, &tb, &bz, &sc, &v,
                        &extra) != 9 ||
            !valid_entry(t, m, n, k, ta, tb, bz, sc, v)) {
            st = SBGEMM_ERR_IO;
            break;
        }
        (*out)[Key(t, m, n, k, ta, tb, bz, sc)] = v;
    }
    std::fclose(f);
    if (st == SBGEMM_SUCCESS && !header) st = SBGEMM_ERR_IO;
    return st;
}

int read_model_file(const char* path, CostModel* M) {
    FILE* f = std::fopen(path, "r");
    if (!f) return SBGEMM_ERR_IO;
    int st = SBGEMM_ERR_IO;
    char buf[512];
    int ver = 0;
    long long np = 0;
    do {
        if (!std::fgets(buf, sizeof buf, f) || std::sscanf(buf, "sbgemm-cost-model %d", &ver) != 1 ||
            (ver != 1 && ver != 2))
            break;
        if (!std::fgets(buf, sizeof buf, f) || std::strncmp(buf, "device ", 7) != 0) break;
        M->device.assign(buf + 7);
        while (!M->device.empty() && (M->device.back() == '\n' || M->device.back() == '\r'))
            M->device.pop_back();
        if (std::fscanf(f, " features %d hidden %d outputs %d", &M->F, &M->H, &M->V) != 3) break;
        if (std::fscanf(f, " log_time_mean %lf log_time_std %lf", &M->mu, &M->sd) != 2) break;
        if (ver == 1) {          // one margin for every storage type
            if (std::fscanf(f, " margin %lf", &M->margin[0]) != 1) break;
            for (int t = 1; t < 6; ++t) M->margin[t] = M->margin[0];
        } else {
            double* g = M->margin;
            if (std::fscanf(f, " margins %lf %lf %lf %lf %lf %lf", g, g + 1, g + 2, g + 3, g + 4,
                            g + 5) != 6)
                break;
        }
        if (std::fscanf(f, " params %lld", &np) != 1) break;
        if (np != sbgemm_mlp_param_count(M->F, M->H, M->V) || np <= 0) break;
        M->params.resize((size_t)np);
        long long i = 0;
        for (; i < np; ++i)
            if (std::fscanf(f, " %f", &M->params[(size_t)i]) != 1) break;
        if (i != np) break;
        char extra;
        if (std::fscanf(f, " %c", &extra) == 1) break;     // trailing content
        st = SBGEMM_SUCCESS;
    } while (false);
    std::fclose(f);
    return st;
}

// margins: one per storage type, 0 <= margin <= 1 (1: the built-in rule's
// variant is always kept for that type)
bool model_args_ok(int F, int H, int V, double sd, const double* margin) {
    if (!(F == 16 && H >= 1 && H <= 4096 && V >= 1 && V <= 64 && std::isfinite(sd) && sd > 0))
        return false;
    for (int t = 0; t < 6; ++t)
        if (!std::isfinite(margin[t]) || margin[t] < 0 || margin[t] > 1) return false;
    return true;
}

int install_model(CostModel&& M) {
    std::lock_guard<std::mutex> lk(g_model_mu);
    g_model = std::move(M);
    g_model.present = true;
    g_model.evaluated = false;
    g_model.eval_status = 0;
    g_model.choice.clear();
    if (g_mode.load() == SBGEMM_SELECTOR_MODEL) return evaluate_model_locked();
    return SBGEMM_SUCCESS;
}

// Environment: SBGEMM_SELECTOR = default | table | model, SBGEMM_TABLE = a
// table file to load, SBGEMM_COST_MODEL = a cost-model file to load.  Read
// once, before the first selection or selector call.
void init_from_env() {
    std::call_once(g_env_once, [] {
        int first = 0;
        auto note = [&](int st) { if (st != 0 && first == 0) first = st; };
        if (const char* p = std::getenv("SBGEMM_TABLE")) {
            if (*p) {
                std::map<Key, int> t;
                const int st = read_table_file(p, &t);
                note(st);
                if (st == SBGEMM_SUCCESS) {
                    std::lock_guard<std::mutex> lk(g_choice_mu);
                    for (auto& kv : t) g_choice[kv.first] = kv.second;
                }
            }
        }
        if (const char* p = std::getenv("SBGEMM_COST_MODEL")) {
            if (*p) {
                CostModel M;
                int st = read_model_file(p, &M);
                if (st == SBGEMM_SUCCESS && !model_args_ok(M.F, M.H, M.V, M.sd, M.margin))
                    st = SBGEMM_ERR_IO;
                note(st);
                if (st == SBGEMM_SUCCESS) {
                    std::lock_guard<std::mutex> lk(g_model_mu);
                    g_model = std::move(M);
                    g_model.present = true;      // evaluated at its first use
                }
            }
        }
        if (const char* p = std::getenv("SBGEMM_SELECTOR")) {
            if (!std::strcmp(p, "default")) g_mode = SBGEMM_SELECTOR_DEFAULT;
            else if (!std::strcmp(p, "table")) g_mode = SBGEMM_SELECTOR_TABLE;
            else if (!std::strcmp(p, "model")) {
                std::lock_guard<std::mutex> lk(g_model_mu);
                if (g_model.present) g_mode = SBGEMM_SELECTOR_MODEL;
                else note(SBGEMM_ERR_INVALID_VALUE);
            } else if (*p) {
                note(SBGEMM_ERR_INVALID_VALUE);
            }
        }
        g_env_status = first;
    });
}

}  // namespace

int size_class(int batch) {
    int c = 0;
    while (batch >= 10 && c < 7) { batch /= 10; ++c; }
    return c;
}

int variants_for(int type, int m, int n, int k) {
    if (m < 1 || n < 1 || k < 1 || m > 16 || n > 16 || k > 16) return 0;
    // shapes without specialised kernels: the generic kernel, and for real
    // and complex fp64 also the tensor-core kernel (public variant 1)
    if (!has_specialized(0, m, n, k))
        return type == SBGEMM_TYPE_D || type == SBGEMM_TYPE_Z ? 2 : 1;
    return has_mma_variant(type, m, n, k) ? kMmaVariant + 1 : kNumPipeVariants + 1;
}

// The variant used without a table entry or cost model (sc: the batch's
// size class, floor(log10 N)):
// - the tensor-core kernel for the 16-bit types at m = n = k = 8, 12 and 16
//   (measured 1.3-1.7x faster at 8 and 16; at m = 12, N = 1e6, binary16:
//   153.6 against 197.2 us with beta = 0, 207.8 against 311.9 us with
//   beta = -0.5);
// - variant 2 (32 KB tiles, two stages: more blocks per SM and a shorter
//   pipeline to fill) for complex64 and for fp32 below 1e6 pairs: over the
//   square N/N sizes 2..16 it took 9% less total time than variant 0 for
//   complex64 at N = 1e5 and 1e6, and 5% less for fp32 at N = 1e5 (up to 20%
//   per size), while fp32 at N = 1e6 measured the same total;
// - the tensor-core kernel (digit-split products) for real fp64 at
//   m = n = k = 13..16, at 12 with beta != 0, and at 16 x 8 x 16: with
//   alpha = 1.5 at N = 1e5 it took 387 / 388 / 383 / 355 us for
//   m = 13 / 14 / 15 / 16 against 494 / 508 / 647 / 738 us on the fp64 FMA
//   pipe with beta = 0 (1.28-2.08x), 413 / 416 / 413 / 383 us against
//   550 / 557 / 733 / 791 us with beta = -0.5 (1.33-2.06x), 416 against
//   434 us at m = 12 with beta != 0 (385 against 333 with beta = 0), and
//   236 us against 403 us for 16 x 8 x 16 (op(A) = T, beta = 1); below
//   m = 12 and on the other FEM shapes the FMA kernels win, as the
//   tensor-core kernel always computes a 16 x 16 x 16 product;
// - for real fp64 shapes without specialised kernels, the tensor-core
//   kernel (public variant 1) when m n k >= 1024 with beta == 0 or >= 1320
//   otherwise: over the 334 such shapes with m, n, k in {4, 8, 11, 13, 14,
//   15, 16}, op N/N, N = 1e5, this rule took 95.0 / 101.7 ms in total
//   (beta == 0 / beta = -0.5) against 94.3 / 100.8 ms for the best variant
//   of each shape and 129.6 / 135.3 ms for the generic kernel alone;
// - the tensor-core kernel for complex128 at m = n = k = 12..16 and at
//   16 x 8 x 16: with alpha = 1.5 at N = 1e5 it took 1.12 / 1.13 / 1.15 /
//   1.16 / 1.12 ms for m = 12 / 13 / 14 / 15 / 16 against 1.28 / 1.95 /
//   2.25 / 2.48 / 2.88 ms on the fp64 FMA pipe with beta = 0 (1.14-2.57x;
//   1.09-2.35x with beta = -0.5), and 0.80 against 1.88 ms for 16 x 8 x 16
//   (op(A) = T, beta = 1); at m = 11 they were even; on the complex128
//   shapes without specialised kernels, the tensor-core kernel (public
//   variant 1) when m n k >= 1024: over the same 334 shapes, 277.1 / 316.4 ms
//   in total against 275.6 / 314.9 ms for the best variant of each and
//   411.4 / 452.0 ms for the generic kernel alone;
// - variant 0 otherwise (fp64 and complex128, bound by the fp64 pipe, showed
//   no difference; the 16-bit CUDA-core kernels were mixed).
int default_variant(int type, int m, int n, int k, int bz, int sc) {
    if (type == SBGEMM_TYPE_Z) {
        if (!has_specialized(0, m, n, k)) return m * n * k >= 1024 ? 1 : 0;
        if (m == n && n == k && m >= 12) return kMmaVariant;
        if (m == 16 && n == 8 && k == 16) return kMmaVariant;
    }
    if (type == SBGEMM_TYPE_D) {
        if (!has_specialized(0, m, n, k)) return m * n * k >= (bz ? 1024 : 1320) ? 1 : 0;
        if (m == n && n == k && (m >= 13 || (m == 12 && !bz))) return kMmaVariant;
        if (m == 16 && n == 8 && k == 16) return kMmaVariant;
    }
    if ((type == SBGEMM_TYPE_H || type == SBGEMM_TYPE_B) && has_mma_variant(type, m, n, k))
        return kMmaVariant;
    if (!has_specialized(0, m, n, k)) return 0;
    if (type == SBGEMM_TYPE_C || (type == SBGEMM_TYPE_S && sc <= 5)) return 2;
    return 0;
}

int select_variant(int type, int m, int n, int k, int ta, int tb, int bz, int sc) {
    init_from_env();
    const int nv = variants_for(type, m, n, k);
    const int mode = g_mode.load(std::memory_order_relaxed);
    if (mode != SBGEMM_SELECTOR_DEFAULT) {
        const int v = lookup_choice(type, m, n, k, ta, tb, bz, sc);
        if (v >= 0 && v < nv) return v;
    }
    if (mode == SBGEMM_SELECTOR_MODEL && nv > 1) {
        const int v = model_choice(type, m, n, k, ta, tb, bz, sc);
        if (v >= 0 && v < nv) return v;
    }
    return default_variant(type, m, n, k, bz, sc);
}

void note_variant(int v) { t_last_variant = v; }

}  // namespace sbg

extern "C" {

sbgemm_status sbgemm_set_choice(int type, int m, int n, int k, int ta, int tb,
                                int beta_zero, int size_class, int variant) {
    sbg::init_from_env();
    if (type < SBGEMM_TYPE_S || type > SBGEMM_TYPE_B) return SBGEMM_ERR_INVALID_VALUE;
    const int nv = sbg::variants_for(type, m, n, k);
    if (nv == 0 || variant >= nv || size_class < 0 || size_class > 7) return SBGEMM_ERR_INVALID_VALUE;
    std::lock_guard<std::mutex> lk(sbg::g_choice_mu);
    sbg::Key key(type, m, n, k, ta ? 1 : 0, tb ? 1 : 0, beta_zero ? 1 : 0, size_class);
    if (variant < 0) sbg::g_choice.erase(key);
    else sbg::g_choice[key] = variant;
    return SBGEMM_SUCCESS;
}

int sbgemm_get_choice(int type, int m, int n, int k, int ta, int tb, int beta_zero, int size_class) {
    if (type < SBGEMM_TYPE_S || type > SBGEMM_TYPE_B || size_class < 0 || size_class > 7) return -1;
    if (sbg::variants_for(type, m, n, k) == 0) return -1;
    return sbg::select_variant(type, m, n, k, ta ? 1 : 0, tb ? 1 : 0, beta_zero ? 1 : 0, size_class);
}

int sbgemm_default_variant(int type, int m, int n, int k, int beta_zero, int size_class) {
    if (type < SBGEMM_TYPE_S || type > SBGEMM_TYPE_B || size_class < 0 || size_class > 7) return -1;
    if (sbg::variants_for(type, m, n, k) == 0) return -1;
    return sbg::default_variant(type, m, n, k, beta_zero ? 1 : 0, size_class);
}

void sbgemm_clear_choices(void) {
    sbg::init_from_env();
    std::lock_guard<std::mutex> lk(sbg::g_choice_mu);
    sbg::g_choice.clear();
}

int sbgemm_last_variant(void) { return sbg::t_last_variant; }

sbgemm_status sbgemm_save_table(const char* path) {
    sbg::init_from_env();
    if (!path) return SBGEMM_ERR_NULL_POINTER;
    std::map<sbg::Key, int> copy;
    {
        std::lock_guard<std::mutex> lk(sbg::g_choice_mu);
        copy = sbg::g_choice;
    }
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return SBGEMM_ERR_IO;
    std::fprintf(f, "sbgemm-table 1\ndevice %s\n", sbg::device_name().c_str());
    std::fprintf(f, "# type m n k ta tb beta_zero size_class variant\n");
    for (auto& kv : copy) {
        const sbg::Key& k = kv.first;
        std::fprintf(f, "%d %d %d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k),
                     std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k), std::get<6>(k),
                     std::get<7>(k), kv.second);
    }
    const bool ok = std::fflush(f) == 0 && !std::ferror(f);
    std::fclose(f);
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return SBGEMM_ERR_IO;
    }
    return SBGEMM_SUCCESS;
}

sbgemm_status sbgemm_load_table(const char* path) {
    sbg::init_from_env();
    if (!path) return SBGEMM_ERR_NULL_POINTER;
    std::map<sbg::Key, int> t;
    const int st = sbg::read_table_file(path, &t);
    if (st != SBGEMM_SUCCESS) return st;
    std::lock_guard<std::mutex> lk(sbg::g_choice_mu);
    for (auto& kv : t) sbg::g_choice[kv.first] = kv.second;
    return SBGEMM_SUCCESS;
}

sbgemm_status sbgemm_set_selector(int mode) {
    sbg::init_from_env();
    if (mode != SBGEMM_SELECTOR_DEFAULT && mode != SBGEMM_SELECTOR_TABLE &&
        mode != SBGEMM_SELECTOR_MODEL)
        return SBGEMM_ERR_INVALID_VALUE;
    if (mode == SBGEMM_SELECTOR_MODEL) {
        std::lock_guard<std::mutex> lk(sbg::g_model_mu);
        if (!sbg::g_model.present) return SBGEMM_ERR_INVALID_VALUE;
        if (!sbg::g_model.evaluated) {
            const int st = sbg::evaluate_model_locked();
            if (st != 0) return st;
        }
    }
    sbg::g_mode = mode;
    return SBGEMM_SUCCESS;
}

sbgemm_status sbgemm_get_selector(int* mode, int* env_status) {
    sbg::init_from_env();
    if (!mode) return SBGEMM_ERR_NULL_POINTER;
    *mode = sbg::g_mode.load();
    if (env_status) *env_status = sbg::g_env_status.load();
    return SBGEMM_SUCCESS;
}

sbgemm_status sbgemm_set_cost_model(int F, int H, int V, const float* params, double log_time_mean,
                                    double log_time_std, const double* margins) {
    sbg::init_from_env();
    if (!params || !margins) return SBGEMM_ERR_NULL_POINTER;
    if (!sbg::model_args_ok(F, H, V, log_time_std, margins) || !std::isfinite(log_time_mean))
        return SBGEMM_ERR_INVALID_VALUE;
    const long long np = sbgemm_mlp_param_count(F, H, V);
    sbg::CostModel M;
    M.F = F; M.H = H; M.V = V;
    M.params.assign(params, params + np);
    for (float x : M.params)
        if (!std::isfinite(x)) return SBGEMM_ERR_INVALID_VALUE;
    M.mu = log_time_mean; M.sd = log_time_std;
    for (int t = 0; t < 6; ++t) M.margin[t] = margins[t];
    M.device = sbg::device_name();
    return sbg::install_model(std::move(M));
}

sbgemm_status sbgemm_save_cost_model(const char* path) {
    sbg::init_from_env();
    if (!path) return SBGEMM_ERR_NULL_POINTER;
    sbg::CostModel M;
    {
        std::lock_guard<std::mutex> lk(sbg::g_model_mu);
        if (!sbg::g_model.present) return SBGEMM_ERR_INVALID_VALUE;
        M.F = sbg::g_model.F; M.H = sbg::g_model.H; M.V = sbg::g_model.V;
        M.params = sbg::g_model.params;
        M.mu = sbg::g_model.mu; M.sd = sbg::g_model.sd;
        for (int t = 0; t < 6; ++t) M.margin[t] = sbg::g_model.margin[t];
        M.device = sbg::g_model.device;
    }
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return SBGEMM_ERR_IO;
    std::fprintf(f, "sbgemm-cost-model 2\ndevice %s\n", M.device.c_str());
    std::fprintf(f, "features %d hidden %d outputs %d\n", M.F, M.H, M.V);
    std::fprintf(f, "log_time_mean %.17g log_time_std %.17g\n", M.mu, M.sd);
    std::fprintf(f, "margins");
    for (int t = 0; t < 6; ++t) std::fprintf(f, " %.17g", M.margin[t]);
    std::fprintf(f, "\n");
    std::fprintf(f, "params %lld\n", (long long)M.params.size());
    for (size_t i = 0; i < M.params.size(); ++i)
        std::fprintf(f, "%.9g%c", M.params[i], (i % 8 == 7 || i + 1 == M.params.size()) ? '\n' : ' ');
    const bool ok = std::fflush(f) == 0 && !std::ferror(f);
    std::fclose(f);
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return SBGEMM_ERR_IO;
    }
    return SBGEMM_SUCCESS;
}

sbgemm_status sbgemm_load_cost_model(const char* path) {
    sbg::init_from_env();
    if (!path) return SBGEMM_ERR_NULL_POINTER;
    sbg::CostModel M;
    int st = sbg::read_model_file(path, &M);
    if (st != SBGEMM_SUCCESS) return st;
    if (!sbg::model_args_ok(M.F, M.H, M.V, M.sd, M.margin)) return SBGEMM_ERR_IO;
    return sbg::install_model(std::move(M));
}

sbgemm_status sbgemm_tune(int type, char transa, char transb, int m, int n, int k,
    const void* alpha, const void* A, int lda, long long lda2, const void* B, int ldb,
    long long ldb2, const void* beta, void* C, int ldc, long long ldc2, int batchCount, int reps,
    void* flush, size_t flush_bytes, void* stream, int* best, float* ms) {
    sbg::init_from_env();
    if (!best || !beta) return SBGEMM_ERR_NULL_POINTER;
    if (type < SBGEMM_TYPE_S || type > SBGEMM_TYPE_B || batchCount < 1 || reps < 1)
        return SBGEMM_ERR_INVALID_VALUE;
    const int nv = sbgemm_num_variants(type, m, n, k);
    if (nv < 1) return SBGEMM_ERR_INVALID_SIZE;
    int bi = -1;
    float bt = 0.f;
    for (int v = 0; v < nv; ++v) {
        float t = 0.f;
        const sbgemm_status st = sbgemm_time_variant(type, transa, transb, m, n, k, alpha, A, lda,
                                                     lda2, B, ldb, ldb2, beta, C, ldc, ldc2,
                                                     batchCount, v, reps, flush, flush_bytes,
                                                     stream, &t);
        if (st != SBGEMM_SUCCESS) return st;
        if (ms) ms[v] = t;
        if (bi < 0 || t < bt) { bi = v; bt = t; }
    }
    *best = bi;
    const int ta = !(transa == 'N' || transa == 'n'), tb = !(transb == 'N' || transb == 'n');
    // beta == 0 of host scalars decides the class (C is then not read)
    bool bz;
    switch (type) {
    case SBGEMM_TYPE_D: bz = *static_cast<const double*>(beta) == 0.0; break;
    case SBGEMM_TYPE_C: { const float* f = static_cast<const float*>(beta); bz = f[0] == 0.f && f[1] == 0.f; break; }
    case SBGEMM_TYPE_Z: { const double* d = static_cast<const double*>(beta); bz = d[0] == 0.0 && d[1] == 0.0; break; }
    default: bz = *static_cast<const float*>(beta) == 0.f;
    }
    return sbgemm_set_choice(type, m, n, k, ta, tb, bz ? 1 : 0, sbg::size_class(batchCount), bi);
}

}  // extern "C"
