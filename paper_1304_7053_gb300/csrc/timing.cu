// Native timing core: CUDA-event timers whose marks can be captured into
// CUDA graphs, and the per-variant timing loop the autotuner runs.
#include <algorithm>
#include <new>
#include <vector>

#include "sbgemm_launch.cuh"

struct sbgemm_timer_s {
    std::vector<cudaEvent_t> ev;
};

namespace sbg {
sbgemm_status gemm_uniform(int type, char transa, char transb, int m, int n, int k,
                           const void* alpha, const void* A, int lda, long long lda2,
                           const void* B, int ldb, long long ldb2,
                           const void* beta, void* C, int ldc, long long ldc2, int batch,
                           int scalar_mode, int variant, cudaStream_t stream);
}

extern "C" {

sbgemm_status sbgemm_timer_create(sbgemm_timer* timer, int n_marks) {
    if (!timer || n_marks < 2 || n_marks > (1 << 20)) return SBGEMM_ERR_INVALID_VALUE;
    sbgemm_timer t = new (std::nothrow) sbgemm_timer_s;
    if (!t) return SBGEMM_ERR_CAPACITY;
    t->ev.resize(n_marks, nullptr);
    for (auto& e : t->ev) {
        cudaError_t st = cudaEventCreateWithFlags(&e, cudaEventDefault);
        if (st != cudaSuccess) {
            for (auto& x : t->ev) if (x) cudaEventDestroy(x);
            delete t;
            return (sbgemm_status)st;
        }
    }
    *timer = t;
    return SBGEMM_SUCCESS;
}

sbgemm_status sbgemm_timer_mark(sbgemm_timer timer, int mark, void* stream) {
    if (!timer || mark < 0 || mark >= (int)timer->ev.size()) return SBGEMM_ERR_INVALID_VALUE;
    // while the stream is being captured an external record becomes an event
    // node of the graph; outside capture the external flag is not allowed and
    // an ordinary record is used
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing((cudaStream_t)stream, &cs);
    if (e != cudaSuccess) return (sbgemm_status)e;
    if (cs == cudaStreamCaptureStatusActive)
        return (sbgemm_status)cudaEventRecordWithFlags(timer->ev[mark], (cudaStream_t)stream,
                                                       cudaEventRecordExternal);
    return (sbgemm_status)cudaEventRecord(timer->ev[mark], (cudaStream_t)stream);
}

sbgemm_status sbgemm_timer_elapsed(sbgemm_timer timer, int from, int to, float* ms) {
    if (!timer || !ms || from < 0 || to < 0 || from >= (int)timer->ev.size() ||
        to >= (int)timer->ev.size())
        return SBGEMM_ERR_INVALID_VALUE;
    cudaError_t st = cudaEventSynchronize(timer->ev[to]);
    if (st != cudaSuccess) return (sbgemm_status)st;
    return (sbgemm_status)cudaEventElapsedTime(ms, timer->ev[from], timer->ev[to]);
}

sbgemm_status sbgemm_timer_destroy(sbgemm_timer timer) {
    if (!timer) return SBGEMM_ERR_INVALID_VALUE;
    for (auto& e : timer->ev) if (e) cudaEventDestroy(e);
    delete timer;
    return SBGEMM_SUCCESS;
}

}  // extern "C"

namespace {

// Read every 16-byte word of a buffer (a sink write nobody takes keeps the
// loads): run before a timed call it evicts L2 with clean lines, so the
// previous call's dirty results are written back outside the timed interval.
__global__ void flush_read_kernel(const uint4* __restrict__ p, size_t n, unsigned* sink) {
    unsigned acc = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const uint4 v = p[i];
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x9E3779B9u && sink) *sink = acc;
}

// Event timestamps can advance in steps of about a microsecond, and where a
// call starts against those steps varies from call to call, so the mean of
// the calls resolves a time below one step where the median snaps to a
// step.  Calls more than 2 us from the median (delayed or preempted) are
// left out.
float robust_mean_ms(std::vector<float> d) {
    std::sort(d.begin(), d.end());
    const float med = d[d.size() / 2];
    double sum = 0.0;
    int n = 0;
    for (float x : d)
        if (x >= med - 0.002f && x <= med + 0.002f) { sum += x; ++n; }
    return (float)(sum / n);
}

}  // namespace

extern "C" {

sbgemm_status sbgemm_time_variant(int type, char transa, char transb, int m, int n, int k,
    const void* alpha, const void* A, int lda, long long lda2,
    const void* B, int ldb, long long ldb2, const void* beta, void* C, int ldc,
    long long ldc2, int batchCount, int variant, int reps, void* flush, size_t flush_bytes,
    void* stream, float* ms_out) {
    if (!ms_out || reps < 1 || reps > 100000 || variant < 0) return SBGEMM_ERR_INVALID_VALUE;
    cudaStream_t s = (cudaStream_t)stream;
    // one untimed call first: the first launch of a variant does host-side
    // set-up (function attributes, occupancy) while the GPU waits
    sbgemm_status st = sbg::gemm_uniform(type, transa, transb, m, n, k, alpha, A, lda, lda2, B,
                                         ldb, ldb2, beta, C, ldc, ldc2, batchCount,
                                         SBGEMM_SCALARS_HOST, variant, s);
    if (st != SBGEMM_SUCCESS) return st;
    sbgemm_timer t = nullptr;
    st = sbgemm_timer_create(&t, 2 * reps);
    if (st != SBGEMM_SUCCESS) return st;
    for (int r = 0; r < reps && st == SBGEMM_SUCCESS; ++r) {
        if (flush && flush_bytes >= 16) {
            const size_t n16 = flush_bytes / 16;
            flush_read_kernel<<<(unsigned)(sbg::num_sms() * 8), 256, 0, s>>>(
                static_cast<const uint4*>(flush), n16, nullptr);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { st = (sbgemm_status)e; break; }
        }
        st = sbgemm_timer_mark(t, 2 * r, stream);
        if (st == SBGEMM_SUCCESS)
            st = sbg::gemm_uniform(type, transa, transb, m, n, k, alpha, A, lda, lda2, B, ldb,
                                   ldb2, beta, C, ldc, ldc2, batchCount, SBGEMM_SCALARS_HOST,
                                   variant, s);
        if (st == SBGEMM_SUCCESS) st = sbgemm_timer_mark(t, 2 * r + 1, stream);
    }
    std::vector<float> d;
    for (int r = 0; r < reps && st == SBGEMM_SUCCESS; ++r) {
        float ms = 0.f;
        st = sbgemm_timer_elapsed(t, 2 * r, 2 * r + 1, &ms);
        d.push_back(ms);
    }
    sbgemm_timer_destroy(t);
    if (st != SBGEMM_SUCCESS) return st;
    *ms_out = robust_mean_ms(d);
    return SBGEMM_SUCCESS;
}

}  // extern "C"
