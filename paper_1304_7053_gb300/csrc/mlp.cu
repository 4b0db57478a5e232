// Cost-model network: a 3-layer perceptron (F inputs, H hidden, V outputs)
// trained and evaluated by these kernels in fp32.
//
//   Z1 = X W1^T + b1,  H1 = relu(Z1)
//   Z2 = H1 W2^T + b2, H2 = relu(Z2)
//   Y  = H2 W3^T + b3
//   L  = sum mask (Y - T)^2 / (2 M),  M = sum mask
// Gradients are the chain rule layer by layer (relu'(0) = 0); the update is
// Adam (Kingma & Ba, ICLR 2015, Algorithm 1) on the gradient of
// L + (l2 / 2) |params|^2 (an L2 penalty on every parameter, added to the
// gradient before the moment estimates).  Every reduction is a plain
// loop in a fixed order (no atomics), so results are reproducible.
//
// Parameters live in one buffer: W1 (H x F), b1 (H), W2 (H x H), b2 (H),
// W3 (V x H), b3 (V), row-major.  The sizes are small (a few thousand rows,
// H = 64), so the kernels use one thread per output element.
#include <cuda_runtime.h>

#include "../../include/sbgemm.h"

namespace {

struct Layout {
    int F, H, V;
    size_t w1, b1, w2, b2, w3, b3, total;
    __host__ __device__ Layout(int f, int h, int v) : F(f), H(h), V(v) {
        w1 = 0;
        b1 = w1 + (size_t)H * F;
        w2 = b1 + H;
        b2 = w2 + (size_t)H * H;
        w3 = b2 + H;
        b3 = w3 + (size_t)V * H;
        total = b3 + V;
    }
};

// out[b, o] = act(sum_i in[b, i] W[o, i] + bias[o]); pre[b, o] keeps the
// pre-activation when requested.
__global__ void dense_fwd(const float* __restrict__ in, int batch, int nin,
                          const float* __restrict__ W, const float* __restrict__ bias, int nout,
                          float* __restrict__ pre, float* __restrict__ out, int relu) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)batch * nout) return;
    const int b = (int)(idx / nout), o = (int)(idx - (long long)b * nout);
    float acc = 0.f;
    const float* x = in + (long long)b * nin;
    const float* w = W + (long long)o * nin;
    for (int i = 0; i < nin; ++i) acc = fmaf(x[i], w[i], acc);
    acc += bias[o];
    if (pre) pre[idx] = acc;
    out[idx] = relu ? fmaxf(acc, 0.f) : acc;
}

// M = sum mask and L = sum mask (Y - T)^2 / (2M), single block tree reduction
// in a fixed order.
__global__ void loss_reduce(const float* __restrict__ Y, const float* __restrict__ T,
                            const float* __restrict__ mask, long long n, float* __restrict__ out) {
    __shared__ double s_l[256], s_m[256];
    double l = 0.0, m = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = (double)Y[i] - (double)T[i];
        l += (double)mask[i] * d * d;
        m += (double)mask[i];
    }
    s_l[threadIdx.x] = l;
    s_m[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            s_l[threadIdx.x] += s_l[threadIdx.x + s];
            s_m[threadIdx.x] += s_m[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s_m[0] > 0 ? (float)(s_l[0] / (2.0 * s_m[0])) : 0.f;
        out[1] = (float)s_m[0];
    }
}

// dY = mask (Y - T) / M
__global__ void loss_grad(const float* __restrict__ Y, const float* __restrict__ T,
                          const float* __restrict__ mask, long long n, const float* __restrict__ lm,
                          float* __restrict__ dY) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float M = lm[1];
    dY[i] = M > 0.f ? mask[i] * (Y[i] - T[i]) / M : 0.f;
}

// dW[o, i] = sum_b dZ[b, o] in[b, i]; db[o] = sum_b dZ[b, o]
__global__ void dense_bwd_w(const float* __restrict__ dZ, const float* __restrict__ in, int batch,
                            int nin, int nout, float* __restrict__ dW, float* __restrict__ db) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nw = (long long)nout * nin;
    if (idx < nw) {
        const int o = (int)(idx / nin), i = (int)(idx - (long long)o * nin);
        float acc = 0.f;
        for (int b = 0; b < batch; ++b) acc = fmaf(dZ[(long long)b * nout + o], in[(long long)b * nin + i], acc);
        dW[idx] = acc;
    } else if (idx < nw + nout) {
        const int o = (int)(idx - nw);
        float acc = 0.f;
        for (int b = 0; b < batch; ++b) acc += dZ[(long long)b * nout + o];
        db[o] = acc;
    }
}

// dIn[b, i] = (sum_o dZ[b, o] W[o, i]) * [pre[b, i] > 0]
__global__ void dense_bwd_x(const float* __restrict__ dZ, const float* __restrict__ W, int batch,
                            int nin, int nout, const float* __restrict__ pre, float* __restrict__ dIn) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)batch * nin) return;
    const int b = (int)(idx / nin), i = (int)(idx - (long long)b * nin);
    float acc = 0.f;
    for (int o = 0; o < nout; ++o) acc = fmaf(dZ[(long long)b * nout + o], W[(long long)o * nin + i], acc);
    dIn[idx] = pre[idx] > 0.f ? acc : 0.f;
}

__global__ void adam_kernel(long long n, float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                            float b2, float eps, float l2, float c1, float c2) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i] + l2 * p[i];      // gradient of L + (l2 / 2) |p|^2
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mhat = mi / c1, vhat = vi / c2;
    p[i] -= lr * mhat / (sqrtf(vhat) + eps);
}

inline unsigned blocks_for(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

bool bad_dims(int F, int H, int V, int batch) {
    return F < 1 || H < 1 || V < 1 || F > 4096 || H > 4096 || V > 4096 || batch < 0;
}

}  // namespace

extern "C" {

long long sbgemm_mlp_param_count(int F, int H, int V) {
    if (bad_dims(F, H, V, 0)) return 0;
    return (long long)Layout(F, H, V).total;
}

sbgemm_status sbgemm_mlp_forward(int F, int H, int V, const float* params, const float* X,
                                 int batch, float* Y, float* work, void* stream) {
    if (bad_dims(F, H, V, batch)) return SBGEMM_ERR_INVALID_VALUE;
    if (batch == 0) return SBGEMM_SUCCESS;
    if (!params || !X || !Y || !work) return SBGEMM_ERR_NULL_POINTER;
    const Layout L(F, H, V);
    cudaStream_t s = (cudaStream_t)stream;
    float* Z1 = work;
    float* H1 = work + (size_t)batch * H;
    float* Z2 = work + 2 * (size_t)batch * H;
    float* H2 = work + 3 * (size_t)batch * H;
    dense_fwd<<<blocks_for((long long)batch * H), 256, 0, s>>>(X, batch, F, params + L.w1, params + L.b1, H, Z1, H1, 1);
    dense_fwd<<<blocks_for((long long)batch * H), 256, 0, s>>>(H1, batch, H, params + L.w2, params + L.b2, H, Z2, H2, 1);
    dense_fwd<<<blocks_for((long long)batch * V), 256, 0, s>>>(H2, batch, H, params + L.w3, params + L.b3, V, nullptr, Y, 0);
    return (sbgemm_status)cudaGetLastError();
}

sbgemm_status sbgemm_mlp_backward(int F, int H, int V, const float* params, const float* X,
                                  int batch, const float* Y, const float* T, const float* mask,
                                  const float* work, float* grads, float* work2, float* loss,
                                  void* stream) {
    if (bad_dims(F, H, V, batch)) return SBGEMM_ERR_INVALID_VALUE;
    if (!params || !X || !Y || !T || !mask || !work || !grads || !work2 || !loss)
        return SBGEMM_ERR_NULL_POINTER;
    const Layout L(F, H, V);
    cudaStream_t s = (cudaStream_t)stream;
    const float* Z1 = work;
    const float* H1 = work + (size_t)batch * H;
    const float* Z2 = work + 2 * (size_t)batch * H;
    const float* H2 = work + 3 * (size_t)batch * H;
    float* dY = work2;                                   // batch x V
    float* dZ2 = work2 + (size_t)batch * V;              // batch x H
    float* dZ1 = dZ2 + (size_t)batch * H;                // batch x H
    const long long nY = (long long)batch * V;
    loss_reduce<<<1, 256, 0, s>>>(Y, T, mask, nY, loss);
    if (batch > 0) loss_grad<<<blocks_for(nY), 256, 0, s>>>(Y, T, mask, nY, loss, dY);
    dense_bwd_w<<<blocks_for((long long)V * H + V), 256, 0, s>>>(dY, H2, batch, H, V, grads + L.w3, grads + L.b3);
    dense_bwd_x<<<blocks_for((long long)batch * H), 256, 0, s>>>(dY, params + L.w3, batch, H, V, Z2, dZ2);
    dense_bwd_w<<<blocks_for((long long)H * H + H), 256, 0, s>>>(dZ2, H1, batch, H, H, grads + L.w2, grads + L.b2);
    dense_bwd_x<<<blocks_for((long long)batch * H), 256, 0, s>>>(dZ2, params + L.w2, batch, H, H, Z1, dZ1);
    dense_bwd_w<<<blocks_for((long long)H * F + H), 256, 0, s>>>(dZ1, X, batch, F, H, grads + L.w1, grads + L.b1);
    return (sbgemm_status)cudaGetLastError();
}

sbgemm_status sbgemm_mlp_adam(long long n, float* params, const float* grads, float* m, float* v,
                              int t, float lr, float beta1, float beta2, float eps, float l2,
                              void* stream) {
    if (n < 0 || t < 1 || !(l2 >= 0.f) || l2 > 1e30f) return SBGEMM_ERR_INVALID_VALUE;
    if (n == 0) return SBGEMM_SUCCESS;
    if (!params || !grads || !m || !v) return SBGEMM_ERR_NULL_POINTER;
    // bias corrections 1 - beta^t, computed on the host in double
    double c1 = 1.0, c2 = 1.0, p1 = 1.0, p2 = 1.0;
    for (int i = 0; i < t; ++i) { p1 *= beta1; p2 *= beta2; }
    c1 -= p1;
    c2 -= p2;
    adam_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, params, grads, m, v, lr, beta1,
                                                                 beta2, eps, l2, (float)c1, (float)c2);
    return (sbgemm_status)cudaGetLastError();
}

}  // extern "C"
