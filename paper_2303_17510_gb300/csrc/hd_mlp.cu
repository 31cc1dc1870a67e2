// hd_mlp.cu -- the learned parameter selector: a small MLP trained on the
// autotuner's own timings, with hand-written forward, backward and Adam
// kernels, and the selector that uses an ensemble of such networks to pick a
// candidate (m, p, q, D, kernel variant) without timing, falling back to the
// timed search when the ensemble is unsure.  The paper has no selector; its
// optimizer (Section 7) is the timed search this stands in for.
//
// Network: h_0 = x; z_l = h_l W_l^T + b_l; h_{l+1} = tanh(z_l) for hidden
// layers; the last layer is linear with one output, the predicted log time of
// one convolution.  Loss: mean squared error.  FP32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "hd_plan.h"

struct hd_mlp {
    std::vector<int> dims;               // layer sizes, dims.back() == 1
    std::vector<int64_t> offW, offb;     // offsets of W_l and b_l in the parameter vector
    int64_t np = 0;
    float* p = nullptr;                  // parameters
    float* g = nullptr;                  // gradients
    float* m = nullptr;                  // Adam first moments
    float* v = nullptr;                  // Adam second moments
    int step = 0;
    int64_t cap = 0;                     // rows the activation buffers hold
    std::vector<float*> z;               // pre-activations per layer
    std::vector<float*> h;               // layer inputs (h[0] = caller's X)
    float* delta0 = nullptr;
    float* delta1 = nullptr;
    float* loss = nullptr;
};

namespace {

__global__ void k_dense(const float* __restrict__ H, int N, int din, const float* __restrict__ W,
                        const float* __restrict__ b, int dout, float* __restrict__ Z, float* __restrict__ Hout,
                        int act) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)N * dout) return;
    const int n = (int)(idx / dout), o = (int)(idx % dout);
    float z = b[o];
    for (int i = 0; i < din; ++i) z = fmaf(H[(int64_t)n * din + i], W[(int64_t)o * din + i], z);
    Z[idx] = z;
    if (Hout) Hout[idx] = act ? tanhf(z) : z;
}

// d loss / d y for the mean squared error, and the loss terms
__global__ void k_loss(const float* __restrict__ Y, const float* __restrict__ t, int N, float* __restrict__ delta,
                       float* __restrict__ terms) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const float d = Y[n] - t[n];
    delta[n] = 2.0f * d / (float)N;
    terms[n] = d * d;
}

// deterministic sum of N values by one block
__global__ void k_sum(const float* __restrict__ x, int N, float* __restrict__ out) {
    __shared__ float s[256];
    float acc = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) acc += x[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0] / (float)N;
}

// gradient of W_l (dout x din) and b_l: one thread per entry, sum over rows
__global__ void k_gradW(const float* __restrict__ delta, int N, int dout, const float* __restrict__ H, int din,
                        float* __restrict__ gW, float* __restrict__ gb) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= dout * (din + 1)) return;
    const int o = idx / (din + 1), i = idx % (din + 1);
    float acc = 0;
    if (i < din) {
        for (int n = 0; n < N; ++n) acc = fmaf(delta[(int64_t)n * dout + o], H[(int64_t)n * din + i], acc);
        gW[(int64_t)o * din + i] = acc;
    } else {
        for (int n = 0; n < N; ++n) acc += delta[(int64_t)n * dout + o];
        gb[o] = acc;
    }
}

// delta of the previous layer: (delta W) * tanh'(z_prev)
__global__ void k_backprop(const float* __restrict__ delta, int N, int dout, const float* __restrict__ W, int din,
                           const float* __restrict__ Zprev, float* __restrict__ dprev) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)N * din) return;
    const int n = (int)(idx / din), i = (int)(idx % din);
    float s = 0;
    for (int o = 0; o < dout; ++o) s = fmaf(delta[(int64_t)n * dout + o], W[(int64_t)o * din + i], s);
    const float th = tanhf(Zprev[idx]);
    dprev[idx] = s * (1.0f - th * th);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

hd_status ensure_cap(hd_mlp* M, int64_t N) {
    if (N <= M->cap) return HD_OK;
    for (float* q : M->z) cudaFree(q);
    for (size_t l = 1; l < M->h.size(); ++l) cudaFree(M->h[l]);
    cudaFree(M->delta0);
    cudaFree(M->delta1);
    cudaFree(M->loss);
    const int K = (int)M->dims.size() - 1;
    int maxd = 1;
    for (int d : M->dims) maxd = std::max(maxd, d);
    M->z.assign(K, nullptr);
    M->h.assign(K + 1, nullptr);
    bool ok = true;
    for (int l = 0; l < K && ok; ++l) ok = cudaMalloc(&M->z[l], sizeof(float) * N * M->dims[l + 1]) == cudaSuccess;
    for (int l = 1; l <= K && ok; ++l) ok = cudaMalloc(&M->h[l], sizeof(float) * N * M->dims[l]) == cudaSuccess;
    ok = ok && cudaMalloc(&M->delta0, sizeof(float) * N * maxd) == cudaSuccess;
    ok = ok && cudaMalloc(&M->delta1, sizeof(float) * N * maxd) == cudaSuccess;
    ok = ok && cudaMalloc(&M->loss, sizeof(float) * (N + 1)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        M->cap = 0;
        return HD_ERR_NOMEM;
    }
    M->cap = N;
    return HD_OK;
}

hd_status forward_impl(hd_mlp* M, const float* X, int64_t N, cudaStream_t st) {
    hd_status s = ensure_cap(M, N);
    if (s != HD_OK) return s;
    const int K = (int)M->dims.size() - 1;
    M->h[0] = const_cast<float*>(X);
    for (int l = 0; l < K; ++l) {
        const int din = M->dims[l], dout = M->dims[l + 1];
        k_dense<<<blocks(N * dout), 256, 0, st>>>(M->h[l], (int)N, din, M->p + M->offW[l], M->p + M->offb[l], dout,
                                                   M->z[l], M->h[l + 1], l < K - 1);
    }
    return cudaGetLastError() == cudaSuccess ? HD_OK : HD_ERR_CUDA;
}

hd_status grad_impl(hd_mlp* M, const float* X, const float* t, int64_t N, cudaStream_t st) {
    hd_status s = forward_impl(M, X, N, st);
    if (s != HD_OK) return s;
    const int K = (int)M->dims.size() - 1;
    k_loss<<<blocks(N), 256, 0, st>>>(M->h[K], t, (int)N, M->delta0, M->loss + 1);
    k_sum<<<1, 256, 0, st>>>(M->loss + 1, (int)N, M->loss);
    float* delta = M->delta0;
    float* other = M->delta1;
    for (int l = K - 1; l >= 0; --l) {
        const int din = M->dims[l], dout = M->dims[l + 1];
        k_gradW<<<blocks((int64_t)dout * (din + 1)), 256, 0, st>>>(delta, (int)N, dout, M->h[l], din, M->g + M->offW[l],
                                                                    M->g + M->offb[l]);
        if (l > 0) {
            k_backprop<<<blocks(N * din), 256, 0, st>>>(delta, (int)N, dout, M->p + M->offW[l], din, M->z[l - 1], other);
            std::swap(delta, other);
        }
    }
    return cudaGetLastError() == cudaSuccess ? HD_OK : HD_ERR_CUDA;
}

}  // namespace

extern "C" {

hd_status hd_mlp_create(hd_mlp** out, int nlayers, const int* dims) {
    if (!out || nlayers < 1 || nlayers > 8 || !dims) return HD_ERR_INVALID;
    *out = nullptr;
    for (int i = 0; i <= nlayers; ++i)
        if (dims[i] <= 0 || dims[i] > 1024) return HD_ERR_INVALID;
    if (dims[nlayers] != 1) return HD_ERR_INVALID;
    hd_mlp* M = new (std::nothrow) hd_mlp;
    if (!M) return HD_ERR_NOMEM;
    M->dims.assign(dims, dims + nlayers + 1);
    int64_t off = 0;
    for (int l = 0; l < nlayers; ++l) {
        M->offW.push_back(off);
        off += (int64_t)dims[l + 1] * dims[l];
        M->offb.push_back(off);
        off += dims[l + 1];
    }
    M->np = off;
    bool ok = cudaMalloc(&M->p, sizeof(float) * off) == cudaSuccess && cudaMalloc(&M->g, sizeof(float) * off) == cudaSuccess &&
              cudaMalloc(&M->m, sizeof(float) * off) == cudaSuccess && cudaMalloc(&M->v, sizeof(float) * off) == cudaSuccess;
    if (ok) ok = cudaMemset(M->p, 0, sizeof(float) * off) == cudaSuccess && cudaMemset(M->m, 0, sizeof(float) * off) == cudaSuccess &&
                 cudaMemset(M->v, 0, sizeof(float) * off) == cudaSuccess && cudaMemset(M->g, 0, sizeof(float) * off) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaFree(M->p);
        cudaFree(M->g);
        cudaFree(M->m);
        cudaFree(M->v);
        delete M;
        return HD_ERR_NOMEM;
    }
    *out = M;
    return HD_OK;
}

int64_t hd_mlp_num_params(const hd_mlp* M) { return M ? M->np : -1; }

hd_status hd_mlp_set_params(hd_mlp* M, const float* host) {
    if (!M || !host) return HD_ERR_INVALID;
    if (cudaMemcpy(M->p, host, sizeof(float) * M->np, cudaMemcpyHostToDevice) != cudaSuccess) return HD_ERR_CUDA;
    cudaMemset(M->m, 0, sizeof(float) * M->np);
    cudaMemset(M->v, 0, sizeof(float) * M->np);
    M->step = 0;
    return HD_OK;
}

hd_status hd_mlp_get_params(const hd_mlp* M, float* host) {
    if (!M || !host) return HD_ERR_INVALID;
    return cudaMemcpy(host, M->p, sizeof(float) * M->np, cudaMemcpyDeviceToHost) == cudaSuccess ? HD_OK : HD_ERR_CUDA;
}

hd_status hd_mlp_forward(hd_mlp* M, const float* X, int64_t N, float* Y, void* stream) {
    if (!M || !X || !Y || N <= 0) return HD_ERR_INVALID;
    hd_status s = forward_impl(M, X, N, (cudaStream_t)stream);
    if (s != HD_OK) return s;
    const int K = (int)M->dims.size() - 1;
    return cudaMemcpyAsync(Y, M->h[K], sizeof(float) * N, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) == cudaSuccess
               ? HD_OK
               : HD_ERR_CUDA;
}

hd_status hd_mlp_gradients(hd_mlp* M, const float* X, const float* t, int64_t N, float* loss, float* grads_host,
                           void* stream) {
    if (!M || !X || !t || N <= 0) return HD_ERR_INVALID;
    hd_status s = grad_impl(M, X, t, N, (cudaStream_t)stream);
    if (s != HD_OK) return s;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return HD_ERR_CUDA;
    if (loss && cudaMemcpy(loss, M->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return HD_ERR_CUDA;
    if (grads_host && cudaMemcpy(grads_host, M->g, sizeof(float) * M->np, cudaMemcpyDeviceToHost) != cudaSuccess)
        return HD_ERR_CUDA;
    return HD_OK;
}

hd_status hd_mlp_train_step(hd_mlp* M, const float* X, const float* t, int64_t N, float lr, float* loss, void* stream) {
    if (!M || !X || !t || N <= 0 || !(lr > 0)) return HD_ERR_INVALID;
    hd_status s = grad_impl(M, X, t, N, (cudaStream_t)stream);
    if (s != HD_OK) return s;
    M->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)M->step), c2 = 1.0f - std::pow(b2, (float)M->step);
    k_adam<<<blocks(M->np), 256, 0, (cudaStream_t)stream>>>(M->p, M->g, M->m, M->v, M->np, lr, b1, b2, 1e-8f, c1, c2);
    if (cudaGetLastError() != cudaSuccess) return HD_ERR_CUDA;
    if (loss) {
        if (cudaMemcpyAsync(loss, M->loss, sizeof(float), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
            return HD_ERR_CUDA;
        if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return HD_ERR_CUDA;
    }
    return HD_OK;
}

hd_status hd_mlp_destroy(hd_mlp* M) {
    if (!M) return HD_OK;
    cudaFree(M->p);
    cudaFree(M->g);
    cudaFree(M->m);
    cudaFree(M->v);
    for (float* q : M->z) cudaFree(q);
    for (size_t l = 1; l < M->h.size(); ++l) cudaFree(M->h[l]);
    cudaFree(M->delta0);
    cudaFree(M->delta1);
    cudaFree(M->loss);
    cudaGetLastError();
    delete M;
    return HD_OK;
}

}  // extern "C"
