// hd_peaks.cu -- arithmetic peak microbenchmark of the current GPU (no
// counterpart in the paper).  The FFT kernels run on the CUDA cores (FP32 or
// FP64 fused multiply-adds, no tensor cores), so their roofline is the
// measured FMA throughput of the device, taken here by kernels of the
// library's own: every thread runs independent chains of dependent FMAs
// (enough chains to cover the pipeline latency), many CTAs per SM.
#include <cuda_runtime.h>

#include <cstdint>

#include "hd_plan.h"

namespace {

constexpr int kChains = 8;

template <class R>
__global__ void __launch_bounds__(256) k_fma_chains(R* out, int iters, R b, R c) {
    R a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = R(threadIdx.x) * R(1e-3) + R(i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = a[i] * b + c;   // contracted to one FMA
    }
    R s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// the packed two-lane FP32 FMA of sm_100 and later (fma.rn.f32x2): half the
// issue slots of scalar FMAs for the same work
__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a, unsigned long long b,
                                                       unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__global__ void __launch_bounds__(256) k_fma_chains_x2(float* out, int iters, float b, float c) {
    unsigned long long a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        const float x = threadIdx.x * 1e-3f + i;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[i]) : "f"(x), "f"(x + 0.5f));
    }
    unsigned long long bb, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fma_f32x2(a[i], bb, cc);
    }
    float s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        float x, y;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[i]));
        s += x + y;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" hd_status hd_alu_peak(int kind, double* tflops) {
    if (!tflops || kind < 0 || kind > 2) return HD_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    const int threads = 256, blocks = sms * 8;
    const int iters = kind == HD_F64 ? 2048 : 16384;   // a few milliseconds per launch
    void* out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_NOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&]() {
        if (kind == HD_F64)
            k_fma_chains<double><<<blocks, threads>>>(static_cast<double*>(out), iters, 0.999, 1e-3);
        else if (kind == HD_F32)
            k_fma_chains<float><<<blocks, threads>>>(static_cast<float*>(out), iters, 0.999f, 1e-3f);
        else
            k_fma_chains_x2<<<blocks, threads>>>(static_cast<float*>(out), iters, 0.999f, 1e-3f);
    };
    const int reps = 5;
    launch();
    cudaEventRecord(e0);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || ms <= 0) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    const double lanes = kind == 2 ? 2.0 : 1.0;   // values per FMA instruction
    const double flops = 2.0 * lanes * kChains * (double)iters * blocks * threads * reps;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return HD_OK;
}
