// Device-rate probe for the rooflines (the paper has no counterpart): the FP32 and FP64 fused
// multiply-add throughput of the CUDA cores, measured with independent FMA chains on every SM
// and timed with CUDA events. It changes no device setting.
#include <cuda_runtime.h>

#include "launchers.h"

namespace dgfs {

namespace {

constexpr int kChains = 8;      // independent dependency chains per thread
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(T* __restrict__ sink, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == T(-1)) sink[blockIdx.x] = s;   // never true for these inputs; keeps the chains live
}

template <typename T>
cudaError_t time_probe(int blocks, int iters, double& tflops) {
    T* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(T) * blocks);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    // a = 1 - 2^-20 and b = 2^-20 keep every chain bounded near 1
    const T a = T(1) - T(1.0 / 1048576.0), b = T(1.0 / 1048576.0);
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // rep 0 warms up
        cudaEventRecord(e0);
        k_fma_probe<T><<<blocks, kThreads>>>(sink, iters, a, b);
        cudaEventRecord(e1);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e == cudaSuccess)
        tflops = 2.0 * kChains * (double)iters * kThreads * blocks / (best * 1e-3) / 1e12;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    return e;
}

}  // namespace

cudaError_t measure_fma_peaks(double& fp32_tflops, double& fp64_tflops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // eight 256-thread blocks per SM; FP64 runs far fewer iterations (its rate is far lower)
    e = time_probe<float>(8 * sms, 1 << 15, fp32_tflops);
    if (e == cudaSuccess) e = time_probe<double>(8 * sms, 1 << 10, fp64_tflops);
    return e;
}

}  // namespace dgfs
