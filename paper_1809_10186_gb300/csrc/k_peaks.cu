// Device-rate probes for the rooflines (the paper has no counterpart): the FP32 and FP64 fused
// multiply-add throughput of the CUDA cores, measured with independent FMA chains on every SM
// and timed with CUDA events; and the issue-to-completion cycles of back-to-back tcgen05 MMAs of
// the shapes the translate kernels use. They change no device setting.
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "launchers.h"
#include "tc_ptx.cuh"

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

// One CTA per SM: the elected lane of warp 0 issues `iters` tcgen05.mma.kind::f16 (M = 128, K = 16,
// N = n, FP32 accumulator in TMEM, fp16 operands that are zero) back to back into one accumulator,
// commits, and waits (bounded) for their completion; cycles[blockIdx.x] = clock64 difference, or
// -1 when the wait gave up. A comes from shared memory (MN-major, no swizzle: the layout of the
// translate kernels' pass-2/3 operands) or from TMEM (their pass-1 operand); B from shared memory
// (K-major).
constexpr int kMmaSmem = 32768;   // A at [0, 16 KB), B at [16 KB, 32 KB)
__global__ void __launch_bounds__(128, 1) k_mma_probe(int n, int a_tmem, int iters, long long* __restrict__ cycles) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tmem;
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kMmaSmem / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(smem)[i] = 0u;
    if (warp == 0) {
        if (threadIdx.x == 0) {
            tc::mbar_init(&bar, 1);
            tc::fence_mbar_init();
        }
        __syncwarp();
        tc::tmem_alloc(&s_tmem, 512);
    }
    tc::fence_proxy_async();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (warp == 0) {
        const uint32_t sb = tc::smem_u32(smem);
        // MN-major A (8-row groups 128 B apart, 8-column K groups 2 KB apart), K-major B (K groups
        // 128 B apart, 8-row groups 256 B apart); D at TMEM column 0, a TMEM A operand at column 256
        const uint64_t da = tc::sdesc_at(tc::sdesc_base(2048, 128), sb >> 4);
        const uint64_t db = tc::sdesc_at(tc::sdesc_base(128, 256), (sb + 16384) >> 4);
        const uint32_t idesc = tc::idesc_f16(false, !a_tmem, false, n, 128);
        // (the operand values do not matter: the accumulator is never read)
        const long long t0 = clock64();
        for (int i = 0; i < iters; ++i) {
            if (a_tmem) tc::mma_ts_warp(tmem, tmem + 256, db, idesc, 1);
            else tc::mma_ss_warp(tmem, da, db, idesc, 1);
        }
        tc::mma_commit_warp(&bar);
        const bool ok = tc::mbar_wait(&bar, 0);
        const long long t1 = clock64();
        if (threadIdx.x == 0) cycles[blockIdx.x] = ok ? t1 - t0 : -1;
        __syncwarp();
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

}  // namespace

cudaError_t measure_mma_cycles(int n, int a_tmem, double& cycles_per_mma) {
    if (n < 16 || n > 256 || n % 16) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // 120 KB of dynamic shared memory keeps one probe CTA per SM (its TMEM allocation takes them all)
    const int smem = 120 * 1024, iters = 4096;
    e = cudaFuncSetAttribute(k_mma_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    long long* d = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d, sizeof(long long) * sms);
    long long worst = 0;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // rep 0 warms up
        k_mma_probe<<<sms, 128, smem>>>(n, a_tmem, iters, d);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        std::vector<long long> h((size_t)sms);
        if (e == cudaSuccess) e = cudaMemcpy(h.data(), d, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
        worst = 0;
        for (long long c : h) {
            if (c < 0) e = cudaErrorTimeout;
            worst = c > worst ? c : worst;
        }
    }
    if (d) cudaFree(d);
    if (e == cudaSuccess) cycles_per_mma = (double)worst / iters;
    return e;
}

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
