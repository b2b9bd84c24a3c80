// Roofline denominators measured on the running GPU: sustained rates of the
// MUFU sin/cos path (XU pipe), FP32 and FP64 fused multiply-add, and the SM
// clock seen while they run.  Each kernel keeps 8 independent dependency
// chains per thread over a grid of 8 blocks per SM, so the pipes, not the
// latencies, bound the rate.  Not part of the force path.
#include <cuda_runtime.h>

#include "../../include/rbsog.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kThreads) k_peak_mufu(int iters, float seed, float *out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = seed + 0.001f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float s, co;
            __sincosf(x[c], &s, &co);
            x[c] = s + co;
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += x[c];
    if (acc == 12345.678f) out[0] = acc;   // keeps the chains alive
}

__global__ void __launch_bounds__(kThreads) k_peak_fma32(int iters, float seed, float *out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = seed + 0.001f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], 0.999999f, 1e-7f);
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += x[c];
    if (acc == 12345.678f) out[0] = acc;
}

__global__ void __launch_bounds__(kThreads) k_peak_fma64(int iters, double seed, double *out) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = seed + 0.001 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], 0.999999999, 1e-9);
    }
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += x[c];
    if (acc == 12345.678) out[0] = acc;
}

// SM cycles and nanoseconds elapsed over a fixed busy loop (clock64 vs the
// global nanosecond timer) give the SM clock.
__global__ void k_clock(int iters, long long *out) {
    long long c0 = clock64();
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    float x = 1.0f;
    // empty volatile asm statements tie the loop between the timer reads
    // (volatile asm is not reordered against volatile asm)
    asm volatile("" : "+f"(x));
    for (int i = 0; i < iters; ++i) x = fmaf(x, 0.9999f, 1e-4f);
    asm volatile("" : "+f"(x));
    long long c1 = clock64();
    unsigned long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (threadIdx.x == 0) {
        out[0] = c1 - c0;
        out[1] = (long long)(t1 - t0);
        if (x == 12345.f) out[2] = 1;
    }
}

}  // namespace

extern "C" rbsog_status rbsog_measure_peaks(int device, double *out) {
    if (!out) return RBSOG_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return RBSOG_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return RBSOG_ECUDA;
    const int blocks = prop.multiProcessorCount * 8;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return RBSOG_ECUDA;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double *dsink = nullptr;
    long long *clk = nullptr;
    rbsog_status status = RBSOG_OK;
    if (cudaMalloc(&dsink, 64) != cudaSuccess || cudaMalloc(&clk, 64) != cudaSuccess) status = RBSOG_ENOMEM;
    auto timed = [&](auto launch, double ops) -> double {
        launch();   // warm-up
        cudaEventRecord(a, st);
        launch();
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        return ops / (ms * 1e-3);
    };
    if (status == RBSOG_OK) {
        const double threads = (double)blocks * kThreads;
        const int im = 2048, i32 = 8192, i64 = 256;
        out[0] = timed([&] { k_peak_mufu<<<blocks, kThreads, 0, st>>>(im, 0.5f, (float *)dsink); },
                       threads * im * kChains * 2.0);
        out[1] = timed([&] { k_peak_fma32<<<blocks, kThreads, 0, st>>>(i32, 0.5f, (float *)dsink); },
                       threads * i32 * kChains);
        out[2] = timed([&] { k_peak_fma64<<<blocks, kThreads, 0, st>>>(i64, 0.5, dsink); },
                       threads * i64 * kChains);
        k_clock<<<prop.multiProcessorCount, 32, 0, st>>>(1 << 20, clk);
        long long h[3] = {0, 0, 0};
        if (cudaMemcpyAsync(h, clk, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            status = RBSOG_ECUDA;
        out[3] = h[1] > 0 ? (double)h[0] / (double)h[1] * 1e3 : 0.0;   // MHz
        out[4] = (double)prop.multiProcessorCount;
    }
    if (cudaGetLastError() != cudaSuccess && status == RBSOG_OK) status = RBSOG_ECUDA;
    cudaFree(dsink);
    cudaFree(clk);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(st);
    return status;
}
