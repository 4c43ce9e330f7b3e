// Arithmetic pipe peaks of the current GPU, measured with CUDA events: the
// denominators of the rooflines the filter's kernels are quoted against.
// The filter is bound by arithmetic, not by HBM (it moves 13-17 bytes per
// pixel), and the figures a vendor states for these pipes are unit counts
// times a clock that the GPU may not hold; so they are measured here.
//
// Each kernel runs kChains independent dependency chains per thread (enough
// instruction-level parallelism to keep its pipe busy) on a grid of
// kBlocksPerSm x 256-thread CTAs per SM, for a fixed number of iterations.
// A result that depends on every chain is written only under a condition
// that never holds, so the compiler keeps all the arithmetic.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fabf.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;
constexpr int kChains = 8;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// cycles[0], cycles[1]: SM clock cycles and global-timer nanoseconds that
// CTA 0's thread 0 spent in its loop (their ratio is the SM clock).
__global__ void __launch_bounds__(kThreads) dfma_loop(double a0, double b, int iters, double* sink,
                                                      unsigned long long* cycles)
{
    double x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = a0 + 1e-3 * (threadIdx.x + j);
    const unsigned long long g0 = global_ns();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], b, -0.25);   // |x| stays bounded for |b| < 1
    }
    const long long t1 = clock64();
    const unsigned long long g1 = global_ns();
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc += x[j];
    if (acc == 1234.5678) sink[threadIdx.x] = acc;
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        cycles[0] = (unsigned long long)(t1 - t0);
        cycles[1] = g1 - g0;
    }
}

__global__ void __launch_bounds__(kThreads) ffma_loop(float a0, float b, int iters, float* sink)
{
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = a0 + 1e-3f * (threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], b, -0.25f);
    }
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc += x[j];
    if (acc == 1234.5678f) sink[threadIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) imad_loop(uint32_t a0, uint32_t b, int iters, uint32_t* sink)
{
    uint32_t x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = a0 + threadIdx.x + 977u * j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = x[j] * b + 0x9E3779B9u;
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc ^= x[j];
    if (acc == 0x12345679u && a0 == 7u) sink[threadIdx.x] = acc;
}

// MUFU: the base-2 exponential approximation, one per chain per iteration.
__device__ __forceinline__ float ex2_approx(float v)
{
    float r;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__global__ void __launch_bounds__(kThreads) mufu_loop(float a0, int iters, float* sink)
{
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = a0 - 1e-3f * (threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = -ex2_approx(x[j]);   // stays in [-1, -0.5]
    }
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc += x[j];
    if (acc == 1234.5678f) sink[threadIdx.x] = acc;
}

template <typename Launch>
cudaError_t time_best(Launch&& launch, int reps, float* best_ms)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    float best = 1e30f;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {   // run 0 is the warm-up
        e = cudaEventRecord(e0, 0);
        launch();
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best_ms = best;
    return e;
}

}  // namespace

extern "C" int fabf_pipe_peaks(double* out)
{
    if (!out) return FABF_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return FABF_ECUDA;
    }
    void* sink = nullptr;
    if (cudaMalloc(&sink, kThreads * sizeof(double) + 256) != cudaSuccess) {
        (void)cudaGetLastError();
        return FABF_ENOMEM;
    }
    unsigned long long* d_cycles = reinterpret_cast<unsigned long long*>(static_cast<char*>(sink) +
                                                                           kThreads * sizeof(double));
    const int blocks = sms * kBlocksPerSm;
    const double threads = (double)blocks * kThreads;
    // iteration counts sized for launches of a few milliseconds each
    const int it64 = 2000, it32 = 100000, itmu = 20000;
    float ms64 = 0, ms32 = 0, msi = 0, msm = 0;
    cudaError_t e = time_best([&] { dfma_loop<<<blocks, kThreads>>>(0.5, 0.75, it64, (double*)sink, d_cycles); },
                              3, &ms64);
    unsigned long long cyc[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(cyc, d_cycles, sizeof(cyc), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = time_best([&] { ffma_loop<<<blocks, kThreads>>>(0.5f, 0.75f, it32, (float*)sink); }, 3, &ms32);
    if (e == cudaSuccess)
        e = time_best([&] { imad_loop<<<blocks, kThreads>>>(3u, 0x01000193u, it32, (uint32_t*)sink); }, 3, &msi);
    if (e == cudaSuccess)
        e = time_best([&] { mufu_loop<<<blocks, kThreads>>>(-0.75f, itmu, (float*)sink); }, 3, &msm);
    cudaFree(sink);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return FABF_ECUDA;
    }
    const double ops64 = threads * kChains * it64, ops32 = threads * kChains * it32, opsm = threads * kChains * itmu;
    out[0] = 2.0 * ops64 / (ms64 * 1e-3) / 1e12;   // FP64 FMA, TFLOP/s (FMA = 2 flops)
    out[1] = 2.0 * ops32 / (ms32 * 1e-3) / 1e12;   // FP32 FMA, TFLOP/s
    out[2] = ops32 / (msi * 1e-3) / 1e12;          // INT32 multiply-add, T ops/s
    out[3] = opsm / (msm * 1e-3) / 1e12;           // MUFU ex2, T ops/s
    // SM clock during the FP64 run: one CTA's clock64 cycles over the
    // global-timer nanoseconds of the same interval
    out[4] = cyc[1] > 0 ? (double)cyc[0] / (double)cyc[1] * 1e3 : 0.0;
    out[5] = (double)sms;
    return FABF_OK;
}
