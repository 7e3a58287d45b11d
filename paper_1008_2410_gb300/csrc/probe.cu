// probe.cu -- throughput probes of the execution units the FMM kernels are bound by (FP32 FMA, FP64 FMA,
// SFU ex2/rcp), so that roofline fractions of the near field and sweep kernels can be quoted against
// measured rather than nominal rates. Each probe runs independent dependency chains in every thread of a
// grid that fills the GPU and is timed with CUDA events.
#include <cstdio>

#include "fmm2d.h"
#include "fmm_internal.cuh"

namespace {

constexpr int CHAINS = 8;

__global__ void k_probe_ffma(float *out, int iters, float a, float b)
{
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c)
        x[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c)
            x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c)
        s += x[c];
    if (s == 1.2345f)
        out[blockIdx.x] = s;
}

__global__ void k_probe_dfma(double *out, int iters, double a, double b)
{
    double x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c)
        x[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c)
            x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c)
        s += x[c];
    if (s == 1.2345)
        out[blockIdx.x] = s;
}

__global__ void k_probe_mufu(float *out, int iters)
{
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c)
        x[c] = -1e-3f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(-y));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c)
        s += x[c];
    if (s == 1.2345f)
        out[blockIdx.x] = s;
}

}  // namespace

extern "C" fmm_status fmm_probe_peaks(double *out, int cap)
{
    if (!out || cap < 4)
        return FMM_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
        return FMM_ECUDA;
    void *buf = nullptr;
    if (cudaMalloc(&buf, 1 << 20) != cudaSuccess)
        return FMM_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int threads = 256, blocks = sms * 8;
    const double lanes = (double)threads * blocks * CHAINS;
    auto timeit = [&](auto launch, int iters) {
        launch(iters / 8);  // warm-up
        cudaEventRecord(e0);
        launch(iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return (double)ms * 1e-3;
    };
    int it = 4096;
    double t = timeit([&](int n) { k_probe_ffma<<<blocks, threads>>>((float *)buf, n, 0.999f, 1e-3f); }, it);
    out[0] = 2.0 * lanes * it / t / 1e12;  // FP32 TFLOP/s (FMA = 2 flops)
    it = 256;
    t = timeit([&](int n) { k_probe_dfma<<<blocks, threads>>>((double *)buf, n, 0.999, 1e-3); }, it);
    out[1] = 2.0 * lanes * it / t / 1e12;  // FP64 TFLOP/s
    it = 1024;
    t = timeit([&](int n) { k_probe_mufu<<<blocks, threads>>>((float *)buf, n); }, it);
    out[2] = 2.0 * lanes * it / t / 1e12;  // SFU results per second, 1e12 (ex2 + rcp)
    out[3] = (double)sms;
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return e == cudaSuccess ? FMM_OK : FMM_ECUDA;
}
