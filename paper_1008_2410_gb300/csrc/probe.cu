// probe.cu -- throughput probes of the execution units the FMM kernels are bound by (FP32 FMA, FP64 FMA,
// SFU ex2/rcp, the tensor core's TF32 MMA issue rate), so that roofline fractions of the near field and sweep kernels can be quoted against
// measured rather than nominal rates. Each probe runs independent dependency chains in every thread of a
// grid that fills the GPU and is timed with CUDA events.
#include <cstdio>
#include <vector>

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

// Issue rate of tcgen05.mma kind::tf32 (M = 128, K = 8, operands zero in shared memory) at a given N: one CTA per
// SM, its first thread issues nmma MMAs into one accumulator, commits them and waits (bounded); out[cta] = the
// clock cycles from the first issue to the commit's completion, 0 on a timeout.
__device__ __forceinline__ uint32_t probe_smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__global__ void __launch_bounds__(128, 1) k_probe_tf32_mma(int N, int nmma, unsigned long long *out)
{
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tbase;
    for (int i = threadIdx.x; i < (40 << 10) / 16; i += blockDim.x)  // A: 128 x 8 at 0, B: up to 256 x 8 at 32 KB
        reinterpret_cast<float4 *>(sm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(probe_smem_u32(&tbase)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(probe_smem_u32(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;
    if (threadIdx.x == 0) {
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | (8u << 24);
        const uint32_t a0 = probe_smem_u32(sm), b0 = probe_smem_u32(sm + (32 << 10));
        // K-major, no swizzle: K-adjacent core matrices 128 B apart, 8-row groups 256 B apart; version 1 at bit 46
        const uint64_t ad = (uint64_t)((a0 >> 4) & 0x3fff) | ((uint64_t)8 << 16) | ((uint64_t)16 << 32) | ((uint64_t)1 << 46);
        const uint64_t bd = (uint64_t)((b0 >> 4) & 0x3fff) | ((uint64_t)8 << 16) | ((uint64_t)16 << 32) | ((uint64_t)1 << 46);
        unsigned long long t0, t1;
        asm volatile("mov.u64 %0, %%clock64;" : "=l"(t0));
        for (int i = 0; i < nmma; ++i)
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                         "l"(ad), "l"(bd), "r"(idesc), "r"(i > 0 ? 1u : 0u));
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(probe_smem_u32(&bar))
                     : "memory");
        uint32_t ok = 0;
        for (int it = 0; it < (1 << 22) && !ok; ++it)
            asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                         : "=r"(ok)
                         : "r"(probe_smem_u32(&bar))
                         : "memory");
        asm volatile("mov.u64 %0, %%clock64;" : "=l"(t1));
        out[blockIdx.x] = ok ? t1 - t0 : 0ull;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
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
    if (cap >= 6) {  // cycles per tcgen05.mma kind::tf32 (M = 128, K = 8) at N = 48 and N = 256, the slowest SM
        const int nmma = 480, smem = 40 << 10;
        cudaFuncSetAttribute(k_probe_tf32_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        unsigned long long *cyc = (unsigned long long *)buf;
        std::vector<unsigned long long> h(sms);
        for (int k = 0; k < 2; ++k) {
            k_probe_tf32_mma<<<sms, 128, smem>>>(k == 0 ? 48 : 256, nmma, cyc);
            unsigned long long mx = 0;
            if (cudaMemcpy(h.data(), cyc, sms * sizeof(unsigned long long), cudaMemcpyDeviceToHost) == cudaSuccess)
                for (unsigned long long c : h)
                    mx = c > mx ? c : mx;
            out[4 + k] = (double)mx / nmma;
        }
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return e == cudaSuccess ? FMM_OK : FMM_ECUDA;
}
