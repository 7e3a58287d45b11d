// m2l_tc.cu -- Fig. 1 stage 6 (M2L, §3) of the precision form on the tensor cores (tcgen05, TMEM).
//
// With radius-scaled coefficients the translation from a source box at offset delta = (dx, dy) box widths
// (a Gaussian integer, max(|dx|, |dy|) in {2, 3}) is the same at every level and factors as
//     b^_l += rho^(l+1) sum_m B[l][m] (rho^m a~_m),   B[l][m] = (-1)^(m+1) C(m+l, m),   rho = 1/delta,
// so the only dense contraction is with the real matrix B, shared by every offset and level. A CTA owns up to
// 128 target boxes of one level, one system and one child position (cx, cy) -- boxes that share their 27
// interaction offsets (children of the parent's neighbours that are not adjacent) -- and walks those offsets.
// Per offset it gathers the 128 source multipoles (zero for sources outside the domain or empty), scales them
// by rho^m (CUDA cores), splits the real and the imaginary parts into two TF32 values each (hi, lo) and issues
//     D_re = A_re B^T,  D_im = A_im B^T   as hi*hi + hi*lo + lo*hi (3xTF32)
// with tcgen05.mma, accumulators in tensor memory. B (hi and lo, built on the host in FP64) is loaded once.
// Each offset gets fresh accumulators (two stages alternate); they are read back with tcgen05.ld, multiplied by
// rho^(l+1) and summed over the 27 offsets in FP32 registers. A single accumulator over all offsets measured
// 7.7e-6 relative error against 3.8e-7 with the per-offset read-back: long accumulation chains inside the
// tensor core lose accuracy.
//
// Each target row is shared by KP / 8 threads, 8 coefficients each, so that the per-offset CUDA-core work
// (gather, scaling, split, read-back) is spread over 4 KP / 8 warps per CTA.
//
// Pipeline (two shared-memory stages s = q & 1 for offset q): the loads of offset q + 1 are issued first;
// then wait for the MMAs of offset q - 2 (stage s), read their accumulators, stage A(q) into s; after a
// barrier one thread issues the MMAs of offset q and commits them to mma_bar[s]. Every wait is bounded: on a
// timeout the CTA sets FMM_DEV_TIMEOUT, lets its MMAs in flight finish (bounded), frees its tensor memory and
// returns without writing.
#include <cstring>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kRows = 128;  // MMA M: target boxes per CTA
constexpr int kNOff = 27;   // interaction offsets per child position

template <int PB>
struct TcShape {
    static constexpr int KP = PB;                    // K: coefficient index m (PB a multiple of 8)
    static constexpr int NP = (PB + 15) / 16 * 16;   // N: output index l, padded to the M = 128 rule
    static constexpr int A_PART = kRows * KP * 4;    // one of re-hi, re-lo, im-hi, im-lo
    static constexpr int B_PART = NP * KP * 4;       // one TF32 part of B
    static constexpr int STAGE_A = 4 * A_PART;
    static constexpr int B_BYTES = 2 * B_PART;
    static constexpr int RHO_BYTES = kNOff * (PB + 1) * 8;  // rho^k, k = 0 .. PB, of the CTA's 27 offsets
    static constexpr int SMEM = 2 * STAGE_A + B_BYTES + RHO_BYTES;
    // accumulators: stage s, part (re 0, im 1) at column (2 s + part) NP; 4 NP columns (a power of two), at
    // most 512 per SM for any number of CTAs that fit in shared memory
    static constexpr int COLS = 4 * NP;
    // G = KP / 8 threads per target row, each owning 8 coefficients (m on input, l on output); warp w holds
    // rows 32 (w % 4) .. + 31 (the tensor-memory lanes it may read) and coefficients 8 (w / 4) .. + 7
    static constexpr int G = KP / 8;
    static constexpr int THREADS = kRows * G;
    static constexpr int MIN_BLOCKS = PB <= 16 ? 3 : PB <= 24 ? 2 : 1;  // as many as shared memory admits
};

// Byte offset of element (row, k) in the K-major, non-swizzled operand layout: 8-row x 16-byte core matrices,
// K-adjacent core matrices 128 bytes apart (leading-dimension offset), 8-row groups KP/4 * 128 bytes apart
// (stride-dimension offset).
__host__ __device__ inline int core_off(int row, int k, int KP)
{
    return ((row >> 3) * (KP >> 2) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start, leading and stride byte offsets (16-byte units),
// descriptor version 1 at bit 46, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 20); ++it)
        if (mbar_try(bar, parity))
            return true;
    return false;
}
__device__ __forceinline__ float tf32_rn(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// Adds rho^(l+1) (D_re[l] + i D_im[l]) for this thread's 8 output coefficients l = l0 + j (those < p) of its
// row into (ar, ai); taddr_* point at column l0 of the stage's two accumulators.
__device__ __forceinline__ void accumulate_tmem(uint32_t taddr_re, uint32_t taddr_im, const float2 *rho, int l0,
                                                int p, float *ar, float *ai)
{
    uint32_t re[8], im[8];
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem_ld8(taddr_re, re);
    tmem_ld8(taddr_im, im);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (l0 + j < p) {
            const float2 r = rho[l0 + j + 1];
            const float dr = __uint_as_float(re[j]), di = __uint_as_float(im[j]);
            ar[j] = fmaf(r.x, dr, fmaf(-r.y, di, ar[j]));
            ai[j] = fmaf(r.x, di, fmaf(r.y, dr, ai[j]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

template <int PB>
__global__ void __launch_bounds__(TcShape<PB>::THREADS, TcShape<PB>::MIN_BLOCKS) k_m2l_tc(Work w, const unsigned char *__restrict__ btab,
                                                    const float2 *__restrict__ rho32, int l32)
{
    using S = TcShape<PB>;
    constexpr int RS = 2 * FMM_PMAX + 2;  // row length of the rho^k table
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t mma_bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_bad;
    __shared__ int2 s_off[kNOff];
    unsigned char *sB = sm + 2 * S::STAGE_A;
    float2 *s_rho = reinterpret_cast<float2 *>(sB + S::B_BYTES);  // [kNOff][PB + 1]

    // work item -> (level l, system, child position, tile of 128 boxes of that position)
    int64_t g = blockIdx.x, tiles = 1;
    int l = l32;
    for (; l <= w.lv.maxdepth; ++l) {
        tiles = l >= 5 ? ((int64_t)1 << (2 * l - 9)) : 1;  // 4^(l-1) boxes per position, 128 per tile
        const int64_t cnt = (int64_t)w.lv.nsys_at[l] * 4 * tiles;
        if (g < cnt)
            break;
        g -= cnt;
    }
    if (l > w.lv.maxdepth)
        return;  // block-uniform
    const int sidx = (int)(g / (4 * tiles));
    const int64_t rem = g - (int64_t)sidx * 4 * tiles;
    const int cls = (int)(rem / tiles);
    const int64_t tile = rem - (int64_t)cls * tiles;
    const SysDev &d = w.sys[sys_at_level(w, l, sidx)];
    const int tid = threadIdx.x, warp = tid >> 5, p = w.p;
    const int row = 32 * (warp & 3) + (tid & 31), m0 = 8 * (warp >> 2);  // this thread's row and coefficients
    const int cx = cls & 1, cy = cls >> 1, ns = 1 << l, nh = ns >> 1;
    const int64_t ib = tile * kRows + row;  // this row's index among the boxes of the child position
    const bool row_ok = ib < (int64_t)nh * nh;
    const int bx = 2 * (int)(ib & (nh - 1)) + cx, by = 2 * (int)(ib >> (l - 1)) + cy;
    const int64_t lev0 = d.box0[l];

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(S::COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        int q = 0;
        for (int ry = -2 - cy; ry <= 3 - cy; ++ry)
            for (int rx = -2 - cx; rx <= 3 - cx; ++rx)
                if (rx < -1 || rx > 1 || ry < -1 || ry > 1)
                    s_off[q++] = make_int2(rx, ry);
        s_bad = 0;
        for (int i = 0; i < 2; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_bar[i])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B (hi, lo) once; 16-byte pieces
    for (int i = tid; i < S::B_BYTES / 16; i += blockDim.x)
        reinterpret_cast<float4 *>(sB)[i] = reinterpret_cast<const float4 *>(btab)[i];
    __syncthreads();  // s_off ready
    for (int i = tid; i < kNOff * (PB + 1); i += blockDim.x) {
        const int q = i / (PB + 1), k = i - q * (PB + 1);
        const int2 o = s_off[q];
        s_rho[i] = rho32[((o.y + 3) * 7 + (o.x + 3)) * RS + k];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B visible to the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t tlane = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + m0;  // this warp's lanes, column m0
    // instruction descriptor: D f32, A and B tf32, both K-major, N = NP, M = 128
    const uint32_t idesc =
        (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(S::NP >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);

    auto gather = [&](int q, float2 *r) {
        const int2 o = s_off[q];
        const int jx = bx + o.x, jy = by + o.y;
        bool v = row_ok && jx >= 0 && jy >= 0 && jx < ns && jy < ns;
        const int64_t sb = lev0 + (int64_t)jy * ns + jx;
        v = v && w.bcount[sb] != 0;
        const float2 *src = w.M32 + sb * p + m0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            r[j] = (v && m0 + j < p) ? src[j] : make_float2(0.f, 0.f);
    };

    float ar[8], ai[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        ar[j] = 0.f;
        ai[j] = 0.f;
    }
    float2 nxt[8];
    gather(0, nxt);
    int committed = -1;  // (thread 0) last offset whose MMAs were committed
    for (int q = 0; q < kNOff; ++q) {
        const int s = q & 1;
        float2 cur[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            cur[j] = nxt[j];
        if (q + 1 < kNOff)
            gather(q + 1, nxt);  // loads in flight while this offset is staged
        if (q >= 2) {
            if (!__all_sync(0xffffffffu, mbar_wait(&mma_bar[s], ((q - 2) >> 1) & 1)))
                s_bad = 1;
            else
                accumulate_tmem(tlane + (2 * s) * S::NP, tlane + (2 * s + 1) * S::NP, s_rho + (q - 2) * (PB + 1),
                                m0, p, ar, ai);
        }
        // A(q): rho^m a~_m, real and imaginary parts, each split hi + lo
        unsigned char *sa = sm + s * S::STAGE_A;
        const float2 *rq = s_rho + q * (PB + 1);
#pragma unroll
        for (int c = 0; c < 2; ++c) {  // the thread's two 4-coefficient chunks
            float re[4], im[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 a = cur[4 * c + j], r = rq[m0 + 4 * c + j];
                re[j] = fmaf(r.x, a.x, -r.y * a.y);
                im[j] = fmaf(r.x, a.y, r.y * a.x);
            }
            const float4 rh = make_float4(tf32_rn(re[0]), tf32_rn(re[1]), tf32_rn(re[2]), tf32_rn(re[3]));
            const float4 rl = make_float4(tf32_rn(re[0] - rh.x), tf32_rn(re[1] - rh.y), tf32_rn(re[2] - rh.z),
                                          tf32_rn(re[3] - rh.w));
            const float4 ih = make_float4(tf32_rn(im[0]), tf32_rn(im[1]), tf32_rn(im[2]), tf32_rn(im[3]));
            const float4 il = make_float4(tf32_rn(im[0] - ih.x), tf32_rn(im[1] - ih.y), tf32_rn(im[2] - ih.z),
                                          tf32_rn(im[3] - ih.w));
            const int off = core_off(row, m0 + 4 * c, S::KP);
            *reinterpret_cast<float4 *>(sa + off) = rh;
            *reinterpret_cast<float4 *>(sa + S::A_PART + off) = rl;
            *reinterpret_cast<float4 *>(sa + 2 * S::A_PART + off) = ih;
            *reinterpret_cast<float4 *>(sa + 3 * S::A_PART + off) = il;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (s_bad)
            break;  // block-uniform: read after the barrier
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sB);
            const uint32_t lbo = 128, sbo = (S::KP / 4) * 128;
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const uint32_t d_acc = tmem + (2 * s + part) * S::NP;
                const uint32_t ap = a0 + 2 * part * S::A_PART;
#pragma unroll
                for (int ks = 0; ks < S::KP / 8; ++ks) {
                    const uint32_t ko = ks * 256;  // 8 TF32 of K = two core matrices
                    const uint64_t ah = sdesc(ap + ko, lbo, sbo), al = sdesc(ap + S::A_PART + ko, lbo, sbo);
                    const uint64_t bh = sdesc(b0 + ko, lbo, sbo), bl = sdesc(b0 + S::B_PART + ko, lbo, sbo);
                    mma_tf32(d_acc, ah, bh, idesc, ks > 0 ? 1u : 0u);
                    mma_tf32(d_acc, ah, bl, idesc, 1u);
                    mma_tf32(d_acc, al, bh, idesc, 1u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mma_bar[s]))
                         : "memory");
            committed = q;
        }
    }
    __syncthreads();
    bool ok = !s_bad;
    if (ok) {
        // offsets kNOff - 2 and kNOff - 1 are still in their accumulators
#pragma unroll
        for (int q = kNOff - 2; q < kNOff; ++q) {
            const int s = q & 1;
            const bool okq = __all_sync(0xffffffffu, mbar_wait(&mma_bar[s], (q >> 1) & 1));
            if (okq)
                accumulate_tmem(tlane + (2 * s) * S::NP, tlane + (2 * s + 1) * S::NP, s_rho + q * (PB + 1), m0, p,
                                ar, ai);
            ok = ok && okq;
        }
    }
    if (ok && row_ok) {
        float2 *dst = w.L32 + (lev0 + (int64_t)by * ns + bx) * p + m0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (m0 + j < p)
                dst[j] = make_float2(ar[j], ai[j]);
    }
    if (!ok && tid == 0) {
        atomicOr(w.status, FMM_DEV_TIMEOUT);
        if (committed >= 0)  // let the last MMAs land before the shared and tensor memory are released
            mbar_wait(&mma_bar[committed & 1], (committed >> 1) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::COLS));
}

template <int PB>
int set_smem_attr()
{
    return cudaFuncSetAttribute(k_m2l_tc<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<PB>::SMEM) ==
                   cudaSuccess
               ? 0
               : -1;
}

int bucket_of(int p) { return p <= 8 ? 8 : p <= 16 ? 16 : p <= 24 ? 24 : 32; }

bool g_tc_ready[64] = {};

}  // namespace

size_t m2l_tc_table_bytes(int p)
{
    switch (bucket_of(p)) {
    case 8:
        return TcShape<8>::B_BYTES;
    case 16:
        return TcShape<16>::B_BYTES;
    case 24:
        return TcShape<24>::B_BYTES;
    default:
        return TcShape<32>::B_BYTES;
    }
}

// TF32 value nearest to x (ties away from zero), the rounding of cvt.rna.tf32.f32.
static float tf32_round_host(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u + 0x1000u) & 0xffffe000u;
    memcpy(&f, &u, 4);
    return f;
}

// B[l][m] = (-1)^(m+1) C(m+l, m) for l, m < p (zero padding elsewhere), hi part then lo part, each [NP rows l]
// [KP columns m] in the operand layout.
void build_m2l_tc_table_host(int p, unsigned char *out)
{
    const int pb = bucket_of(p), KP = pb, NP = (pb + 15) / 16 * 16;
    const size_t part = (size_t)NP * KP * 4;
    memset(out, 0, 2 * part);
    for (int l = 0; l < p; ++l)
        for (int m = 0; m < p; ++m) {
            double c = 1.0;
            for (int i = 1; i <= m; ++i)
                c = c * (double)(l + i) / (double)i;  // C(m + l, m)
            const double v = (m & 1) ? c : -c;
            const float hi = tf32_round_host(v), lo = tf32_round_host(v - (double)hi);
            const int off = core_off(l, m, KP);
            memcpy(out + off, &hi, 4);
            memcpy(out + part + off, &lo, 4);
        }
}

int prepare_m2l_tc()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return -1;
    if (g_tc_ready[dev])
        return 0;
    if (set_smem_attr<8>() || set_smem_attr<16>() || set_smem_attr<24>() || set_smem_attr<32>())
        return -1;
    g_tc_ready[dev] = 1;
    return 0;
}

int64_t m2l_tc_items(const Work &w, int l32)
{
    int64_t n = 0;
    for (int l = l32; l <= w.lv.maxdepth; ++l) {
        const int64_t tiles = l >= 5 ? ((int64_t)1 << (2 * l - 9)) : 1;
        n += (int64_t)w.lv.nsys_at[l] * 4 * tiles;
    }
    return n;
}

int launch_m2l_tc(const Work &w, const Tables &t, int l32, cudaStream_t s)
{
    const int64_t items = m2l_tc_items(w, l32);
    if (items == 0)
        return 0;
    const unsigned blocks = (unsigned)items;
    switch (bucket_of(w.p)) {
    case 8:
        k_m2l_tc<8><<<blocks, TcShape<8>::THREADS, TcShape<8>::SMEM, s>>>(w, t.m2l_tc, t.rho32, l32);
        break;
    case 16:
        k_m2l_tc<16><<<blocks, TcShape<16>::THREADS, TcShape<16>::SMEM, s>>>(w, t.m2l_tc, t.rho32, l32);
        break;
    case 24:
        k_m2l_tc<24><<<blocks, TcShape<24>::THREADS, TcShape<24>::SMEM, s>>>(w, t.m2l_tc, t.rho32, l32);
        break;
    default:
        k_m2l_tc<32><<<blocks, TcShape<32>::THREADS, TcShape<32>::SMEM, s>>>(w, t.m2l_tc, t.rho32, l32);
        break;
    }
    return 1;
}

}  // namespace fmm
