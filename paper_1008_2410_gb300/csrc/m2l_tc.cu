// m2l_tc.cu -- Fig. 1 stage 6 (M2L, §3) of the precision form on the tensor cores (tcgen05, TMEM).
//
// With radius-scaled coefficients the translation from a source box at offset delta = (dx, dy) box widths
// (a Gaussian integer, max(|dx|, |dy|) in {2, 3}) is the same matrix at every level:
//     b^_l += sum_m T[l][m] a~_m,   T[l][m] = (-1)^(m+1) C(m + l, m) rho^(m+l+1),   rho = 1 / delta.
// Over the reals, with real and imaginary parts interleaved (input k = 2m + {0, 1}, output n = 2l + {0, 1}),
// each of the 40 offsets is one 2p x 2p real matrix B_delta; the host builds them in FP64 and stores every
// entry as a TF32 pair (hi, lo). A translation is a row of A (a source box's 2p numbers, split hi + lo as well)
// times B_delta^T, evaluated as hi*hi + hi*lo + lo*hi (3xTF32) by tcgen05.mma into tensor memory.
//
// The boxes of a level fall into four classes by child position c = (cx, cy). A box of class c at class
// coordinates (i, j) (its parent's coordinates) takes its 27 interaction-list sources from the children of the
// parent's 3 x 3 neighbours: boxes of class c' at class coordinates (i + ox, j + oy), ox, oy in {-1, 0, 1}.
// On a class grid whose rows carry one zero column at either end (row length Lc = 2^(l-1) + 2), the sources
// of 128 consecutive target positions q0 .. q0 + 127 at one offset are 128 consecutive positions, starting at
// (1 + oy) Lc + 1 + ox in the window [q0 - Lc - 1, q0 + Lc + 129) of class c'. A first kernel writes every
// level's multipoles in that form once per evaluation (per class, TF32 hi and lo planes of 16-byte K chunks, one
// position per chunk, zeros for padding and empty boxes); a CTA (128 target positions of one class) then takes
// each source class's window by bulk asynchronous copies (one contiguous run per plane), and every offset's A
// operand is a shared-memory descriptor into it (8-row core matrices 128 bytes apart, K planes one window
// apart). Per offset no CUDA-core work remains but reading the accumulator back.
//
// Per offset: the B pair arrives by a bulk copy into a ring of slots; one thread issues the 3 KP / 8 MMAs into
// one of two accumulators and commits them to an mbarrier; then the 128 threads (one per target position and
// tensor-memory lane) read the previous offset's accumulator and add it to their 2p registers, so the tensor
// core never accumulates over more than one offset. Two window buffers alternate: the copies of the source
// class after next start as soon as the MMAs of a class have completed. Every wait is bounded: on a timeout the
// CTA sets FMM_DEV_TIMEOUT, lets its MMAs and copies in flight land (bounded), frees its tensor memory and
// returns without writing.
//
// Levels whose class grid is wider than 64 boxes (their windows do not fit twice) and p > 20 take the CUDA-core
// kernel (sweep.cu).
#include <complex>
#include <cstring>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kRows = 128;        // MMA M: target positions per CTA
constexpr int kNOff = 27;         // interaction offsets per class
constexpr int kMaxClassWidth = 64;  // widest class grid (level 7) whose two windows fit in shared memory
constexpr int kPMaxTc = 20;
constexpr int kNDelta = 49;       // offset table index (dy + 3) * 7 + (dx + 3)
constexpr int kReplicas = 8;      // copies of the B table, CTA i reading copy i % 8: every CTA of a class streams the
                                  // same 27 matrices, and one copy would concentrate those reads on a few L2 slices

template <int PB>
struct TcShape {
    static constexpr int KP = (2 * PB + 7) / 8 * 8;     // K: 2p real inputs, padded to the MMA's K step
    static constexpr int NP = (2 * PB + 15) / 16 * 16;  // N: 2p real outputs, padded to the M = 128 rule
    static constexpr int KC = KP / 4;                   // 16-byte K chunks (window planes)
    static constexpr int NG = KP / 8;                   // 8-row groups of B that may hold nonzero rows
    static constexpr int B_PART = NP * KP * 4;          // one TF32 part of B_delta in the operand layout
    static constexpr int B_LOAD = NG * KC * 128;        // bytes of a part that are copied (the rest is zero)
    static constexpr int B_SLOT = 2 * B_PART;
    static constexpr int NSLOT = 3;
    static constexpr int RD = KP / 8;                   // 8-column read-backs per offset
};

// Window length: the 2 Lc + 130 positions a tile reads.
__host__ __device__ inline int window_len(int Lc) { return 2 * Lc + 130; }

template <int PB>
constexpr size_t smem_bytes(int ws)
{
    using S = TcShape<PB>;
    return 2 * (size_t)(2 * S::KC * ws * 16) + (size_t)S::NSLOT * S::B_SLOT;
}

// Byte offset of element (row, k) in the K-major, non-swizzled operand layout of B: 8-row x 16-byte core
// matrices, K-adjacent core matrices 128 bytes apart (leading-dimension offset), 8-row groups KP/4 * 128 bytes
// apart (stride-dimension offset).
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
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// plain (non-multicast) bulk copy from this GPU's global memory into this CTA's shared memory
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
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
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Window source layout, built per evaluation by k_m2l_tc_layout: for every level l <= 7 (from level 2), system
// at l and class c', 2 (hi, lo) x KC planes of NPOS(l) 16-byte chunks; chunk P of plane kc holds coefficients
// m = 2 kc, 2 kc + 1 (re, im each) of the box at padded position qq = P - Lc - 1 (row qq / Lc, column qq % Lc - 1)
// of the class grid, or zeros (outside the grid, padding column, empty box, m >= p). A tile's window is then one
// contiguous run of 2 Lc + 130 chunks per plane, starting at P = q0.
__host__ __device__ inline int npos_of(int l)
{
    const int nc = 1 << (l - 1), Lc = nc + 2;
    return (nc + 2) * Lc + 130;
}
// float4 offset of the planes of (level l, system index sidx at l, class c)
__host__ __device__ inline int64_t layout_base(const LevelInfo &lv, int KC, int l, int sidx, int c)
{
    int64_t b = 0;
    for (int k = 2; k < l; ++k)
        b += (int64_t)lv.nsys_at[k] * 8 * KC * npos_of(k);
    return b + (int64_t)(sidx * 4 + c) * 2 * KC * npos_of(l);
}

// Block (plane (level, system, class, K chunk), run of 256 positions), nch runs per plane; a thread writes
// position P's hi and lo chunks.
template <int PB>
__global__ void __launch_bounds__(256) k_m2l_tc_layout(Work w, int l_lo, int l_hi, int nch)
{
    using S = TcShape<PB>;
    int64_t g = blockIdx.x / nch;
    const int run = (int)(blockIdx.x % nch);
    int l = l_lo;
    for (; l <= l_hi; ++l) {
        const int64_t cnt = (int64_t)w.lv.nsys_at[l] * 4 * S::KC;
        if (g < cnt)
            break;
        g -= cnt;
    }
    if (l > l_hi)
        return;  // block-uniform
    const int kc = (int)(g % S::KC), r = (int)(g / S::KC), c = r & 3, sidx = r >> 2;
    const SysDev &d = w.sys[sys_at_level(w, l, sidx)];
    const int p = w.p, ns = 1 << l, nc = ns >> 1, Lc = nc + 2, np_ = npos_of(l);
    const int m0 = 2 * kc, m1 = 2 * kc + 1;
    const int64_t lev0 = d.box0[l];
    float4 *dst = w.mtc + layout_base(w.lv, S::KC, l, sidx, c) + (int64_t)kc * np_;
    const int P = run * blockDim.x + threadIdx.x;
    if (P < np_) {
        const int qq = P - Lc - 1;
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
        if (qq >= 0 && qq < nc * Lc) {
            const int row = qq / Lc, colp = qq - row * Lc;
            if (colp >= 1 && colp <= nc) {
                const int64_t box = lev0 + (int64_t)(2 * row + (c >> 1)) * ns + 2 * (colp - 1) + (c & 1);
                if (w.bcount[box] != 0) {
                    const float2 *src = w.M32 + box * p;
                    if (m0 < p)
                        a0 = src[m0];
                    if (m1 < p)
                        a1 = src[m1];
                }
            }
        }
        const float4 hi = make_float4(tf32_rn(a0.x), tf32_rn(a0.y), tf32_rn(a1.x), tf32_rn(a1.y));
        const float4 lo = make_float4(tf32_rn(a0.x - hi.x), tf32_rn(a0.y - hi.y), tf32_rn(a1.x - hi.z),
                                      tf32_rn(a1.y - hi.w));
        dst[P] = hi;
        dst[(int64_t)S::KC * np_ + P] = lo;
    }
}

// Waits for the phase of the given parity, or gives up when another role of the CTA has failed (*bad) or after
// a bounded number of polls (then sets *bad).
__device__ __forceinline__ bool wait_or_bad(uint64_t *bar, uint32_t parity, volatile int *bad)
{
    for (int it = 0; it < (1 << 20); ++it) {
        if (mbar_try(bar, parity))
            return true;
        if ((it & 15) == 15 && *bad)
            return false;
    }
    *bad = 1;
    return false;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Roles: warps 0-3 read the accumulators back (warp w owns tensor-memory lanes 32 w .. 32 w + 31, i.e. target
// positions), one thread of warp 4 issues the MMAs, one thread of warp 5 issues the bulk copies. Hand-offs go
// through mbarriers: B slots (full / empty), window buffers (full / empty) and NS accumulator stages
// (full / empty); the MMA thread frees a B slot, a window buffer or signals a stage by tcgen05.commit.
constexpr int kThreads = 192;
constexpr int kStages = 3;  // accumulator stages; each holds three accumulators (hi*hi, hi*lo, lo*hi) of NP columns
constexpr int kParts = 3;
__host__ __device__ constexpr int tmem_cols(int np) { return kStages * kParts * np <= 256 ? 256 : 512; }

template <int PB>
__global__ void __launch_bounds__(kThreads, 1) k_m2l_tc(Work w, const unsigned char *__restrict__ btab, int l_lo,
                                                        int l_hi, int ws)
{
    using S = TcShape<PB>;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bfull[S::NSLOT], bempty[S::NSLOT], wfull[2], wempty[2], tfull[kStages],
        tempty[kStages];
    __shared__ uint32_t tmem_base;
    __shared__ int s_bad;
    __shared__ int s_gq[5];         // first offset of each source class in the CTA's list; s_gq[4] = 27
    __shared__ int s_delta[kNOff];  // B table index of each offset
    __shared__ int s_a0[kNOff];     // window position of each offset's first A row
    const int WB = 2 * S::KC * ws * 16;  // one window buffer: hi planes, then lo planes
    unsigned char *const sB = sm + 2 * WB;
    volatile int *bad = &s_bad;

    // block -> (level, system, class, tile of 128 positions); finest level first
    int64_t g = blockIdx.x;
    int l = l_hi, tiles = 1;
    for (; l >= l_lo; --l) {
        const int ncl = 1 << (l - 1);
        tiles = (ncl * (ncl + 2) + kRows - 1) / kRows;
        const int64_t cnt = (int64_t)w.lv.nsys_at[l] * 4 * tiles;
        if (g < cnt)
            break;
        g -= cnt;
    }
    if (l < l_lo)
        return;  // block-uniform
    const int sidx = (int)(g / (4 * tiles));
    const int rem = (int)(g - (int64_t)sidx * 4 * tiles);
    const int cls = rem / tiles, tile = rem - cls * tiles;
    const SysDev &d = w.sys[sys_at_level(w, l, sidx)];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, p = w.p;
    const int cx = cls & 1, cy = cls >> 1, ns = 1 << l, nc = ns >> 1, Lc = nc + 2;
    const int q0 = tile * kRows;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(tmem_cols(S::NP)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        int q = 0;
        for (int gs = 0; gs < 4; ++gs) {
            s_gq[gs] = q;
            for (int ry = -2 - cy; ry <= 3 - cy; ++ry)
                for (int rx = -2 - cx; rx <= 3 - cx; ++rx) {
                    if (rx >= -1 && rx <= 1 && ry >= -1 && ry <= 1)
                        continue;  // adjacent: near field
                    const int ux = cx + rx + 4, uy = cy + ry + 4;  // source box = 2 (i, j) + (ux, uy) - 4
                    if ((ux & 1) + 2 * (uy & 1) != gs)
                        continue;
                    s_delta[q] = (ry + 3) * 7 + (rx + 3);
                    s_a0[q] = (1 + (uy >> 1) - 2) * Lc + 1 + (ux >> 1) - 2;
                    ++q;
                }
        }
        s_gq[4] = q;
        s_bad = 0;
        for (int i = 0; i < S::NSLOT; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bempty[i])));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&wfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&wempty[i])));
        }
        for (int i = 0; i < kStages; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&tempty[i])));  // one per warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // zeros that no copy overwrites: B rows >= 8 NG of every slot
    {
        constexpr int zb = (S::B_PART - S::B_LOAD) / 16;
        if constexpr (zb > 0) {
            for (int i = tid; i < S::NSLOT * 2 * zb; i += kThreads) {
                const int part = i / zb, j = i - part * zb;
                reinterpret_cast<float4 *>(sB + part * S::B_PART + S::B_LOAD)[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
    fence_async_smem();  // those zeros, visible to the tensor core
    tc_before_sync();
    __syncthreads();     // offset lists, barriers and tensor memory ready
    tc_after_sync();
    const uint32_t tmem = tmem_base;

    float acc[S::KP];
#pragma unroll
    for (int k = 0; k < S::KP; ++k)
        acc[k] = 0.f;

    // The copy and MMA warps run their loops with all 32 lanes (waits by every lane, so each warp stays
    // converged); lane 0 alone issues the copies, MMAs and commits.
    auto warp_wait = [&](uint64_t *bar, uint32_t parity) {
        return __all_sync(0xffffffffu, wait_or_bad(bar, parity, bad));
    };
    if (warp == 5) {
        // ---------------- copies: windows (source classes) and B_delta, in the order the MMAs use them
        const int np_ = npos_of(l);
        const uint32_t wrun = (uint32_t)(2 * Lc + 130) * 16u;  // bytes of one plane's window
        int nb = 0, nw = 0;  // copies of B and of windows issued
        auto load_window = [&](int gs) {
            if (lane == 0) {
                uint64_t *bar = &wfull[gs & 1];
                const float4 *src = w.mtc + layout_base(w.lv, S::KC, l, sidx, gs) + q0;
                unsigned char *dst = sm + (gs & 1) * WB;
                mbar_expect_tx(bar, 2u * S::KC * wrun);
                for (int pl = 0; pl < 2 * S::KC; ++pl)
                    bulk_g2s(dst + (size_t)pl * ws * 16, src + (int64_t)pl * np_, wrun, bar);
            }
            __syncwarp();
            nw = gs + 1;
        };
        load_window(0);
        load_window(1);
        int gs = 0;
        for (int q = 0; q < kNOff; ++q) {
            const int slot = q % S::NSLOT;
            if (q >= S::NSLOT && !warp_wait(&bempty[slot], (uint32_t)(q / S::NSLOT - 1) & 1u))
                break;
            if (lane == 0) {
                const unsigned char *src =
                    btab + ((size_t)(blockIdx.x % kReplicas) * kNDelta + s_delta[q]) * S::B_SLOT;
                mbar_expect_tx(&bfull[slot], 2 * S::B_LOAD);
                bulk_g2s(sB + slot * S::B_SLOT, src, S::B_LOAD, &bfull[slot]);
                bulk_g2s(sB + slot * S::B_SLOT + S::B_PART, src + S::B_PART, S::B_LOAD, &bfull[slot]);
            }
            __syncwarp();
            nb = q + 1;
            // three B of class gs + 1 are on their way: wait for class gs's MMAs, then its buffer takes gs + 2
            if (gs + 2 < 4 && q == s_gq[gs + 1] + 2) {
                if (!warp_wait(&wempty[gs & 1], (uint32_t)(gs >> 1) & 1u))
                    break;
                load_window(gs + 2);
                ++gs;
            }
        }
        // every copy lands before the CTA may exit (bounded): the last one issued into each slot and buffer
        for (int q = nb - S::NSLOT < 0 ? 0 : nb - S::NSLOT; q < nb; ++q)
            mbar_wait(&bfull[q % S::NSLOT], (uint32_t)(q / S::NSLOT) & 1u);
        for (int gs = nw - 2 < 0 ? 0 : nw - 2; gs < nw; ++gs)
            mbar_wait(&wfull[gs & 1], (uint32_t)(gs >> 1) & 1u);
    } else if (warp == 4) {
        // ---------------- MMAs
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(S::NP >> 3) << 17) |
                               ((uint32_t)(kRows >> 4) << 24);  // D f32, A, B tf32 K-major, N = NP, M = 128
        const uint32_t lbo_a = (uint32_t)ws * 16u, plane2 = 2u * (uint32_t)ws * 16u;
        int committed = -1;
        int gs = 0;
        for (int q = 0; q < kNOff; ++q) {
            if (q == s_gq[gs] && !warp_wait(&wfull[gs & 1], (uint32_t)(gs >> 1) & 1u))
                break;
            const int slot = q % S::NSLOT, st = q % kStages;
            if (!warp_wait(&bfull[slot], (uint32_t)(q / S::NSLOT) & 1u))
                break;
            if (q >= kStages && !warp_wait(&tempty[st], (uint32_t)(q / kStages - 1) & 1u))
                break;
            const bool last_of_class = q + 1 == s_gq[gs + 1];
            if (lane == 0) {
                tc_after_sync();
                const uint32_t ah0 = smem_u32(sm + (gs & 1) * WB) + (uint32_t)s_a0[q] * 16u;
                const uint32_t al0 = ah0 + (uint32_t)(S::KC * ws * 16);
                const uint32_t bh0 = smem_u32(sB + slot * S::B_SLOT), bl0 = bh0 + S::B_PART;
                // three independent accumulation chains (hi*hi, hi*lo, lo*hi) so that consecutive MMAs do not wait
                // for each other's accumulator
                const uint32_t d_acc = tmem + (uint32_t)(st * kParts * S::NP);
#pragma unroll
                for (int ks = 0; ks < S::KP / 8; ++ks) {
                    const uint64_t ah = sdesc(ah0 + ks * plane2, lbo_a, 128), al = sdesc(al0 + ks * plane2, lbo_a, 128);
                    const uint64_t bh = sdesc(bh0 + ks * 256, 128, S::KC * 128),
                                   bl = sdesc(bl0 + ks * 256, 128, S::KC * 128);
                    const uint32_t acc_on = ks > 0 ? 1u : 0u;
                    mma_tf32(d_acc, ah, bh, idesc, acc_on);
                    mma_tf32(d_acc + S::NP, ah, bl, idesc, acc_on);
                    mma_tf32(d_acc + 2 * S::NP, al, bh, idesc, acc_on);
                }
                tc_commit(&tfull[st]);
                tc_commit(&bempty[slot]);
                if (last_of_class)
                    tc_commit(&wempty[gs & 1]);
            }
            __syncwarp();
            if (last_of_class)
                ++gs;
            committed = q;
        }
        if (committed >= 0)  // the last MMAs land before shared and tensor memory are released (bounded)
            mbar_wait(&tfull[committed % kStages], (uint32_t)(committed / kStages) & 1u);
    } else {
        // ---------------- read-back: warps 0-3, one target position per thread
        const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);
        for (int q = 0; q < kNOff; ++q) {
            const int st = q % kStages;
            if (!__all_sync(0xffffffffu, wait_or_bad(&tfull[st], (uint32_t)(q / kStages) & 1u, bad)))
                break;
            tc_after_sync();
            uint32_t r[kParts][S::RD][8];
#pragma unroll
            for (int pt = 0; pt < kParts; ++pt)
#pragma unroll
                for (int j = 0; j < S::RD; ++j)
                    tmem_ld8(tlane + (uint32_t)((st * kParts + pt) * S::NP + 8 * j), r[pt][j]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            tc_before_sync();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&tempty[st]);
#pragma unroll
            for (int j = 0; j < S::RD; ++j)
#pragma unroll
                for (int i = 0; i < 8; ++i)  // the small products first
                    acc[8 * j + i] += (__uint_as_float(r[1][j][i]) + __uint_as_float(r[2][j][i])) +
                                      __uint_as_float(r[0][j][i]);
        }
    }
    tc_before_sync();
    __syncthreads();
    const bool ok = !s_bad;
    if (ok && warp < 4) {
        const int tq = q0 + tid, row = tq / Lc, colp = tq - row * Lc;
        if (row < nc && colp >= 1 && colp <= nc) {
            const int64_t box = d.box0[l] + (int64_t)(2 * row + cy) * ns + 2 * (colp - 1) + cx;
            if (w.bcount[box] != 0) {
                float2 *dst = w.L32 + box * p;
#pragma unroll
                for (int m = 0; m < PB; ++m)
                    if (m < p)
                        dst[m] = make_float2(acc[2 * m], acc[2 * m + 1]);
            }
        }
    }
    if (!ok && tid == 0)
        atomicOr(w.status, FMM_DEV_TIMEOUT);
    if (warp == 0) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols(S::NP)));
    }
}

template <int PB>
int set_smem_attr()
{
    return cudaFuncSetAttribute(k_m2l_tc<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes<PB>(window_len(kMaxClassWidth + 2))) == cudaSuccess
               ? 0
               : -1;
}

int bucket_of(int p) { return p <= 8 ? 8 : p <= 12 ? 12 : p <= 16 ? 16 : 20; }

template <int PB>
constexpr size_t table_bytes()
{
    return (size_t)kReplicas * kNDelta * TcShape<PB>::B_SLOT;
}

bool g_tc_ready[64] = {};

// TF32 value nearest to x (ties away from zero), the rounding of cvt.rna.tf32.f32.
float tf32_round_host(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u + 0x1000u) & 0xffffe000u;
    memcpy(&f, &u, 4);
    return f;
}

template <int PB>
void build_table(int p, unsigned char *out)
{
    using S = TcShape<PB>;
    memset(out, 0, table_bytes<PB>());
    std::vector<std::complex<double>> pw(2 * PB + 1);
    const size_t one = (size_t)kNDelta * S::B_SLOT;
    for (int dy = -3; dy <= 3; ++dy)
        for (int dx = -3; dx <= 3; ++dx) {
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1)
                continue;
            const std::complex<double> rho = 1.0 / std::complex<double>(dx, dy);
            pw[0] = 1.0;
            for (int k = 1; k <= 2 * p; ++k)
                pw[k] = pw[k - 1] * rho;
            unsigned char *hi = out + (size_t)((dy + 3) * 7 + (dx + 3)) * S::B_SLOT, *lo = hi + S::B_PART;
            for (int l = 0; l < p; ++l)
                for (int m = 0; m < p; ++m) {
                    double c = 1.0;
                    for (int i = 1; i <= m; ++i)
                        c = c * (double)(l + i) / (double)i;  // C(m + l, m)
                    const std::complex<double> t = ((m & 1) ? c : -c) * pw[m + l + 1];
                    // rows n = 2l (real part of b_l), 2l + 1 (imaginary); columns k = 2m (Re a_m), 2m + 1 (Im a_m)
                    const double e[2][2] = {{t.real(), -t.imag()}, {t.imag(), t.real()}};
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b) {
                            const float h = tf32_round_host(e[a][b]), r = tf32_round_host(e[a][b] - (double)h);
                            const int off = core_off(2 * l + a, 2 * m + b, S::KP);
                            memcpy(hi + off, &h, 4);
                            memcpy(lo + off, &r, 4);
                        }
                }
        }
    for (int rep = 1; rep < kReplicas; ++rep)
        memcpy(out + rep * one, out, one);
}

template <int PB>
int launch_bucket(const Work &w, const Tables &t, int l_lo, int l_hi, int64_t items, cudaStream_t s)
{
    int64_t planes = 0;
    for (int l = l_lo; l <= l_hi; ++l)
        planes += (int64_t)w.lv.nsys_at[l] * 4 * TcShape<PB>::KC;
    const int nch = (npos_of(l_hi) + 255) / 256;
    k_m2l_tc_layout<PB><<<(unsigned)(planes * nch), 256, 0, s>>>(w, l_lo, l_hi, nch);
    const int ws = window_len((1 << (l_hi - 1)) + 2);
    k_m2l_tc<PB><<<(unsigned)items, kThreads, smem_bytes<PB>(ws), s>>>(w, t.m2l_tc, l_lo, l_hi, ws);
    return 2;
}

}  // namespace

bool m2l_tc_supported(int p) { return p >= 1 && p <= kPMaxTc; }

int m2l_tc_max_level() { return 7; }  // the finest level whose class grid (2^(l-1) boxes wide) is <= kMaxClassWidth

size_t m2l_tc_table_bytes(int p)
{
    switch (bucket_of(p < kPMaxTc ? p : kPMaxTc)) {
    case 8:
        return table_bytes<8>();
    case 12:
        return table_bytes<12>();
    case 16:
        return table_bytes<16>();
    default:
        return table_bytes<20>();
    }
}

// B_delta (hi, lo) of the 40 offsets for p (zeros for p > 20, which never runs here), in the layout above,
// indexed (dy + 3) * 7 + (dx + 3), the 9 near offsets zero; the whole table kReplicas times.
void build_m2l_tc_table_host(int p, unsigned char *out)
{
    if (!m2l_tc_supported(p)) {
        memset(out, 0, m2l_tc_table_bytes(p));
        return;
    }
    switch (bucket_of(p)) {
    case 8:
        build_table<8>(p, out);
        break;
    case 12:
        build_table<12>(p, out);
        break;
    case 16:
        build_table<16>(p, out);
        break;
    default:
        build_table<20>(p, out);
        break;
    }
}

int prepare_m2l_tc()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return -1;
    if (g_tc_ready[dev])
        return 0;
    if (set_smem_attr<8>() || set_smem_attr<12>() || set_smem_attr<16>() || set_smem_attr<20>())
        return -1;
    g_tc_ready[dev] = 1;
    return 0;
}

size_t m2l_tc_layout_bytes(const LevelInfo &lv, int p)
{
    if (!m2l_tc_supported(p))
        return 0;
    const int kc = bucket_of(p) == 8 ? TcShape<8>::KC : bucket_of(p) == 12 ? TcShape<12>::KC
                                                       : bucket_of(p) == 16 ? TcShape<16>::KC
                                                                            : TcShape<20>::KC;
    const int lt = lv.maxdepth < m2l_tc_max_level() ? lv.maxdepth : m2l_tc_max_level();
    return lt < 2 ? 0 : (size_t)layout_base(lv, kc, lt + 1, 0, 0) * 16;
}

int launch_m2l_tc(const Work &w, const Tables &t, int l_lo, int l_hi, cudaStream_t s)
{
    if (!m2l_tc_supported(w.p) || !w.mtc || l_hi > m2l_tc_max_level() || l_lo < 2 || l_hi < l_lo)
        return 0;
    int64_t items = 0;
    for (int l = l_lo; l <= l_hi; ++l) {
        const int nc = 1 << (l - 1);
        items += (int64_t)w.lv.nsys_at[l] * 4 * ((nc * (nc + 2) + kRows - 1) / kRows);
    }
    if (items == 0)
        return 0;
    switch (bucket_of(w.p)) {
    case 8:
        return launch_bucket<8>(w, t, l_lo, l_hi, items, s);
    case 12:
        return launch_bucket<12>(w, t, l_lo, l_hi, items, s);
    case 16:
        return launch_bucket<16>(w, t, l_lo, l_hi, items, s);
    default:
        return launch_bucket<20>(w, t, l_lo, l_hi, items, s);
    }
}

}  // namespace fmm
