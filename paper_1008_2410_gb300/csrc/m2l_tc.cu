// m2l_tc.cu -- Fig. 1 stage 6 (M2L, §3) of the precision form on the tensor cores (tcgen05, TMEM).
//
// With radius-scaled coefficients the translation from a source box at offset delta = (dx, dy) box widths
// (a Gaussian integer, max(|dx|, |dy|) in {2, 3}) is the same matrix at every level:
//     b^_l += sum_m T[l][m] a~_m,   T[l][m] = (-1)^(m+1) C(m + l, m) rho^(m+l+1),   rho = 1 / delta.
// Over the reals, with real and imaginary parts interleaved (input k = 2m + {0, 1}, output n = 2l + {0, 1}),
// each of the 40 offsets is one 2p x 2p real matrix T_delta; the host builds it in FP64 and stores every entry
// as a TF32 pair (hi, lo).
//
// Shape. A tcgen05.mma of kind::tf32 with M = 128 and K = 8 costs 47 cycles at N = 48 and 129 at N = 256
// (fmm_probe_peaks, GB300), so the work per instruction grows far faster than its cost with N; the contraction
// is laid out with the targets as N = 256:
//     D[n][t] += sum_k A[n][k] W[t][k],   A = [T_hi ; T_lo] (rows 0 .. 2p and R .. R + 2p, R = 2p rounded up to 8),
// W = the source window, once with its hi part and once with its lo part into the same accumulator, so that the
// two row blocks of D sum to T_hi W_hi + T_hi W_lo + T_lo W_hi + T_lo W_lo. A's rows from 2R on are never read
// back: they may hold whatever follows the slice in shared memory.
//
// Which sources. The boxes of a level fall into four classes by child position c = (cx, cy). A box of class c
// at class coordinates (i, j) (its parent's coordinates) takes its 27 interaction-list sources from the children
// of the parent's 3 x 3 neighbours: boxes of class c' at class coordinates (i + ox, j + oy), ox, oy in
// {-1, 0, 1}. On a class grid whose rows carry one zero column at either end (row length Lc = 2^(l-1) + 2), the
// sources of 256 consecutive target positions q0 .. q0 + 255 at one offset are 256 consecutive positions,
// starting at (1 + oy) Lc + 1 + ox in the window [q0 - Lc - 1, q0 + Lc + 257) of class c'. A first kernel writes
// each level's multipoles in that form (per class, TF32 hi and lo planes of 16-byte K chunks, one position per
// chunk, zeros for padding and empty boxes); every offset's B operand is then a shared-memory descriptor into one
// bulk-copied window (8-row core matrices 128 bytes apart, K planes one window apart).
//
// Work. A CTA takes 256 target positions of class c and the 5 .. 8 offsets whose sources are of class c': four
// CTAs share a tile. K is streamed in steps of 8 through two stages: a stage holds the window's hi and lo planes
// of that step and the K slices of A of all the CTA's offsets (one bulk copy from a table ordered by (c, c', K
// step, offset)), about 47 KB, so that two CTAs share an SM and one's copies and read-back overlap the other's
// MMAs. Roles: one warp copies, one thread issues the MMAs (stages are released by tcgen05.commit), four warps
// read the 256-column accumulator back through a shared-memory transpose into a partial local expansion per
// (box, c'); the fourth CTA of a tile to finish (an atomic count) sums the four partials in a fixed order into
// the level's locals, so results do not depend on scheduling. Every wait is bounded: on a timeout the CTA sets
// FMM_DEV_TIMEOUT and still completes the count.
//
// Levels whose class grid is wider than 64 boxes (windows too large for shared memory) and p > 20 take the
// CUDA-core kernel (sweep.cu).
#include <complex>
#include <cstring>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kN = 256;            // MMA N: target positions per CTA
constexpr int kM = 128;            // MMA M: output rows
constexpr int kMaxOff = 8;         // offsets of one (class, source class) pair, at most
constexpr int kMaxClassWidth = 64;  // widest class grid (level 7) whose window fits in shared memory
constexpr int kPMaxTc = 20;
constexpr int kThreads = 192;      // warps 0-3 read back, warp 4 issues the MMAs, warp 5 copies

template <int PB>
struct TcShape {
    static constexpr int KP = (2 * PB + 7) / 8 * 8;  // K: 2p real inputs, padded to the MMA's K step
    static constexpr int KC = KP / 4;                // 16-byte K chunks (window planes)
    static constexpr int NKS = KP / 8;               // K steps
    static constexpr int R = KP;                     // first row of T_lo in A
    static constexpr int AS = 2 * R / 8 * 256;       // one K slice of A: 2R rows of two 16-byte chunks
    static constexpr int A_OVER = (kM - 2 * R) / 8 * 256;  // rows 2R .. 127 of the last slice, read but unused
    static constexpr int A_STAGE = kMaxOff * AS + A_OVER;
};

// Window of a tile: the 2 Lc + 258 positions its offsets read.
__host__ __device__ inline int window_len(int Lc) { return 2 * Lc + 258; }
// Positions per class and plane in the source layout: rows -1 .. nc of the padded grid plus the overhang of the
// last tile's window.
__host__ __device__ inline int npos_of(int l)
{
    const int nc = 1 << (l - 1), Lc = nc + 2;
    return (nc + 2) * Lc + 258;
}
__host__ __device__ inline int tiles_of(int l)
{
    const int nc = 1 << (l - 1);
    return (nc * (nc + 2) + kN - 1) / kN;
}

// Shared memory: two stages of (window planes of one K step: hi 2 ks, 2 ks + 1, lo 2 ks, 2 ks + 1; A slices),
// reused after the MMAs by the read-back transpose [2R][kN + 1] floats.
template <int PB>
__host__ __device__ constexpr size_t stage_bytes(int ws)
{
    return (size_t)4 * ws * 16 + TcShape<PB>::A_STAGE;
}
template <int PB>
constexpr size_t smem_bytes(int ws)
{
    const size_t main = 2 * stage_bytes<PB>(ws);
    const size_t tr = (size_t)2 * TcShape<PB>::R * (kN + 1) * 4;
    return main > tr ? main : tr;
}

// The offsets of target class c whose sources are of class c', in a fixed order (the table and the kernel agree):
// table index (dy + 3) * 7 + (dx + 3) and window position of the first source; returns their number.
__host__ __device__ inline int pair_offsets(int c, int cs, int Lc, int *delta, int *b0)
{
    const int cx = c & 1, cy = c >> 1;
    int q = 0;
    for (int ry = -2 - cy; ry <= 3 - cy; ++ry)
        for (int rx = -2 - cx; rx <= 3 - cx; ++rx) {
            if (rx >= -1 && rx <= 1 && ry >= -1 && ry <= 1)
                continue;  // adjacent: near field
            const int ux = cx + rx + 4, uy = cy + ry + 4;  // source box = 2 (i, j) + (ux, uy) - 4
            if ((ux & 1) + 2 * (uy & 1) != cs)
                continue;
            if (delta)
                delta[q] = (ry + 3) * 7 + (rx + 3);
            if (b0)
                b0[q] = (1 + (uy >> 1) - 2) * Lc + 1 + (ux >> 1) - 2;
            ++q;
        }
    return q;
}

// Byte offset of element (row, kk) in one K slice of A (K-major, non-swizzled operand layout): 8-row x 16-byte
// core matrices, the slice's two K-adjacent core matrices 128 bytes apart (leading-dimension offset), 8-row
// groups 256 bytes apart (stride-dimension offset).
__host__ __device__ inline int slice_off(int row, int kk)
{
    return ((row >> 3) * 2 + (kk >> 2)) * 128 + (row & 7) * 16 + (kk & 3) * 4;
}

// Offsets into the workspace arrays, levels from 2 up, systems in order.
// Source layout (Work::mtc, float4): per (level, system, class c'), 2 (hi, lo) x KC planes of npos_of(l) chunks.
__host__ __device__ inline int64_t layout_base(const LevelInfo &lv, int KC, int l, int sidx, int c)
{
    int64_t b = 0;
    for (int k = 2; k < l; ++k)
        b += (int64_t)lv.nsys_at[k] * 8 * KC * npos_of(k);
    return b + (int64_t)(sidx * 4 + c) * 2 * KC * npos_of(l);
}
// Partials (Work::m2l_part, float2): per (level, system, box), four records of p coefficients (one per c').
__host__ __device__ inline int64_t part_base(const LevelInfo &lv, int l, int sidx)
{
    int64_t b = 0;
    for (int k = 2; k < l; ++k)
        b += (int64_t)lv.nsys_at[k] << (2 * k);
    return b + ((int64_t)sidx << (2 * l));
}
// Counters (Work::m2l_cnt): per (level, system, class, tile).
__host__ __device__ inline int64_t count_base(const LevelInfo &lv, int l, int sidx)
{
    int64_t b = 0;
    for (int k = 2; k < l; ++k)
        b += (int64_t)lv.nsys_at[k] * 4 * tiles_of(k);
    return b + (int64_t)sidx * 4 * tiles_of(l);
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
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Per-level offsets of one layout launch, computed on the host: for level lev[k], its first thread, the float4
// offset of its planes and the positions per plane; and the range of tile counters the launch zeroes.
struct LayoutPlan {
    int nlev;
    int lev[FMM_MAXL];
    int npos[FMM_MAXL];
    int64_t t0[FMM_MAXL + 1];
    int64_t base[FMM_MAXL];
    int64_t c0, c1;
};

// Source layout of levels l_lo .. l_hi: a thread per (level, system, class, K chunk, position P) writes the hi
// and lo chunks of coefficients 2 kc, 2 kc + 1 of the box at P; the first threads also zero the levels' tile
// counters (there are fewer counters than threads).
template <int PB>
__global__ void __launch_bounds__(256) k_m2l_tc_layout(Work w, LayoutPlan pl)
{
    using S = TcShape<PB>;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < pl.c1 - pl.c0)
        w.m2l_cnt[pl.c0 + g] = 0;
    int k = 0;
    while (k < pl.nlev && g >= pl.t0[k + 1])
        ++k;
    if (k >= pl.nlev)
        return;
    const int l = pl.lev[k];
    const unsigned np_ = (unsigned)pl.npos[k], gl = (unsigned)(g - pl.t0[k]);  // a level's positions < 2^32
    const unsigned P = gl % np_, r = gl / np_;
    const int kc = (int)(r % S::KC), c = (int)(r / S::KC) & 3, sidx = (int)(r / S::KC) >> 2;
    const int p = w.p, ns = 1 << l, nc = ns >> 1, Lc = nc + 2, qq = (int)P - Lc - 1;
    float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
    if (qq >= 0 && qq < nc * Lc) {
        const int row = qq / Lc, colp = qq - row * Lc;
        if (colp >= 1 && colp <= nc) {
            const SysDev &d = w.sys[sys_at_level(w, l, sidx)];
            const int64_t box = d.box0[l] + (int64_t)(2 * row + (c >> 1)) * ns + 2 * (colp - 1) + (c & 1);
            if (w.bcount[box] != 0) {
                const float2 *src = w.M32 + box * p;
                if (2 * kc < p)
                    a0 = src[2 * kc];
                if (2 * kc + 1 < p)
                    a1 = src[2 * kc + 1];
            }
        }
    }
    const float4 hi = make_float4(tf32_rn(a0.x), tf32_rn(a0.y), tf32_rn(a1.x), tf32_rn(a1.y));
    const float4 lo = make_float4(tf32_rn(a0.x - hi.x), tf32_rn(a0.y - hi.y), tf32_rn(a1.x - hi.z),
                                  tf32_rn(a1.y - hi.w));
    float4 *dst = w.mtc + pl.base[k] + (int64_t)(sidx * 4 + c) * 2 * S::KC * np_ + (int64_t)kc * np_ + P;
    dst[0] = hi;
    dst[(int64_t)S::KC * np_] = lo;
}

template <int PB>
__global__ void __launch_bounds__(kThreads, 2) k_m2l_tc(Work w, const unsigned char *__restrict__ atab, int l_lo,
                                                        int l_hi, int ws)
{
    using S = TcShape<PB>;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t sfull[2], sempty[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_bad, s_last, s_nq;
    __shared__ int s_b0[kMaxOff];  // window position of each offset's first source
    __shared__ int s_dst[kN];      // level-local box of each target position, or -1 (padding, outside, empty)
    const int SB = (int)stage_bytes<PB>(ws);
    float *const stg = reinterpret_cast<float *>(sm);  // read-back transpose [2R][kN + 1], after the MMAs
    volatile int *bad = &s_bad;

    // block -> (level, system, class c, tile, source class c'); finest level first, a tile's four CTAs adjacent
    int64_t g = blockIdx.x;
    int l = l_hi;
    for (; l >= l_lo; --l) {
        const int64_t cnt = (int64_t)w.lv.nsys_at[l] * 16 * tiles_of(l);
        if (g < cnt)
            break;
        g -= cnt;
    }
    if (l < l_lo)
        return;  // block-uniform
    const int tiles = tiles_of(l);
    const int csrc = (int)(g & 3), tile = (int)((g >> 2) % tiles), r = (int)((g >> 2) / tiles);
    const int cls = r & 3, sidx = r >> 2;
    const SysDev &d = w.sys[sys_at_level(w, l, sidx)];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, p = w.p;
    const int cx = cls & 1, cy = cls >> 1, ns = 1 << l, nc = ns >> 1, Lc = nc + 2;
    const int q0 = tile * kN;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_nq = pair_offsets(cls, csrc, Lc, nullptr, s_b0);
        s_bad = 0;
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sempty[i])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int j = tid; j < kN; j += kThreads) {
        const int tq = q0 + j, row = tq / Lc, colp = tq - row * Lc;
        int lb = -1;
        if (row < nc && colp >= 1 && colp <= nc) {
            lb = (2 * row + cy) * ns + 2 * (colp - 1) + cx;
            if (w.bcount[d.box0[l] + lb] == 0)
                lb = -1;
        }
        s_dst[j] = lb;
    }
    tc_before_sync();
    __syncthreads();  // offset list, barriers and tensor memory ready
    tc_after_sync();
    const uint32_t tmem = tmem_base;
    const int nq = s_nq;
    auto warp_wait = [&](uint64_t *bar, uint32_t parity) {
        return __all_sync(0xffffffffu, wait_or_bad(bar, parity, bad));
    };

    if (warp == 5) {
        // ---------------- copies: per K step, the window's four planes and the A slices of the offsets
        const uint32_t wrun = (uint32_t)window_len(Lc) * 16u;
        const float4 *wsrc = w.mtc + layout_base(w.lv, S::KC, l, sidx, csrc) + q0;
        const int np_ = npos_of(l);
        const unsigned char *asrc = atab + (size_t)((cls * 4 + csrc) * S::NKS) * kMaxOff * S::AS;
        int ns_ = 0;
        for (int ks = 0; ks < S::NKS; ++ks) {
            const int st = ks & 1;
            if (ks >= 2 && !warp_wait(&sempty[st], (uint32_t)((ks >> 1) - 1) & 1u))
                break;
            if (lane == 0) {
                unsigned char *dst = sm + st * SB;
                mbar_expect_tx(&sfull[st], 4u * wrun + (uint32_t)(nq * S::AS));
                for (int pl = 0; pl < 4; ++pl) {  // hi 2 ks, hi 2 ks + 1, lo 2 ks, lo 2 ks + 1
                    const int plane = (pl >> 1) * S::KC + 2 * ks + (pl & 1);
                    bulk_g2s(dst + (size_t)pl * ws * 16, wsrc + (int64_t)plane * np_, wrun, &sfull[st]);
                }
                bulk_g2s(dst + 4 * ws * 16, asrc + (size_t)ks * kMaxOff * S::AS, (uint32_t)(nq * S::AS), &sfull[st]);
            }
            __syncwarp();
            ns_ = ks + 1;
        }
        // every copy lands before the CTA may exit (bounded): the last fill of each stage
        for (int ks = ns_ - 2 < 0 ? 0 : ns_ - 2; ks < ns_; ++ks)
            mbar_wait(&sfull[ks & 1], (uint32_t)(ks >> 1) & 1u);
    } else if (warp == 4) {
        // ---------------- MMAs: D (256 columns) += A W_hi + A W_lo
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN >> 3) << 17) |
                               ((uint32_t)(kM >> 4) << 24);  // D f32, A, B tf32 K-major, N = 256, M = 128
        const uint32_t lbo_w = (uint32_t)ws * 16u;
        int committed = -1;
        for (int ks = 0; ks < S::NKS; ++ks) {
            const int st = ks & 1;
            if (!warp_wait(&sfull[st], (uint32_t)(ks >> 1) & 1u))
                break;
            if (lane == 0) {
                tc_after_sync();
                const uint32_t wbase = smem_u32(sm + st * SB), abase = wbase + 4u * ws * 16u;
                for (int q = 0; q < nq; ++q) {
                    const uint64_t a = sdesc(abase + (uint32_t)(q * S::AS), 128, 256);
                    const uint32_t wh = wbase + (uint32_t)s_b0[q] * 16u;
                    const uint64_t bh = sdesc(wh, lbo_w, 128), bl = sdesc(wh + 2u * ws * 16u, lbo_w, 128);
                    mma_tf32(tmem, a, bh, idesc, (ks > 0 || q > 0) ? 1u : 0u);
                    mma_tf32(tmem, a, bl, idesc, 1u);
                }
                tc_commit(&sempty[st]);
                if (ks + 1 == S::NKS)
                    tc_commit(&done);
            }
            __syncwarp();
            committed = ks;
        }
        if (committed + 1 != S::NKS)
            *bad = 1;
        if (committed >= 0)  // the MMAs land before shared and tensor memory are reused (bounded)
            mbar_wait(&sempty[committed & 1], (uint32_t)(committed >> 1) & 1u);
    } else {
        // ---------------- read-back: the accumulator is final once `done` completes
        if (warp_wait(&done, 0u)) {
            tc_after_sync();
            const int row = 32 * warp + lane;  // this thread's tensor-memory lane = output row
            const bool keep = row < 2 * S::R;
            const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
            for (int c0 = 0; c0 < kN; c0 += 32) {
                uint32_t h[4][8];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    tmem_ld8(tl + (uint32_t)(c0 + 8 * j), h[j]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (keep) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            stg[row * (kN + 1) + c0 + 8 * j + i] = __uint_as_float(h[j][i]);
                }
            }
        }
    }
    tc_before_sync();
    __syncthreads();  // the transpose is complete (or the CTA failed); every copy and MMA has landed

    // partial of this source class for the tile's target boxes, element (target j, coefficient m) per thread,
    // consecutive threads on consecutive coefficients: rows 2m (+ 1) of T_hi plus those of T_lo
    const int64_t pb = part_base(w.lv, l, sidx);
    const bool ok = !s_bad;
    {
        int j = tid / p, m = tid - j * p;
        const int dj = kThreads / p, dm = kThreads - dj * p;
        for (int e = tid; e < kN * p; e += kThreads) {
            const int lb = s_dst[j];
            if (lb >= 0) {
                float re = 0.f, im = 0.f;
                if (ok) {
                    re = stg[(2 * m) * (kN + 1) + j] + stg[(S::R + 2 * m) * (kN + 1) + j];
                    im = stg[(2 * m + 1) * (kN + 1) + j] + stg[(S::R + 2 * m + 1) * (kN + 1) + j];
                }
                w.m2l_part[((pb + lb) * 4 + csrc) * p + m] = make_float2(re, im);
            }
            j += dj;
            m += dm;
            if (m >= p) {
                m -= p;
                ++j;
            }
        }
    }
    __threadfence();
    __syncthreads();
    int *const counter = w.m2l_cnt + count_base(w.lv, l, sidx) + cls * tiles + tile;
    if (tid == 0) {
        if (!ok)
            atomicOr(w.status, FMM_DEV_TIMEOUT);
        s_last = atomicAdd(counter, 1) == 3;
    }
    __syncthreads();
    if (s_last) {
        // the fourth CTA of the tile: locals = partials of source classes 0, 1, 2, 3, added in that order
        __threadfence();
        int j = tid / p, m = tid - j * p;
        const int dj = kThreads / p, dm = kThreads - dj * p;
#pragma unroll 4
        for (int e = tid; e < kN * p; e += kThreads) {
            const int lb = s_dst[j];
            if (lb >= 0) {
                const float2 *src = w.m2l_part + (pb + lb) * 4 * p + m;
                const float2 a = __ldcg(src), b = __ldcg(src + p), c = __ldcg(src + 2 * p), f = __ldcg(src + 3 * p);
                w.L32[(d.box0[l] + lb) * p + m] = make_float2(((a.x + b.x) + c.x) + f.x, ((a.y + b.y) + c.y) + f.y);
            }
            j += dj;
            m += dm;
            if (m >= p) {
                m -= p;
                ++j;
            }
        }
    }
    if (warp == 0) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kN));
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
int kc_of(int p) { return (2 * bucket_of(p) + 7) / 8 * 2; }

template <int PB>
constexpr size_t table_bytes()
{
    return (size_t)16 * TcShape<PB>::NKS * kMaxOff * TcShape<PB>::AS;
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

// A slices ordered by (target class c, source class c', K step ks, offset q of pair_offsets(c, c')): rows 2l + u
// (u = 0 real, 1 imaginary part of b_l) hold T_hi, rows R + 2l + u hold T_lo, columns kk = k - 8 ks with
// k = 2m (Re a~_m), 2m + 1 (Im a~_m).
template <int PB>
void build_table(int p, unsigned char *out)
{
    using S = TcShape<PB>;
    memset(out, 0, table_bytes<PB>());
    for (int c = 0; c < 4; ++c)
        for (int cs = 0; cs < 4; ++cs) {
            int delta[kMaxOff];
            const int nq = pair_offsets(c, cs, 0, delta, nullptr);
            for (int q = 0; q < nq; ++q) {
                const int dx = delta[q] % 7 - 3, dy = delta[q] / 7 - 3;
                const std::complex<double> rho = 1.0 / std::complex<double>(dx, dy);
                std::vector<std::complex<double>> pw(2 * p + 1);
                pw[0] = 1.0;
                for (int k = 1; k <= 2 * p; ++k)
                    pw[k] = pw[k - 1] * rho;
                for (int l = 0; l < p; ++l)
                    for (int m = 0; m < p; ++m) {
                        double cb = 1.0;
                        for (int i = 1; i <= m; ++i)
                            cb = cb * (double)(l + i) / (double)i;  // C(m + l, m)
                        const std::complex<double> t = ((m & 1) ? cb : -cb) * pw[m + l + 1];
                        const double e[2][2] = {{t.real(), -t.imag()}, {t.imag(), t.real()}};
                        for (int u = 0; u < 2; ++u)
                            for (int v = 0; v < 2; ++v) {
                                const int k = 2 * m + v, ks = k >> 3, kk = k & 7;
                                unsigned char *a =
                                    out + ((size_t)((c * 4 + cs) * S::NKS + ks) * kMaxOff + q) * S::AS;
                                const float h = tf32_round_host(e[u][v]), lo = tf32_round_host(e[u][v] - (double)h);
                                memcpy(a + slice_off(2 * l + u, kk), &h, 4);
                                memcpy(a + slice_off(S::R + 2 * l + u, kk), &lo, 4);
                            }
                    }
            }
        }
}

template <int PB>
int launch_bucket(const Work &w, const Tables &t, int l_lo, int l_hi, int64_t items, cudaStream_t s)
{
    LayoutPlan pl{};
    pl.t0[0] = 0;
    for (int l = l_lo; l <= l_hi; ++l) {
        const int k = pl.nlev++;
        pl.lev[k] = l;
        pl.npos[k] = npos_of(l);
        pl.base[k] = layout_base(w.lv, TcShape<PB>::KC, l, 0, 0);
        pl.t0[k + 1] = pl.t0[k] + (int64_t)w.lv.nsys_at[l] * 4 * TcShape<PB>::KC * npos_of(l);
    }
    pl.c0 = count_base(w.lv, l_lo, 0);
    pl.c1 = count_base(w.lv, l_hi + 1, 0);
    const int64_t threads = pl.t0[pl.nlev] > pl.c1 - pl.c0 ? pl.t0[pl.nlev] : pl.c1 - pl.c0;
    k_m2l_tc_layout<PB><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(w, pl);
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

// The A slices for p (zeros for p > 20, which never runs here), in the order above.
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

static int tc_top(const LevelInfo &lv) { return lv.maxdepth < m2l_tc_max_level() ? lv.maxdepth : m2l_tc_max_level(); }

size_t m2l_tc_layout_bytes(const LevelInfo &lv, int p)
{
    const int lt = tc_top(lv);
    return !m2l_tc_supported(p) || lt < 2 ? 0 : (size_t)layout_base(lv, kc_of(p), lt + 1, 0, 0) * 16;
}

size_t m2l_tc_part_bytes(const LevelInfo &lv, int p)
{
    const int lt = tc_top(lv);
    return !m2l_tc_supported(p) || lt < 2 ? 0 : (size_t)part_base(lv, lt + 1, 0) * 4 * p * sizeof(float2);
}

size_t m2l_tc_count_bytes(const LevelInfo &lv, int p)
{
    const int lt = tc_top(lv);
    return !m2l_tc_supported(p) || lt < 2 ? 0 : (size_t)count_base(lv, lt + 1, 0) * sizeof(int);
}

int launch_m2l_tc(const Work &w, const Tables &t, int l_lo, int l_hi, cudaStream_t s)
{
    if (!m2l_tc_supported(w.p) || !w.mtc || !w.m2l_part || !w.m2l_cnt || l_hi > m2l_tc_max_level() || l_lo < 2 ||
        l_hi < l_lo)
        return 0;
    int64_t items = 0;
    for (int l = l_lo; l <= l_hi; ++l)
        items += (int64_t)w.lv.nsys_at[l] * 16 * tiles_of(l);
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
