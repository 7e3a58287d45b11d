// p2p.cu -- Fig. 1 stage 9: near-field direct evaluation of the regularised kernel (Eq. 6) between
// particles in the same or adjacent leaves, and its adjoint.
//
// Each pair is evaluated from the target's side (§3: "each particle pair twice, once from each end"), so
// a target accumulates in registers and nothing is written concurrently. One thread block owns one target
// leaf; its 3 x 3 neighbourhood is three contiguous runs of the leaf-ordered particles (rows iy-1, iy, iy+1
// of columns ix-1..ix+1), staged through shared memory in tiles.
//
// Precision form (FMM_MIXED): coordinates are leaf-relative in leaf units, split hi + lo in FP32; the shift
// by the integer leaf offset is exact (Fast2Sum folds its rounding error into lo). For leaves up to about 38
// sigma wide one float per coordinate suffices (the source's hi, the target's shifted value rounded once);
// wider leaves keep both parts, so a difference has the FP64 coordinates' resolution. exp and 1/r^2 use the SFU (ex2.approx, rcp.approx); for r^2 / 2 sigma^2 < 1/2
// the factor (1 - e^-y)/y comes from its Taylor series instead of 1 - e^-y, which cancels. Two targets share
// each packed f32x2 instruction. Per-target sums are FP32 within a row of source leaves and compensated
// (TwoSum) across rows. Tiles arrive by bulk asynchronous copies (cp.async.bulk, the TMA engine) into shared
// memory, completed on an mbarrier with a bounded wait.
#include "fmm_internal.cuh"

#include <type_traits>

namespace fmm {

#define TWO_PI 6.283185307179586476925

// ------------------------------------------------------------------ FP64 form

#define TILE64 512

__global__ void __launch_bounds__(64) k_p2p64(Work w)
{
    __shared__ double shx[TILE64], shy[TILE64], shg[TILE64];
    int leaf = blockIdx.x;
    int s0 = w.start[leaf], c = w.start[leaf + 1] - s0;
    if (c == 0)
        return;
    int k = w.nsys == 1 ? 0 : find_sys_by_leaf(w.sys, w.nsys, leaf);
    const SysDev &d = w.sys[k];
    int L = d.depth, ns = 1 << L, local = leaf - (int)d.leaf0;
    int ix = local & (ns - 1), iy = local >> L;
    double k2 = 1.0 / (2.0 * d.sigma * d.sigma);
    int jx0 = ix > 0 ? ix - 1 : 0, jx1 = ix < ns - 1 ? ix + 1 : ns - 1;
    for (int t0 = 0; t0 < c; t0 += blockDim.x) {
        int tpos = s0 + t0 + threadIdx.x;
        bool valid = t0 + threadIdx.x < c;
        double xt = valid ? w.sx[tpos] : 0.0, yt = valid ? w.sy[tpos] : 0.0;
        double au = 0.0, av = 0.0;
        for (int dy = -1; dy <= 1; ++dy) {
            int row = iy + dy;
            if (row < 0 || row >= ns)
                continue;
            int r0 = w.start[d.leaf0 + row * ns + jx0], r1 = w.start[d.leaf0 + row * ns + jx1 + 1];
            for (int q0 = r0; q0 < r1; q0 += TILE64) {
                int m = min(TILE64, r1 - q0);
                __syncthreads();
                for (int j = threadIdx.x; j < m; j += blockDim.x) {
                    shx[j] = w.sx[q0 + j];
                    shy[j] = w.sy[q0 + j];
                    shg[j] = w.sg[q0 + j];
                }
                __syncthreads();
                if (valid) {
                    for (int j = 0; j < m; ++j) {
                        double ax = xt - shx[j], ay = yt - shy[j];
                        double r2 = ax * ax + ay * ay;
                        if (r2 > 0.0) {
                            double f = -expm1(-r2 * k2) / r2 * shg[j];
                            au -= ay * f;
                            av += ax * f;
                        }
                    }
                }
            }
        }
        if (valid)
            w.near64[tpos] = make_double2(au / TWO_PI, av / TWO_PI);
    }
}

// ------------------------------------------------------------------ precision form

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase with the given parity; gives up after a bounded number of polls (each try_wait may also
// suspend the thread for a short, hardware-defined time) and reports a timeout in the status word instead of
// hanging.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned int *status,
                                                  int polls = 1 << 20)
{
    for (int it = 0; it < polls; ++it)
        if (mbar_try_wait(bar, parity))
            return true;
    atomicOr(status, FMM_DEV_TIMEOUT);
    return false;
}

// Self-test of the timeout path: one thread initialises an mbarrier that expects one arrival, never arrives and
// never starts a copy, then waits on it with the bounded wait above, so the wait runs out after `polls` polls and
// the status word gets the timeout bit. Nothing is in flight when the kernel returns.
__global__ void k_wait_timeout_selftest(unsigned int *status, int polls)
{
    __shared__ __align__(8) uint64_t bar;
    mbar_init(&bar, 1);
    fence_proxy_async();
    mbar_wait_bounded(&bar, 0, status, polls);
}

int launch_wait_timeout_selftest(const Work &w, int polls, cudaStream_t s)
{
    k_wait_timeout_selftest<<<1, 1, 0, s>>>(w.status, polls);
    return 1;
}

// Packed FP32 pairs (one 64-bit register pair, two targets): sm_100-class f32x2 arithmetic.
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk2(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void up2(f2 v, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// In units where r'^2 is the exponent of 2: exp(-r^2 / 2 sigma^2) = 2^-(r'^2), y = r'^2 ln 2. Below y = 1/2
// the factor (1 - e^-y)/y comes from the product form of small_q2 below: 1 - 2^-(r'^2) from the SFU loses
// 2^-22.5 / y of its relative accuracy there. r' = 0 (a particle and itself, or coincident particles, which
// always share a leaf) needs no special factor: with 1/r'^2 clamped, g (1 - e) / r'^2 = 0 exactly.
#define P2P_THR 0.72134752044448170f
#define P2P_RMIN2 0x1p-16f  // floor of r'^2 in the plain factor of tested pairs (the series replaces it below P2P_THR)
#define P2P_LN2 0.69314718055994531f
#ifndef P2P_UNROLL
#define P2P_UNROLL 1  // source loop unroll of the near-field kernel
#endif
#ifndef P2P_MIN_BLOCKS
#define P2P_MIN_BLOCKS 18  // minimum resident blocks per SM requested from the register allocator (56 registers)
#endif
#ifndef P2P_MIN_BLOCKS2
#define P2P_MIN_BLOCKS2 24  // the same for the two-targets-per-lane instance (40 registers)
#endif
#ifndef P2P_TILE2
#define P2P_TILE2 288  // sources per shared-memory tile of the two-per-lane instance (one-float coordinates)
#endif
#ifndef P2P_TILE4
#define P2P_TILE4 448  // the same with four leaves per block (a row of six source leaves)
#endif
constexpr int kP2PUnroll = P2P_UNROLL;

// (1 - 2^-a) / a for both halves of a packed pair a = r'^2 below the series threshold, written as
// ln2 * 2^(-a/2) * sinh(t) / t with t = a ln2 / 2 <= 1/4 (the identity 1 - e^-y = 2 e^(-y/2) sinh(y/2)): the SFU's
// 2^(-a/2) keeps its relative accuracy (no cancellation), and sinh(t)/t = sum_k t^(2k) / (2k+1)! to t^6 truncates
// below 5e-11. Coefficients: ln2 (ln2/2)^(2k) / (2k+1)!, k = 0..3, a polynomial in a^2.
#define P2P_SQ0 6.931471806e-01f
#define P2P_SQ1 1.387602717e-02f
#define P2P_SQ2 8.333473842e-05f
#define P2P_SQ3 2.383239657e-07f
__device__ __forceinline__ f2 small_q2(f2 r2)
{
    float ra, rb;
    up2(r2, ra, rb);
    const f2 h = pk2(ex2_approx(-0.5f * ra), ex2_approx(-0.5f * rb));
    const f2 v = mul2(r2, r2);
    f2 t = fma2(v, pk2(P2P_SQ3, P2P_SQ3), pk2(P2P_SQ2, P2P_SQ2));
    t = fma2(v, t, pk2(P2P_SQ1, P2P_SQ1));
    t = fma2(v, t, pk2(P2P_SQ0, P2P_SQ0));
    return mul2(h, t);
}

// Error-free packed sum: s + c += x (Knuth's TwoSum on both halves).
__device__ __forceinline__ void two_sum2(f2 &s, f2 &c, f2 x)
{
    f2 t = add2(s, x);
    f2 bp = sub2(t, s);
    f2 e = add2(sub2(s, sub2(t, bp)), sub2(x, bp));
    c = add2(c, e);
    s = t;
}

// Sources j0..j1 of one source leaf against KT targets per lane (KT/2 packed pairs), accumulated into PU, PV.
// The lane's targets (entries lane + 32 q, q < KT, only those < tcnt, of the pass's staged targets TT: x hi, x lo,
// y hi, y lo) are re-expressed relative to the source leaf's centre: hi - dc s by Fast2Sum (|dc s| >= |hi|), error
// into lo.
// SPLIT keeps the sources' lo parts (differences at FP64-level resolution); otherwise each coordinate is one
// float (the target's rounded once from its exact shifted hi + lo) and a difference costs one instruction.
// Only sources j0..t1 and ja..jb are tested for small r and take the exponential (the targets' own leaf: all of
// them); the others lie more than 6 sigma from every target (outside the band of their leaf that faces the
// targets' leaf), where 1 - exp(-r^2 / 2 sigma^2) is 1 in FP32, and run without either: [t1, ja) and [jb, j1)
// first, then the band.
template <int KT, bool SELF, bool SPLIT>
__device__ __forceinline__ void p2p_segment(const Work &w, const float4 *__restrict__ EH,
                                            const float4 *__restrict__ EL, const float4 *__restrict__ EG, int j0,
                                            int j1, int t1, int ja, int jb, float sdx, float sdy,
                                            const float4 *__restrict__ TT, int tcnt, f2 *PU, f2 *PV)
{
    constexpr int NP = KT / 2;
    const int lane = threadIdx.x & 31;
    f2 AHX[NP], ALX[NP], AHY[NP], ALY[NP];
#pragma unroll
    for (int pr = 0; pr < NP; ++pr) {
        float hx[2], lx[2], hy[2], ly[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = lane + 32 * (2 * pr + h);
            const float4 t = e < tcnt ? TT[e] : make_float4(0.f, 0.f, 0.f, 0.f);
            hx[h] = t.x - sdx;
            lx[h] = t.y + (t.x - (hx[h] + sdx));
            hy[h] = t.z - sdy;
            ly[h] = t.w + (t.z - (hy[h] + sdy));
            if (!SPLIT) {
                hx[h] += lx[h];
                hy[h] += ly[h];
            }
        }
        AHX[pr] = pk2(hx[0], hx[1]);
        AHY[pr] = pk2(hy[0], hy[1]);
        if (SPLIT) {
            ALX[pr] = pk2(lx[0], lx[1]);
            ALY[pr] = pk2(ly[0], ly[1]);
        }
    }
    // One source against the lane's targets; `tst` (a std::bool_constant) selects the small-r test. Every pair
    // first takes the plain factor g (1 - e) / r'^2, with r'^2 clamped below at P2P_RMIN2 where it is tested (so
    // that it stays bounded: (1 - e) / r'^2 <= ln 2 + 2^-22 / P2P_RMIN2); for the rare warp with a pair at
    // 0 < r < sigma the source is re-read, the plain factor recomputed bit for bit and replaced by the series
    // through the difference, so none of the series' registers are live on the common path.
    auto plain = [&](int j, auto tst, f2 *dx, f2 *dy, f2 *r2, f2 *gf) {
        constexpr bool TEST = decltype(tst)::value;
        const float4 h = EH[j], g = EG[j], l = SPLIT ? EL[j] : h;
        const f2 sxh = pk2(h.x, h.y), syh = pk2(h.z, h.w);
        const f2 gp = pk2(g.x, g.y), gn = pk2(g.z, g.w);
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
            if (SPLIT) {
                dx[pr] = add2(sub2(AHX[pr], sxh), sub2(ALX[pr], pk2(l.x, l.y)));
                dy[pr] = add2(sub2(AHY[pr], syh), sub2(ALY[pr], pk2(l.z, l.w)));
            } else {
                dx[pr] = sub2(AHX[pr], sxh);
                dy[pr] = sub2(AHY[pr], syh);
            }
            r2[pr] = fma2(dx[pr], dx[pr], mul2(dy[pr], dy[pr]));
            float ra, rb;
            up2(r2[pr], ra, rb);
            if (TEST) {
                const float ea = ex2_approx(-ra), eb = ex2_approx(-rb);
                const f2 q = pk2(rcp_approx(fmaxf(ra, P2P_RMIN2)), rcp_approx(fmaxf(rb, P2P_RMIN2)));
                gf[pr] = mul2(fma2(pk2(ea, eb), gn, gp), q);  // g (1 - e) / r'^2
            } else {
                // outside the bands r > 6 sigma: e < 2^-25, and 1 - e is 1 in FP32
                gf[pr] = mul2(gp, pk2(rcp_approx(ra), rcp_approx(rb)));  // g / r'^2
            }
        }
    };
    auto source = [&](int j, auto tst) {
        constexpr bool TEST = decltype(tst)::value;
        f2 dx[NP], dy[NP], r2[NP], gf[NP];
        plain(j, tst, dx, dy, r2, gf);
        bool close = false;
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
            float ra, rb;
            up2(r2[pr], ra, rb);
            if (SELF)  // r' = 0 (a particle and itself) needs nothing: (1 - e) = 0 exactly; as unsigned, the bit
                       // pattern minus one maps it to the largest value
                close |= (__float_as_uint(ra) - 1u < __float_as_uint(P2P_THR)) |
                         (__float_as_uint(rb) - 1u < __float_as_uint(P2P_THR));
            else if (TEST)
                close |= (ra < P2P_THR) | (rb < P2P_THR);
            PU[pr] = fma2(dy[pr], gf[pr], PU[pr]);  // u accumulates -dy g f: negated at the end
            PV[pr] = fma2(dx[pr], gf[pr], PV[pr]);
        }
        // rare (0 < r < sigma): warp-uniform branch to the series, off the common path
        if (TEST && __any_sync(0xffffffffu, close)) {
            plain(j, tst, dx, dy, r2, gf);
            const float gs = EG[j].x;
#pragma unroll
            for (int pr = 0; pr < NP; ++pr) {
                float ra, rb, fa, fb, sa, sb;
                up2(r2[pr], ra, rb);
                up2(gf[pr], fa, fb);
                up2(small_q2(r2[pr]), sa, sb);
                const float da = ra < P2P_THR ? fmaf(gs, sa, -fa) : 0.f;
                const float db = rb < P2P_THR ? fmaf(gs, sb, -fb) : 0.f;
                const f2 dd = pk2(da, db);  // series minus plain (zero where r' = 0: dx = dy = 0)
                PU[pr] = fma2(dy[pr], dd, PU[pr]);
                PV[pr] = fma2(dx[pr], dd, PV[pr]);
            }
        }
    };
    if (!SELF) {
        int lo = t1, hi = ja;
#pragma unroll 1
        for (int ph = 0; ph < 2; ++ph) {
#pragma unroll(kP2PUnroll)
            for (int j = lo; j < hi; ++j)
                source(j, std::false_type{});
            lo = jb;
            hi = j1;
        }
    }
    int lo = j0, hi = t1;
#pragma unroll 1
    for (int ph = 0; ph < 2; ++ph) {
#pragma unroll(kP2PUnroll)
        for (int j = lo; j < hi; ++j)
            source(j, std::true_type{});
        lo = ja;
        hi = jb;
    }
}

// The remainder of a pass: r targets spread over the warp's 64 slots (slot s = lane + 32 h, h = 0, 1, one half of
// a packed pair each). Slot s takes target s mod r and the sources j0 + s / r + G k, k = 0, 1, ... (G = 64 / r
// source groups), so a few leftover targets keep every lane busy for 1/G of the sources instead of all lanes
// busy for all of them; slots s >= G r carry zero charge. One-float coordinates only (not the split form).
// The slot geometry is recomputed per call (it is cheap) so that nothing of it stays live across the tile loop.
struct RemSlots {
    int e[2], g[2];  // per half: target position in leaf order, source group
    bool a[2];       // per half: slot in use
    int G;
    __device__ __forceinline__ RemSlots(int rbase, int r)  // rbase: first remainder target in the staged copy
    {
        const int lane = threadIdx.x & 31;
        G = 64 / r;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int sl = lane + 32 * h;
            a[h] = sl < G * r;
            e[h] = rbase + (a[h] ? sl % r : 0);
            g[h] = a[h] ? sl / r : 0;
        }
    }
};

template <bool SELF>
__device__ __forceinline__ void p2p_segment_rem(const float4 *__restrict__ EH, const float4 *__restrict__ EG,
                                                int j0, int j1, float sdx, float sdy,
                                                const float4 *__restrict__ TT, int rbase, int r, f2 &PU, f2 &PV)
{
    const RemSlots R(rbase, r);
    float hx[2], hy[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float4 t = TT[R.e[h]];
        const float ax = t.x - sdx, ay = t.z - sdy;
        hx[h] = ax + (t.y + (t.x - (ax + sdx)));
        hy[h] = ay + (t.w + (t.z - (ay + sdy)));
    }
    const f2 AX = pk2(hx[0], hx[1]), AY = pk2(hy[0], hy[1]);
    const int G = R.G;
    for (int b = j0; b < j1; b += G) {
        const int ja = b + R.g[0], jb = b + R.g[1];
        const bool va = R.a[0] && ja < j1, vb = R.a[1] && jb < j1;
        const float4 ha = EH[va ? ja : j0], hb = EH[vb ? jb : j0];
        const float ga = va ? EG[ja].x : 0.f, gb = vb ? EG[jb].x : 0.f;
        const f2 dx = sub2(AX, pk2(ha.x, hb.x)), dy = sub2(AY, pk2(ha.z, hb.z));
        const f2 r2 = fma2(dx, dx, mul2(dy, dy));
        float ra, rb;
        up2(r2, ra, rb);
        const float ea = ex2_approx(-ra), eb = ex2_approx(-rb);
        f2 q;
        float rmin;
        if (SELF) {
            q = pk2(rcp_approx(fmaxf(ra, 1e-30f)), rcp_approx(fmaxf(rb, 1e-30f)));
            rmin = __uint_as_float(min(__float_as_uint(ra) - 1u, __float_as_uint(rb) - 1u));
        } else {
            q = pk2(rcp_approx(ra), rcp_approx(rb));
            rmin = fminf(ra, rb);
        }
        f2 og = fma2(pk2(ea, eb), pk2(-ga, -gb), pk2(ga, gb));  // g (1 - e)
        if (__any_sync(0xffffffffu, SELF ? (__float_as_uint(rmin) < __float_as_uint(P2P_THR)) : (rmin < P2P_THR))) {
            float qa, qb, oa, ob, sa, sb;
            up2(q, qa, qb);
            up2(og, oa, ob);
            up2(small_q2(r2), sa, sb);
            if (ra < P2P_THR) {
                qa = sa;
                oa = ga;
            }
            if (rb < P2P_THR) {
                qb = sb;
                ob = gb;
            }
            q = pk2(qa, qb);
            og = pk2(oa, ob);
        }
        const f2 gf = mul2(og, q);
        PU = fma2(dy, gf, PU);  // u accumulates -dy g f: negated at the end
        PV = fma2(dx, gf, PV);
    }
}

// LPB leaves per block (1, 2 or 4, one warp each; with 2 or 4 the leaves are consecutive in one row and share
// their 3 x (LPB + 2) source neighbourhood). Each warp takes its leaf's targets in passes of at most 32 * ktmax. With
// ktmax = 4 (one-float coordinates) the passes hold 128 targets, four per lane, except the last: from 97 targets
// on it is the same, otherwise a main group of up to 64 targets, two per lane, every lane meeting the same source,
// plus the rest (r <= 32 after a full main group, or a whole pass of r <= 32) spread over the 64 slots with
// G = 64 / r source groups (p2p_segment_rem); the G partial sums of each remainder target are added at the end.
// With ktmax = 2 (a second instance, KTM = 2, compiled for fewer registers and so more warps per SM) a pass holds
// either a main group of up to 64 targets or a remainder of at most 32, never both, so one set of accumulators is
// live; in the split form passes are balanced, at most 64 targets, two per lane. Sources arrive by bulk copies into
// shared memory; each slot's sum over one tile (plain FP32) is added to its total with an error-free TwoSum.
// Register budget of the two instances (minimum resident blocks per SM, of 64 threads; of 128 with four leaves).
template <int LPB, int KTM>
struct P2PBounds {
    static constexpr int threads = LPB == 4 ? 128 : 64;
    static constexpr int min_blocks = (KTM == 4 ? P2P_MIN_BLOCKS : P2P_MIN_BLOCKS2) / (LPB == 4 ? 2 : 1);
};

template <int LPB, int KTM>
__global__ void __launch_bounds__(P2PBounds<LPB, KTM>::threads, P2PBounds<LPB, KTM>::min_blocks)
    k_p2p32(Work w, int tile, int ktmax, int skip_plain)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int4 segtab[LPB][3];  // per warp, per source column of the current row: first, end, band first, end
    __shared__ int segt1[LPB][3];    // the same: end of a second band run at the leaf's front (empty but above)
    // EH, EG, then EL (only the split form reads EL, so one-float launches allocate 32 bytes per source), then
    // each warp's targets of the current pass (p2p_smem_bytes)
    float4 *EH = reinterpret_cast<float4 *>(smem_raw), *EG = EH + tile, *EL = EG + tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *TT = EH + (size_t)tile * (w.p2p_all_plain ? 2 : 3) + warp * (KTM == 4 ? 128 : 64);
    const int first = blockIdx.x * LPB;
    if (first >= w.nleaf)
        return;
    const int k = w.nsys == 1 ? 0 : find_sys_by_leaf(w.sys, w.nsys, first);
    const SysDev &d = w.sys[k];
    const int L = d.depth, ns = 1 << L, local0 = first - (int)d.leaf0;
    const int ix0 = local0 & (ns - 1), iy = local0 >> L;
    const int myleaf = first + warp;
    const int my_s0 = w.start[myleaf], my_c = w.start[myleaf + 1] - my_s0;
    const bool split = d.s_unit > P2P_SPLIT_S;  // block-uniform; the split form runs 2 targets per lane
    if (skip_plain && !split)
        return;  // this system's near field is the symmetric kernel's
    (void)ktmax;
    const bool rem_form = !split;
    const bool bands = w.cls_off != nullptr && d.bnd_ok;  // leaves ordered by boundary class (block-uniform)
    // passes: KTM = 4, 128 targets (the last one the rest); KTM = 2, 64 targets, then the rest as one pass
    // (a main group of 33..63, or a remainder of at most 32); split form: balanced passes of at most 64
    const int full_pass = KTM == 4 ? 128 : 64;
    const int per_pass = rem_form ? full_pass : 64;
    int npass = (my_c + per_pass - 1) / per_pass;
#pragma unroll
    for (int q = 1; q < LPB; ++q) {  // the block runs as many passes as its fullest leaf needs
        const int other = first + (warp ^ q);
        const int oc = w.start[other + 1] - w.start[other];
        npass = max(npass, (oc + per_pass - 1) / per_pass);
    }
    if (npass == 0)
        return;  // block-uniform: every leaf of the block is empty
    const int my_np = (my_c + per_pass - 1) / per_pass;
    // the remainder's accumulators: a slot pair of their own where a pass holds both groups (KTM = 4), the main
    // group's where a pass holds one or the other (KTM = 2: one accumulator set live)
    constexpr int RI = KTM == 4 ? 1 : 0;
    const float s = d.s_unit;
    const int c_lo = ix0 - 1, ncol = LPB + 2;  // block columns c_lo .. c_lo + ncol - 1
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_proxy_async();
    }
    __syncthreads();
    uint32_t phase = 0;
    for (int pass = 0; pass < npass; ++pass) {
        int t_lo = 0, t_cnt = 0;
        if (pass < my_np) {
            if (rem_form) {  // full passes, the rest in the last
                t_lo = full_pass * pass;
                t_cnt = min(full_pass, my_c - t_lo);
            } else {  // balanced passes
                t_lo = (int)((int64_t)pass * my_c / my_np);
                t_cnt = (int)((int64_t)(pass + 1) * my_c / my_np) - t_lo;
            }
        }
        const int tbase = my_s0 + t_lo;
        // the pass's targets, staged once (x hi, x lo, y hi, y lo): every segment re-reads them
        __syncwarp();
        for (int e = lane; e < full_pass; e += 32) {
            float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e < t_cnt) {
                const float4 th = w.eh[tbase + e], tl = w.el[tbase + e];
                t = make_float4(th.x, tl.x, th.z, tl.z);
            }
            TT[e] = t;
        }
        __syncwarp();
        // layout of the pass: more than 96 targets, four per lane (two packed pairs, broadcast sources); else a
        // main group of up to 64, two per lane, and a remainder of at most 32 over the slots (source groups); a
        // pass of 33..63 targets is all main group, one of at most 32 all remainder
        const bool kt4 = KTM == 4 && rem_form && t_cnt > 96;
        const int n_main = !rem_form || kt4 ? t_cnt : (t_cnt >= 64 ? 64 : (t_cnt > 32 ? t_cnt : 0));
        const int r = t_cnt - n_main;  // KTM = 2: n_main and r are never both non-zero
        f2 SU[2] = {0ull, 0ull}, CU[2] = {0ull, 0ull}, SV[2] = {0ull, 0ull}, CV[2] = {0ull, 0ull};
        for (int dyr = -1; dyr <= 1; ++dyr) {
            const int row = iy + dyr;
            if (row < 0 || row >= ns || (w.p2p_rows && dyr != (int)blockIdx.y - 1))
                continue;  // with p2p_rows each block takes one source row (blockIdx.y)
            const int rowleaf = (int)d.leaf0 + row * ns;
            const int ca = max(c_lo, 0), cz = min(c_lo + ncol - 1, ns - 1);
            const int r0 = w.start[rowleaf + ca], r1 = w.start[rowleaf + cz + 1];
            if (r1 <= r0)
                continue;
            // this warp's three source leaves of the row (columns ix-1, ix, ix+1): their sorted ranges and the part
            // tested for small r, the band facing the targets' leaf (a run of its boundary classes: a corner or a
            // side with its two corners; for the leaf above, whose facing side is cut by the cyclic class order,
            // classes 6-7 and class 0 at the front); the targets' own leaf, and systems without bands, are tested
            // throughout
            __syncwarp();
            if (lane < 3) {
                const int col = ix0 + warp - 1 + lane;
                int4 t = make_int4(0, 0, 0, 0);
                int t1 = 0;
                if (col >= 0 && col < ns) {
                    t.x = w.start[rowleaf + col];
                    t.y = w.start[rowleaf + col + 1];
                    t.z = t.x;
                    t.w = t.y;
                    t1 = t.x;
                    if (bands && !(lane == 1 && dyr == 0)) {
                        const int *o = w.cls_off + (int64_t)(rowleaf + col) * 8;  // o[k - 1]: first of class k
                        const int dir = (dyr + 1) * 3 + lane;  // source leaf at (lane - 1, dyr) from the targets'
                        const int ka = (int)((0x066004224ull >> (4 * dir)) & 15ull);
                        const int kb = (int)((0x187307355ull >> (4 * dir)) & 15ull);
                        t.z = ka == 0 ? t.x : o[ka - 1];
                        t.w = o[kb - 1];
                        if (dir == 7)
                            t1 = o[0];  // class 0 (bottom-left corner) also faces the targets' leaf below
                    }
                }
                segtab[warp][lane] = t;
                segt1[warp][lane] = t1;
            }
            __syncwarp();
            f2 PU[2] = {0ull, 0ull}, PV[2] = {0ull, 0ull};
            for (int q0 = r0; q0 < r1; q0 += tile) {
                const int m = min(tile, r1 - q0);
                __syncthreads();  // everyone is done with the previous tile
                if (threadIdx.x == 0) {
                    fence_proxy_async();
                    mbar_expect_tx(&bar, (uint32_t)m * (split ? 48u : 32u));
                    bulk_g2s(EH, w.eh + q0, (uint32_t)m * 16u, &bar);
                    bulk_g2s(EG, w.eg + q0, (uint32_t)m * 16u, &bar);
                    if (split)
                        bulk_g2s(EL, w.el + q0, (uint32_t)m * 16u, &bar);
                }
                bool ok = mbar_wait_bounded(&bar, phase, w.status);
                if (!__syncthreads_and(ok)) {
                    if (!ok)
                        mbar_wait_bounded(&bar, phase, w.status);  // let a late copy land before exiting
                    return;
                }
                phase ^= 1;
                if (t_cnt == 0)
                    continue;
#pragma unroll
                for (int k3 = 0; k3 < 3; ++k3) {
                    const int4 sg = segtab[warp][k3];  // columns ix-1, ix, ix+1 (empty outside the grid)
                    const int j0 = max(q0, sg.x) - q0, j1 = min(q0 + m, sg.y) - q0;
                    if (j0 >= j1)
                        continue;
                    const float sdx = (float)(k3 - 1) * s, sdy = (float)dyr * s;
                    const bool self = k3 == 1 && dyr == 0;
                    // tested: [j0, t1) and [ja, jb)
                    const int t1 = min(max(segt1[warp][k3] - q0, j0), j1);
                    const int ja = min(max(sg.z - q0, t1), j1), jb = max(min(sg.w - q0, j1), ja);
#define P2P_SEG(SELF, SPLIT) \
    p2p_segment<2, SELF, SPLIT>(w, EH, EL, EG, j0, j1, t1, ja, jb, sdx, sdy, TT, n_main, PU, PV)
                    if (KTM == 4 && kt4) {
                        if (self)
                            p2p_segment<KTM, true, false>(w, EH, EL, EG, j0, j1, t1, ja, jb, sdx, sdy, TT, n_main, PU,
                                                          PV);
                        else
                            p2p_segment<KTM, false, false>(w, EH, EL, EG, j0, j1, t1, ja, jb, sdx, sdy, TT, n_main,
                                                           PU, PV);
                    } else if (n_main > 0) {
                        if (split) {
                            if (self)
                                P2P_SEG(true, true);
                            else
                                P2P_SEG(false, true);
                        } else {
                            if (self)
                                P2P_SEG(true, false);
                            else
                                P2P_SEG(false, false);
                        }
                    }
#undef P2P_SEG
                    if (r > 0) {
                        if (self)
                            p2p_segment_rem<true>(EH, EG, j0, j1, sdx, sdy, TT, n_main, r, PU[RI], PV[RI]);
                        else
                            p2p_segment_rem<false>(EH, EG, j0, j1, sdx, sdy, TT, n_main, r, PU[RI], PV[RI]);
                    }
                }
                // compensated totals: plain FP32 sums cover at most one tile of sources
#pragma unroll
                for (int pr = 0; pr < (KTM == 4 ? 2 : 1); ++pr) {
                    two_sum2(SU[pr], CU[pr], PU[pr]);
                    two_sum2(SV[pr], CV[pr], PV[pr]);
                    PU[pr] = 0ull;
                    PV[pr] = 0ull;
                }
            }
        }
        const float snear = d.snear;
        float2 *dst = w.p2p_rows ? w.nearp + (int64_t)blockIdx.y * w.n : w.near32;  // rows: one row's part
        const int dstride = w.p2p_rows ? 1 : w.nf_stride;
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {  // main group: targets lane + 32 (2 pr + h); pr = 1 only with kt4
            if (pr == 1 && !kt4)
                break;
            if (n_main == 0)
                break;
            float su[2], cu[2], sv[2], cv[2];
            up2(SU[pr], su[0], su[1]);
            up2(CU[pr], cu[0], cu[1]);
            up2(SV[pr], sv[0], sv[1]);
            up2(CV[pr], cv[0], cv[1]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e = lane + 32 * (2 * pr + h);
                if (e < n_main)
                    dst[(int64_t)(tbase + e) * dstride] = make_float2(-(su[h] + cu[h]) * snear, (sv[h] + cv[h]) * snear);
            }
        }
        // remainder: the G partial sums of each target (slots t, t + r, ..., t + (G - 1) r), added in FP64 through
        // this warp's part of the (now idle) source tile
        if (__syncthreads_or(r > 0)) {
            float2 *red = reinterpret_cast<float2 *>(EH) + 64 * warp;
            if (r > 0) {
                float su[2], cu[2], sv[2], cv[2];
                up2(SU[RI], su[0], su[1]);
                up2(CU[RI], cu[0], cu[1]);
                up2(SV[RI], sv[0], sv[1]);
                up2(CV[RI], cv[0], cv[1]);
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    red[lane + 32 * h] = make_float2(su[h] + cu[h], sv[h] + cv[h]);
                __syncwarp();
                const int G = 64 / r;
                for (int t = lane; t < r; t += 32) {
                    double au = 0.0, av = 0.0;
                    for (int gq = 0; gq < G; ++gq) {
                        const float2 part = red[t + gq * r];
                        au += (double)part.x;
                        av += (double)part.y;
                    }
                    dst[(int64_t)(tbase + n_main + t) * dstride] = make_float2(-(float)au * snear, (float)av * snear);
                }
            }
            __syncthreads();  // the tile is free again before the next pass copies into it
        }
    }
}

// ------------------------------------------------------------------ precision form, symmetric near field

// Each unordered pair of particles in adjacent leaves is evaluated once and acts on both (the kernel is odd:
// K(-z) = -K(z)). A warp owns a target leaf A and visits A itself and its four "forward" neighbours
// B = A + c_p2p_fwd[d]; every other adjacent pair of leaves is some other warp's forward pair. Everything is in
// A's frame (targets rounded once from hi + lo; forward sources shifted by their leaf offset when staged).
// Sources arrive in chunks of 32, one per lane, in shared memory (A's own particles first, then the forward
// leaves' particles back to back, so only the stream's ends are padded); in step k of a chunk lane l pairs its
// KT targets with source (l + k) mod 32, so the 32 lanes meet 32 different sources, and the source's running
// reaction travels with it (one lane shuffle per step), back at its own lane after 32 steps. The reactions on
// forward particles go to nearp[d] (written by this warp only, so sums are deterministic); the final sum adds
// the four backward contributions in a fixed order. Systems whose leaves are wider than the one-float bound
// (P2P_SPLIT_S) are left to k_p2p32.
__constant__ int2 c_p2p_fwd[4] = {{1, 0}, {1, 1}, {0, 1}, {-1, 1}};

__device__ __forceinline__ f2 shfl2(f2 v, int src)
{
    return __shfl_sync(0xffffffffu, v, src);
}

// One chunk of 32 sources (SH, SG in shared memory) against the lane's KT targets. SELF: the sources are the
// targets' own leaf (r' = 0 occurs; no reaction). SYM: accumulate the reaction on the source in RU, RV and
// rotate it with the source.
template <int KT, bool SELF, bool SYM>
__device__ __forceinline__ void p2ps_chunk(const float4 *__restrict__ SH, const float4 *__restrict__ SG, int lane,
                                           const f2 *AX, const f2 *AY, const f2 *GT, const f2 *GTN, f2 *PU, f2 *PV,
                                           f2 &RU, f2 &RV)
{
    constexpr int NP = KT / 2;
#pragma unroll 1
    for (int k = 0; k < 32; ++k) {
        const int m = (lane + k) & 31;
        const float4 h = SH[m], g = SG[m];
        const f2 sxh = pk2(h.x, h.y), syh = pk2(h.z, h.w);
        const f2 gp = pk2(g.x, g.y), gn = pk2(g.z, g.w);
        f2 dx[NP], dy[NP], e[NP], q[NP], r2[NP];
        float rmin = 3.0e38f;
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
            dx[pr] = sub2(AX[pr], sxh);
            dy[pr] = sub2(AY[pr], syh);
            r2[pr] = fma2(dx[pr], dx[pr], mul2(dy[pr], dy[pr]));
            float ra, rb;
            up2(r2[pr], ra, rb);
            e[pr] = pk2(ex2_approx(-ra), ex2_approx(-rb));
            if (SELF) {
                q[pr] = pk2(rcp_approx(fmaxf(ra, 1e-30f)), rcp_approx(fmaxf(rb, 1e-30f)));
                rmin = __uint_as_float(min(__float_as_uint(rmin), min(__float_as_uint(ra) - 1u, __float_as_uint(rb) - 1u)));
            } else {
                q[pr] = pk2(rcp_approx(ra), rcp_approx(rb));
                rmin = fminf(rmin, fminf(ra, rb));
            }
        }
        // rare (0 < r < sigma): the series gives (1 - e) q directly; e := 0, q := series
        if (__any_sync(0xffffffffu, SELF ? (__float_as_uint(rmin) < __float_as_uint(P2P_THR)) : (rmin < P2P_THR))) {
#pragma unroll
            for (int pr = 0; pr < NP; ++pr) {
                float ra, rb, qa, qb, ea, eb, sa, sb;
                up2(r2[pr], ra, rb);
                up2(q[pr], qa, qb);
                up2(e[pr], ea, eb);
                up2(small_q2(r2[pr]), sa, sb);
                if (ra < P2P_THR) {
                    qa = sa;
                    ea = 0.f;
                }
                if (rb < P2P_THR) {
                    qb = sb;
                    eb = 0.f;
                }
                q[pr] = pk2(qa, qb);
                e[pr] = pk2(ea, eb);
            }
        }
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
            const f2 gf = mul2(fma2(e[pr], gn, gp), q[pr]);  // gamma_s (1 - e) q
            PU[pr] = fma2(dy[pr], gf, PU[pr]);                // u accumulates -dy g f: negated at the end
            PV[pr] = fma2(dx[pr], gf, PV[pr]);
            if (SYM) {
                const f2 gr = mul2(fma2(e[pr], GTN[pr], GT[pr]), q[pr]);  // gamma_t (1 - e) q
                RU = fma2(dy[pr], gr, RU);  // reaction on the source: u += +dy g f, v += -dx g f
                RV = fma2(dx[pr], gr, RV);
            }
        }
        if (SYM) {  // the source of step k + 1 in this lane sits in lane + 1 now
            RU = shfl2(RU, (lane + 1) & 31);
            RV = shfl2(RV, (lane + 1) & 31);
        }
    }
}

#ifndef P2PS_MIN_BLOCKS
#define P2PS_MIN_BLOCKS 6  // minimum resident 128-thread blocks per SM for the symmetric kernel (80 registers)
#endif

// Source stream of one target leaf A: A's own particles (padded to a multiple of 32), then the particles of
// its forward neighbours in order d = 0..3, shifted into A's frame when they are staged. Stream position ->
// (source index, forward direction d or -1 for A itself, or padding).
struct SymStream {
    int a0, ac, selfpad, total;
    int fb0[4], fpre[5];  // first particle of forward leaf d, prefix of their counts
    float fsx[4], fsy[4];  // shift of leaf d into A's frame (leaf offset x s)
};

__device__ __forceinline__ void stream_load(const Work &w, const SymStream &S, int pos, float4 &h, float4 &g,
                                            int &src, int &dir)
{
    src = -1;
    dir = -1;
    h = make_float4(-1.0e4f, -1.0e4f, -1.0e4f, -1.0e4f);  // padding: far away, no charge
    g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pos < S.ac) {
        src = S.a0 + pos;
        h = w.eh[src];
        g = w.eg[src];
    } else if (pos >= S.selfpad && pos < S.total) {
        const int f = pos - S.selfpad;
        // the last leaf d whose prefix is <= f (prefixes never decrease; selects keep S in registers)
        int dd = 0, fb = S.fb0[0], fp = 0;
        float sx = S.fsx[0], sy = S.fsy[0];
#pragma unroll
        for (int q = 1; q < 4; ++q)
            if (f >= S.fpre[q]) {
                dd = q;
                fb = S.fb0[q];
                fp = S.fpre[q];
                sx = S.fsx[q];
                sy = S.fsy[q];
            }
        dir = dd;
        src = fb + (f - fp);
        const float4 hb = w.eh[src];
        h = make_float4(hb.x + sx, hb.y + sx, hb.z + sy, hb.w + sy);
        g = w.eg[src];
    }
}

template <int LW>
__global__ void __launch_bounds__(32 * LW, P2PS_MIN_BLOCKS) k_p2p32s(Work w, int ktmax)
{
    __shared__ float4 sh_h[LW][32], sh_g[LW][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int A = blockIdx.x * LW + warp;
    if (A >= w.nleaf)
        return;  // warp-uniform; warps never synchronise with each other
    const int k = w.nsys == 1 ? 0 : find_sys_by_leaf(w.sys, w.nsys, A);
    const SysDev &d = w.sys[k];
    if (d.s_unit > P2P_SPLIT_S)
        return;  // split-coordinate system: k_p2p32
    const int L = d.depth, ns = 1 << L, local = A - (int)d.leaf0;
    const int ax = local & (ns - 1), ay = local >> L;
    SymStream S;
    S.a0 = w.start[A];
    S.ac = w.start[A + 1] - S.a0;
    if (S.ac == 0)
        return;
    const float s = d.s_unit, snear = d.snear;
    const int n = w.n;
    S.selfpad = (S.ac + 31) & ~31;
    S.fpre[0] = 0;
#pragma unroll
    for (int dd = 0; dd < 4; ++dd) {
        const int2 o = c_p2p_fwd[dd];
        const int bx = ax + o.x, by = ay + o.y;
        int cnt = 0, b0 = 0;
        if (bx >= 0 && bx < ns && by < ns) {
            const int B = (int)d.leaf0 + by * ns + bx;
            b0 = w.start[B];
            cnt = w.start[B + 1] - b0;
        }
        S.fb0[dd] = b0;
        S.fpre[dd + 1] = S.fpre[dd] + cnt;
        S.fsx[dd] = (float)o.x * s;
        S.fsy[dd] = (float)o.y * s;
    }
    S.total = S.selfpad + S.fpre[4];
    float4 *SH = sh_h[warp], *SG = sh_g[warp];
    const int per_pass = 32 * ktmax;
    const int np = (S.ac + per_pass - 1) / per_pass;
    for (int pass = 0; pass < np; ++pass) {
        const int t_lo = (int)((int64_t)pass * S.ac / np);
        const int t_cnt = (int)((int64_t)(pass + 1) * S.ac / np) - t_lo;
        const int kt = t_cnt <= 64 ? 2 : 4;
        const int tbase = S.a0 + t_lo;
        // the lane's targets in A's frame, one float per coordinate; charges (and negated) per packed pair
        f2 AX[2], AY[2], GT[2], GTN[2];
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
            float hx[2], hy[2], gv[2];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int e = lane + 32 * (2 * pr + hh);
                if (e < t_cnt) {
                    const float4 th = w.eh[tbase + e], tl = w.el[tbase + e];
                    hx[hh] = th.x + tl.x;
                    hy[hh] = th.z + tl.z;
                    gv[hh] = w.eg[tbase + e].x;
                } else {
                    hx[hh] = 1.0e4f;  // padding target: far away, no charge
                    hy[hh] = 1.0e4f;
                    gv[hh] = 0.f;
                }
            }
            AX[pr] = pk2(hx[0], hx[1]);
            AY[pr] = pk2(hy[0], hy[1]);
            GT[pr] = pk2(gv[0], gv[1]);
            GTN[pr] = pk2(-gv[0], -gv[1]);
        }
        f2 SU[2] = {0ull, 0ull}, CU[2] = {0ull, 0ull}, SV[2] = {0ull, 0ull}, CV[2] = {0ull, 0ull};
        float4 nh, ng;
        int nsrc, ndir;
        stream_load(w, S, lane, nh, ng, nsrc, ndir);
        for (int c0 = 0; c0 < S.total; c0 += 32) {
            const int src = nsrc, dir = ndir;
            __syncwarp();  // the previous chunk is no longer read
            SH[lane] = nh;
            SG[lane] = ng;
            __syncwarp();
            if (c0 + 32 < S.total)
                stream_load(w, S, c0 + 32 + lane, nh, ng, nsrc, ndir);  // next chunk, in flight meanwhile
            f2 PU[2] = {0ull, 0ull}, PV[2] = {0ull, 0ull}, RU = 0ull, RV = 0ull;
            if (c0 < S.selfpad) {
                if (kt == 2)
                    p2ps_chunk<2, true, false>(SH, SG, lane, AX, AY, GT, GTN, PU, PV, RU, RV);
                else
                    p2ps_chunk<4, true, false>(SH, SG, lane, AX, AY, GT, GTN, PU, PV, RU, RV);
            } else {
                if (kt == 2)
                    p2ps_chunk<2, false, true>(SH, SG, lane, AX, AY, GT, GTN, PU, PV, RU, RV);
                else
                    p2ps_chunk<4, false, true>(SH, SG, lane, AX, AY, GT, GTN, PU, PV, RU, RV);
                if (dir >= 0) {  // reaction on this lane's source (pass 0 writes, later passes add)
                    float ru0, ru1, rv0, rv1;
                    up2(RU, ru0, ru1);
                    up2(RV, rv0, rv1);
                    float2 r = make_float2((ru0 + ru1) * snear, -(rv0 + rv1) * snear);
                    float2 *dst = w.nearp + (int64_t)dir * n + src;
                    if (pass > 0) {
                        const float2 old = *dst;
                        r.x += old.x;
                        r.y += old.y;
                    }
                    *dst = r;
                }
            }
#pragma unroll
            for (int pr = 0; pr < 2; ++pr) {
                two_sum2(SU[pr], CU[pr], PU[pr]);
                two_sum2(SV[pr], CV[pr], PV[pr]);
            }
        }
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
            float su[2], cu[2], svv[2], cv[2];
            up2(SU[pr], su[0], su[1]);
            up2(CU[pr], cu[0], cu[1]);
            up2(SV[pr], svv[0], svv[1]);
            up2(CV[pr], cv[0], cv[1]);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int e = lane + 32 * (2 * pr + hh);
                if (e < t_cnt)
                    w.near32[(int64_t)(tbase + e) * w.nf_stride] =
                        make_float2(-(su[hh] + cu[hh]) * snear, (svv[hh] + cv[hh]) * snear);
            }
        }
    }
}

// Per-device kernel attributes of the near field (once, before any stream capture): the largest shared-memory
// carveout, so that the two-per-lane instance reaches its register-limited 24 blocks per SM.
static int g_p2p_ready[64];

int prepare_p2p()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return -1;
    if (g_p2p_ready[dev])
        return 0;
    const int c = cudaSharedmemCarveoutMaxShared;
    if (cudaFuncSetAttribute(k_p2p32<1, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, c) != cudaSuccess ||
        cudaFuncSetAttribute(k_p2p32<2, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, c) != cudaSuccess ||
        cudaFuncSetAttribute(k_p2p32<1, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, c) != cudaSuccess ||
        cudaFuncSetAttribute(k_p2p32<2, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, c) != cudaSuccess)
        return -1;
    g_p2p_ready[dev] = 1;
    return 0;
}

int launch_p2p(const Work &w, int threads, int kt, cudaStream_t s)
{
    if (w.nleaf == 0)
        return 0;
    if (!w.mixed) {
        k_p2p64<<<w.nleaf, 64, 0, s>>>(w);
        return 1;
    }
    int ktmax = kt == 2 ? 2 : 4;
    int nl = 0;
    if (threads == 128 && w.p2p_sym) {
        // symmetric near field for the one-float systems; k_p2p32 only where a system may need split coordinates
        constexpr int LW = 4;
        k_p2p32s<LW><<<(w.nleaf + LW - 1) / LW, 32 * LW, 0, s>>>(w, ktmax);
        ++nl;
        if (!w.p2p_all_plain) {
            const int tile = 192;
            k_p2p32<1, 2><<<w.nleaf, 32, (size_t)tile * 48 + 64 * 16, s>>>(w, tile, 2, 1);
            ++nl;
        }
        return nl;
    }
    // shared memory per block: 32 bytes per source when every system keeps one-float coordinates, else 48; the
    // four-per-lane instance runs up to 17 blocks per SM (tile 256, 56 registers), the two-per-lane instance up to 20 (tile 288,
    // or 192 with split coordinates), where a larger tile (fewer block-wide waits) measured faster than more blocks
    const int tile = ktmax == 4 ? 256 : (w.p2p_all_plain ? P2P_TILE2 : 192);
    // plus the staged targets of a pass, 16 bytes each for up to 32 ktmax targets per warp (two warps)
    const size_t sm = (size_t)tile * (w.p2p_all_plain ? 32 : 48) + (size_t)2 * 32 * ktmax * 16;
    if (threads == 256 && w.lv.nsys_at[2] == w.nsys) {
        // four leaves per block (every system at least 4 leaves wide): a 3 x 6 source neighbourhood for four
        // target leaves, twice the warps per block at the same per-warp register budget
        const int tile4 = w.p2p_all_plain ? P2P_TILE4 : 288;
        const size_t sm4 = (size_t)tile4 * (w.p2p_all_plain ? 32 : 48) + (size_t)4 * 32 * ktmax * 16;
        if (ktmax == 4)
            k_p2p32<4, 4><<<(w.nleaf + 3) / 4, 128, sm4, s>>>(w, tile4, ktmax, 0);
        else
            k_p2p32<4, 2><<<(w.nleaf + 3) / 4, 128, sm4, s>>>(w, tile4, ktmax, 0);
        return 1;
    }
    if (threads == 192 && w.p2p_rows) {
        // the target-side kernel with each of the three source rows of a leaf pair in its own block: three
        // times the blocks at a third of the length, so the last wave leaves less of the GPU idle
        const bool pr2 = w.lv.nsys_at[1] == w.nsys;
        const dim3 grid(pr2 ? (w.nleaf + 1) / 2 : w.nleaf, 3);
        if (pr2) {
            if (ktmax == 4)
                k_p2p32<2, 4><<<grid, 64, sm, s>>>(w, tile, ktmax, 0);
            else
                k_p2p32<2, 2><<<grid, 64, sm, s>>>(w, tile, ktmax, 0);
        } else {
            if (ktmax == 4)
                k_p2p32<1, 4><<<grid, 32, sm, s>>>(w, tile, ktmax, 0);
            else
                k_p2p32<1, 2><<<grid, 32, sm, s>>>(w, tile, ktmax, 0);
        }
        return 1;
    }
    // two leaves per block needs every system's leaves to pair up within rows (depth >= 1)
    bool pairs = (threads == 64 || threads == 256) && w.lv.nsys_at[1] == w.nsys;
    if (pairs) {
        if (ktmax == 4)
            k_p2p32<2, 4><<<(w.nleaf + 1) / 2, 64, sm, s>>>(w, tile, ktmax, 0);
        else
            k_p2p32<2, 2><<<(w.nleaf + 1) / 2, 64, sm, s>>>(w, tile, ktmax, 0);
    } else {
        if (ktmax == 4)
            k_p2p32<1, 4><<<w.nleaf, 32, sm, s>>>(w, tile, ktmax, 0);
        else
            k_p2p32<1, 2><<<w.nleaf, 32, sm, s>>>(w, tile, ktmax, 0);
    }
    return 1;
}

// ------------------------------------------------------------------ adjoint near field (FP64)

// For target k and neighbour m (z = z_k - z_m), with K = (Ku, Kv) of Eq. 6 and its Jacobian J:
//   dgamma_k += -(gu_m Ku(z) + gv_m Kv(z))
//   dx_k     += (gamma_m gu_k - gamma_k gu_m) dKu/da + (gamma_m gv_k - gamma_k gv_m) dKv/da
//   dy_k     += (gamma_m gu_k - gamma_k gu_m) dKu/db + (gamma_m gv_k - gamma_k gv_m) dKv/db
// (K is odd and its Jacobian even in z). Writes the near part in caller order (the far part is added later).
__global__ void __launch_bounds__(64) k_adjoint_p2p64(Work w, double *__restrict__ odg, double *__restrict__ odx,
                                                     double *__restrict__ ody, int skip_plain)
{
    __shared__ double shx[256], shy[256], shg[256], shu[256], shv[256];
    int leaf = blockIdx.x;
    int s0 = w.start[leaf], c = w.start[leaf + 1] - s0;
    if (c == 0)
        return;
    int k = w.nsys == 1 ? 0 : find_sys_by_leaf(w.sys, w.nsys, leaf);
    const SysDev &d = w.sys[k];
    if (skip_plain && !(d.s_unit > P2P_SPLIT_S))
        return;  // this system's near field is the FP32 kernel's
    int L = d.depth, ns = 1 << L, local = leaf - (int)d.leaf0;
    int ix = local & (ns - 1), iy = local >> L;
    double k2 = 1.0 / (2.0 * d.sigma * d.sigma);
    int jx0 = ix > 0 ? ix - 1 : 0, jx1 = ix < ns - 1 ? ix + 1 : ns - 1;
    for (int t0 = 0; t0 < c; t0 += blockDim.x) {
        int tpos = s0 + t0 + threadIdx.x;
        bool valid = t0 + threadIdx.x < c;
        double xt = 0, yt = 0, gt = 0, gut = 0, gvt = 0;
        if (valid) {
            xt = w.sx[tpos];
            yt = w.sy[tpos];
            gt = w.sg[tpos];
            gut = w.sgu[tpos];
            gvt = w.sgv[tpos];
        }
        double ag = 0, ax = 0, ay = 0;
        for (int dy = -1; dy <= 1; ++dy) {
            int row = iy + dy;
            if (row < 0 || row >= ns)
                continue;
            int r0 = w.start[d.leaf0 + row * ns + jx0], r1 = w.start[d.leaf0 + row * ns + jx1 + 1];
            for (int q0 = r0; q0 < r1; q0 += 256) {
                int m = min(256, r1 - q0);
                __syncthreads();
                for (int j = threadIdx.x; j < m; j += blockDim.x) {
                    shx[j] = w.sx[q0 + j];
                    shy[j] = w.sy[q0 + j];
                    shg[j] = w.sg[q0 + j];
                    shu[j] = w.sgu[q0 + j];
                    shv[j] = w.sgv[q0 + j];
                }
                __syncthreads();
                if (!valid)
                    continue;
                for (int j = 0; j < m; ++j) {
                    double a = xt - shx[j], b = yt - shy[j];
                    double s = a * a + b * b;
                    if (s == 0.0)
                        continue;
                    double e = exp(-s * k2);
                    double om = -expm1(-s * k2);
                    double f = om / (TWO_PI * s);
                    double fp = (k2 * e * s - om) / (TWO_PI * s * s);
                    double ku = -b * f, kv = a * f;
                    double J0 = -2.0 * a * b * fp, J1 = -(f + 2.0 * b * b * fp);
                    double J2 = f + 2.0 * a * a * fp, J3 = 2.0 * a * b * fp;
                    double cu = shg[j] * gut - gt * shu[j], cv = shg[j] * gvt - gt * shv[j];
                    ag -= shu[j] * ku + shv[j] * kv;
                    ax += cu * J0 + cv * J2;
                    ay += cu * J1 + cv * J3;
                }
            }
        }
        if (valid) {
            int i = w.perm[tpos];
            if (odg)
                odg[i] = ag;
            if (odx)
                odx[i] = ax;
            if (ody)
                ody[i] = ay;
        }
    }
}

// Precision form of the same near-field adjoint. Lengths in units r' = lambda r, lambda = s / w_L, with s the
// system's s_unit, so that exp(-r^2 / 2 sigma^2) = 2^-(r'^2) (the forward's units); F(t) = (1 - 2^-t) / t and
// F'(t) at t = r'^2 give, with C = lambda * snear (snear = lambda / 2 pi):
//   Ku = -b' F snear,  Kv = a' F snear,
//   dKu/da = -2 a'b' F' C,  dKu/db = -(F + 2 b'^2 F') C,  dKv/da = (F + 2 a'^2 F') C,  dKv/db = 2 a'b' F' C,
// F' = (ln2 2^-t - F) / t. Below t = 1/(2 ln2) both come from series in y = t ln2 (g(y) = (1 - e^-y)/y and
// g'(y), the terms of their Taylor series, F = ln2 g, F' = ln2^2 g'), behind a warp-uniform branch. Coordinates
// relative to the target leaf's centre, formed in FP64 and rounded once to FP32 (|a'| <= 1.5 s); one target per
// thread, sources staged per row of leaves in shared memory as FP32; FP32 sums per row, FP64 across rows.
__device__ __forceinline__ void adj_small(float t, float &F, float &Fp)
{
    const float y = t * P2P_LN2;
    // g(y) = sum_k (-y)^k / (k+1)!, g'(y) = sum_{k>=1} k (-y)^(k-1) (-1) / (k+1)!, to y^8
    float g = 1.0f / 362880.0f;
    g = fmaf(g, -y, 1.0f / 40320.0f);
    g = fmaf(g, -y, 1.0f / 5040.0f);
    g = fmaf(g, -y, 1.0f / 720.0f);
    g = fmaf(g, -y, 1.0f / 120.0f);
    g = fmaf(g, -y, 1.0f / 24.0f);
    g = fmaf(g, -y, 1.0f / 6.0f);
    g = fmaf(g, -y, 0.5f);
    g = fmaf(g, -y, 1.0f);
    float d = -9.0f / 3628800.0f;
    d = fmaf(d, y, 8.0f / 362880.0f);
    d = fmaf(d, y, -7.0f / 40320.0f);
    d = fmaf(d, y, 6.0f / 5040.0f);
    d = fmaf(d, y, -5.0f / 720.0f);
    d = fmaf(d, y, 4.0f / 120.0f);
    d = fmaf(d, y, -3.0f / 24.0f);
    d = fmaf(d, y, 2.0f / 6.0f);
    d = fmaf(d, y, -0.5f);
    F = P2P_LN2 * g;
    Fp = (P2P_LN2 * P2P_LN2) * d;
}

#define ADJ_TILE 256

__global__ void __launch_bounds__(64) k_adjoint_p2p32(Work w, double *__restrict__ odg, double *__restrict__ odx,
                                                      double *__restrict__ ody)
{
    __shared__ float shx[ADJ_TILE], shy[ADJ_TILE], shg[ADJ_TILE], shu[ADJ_TILE], shv[ADJ_TILE];
    const int leaf = blockIdx.x;
    const int s0 = w.start[leaf], c = w.start[leaf + 1] - s0;
    if (c == 0)
        return;
    const int k = w.nsys == 1 ? 0 : find_sys_by_leaf(w.sys, w.nsys, leaf);
    const SysDev &d = w.sys[k];
    if (d.s_unit > P2P_SPLIT_S)
        return;  // leaves wider than the one-float bound: the FP64 kernel
    const int L = d.depth, ns = 1 << L, local = leaf - (int)d.leaf0;
    const int ix = local & (ns - 1), iy = local >> L;
    const double lam = (double)d.s_unit / d.wl;
    const double cx = d.x0 + (ix + 0.5) * d.wl, cy = d.y0 + (iy + 0.5) * d.wl;
    const float snear = d.snear, C = (float)(lam * (double)d.snear);
    const int jx0 = ix > 0 ? ix - 1 : 0, jx1 = ix < ns - 1 ? ix + 1 : ns - 1;
    for (int t0 = 0; t0 < c; t0 += blockDim.x) {
        const int tpos = s0 + t0 + threadIdx.x;
        const bool valid = t0 + threadIdx.x < c;
        float xt = 0.f, yt = 0.f, gt = 0.f, gut = 0.f, gvt = 0.f;
        if (valid) {
            xt = (float)((w.sx[tpos] - cx) * lam);
            yt = (float)((w.sy[tpos] - cy) * lam);
            gt = (float)w.sg[tpos];
            gut = (float)w.sgu[tpos];
            gvt = (float)w.sgv[tpos];
        }
        double ag = 0.0, ax = 0.0, ay = 0.0;
        for (int dyr = -1; dyr <= 1; ++dyr) {
            const int row = iy + dyr;
            if (row < 0 || row >= ns)
                continue;
            const int r0 = w.start[d.leaf0 + row * ns + jx0], r1 = w.start[d.leaf0 + row * ns + jx1 + 1];
            float pg = 0.f, px = 0.f, py = 0.f;
            for (int q0 = r0; q0 < r1; q0 += ADJ_TILE) {
                const int m = min(ADJ_TILE, r1 - q0);
                __syncthreads();
                for (int j = threadIdx.x; j < m; j += blockDim.x) {
                    shx[j] = (float)((w.sx[q0 + j] - cx) * lam);
                    shy[j] = (float)((w.sy[q0 + j] - cy) * lam);
                    shg[j] = (float)w.sg[q0 + j];
                    shu[j] = (float)w.sgu[q0 + j];
                    shv[j] = (float)w.sgv[q0 + j];
                }
                __syncthreads();
                for (int j = 0; j < m; ++j) {
                    const float a = xt - shx[j], b = yt - shy[j];
                    const float t = fmaf(a, a, b * b);
                    const float e = ex2_approx(-t), q = rcp_approx(fmaxf(t, 1e-30f));
                    float F = (1.0f - e) * q;
                    float Fp = fmaf(P2P_LN2, e, -F) * q;
                    if (__any_sync(0xffffffffu, t < P2P_THR)) {
                        if (t < P2P_THR) {
                            float Fs, Fps;
                            adj_small(t, Fs, Fps);
                            F = Fs;
                            Fp = Fps;
                        }
                    }
                    if (t > 0.f) {  // a particle and itself, or coincident particles: K = 0
                        // dgamma_k -= gu_m Ku + gv_m Kv = F (gu_m b' - gv_m a') (times snear)
                        pg = fmaf(F, fmaf(shu[j], b, -shv[j] * a), pg);
                        const float cu = fmaf(shg[j], gut, -gt * shu[j]), cv = fmaf(shg[j], gvt, -gt * shv[j]);
                        const float A = 2.0f * a * b * Fp;
                        const float B1 = fmaf(2.0f * a * a, Fp, F), B2 = fmaf(2.0f * b * b, Fp, F);
                        px = fmaf(cv, B1, fmaf(-cu, A, px));  // cu dKu/da + cv dKv/da (times C)
                        py = fmaf(cv, A, fmaf(-cu, B2, py));  // cu dKu/db + cv dKv/db (times C)
                    }
                }
            }
            ag += (double)pg;
            ax += (double)px;
            ay += (double)py;
        }
        if (valid) {
            const int i = w.perm[tpos];
            if (odg)
                odg[i] = ag * snear;
            if (odx)
                odx[i] = ax * C;
            if (ody)
                ody[i] = ay * C;
        }
    }
}

int launch_adjoint_p2p(const Work &w, double *dg, double *dx, double *dy, int fp32, cudaStream_t s)
{
    if (w.nleaf == 0)
        return 0;
    if (!fp32) {
        k_adjoint_p2p64<<<w.nleaf, 64, 0, s>>>(w, dg, dx, dy, 0);
        return 1;
    }
    // one-float systems in FP32, systems with wider leaves in FP64
    k_adjoint_p2p32<<<w.nleaf, 64, 0, s>>>(w, dg, dx, dy);
    k_adjoint_p2p64<<<w.nleaf, 64, 0, s>>>(w, dg, dx, dy, 1);
    return 2;
}

}  // namespace fmm
