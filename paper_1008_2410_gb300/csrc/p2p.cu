// p2p.cu -- Fig. 1 stage 9: near-field direct evaluation of the regularised kernel (Eq. 6) between
// particles in the same or adjacent leaves, and its adjoint.
//
// Each pair is evaluated from the target's side (§3: "each particle pair twice, once from each end"), so
// a target accumulates in registers and nothing is written concurrently. One thread block owns one target
// leaf; its 3 x 3 neighbourhood is three contiguous runs of the leaf-ordered particles (rows iy-1, iy, iy+1
// of columns ix-1..ix+1), staged through shared memory in tiles.
//
// Precision form (FMM_MIXED): coordinates are leaf-relative in leaf units, split hi + lo in FP32; the shift
// by the integer leaf offset is exact (Fast2Sum folds its rounding error into lo), so a difference keeps the
// FP64 coordinates' resolution. exp and 1/r^2 use the SFU (ex2.approx, rcp.approx); for r^2 / 2 sigma^2 < 1/2
// the factor (1 - e^-y)/y comes from its Taylor series instead of 1 - e^-y, which cancels. Per-target sums are
// FP32 per source-leaf segment and compensated (Neumaier) across segments. Tiles arrive by bulk asynchronous
// copies (cp.async.bulk, the TMA engine) into shared memory, completed on an mbarrier with a bounded wait.
#include "fmm_internal.cuh"

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
// Waits for the phase with the given parity; gives up after a bounded number of polls and reports a timeout
// in the status word instead of hanging.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned int *status)
{
    for (int it = 0; it < (1 << 20); ++it)
        if (mbar_try_wait(bar, parity))
            return true;
    atomicOr(status, FMM_DEV_TIMEOUT);
    return false;
}

// (1 - e^-y)/y for y in [0, 1/2): Taylor series sum_k (-y)^k / (k+1)!, 10 terms (truncation < 3e-11).
__device__ __forceinline__ float small_y_factor(float y)
{
    float s = 1.0f / 39916800.0f;  // 1/11!
    s = fmaf(s, -y, 1.0f / 3628800.0f);
    s = fmaf(s, -y, 1.0f / 362880.0f);
    s = fmaf(s, -y, 1.0f / 40320.0f);
    s = fmaf(s, -y, 1.0f / 5040.0f);
    s = fmaf(s, -y, 1.0f / 720.0f);
    s = fmaf(s, -y, 1.0f / 120.0f);
    s = fmaf(s, -y, 1.0f / 24.0f);
    s = fmaf(s, -y, 1.0f / 6.0f);
    s = fmaf(s, -y, 0.5f);
    s = fmaf(s, -y, 1.0f);
    return s;
}

__device__ __forceinline__ void neumaier(float &s, float &c, float x)
{
    float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
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

// In units where r'^2 is the exponent of 2: exp(-r^2 / 2 sigma^2) = 2^-(r'^2), y = r'^2 ln 2. The series
// replaces 1 - 2^-(r'^2) when y < 1/2, i.e. r'^2 < (1/2) / ln 2.
#define P2P_THR 0.72134752044448170f
#define P2P_LN2 0.69314718055994531f

// Targets of one lane for one pass: up to 4 (two packed pairs); split coordinates and compensated sums.
struct Targets {
    float hx[4], hy[4], lx[4], ly[4];
    float su[4], cu[4], sv[4], cv[4];
};

// Sources j0..j1 of one source leaf against KT targets per lane (KT/2 packed pairs). The targets are first
// re-expressed relative to that leaf's centre, exactly: hi - dc s by Fast2Sum (|dc s| >= |hi|), its error into lo.
template <int KT>
__device__ __forceinline__ void p2p_segment(const float4 *__restrict__ EH, const float4 *__restrict__ EL,
                                            const float4 *__restrict__ EG, int j0, int j1, float sdx, float sdy,
                                            Targets &t)
{
    constexpr int NP = KT / 2;
    f2 AHX[NP], ALX[NP], AHY[NP], ALY[NP], PU[NP], PV[NP];
#pragma unroll
    for (int pr = 0; pr < NP; ++pr) {
        float hx0 = t.hx[2 * pr] - sdx, hx1 = t.hx[2 * pr + 1] - sdx;
        float lx0 = t.lx[2 * pr] + (t.hx[2 * pr] - (hx0 + sdx)), lx1 = t.lx[2 * pr + 1] + (t.hx[2 * pr + 1] - (hx1 + sdx));
        float hy0 = t.hy[2 * pr] - sdy, hy1 = t.hy[2 * pr + 1] - sdy;
        float ly0 = t.ly[2 * pr] + (t.hy[2 * pr] - (hy0 + sdy)), ly1 = t.ly[2 * pr + 1] + (t.hy[2 * pr + 1] - (hy1 + sdy));
        AHX[pr] = pk2(hx0, hx1);
        ALX[pr] = pk2(lx0, lx1);
        AHY[pr] = pk2(hy0, hy1);
        ALY[pr] = pk2(ly0, ly1);
        PU[pr] = 0ull;
        PV[pr] = 0ull;
    }
    for (int j = j0; j < j1; ++j) {
        const float4 h = EH[j], l = EL[j], g = EG[j];
        const f2 sxh = pk2(h.x, h.y), syh = pk2(h.z, h.w), sxl = pk2(l.x, l.y), syl = pk2(l.z, l.w);
        const f2 gp = pk2(g.x, g.y), gn = pk2(g.z, g.w);
        f2 dx[NP], dy[NP], r2[NP], q[NP], og[NP];
        float rmin = 3.0e38f;
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
            dx[pr] = add2(sub2(AHX[pr], sxh), sub2(ALX[pr], sxl));
            dy[pr] = add2(sub2(AHY[pr], syh), sub2(ALY[pr], syl));
            r2[pr] = fma2(dx[pr], dx[pr], mul2(dy[pr], dy[pr]));
            float ra, rb;
            up2(r2[pr], ra, rb);
            const float ea = ex2_approx(-ra), eb = ex2_approx(-rb);
            q[pr] = pk2(rcp_approx(ra), rcp_approx(rb));
            og[pr] = fma2(pk2(ea, eb), gn, gp);  // g (1 - e)
            rmin = fminf(rmin, fminf(ra, rb));
        }
        // rare (r < sigma): warp-uniform branch to the series for (1 - e^-y) / y
        if (__any_sync(0xffffffffu, rmin < P2P_THR)) {
#pragma unroll
            for (int pr = 0; pr < NP; ++pr) {
                float ra, rb, qa, qb, oa, ob;
                up2(r2[pr], ra, rb);
                up2(q[pr], qa, qb);
                up2(og[pr], oa, ob);
                if (ra < P2P_THR) {
                    qa = P2P_LN2 * small_y_factor(P2P_LN2 * ra);
                    oa = g.x;
                }
                if (rb < P2P_THR) {
                    qb = P2P_LN2 * small_y_factor(P2P_LN2 * rb);
                    ob = g.x;
                }
                q[pr] = pk2(qa, qb);
                og[pr] = pk2(oa, ob);
            }
        }
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
            const f2 gf = mul2(og[pr], q[pr]);
            PU[pr] = fma2(dy[pr], gf, PU[pr]);  // u accumulates -dy g f: negated at the end
            PV[pr] = fma2(dx[pr], gf, PV[pr]);
        }
    }
#pragma unroll
    for (int pr = 0; pr < NP; ++pr) {
        float a, b;
        up2(PU[pr], a, b);
        neumaier(t.su[2 * pr], t.cu[2 * pr], a);
        neumaier(t.su[2 * pr + 1], t.cu[2 * pr + 1], b);
        up2(PV[pr], a, b);
        neumaier(t.sv[2 * pr], t.cv[2 * pr], a);
        neumaier(t.sv[2 * pr + 1], t.cv[2 * pr + 1], b);
    }
}

// LPB leaves per block (1 or 2, one warp each; with 2 the leaves are the pair (2j, 2j+1) of one row and share
// their 3 x 4 source neighbourhood). Each warp takes its leaf's targets in passes of at most 32 * ktmax, with
// 2 or 4 targets per lane chosen by the pass size. Sources arrive by bulk copies into shared memory.
template <int LPB>
__global__ void __launch_bounds__(64) k_p2p32(Work w, int tile, int ktmax)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    float4 *EH = reinterpret_cast<float4 *>(smem_raw), *EL = EH + tile, *EG = EL + tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int first = blockIdx.x * LPB;
    if (first >= w.nleaf)
        return;
    const int k = w.nsys == 1 ? 0 : find_sys_by_leaf(w.sys, w.nsys, first);
    const SysDev &d = w.sys[k];
    const int L = d.depth, ns = 1 << L, local0 = first - (int)d.leaf0;
    const int ix0 = local0 & (ns - 1), iy = local0 >> L;
    const int myleaf = first + warp;
    const int my_s0 = w.start[myleaf], my_c = w.start[myleaf + 1] - my_s0;
    const int per_pass = 32 * ktmax;
    int npass = (my_c + per_pass - 1) / per_pass;
    if (LPB == 2) {
        const int other = first + (warp ^ 1);
        const int oc = w.start[other + 1] - w.start[other];
        npass = max(npass, (oc + per_pass - 1) / per_pass);
    }
    if (npass == 0)
        return;  // block-uniform: every leaf of the block is empty
    const int my_np = (my_c + per_pass - 1) / per_pass;
    const float s = d.s_unit, snear = d.snear;
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
            t_lo = (int)((int64_t)pass * my_c / my_np);
            t_cnt = (int)((int64_t)(pass + 1) * my_c / my_np) - t_lo;
        }
        const int kt = t_cnt == 0 ? 0 : (t_cnt <= 64 ? 2 : 4);
        Targets t;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int e = lane + 32 * q;
            float4 hh = make_float4(0.f, 0.f, 0.f, 0.f), ll = hh;
            if (e < t_cnt) {
                hh = w.eh[my_s0 + t_lo + e];
                ll = w.el[my_s0 + t_lo + e];
            }
            t.hx[q] = hh.x;
            t.hy[q] = hh.z;
            t.lx[q] = ll.x;
            t.ly[q] = ll.z;
            t.su[q] = t.cu[q] = t.sv[q] = t.cv[q] = 0.f;
        }
        for (int dyr = -1; dyr <= 1; ++dyr) {
            const int row = iy + dyr;
            if (row < 0 || row >= ns)
                continue;
            const int rowleaf = (int)d.leaf0 + row * ns;
            const int ca = max(c_lo, 0), cz = min(c_lo + ncol - 1, ns - 1);
            const int r0 = w.start[rowleaf + ca], r1 = w.start[rowleaf + cz + 1];
            if (r1 <= r0)
                continue;
            int cb[LPB + 3];
#pragma unroll
            for (int cc = 0; cc < ncol; ++cc) {
                const int col = c_lo + cc;
                cb[cc] = col < 0 ? r0 : (col >= ns ? r1 : w.start[rowleaf + col]);
            }
            cb[ncol] = r1;
            for (int q0 = r0; q0 < r1; q0 += tile) {
                const int m = min(tile, r1 - q0);
                __syncthreads();  // everyone is done with the previous tile
                if (threadIdx.x == 0) {
                    fence_proxy_async();
                    mbar_expect_tx(&bar, (uint32_t)m * 48u);
                    bulk_g2s(EH, w.eh + q0, (uint32_t)m * 16u, &bar);
                    bulk_g2s(EL, w.el + q0, (uint32_t)m * 16u, &bar);
                    bulk_g2s(EG, w.eg + q0, (uint32_t)m * 16u, &bar);
                }
                bool ok = mbar_wait_bounded(&bar, phase, w.status);
                if (!__syncthreads_and(ok)) {
                    if (!ok)
                        mbar_wait_bounded(&bar, phase, w.status);  // let a late copy land before exiting
                    return;
                }
                phase ^= 1;
                if (kt == 0)
                    continue;
#pragma unroll
                for (int k3 = 0; k3 < 3; ++k3) {
                    const int cc = warp + k3;  // this warp's columns ix-1, ix, ix+1
                    const int j0 = max(q0, cb[cc]) - q0, j1 = min(q0 + m, cb[cc + 1]) - q0;
                    if (j0 >= j1)
                        continue;
                    const float sdx = (float)(k3 - 1) * s, sdy = (float)dyr * s;
                    if (kt == 2)
                        p2p_segment<2>(EH, EL, EG, j0, j1, sdx, sdy, t);
                    else
                        p2p_segment<4>(EH, EL, EG, j0, j1, sdx, sdy, t);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = lane + 32 * q;
            if (e < t_cnt)
                w.near32[my_s0 + t_lo + e] = make_float2(-(t.su[q] + t.cu[q]) * snear, (t.sv[q] + t.cv[q]) * snear);
        }
    }
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
    // two leaves per block needs every system's leaves to pair up within rows (depth >= 1)
    bool pairs = threads == 64 && w.lv.nsys_at[1] == w.nsys;
    int tile = pairs ? 320 : 256;
    size_t sm = (size_t)tile * 48;
    if (pairs)
        k_p2p32<2><<<(w.nleaf + 1) / 2, 64, sm, s>>>(w, tile, ktmax);
    else
        k_p2p32<1><<<w.nleaf, 32, sm, s>>>(w, tile, ktmax);
    return 1;
}

// ------------------------------------------------------------------ adjoint near field (FP64)

// For target k and neighbour m (z = z_k - z_m), with K = (Ku, Kv) of Eq. 6 and its Jacobian J:
//   dgamma_k += -(gu_m Ku(z) + gv_m Kv(z))
//   dx_k     += (gamma_m gu_k - gamma_k gu_m) dKu/da + (gamma_m gv_k - gamma_k gv_m) dKv/da
//   dy_k     += (gamma_m gu_k - gamma_k gu_m) dKu/db + (gamma_m gv_k - gamma_k gv_m) dKv/db
// (K is odd and its Jacobian even in z). Writes the near part in caller order (the far part is added later).
__global__ void __launch_bounds__(64) k_adjoint_p2p64(Work w, double *__restrict__ odg, double *__restrict__ odx,
                                                     double *__restrict__ ody)
{
    __shared__ double shx[256], shy[256], shg[256], shu[256], shv[256];
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

int launch_adjoint_p2p(const Work &w, double *dg, double *dx, double *dy, cudaStream_t s)
{
    if (w.nleaf == 0)
        return 0;
    k_adjoint_p2p64<<<w.nleaf, 64, 0, s>>>(w, dg, dx, dy);
    return 1;
}

}  // namespace fmm
