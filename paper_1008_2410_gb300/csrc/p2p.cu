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

// One block per target leaf; `KT` targets per thread; tiles of `tile` sources (a multiple of 4).
template <int KT>
__global__ void __launch_bounds__(128) k_p2p32(Work w, int tile)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    float4 *spos = reinterpret_cast<float4 *>(smem_raw);
    float *sgam = reinterpret_cast<float *>(smem_raw + (size_t)tile * sizeof(float4));
    const int leaf = blockIdx.x;
    const int s0 = w.start[leaf], c = w.start[leaf + 1] - s0;
    if (c == 0)
        return;
    const int k = w.nsys == 1 ? 0 : find_sys_by_leaf(w.sys, w.nsys, leaf);
    const SysDev &d = w.sys[k];
    const int L = d.depth, ns = 1 << L, local = leaf - (int)d.leaf0;
    const int ix = local & (ns - 1), iy = local >> L;
    const float kappa = d.kappa, cexp = d.cexp, ythr = d.ythr, snear = d.snear;
    const int jx0 = ix > 0 ? ix - 1 : 0, jx1 = ix < ns - 1 ? ix + 1 : ns - 1;
    const int tid = threadIdx.x, T = blockDim.x;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_proxy_async();
    }
    __syncthreads();
    uint32_t phase = 0;
    for (int t0 = 0; t0 < c; t0 += T * KT) {
        float thx[KT], thy[KT], tlx[KT], tly[KT];
        float su[KT], cu[KT], sv[KT], cv[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            int e = t0 + tid + q * T;
            float4 tp = e < c ? w.pos4[s0 + e] : make_float4(0.f, 0.f, 0.f, 0.f);
            thx[q] = tp.x;
            thy[q] = tp.y;
            tlx[q] = tp.z;
            tly[q] = tp.w;
            su[q] = cu[q] = sv[q] = cv[q] = 0.f;
        }
        for (int dy = -1; dy <= 1; ++dy) {
            const int row = iy + dy;
            if (row < 0 || row >= ns)
                continue;
            const int rowleaf = (int)d.leaf0 + row * ns;
            const int r0 = w.start[rowleaf + jx0], r1 = w.start[rowleaf + jx1 + 1];
            if (r1 <= r0)
                continue;
            int cb[4];  // column boundaries inside the row run (columns ix-1, ix, ix+1)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                int col = ix - 1 + q;
                cb[q] = (col < jx0) ? r0 : (col > jx1 ? r1 : w.start[rowleaf + col]);
            }
            cb[3] = r1;
            for (int q0 = r0 & ~3; q0 < r1; q0 += tile) {
                const int a = q0, b = min(q0 + tile, (r1 + 3) & ~3);
                __syncthreads();  // everyone is done with the previous tile
                if (tid == 0) {
                    fence_proxy_async();
                    mbar_expect_tx(&bar, (uint32_t)(b - a) * 20u);
                    bulk_g2s(spos, w.pos4 + a, (uint32_t)(b - a) * 16u, &bar);
                    bulk_g2s(sgam, w.g32 + a, (uint32_t)(b - a) * 4u, &bar);
                }
                bool ok = mbar_wait_bounded(&bar, phase, w.status);
                if (!__syncthreads_and(ok)) {
                    // the copy never completed: give it one more bounded wait before the block exits
                    if (!ok)
                        mbar_wait_bounded(&bar, phase, w.status);
                    return;
                }
                phase ^= 1;
                const int lo = max(a, r0), hi = min(q0 + tile, r1);
#pragma unroll 1
                for (int col = 0; col < 3; ++col) {
                    const int j0 = max(lo, cb[col]) - a, j1 = min(hi, cb[col + 1]) - a;
                    if (j0 >= j1)
                        continue;
                    // target relative to this source leaf's centre, zeta_t - (dc, dy), kept exact as hi + lo
                    const float dc = (float)(col - 1), dr = (float)dy;
                    float ahx[KT], alx[KT], ahy[KT], aly[KT], pu[KT], pv[KT];
#pragma unroll
                    for (int q = 0; q < KT; ++q) {
                        float sx = thx[q] - dc;
                        ahx[q] = sx;
                        alx[q] = tlx[q] + (thx[q] - (sx + dc));
                        float sy = thy[q] - dr;
                        ahy[q] = sy;
                        aly[q] = tly[q] + (thy[q] - (sy + dr));
                        pu[q] = pv[q] = 0.f;
                    }
                    for (int j = j0; j < j1; ++j) {
                        const float4 sp = spos[j];
                        const float g = sgam[j];
                        float dxv[KT], dyv[KT], r2v[KT], fv[KT];
                        float rmin = 3.0e38f;
#pragma unroll
                        for (int q = 0; q < KT; ++q) {
                            dxv[q] = (ahx[q] - sp.x) + (alx[q] - sp.z);
                            dyv[q] = (ahy[q] - sp.y) + (aly[q] - sp.w);
                            float r2 = fmaf(dxv[q], dxv[q], dyv[q] * dyv[q]);
                            float e = ex2_approx(r2 * cexp);
                            float rr = rcp_approx(fmaxf(r2, 1e-30f));
                            fv[q] = fmaf(-e, rr, rr);  // (1 - e^-y) / r^2
                            r2v[q] = r2;
                            rmin = fminf(rmin, r2);
                        }
                        // rare (r < sigma): warp-uniform branch to the series, off the common path
                        if (__any_sync(0xffffffffu, rmin < ythr)) {
#pragma unroll
                            for (int q = 0; q < KT; ++q)
                                if (r2v[q] < ythr)
                                    fv[q] = kappa * small_y_factor(kappa * r2v[q]);
                        }
#pragma unroll
                        for (int q = 0; q < KT; ++q) {
                            const float gf = g * fv[q];
                            pu[q] = fmaf(-dyv[q], gf, pu[q]);
                            pv[q] = fmaf(dxv[q], gf, pv[q]);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < KT; ++q) {
                        neumaier(su[q], cu[q], pu[q]);
                        neumaier(sv[q], cv[q], pv[q]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            int e = t0 + tid + q * T;
            if (e < c)
                w.near32[s0 + e] = make_float2((su[q] + cu[q]) * snear, (sv[q] + cv[q]) * snear);
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
    if (threads <= 0)
        threads = 64;
    int tile = 8 * threads;  // 256 / 512 / 1024 sources: 5, 10, 20 KiB of shared memory per block
    size_t sm = (size_t)tile * 20;
    if (kt == 2)
        k_p2p32<2><<<w.nleaf, threads, sm, s>>>(w, tile);
    else if (kt == 4)
        k_p2p32<4><<<w.nleaf, threads, sm, s>>>(w, tile);
    else
        k_p2p32<1><<<w.nleaf, threads, sm, s>>>(w, tile);
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
