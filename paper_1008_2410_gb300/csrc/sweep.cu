// sweep.cu -- Fig. 1 stages 4-8 and 10: P2M, M2M, M2L, L2L, and the fused L2P + sum + unsort.
//
// Expansions (§3: a t-term multipole with coefficients sum_p Gamma_p (x_p - x_c)^m, times -i/2pi) are kept
// radius-scaled: a~_m = sum_j q'_j zeta_j^m with zeta = (z - c)/w_l and q' = -i gamma; locals
// b^_l = w_l^(l+1) b_l. In these units every translation matrix is the same on every level:
//   M2M  a~'_n = sum_{m<=n} C(n, m) delta^(n-m) 2^-m a~_m,          delta = (c_child - c_parent)/w_parent
//   M2L  b^_l  = sum_m (-1)^(m+1) C(m+l, m) rho^(m+l+1) a~_m,       rho = w / (c_source - c_target)
//   L2L  b^'_k = sum_{l>=k} C(l, k) delta^(l-k) 2^-(l+1) b^_l,     delta = (c_child - c_parent)/w_child
// and the far field at z is w = u - i v = (1 / (2 pi w_L)) sum_l b^_l zeta^l. M2L is evaluated in the
// factored form b^_l = rho^(l+1) sum_m C(m+l, m) [(-1)^(m+1) rho^m a~_m]: a real p x p contraction between
// two diagonal complex scalings, 2p^2 + 12p flops per translation instead of 8p^2.
#include <type_traits>

#include "fmm_internal.cuh"

namespace fmm {

template <typename R>
struct cx {
    R re, im;
};
template <typename R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b)
{
    return {a.re + b.re, a.im + b.im};
}

template <typename R>
struct store_of;
template <>
struct store_of<double> {
    typedef double2 T;
};
template <>
struct store_of<float> {
    typedef float2 T;
};

template <typename R, typename S>
__device__ __forceinline__ cx<R> ldc(const S *p, int64_t i)
{
    S v = p[i];
    return {(R)v.x, (R)v.y};
}
template <typename R>
__device__ __forceinline__ void stc(double2 *p, int64_t i, cx<R> v)
{
    p[i] = make_double2((double)v.re, (double)v.im);
}
template <typename R>
__device__ __forceinline__ void stc(float2 *p, int64_t i, cx<R> v)
{
    p[i] = make_float2((float)v.re, (float)v.im);
}

// ------------------------------------------------------------------ stage 4: P2M (one warp per leaf)

// Compute type R; coefficients written to the leaf level's array (FP64 or FP32). PM >= p terms are
// accumulated (the first p are the p-term expansion; the rest are discarded).
template <int PM, typename R>
__global__ void __launch_bounds__(64) k_p2m(Work w, int adj)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R> *sh = reinterpret_cast<cx<R> *>(smem_raw) + (threadIdx.x >> 5) * 32 * (PM + 1);
    int lane = threadIdx.x & 31;
    int64_t leaf = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (leaf >= w.nleaf)
        return;
    int k = w.nsys == 1 ? 0 : find_sys_by_leaf(w.sys, w.nsys, leaf);
    const SysDev &d = w.sys[k];
    int L = d.depth;
    if (L < 2)
        return;
    int local = (int)(leaf - d.leaf0);
    int64_t box = d.box0[L] + local;
    int s0 = w.start[leaf], c = w.start[leaf + 1] - s0;
    if (lane == 0)
        w.bcount[box] = c;
    if (c == 0)
        return;
    int ix = local & ((1 << L) - 1), iy = local >> L;
    double scale = d.scale;
    cx<R> a[PM];
#pragma unroll
    for (int m = 0; m < PM; ++m)
        a[m] = {(R)0, (R)0};
    for (int j = s0 + lane; j < s0 + c; j += 32) {
        cx<R> z, q;
        if (w.mixed) {
            float4 hh = w.eh[j], ll = w.el[j];
            z = {(R)((hh.x + ll.x) * d.inv_s), (R)((hh.z + ll.z) * d.inv_s)};
            q = {(R)0, -(R)w.eg[j].x};
        } else {
            z = {(R)((w.sx[j] - d.x0) * scale - (ix + 0.5)), (R)((w.sy[j] - d.y0) * scale - (iy + 0.5))};
            if (adj)
                q = {(R)w.sgu[j], (R)w.sgv[j]};
            else
                q = {(R)0, -(R)w.sg[j]};
        }
        cx<R> pw = q;
#pragma unroll
        for (int m = 0; m < PM; ++m) {
            a[m] = cadd(a[m], pw);
            pw = cmul(pw, z);
        }
    }
#pragma unroll
    for (int m = 0; m < PM; ++m)
        sh[lane * (PM + 1) + m] = a[m];
    __syncwarp();
    if (lane < w.p) {
        cx<R> s = {(R)0, (R)0};
        for (int r = 0; r < 32; ++r)
            s = cadd(s, sh[r * (PM + 1) + lane]);
        int64_t idx = box * w.p + lane;
        if (level_fp64(w, L))
            stc(adj ? w.AM64 : w.M64, idx, s);
        else
            stc(w.M32, idx, s);
    }
}

template <int PM>
static void p2m_dispatch(const Work &w, int adj, cudaStream_t s)
{
    int blocks = (int)(((int64_t)w.nleaf * 32 + 63) / 64);
    // FP32 accumulation only when every system's leaf level is an FP32 level; the FP64 kernel writes either.
    if (w.mixed && w.lv.mindepth2 > w.coarse_level) {
        size_t sm = 2 * 32 * (PM + 1) * sizeof(cx<float>);
        k_p2m<PM, float><<<blocks, 64, sm, s>>>(w, adj);
    } else {
        size_t sm = 2 * 32 * (PM + 1) * sizeof(cx<double>);
        k_p2m<PM, double><<<blocks, 64, sm, s>>>(w, adj);
    }
}

int launch_p2m(const Work &w, const Tables &t, int adj, cudaStream_t s)
{
    (void)t;
    if (w.p <= 8)
        p2m_dispatch<8>(w, adj, s);
    else if (w.p <= 16)
        p2m_dispatch<16>(w, adj, s);
    else if (w.p <= 20)
        p2m_dispatch<20>(w, adj, s);
    else if (w.p <= 24)
        p2m_dispatch<24>(w, adj, s);
    else
        p2m_dispatch<32>(w, adj, s);
    return 1;
}

// ------------------------------------------------------------------ stage 5: M2M (warp per parent box)

template <typename RA>
__device__ __forceinline__ cx<RA> ld_tab(const double2 *__restrict__ t64, const float2 *__restrict__ t32, int i)
{
    if constexpr (std::is_same<RA, double>::value) {
        double2 t = t64[i];
        return {(RA)t.x, (RA)t.y};
    } else {
        float2 t = t32[i];
        return {(RA)t.x, (RA)t.y};
    }
}

// One warp per parent box, lane n = coefficient. The four children's expansions are staged in shared memory
// with coalesced loads; the table is stored [child][m][n] so that lanes read consecutive entries.
template <int PM, typename RA, typename SC, typename SP>
__global__ void __launch_bounds__(128) k_m2m(Work w, const double2 *__restrict__ tab64,
                                             const float2 *__restrict__ tab32, int l, const SC *__restrict__ child,
                                             SP *parent)
{
    __shared__ cx<RA> sh[4][4][FMM_PMAX];
    const int p = w.p, lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int64_t nb = (int64_t)1 << (2 * l);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= (int64_t)w.lv.nsys_at[l + 1] * nb)
        return;
    const int b = (int)(gw & (nb - 1));
    const int sidx = (int)(gw >> (2 * l));
    const SysDev &d = w.sys[sys_at_level(w, l + 1, sidx)];
    const int ns = 1 << l, bx = b & (ns - 1), by = b >> l;
    const int64_t pbox = d.box0[l] + b;
    int cnt[4], count = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int64_t cbox = d.box0[l + 1] + (int64_t)(2 * by + (c >> 1)) * (2 * ns) + (2 * bx + (c & 1));
        cnt[c] = w.bcount[cbox];
        count += cnt[c];
        if (lane < p)
            sh[wi][c][lane] = cnt[c] ? ldc<RA>(child, cbox * p + lane) : cx<RA>{(RA)0, (RA)0};
    }
    if (lane == 0)
        w.bcount[pbox] = count;
    if (count == 0)
        return;
    __syncwarp();
    if (lane >= p)
        return;
    // compile-time trip count (entries with m > n are zero in the table): every load issues at once
    cx<RA> acc = {(RA)0, (RA)0};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (!cnt[c])
            continue;
#pragma unroll
        for (int m = 0; m < PM; ++m)
            if (m < p)
                acc = cadd(acc, cmul(ld_tab<RA>(tab64, tab32, (c * FMM_PMAX + m) * FMM_PMAX + lane), sh[wi][c][m]));
    }
    stc(parent, pbox * p + lane, acc);
}

template <int PM>
static void m2m_launch(const Work &w, const Tables &t, int l, int adj, unsigned blocks, cudaStream_t s)
{
    const bool pd = level_fp64(w, l), cd = level_fp64(w, l + 1);
    double2 *M64 = adj ? w.AM64 : w.M64;
    if (pd && cd)
        k_m2m<PM, double, double2, double2><<<blocks, 128, 0, s>>>(w, t.m2m64, t.m2m32, l, M64, M64);
    else if (pd)
        k_m2m<PM, double, float2, double2><<<blocks, 128, 0, s>>>(w, t.m2m64, t.m2m32, l, w.M32, M64);
    else
        k_m2m<PM, float, float2, float2><<<blocks, 128, 0, s>>>(w, t.m2m64, t.m2m32, l, w.M32, w.M32);
}

int launch_m2m(const Work &w, const Tables &t, int l, int adj, cudaStream_t s, int prio)
{
    (void)prio;
    const int64_t warps = (int64_t)w.lv.nsys_at[l + 1] * ((int64_t)1 << (2 * l));
    if (warps == 0)
        return 0;
    const unsigned blocks = (unsigned)((warps * 32 + 127) / 128);
    if (w.p <= 8)
        m2m_launch<8>(w, t, l, adj, blocks, s);
    else if (w.p <= 16)
        m2m_launch<16>(w, t, l, adj, blocks, s);
    else if (w.p <= 20)
        m2m_launch<20>(w, t, l, adj, blocks, s);
    else if (w.p <= 24)
        m2m_launch<24>(w, t, l, adj, blocks, s);
    else
        m2m_launch<32>(w, t, l, adj, blocks, s);
    return 1;
}

// ------------------------------------------------------------------ stage 6: M2L (warp per target box, all levels)

// One warp per target box, lane l = local coefficient. The interaction list (children of the parent's
// neighbours that are not adjacent, at most 27, empty boxes skipped) is built once; sources are then taken two
// at a time: lane m scales a~_m by (-1)^(m+1) rho^m into shared memory, and lane l contracts with its column of
// binomials C(m + l, m), held in registers, before the rho^(l+1) scaling.
template <int PM, typename R, typename S>
__device__ void m2l_box(const Work &w, const typename store_of<R>::T *__restrict__ rho, const R *__restrict__ binom,
                        const S *__restrict__ M, S *Loc, const SysDev &d, int l, int b, cx<R> *alpha, int2 *list)
{
    const int lane = threadIdx.x & 31, p = w.p;
    const int ns = 1 << l, bx = b & (ns - 1), by = b >> l;
    const int px = bx >> 1, py = by >> 1;
    const int RS = 2 * FMM_PMAX + 2;
    // interaction list: lanes 0..35 cover the 6 x 6 children block of the parent's 3 x 3 neighbourhood
    int cnt = 0;
    for (int base = 0; base < 36; base += 32) {
        int q = base + lane;
        bool ok = false;
        int2 ent = make_int2(0, 0);
        if (q < 36) {
            int jx = 2 * (px - 1) + q % 6, jy = 2 * (py - 1) + q / 6;
            int ddx = jx - bx, ddy = jy - by;
            if (jx >= 0 && jy >= 0 && jx < ns && jy < ns && !(ddx >= -1 && ddx <= 1 && ddy >= -1 && ddy <= 1)) {
                int64_t sb = d.box0[l] + (int64_t)jy * ns + jx;
                if (w.bcount[sb] != 0) {
                    ok = true;
                    ent = make_int2((int)(sb - d.box0[l]), (ddy + 3) * 7 + (ddx + 3));
                }
            }
        }
        unsigned m = __ballot_sync(0xffffffffu, ok);
        if (ok)
            list[cnt + __popc(m & ((1u << lane) - 1))] = ent;
        cnt += __popc(m);
    }
    __syncwarp();
    R cb[PM];
#pragma unroll
    for (int m = 0; m < PM; ++m)
        cb[m] = (m < p && lane < p) ? binom[m * FMM_PMAX + lane] : (R)0;
    cx<R> acc = {(R)0, (R)0};
    for (int s = 0; s < cnt; s += 2) {
        const bool two = s + 1 < cnt;
        const int2 e0 = list[s], e1 = two ? list[s + 1] : list[s];
        const typename store_of<R>::T *rp0 = rho + e0.y * RS, *rp1 = rho + e1.y * RS;
        if (lane < p) {
            const R sg = (lane & 1) ? (R)1 : (R)-1;  // (-1)^(m+1)
            cx<R> a0 = ldc<R>(M, (d.box0[l] + e0.x) * (int64_t)p + lane);
            auto r0 = rp0[lane];
            cx<R> t0 = cmul(cx<R>{(R)r0.x, (R)r0.y}, a0);
            alpha[lane] = {sg * t0.re, sg * t0.im};
            cx<R> t1 = {(R)0, (R)0};
            if (two) {
                cx<R> a1 = ldc<R>(M, (d.box0[l] + e1.x) * (int64_t)p + lane);
                auto r1 = rp1[lane];
                t1 = cmul(cx<R>{(R)r1.x, (R)r1.y}, a1);
            }
            alpha[32 + lane] = {sg * t1.re, sg * t1.im};
        } else {
            alpha[lane] = {(R)0, (R)0};  // entries m >= p meet zero binomials: keep them finite
            alpha[32 + lane] = {(R)0, (R)0};
        }
        __syncwarp();
        cx<R> b0 = {(R)0, (R)0}, b1 = {(R)0, (R)0};
#pragma unroll
        for (int m = 0; m < PM; ++m) {
            const cx<R> am = alpha[m], an = alpha[32 + m];
            b0.re = fma(cb[m], am.re, b0.re);
            b0.im = fma(cb[m], am.im, b0.im);
            b1.re = fma(cb[m], an.re, b1.re);
            b1.im = fma(cb[m], an.im, b1.im);
        }
        if (lane < p) {
            auto q0 = rp0[lane + 1];
            acc = cadd(acc, cmul(cx<R>{(R)q0.x, (R)q0.y}, b0));
            if (two) {
                auto q1 = rp1[lane + 1];
                acc = cadd(acc, cmul(cx<R>{(R)q1.x, (R)q1.y}, b1));
            }
        }
        __syncwarp();
    }
    if (lane < p)
        stc(Loc, (d.box0[l] + b) * (int64_t)p + lane, acc);
}

template <int PM>
__global__ void __launch_bounds__(128) k_m2l(Work w, Tables t, int adj, int64_t gw0, int64_t gw1)
{
    __shared__ __align__(16) double2 alpha_sh[4][64];
    __shared__ int2 list_sh[4][40];
    int64_t gw = gw0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (gw >= gw1)
        return;
    int l = 2;
    while (l < w.lv.maxdepth && gw >= w.lv.m2l_item0[l + 1])
        ++l;
    if (l > w.lv.maxdepth || gw >= w.lv.m2l_item0[l + 1])
        return;
    int64_t g = gw - w.lv.m2l_item0[l];
    int b = (int)(g & (((int64_t)1 << (2 * l)) - 1));
    int sidx = (int)(g >> (2 * l));
    const SysDev &d = w.sys[sys_at_level(w, l, sidx)];
    if (w.bcount[d.box0[l] + b] == 0)
        return;
    int wi = threadIdx.x >> 5;
    if (level_fp64(w, l)) {
        double2 *M = adj ? w.AM64 : w.M64, *Lc = adj ? w.AL64 : w.L64;
        m2l_box<PM, double, double2>(w, t.rho64, t.binom64, M, Lc, d, l, b,
                                     reinterpret_cast<cx<double> *>(alpha_sh[wi]), list_sh[wi]);
    } else {
        m2l_box<PM, float, float2>(w, t.rho32, t.binom32, w.M32, w.L32, d, l, b,
                                   reinterpret_cast<cx<float> *>(alpha_sh[wi]), list_sh[wi]);
    }
}

// Precision form, FP32 levels: one warp per target box with lane q = source q of its interaction list (at most
// 27: the children of the parent's 3 x 3 neighbours that are not adjacent, taken from a per-parity offset table).
// Lane q forms x_m = (-1)^(m+1) rho^m a~_m, contracts it with the binomials C(m + l, m) by prefix sums (below),
// scales by rho^(l+1), and the 27 partial locals are summed per coefficient through shared memory. P >= p terms
// are evaluated (zero-padded).
__constant__ int2 c_m2l_off[4][27];

static int g_const_ready[64];

static bool m2l_constants_ready()
{
    int dev = 0;
    return cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && g_const_ready[dev];
}

// Uploads the offset table of k_m2l_src to the current device once (synchronises the stream: call it before
// any stream capture).
int upload_m2l_constants(cudaStream_t s)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return -1;
    if (g_const_ready[dev])
        return 0;
    static int2 off[4][27];
    for (int cls = 0; cls < 4; ++cls) {
        int cx = cls & 1, cy = cls >> 1, q = 0;
        for (int ry = -2 - cy; ry <= 3 - cy; ++ry)
            for (int rx = -2 - cx; rx <= 3 - cx; ++rx)
                if (rx < -1 || rx > 1 || ry < -1 || ry > 1)
                    off[cls][q++] = make_int2(rx, ry);
    }
    if (cudaMemcpyToSymbolAsync(c_m2l_off, off, sizeof off, 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return -1;
    g_const_ready[dev] = 1;
    return 0;
}

// packed FP32 pairs (real, imaginary) for the additions of the lane-per-source M2L
typedef unsigned long long m2l_f2;
__device__ __forceinline__ m2l_f2 m2l_pk2(float a, float b)
{
    m2l_f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void m2l_up2(m2l_f2 v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ m2l_f2 m2l_add2(m2l_f2 a, m2l_f2 b)
{
    m2l_f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

template <int P>
__global__ void __launch_bounds__(128) k_m2l_src(Work w, int64_t gw0, int64_t gw1)
{
    __shared__ float2 part[4][27][P + 1];
    const int64_t gw = gw0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (gw >= gw1)
        return;
    int l = 2;
    while (l < w.lv.maxdepth && gw >= w.lv.m2l_item0[l + 1])
        ++l;
    const int64_t g = gw - w.lv.m2l_item0[l];
    const int b = (int)(g & (((int64_t)1 << (2 * l)) - 1));
    const int sidx = (int)(g >> (2 * l));
    const SysDev &d = w.sys[sys_at_level(w, l, sidx)];
    if (w.bcount[d.box0[l] + b] == 0)
        return;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, p = w.p;
    const int ns = 1 << l, bx = b & (ns - 1), by = b >> l;
    const int cls = (by & 1) * 2 + (bx & 1);
    bool valid = false;
    int64_t sb = 0;
    float rr = 0.f, ri = 0.f;
    if (lane < 27) {
        const int2 o = c_m2l_off[cls][lane];
        const int jx = bx + o.x, jy = by + o.y;
        if (jx >= 0 && jy >= 0 && jx < ns && jy < ns) {
            sb = d.box0[l] + (int64_t)jy * ns + jx;
            valid = w.bcount[sb] != 0;
            const float den = (float)(o.x * o.x + o.y * o.y);
            rr = (float)o.x / den;  // rho = 1 / (dx + i dy)
            ri = -(float)o.y / den;
        }
    }
    if (valid) {
        m2l_f2 X[P];
        const float2 *src = w.M32 + sb * p;
        float pr = 1.f, pi = 0.f;
#pragma unroll
        for (int m = 0; m < P; ++m) {
            float2 a = m < p ? src[m] : make_float2(0.f, 0.f);
            const float sg = (m & 1) ? 1.f : -1.f;  // (-1)^(m+1)
            X[m] = m2l_pk2(sg * (pr * a.x - pi * a.y), sg * (pr * a.y + pi * a.x));
            const float t = pr * rr - pi * ri;
            pi = pr * ri + pi * rr;
            pr = t;
        }
        // y_l = sum_m C(m+l, m) x_m: with u = 1/(1 - s), sum_l y_l s^l = u X(u) = u (x_0 + u (x_1 + ... + u x_{P-1})),
        // and multiplying a truncated series by u is a prefix sum of its coefficients: P prefix sums of P terms,
        // additions only (re and im packed), no binomial table
        m2l_f2 T[P];
        T[0] = X[P - 1];
#pragma unroll
        for (int k = 1; k < P; ++k)
            T[k] = 0ull;
#pragma unroll
        for (int m = P - 2; m >= -1; --m) {
#pragma unroll
            for (int k = 1; k < P; ++k)
                T[k] = m2l_add2(T[k], T[k - 1]);
            if (m >= 0)
                T[0] = m2l_add2(T[0], X[m]);
        }
        float qr = rr, qi = ri;  // rho^(l+1)
#pragma unroll
        for (int ll = 0; ll < P; ++ll) {
            float br, bi;
            m2l_up2(T[ll], br, bi);
            part[wi][lane][ll] = make_float2(qr * br - qi * bi, qr * bi + qi * br);
            const float t = qr * rr - qi * ri;
            qi = qr * ri + qi * rr;
            qr = t;
        }
    } else if (lane < 27) {
#pragma unroll
        for (int ll = 0; ll < P; ++ll)
            part[wi][lane][ll] = make_float2(0.f, 0.f);
    }
    __syncwarp();
    if (lane < p) {
        float sr = 0.f, si = 0.f;
#pragma unroll 9
        for (int q = 0; q < 27; ++q) {
            const float2 v = part[wi][q][lane];
            sr += v.x;
            si += v.y;
        }
        w.L32[(d.box0[l] + b) * (int64_t)p + lane] = make_float2(sr, si);
    }
}

template <int P>
static void m2l_src_launch(const Work &w, int64_t a, int64_t b, cudaStream_t s)
{
    if (b <= a)
        return;
    unsigned blocks = (unsigned)(((b - a) * 32 + 127) / 128);
    k_m2l_src<P><<<blocks, 128, 0, s>>>(w, a, b);
}

template <int PM>
static void m2l_box_launch(const Work &w, const Tables &t, int adj, int64_t a, int64_t b, cudaStream_t s)
{
    if (b <= a)
        return;
    unsigned blocks = (unsigned)(((b - a) * 32 + 127) / 128);
    k_m2l<PM><<<blocks, 128, 0, s>>>(w, t, adj, a, b);
}

int launch_m2l(const Work &w, const Tables &t, int adj, cudaStream_t s, int prio)
{
    (void)prio;
    const int64_t total = w.lv.m2l_item0[w.lv.maxdepth + 1];
    if (w.lv.maxdepth < 2 || total == 0)
        return 0;
    // FP64 levels (all levels of the plain form; levels <= coarse_level of the precision form): lane = coefficient
    int l32 = w.mixed ? max(2, w.coarse_level + 1) : w.lv.maxdepth + 1;  // first FP32 level
    if (!m2l_constants_ready())
        l32 = w.lv.maxdepth + 1;  // constants not uploaded on this device: the lane-per-coefficient kernel for all
    const int64_t split = l32 > w.lv.maxdepth ? total : w.lv.m2l_item0[l32];
    int n = 0;
    if (split > 0) {
        if (w.p <= 8)
            m2l_box_launch<8>(w, t, adj, 0, split, s);
        else if (w.p <= 12)
            m2l_box_launch<12>(w, t, adj, 0, split, s);
        else if (w.p <= 16)
            m2l_box_launch<16>(w, t, adj, 0, split, s);
        else if (w.p <= 20)
            m2l_box_launch<20>(w, t, adj, 0, split, s);
        else if (w.p <= 24)
            m2l_box_launch<24>(w, t, adj, 0, split, s);
        else
            m2l_box_launch<32>(w, t, adj, 0, split, s);
        ++n;
    }
    // FP32 levels: the tensor cores take l32 .. the finest level they cover, the CUDA cores the rest
    int64_t src0 = split;
    if (split < total && w.m2l_tc && t.m2l_tc && m2l_tc_supported(w.p)) {
        const int lt = min(w.lv.maxdepth, m2l_tc_max_level());
        const int k = lt >= l32 ? launch_m2l_tc(w, t, l32, lt, s) : 0;
        if (k > 0) {
            n += k;
            src0 = w.lv.m2l_item0[lt + 1];
        }
    }
    if (src0 < total) {
        if (w.p <= 8)
            m2l_src_launch<8>(w, src0, total, s);
        else if (w.p <= 12)
            m2l_src_launch<12>(w, src0, total, s);
        else if (w.p <= 14)
            m2l_src_launch<14>(w, src0, total, s);
        else if (w.p <= 16)
            m2l_src_launch<16>(w, src0, total, s);
        else if (w.p <= 17)
            m2l_src_launch<17>(w, src0, total, s);
        else if (w.p <= 20)
            m2l_src_launch<20>(w, src0, total, s);
        else if (w.p <= 24)
            m2l_src_launch<24>(w, src0, total, s);
        else
            m2l_src_launch<32>(w, src0, total, s);
        ++n;
    }
    return n;
}

// ------------------------------------------------------------------ level exchange of sharded evaluations

// Level l's multipoles (radius-scaled, in the level's storage precision) and box particle counts of the first
// system, to dst (4^l * p double2, boxes row-major) and cnt (4^l); boxes without particles give zeros (their
// multipoles are never written by P2M / M2M).
__global__ void k_level_export(Work w, int l, double2 *__restrict__ dst, long long *__restrict__ cnt)
{
    const SysDev &d = w.sys[0];
    const int p = w.p;
    const int64_t nb = (int64_t)1 << (2 * l), i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nb * p)
        return;
    const int64_t b = i / p, box = d.box0[l] + b;
    const int c = w.bcount[box];
    if (i - b * p == 0)
        cnt[b] = c;
    double2 v = make_double2(0.0, 0.0);
    if (c != 0) {
        if (level_fp64(w, l)) {
            v = w.M64[box * p + (i - b * p)];
        } else {
            const float2 f = w.M32[box * p + (i - b * p)];
            v = make_double2((double)f.x, (double)f.y);
        }
    }
    dst[i] = v;
}

// The reverse: level l's multipoles and counts of the first system from src / cnt (same layout).
__global__ void k_level_import(Work w, int l, const double2 *__restrict__ src, const long long *__restrict__ cnt)
{
    const SysDev &d = w.sys[0];
    const int p = w.p;
    const int64_t nb = (int64_t)1 << (2 * l), i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nb * p)
        return;
    const int64_t b = i / p, box = d.box0[l] + b;
    if (i - b * p == 0)
        w.bcount[box] = (int)cnt[b];
    const double2 v = src[i];
    if (level_fp64(w, l))
        w.M64[box * p + (i - b * p)] = v;
    else
        w.M32[box * p + (i - b * p)] = make_float2((float)v.x, (float)v.y);
}

int launch_level_export(const Work &w, int l, double2 *dst, long long *cnt, cudaStream_t s)
{
    const int64_t items = ((int64_t)1 << (2 * l)) * w.p;
    k_level_export<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(w, l, dst, cnt);
    return 1;
}

int launch_level_import(const Work &w, int l, const double2 *src, const long long *cnt, cudaStream_t s)
{
    const int64_t items = ((int64_t)1 << (2 * l)) * w.p;
    k_level_import<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(w, l, src, cnt);
    return 1;
}

// ------------------------------------------------------------------ stage 7: L2L (block = the 4 children of a parent)

// Four warps, one per child of one parent box at level l, lane k = coefficient; the parent's local expansion is
// staged once in shared memory; the table is stored [child][j][k] so that lanes read consecutive entries.
template <int PM, typename RA, typename SPa, typename SCh>
__global__ void __launch_bounds__(128) k_l2l(Work w, const double2 *__restrict__ tab64,
                                             const float2 *__restrict__ tab32, int l, const SPa *__restrict__ parent,
                                             SCh *child)
{
    __shared__ cx<RA> sh[FMM_PMAX];
    const int p = w.p, lane = threadIdx.x & 31, c = threadIdx.x >> 5;
    const int64_t nb = (int64_t)1 << (2 * l);
    const int64_t g = blockIdx.x;  // parent box over the systems that have level l + 1
    if (g >= (int64_t)w.lv.nsys_at[l + 1] * nb)
        return;
    const int b = (int)(g & (nb - 1));
    const int sidx = (int)(g >> (2 * l));
    const SysDev &d = w.sys[sys_at_level(w, l + 1, sidx)];
    const int64_t pbox = d.box0[l] + b;
    if (w.bcount[pbox] == 0)
        return;  // block-uniform: no child has particles
    if (threadIdx.x < p)
        sh[threadIdx.x] = ldc<RA>(parent, pbox * p + threadIdx.x);
    __syncthreads();
    const int ns = 1 << l, bx = b & (ns - 1), by = b >> l;
    const int64_t cbox = d.box0[l + 1] + (int64_t)(2 * by + (c >> 1)) * (2 * ns) + (2 * bx + (c & 1));
    if (lane >= p || w.bcount[cbox] == 0)
        return;
    cx<RA> acc = ldc<RA>(child, cbox * p + lane);
#pragma unroll
    for (int j = 0; j < PM; ++j)  // entries with j < k are zero in the table
        if (j < p)
            acc = cadd(acc, cmul(ld_tab<RA>(tab64, tab32, (c * FMM_PMAX + j) * FMM_PMAX + lane), sh[j]));
    stc(child, cbox * p + lane, acc);
}

template <int PM>
static void l2l_launch(const Work &w, const Tables &t, int l, int adj, unsigned blocks, cudaStream_t s)
{
    const bool pd = level_fp64(w, l), cd = level_fp64(w, l + 1);
    double2 *L64 = adj ? w.AL64 : w.L64;
    if (pd && cd)
        k_l2l<PM, double, double2, double2><<<blocks, 128, 0, s>>>(w, t.l2l64, t.l2l32, l, L64, L64);
    else if (pd)
        k_l2l<PM, double, double2, float2><<<blocks, 128, 0, s>>>(w, t.l2l64, t.l2l32, l, L64, w.L32);
    else
        k_l2l<PM, float, float2, float2><<<blocks, 128, 0, s>>>(w, t.l2l64, t.l2l32, l, w.L32, w.L32);
}

int launch_l2l(const Work &w, const Tables &t, int l, int adj, cudaStream_t s, int prio)
{
    (void)prio;
    const int64_t blocks = (int64_t)w.lv.nsys_at[l + 1] * ((int64_t)1 << (2 * l));
    if (blocks == 0)
        return 0;
    if (w.p <= 8)
        l2l_launch<8>(w, t, l, adj, (unsigned)blocks, s);
    else if (w.p <= 16)
        l2l_launch<16>(w, t, l, adj, (unsigned)blocks, s);
    else if (w.p <= 20)
        l2l_launch<20>(w, t, l, adj, (unsigned)blocks, s);
    else if (w.p <= 24)
        l2l_launch<24>(w, t, l, adj, (unsigned)blocks, s);
    else
        l2l_launch<32>(w, t, l, adj, (unsigned)blocks, s);
    return 1;
}

// ------------------------------------------------------------------ stages 8 + 10: L2P, sum, unsort

template <typename R, typename S>
__device__ __forceinline__ cx<R> horner(const S *__restrict__ b, int64_t base, int p, cx<R> z)
{
    cx<R> acc = ldc<R>(b, base + p - 1);
    for (int l = p - 2; l >= 0; --l)
        acc = cadd(cmul(acc, z), ldc<R>(b, base + l));
    return acc;
}

// Horner with a compile-time bound PM >= p: the coefficient loads are independent of the recurrence and all
// issue before it starts.
template <int PM, typename R, typename S>
__device__ __forceinline__ cx<R> horner_u(const S *__restrict__ b, int64_t base, int p, cx<R> z)
{
    cx<R> c[PM];
#pragma unroll
    for (int l = 0; l < PM; ++l)
        c[l] = l < p ? ldc<R>(b, base + l) : cx<R>{(R)0, (R)0};
    cx<R> acc = c[PM - 1];
#pragma unroll
    for (int l = PM - 2; l >= 0; --l)
        acc = cadd(cmul(acc, z), c[l]);
    return acc;
}

// Stage 8 alone for the precision form: the FP32 far field of every particle whose leaf level is FP32, in leaf
// order (runs on the sweep stream, so that only the sum below waits for the near field).
template <int PM>
__global__ void k_l2p32(Work w)
{
    int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= w.n)
        return;
    int k = w.nsys == 1 ? 0 : find_sys_by_particle(w.sys, w.nsys, pos);
    const SysDev &d = w.sys[k];
    int L = d.depth;
    if (L < 2 || level_fp64(w, L))
        return;
    int64_t base = (d.box0[L] + (int)(w.sleaf[pos] - d.leaf0)) * (int64_t)w.p;
    float4 hh = w.eh[pos], ll = w.el[pos];
    cx<float> z = {(hh.x + ll.x) * d.inv_s, (hh.z + ll.z) * d.inv_s};
    cx<float> s = horner_u<PM, float>(w.L32, base, w.p, z);
    float fs = (float)d.far_scale;
    w.far32[(int64_t)pos * w.nf_stride] = make_float2(s.re * fs, -s.im * fs);
}

int launch_l2p(const Work &w, cudaStream_t s)
{
    if (!w.mixed || !w.far32)
        return 0;
    const unsigned nb = (unsigned)((w.n + 255) / 256);
    if (w.p <= 8)
        k_l2p32<8><<<nb, 256, 0, s>>>(w);
    else if (w.p <= 16)
        k_l2p32<16><<<nb, 256, 0, s>>>(w);
    else if (w.p <= 20)
        k_l2p32<20><<<nb, 256, 0, s>>>(w);
    else if (w.p <= 24)
        k_l2p32<24><<<nb, 256, 0, s>>>(w);
    else
        k_l2p32<32><<<nb, 256, 0, s>>>(w);
    return 1;
}

// Stage 10 in caller order: thread i gathers its particle's near and far parts from leaf-order position
// iperm[i] and writes u[i], v[i] contiguously (so the outputs may also be page-locked host memory).
template <int PM>
__global__ void k_combine(Work w, int use_near, int use_far, double *__restrict__ u, double *__restrict__ v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && w.status_host)
        *w.status_host = *w.status;  // every earlier stage has finished: hand the status word to the host
    if (i >= w.n)
        return;
    int pos = w.iperm[i];
    int k = w.nsys == 1 ? 0 : find_sys_by_particle(w.sys, w.nsys, pos);
    const SysDev &d = w.sys[k];
    int L = d.depth;
    bool far = use_far && L >= 2;
    // first local coefficient of the particle's leaf (read only where the far field is evaluated here)
    auto leaf_base = [&]() { return (d.box0[L] + (int)(w.sleaf[pos] - d.leaf0)) * (int64_t)w.p; };
    if (w.mixed && !level_fp64(w, L)) {
        // precision form: FP32 far field and sum, one conversion to FP64 at the end
        float fu = 0.f, fv = 0.f;
        if (far && w.far32) {
            const float2 f = w.far32[(int64_t)pos * w.nf_stride];  // k_l2p32
            fu = f.x;
            fv = f.y;
        } else if (far) {
            float4 hh = w.eh[pos], ll = w.el[pos];
            cx<float> z = {(hh.x + ll.x) * d.inv_s, (hh.z + ll.z) * d.inv_s};
            cx<float> s = horner_u<PM, float>(w.L32, leaf_base(), w.p, z);
            float fs = (float)d.far_scale;
            fu = s.re * fs;
            fv = -s.im * fs;
        }
        float2 t = make_float2(0.f, 0.f);
        if (use_near && w.p2p_rows) {  // the three source rows' parts, fixed order
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float2 q = w.nearp[(int64_t)r * w.n + pos];
                t.x += q.x;
                t.y += q.y;
            }
        } else if (use_near) {
            t = w.near32[(int64_t)pos * w.nf_stride];
        }
        if (use_near && w.p2p_sym && d.s_unit <= P2P_SPLIT_S) {
            // symmetric near field: add the reactions from the four backward neighbour leaves, fixed order
            const int ns = 1 << L, local = (int)(w.sleaf[pos] - d.leaf0);
            const int ix = local & (ns - 1), iy = local >> L;
            const int2 fwd[4] = {{1, 0}, {1, 1}, {0, 1}, {-1, 1}};
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) {
                const int ax = ix - fwd[dd].x, ay = iy - fwd[dd].y;
                if (ax < 0 || ax >= ns || ay < 0)
                    continue;
                const int A = (int)d.leaf0 + ay * ns + ax;
                if (w.start[A + 1] == w.start[A])
                    continue;  // empty leaf: its warp wrote nothing
                const float2 r = w.nearp[(int64_t)dd * w.n + pos];
                t.x += r.x;
                t.y += r.y;
            }
        }
        u[i] = (double)(t.x + fu);
        v[i] = (double)(t.y + fv);
        return;
    }
    double fu = 0.0, fv = 0.0;
    if (far) {
        cx<double> z;
        if (w.mixed) {
            float4 hh = w.eh[pos], ll = w.el[pos];
            z = {((double)hh.x + (double)ll.x) / (double)d.s_unit, ((double)hh.z + (double)ll.z) / (double)d.s_unit};
        } else {
            int local = (int)(w.sleaf[pos] - d.leaf0);
            int ix = local & ((1 << L) - 1), iy = local >> L;
            z = {(w.sx[pos] - d.x0) * d.scale - (ix + 0.5), (w.sy[pos] - d.y0) * d.scale - (iy + 0.5)};
        }
        cx<double> s = horner<double>(w.L64, leaf_base(), w.p, z);
        fu = s.re * d.far_scale;
        fv = -s.im * d.far_scale;
    }
    double nu = 0.0, nv = 0.0;
    if (use_near) {
        if (w.mixed) {
            float2 t = w.near32[(int64_t)pos * w.nf_stride];
            nu = t.x;
            nv = t.y;
        } else {
            double2 t = w.near64[pos];
            nu = t.x;
            nv = t.y;
        }
    }
    u[i] = nu + fu;
    v[i] = nv + fv;
}

// The common precision-form case of stage 10 (the near field from the target-side kernel, the far field from
// k_l2p32, every leaf level FP32): the same sums as k_combine in a kernel small enough to keep every warp slot
// of an SM resident, two particles per thread, so that the dependent gathers through iperm overlap.
__global__ void __launch_bounds__(256) k_combine32(Work w, int use_near, int use_far, double *__restrict__ u,
                                                   double *__restrict__ v)
{
    const int i0 = blockIdx.x * 512 + threadIdx.x;
    if (i0 == 0 && w.status_host)
        *w.status_host = *w.status;  // every earlier stage has finished: hand the status word to the host
    int pos[2];
#pragma unroll
    for (int h = 0; h < 2; ++h)
        pos[h] = i0 + 256 * h < w.n ? w.iperm[i0 + 256 * h] : -1;
    float2 t[2], f[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (w.nf_stride == 2 && pos[h] >= 0) {  // near and far side by side: one 16-byte gather
            const float4 q = reinterpret_cast<const float4 *>(w.near32)[pos[h]];
            t[h] = use_near ? make_float2(q.x, q.y) : make_float2(0.f, 0.f);
            f[h] = use_far ? make_float2(q.z, q.w) : make_float2(0.f, 0.f);
        } else {
            t[h] = use_near && pos[h] >= 0 ? w.near32[(int64_t)pos[h] * w.nf_stride] : make_float2(0.f, 0.f);
            f[h] = use_far && pos[h] >= 0 ? w.far32[(int64_t)pos[h] * w.nf_stride] : make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (pos[h] >= 0) {
            u[i0 + 256 * h] = (double)(t[h].x + f[h].x);
            v[i0 + 256 * h] = (double)(t[h].y + f[h].y);
        }
}

int launch_combine(const Work &w, int use_near, int use_far, double *u, double *v, cudaStream_t s)
{
    const unsigned nb = (unsigned)((w.n + 255) / 256);
    const int lmin = w.coarse_level + 1 > 2 ? w.coarse_level + 1 : 2;  // every system this deep: all leaves FP32
    if (w.mixed && !w.p2p_rows && !w.p2p_sym && (!use_far || w.far32) && lmin <= FMM_MAXL &&
        w.lv.nsys_at[lmin] == w.nsys) {
        k_combine32<<<(unsigned)((w.n + 511) / 512), 256, 0, s>>>(w, use_near, use_far, u, v);
        return 1;
    }
    if (w.p <= 8)
        k_combine<8><<<nb, 256, 0, s>>>(w, use_near, use_far, u, v);
    else if (w.p <= 16)
        k_combine<16><<<nb, 256, 0, s>>>(w, use_near, use_far, u, v);
    else if (w.p <= 20)
        k_combine<20><<<nb, 256, 0, s>>>(w, use_near, use_far, u, v);
    else if (w.p <= 24)
        k_combine<24><<<nb, 256, 0, s>>>(w, use_near, use_far, u, v);
    else
        k_combine<32><<<nb, 256, 0, s>>>(w, use_near, use_far, u, v);
    return 1;
}

// ------------------------------------------------------------------ adjoint: far-field part (FP64)

// With G = gu + i gv, q = -i gamma / 2pi, w the forward far field and phi(z) = sum_i G_i / (z - z_i) the far
// field of the adjoint charges (same tree, same truncation), the transpose of the far-field operator is
// (T^T G)_j = -phi(z_j) because the truncated operator is antisymmetric. Hence
//   dL/dgamma_j = -Im phi(z_j) / 2pi,  dL/dx_j = Re(G_j w'(z_j)) - Re(q_j phi'(z_j)),
//   dL/dy_j = -Im(G_j w'(z_j)) + Im(q_j phi'(z_j)).
__global__ void k_adjoint_far(Work w)
{
    int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= w.n)
        return;
    int k = w.nsys == 1 ? 0 : find_sys_by_particle(w.sys, w.nsys, pos);
    const SysDev &d = w.sys[k];
    int L = d.depth;
    double dg = 0.0, dx = 0.0, dy = 0.0;
    if (L >= 2) {
        int local = (int)(w.sleaf[pos] - d.leaf0);
        int64_t base = (d.box0[L] + local) * (int64_t)w.p;
        int ix = local & ((1 << L) - 1), iy = local >> L;
        double scale = d.scale, wl = d.wl;
        cx<double> z = {(w.sx[pos] - d.x0) * scale - (ix + 0.5), (w.sy[pos] - d.y0) * scale - (iy + 0.5)};
        // forward derivative w' and adjoint phi, phi' by Horner on the polynomial and its derivative
        cx<double> bw = {0, 0}, bwd = {0, 0}, ph = {0, 0}, phd = {0, 0};
        for (int l = w.p - 1; l >= 0; --l) {
            cx<double> bl = ldc<double>(w.L64, base + l), Bl = ldc<double>(w.AL64, base + l);
            bwd = cadd(cmul(bwd, z), bw);
            bw = cadd(cmul(bw, z), bl);
            phd = cadd(cmul(phd, z), ph);
            ph = cadd(cmul(ph, z), Bl);
        }
        const double twopi = 2.0 * 3.14159265358979323846;
        cx<double> wp = {bwd.re / (twopi * wl * wl), bwd.im / (twopi * wl * wl)};
        cx<double> phi = {ph.re / wl, ph.im / wl};
        cx<double> phip = {phd.re / (wl * wl), phd.im / (wl * wl)};
        cx<double> G = {w.sgu[pos], w.sgv[pos]};
        cx<double> q = {0.0, -w.sg[pos] / twopi};
        cx<double> Gw = cmul(G, wp), qp = cmul(q, phip);
        dg = -phi.im / twopi;
        dx = Gw.re - qp.re;
        dy = -Gw.im + qp.im;
    }
    w.adj_far[pos] = dg;
    w.adj_far[(int64_t)w.n + pos] = dx;
    w.adj_far[2 * (int64_t)w.n + pos] = dy;
}

int launch_adjoint_far(const Work &w, cudaStream_t s)
{
    k_adjoint_far<<<(w.n + 255) / 256, 256, 0, s>>>(w);
    return 1;
}

__global__ void k_adjoint_add(Work w, double *__restrict__ dg, double *__restrict__ dx, double *__restrict__ dy)
{
    int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= w.n)
        return;
    int i = w.perm[pos];
    int64_t n = w.n;
    if (dg)
        dg[i] += w.adj_far[pos];
    if (dx)
        dx[i] += w.adj_far[n + pos];
    if (dy)
        dy[i] += w.adj_far[2 * n + pos];
}

int launch_adjoint_combine(const Work &w, double *dg, double *dx, double *dy, cudaStream_t s)
{
    k_adjoint_add<<<(w.n + 255) / 256, 256, 0, s>>>(w, dg, dx, dy);
    return 1;
}

// ------------------------------------------------------------------ tables

static double binom_host(int n, int k)
{
    if (k < 0 || k > n)
        return 0.0;
    double c = 1.0;
    for (int i = 1; i <= k; ++i)
        c = c * (double)(n - k + i) / (double)i;
    return c;
}

// m2m[c][m][n] = C(n, m) delta_c^(n-m) 2^-m (m <= n), delta_c = ((cx - 1/2) + i (cy - 1/2)) / 2;
// l2l[c][j][k] = C(j, k) delta_c^(j-k) 2^-(j+1) (j >= k), delta_c = (cx - 1/2) + i (cy - 1/2);
// rho[o][k] = (1/delta_o)^k, delta_o = dx + i dy; binom[m][l] = C(m + l, m).
// Both translation tables are stored with the output index last, so a warp whose lanes are outputs reads
// consecutive entries.
void build_tables_host(int p, double2 *m2m, double2 *l2l, double2 *rho, double *binom)
{
    (void)p;
    const int P = FMM_PMAX;
    for (int c = 0; c < 4; ++c) {
        double ddx = (c & 1) - 0.5, ddy = (c >> 1) - 0.5;
        double pre[2 * FMM_PMAX][2], prl[2 * FMM_PMAX][2];
        pre[0][0] = 1.0;
        pre[0][1] = 0.0;
        prl[0][0] = 1.0;
        prl[0][1] = 0.0;
        for (int k = 1; k < P; ++k) {
            double ar = 0.5 * ddx, ai = 0.5 * ddy;  // M2M delta
            pre[k][0] = pre[k - 1][0] * ar - pre[k - 1][1] * ai;
            pre[k][1] = pre[k - 1][0] * ai + pre[k - 1][1] * ar;
            prl[k][0] = prl[k - 1][0] * ddx - prl[k - 1][1] * ddy;  // L2L delta
            prl[k][1] = prl[k - 1][0] * ddy + prl[k - 1][1] * ddx;
        }
        for (int n = 0; n < P; ++n)      // output coefficient
            for (int m = 0; m < P; ++m) {  // input coefficient
                double2 t = make_double2(0.0, 0.0), s = make_double2(0.0, 0.0);
                if (m <= n) {
                    double f = binom_host(n, m) * ldexp(1.0, -m);
                    t = make_double2(f * pre[n - m][0], f * pre[n - m][1]);
                }
                m2m[(c * P + m) * P + n] = t;
                if (m >= n) {  // l2l: output k = n, input j = m >= k
                    double f = binom_host(m, n) * ldexp(1.0, -(m + 1));
                    s = make_double2(f * prl[m - n][0], f * prl[m - n][1]);
                }
                l2l[(c * P + m) * P + n] = s;
            }
    }
    const int RS = 2 * FMM_PMAX + 2;
    for (int oy = -3; oy <= 3; ++oy)
        for (int ox = -3; ox <= 3; ++ox) {
            int o = (oy + 3) * 7 + (ox + 3);
            double den = (double)(ox * ox + oy * oy);
            double rr = den > 0 ? ox / den : 0.0, ri = den > 0 ? -oy / den : 0.0;  // 1/(ox + i oy)
            double pr = 1.0, pi = 0.0;
            for (int k = 0; k < RS; ++k) {
                rho[o * RS + k] = make_double2(pr, pi);
                double nr = pr * rr - pi * ri, ni = pr * ri + pi * rr;
                pr = nr;
                pi = ni;
            }
        }
    for (int m = 0; m < P; ++m)
        for (int l = 0; l < P; ++l)
            binom[m * P + l] = binom_host(m + l, m);
}

}  // namespace fmm
