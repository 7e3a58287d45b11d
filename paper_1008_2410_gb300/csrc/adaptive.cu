// adaptive.cu -- the FMM on an adaptive quadtree, for uneven particle densities (the paper's closing section
// names them as the step beyond its uniform tree).
//
// Tree. Particles are binned at the maximum depth L in Morton order (binning.cu with Work::morton), so every
// box of every level owns one contiguous run of the sorted particles: box m of level l holds
// start[m << 2(L - l)] .. start[(m + 1) << 2(L - l)). A box is split while it holds more than B particles and
// its level is below L. Hence box (l, m) exists iff l == 0 or its parent holds more than B particles, and
// nothing about the tree is stored: every kernel reads it off `start`.
//
// Lists (Carrier, Greengard and Rokhlin), walked on the fly:
//   U(b), leaf b: leaves adjacent to b, b included          -> exact K_sigma (Eq. 6), stage 9
//   V(b): boxes of b's level whose parent is adjacent to b's parent, not adjacent to b   -> M2L, stage 6
//   W(b), leaf b: boxes below b's colleagues whose parent is adjacent to b but which are not themselves
//         adjacent to b                                    -> multipole evaluated at b's particles
//   X(b): leaves c with b in W(c), i.e. coarser leaves adjacent to b's parent and not to b -> P2L
// Expansions exist on levels >= 2 (levels 0 and 1 hold no well separated pair). They use the uniform tree's
// radius scaling, so its level-independent tables (M2M, L2L, binomials, powers of 1/delta) serve here too;
// zeta = (z - c) / w for a box of side w, charges q' = -i gamma (1 / 2pi applied at the end):
//   multipole  a~_m = sum_j q'_j zeta_j^m
//   local      b^_k = w^(k+1) b_k, so that the far field at z is (1/w) sum_k b^_k zeta^k
//   M2M        a~P_n = sum_{m<=n} C(n, m) delta^(n-m) 2^-m a~C_m,        delta = (c_child - c_parent) / w_parent
//   M2L        b^_k += rho^(k+1) sum_m C(m+k, m) (-1)^(m+1) rho^m a~_m,  rho = 1 / delta, delta = (c_src - c_tgt) / w
//   L2L        b^C_k = sum_{j>=k} C(j, k) 2^-(j+1) delta^(j-k) b^P_j,   delta = (c_child - c_parent) / w_child
//   P2L        b^_k += -sum_j q'_j / s_j^(k+1),                        s_j = (z_j - c) / w
//   M2P        w(z) += (1/w_s) sum_m a~_m / t^(m+1),                   t = (z - c_s) / w_s
// Two forms: FP64 throughout, or the precision form (FP32 expansions and FP32 near field on hi + lo split
// coordinates, FP64 sums per source leaf and at the end).
#include <type_traits>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr double kTwoPi = 6.283185307179586476925;
constexpr int kStack = 48;  // DFS stack of the U / W walk; depth <= 2 (L - l) + 2 <= 26 for L <= 12
constexpr int kRS = 2 * FMM_PMAX + 2;  // row length of the 1/delta power table

struct Tree {
    const int *start;
    int L, B;
};

__device__ __forceinline__ int box_count(const Tree &t, int l, unsigned m)
{
    const int sh = 2 * (t.L - l);
    return t.start[(size_t)(m + 1) << sh] - t.start[(size_t)m << sh];
}

__device__ __forceinline__ int box_first(const Tree &t, int l, unsigned m) { return t.start[(size_t)m << (2 * (t.L - l))]; }

__device__ __forceinline__ bool box_exists(const Tree &t, int l, int x, int y)
{
    return l == 0 || box_count(t, l - 1, morton2((unsigned)x >> 1, (unsigned)y >> 1)) > t.B;
}

__device__ __forceinline__ bool box_split(const Tree &t, int l, int x, int y)
{
    return l < t.L && box_count(t, l, morton2(x, y)) > t.B;
}

// closed squares touch or overlap (ranges of depth-L cells)
__device__ __forceinline__ bool adjacent(int L, int l1, int x1, int y1, int l2, int x2, int y2)
{
    const int s1 = L - l1, s2 = L - l2;
    const int ax0 = x1 << s1, ax1 = ((x1 + 1) << s1) - 1, ay0 = y1 << s1, ay1 = ((y1 + 1) << s1) - 1;
    const int bx0 = x2 << s2, bx1 = ((x2 + 1) << s2) - 1, by0 = y2 << s2, by1 = ((y2 + 1) << s2) - 1;
    return ax0 <= bx1 + 1 && bx0 <= ax1 + 1 && ay0 <= by1 + 1 && by0 <= ay1 + 1;
}

// Deepest existing box covering cell (x, y) of level l (a leaf whenever it is coarser than l).
__device__ __forceinline__ void covering_box(const Tree &t, int &l, int &x, int &y)
{
    while (l > 0 && !box_exists(t, l, x, y)) {
        --l;
        x >>= 1;
        y >>= 1;
    }
}

__device__ __forceinline__ int pack_box(int l, int x, int y) { return (l << 26) | (x << 13) | y; }

// complex arithmetic in R (double or float)
template <typename R>
struct cpx {
    R re, im;
};
template <typename R>
__device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cpx<R> cadd(cpx<R> a, cpx<R> b)
{
    return {a.re + b.re, a.im + b.im};
}

// Storage of the expansions: FP64 form double2 (M64 / L64), precision form float2 (M32 / L32).
template <typename R>
struct Store;
template <>
struct Store<double> {
    using S = double2;
    using V2 = double4_16a;  // two complex coefficients
    __device__ static double2 *mp(const Work &w) { return w.M64; }
    __device__ static double2 *loc(const Work &w) { return w.L64; }
    __device__ static const double2 *m2m(const Tables &t) { return t.m2m64; }
    __device__ static const double2 *l2l(const Tables &t) { return t.l2l64; }
    __device__ static const double2 *rho(const Tables &t) { return t.rho64; }
    __device__ static const double *binom(const Tables &t) { return t.binom64; }
};
template <>
struct Store<float> {
    using S = float2;
    using V2 = float4;  // two complex coefficients
    __device__ static float2 *mp(const Work &w) { return w.M32; }
    __device__ static float2 *loc(const Work &w) { return w.L32; }
    __device__ static const float2 *m2m(const Tables &t) { return t.m2m32; }
    __device__ static const float2 *l2l(const Tables &t) { return t.l2l32; }
    __device__ static const float2 *rho(const Tables &t) { return t.rho32; }
    __device__ static const float *binom(const Tables &t) { return t.binom32; }
};

template <typename R, typename S>
__device__ __forceinline__ cpx<R> ld(const S *p)
{
    const S v = *p;
    return {(R)v.x, (R)v.y};
}
template <typename R, typename S>
__device__ __forceinline__ void st(S *p, cpx<R> v)
{
    p->x = v.re;
    p->y = v.im;
}

template <typename R>
__device__ __forceinline__ typename Store<R>::S *mp_of(const Work &w, int l, unsigned m)
{
    return Store<R>::mp(w) + ((size_t)w.sys[0].box0[l] + m) * w.p;
}
template <typename R>
__device__ __forceinline__ typename Store<R>::S *loc_of(const Work &w, int l, unsigned m)
{
    return Store<R>::loc(w) + ((size_t)w.sys[0].box0[l] + m) * w.p;
}

__device__ __forceinline__ double2 centre(const SysDev &d, int l, int x, int y)
{
    const double w = ldexp(d.S, -l);
    return make_double2(d.x0 + (x + 0.5) * w, d.y0 + (y + 0.5) * w);
}

// ------------------------------------------------------------------ existing boxes of every level

// The boxes of level l + 1 are the four children of each box of level l holding more than B particles. One
// thread per box of levels 1 .. L-1; each level's index range is padded to a multiple of 32 so that a warp
// appends its children with one atomic.
__global__ void k_ad_enum(Work w)
{
    const SysDev &d = w.sys[0];
    const Tree t{w.start, d.depth, w.adapt_cap};
    const int L = d.depth;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int lp = 1;
    int64_t base = 0;
    while (lp < L && g >= base + (((1ll << (2 * lp)) + 31) & ~31ll)) {
        base += ((1ll << (2 * lp)) + 31) & ~31ll;
        ++lp;
    }
    if (lp >= L)
        return;  // whole warps leave together: every level range is a multiple of 32
    const int64_t m = g - base;
    const bool split = m < (1ll << (2 * lp)) && box_count(t, lp, (unsigned)m) > t.B;
    const unsigned mask = __ballot_sync(0xffffffffu, split);
    if (!mask)
        return;
    const int lane = threadIdx.x & 31;
    int pos = 0;
    if (lane == __ffs(mask) - 1)
        pos = atomicAdd(&w.ad_cnt[lp + 1], 4 * __popc(mask));
    pos = __shfl_sync(0xffffffffu, pos, __ffs(mask) - 1) + 4 * __popc(mask & ((1u << lane) - 1));
    if (split) {
        int *lst = w.ad_list + d.box0[lp + 1];
        for (int c = 0; c < 4; ++c)
            lst[pos + c] = (int)(4 * m + c);
    }
}

int64_t enum_threads(int L)
{
    int64_t t = 0;
    for (int l = 1; l < L; ++l)
        t += ((1ll << (2 * l)) + 31) & ~31ll;
    return t;
}

constexpr int kSweepBlocks = 152 * 16;  // grid of the list-driven sweep kernels (4 warps per block)

// Sum over a warp's lanes of PM complex partial sums per lane (lanes >= used hold zeros): in the precision form
// through shared memory, one row per lane and lane k adding column k (PM stores and `used` loads per lane, against
// a butterfly of 2 PM log2(32) shuffles); in the FP64 form by the butterfly. Lane k < PM returns coefficient k.
template <typename R, int PM>
__device__ __forceinline__ cpx<R> warp_coeff_sum(cpx<R> *acc, int lane, int used)
{
    if constexpr (std::is_same<R, float>::value) {
        __shared__ float2 red[4][32][PM + 1];
        float2(*row)[PM + 1] = red[threadIdx.x >> 5];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < PM; ++k)
            row[lane][k] = make_float2(acc[k].re, acc[k].im);
        __syncwarp();
        cpx<R> s = {0.f, 0.f};
        if (lane < PM)
            for (int r = 0; r < used; ++r) {
                const float2 v = row[r][lane];
                s.re += v.x;
                s.im += v.y;
            }
        __syncwarp();
        return s;
    } else {
        (void)used;
#pragma unroll
        for (int k = 0; k < PM; ++k)
            for (int o = 16; o > 0; o >>= 1) {
                acc[k].re += __shfl_xor_sync(0xffffffffu, acc[k].re, o);
                acc[k].im += __shfl_xor_sync(0xffffffffu, acc[k].im, o);
            }
        cpx<R> s = acc[0];
#pragma unroll
        for (int k = 1; k < PM; ++k)
            if (lane == k)
                s = acc[k];
        return s;
    }
}

// ------------------------------------------------------------------ stage 4: P2M at the leaves of level l

// One warp per leaf; lane = particle (32 at a time), each lane accumulating the PM coefficients of its particles
// in registers (powers by repeated multiplication), then a butterfly sum over the warp. Positions relative to
// the box centre are formed in FP64.
template <typename R, int PM>
__global__ void __launch_bounds__(128) k_ad_p2m(Work w, int l)
{
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const SysDev &d = w.sys[0];
    const Tree t{w.start, d.depth, w.adapt_cap};
    const int nbx = w.ad_cnt[l], p = w.p;
    const double iw = ldexp(1.0, l) / d.S;
    for (int idx = blockIdx.x * 4 + wi; idx < nbx; idx += gridDim.x * 4) {
        const unsigned m = (unsigned)w.ad_list[d.box0[l] + idx];
        const int bx = (int)compact1(m), by = (int)compact1(m >> 1);
        if (box_split(t, l, bx, by))
            continue;
        const int j0 = box_first(t, l, m), cnt = box_count(t, l, m);
        const double2 c = centre(d, l, bx, by);
        cpx<R> acc[PM];
#pragma unroll
        for (int k = 0; k < PM; ++k)
            acc[k] = {(R)0, (R)0};
        for (int e = lane; e < cnt; e += 32) {
            const int j = j0 + e;
            const cpx<R> z = {(R)((w.sx[j] - c.x) * iw), (R)((w.sy[j] - c.y) * iw)};
            const R g = (R)w.sg[j];
            cpx<R> pw = {(R)0, -g};  // q' = -i gamma
#pragma unroll
            for (int k = 0; k < PM; ++k) {
                acc[k] = cadd(acc[k], pw);
                pw = cmul(pw, z);
            }
        }
        const cpx<R> sum = warp_coeff_sum<R, PM>(acc, lane, min(cnt, 32));
        if (lane < p)
            st(mp_of<R>(w, l, m) + lane, sum);
    }
}

// ------------------------------------------------------------------ stage 5: M2M into the split boxes of level l

template <typename R>
__global__ void __launch_bounds__(128) k_ad_m2m(Work w, Tables tb, int l)
{
    __shared__ cpx<R> sa[4][4][FMM_PMAX];
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const SysDev &d = w.sys[0];
    const Tree t{w.start, d.depth, w.adapt_cap};
    const int nbx = w.ad_cnt[l], p = w.p, P = FMM_PMAX;
    const auto *T = Store<R>::m2m(tb);  // [c][input m][output n]
    for (int idx = blockIdx.x * 4 + wi; idx < nbx; idx += gridDim.x * 4) {
        const unsigned m = (unsigned)w.ad_list[d.box0[l] + idx];
        const int bx = (int)compact1(m), by = (int)compact1(m >> 1);
        if (!box_split(t, l, bx, by))
            continue;
        __syncwarp();
        for (int c = 0; c < 4; ++c)
            if (lane < p)
                sa[wi][c][lane] = ld<R>(mp_of<R>(w, l + 1, 4 * m + c) + lane);
        __syncwarp();
        if (lane < p) {
            cpx<R> acc = {(R)0, (R)0};
            for (int c = 0; c < 4; ++c)
                for (int k = 0; k <= lane; ++k)
                    acc = cadd(acc, cmul(ld<R>(T + (c * P + k) * P + lane), sa[wi][c][k]));
            st(mp_of<R>(w, l, m) + lane, acc);
        }
    }
}

// ------------------------------------------------------------------ X list: P2L into the locals of level l

// One warp per existing box of level l. Lanes 0..7 each take one of the parent's neighbour cells, find the leaf
// covering it and keep it if it is coarser, not adjacent to the box and not already found by a lower lane; then
// the particles of the kept leaves run one per lane, each lane accumulating all p coefficients
// b^_k = -sum_j q'_j s_j^-(k+1), s_j = (z_j - c) / w, in registers (powers by repeated multiplication, 1 / s_j
// formed in FP64), and a butterfly sum over the warp gives the box's X part. Writes every existing box's local
// (zero without an X list); the downward pass adds L2L and M2L to it.
template <typename R, int PM>
__global__ void __launch_bounds__(128) k_ad_p2l(Work w, int l)
{
    const int lane = threadIdx.x & 31;
    const SysDev &d = w.sys[0];
    const Tree t{w.start, d.depth, w.adapt_cap};
    const int nbx = w.ad_cnt[l], p = w.p, L = d.depth, nside = 1 << l;
    const double iw = ldexp(1.0, l) / d.S;
    for (int idx = blockIdx.x * 4 + (threadIdx.x >> 5); idx < nbx; idx += gridDim.x * 4) {
        const unsigned m = (unsigned)w.ad_list[d.box0[l] + idx];
        const int bx = (int)compact1(m), by = (int)compact1(m >> 1), px = bx >> 1, py = by >> 1;
        int xid = -1;
        if (lane < 8) {
            const int dxy = lane < 4 ? lane : lane + 1;  // 3 x 3 block without its centre
            int lq = l - 1, qx = px + dxy % 3 - 1, qy = py + dxy / 3 - 1;
            if (qx >= 0 && qy >= 0 && qx < (nside >> 1) && qy < (nside >> 1)) {
                covering_box(t, lq, qx, qy);
                if (!(lq == l - 1 && box_split(t, lq, qx, qy)) && !adjacent(L, l, bx, by, lq, qx, qy) &&
                    box_count(t, lq, morton2(qx, qy)) > 0)
                    xid = pack_box(lq, qx, qy);
            }
        }
        bool keep = xid >= 0;
        for (int o = 0; o < 8; ++o) {
            const int other = __shfl_sync(0xffffffffu, xid, o);
            keep = keep && !(o < lane && other == xid);
        }
        unsigned xm = __ballot_sync(0xffffffffu, keep);
        auto *dst = loc_of<R>(w, l, m);
        if (!xm) {
            if (lane < p)
                st(dst + lane, cpx<R>{(R)0, (R)0});
            continue;
        }
        cpx<R> acc[PM];
#pragma unroll
        for (int k = 0; k < PM; ++k)
            acc[k] = {(R)0, (R)0};
        const double2 c = centre(d, l, bx, by);
        int used = 0;  // lanes that took a particle
        while (xm) {
            const int src = __ffs(xm) - 1;
            xm &= xm - 1;
            const int id = __shfl_sync(0xffffffffu, xid, src);
            const int lq = id >> 26, qx = (id >> 13) & 0x1fff, qy = id & 0x1fff;
            const unsigned mq = morton2(qx, qy);
            const int j0 = box_first(t, lq, mq), cnt = box_count(t, lq, mq);
            used = max(used, min(cnt, 32));
            for (int e = lane; e < cnt; e += 32) {
                const int j = j0 + e;
                const double ax = (w.sx[j] - c.x) * iw, ay = (w.sy[j] - c.y) * iw;
                const double id2 = 1.0 / (ax * ax + ay * ay);
                const cpx<R> is = {(R)(ax * id2), (R)(-ay * id2)};
                const R g = (R)w.sg[j];
                cpx<R> pw = {-g * is.im, g * is.re};  // -q' / s with q' = -i gamma: i gamma / s
#pragma unroll
                for (int k = 0; k < PM; ++k) {
                    acc[k] = cadd(acc[k], pw);
                    pw = cmul(pw, is);
                }
            }
        }
        const cpx<R> sum = warp_coeff_sum<R, PM>(acc, lane, used);
        if (lane < p)
            st(dst + lane, sum);
    }
}

// ------------------------------------------------------------------ stages 6-7: locals of level l (L2L + V + X)

// One warp per existing box of level l, lane k = local coefficient: adds L2L from the parent and M2L over V to the
// X-list part left by k_ad_p2l. The binomial column C(m + k, m) stays in registers (PM >= p, entries m >= p zero)
// and the V sources are taken two at a time.
template <typename R, int PM>
__global__ void __launch_bounds__(128) k_ad_down(Work w, Tables tb, int l)
{
    __shared__ __align__(16) cpx<R> sa[4][2][32];
    __shared__ int vl[4][28];
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const SysDev &d = w.sys[0];
    const Tree t{w.start, d.depth, w.adapt_cap};
    const int nbx = w.ad_cnt[l], p = w.p, P = FMM_PMAX, nside = 1 << l;
    const int k = lane < p ? lane : p - 1;  // lanes >= p shadow the last coefficient and do not store
    const auto *rho = Store<R>::rho(tb);
    const auto *binom = Store<R>::binom(tb);
    R cb[PM];
#pragma unroll
    for (int mm = 0; mm < PM; ++mm)
        cb[mm] = mm < p ? (R)binom[mm * P + k] : (R)0;
    for (int idx = blockIdx.x * 4 + wi; idx < nbx; idx += gridDim.x * 4) {
        const unsigned m = (unsigned)w.ad_list[d.box0[l] + idx];
        const int bx = (int)compact1(m), by = (int)compact1(m >> 1);
        // the X-list part (k_ad_p2l) is already in the local
        cpx<R> acc = lane < p ? ld<R>(loc_of<R>(w, l, m) + lane) : cpx<R>{(R)0, (R)0};
        __syncwarp();
        // L2L from the parent
        if (l >= 3) {
            if (lane < p)
                sa[wi][0][lane] = ld<R>(loc_of<R>(w, l - 1, m >> 2) + lane);
            __syncwarp();
            const auto *T = Store<R>::l2l(tb) + (((by & 1) << 1) | (bx & 1)) * P * P;  // [input j][output k]
            for (int j = k; j < p; ++j)
                acc = cadd(acc, cmul(ld<R>(T + j * P + k), sa[wi][0][j]));
            __syncwarp();
        }
        // V: M2L from the children of the parent's neighbours that are not adjacent to b (factored form). The 36
        // candidates of the parent's 6 x 6 children block are tested one per lane and compacted by ballot.
        const int px = bx >> 1, py = by >> 1;
        int nv = 0;
        for (int base = 0; base < 36; base += 32) {
            const int q = base + lane;
            bool ok = false;
            int ent = 0;
            if (q < 36) {
                const int sx = 2 * px - 2 + q % 6, sy = 2 * py - 2 + q / 6;
                if (sx >= 0 && sy >= 0 && sx < nside && sy < nside && !(abs(sx - bx) <= 1 && abs(sy - by) <= 1) &&
                    box_exists(t, l, sx, sy)) {
                    const unsigned ms = morton2(sx, sy);
                    ok = box_count(t, l, ms) > 0;
                    ent = (((sy - by + 3) * 7 + (sx - bx + 3)) << 24) | (int)ms;
                }
            }
            const unsigned mk = __ballot_sync(0xffffffffu, ok);
            if (ok)
                vl[wi][nv + __popc(mk & ((1u << lane) - 1))] = ent;
            nv += __popc(mk);
        }
        __syncwarp();
        for (int sidx = 0; sidx < nv; sidx += 2) {
            const int e0 = vl[wi][sidx], e1 = sidx + 1 < nv ? vl[wi][sidx + 1] : -1;
            const auto *r0 = rho + (e0 >> 24) * kRS;
            const auto *r1 = rho + ((e1 >= 0 ? e1 : e0) >> 24) * kRS;
            if (lane < p) {  // alpha_m = (-1)^(m+1) rho^m a~_m
                const cpx<R> a0 = cmul(ld<R>(r0 + lane), ld<R>(mp_of<R>(w, l, e0 & 0xffffff) + lane));
                sa[wi][0][lane] = (lane & 1) ? a0 : cpx<R>{-a0.re, -a0.im};
                cpx<R> a1 = {(R)0, (R)0};
                if (e1 >= 0)
                    a1 = cmul(ld<R>(r1 + lane), ld<R>(mp_of<R>(w, l, e1 & 0xffffff) + lane));
                sa[wi][1][lane] = (lane & 1) ? a1 : cpx<R>{-a1.re, -a1.im};
            } else {
                sa[wi][0][lane] = {(R)0, (R)0};
                sa[wi][1][lane] = {(R)0, (R)0};
            }
            __syncwarp();
            cpx<R> s0 = {(R)0, (R)0}, s1 = {(R)0, (R)0};
            using V2 = typename Store<R>::V2;  // two coefficients in one shared-memory load (16 B for FP32)
            const V2 *q0 = reinterpret_cast<const V2 *>(sa[wi][0]), *q1 = reinterpret_cast<const V2 *>(sa[wi][1]);
#pragma unroll
            for (int mm = 0; mm < PM; mm += 2) {
                const V2 a = q0[mm >> 1], b = q1[mm >> 1];
                s0.re = fma(cb[mm], a.x, s0.re);
                s0.im = fma(cb[mm], a.y, s0.im);
                s1.re = fma(cb[mm], b.x, s1.re);
                s1.im = fma(cb[mm], b.y, s1.im);
                s0.re = fma(cb[mm + 1], a.z, s0.re);
                s0.im = fma(cb[mm + 1], a.w, s0.im);
                s1.re = fma(cb[mm + 1], b.z, s1.re);
                s1.im = fma(cb[mm + 1], b.w, s1.im);
            }
            acc = cadd(acc, cmul(ld<R>(r0 + k + 1), s0));
            if (e1 >= 0)
                acc = cadd(acc, cmul(ld<R>(r1 + k + 1), s1));
            __syncwarp();
        }
        if (lane < p)
            st(loc_of<R>(w, l, m) + lane, acc);
    }
}

// Precision form: the same locals with the V list one source per lane. Lane q takes V source q (at most 27: the
// 36 cells of the parent's 6 x 6 children block, compacted by ballot), forms x_m = (-1)^(m+1) rho^m a~_m, contracts
// it with the binomials C(m + k, m) by prefix sums (sum_k y_k s^k = u X(u) with u = 1/(1 - s), and multiplying a
// truncated series by u is a prefix sum of its coefficients: P (P - 1) packed additions, no table), scales by
// rho^(k+1) and leaves its partial local in shared memory; lane k then adds the V sources' partials of coefficient
// k, the parent's L2L and the X part. P >= p terms (zero padded).
typedef unsigned long long ad_f2;
__device__ __forceinline__ ad_f2 ad_pk2(float a, float b)
{
    ad_f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void ad_up2(ad_f2 v, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ ad_f2 ad_add2(ad_f2 a, ad_f2 b)
{
    ad_f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

template <int P>
__global__ void __launch_bounds__(128) k_ad_down32(Work w, Tables tb, int l)
{
    __shared__ float2 part[4][27][P + 1];
    __shared__ float2 sp[4][FMM_PMAX];
    __shared__ int vl[4][28];
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const SysDev &d = w.sys[0];
    const Tree t{w.start, d.depth, w.adapt_cap};
    const int nbx = w.ad_cnt[l], p = w.p, PP = FMM_PMAX, nside = 1 << l;
    for (int idx = blockIdx.x * 4 + wi; idx < nbx; idx += gridDim.x * 4) {
        const unsigned m = (unsigned)w.ad_list[d.box0[l] + idx];
        const int bx = (int)compact1(m), by = (int)compact1(m >> 1);
        // V candidates: the 36 cells of the parent's 6 x 6 children block, one per lane, compacted by ballot
        const int px = bx >> 1, py = by >> 1;
        int nv = 0;
        for (int base = 0; base < 36; base += 32) {
            const int q = base + lane;
            bool ok = false;
            int ent = 0;
            if (q < 36) {
                const int sx = 2 * px - 2 + q % 6, sy = 2 * py - 2 + q / 6;
                if (sx >= 0 && sy >= 0 && sx < nside && sy < nside && !(abs(sx - bx) <= 1 && abs(sy - by) <= 1) &&
                    box_exists(t, l, sx, sy)) {
                    const unsigned ms = morton2(sx, sy);
                    ok = box_count(t, l, ms) > 0;
                    ent = (((sy - by + 3) * 7 + (sx - bx + 3)) << 24) | (int)ms;
                }
            }
            const unsigned mk = __ballot_sync(0xffffffffu, ok);
            if (ok)
                vl[wi][nv + __popc(mk & ((1u << lane) - 1))] = ent;
            nv += __popc(mk);
        }
        // the parent's local for the L2L below
        if (l >= 3 && lane < p)
            sp[wi][lane] = loc_of<float>(w, l - 1, m >> 2)[lane];
        __syncwarp();
        if (lane < nv) {
            const int e = vl[wi][lane];
            const int off = e >> 24;
            const int ox = off % 7 - 3, oy = off / 7 - 3;
            const float den = (float)(ox * ox + oy * oy);
            const float rr = (float)ox / den, ri = -(float)oy / den;  // rho = 1 / (dx + i dy)
            const float2 *src = mp_of<float>(w, l, (unsigned)(e & 0xffffff));
            ad_f2 X[P];
            float pr = 1.f, pi = 0.f;
#pragma unroll
            for (int mm = 0; mm < P; ++mm) {
                const float2 a = mm < p ? src[mm] : make_float2(0.f, 0.f);
                const float sg = (mm & 1) ? 1.f : -1.f;  // (-1)^(m+1)
                X[mm] = ad_pk2(sg * (pr * a.x - pi * a.y), sg * (pr * a.y + pi * a.x));
                const float tt = pr * rr - pi * ri;
                pi = pr * ri + pi * rr;
                pr = tt;
            }
            ad_f2 T[P];
            T[0] = X[P - 1];
#pragma unroll
            for (int k = 1; k < P; ++k)
                T[k] = 0ull;
#pragma unroll
            for (int mm = P - 2; mm >= -1; --mm) {
#pragma unroll
                for (int k = 1; k < P; ++k)
                    T[k] = ad_add2(T[k], T[k - 1]);
                if (mm >= 0)
                    T[0] = ad_add2(T[0], X[mm]);
            }
            float qr = rr, qi = ri;  // rho^(k+1)
#pragma unroll
            for (int k = 0; k < P; ++k) {
                float br, bi;
                ad_up2(T[k], br, bi);
                part[wi][lane][k] = make_float2(qr * br - qi * bi, qr * bi + qi * br);
                const float tt = qr * rr - qi * ri;
                qi = qr * ri + qi * rr;
                qr = tt;
            }
        }
        __syncwarp();
        if (lane < p) {
            float2 acc = loc_of<float>(w, l, m)[lane];  // the X-list part (k_ad_p2l)
            if (l >= 3) {
                const float2 *T = Store<float>::l2l(tb) + (((by & 1) << 1) | (bx & 1)) * PP * PP;  // [input j][output k]
                for (int j = lane; j < p; ++j) {
                    const float2 c = T[j * PP + lane], a = sp[wi][j];
                    acc.x += c.x * a.x - c.y * a.y;
                    acc.y += c.x * a.y + c.y * a.x;
                }
            }
            float sr = 0.f, si = 0.f;
            for (int q = 0; q < nv; ++q) {
                const float2 v = part[wi][q][lane];
                sr += v.x;
                si += v.y;
            }
            acc.x += sr;
            acc.y += si;
            loc_of<float>(w, l, m)[lane] = acc;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ leaf of a sorted particle, U / W walk

// The leaf is the first level whose box around the particle holds at most B particles (or level L); the count of
// that box never grows with the level, so the level is found by bisection.
__device__ __forceinline__ void particle_leaf(const Tree &t, unsigned kf, int &l, int &x, int &y)
{
    int lo = 0, hi = t.L;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (box_count(t, mid, kf >> (2 * (t.L - mid))) <= t.B)
            hi = mid;
        else
            lo = mid + 1;
    }
    const int lv = lo;
    const unsigned m = kf >> (2 * (t.L - lv));
    l = lv;
    x = (int)compact1(m);
    y = (int)compact1(m >> 1);
}

// The U / W walk around leaf (l, bx, by): calls near(j0, j1) for the particles of every U leaf and
// far(ls, sx, sy) for every W box (non-empty ones only).
template <class Near, class Far>
__device__ __forceinline__ void walk_uw(const Work &w, const Tree &t, int l, int bx, int by, Near near, Far far)
{
    const int L = t.L, nside = 1 << l;
    {
        const unsigned mb = morton2(bx, by);
        const int j0 = box_first(t, l, mb);
        near(j0, j0 + box_count(t, l, mb));
    }
    int coarse[8];
    int ncoarse = 0;
    int stack[kStack];
    for (int dy = -1; dy <= 1; ++dy) {
        for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0)
                continue;
            int lq = l, qx = bx + dx, qy = by + dy;
            if (qx < 0 || qy < 0 || qx >= nside || qy >= nside)
                continue;
            if (!box_exists(t, l, qx, qy)) {  // a coarser leaf adjacent to b, possibly met from another cell
                covering_box(t, lq, qx, qy);
                const int id = pack_box(lq, qx, qy);
                bool dup = false;
                for (int e = 0; e < ncoarse; ++e)
                    dup |= coarse[e] == id;
                if (dup)
                    continue;
                coarse[ncoarse++] = id;
                const unsigned mq = morton2(qx, qy);
                const int j0 = box_first(t, lq, mq);
                near(j0, j0 + box_count(t, lq, mq));
                continue;
            }
            if (!box_split(t, l, qx, qy)) {
                const unsigned mq = morton2(qx, qy);
                const int j0 = box_first(t, l, mq);
                near(j0, j0 + box_count(t, l, mq));
                continue;
            }
            int sp = 0;
            stack[sp++] = pack_box(l, qx, qy);
            while (sp > 0) {
                const int id = stack[--sp];
                const int ls = id >> 26, sx = (id >> 13) & 0x1fff, sy = id & 0x1fff;
                for (int c = 0; c < 4; ++c) {
                    const int cl = ls + 1, cx = 2 * sx + (c & 1), cy = 2 * sy + (c >> 1);
                    const unsigned mc = morton2(cx, cy);
                    const int cnt = box_count(t, cl, mc);
                    if (!adjacent(L, l, bx, by, cl, cx, cy)) {
                        if (cnt > 0)
                            far(cl, cx, cy);
                    } else if (cl < L && cnt > t.B) {
                        if (sp < kStack)
                            stack[sp++] = pack_box(cl, cx, cy);
                        else
                            atomicOr(w.status, FMM_DEV_BOUNDS);
                    } else if (cnt > 0) {
                        const int j0 = box_first(t, cl, mc);
                        near(j0, j0 + cnt);
                    }
                }
            }
        }
    }
}

// W list: a multipole a~ (p terms) evaluated at t = (ax, ay) = (z - c_s) / w_s: sum_m a~_m / t^(m+1). Out of line
// (scalar arguments only, so that no large structure is copied to the stack), which keeps the walk's registers
// low.
template <typename R>
__device__ __noinline__ double2 m2p_eval(const typename Store<R>::S *a, int p, double ax, double ay)
{
    const double id2 = 1.0 / (ax * ax + ay * ay);
    const cpx<R> uinv = {(R)(ax * id2), (R)(-ay * id2)};
    cpx<R> s = {(R)0, (R)0};
    for (int mm = p - 1; mm >= 0; --mm)
        s = cmul(cadd(s, ld<R>(a + mm)), uinv);
    return make_double2((double)s.re, (double)s.im);
}

// The multipole of W box (ls, sx, sy) at (xi, yi), (1/w_s) sum_m a~_m / t^(m+1), t formed in FP64, added to
// (wr, wi) (complex velocity w = u - i v without 1 / 2pi).
template <typename R>
__device__ __forceinline__ void m2p_add(const Work &w, const SysDev &d, double xi, double yi, int ls, int sx, int sy,
                                        double &wr, double &wi)
{
    const double2 c = centre(d, ls, sx, sy);
    const double iws = ldexp(1.0, ls) / d.S;
    const double2 r = m2p_eval<R>(mp_of<R>(w, ls, morton2(sx, sy)), w.p, (xi - c.x) * iws, (yi - c.y) * iws);
    wr += r.x * iws;
    wi += r.y * iws;
}

// Stage 8, L2P: the local expansion of leaf (l, bx, by), l >= 2, at (xi, yi): (1/w) sum_k b^_k zeta^k with
// zeta = (z - c) / w formed in FP64; returned as the complex velocity w = u - i v without 1 / 2pi.
template <typename R>
__device__ __forceinline__ double2 l2p_eval(const Work &w, const SysDev &d, int l, int bx, int by, double xi, double yi)
{
    const double2 c = centre(d, l, bx, by);
    const double iw = ldexp(1.0, l) / d.S;
    const cpx<R> z = {(R)((xi - c.x) * iw), (R)((yi - c.y) * iw)};
    const auto *b = loc_of<R>(w, l, morton2(bx, by));
    cpx<R> s = {(R)0, (R)0};
    for (int k = w.p - 1; k >= 0; --k)
        s = cadd(cmul(s, z), ld<R>(b + k));
    return make_double2((double)s.re * iw, (double)s.im * iw);
}

// ------------------------------------------------------------------ stages 8-10: U, W, L2P, sum, unsort

// One thread per target, after the whole sweep: one walk of U and W, the exact K_sigma over U (use_near), the
// multipoles of W and the leaf's local expansion (use_far), the sum written in the caller's order.

__global__ void __launch_bounds__(128) k_ad_near(Work w, unsigned long long *pairs, int use_near, int use_far, double *u,
                                                double *v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w.n)
        return;
    const SysDev &d = w.sys[0];
    const Tree t{w.start, d.depth, w.adapt_cap};
    int l, bx, by;
    particle_leaf(t, (unsigned)w.sleaf[i], l, bx, by);
    const double xi = w.sx[i], yi = w.sy[i];
    const double k2 = 1.0 / (2.0 * d.sigma * d.sigma);
    double su = 0.0, sv = 0.0, wr = 0.0, wi = 0.0;
    long long np = -1;  // ordered pairs (i, j), j != i
    auto near = [&](int j0, int j1) {
        np += j1 - j0;
        if (!use_near)
            return;
        for (int j = j0; j < j1; ++j) {
            const double ax = xi - w.sx[j], ay = yi - w.sy[j];
            const double r2 = ax * ax + ay * ay;
            if (r2 > 0.0) {
                const double f = w.sg[j] * (-expm1(-r2 * k2)) / (kTwoPi * r2);
                su -= ay * f;
                sv += ax * f;
            }
        }
    };
    auto far = [&](int ls, int sx, int sy) {
        if (use_far)
            m2p_add<double>(w, d, xi, yi, ls, sx, sy, wr, wi);
    };
    walk_uw(w, t, l, bx, by, near, far);
    if (use_far && l >= 2) {
        const double2 b = l2p_eval<double>(w, d, l, bx, by, xi, yi);
        wr += b.x;
        wi += b.y;
    }
    const int pos = w.perm[i];
    u[pos] = su + wr / kTwoPi;
    v[pos] = sv - wi / kTwoPi;
    if (pairs && use_near)
        atomicAdd(pairs, (unsigned long long)np);
}

// Precision form: positions in units u = sigma sqrt(2 / log2 e), X = (x - x0) / u, split into hi + lo floats
// (eh = (xh, yh, xl, yl), written with the circulation eg.x by the leaf-order kernel) so that a displacement
// (hi_i - hi_j) + (lo_i - lo_j) keeps about 2^-24 of its own size. In these units exp(-r^2 / 2 sigma^2) = 2^-(R^2),
// R = r / u.

__device__ __forceinline__ float ex2_approx(float v)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float rcp_approx(float v)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// q(R^2) = (1 - 2^-R^2) / R^2 = ln2 f(x), f(x) = (1 - e^-x) / x, x = R^2 ln 2: the Taylor series
// f = sum_k (-x)^k / (k+1)! below x = 1/2 (truncation < 1e-8 relative), the exponential above (cancellation
// < 2e-7 relative).
__device__ __forceinline__ float blob_q(float R2)
{
    constexpr float kLn2 = 0.693147180559945309f;
    if (R2 < 0.5f / kLn2) {
        const float x = R2 * kLn2;
        float s = 1.0f / 362880.0f;
        s = fmaf(s, -x, 1.0f / 40320.0f);
        s = fmaf(s, -x, 1.0f / 5040.0f);
        s = fmaf(s, -x, 1.0f / 720.0f);
        s = fmaf(s, -x, 1.0f / 120.0f);
        s = fmaf(s, -x, 1.0f / 24.0f);
        s = fmaf(s, -x, 1.0f / 6.0f);
        s = fmaf(s, -x, 0.5f);
        return kLn2 * fmaf(s, -x, 1.0f);
    }
    return (1.0f - ex2_approx(-R2)) * rcp_approx(R2);
}

// Pairs of one target with the sources [j0, j1): FP32 terms in two chains (even and odd sources), returned as an
// FP32 partial (sum of -dY q g, sum of dX q g).
__device__ __forceinline__ float2 near_range(const Work &w, float4 pi, int j0, int j1)
{
    float pu0 = 0.0f, pv0 = 0.0f, pu1 = 0.0f, pv1 = 0.0f;
    int j = j0;
#pragma unroll 4
    for (; j + 1 < j1; j += 2) {
        const float4 pa = w.eh[j], pb = w.eh[j + 1];
        const float ga = w.eg[j].x, gb = w.eg[j + 1].x;
        const float ax = (pi.x - pa.x) + (pi.z - pa.z), ay = (pi.y - pa.y) + (pi.w - pa.w);
        const float bx = (pi.x - pb.x) + (pi.z - pb.z), by = (pi.y - pb.y) + (pi.w - pb.w);
        const float fa = ga * blob_q(fmaf(ax, ax, ay * ay)), fb = gb * blob_q(fmaf(bx, bx, by * by));
        pu0 = fmaf(-ay, fa, pu0);
        pv0 = fmaf(ax, fa, pv0);
        pu1 = fmaf(-by, fb, pu1);
        pv1 = fmaf(bx, fb, pv1);
    }
    if (j < j1) {
        const float4 pa = w.eh[j];
        const float ga = w.eg[j].x;
        const float ax = (pi.x - pa.x) + (pi.z - pa.z), ay = (pi.y - pa.y) + (pi.w - pa.w);
        const float fa = ga * blob_q(fmaf(ax, ax, ay * ay));
        pu0 = fmaf(-ay, fa, pu0);
        pv0 = fmaf(ax, fa, pv0);
    }
    return make_float2(pu0 + pu1, pv0 + pv1);
}

// K_sigma in units u: K = (-dY, dX) q(R^2) / (2 pi u). The walk only records the U source ranges (in shared
// memory, range-major so that a warp's accesses fall in distinct banks) and evaluates the W multipoles; one loop
// over the recorded ranges then runs the pairs, so that lanes whose leaves reach their sources through different
// branches of the walk meet in the same loop. FP32 sums per range, FP64 across ranges.
constexpr int kRanges = 16;
__global__ void __launch_bounds__(128, 8) k_ad_near32(Work w, unsigned long long *pairs, int use_near, int use_far,
                                                       double *u, double *v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w.n)
        return;
    const SysDev &d = w.sys[0];
    const Tree t{w.start, d.depth, w.adapt_cap};
    int l, bx, by;
    particle_leaf(t, (unsigned)w.sleaf[i], l, bx, by);
    const float4 pi = w.eh[i];
    double su = 0.0, sv = 0.0, wr = 0.0, wi = 0.0;
    long long np = -1;
    __shared__ int2 rg_s[kRanges][128];
    int2 *rg = &rg_s[0][threadIdx.x];  // range r of this thread at rg[128 r]
    int nr = 0;
    auto run = [&]() {
        for (int r = 0; r < nr; ++r) {
            const int2 q = rg[128 * r];
            const float2 part = near_range(w, pi, q.x, q.y);
            su += (double)part.x;
            sv += (double)part.y;
        }
        nr = 0;
    };
    auto near = [&](int j0, int j1) {
        np += j1 - j0;
        if (!use_near || j1 <= j0)
            return;
        if (nr == kRanges)
            run();
        rg[128 * nr++] = make_int2(j0, j1);
    };
    auto far = [&](int ls, int sx, int sy) {
        if (use_far)
            m2p_add<float>(w, d, w.sx[i], w.sy[i], ls, sx, sy, wr, wi);
    };
    walk_uw(w, t, l, bx, by, near, far);
    run();
    const double sc = d.iu / kTwoPi;  // 1 / (2 pi u)
    if (use_far && l >= 2) {
        const double2 b = l2p_eval<float>(w, d, l, bx, by, w.sx[i], w.sy[i]);
        wr += b.x;
        wi += b.y;
    }
    const int pos = w.perm[i];
    u[pos] = su * sc + wr / kTwoPi;
    v[pos] = sv * sc - wi / kTwoPi;
    if (pairs && use_near)
        atomicAdd(pairs, (unsigned long long)np);
}

template <typename R, int PM>
int sweep_levels(const Work &w, const Tables &t, int part, cudaStream_t s)
{
    const int L = w.maxdepth;
    int nl = 0;
    if (part == 0) {  // box lists, P2L over X (particles only), then upward: P2M, M2M
        const int64_t ne = enum_threads(L);
        k_ad_enum<<<(unsigned)((ne + 127) / 128), 128, 0, s>>>(w);
        ++nl;
        for (int l = 2; l <= L; ++l, ++nl)
            k_ad_p2l<R, PM><<<kSweepBlocks, 128, 0, s>>>(w, l);
        for (int l = 2; l <= L; ++l, ++nl)
            k_ad_p2m<R, PM><<<kSweepBlocks, 128, 0, s>>>(w, l);
        for (int l = L - 1; l >= 2; --l, ++nl)
            k_ad_m2m<R><<<kSweepBlocks, 128, 0, s>>>(w, t, l);
    } else {  // downward: L2L + M2L (V list) over the X part, per level
        for (int l = 2; l <= L; ++l, ++nl) {
            if constexpr (std::is_same<R, float>::value)
                k_ad_down32<PM><<<kSweepBlocks, 128, 0, s>>>(w, t, l);
            else
                k_ad_down<R, PM><<<kSweepBlocks, 128, 0, s>>>(w, t, l);
        }
    }
    return nl;
}

template <typename R>
int sweep_bucket(const Work &w, const Tables &t, int part, cudaStream_t s)
{
    if (w.p <= 8)
        return sweep_levels<R, 8>(w, t, part, s);
    if (w.p <= 16)
        return sweep_levels<R, 16>(w, t, part, s);
    if (w.p <= 20)
        return sweep_levels<R, 20>(w, t, part, s);
    if (w.p <= 24)
        return sweep_levels<R, 24>(w, t, part, s);
    return sweep_levels<R, 32>(w, t, part, s);
}

}  // namespace

int launch_adaptive_up(const Work &w, const Tables &t, cudaStream_t s)
{
    return w.ad_mixed ? sweep_bucket<float>(w, t, 0, s) : sweep_bucket<double>(w, t, 0, s);
}

int launch_adaptive_down(const Work &w, const Tables &t, cudaStream_t s)
{
    return w.ad_mixed ? sweep_bucket<float>(w, t, 1, s) : sweep_bucket<double>(w, t, 1, s);
}


int launch_adaptive_near(const Work &w, unsigned long long *pairs, int use_near, int use_far, double *u, double *v,
                         cudaStream_t s)
{
    if (w.ad_mixed)
        k_ad_near32<<<(w.n + 127) / 128, 128, 0, s>>>(w, pairs, use_near, use_far, u, v);
    else
        k_ad_near<<<(w.n + 127) / 128, 128, 0, s>>>(w, pairs, use_near, use_far, u, v);
    return 1;
}

}  // namespace fmm
