// binning.cu -- Fig. 1 stages 1-2: root square, leaf keys, counting sort into leaf order, gather of the
// particle data into the layout the near-field and expansion kernels read.
//
// The root square and leaf rule are this library's reading of the paper (which leaves them open): an
// explicit square, or the particles' bounding box centred with side extent * (1 + 2^-20); the leaf column
// is floor((x - x0) * (2^L / S)) in IEEE double without FMA contraction, clamped to [0, 2^L - 1].
// Within a leaf, particles keep the caller's order, so every run gives bit-identical results; the uniform tree's
// precision form orders each leaf by boundary class first (the band of width sigma along each side that the
// near field of the adjacent leaves must test for small r, see k_keys) and by caller index within a class.
#include "fmm_internal.cuh"

namespace fmm {

// Order-preserving map of doubles onto unsigned integers (for atomicMin / atomicMax).
__device__ inline unsigned long long ord_of(double d)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(d);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ inline double double_of(unsigned long long u)
{
    unsigned long long b = (u & 0x8000000000000000ull) ? (u & ~0x8000000000000000ull) : ~u;
    return __longlong_as_double((long long)b);
}

// ------------------------------------------------------------------ stage 1: bounding box

__global__ void k_bbox(const SysDev *__restrict__ sys, int nsys, int n, const double *__restrict__ x,
                       const double *__restrict__ y, unsigned long long *minmax)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = i < n;
    int k = valid ? (nsys == 1 ? 0 : find_sys_by_particle(sys, nsys, i)) : -1;
    bool use = valid && !sys[k].explicit_domain && isfinite(x[i]) && isfinite(y[i]);
    unsigned long long xmn = use ? ord_of(x[i]) : ~0ull, xmx = use ? ord_of(x[i]) : 0ull;
    unsigned long long ymn = use ? ord_of(y[i]) : ~0ull, ymx = use ? ord_of(y[i]) : 0ull;
    int k0 = __shfl_sync(0xffffffffu, k, 0);
    if (__all_sync(0xffffffffu, k == k0 || k < 0)) {
        for (int o = 16; o > 0; o >>= 1) {
            xmn = min(xmn, __shfl_xor_sync(0xffffffffu, xmn, o));
            xmx = max(xmx, __shfl_xor_sync(0xffffffffu, xmx, o));
            ymn = min(ymn, __shfl_xor_sync(0xffffffffu, ymn, o));
            ymx = max(ymx, __shfl_xor_sync(0xffffffffu, ymx, o));
        }
        if ((threadIdx.x & 31) == 0 && k0 >= 0 && xmx != 0ull) {
            atomicMin(&minmax[4 * k0 + 0], xmn);
            atomicMax(&minmax[4 * k0 + 1], xmx);
            atomicMin(&minmax[4 * k0 + 2], ymn);
            atomicMax(&minmax[4 * k0 + 3], ymx);
        }
    } else if (use) {
        atomicMin(&minmax[4 * k + 0], xmn);
        atomicMax(&minmax[4 * k + 1], xmx);
        atomicMin(&minmax[4 * k + 2], ymn);
        atomicMax(&minmax[4 * k + 3], ymx);
    }
}

// Constants every kernel reads, from the root square, depth and sigma; the host computes them for an explicit
// square, the domain kernel for a bounding-box square. Only IEEE operations without a multiply-add (so no
// contraction into an FMA on either side), so host and device give the same bits.
__host__ __device__ void derive_constants(SysDev &d)
{
    int L = d.depth;
    d.scale = ldexp(1.0, L) / d.S;
#ifdef __CUDA_ARCH__
    d.xe = __dadd_rn(d.x0, d.S);
    d.ye = __dadd_rn(d.y0, d.S);
#else
    d.xe = d.x0 + d.S;
    d.ye = d.y0 + d.S;
#endif
    d.wl = ldexp(d.S, -L);
    d.far_scale = 1.0 / (6.283185307179586476925 * d.wl);
    double kap = d.wl * d.wl / (2.0 * d.sigma * d.sigma);
    float s = (float)sqrt(1.4426950408889634074 * kap);
    d.s_unit = s;
    d.inv_s = 1.0f / s;
    d.snear = (float)((double)s * d.far_scale);
    d.iu = sqrt(1.4426950408889634074 / (2.0 * d.sigma * d.sigma));
    // band width delta = 6 sigma (1 + 2^-8) in leaf widths: a pair farther apart has exp(-r^2 / 2 sigma^2) <
    // 2^-25, so 1 - exp rounds to 1 in FP32 and the near field skips the exponential outside the bands; the
    // bands also hold every pair below the series threshold (r < sigma), with room for FP32 rounding
    const double om = 6.0 * d.sigma * (1.0 + 0x1p-8) / d.wl;
    d.bnd_ok = om < 0.5 ? 1 : 0;
    d.fbnd = d.bnd_ok ? (long long)floor((0.5 - om) * 0x1p52) : 0;
}

__global__ void k_domain_finalize(SysDev *sys, int nsys, const unsigned long long *minmax)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsys)
        return;
    SysDev &d = sys[k];
    if (!d.explicit_domain) {
        if (d.np == 0 || minmax[4 * k + 1] == 0ull) {
            d.x0 = 0.0;
            d.y0 = 0.0;
            d.S = 1.0;
        } else {
            double xmin = double_of(minmax[4 * k + 0]), xmax = double_of(minmax[4 * k + 1]);
            double ymin = double_of(minmax[4 * k + 2]), ymax = double_of(minmax[4 * k + 3]);
            double ex = __dsub_rn(xmax, xmin), ey = __dsub_rn(ymax, ymin);
            double ext = ex > ey ? ex : ey;
            double side = __dmul_rn(ext, 1.0 + 0x1p-20);
            if (side < 1e-300)
                side = 1e-300;
            double cx = __dmul_rn(0.5, __dadd_rn(xmin, xmax)), cy = __dmul_rn(0.5, __dadd_rn(ymin, ymax));
            double half = __dmul_rn(0.5, side);
            d.x0 = __dsub_rn(cx, half);
            d.y0 = __dsub_rn(cy, half);
            d.S = side;
        }
    }
    derive_constants(d);
}

__global__ void k_minmax_init(unsigned long long *minmax, int nsys)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nsys) {
        minmax[4 * k + 0] = ~0ull;
        minmax[4 * k + 1] = 0ull;
        minmax[4 * k + 2] = ~0ull;
        minmax[4 * k + 3] = 0ull;
    }
}

int launch_bbox(const Work &w, const double *x, const double *y, cudaStream_t s)
{
    k_minmax_init<<<(w.nsys + 127) / 128, 128, 0, s>>>(w.minmax, w.nsys);
    k_bbox<<<(w.n + 255) / 256, 256, 0, s>>>(w.sys, w.nsys, w.n, x, y, w.minmax);
    return 2;
}

int launch_domain_finalize(const Work &w, cudaStream_t s)
{
    k_domain_finalize<<<(w.nsys + 127) / 128, 128, 0, s>>>(w.sys, w.nsys, w.minmax);
    return 1;
}

// ------------------------------------------------------------------ stage 2: leaf keys and histogram

__device__ __forceinline__ bool not_finite(double v)
{
    return ((__double_as_longlong(v) >> 52) & 0x7ff) == 0x7ff;
}

// Leaf-relative position from the bit pattern of t = (c - c0) * scale (exact IEEE double, t >= 0 for points in
// the square): returns floor(t) and F = (t - floor(t) - 1/2) * 2^52 as a signed integer, using integer
// operations only. Callers clamp the index (t >= 2^31, not a valid point, returns 2^30).
__device__ __forceinline__ int leaf_frac(double t, long long *F)
{
    const unsigned long long T = (unsigned long long)__double_as_longlong(t);
    const int be = (int)((T >> 52) & 0x7ff);
    if (be == 0 || (T >> 63)) {  // zero, subnormal or negative: fraction 0
        *F = -(1ll << 51);
        return 0;
    }
    const int e = be - 1023;
    const unsigned long long m = (T & 0xfffffffffffffull) | (1ull << 52);
    if (e < 0) {  // t in (0, 1): t 2^52 = m 2^e
        *F = (long long)(e > -53 ? (m >> (-e)) : 0ull) - (1ll << 51);
        return 0;
    }
    if (e > 30) {  // far outside any valid square: the caller clamps it to the last leaf
        *F = 0;
        return 1 << 30;
    }
    const int sh = 52 - e;
    *F = (long long)((m & ((1ull << sh) - 1)) << e) - (1ll << 51);
    return (int)(m >> sh);
}

// s * F * 2^-52 as hi + lo floats (about 46 bits): F = A' 2^29 + B' with A' exact in float.
__device__ __forceinline__ void frac_to_split(long long F, float s, float *hi, float *lo)
{
    const float A = __int2float_rn((int)(F >> 29)) * 0x1p-23f;
    const float B = __uint2float_rn((unsigned)(F & 0x1fffffffll)) * 0x1p-52f;
    const float ph = A * s;
    float pl = fmaf(A, s, -ph);
    pl = fmaf(B, s, pl);
    const float h = ph + pl;
    *hi = h;
    *lo = pl - (h - ph);
}

// IEEE order of doubles as signed integers (for the upper-edge test without the FP64 pipe).
__device__ __forceinline__ long long ordered(double v)
{
    long long b = __double_as_longlong(v);
    return b < 0 ? (long long)(0x8000000000000000ull - (unsigned long long)b) : b;
}

// Key, boundary class and the caller-order records of particle i (everything but its arrival slot); returns the
// global leaf.
__device__ __forceinline__ int key_of(const Work &w, const double *__restrict__ x, const double *__restrict__ y,
                                      const double *__restrict__ g, int i, int &cls)
{
    int k = w.nsys == 1 ? 0 : find_sys_by_particle(w.sys, w.nsys, i);
    const SysDev &d = w.sys[k];
    const double xi = x[i], yi = y[i];
    const int L = d.depth, nside = 1 << L;
    // the only FP64 operations: the two roundings of the leaf rule, t = (c - c0) * (2^L / S)
    const double dx = __dsub_rn(xi, d.x0), dy = __dsub_rn(yi, d.y0);
    const double tx = __dmul_rn(dx, d.scale), ty = __dmul_rn(dy, d.scale);
    long long Fx, Fy;
    int ix = leaf_frac(tx, &Fx), iy = leaf_frac(ty, &Fy);
    if (ix > nside - 1) {  // t >= 2^L: a point on the square's upper edge goes to the last leaf (zeta = 1/2)
        Fx += 1ll << 52;
        ix = nside - 1;
    }
    if (iy > nside - 1) {
        Fy += 1ll << 52;
        iy = nside - 1;
    }
    bool bad = not_finite(xi) || not_finite(yi);
    if (d.explicit_domain)  // outside: c < c0 (sign of c - c0) or c > c0 + S
        bad = bad || __double_as_longlong(dx) < 0 || __double_as_longlong(dy) < 0 || ordered(xi) > ordered(d.xe) ||
              ordered(yi) > ordered(d.ye);
    if (bad) {
        atomicOr(w.status, FMM_DEV_OUTSIDE);
        if (not_finite(xi))
            ix = 0;
        if (not_finite(yi))
            iy = 0;
    }
    const int kk = (int)(d.leaf0 + (w.morton ? (int64_t)morton2(ix, iy) : (int64_t)iy * nside + ix));
    // boundary class (precision form, uniform tree): band (left, middle, right) x (bottom, middle, top) of the
    // leaf, from the exact fraction F = zeta 2^52 (a point on the square's upper edge has F = 2^51: right or top
    // band). Numbered around the leaf so that the band facing each of the 8 neighbours is a run of classes: 0 LB,
    // 1 LM, 2 LT, 3 MT, 4 RT, 5 RM, 6 RB, 7 MB, 8 MM (the interior, last); everything is class 8 where the bands
    // would overlap.
    cls = 8;
    if (w.cls_off && d.bnd_ok) {
        const int cx = Fx < -d.fbnd ? 0 : (Fx > d.fbnd ? 2 : 1);
        const int cy = Fy < -d.fbnd ? 0 : (Fy > d.fbnd ? 2 : 1);
        cls = (int)((0x432581670ull >> (4 * (3 * cy + cx))) & 15ull);
    }
    w.key[i] = kk;
    if (w.mixed) {
        float hx, lx, hy, ly;
        frac_to_split(Fx, d.s_unit, &hx, &lx);
        frac_to_split(Fy, d.s_unit, &hy, &ly);
        w.pos4u[2 * (int64_t)i] = make_float4(hx, hy, lx, ly);
        if (w.cls_off)
            w.cls8[i] = (unsigned char)cls;
        w.pos4u[2 * (int64_t)i + 1] = make_float4(__double2float_rn(g[i]), 0.f, 0.f, 0.f);
    } else if (w.rec64) {
        Rec64 r;
        r.x = xi;
        r.y = yi;
        r.g = g[i];
        r.pad = 0.0;
        w.rec64[i] = r;
    }
    return kk;
}

// KPT particles per thread (block: 256 threads, 256 KPT consecutive particles, coalesced per step): their keys and
// records first, then their arrival slots by returning atomics. Measured at 2^20: 32 us with one particle per
// thread, 37 us with four (the leaf counters' atomics, not their latency, bound the kernel).
constexpr int KPT = 1;
__global__ void __launch_bounds__(256) k_keys(Work w, const double *__restrict__ x, const double *__restrict__ y,
                                              const double *__restrict__ g)
{
    const int base = blockIdx.x * (256 * KPT) + threadIdx.x;
    int kk[KPT], cls[KPT], sl[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        const int i = base + 256 * j;
        kk[j] = i < w.n ? key_of(w, x, y, g, i, cls[j]) : -1;
    }
#pragma unroll
    for (int j = 0; j < KPT; ++j)
        sl[j] = kk[j] >= 0 ? atomicAdd(&w.cnt[kk[j]], 1) : 0;  // arrival slot inside the leaf (order fixed later)
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        const int i = base + 256 * j;
        if (kk[j] < 0)
            continue;
        w.slot[i] = sl[j];
        if (w.bkt) {  // the entry straight into its leaf's bucket; a full bucket sends the evaluation to the scatter
            if (sl[j] < w.bkt_cap)
                w.bkt[(int64_t)kk[j] * w.bkt_cap + sl[j]] = make_int2(i, cls[j]);
            else
                w.cnt[w.nleaf] = 1;
        }
    }
}

int launch_keys(const Work &w, const double *x, const double *y, const double *g, cudaStream_t s)
{
    k_keys<<<(w.n + 256 * KPT - 1) / (256 * KPT), 256, 0, s>>>(w, x, y, g);
    return 1;
}

// ------------------------------------------------------------------ exclusive scan cnt -> start

#define SCAN_BLOCK 1024

__global__ void k_scan_block(const int *__restrict__ in, int nin, int *__restrict__ out, int *__restrict__ bsum)
{
    __shared__ int sh[SCAN_BLOCK / 32];
    int base = blockIdx.x * SCAN_BLOCK;
    int t = threadIdx.x;  // 256 threads, 4 values each
    int v[4], s = 0;
    for (int j = 0; j < 4; ++j) {
        int idx = base + t * 4 + j;
        v[j] = idx < nin ? in[idx] : 0;
        s += v[j];
    }
    int lane = t & 31, wid = t >> 5;
    int inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += u;
    }
    if (lane == 31)
        sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int ws = lane < 8 ? sh[lane] : 0;
        int wi = ws;
        for (int o = 1; o < 8; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o)
                wi += u;
        }
        if (lane < 8)
            sh[lane] = wi - ws;
        if (lane == 7)
            bsum[blockIdx.x] = wi;
    }
    __syncthreads();
    int ex = sh[wid] + inc - s;
    for (int j = 0; j < 4; ++j) {
        int idx = base + t * 4 + j;
        if (idx < nin)
            out[idx] = ex;
        ex += v[j];
    }
}

__global__ void k_scan_top(int *bsum, int nb, int *total_out)
{
    __shared__ int sh[32];
    __shared__ int carry_sh;
    int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0)
        carry_sh = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        int idx = base + t;
        int v = idx < nb ? bsum[idx] : 0;
        int inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o)
                inc += u;
        }
        if (lane == 31)
            sh[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            int ws = sh[lane], wi = ws;
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o)
                    wi += u;
            }
            sh[lane] = wi - ws;
        }
        __syncthreads();
        int carry = carry_sh;
        int ex = carry + sh[wid] + inc - v;
        if (idx < nb)
            bsum[idx] = ex;
        __syncthreads();
        if (t == 1023)
            carry_sh = ex + v;
        __syncthreads();
    }
    if (t == 0)
        *total_out = carry_sh;
}

__global__ void k_scan_add(int *out, int nin, const int *__restrict__ bsum)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < nin)
        out[idx] += bsum[idx / SCAN_BLOCK];
}

// Whole scan in one block when the leaf count is small (one launch instead of three).
__global__ void __launch_bounds__(1024) k_scan_single(const int *__restrict__ in, int nin, int *__restrict__ out)
{
    __shared__ int sh[32];
    __shared__ int carry_sh;
    int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0)
        carry_sh = 0;
    __syncthreads();
    for (int base = 0; base < nin; base += 4096) {
        int v[4], s = 0;
        for (int j = 0; j < 4; ++j) {
            int idx = base + t * 4 + j;
            v[j] = idx < nin ? in[idx] : 0;
            s += v[j];
        }
        int inc = s;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o)
                inc += u;
        }
        if (lane == 31)
            sh[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            int ws = sh[lane], wi = ws;
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o)
                    wi += u;
            }
            sh[lane] = wi - ws;
        }
        __syncthreads();
        int ex = carry_sh + sh[wid] + inc - s;
        for (int j = 0; j < 4; ++j) {
            int idx = base + t * 4 + j;
            if (idx < nin)
                out[idx] = ex;
            ex += v[j];
        }
        __syncthreads();
        if (t == 1023)
            carry_sh = ex;
        __syncthreads();
    }
    if (t == 0)
        out[nin] = carry_sh;
}

// Up to 16384 counts: thread t owns the 16 consecutive counts from 16 t, all loaded at once (one memory round
// trip), then a block-wide exclusive scan of the per-thread sums. out[nin] = total.
__global__ void __launch_bounds__(1024) k_scan_16k(const int *__restrict__ in, int nin, int *__restrict__ out)
{
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, b0 = 16 * t;
    int v[16];
    if (b0 + 16 <= nin) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int4 a = reinterpret_cast<const int4 *>(in + b0)[q];
            v[4 * q] = a.x;
            v[4 * q + 1] = a.y;
            v[4 * q + 2] = a.z;
            v[4 * q + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            v[j] = b0 + j < nin ? in[b0 + j] : 0;
    }
    int s = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j)
        s += v[j];
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += u;
    }
    if (lane == 31)
        wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int ws = wsum[lane];
        int wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o)
                wi += u;
        }
        wsum[lane] = wi - ws;
    }
    __syncthreads();
    int ex = wsum[wid] + inc - s;
    if (b0 + 16 <= nin) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int4 a;
            a.x = ex;
            ex += v[4 * q];
            a.y = ex;
            ex += v[4 * q + 1];
            a.z = ex;
            ex += v[4 * q + 2];
            a.w = ex;
            ex += v[4 * q + 3];
            reinterpret_cast<int4 *>(out + b0)[q] = a;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (b0 + j < nin)
                out[b0 + j] = ex;
            ex += v[j];
        }
    }
    if (t == 1023)
        out[nin] = ex;  // the total (the padding counts are zero)
}

int launch_scan(const Work &w, cudaStream_t s)
{
    if (w.nleaf <= 16384) {
        k_scan_16k<<<1, 1024, 0, s>>>(w.cnt, w.nleaf, w.start);
        return 1;
    }
    if (w.nleaf <= 65536) {
        k_scan_single<<<1, 1024, 0, s>>>(w.cnt, w.nleaf, w.start);
        return 1;
    }
    int nb = (w.nleaf + SCAN_BLOCK - 1) / SCAN_BLOCK;
    k_scan_block<<<nb, 256, 0, s>>>(w.cnt, w.nleaf, w.start, w.scan_tmp);
    k_scan_top<<<1, 1024, 0, s>>>(w.scan_tmp, nb, w.start + w.nleaf);
    k_scan_add<<<(w.nleaf + 255) / 256, 256, 0, s>>>(w.start, w.nleaf, w.scan_tmp);
    return 3;
}

// ------------------------------------------------------------------ counting-sort scatter and in-leaf order

__global__ void k_scatter(Work w, const unsigned char *__restrict__ cls8, const int *__restrict__ overflow)
{
    if (overflow && *overflow == 0)
        return;  // with leaf buckets the scatter runs only after one overflowed
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += gridDim.x * blockDim.x) {
        const int k = w.key[i];
        // caller index and leaf (or boundary class), at the leaf's arrival slot
        w.tmp[w.start[k] + w.slot[i]] = make_int2(i, cls8 ? (int)cls8[i] : k);
    }
}

int launch_scatter_sort(const Work &w, cudaStream_t s)
{
    // with leaf buckets usually nothing to do: a grid of a few blocks per SM, which checks the flag and returns
    const unsigned nb = (unsigned)((w.n + 255) / 256);
    k_scatter<<<w.bkt ? (nb < 152u * 4u ? nb : 152u * 4u) : nb, 256, 0, s>>>(
        w, w.cls_off ? w.cls8 : nullptr, w.bkt ? w.cnt + w.nleaf : nullptr);
    return 1;
}

#define SORT_TILE 256

// Writes the leaf-ordered copies of caller particle v at sorted position pos: FP64 form (x, y, gamma [, gu, gv]);
// precision form the duplicated split records eh = (xh, xh, yh, yh), el = (xl, xl, yl, yl), eg = (g, g, -g, -g),
// from its caller-order record (p, gg) read in advance by the caller.
__device__ __forceinline__ void place_particle(const Work &w, int v, int pos, int leaf, const double *__restrict__ x,
                                               const double *__restrict__ y, const double *__restrict__ g,
                                               const double *__restrict__ gu, const double *__restrict__ gv, int mixed,
                                               float4 p = float4{}, float gg = 0.f)
{
    w.perm[pos] = v;
    if (!w.morton)  // the adaptive tree reads no inverse permutation
        w.iperm[v] = pos;
    w.sleaf[pos] = leaf;
    if (mixed) {
        w.eh[pos] = make_float4(p.x, p.x, p.y, p.y);
        w.el[pos] = make_float4(p.z, p.z, p.w, p.w);
        w.eg[pos] = make_float4(gg, gg, -gg, -gg);
    } else {
        double xv, yv, gv0;
        if (w.rec64) {
            const Rec64 r = w.rec64[v];
            xv = r.x;
            yv = r.y;
            gv0 = r.g;
        } else {
            xv = x[v];
            yv = y[v];
            gv0 = g[v];
        }
        w.sx[pos] = xv;
        w.sy[pos] = yv;
        w.sg[pos] = gv0;
        if (gu) {
            w.sgu[pos] = gu[v];
            w.sgv[pos] = gv[v];
        }
        if (w.ad_mixed) {  // adaptive precision form: hi + lo floats in units u = sigma sqrt(2 / log2 e)
            const SysDev &d = w.sys[0];
            const double X = (xv - d.x0) * d.iu, Y = (yv - d.y0) * d.iu;
            const float hx = (float)X, hy = (float)Y;
            w.eh[pos] = make_float4(hx, hy, (float)(X - (double)hx), (float)(Y - (double)hy));
            w.eg[pos].x = (float)gv0;
        }
    }
}

// Ranks one leaf's entries ent[0..c) (keys all distinct) with the whole block: by caller index, or with `cls`
// (.y holds the boundary class) by (class, caller index); then writes the first position of classes 1..8 of the
// leaf. K = unsigned packs (class, index) into 32 bits, for caller indices below 2^28.
template <typename K>
__device__ __forceinline__ K rank_key(int2 e, bool cls)
{
    if (sizeof(K) == 4)
        return (K)(((cls ? (unsigned)e.y : 0u) << 28) | (unsigned)e.x);
    return (K)(((cls ? (unsigned long long)(unsigned)e.y : 0ull) << 32) | (unsigned)e.x);
}

template <typename K>
__device__ __forceinline__ void order_leaf_block(const Work &w, int leaf, const int2 *__restrict__ ent, K *tile,
                                                 int *ccount, bool cls, const double *x, const double *y,
                                                 const double *g, const double *gu, const double *gv, int mixed)
{
    const int s0 = w.start[leaf], c = w.start[leaf + 1] - s0;
    if (cls && threadIdx.x < 9)
        ccount[threadIdx.x] = 0;
    for (int e0 = 0; e0 < c; e0 += blockDim.x) {
        const int e = e0 + threadIdx.x;
        const int2 me = e < c ? ent[e] : make_int2(0, 0);
        float4 rec = float4{};
        float rg = 0.f;
        if (mixed && e < c) {  // the random read of the caller-order record overlaps the ranking
            rec = w.pos4u[2 * (int64_t)me.x];
            rg = w.pos4u[2 * (int64_t)me.x + 1].x;
        }
        const K v = rank_key<K>(me, cls);
        int rank = 0;
        for (int f0 = 0; f0 < c; f0 += SORT_TILE) {
            const int m = min(SORT_TILE, c - f0);
            constexpr int V = 16 / sizeof(K);  // keys per 16-byte shared-memory read
            const int mv = (m + V - 1) / V;    // the tile padded with the largest key, which no entry reaches
            __syncthreads();
            for (int j = threadIdx.x; j < mv * V; j += blockDim.x)
                tile[j] = j < m ? rank_key<K>(ent[f0 + j], cls) : ~K(0);
            __syncthreads();
            if (e < c) {
                if constexpr (sizeof(K) == 4) {
                    const uint4 *t4 = reinterpret_cast<const uint4 *>(tile);
                    for (int j = 0; j < mv; ++j) {
                        const uint4 q = t4[j];
                        rank += (q.x < v) + (q.y < v) + (q.z < v) + (q.w < v);
                    }
                } else {
                    const ulonglong2 *t2 = reinterpret_cast<const ulonglong2 *>(tile);
                    for (int j = 0; j < mv; ++j) {
                        const ulonglong2 q = t2[j];
                        rank += (q.x < v) + (q.y < v);
                    }
                }
            }
        }
        if (e < c) {
            place_particle(w, me.x, s0 + rank, leaf, x, y, g, gu, gv, mixed, rec, rg);
            if (cls)
                atomicAdd(&ccount[me.y], 1);
        }
    }
    if (cls) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int pos = s0;
            for (int k = 0; k < 8; ++k) {
                pos += ccount[k];
                w.cls_off[(int64_t)leaf * 8 + k] = pos;  // first position of class k + 1
            }
        }
    }
}

// Leaf order: each leaf's arrival order (atomic slots) is replaced by the caller's order, so that every run gives
// bit-identical results. The adaptive tree's cells: one thread per sorted position: its entry (caller index v, leaf) says which leaf run it
// is in; its rank is the number of entries of that run with a smaller caller index (the run's entries are read by
// every thread of the run, so a warp's reads of one leaf coalesce). Leaves holding more than kSmallLeaf particles
// are listed (by their first position) and ranked with a whole block each instead, through shared-memory tiles.
constexpr int kSmallLeaf = 128;

__global__ void __launch_bounds__(256) k_leaf_rank(Work w, const double *__restrict__ x, const double *__restrict__ y,
                                                   const double *__restrict__ g, const double *__restrict__ gu,
                                                   const double *__restrict__ gv, int mixed)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.n)
        return;
    const int2 e = w.tmp[p];
    const int leaf = e.y, s0 = w.start[leaf], c = w.start[leaf + 1] - s0;
    if (c > kSmallLeaf) {
        if (p == s0)
            w.big[atomicAdd(w.big_cnt, 1)] = leaf;
        return;
    }
    float4 rec = float4{};
    float rg = 0.f;
    if (mixed) {
        rec = w.pos4u[2 * (int64_t)e.x];
        rg = w.pos4u[2 * (int64_t)e.x + 1].x;
    }
    int rank = 0;
    for (int q = s0; q < s0 + c; ++q)
        rank += w.tmp[q].x < e.x;
    place_particle(w, e.x, s0 + rank, leaf, x, y, g, gu, gv, mixed, rec, rg);
}

__global__ void __launch_bounds__(128) k_leaf_big(Work w, const double *__restrict__ x, const double *__restrict__ y,
                                                  const double *__restrict__ g, const double *__restrict__ gu,
                                                  const double *__restrict__ gv, int mixed)
{
    __shared__ __align__(16) unsigned long long tile[SORT_TILE];
    const int nb = *w.big_cnt;
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {  // block-uniform
        const int leaf = w.big[b];
        order_leaf_block<unsigned long long>(w, leaf, w.tmp + w.start[leaf], tile, nullptr, false, x, y, g, gu, gv,
                                             mixed);
    }
}

// The uniform tree (tens of particles in each of at most millions of leaves): one block per leaf.
__global__ void __launch_bounds__(64) k_leaf_block(Work w, const double *__restrict__ x, const double *__restrict__ y,
                                                   const double *__restrict__ g, const double *__restrict__ gu,
                                                   const double *__restrict__ gv, int mixed)
{
    __shared__ __align__(16) unsigned long long tile[SORT_TILE];
    __shared__ int ccount[9];
    const int leaf = blockIdx.x;
    // no bucket overflowed: the leaf's bucket, else its run of the scattered list
    const int2 *ent = w.bkt && w.cnt[w.nleaf] == 0 ? w.bkt + (int64_t)leaf * w.bkt_cap : w.tmp + w.start[leaf];
    if (w.n <= (1 << 28))  // (class, caller index) in 32 bits
        order_leaf_block<unsigned>(w, leaf, ent, reinterpret_cast<unsigned *>(tile), ccount, w.cls_off != nullptr,
                                   x, y, g, gu, gv, mixed);
    else
        order_leaf_block<unsigned long long>(w, leaf, ent, tile, ccount, w.cls_off != nullptr, x, y, g, gu, gv,
                                             mixed);
}

int launch_gather(const Work &w, const double *x, const double *y, const double *g, const double *gu,
                  const double *gv, cudaStream_t s)
{
    const int mixed = (w.mixed && !gu) ? 1 : 0;
    if (!w.morton) {  // measured as fast as the per-position ranking there, in one launch
        k_leaf_block<<<w.nleaf, 64, 0, s>>>(w, x, y, g, gu, gv, mixed);
        return 1;
    }
    // the adaptive tree's depth-L cells (millions, mostly empty, a few tens of particles at most)
    cudaMemsetAsync(w.big_cnt, 0, sizeof(int), s);
    k_leaf_rank<<<(w.n + 255) / 256, 256, 0, s>>>(w, x, y, g, gu, gv, mixed);
    const int most = w.n / (kSmallLeaf + 1) + 1;  // leaves that can hold more than kSmallLeaf particles
    k_leaf_big<<<min(most, 152 * 8), 128, 0, s>>>(w, x, y, g, gu, gv, mixed);
    return 2;
}

// ------------------------------------------------------------------ ordered near-field pair count

__global__ void k_pair_count(const SysDev *__restrict__ sys, int nsys, int nleaf, const int *__restrict__ start,
                             unsigned long long *out)
{
    int leaf = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = 0;
    if (leaf < nleaf) {
        int k = nsys == 1 ? 0 : find_sys_by_leaf(sys, nsys, leaf);
        const SysDev &d = sys[k];
        int L = d.depth, ns = 1 << L, local = (int)(leaf - d.leaf0);
        int ix = local & (ns - 1), iy = local >> L;
        long long own = start[leaf + 1] - start[leaf], nb = 0;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int jx = ix + dx, jy = iy + dy;
                if (jx < 0 || jy < 0 || jx >= ns || jy >= ns)
                    continue;
                int j = (int)(d.leaf0 + (int64_t)jy * ns + jx);
                nb += start[j + 1] - start[j];
            }
        c = (unsigned long long)(own * nb - own);
    }
    for (int o = 16; o > 0; o >>= 1)
        c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c)
        atomicAdd(out, c);
}

int launch_pair_count(const Work &w, cudaStream_t s)
{
    k_pair_count<<<(w.nleaf + 255) / 256, 256, 0, s>>>(w.sys, w.nsys, w.nleaf, w.start, w.pair_count);
    return 1;
}

}  // namespace fmm
