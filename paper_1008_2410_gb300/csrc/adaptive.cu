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
// Expansions exist on levels >= 2 (levels 0 and 1 hold no well separated pair) and are radius scaled, with
// zeta = (z - c) / w for a box of side w and charges q' = -i gamma (1 / 2pi applied at the end):
//   multipole  a~_m = sum_j q'_j zeta_j^m
//   local      b~_k = w^k b_k, so that the far field at z is sum_k b~_k zeta^k
//   M2M        a~P_n = sum_{m<=n} C(n, m) delta^(n-m) 2^-m a~C_m,      delta = (c_child - c_parent) / w_parent
//   M2L        b~_k += (1/w) sum_m a~_m (-1)^(m+1) C(m+k, m) / delta^(m+k+1),  delta = (c_src - c_tgt) / w
//   L2L        b~C_k = 2^-k sum_{j>=k} C(j, k) delta^(j-k) b~P_j,      delta = (c_child - c_parent) / w_parent
//   P2L        b~_k += -(1/w) sum_j q'_j / s_j^(k+1),   s_j = (z_j - c) / w
//   M2P        w(z) += (1/w_s) sum_m a~_m / t^(m+1),    t = (z - c_s) / w_s
// This path computes in FP64 throughout.
#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr double kTwoPi = 6.283185307179586476925;
constexpr int kStack = 48;  // DFS stack of the U / W walk; depth <= 2 (L - l) + 2 <= 26 for L <= 12

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

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cinv(double2 a)
{
    const double d = 1.0 / (a.x * a.x + a.y * a.y);
    return make_double2(a.x * d, -a.y * d);
}
__device__ __forceinline__ double2 cpow(double2 a, int e)  // a^e, e >= 0, by repeated squaring
{
    double2 r = make_double2(1.0, 0.0);
    while (e > 0) {
        if (e & 1)
            r = cmul(r, a);
        a = cmul(a, a);
        e >>= 1;
    }
    return r;
}

__device__ __forceinline__ double2 centre(const SysDev &d, int l, int x, int y)
{
    const double w = ldexp(d.S, -l);
    return make_double2(d.x0 + (x + 0.5) * w, d.y0 + (y + 0.5) * w);
}

__device__ __forceinline__ double2 *mp_of(const Work &w, int l, unsigned m)
{
    return w.M64 + ((size_t)w.sys[0].box0[l] + m) * w.p;
}
__device__ __forceinline__ double2 *loc_of(const Work &w, int l, unsigned m)
{
    return w.L64 + ((size_t)w.sys[0].box0[l] + m) * w.p;
}

// ------------------------------------------------------------------ stage 4: P2M at the leaves of level l

__global__ void __launch_bounds__(128) k_ad_p2m(Work w, int l)
{
    const unsigned m = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const SysDev &d = w.sys[0];
    const Tree t{w.start, d.depth, w.adapt_cap};
    if (m >= (1u << (2 * l)))
        return;
    const int bx = (int)compact1(m), by = (int)compact1(m >> 1);
    if (!box_exists(t, l, bx, by) || box_split(t, l, bx, by))
        return;
    const int j0 = box_first(t, l, m), j1 = j0 + box_count(t, l, m);
    const double2 c = centre(d, l, bx, by);
    const double iw = ldexp(1.0, l) / d.S;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = j0; j < j1; ++j) {
        const double2 z = make_double2((w.sx[j] - c.x) * iw, (w.sy[j] - c.y) * iw);
        const double2 q = make_double2(0.0, -w.sg[j]);
        acc = cadd(acc, cmul(q, cpow(z, lane)));
    }
    if (lane < w.p)
        mp_of(w, l, m)[lane] = acc;
}

// ------------------------------------------------------------------ stage 5: M2M into the split boxes of level l

__global__ void __launch_bounds__(128) k_ad_m2m(Work w, int l)
{
    __shared__ double2 sa[4][4][FMM_PMAX];
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned m = blockIdx.x * 4 + wi;
    const SysDev &d = w.sys[0];
    const Tree t{w.start, d.depth, w.adapt_cap};
    if (m >= (1u << (2 * l)))
        return;
    const int bx = (int)compact1(m), by = (int)compact1(m >> 1);
    if (!box_exists(t, l, bx, by) || !box_split(t, l, bx, by))
        return;
    const int p = w.p;
    for (int c = 0; c < 4; ++c)
        if (lane < p)
            sa[wi][c][lane] = mp_of(w, l + 1, 4 * m + c)[lane];
    __syncwarp();
    if (lane >= p)
        return;
    const int n = lane;
    double2 acc = make_double2(0.0, 0.0);
    for (int c = 0; c < 4; ++c) {
        const double2 dl = make_double2(((c & 1) - 0.5) * 0.5, ((c >> 1) - 0.5) * 0.5);
        double2 pw = make_double2(1.0, 0.0);  // delta^(n - k), k from n down to 0
        double C = 1.0;                       // C(n, k)
        for (int k = n; k >= 0; --k) {
            acc = cadd(acc, cscale(cmul(pw, sa[wi][c][k]), C * ldexp(1.0, -k)));
            pw = cmul(pw, dl);
            C = C * (double)k / (double)(n - k + 1);
        }
    }
    mp_of(w, l, m)[n] = acc;
}

// ------------------------------------------------------------------ stages 6-7: locals of level l (L2L + V + X)

__global__ void __launch_bounds__(128) k_ad_down(Work w, int l)
{
    __shared__ double2 sa[4][FMM_PMAX];
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned m = blockIdx.x * 4 + wi;
    const SysDev &d = w.sys[0];
    const Tree t{w.start, d.depth, w.adapt_cap};
    if (m >= (1u << (2 * l)))
        return;
    const int bx = (int)compact1(m), by = (int)compact1(m >> 1);
    if (!box_exists(t, l, bx, by))
        return;
    const int p = w.p, L = d.depth, nside = 1 << l;
    const int k = lane < p ? lane : p - 1;  // lanes >= p shadow the last coefficient and do not store
    const double iw = ldexp(1.0, l) / d.S;
    double2 acc = make_double2(0.0, 0.0);
    // L2L from the parent
    if (l >= 3) {
        if (lane < p)
            sa[wi][lane] = loc_of(w, l - 1, m >> 2)[lane];
        __syncwarp();
        const double2 dl = make_double2(((bx & 1) - 0.5) * 0.5, ((by & 1) - 0.5) * 0.5);
        double2 pw = make_double2(1.0, 0.0);  // delta^(j - k)
        double C = 1.0;                       // C(j, k)
        double2 s = make_double2(0.0, 0.0);
        for (int j = k; j < p; ++j) {
            s = cadd(s, cscale(cmul(pw, sa[wi][j]), C));
            pw = cmul(pw, dl);
            C = C * (double)(j + 1) / (double)(j + 1 - k);
        }
        acc = cscale(s, ldexp(1.0, -k));
        __syncwarp();
    }
    // V: M2L from the children of the parent's neighbours that are not adjacent to b
    const int px = bx >> 1, py = by >> 1;
    for (int sy = 2 * py - 2; sy <= 2 * py + 3; ++sy) {
        for (int sx = 2 * px - 2; sx <= 2 * px + 3; ++sx) {
            if (sx < 0 || sy < 0 || sx >= nside || sy >= nside)
                continue;
            if (abs(sx - bx) <= 1 && abs(sy - by) <= 1)
                continue;
            if (!box_exists(t, l, sx, sy))
                continue;
            const unsigned ms = morton2(sx, sy);
            if (box_count(t, l, ms) == 0)
                continue;
            if (lane < p)
                sa[wi][lane] = mp_of(w, l, ms)[lane];
            __syncwarp();
            const double2 inv = cinv(make_double2((double)(sx - bx), (double)(sy - by)));
            double2 pw = cpow(inv, k + 1);  // delta^-(m + k + 1)
            double C = 1.0;                 // C(m + k, m)
            double2 s = make_double2(0.0, 0.0);
            for (int mm = 0; mm < p; ++mm) {
                const double sg = (mm & 1) ? C : -C;
                s = cadd(s, cscale(cmul(pw, sa[wi][mm]), sg));
                pw = cmul(pw, inv);
                C = C * (double)(mm + k + 1) / (double)(mm + 1);
            }
            acc = cadd(acc, cscale(s, iw));
            __syncwarp();
        }
    }
    // X: P2L from the coarser leaves adjacent to the parent but not to b
    int seen[8];
    int nseen = 0;
    for (int dy = -1; dy <= 1; ++dy) {
        for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0)
                continue;
            int lq = l - 1, qx = px + dx, qy = py + dy;
            if (qx < 0 || qy < 0 || qx >= (nside >> 1) || qy >= (nside >> 1))
                continue;
            covering_box(t, lq, qx, qy);
            if (lq == l - 1 && box_split(t, lq, qx, qy))
                continue;
            if (adjacent(L, l, bx, by, lq, qx, qy))
                continue;
            const int id = pack_box(lq, qx, qy);
            bool dup = false;
            for (int e = 0; e < nseen; ++e)
                dup |= seen[e] == id;
            if (dup)
                continue;
            seen[nseen++] = id;
            const unsigned mq = morton2(qx, qy);
            const int j0 = box_first(t, lq, mq), j1 = j0 + box_count(t, lq, mq);
            const double2 c = centre(d, l, bx, by);
            double2 s = make_double2(0.0, 0.0);
            for (int j = j0; j < j1; ++j) {
                const double2 inv = cinv(make_double2((w.sx[j] - c.x) * iw, (w.sy[j] - c.y) * iw));
                const double2 q = make_double2(0.0, -w.sg[j]);
                s = cadd(s, cmul(q, cpow(inv, k + 1)));
            }
            acc = cadd(acc, cscale(s, -iw));
        }
    }
    if (lane < p)
        loc_of(w, l, m)[lane] = acc;
}

// ------------------------------------------------------------------ leaf of a sorted particle

__device__ __forceinline__ void particle_leaf(const Tree &t, unsigned kf, int &l, int &x, int &y)
{
    int lv = 0;
    while (lv < t.L && box_count(t, lv, kf >> (2 * (t.L - lv))) > t.B)
        ++lv;
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

// ------------------------------------------------------------------ stage 9: near field over U

__global__ void __launch_bounds__(128) k_ad_near(Work w)
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
    double su = 0.0, sv = 0.0;
    auto near = [&](int j0, int j1) {
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
    auto none = [](int, int, int) {};
    walk_uw(w, t, l, bx, by, near, none);
    w.near64[i] = make_double2(su, sv);
}

// ------------------------------------------------------------------ stages 8 + 10: L2P, W, sum, unsort

__global__ void __launch_bounds__(128) k_ad_final(Work w, int use_near, int use_far, double *u, double *v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w.n)
        return;
    const SysDev &d = w.sys[0];
    double ru = 0.0, rv = 0.0;
    if (use_far) {
        const Tree t{w.start, d.depth, w.adapt_cap};
        int l, bx, by;
        particle_leaf(t, (unsigned)w.sleaf[i], l, bx, by);
        const double xi = w.sx[i], yi = w.sy[i];
        const int p = w.p;
        double2 wf = make_double2(0.0, 0.0);
        if (l >= 2) {
            const double2 c = centre(d, l, bx, by);
            const double iw = ldexp(1.0, l) / d.S;
            const double2 z = make_double2((xi - c.x) * iw, (yi - c.y) * iw);
            const double2 *b = loc_of(w, l, morton2(bx, by));
            for (int k = p - 1; k >= 0; --k)
                wf = cadd(cmul(wf, z), b[k]);
        }
        auto none = [](int, int) {};
        auto far = [&](int ls, int sx, int sy) {
            const double2 c = centre(d, ls, sx, sy);
            const double iws = ldexp(1.0, ls) / d.S;
            const double2 uinv = cinv(make_double2((xi - c.x) * iws, (yi - c.y) * iws));
            const double2 *a = mp_of(w, ls, morton2(sx, sy));
            double2 s = make_double2(0.0, 0.0);
            for (int mm = p - 1; mm >= 0; --mm)
                s = cmul(cadd(s, a[mm]), uinv);
            wf = cadd(wf, cscale(s, iws));
        };
        walk_uw(w, t, l, bx, by, none, far);
        ru = wf.x / kTwoPi;
        rv = -wf.y / kTwoPi;
    }
    if (use_near) {
        const double2 nr = w.near64[i];
        ru += nr.x;
        rv += nr.y;
    }
    const int pos = w.perm[i];
    u[pos] = ru;
    v[pos] = rv;
}

}  // namespace

int launch_adaptive_sweep(const Work &w, cudaStream_t s)
{
    const int L = w.maxdepth;
    int nl = 0;
    for (int l = 2; l <= L; ++l, ++nl)
        k_ad_p2m<<<(unsigned)(((1ull << (2 * l)) + 3) / 4), 128, 0, s>>>(w, l);
    for (int l = L - 1; l >= 2; --l, ++nl)
        k_ad_m2m<<<(unsigned)(((1ull << (2 * l)) + 3) / 4), 128, 0, s>>>(w, l);
    for (int l = 2; l <= L; ++l, ++nl)
        k_ad_down<<<(unsigned)(((1ull << (2 * l)) + 3) / 4), 128, 0, s>>>(w, l);
    return nl;
}

int launch_adaptive_near(const Work &w, cudaStream_t s)
{
    k_ad_near<<<(w.n + 127) / 128, 128, 0, s>>>(w);
    return 1;
}

int launch_adaptive_final(const Work &w, int use_near, int use_far, double *u, double *v, cudaStream_t s)
{
    k_ad_final<<<(w.n + 127) / 128, 128, 0, s>>>(w, use_near, use_far, u, v);
    return 1;
}

}  // namespace fmm
