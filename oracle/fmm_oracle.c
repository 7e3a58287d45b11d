/*
 * fmm_oracle.c -- plain, slow, FP64 CPU oracle for one 2D vortex-blob velocity evaluation.
 *
 * TEST INFRASTRUCTURE. Only the tests, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this library. It shares no code, header, table or helper with the CUDA library in
 * paper_1008_2410_gb300/csrc, and it includes nothing from there.
 *
 * What it computes (M. G. Knepley, "Removing the Barrier to Scalability in Parallel FMM"):
 *   Eq. 6   K_sigma(z) = (-v, u) (1 - exp(-|z|^2 / 2 sigma^2)) / (2 pi |z|^2),  z = (u, v);  K_sigma(0) = 0
 *   Eq. 7   u_sigma(z_i) = sum_j gamma_j K_sigma(z_i - z_j)                     (the O(N^2) direct sum)
 *   §2 end  the far field uses expansions of the un-regularised 1/|z|^2 kernel; the exact K_sigma is used
 *           only between particles in the same or adjacent finest-level cells
 *   §3      multipole coefficient m:  a_m = (-i / 2pi) sum_p Gamma_p (z_p - z_c)^m,  t terms (m = 0 .. t-1)
 *   Fig. 1  stages 1 tree, 2 binning, 3 interaction lists, 4 P2M, 5 M2M, 6 M2L, 7 L2L, 8 L2P,
 *           9 near-field direct evaluation, 10 sum
 *   Eq. 3   (2D Euler) the particles move with the local velocity and keep their circulation
 *
 * Complex velocity: w = u - i v. For a point vortex, u - i v = q / (z - z_j) with q = -i gamma / (2 pi),
 * which is Eq. 6 without the Gaussian factor. Coefficients here are the plain (unscaled) ones of the
 * paper's §3 formula; the translation formulas (M2M, M2L, L2L), which the paper delegates to PetFMM, are
 * the binomial re-expansions of 1/(z - z_j), written out in each function below.
 *
 * Readings where the paper is silent:
 *   - root square: given, or centred on the bounding box with side extent*(1 + 2^-20) (minimum 1e-300);
 *   - leaf of a point: ix = floor((x - x0) * (2^L / S)), clamped to [0, 2^L - 1];
 *   - p terms (m = 0..p-1) for both multipole and local expansions;
 *   - M2M on levels L-1..2, M2L on levels 2..L, L2L into levels 3..L (§3 sums); depth <= 1 is all near field;
 *   - a particle does not act on itself; distinct coincident particles contribute K_sigma(0) = 0.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

typedef double complex cplx;

/* ---------------------------------------------------------------- Eq. 6: the regularised kernel */

/* K_sigma at displacement (a, b): writes (ku, kv). 1 - exp(-x) is evaluated as -expm1(-x), which is the
 * same quantity without cancellation for small x. Displacement zero gives 0 (the limit of Eq. 6). */
void oracle_kernel(double a, double b, double sigma, double *ku, double *kv)
{
    double r2 = a * a + b * b;
    if (r2 == 0.0) {
        *ku = 0.0;
        *kv = 0.0;
        return;
    }
    double f = -expm1(-r2 / (2.0 * sigma * sigma)) / (2.0 * ORACLE_PI * r2);
    *ku = -b * f;
    *kv = a * f;
}

/* Point-vortex (un-regularised) kernel used for the far field (§2, last paragraph). */
static void point_vortex_kernel(double a, double b, double *ku, double *kv)
{
    double r2 = a * a + b * b;
    double f = 1.0 / (2.0 * ORACLE_PI * r2);
    *ku = -b * f;
    *kv = a * f;
}

/* ---------------------------------------------------------------- Eq. 7: the direct sum */

/* u_i = sum_{j != i} gamma_j K_sigma(z_i - z_j) for the targets listed in tidx (all n if tidx == NULL,
 * then nt must be n). Output k belongs to target tidx[k]. */
void oracle_direct(int64_t n, const double *x, const double *y, const double *g, double sigma,
                   int64_t nt, const int64_t *tidx, double *u, double *v)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < nt; ++k) {
        int64_t i = tidx ? tidx[k] : k;
        double su = 0.0, sv = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double ku, kv;
            oracle_kernel(x[i] - x[j], y[i] - y[j], sigma, &ku, &kv);
            su += g[j] * ku;
            sv += g[j] * kv;
        }
        u[k] = su;
        v[k] = sv;
    }
}

/* ---------------------------------------------------------------- stage 1: root square and leaves */

/* Default root square: centre of the bounding box, side = extent * (1 + 2^-20), at least 1e-300.
 * out = {x0, y0, S}; the square is [x0, x0 + S] x [y0, y0 + S]. */
void oracle_default_domain(int64_t n, const double *x, const double *y, double *out)
{
    if (n <= 0) {
        out[0] = 0.0;
        out[1] = 0.0;
        out[2] = 1.0;
        return;
    }
    double xmin = x[0], xmax = x[0], ymin = y[0], ymax = y[0];
    for (int64_t i = 1; i < n; ++i) {
        if (x[i] < xmin) xmin = x[i];
        if (x[i] > xmax) xmax = x[i];
        if (y[i] < ymin) ymin = y[i];
        if (y[i] > ymax) ymax = y[i];
    }
    double ex = xmax - xmin, ey = ymax - ymin;
    double ext = ex > ey ? ex : ey;
    double side = ext * (1.0 + 0x1p-20);
    if (side < 1e-300)
        side = 1e-300;
    double cx = 0.5 * (xmin + xmax), cy = 0.5 * (ymin + ymax);
    double half = 0.5 * side;
    out[0] = cx - half;
    out[1] = cy - half;
    out[2] = side;
}

/* Leaf column (or row) of coordinate c: floor((c - c0) * scale), clamped to [0, nside - 1]. */
static int leaf_coord(double c, double c0, double scale, int nside)
{
    double t = (c - c0) * scale;
    double f = floor(t);
    if (f < 0.0)
        return 0;
    if (f > (double)(nside - 1))
        return nside - 1;
    return (int)f;
}

/* Leaf coordinates of every particle at depth L. With check != 0 a point outside the closed square is an
 * error (returns -1); otherwise out-of-square points are clamped. Returns 0 on success. */
int oracle_leaf_coords(int64_t n, const double *x, const double *y, int L, const double *dom, int check,
                       int32_t *ix, int32_t *iy)
{
    int nside = 1 << L;
    double scale = ldexp(1.0, L) / dom[2];
    double xe = dom[0] + dom[2], ye = dom[1] + dom[2];
    for (int64_t i = 0; i < n; ++i) {
        if (check && (!(x[i] >= dom[0]) || !(x[i] <= xe) || !(y[i] >= dom[1]) || !(y[i] <= ye)))
            return -1;
        ix[i] = leaf_coord(x[i], dom[0], scale, nside);
        iy[i] = leaf_coord(y[i], dom[1], scale, nside);
    }
    return 0;
}

/* ---------------------------------------------------------------- stages 4..8: expansions */

/* Binomial coefficient C(n, k) in double (exact while it fits 53 bits). */
static double binom(int n, int k)
{
    if (k < 0 || k > n)
        return 0.0;
    if (k > n - k)
        k = n - k;
    double c = 1.0;
    for (int i = 1; i <= k; ++i)
        c = c * (double)(n - k + i) / (double)i;
    return nearbyint(c);
}

/* Stage 4, §3 multipole coefficient: a_m += sum_j q_j (z_j - c)^m, m = 0..p-1, for complex charges q_j.
 * For vortex blobs q_j = -i gamma_j / (2 pi). a holds p complex values (re, im interleaved). */
void oracle_p2m(int64_t np, const double *x, const double *y, const double *qre, const double *qim,
                double cx, double cy, int p, double *a_out)
{
    cplx *a = (cplx *)a_out;
    for (int64_t j = 0; j < np; ++j) {
        cplx q = qre[j] + I * qim[j];
        cplx dz = (x[j] - cx) + I * (y[j] - cy);
        cplx pw = 1.0;
        for (int m = 0; m < p; ++m) {
            a[m] += q * pw;
            pw *= dz;
        }
    }
}

/* Far value of a multipole about c at displacement dz = z - c: sum_m a_m / dz^(m+1). */
void oracle_multipole_eval(int p, const double *a_in, double dzx, double dzy, double *w_out)
{
    const cplx *a = (const cplx *)a_in;
    cplx dz = dzx + I * dzy, inv = 1.0 / dz, pw = inv, w = 0.0;
    for (int m = 0; m < p; ++m) {
        w += a[m] * pw;
        pw *= inv;
    }
    w_out[0] = creal(w);
    w_out[1] = cimag(w);
}

/* Stage 5, M2M: the expansion about the parent centre of a child multipole, d = c_child - c_parent.
 * From (z_j - c_parent)^n = ((z_j - c_child) + d)^n:  b_n += sum_{m<=n} C(n, m) d^(n-m) a_m. Accumulates. */
void oracle_m2m(int p, const double *a_in, double dx, double dy, double *b_out)
{
    const cplx *a = (const cplx *)a_in;
    cplx *b = (cplx *)b_out;
    cplx d = dx + I * dy;
    cplx dp[64];
    dp[0] = 1.0;
    for (int k = 1; k < p; ++k)
        dp[k] = dp[k - 1] * d;
    for (int n = 0; n < p; ++n)
        for (int m = 0; m <= n; ++m)
            b[n] += binom(n, m) * dp[n - m] * a[m];
}

/* Stage 6, M2L: the local expansion about c_T of a multipole about c_S, d = c_S - c_T. From
 * 1/(zeta - d)^(m+1) = (-d)^-(m+1) sum_l C(m+l, l) (zeta/d)^l with zeta = z - c_T:
 *     b_l += sum_m a_m (-1)^(m+1) C(m+l, m) / d^(m+l+1).   Accumulates. */
void oracle_m2l(int p, const double *a_in, double dx, double dy, double *b_out)
{
    const cplx *a = (const cplx *)a_in;
    cplx *b = (cplx *)b_out;
    cplx d = dx + I * dy, inv = 1.0 / d;
    cplx ip[130];
    ip[0] = 1.0;
    for (int k = 1; k <= 2 * p; ++k)
        ip[k] = ip[k - 1] * inv;
    for (int l = 0; l < p; ++l) {
        cplx s = 0.0;
        for (int m = 0; m < p; ++m) {
            double sign = (m % 2 == 0) ? -1.0 : 1.0; /* (-1)^(m+1) */
            s += a[m] * (sign * binom(m + l, m)) * ip[m + l + 1];
        }
        b[l] += s;
    }
}

/* Stage 7, L2L: the local expansion about the child centre, d = c_child - c_parent. From
 * (z - c_parent)^l = ((z - c_child) + d)^l:  b'_k += sum_{l>=k} C(l, k) d^(l-k) b_l.   Accumulates. */
void oracle_l2l(int p, const double *b_in, double dx, double dy, double *c_out)
{
    const cplx *b = (const cplx *)b_in;
    cplx *c = (cplx *)c_out;
    cplx d = dx + I * dy;
    cplx dp[64];
    dp[0] = 1.0;
    for (int k = 1; k < p; ++k)
        dp[k] = dp[k - 1] * d;
    for (int k = 0; k < p; ++k)
        for (int l = k; l < p; ++l)
            c[k] += binom(l, k) * dp[l - k] * b[l];
}

/* Stage 8, L2P: w = sum_l b_l dz^l at dz = z - c (w = u - i v). */
void oracle_l2p(int p, const double *b_in, double dzx, double dzy, double *w_out)
{
    const cplx *b = (const cplx *)b_in;
    cplx dz = dzx + I * dzy, pw = 1.0, w = 0.0;
    for (int l = 0; l < p; ++l) {
        w += b[l] * pw;
        pw *= dz;
    }
    w_out[0] = creal(w);
    w_out[1] = cimag(w);
}

/* ---------------------------------------------------------------- the uniform quadtree */

typedef struct {
    int L, p;
    double x0, y0, S;
    int32_t *ix, *iy;      /* leaf coordinates per particle */
    int64_t *start, *list; /* leaf l holds list[start[l] .. start[l+1]) in input order */
    cplx **mp, **loc;      /* per level: 4^l boxes x p coefficients */
} tree_t;

static double box_width(const tree_t *t, int l) { return t->S / ldexp(1.0, l); }

static cplx box_centre(const tree_t *t, int l, int bx, int by)
{
    double w = box_width(t, l);
    return (t->x0 + (bx + 0.5) * w) + I * (t->y0 + (by + 0.5) * w);
}

static void tree_free(tree_t *t)
{
    free(t->ix);
    free(t->iy);
    free(t->start);
    free(t->list);
    if (t->mp)
        for (int l = 0; l <= t->L; ++l)
            free(t->mp[l]);
    if (t->loc)
        for (int l = 0; l <= t->L; ++l)
            free(t->loc[l]);
    free(t->mp);
    free(t->loc);
}

/* Stages 1-2: root square, leaf of every particle, per-leaf lists kept in input order. */
static int tree_build(tree_t *t, int64_t n, const double *x, const double *y, int L, int p, const double *dom)
{
    memset(t, 0, sizeof(*t));
    t->L = L;
    t->p = p;
    double d[3];
    int check = dom != NULL;
    if (dom) {
        d[0] = dom[0];
        d[1] = dom[1];
        d[2] = dom[2];
    } else {
        oracle_default_domain(n, x, y, d);
    }
    t->x0 = d[0];
    t->y0 = d[1];
    t->S = d[2];
    int64_t nl = (int64_t)1 << (2 * L);
    t->ix = malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    t->iy = malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    t->start = calloc((size_t)nl + 1, sizeof(int64_t));
    t->list = malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    t->mp = calloc((size_t)L + 1, sizeof(cplx *));
    t->loc = calloc((size_t)L + 1, sizeof(cplx *));
    if (!t->ix || !t->iy || !t->start || !t->list || !t->mp || !t->loc)
        return -2;
    if (oracle_leaf_coords(n, x, y, L, d, check, t->ix, t->iy) != 0)
        return -1;
    int nside = 1 << L;
    for (int64_t i = 0; i < n; ++i)
        t->start[(int64_t)t->iy[i] * nside + t->ix[i] + 1]++;
    for (int64_t l = 0; l < nl; ++l)
        t->start[l + 1] += t->start[l];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)nl);
    if (!fill)
        return -2;
    memcpy(fill, t->start, sizeof(int64_t) * (size_t)nl);
    for (int64_t i = 0; i < n; ++i)
        t->list[fill[(int64_t)t->iy[i] * nside + t->ix[i]]++] = i;
    free(fill);
    for (int l = 0; l <= L; ++l) {
        t->mp[l] = calloc((size_t)p << (2 * l), sizeof(cplx));
        t->loc[l] = calloc((size_t)p << (2 * l), sizeof(cplx));
        if (!t->mp[l] || !t->loc[l])
            return -2;
    }
    return 0;
}

/* Stage 3: interaction list of box (bx, by) at level l >= 2: the children of the parent's neighbours
 * (the parent included) that are not adjacent to the box. Returns the count (at most 27). */
static int interaction_list(int l, int bx, int by, int *sx, int *sy)
{
    int n = 0, np = 1 << (l - 1), px = bx >> 1, py = by >> 1;
    for (int qy = py - 1; qy <= py + 1; ++qy)
        for (int qx = px - 1; qx <= px + 1; ++qx) {
            if (qx < 0 || qy < 0 || qx >= np || qy >= np)
                continue;
            for (int cy = 0; cy < 2; ++cy)
                for (int cx = 0; cx < 2; ++cx) {
                    int jx = 2 * qx + cx, jy = 2 * qy + cy;
                    if (abs(jx - bx) <= 1 && abs(jy - by) <= 1)
                        continue;
                    sx[n] = jx;
                    sy[n] = jy;
                    ++n;
                }
        }
    return n;
}

/* Size of the interaction list of every box at level l (row-major), for tests of stage 3. */
void oracle_interaction_list_sizes(int l, int32_t *sizes)
{
    int ns = 1 << l, sx[36], sy[36];
    for (int by = 0; by < ns; ++by)
        for (int bx = 0; bx < ns; ++bx)
            sizes[by * ns + bx] = interaction_list(l, bx, by, sx, sy);
}

/* Stages 4-7 for complex charges q (re/im arrays): P2M at the leaves, M2M upward, M2L on every box marked
 * in `need` (or every box if need == NULL), then L2L downward into the marked boxes. */
static void upward_downward(tree_t *t, const double *x, const double *y, const double *qre, const double *qim,
                            unsigned char **need)
{
    int L = t->L, p = t->p;
    if (L < 2)
        return;
    /* stage 4: P2M on every leaf */
    int nside = 1 << L;
    for (int by = 0; by < nside; ++by)
        for (int bx = 0; bx < nside; ++bx) {
            int64_t b = (int64_t)by * nside + bx;
            cplx c = box_centre(t, L, bx, by);
            for (int64_t k = t->start[b]; k < t->start[b + 1]; ++k) {
                int64_t j = t->list[k];
                oracle_p2m(1, x + j, y + j, qre + j, qim + j, creal(c), cimag(c), p, (double *)(t->mp[L] + b * p));
            }
        }
    /* stage 5: M2M, levels L-1 .. 2 */
    for (int l = L - 1; l >= 2; --l) {
        int ns = 1 << l;
        for (int by = 0; by < ns; ++by)
            for (int bx = 0; bx < ns; ++bx) {
                cplx cp = box_centre(t, l, bx, by);
                for (int cy = 0; cy < 2; ++cy)
                    for (int cx = 0; cx < 2; ++cx) {
                        int jx = 2 * bx + cx, jy = 2 * by + cy;
                        cplx cc = box_centre(t, l + 1, jx, jy);
                        cplx d = cc - cp;
                        oracle_m2m(p, (double *)(t->mp[l + 1] + ((int64_t)jy * 2 * ns + jx) * p), creal(d), cimag(d),
                                   (double *)(t->mp[l] + ((int64_t)by * ns + bx) * p));
                    }
            }
    }
    /* stage 6: M2L, levels 2 .. L */
    for (int l = 2; l <= L; ++l) {
        int ns = 1 << l;
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t b = 0; b < (int64_t)ns * ns; ++b) {
            if (need && !need[l][b])
                continue;
            int bx = (int)(b % ns), by = (int)(b / ns), sx[36], sy[36];
            cplx ct = box_centre(t, l, bx, by);
            int cnt = interaction_list(l, bx, by, sx, sy);
            for (int s = 0; s < cnt; ++s) {
                cplx d = box_centre(t, l, sx[s], sy[s]) - ct;
                oracle_m2l(p, (double *)(t->mp[l] + ((int64_t)sy[s] * ns + sx[s]) * p), creal(d), cimag(d),
                           (double *)(t->loc[l] + b * p));
            }
        }
    }
    /* stage 7: L2L, levels 2 -> 3 -> ... -> L */
    for (int l = 2; l < L; ++l) {
        int ns = 1 << (l + 1);
        for (int64_t b = 0; b < (int64_t)ns * ns; ++b) {
            if (need && !need[l + 1][b])
                continue;
            int bx = (int)(b % ns), by = (int)(b / ns);
            cplx d = box_centre(t, l + 1, bx, by) - box_centre(t, l, bx >> 1, by >> 1);
            oracle_l2l(p, (double *)(t->loc[l] + ((int64_t)(by >> 1) * (ns >> 1) + (bx >> 1)) * p), creal(d),
                       cimag(d), (double *)(t->loc[l + 1] + b * p));
        }
    }
}

/* Marks the leaves of the targets and all their ancestors (NULL targets: returns NULL = everything). */
static unsigned char **mark_needed(const tree_t *t, int64_t nt, const int64_t *tidx)
{
    if (!tidx)
        return NULL;
    int L = t->L;
    unsigned char **need = calloc((size_t)L + 1, sizeof(unsigned char *));
    for (int l = 0; l <= L; ++l)
        need[l] = calloc((size_t)1 << (2 * l), 1);
    int nside = 1 << L;
    for (int64_t k = 0; k < nt; ++k) {
        int64_t i = tidx[k];
        int bx = t->ix[i], by = t->iy[i];
        for (int l = L; l >= 0; --l) {
            need[l][(int64_t)by * (1 << l) + bx] = 1;
            bx >>= 1;
            by >>= 1;
        }
    }
    (void)nside;
    return need;
}

static void free_needed(unsigned char **need, int L)
{
    if (!need)
        return;
    for (int l = 0; l <= L; ++l)
        free(need[l]);
    free(need);
}

/* ---------------------------------------------------------------- the serial FMM */

/* One FMM velocity evaluation (Fig. 1 stages 1-10) at the targets tidx (all particles if NULL; then nt = n).
 * dom = {x0, y0, S} or NULL for the default square. *npairs (if not NULL) receives the number of ordered
 * near-field pairs evaluated (i != j). Returns 0, -1 for a point outside an explicit square, -2 on OOM. */
/* parts: 1 = stage 9 (near field) only, 2 = stages 4-8 (far field) only, 3 = both (the FMM). */
int oracle_fmm_parts(int64_t n, const double *x, const double *y, const double *g, double sigma, int L, int p,
                     const double *dom, int64_t nt, const int64_t *tidx, double *u, double *v, int64_t *npairs,
                     int parts)
{
    if (npairs)
        *npairs = 0;
    if (n <= 0 || nt <= 0)
        return 0;
    tree_t t;
    int rc = tree_build(&t, n, x, y, L, p, dom);
    if (rc != 0) {
        tree_free(&t);
        return rc;
    }
    double *qre = calloc((size_t)(n ? n : 1), sizeof(double));
    double *qim = malloc(sizeof(double) * (size_t)(n ? n : 1));
    for (int64_t j = 0; j < n; ++j)
        qim[j] = -g[j] / (2.0 * ORACLE_PI); /* q_j = -i gamma_j / (2 pi) */
    unsigned char **need = mark_needed(&t, nt, tidx);
    if (parts & 2)
        upward_downward(&t, x, y, qre, qim, need);
    int nside = 1 << L;
    int64_t pairs = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : pairs)
    for (int64_t k = 0; k < nt; ++k) {
        int64_t i = tidx ? tidx[k] : k;
        int bx = t.ix[i], by = t.iy[i];
        /* stage 9: near field over the leaf and its neighbours, exact K_sigma */
        double su = 0.0, sv = 0.0;
        for (int ny = by - 1; ny <= by + 1 && (parts & 1); ++ny)
            for (int nx = bx - 1; nx <= bx + 1; ++nx) {
                if (nx < 0 || ny < 0 || nx >= nside || ny >= nside)
                    continue;
                int64_t b = (int64_t)ny * nside + nx;
                for (int64_t s = t.start[b]; s < t.start[b + 1]; ++s) {
                    int64_t j = t.list[s];
                    if (j == i)
                        continue;
                    double ku, kv;
                    oracle_kernel(x[i] - x[j], y[i] - y[j], sigma, &ku, &kv);
                    su += g[j] * ku;
                    sv += g[j] * kv;
                    pairs++;
                }
            }
        /* stage 8: far field from the leaf's local expansion */
        double w[2] = {0.0, 0.0};
        if (L >= 2 && (parts & 2)) {
            cplx c = box_centre(&t, L, bx, by);
            oracle_l2p(p, (double *)(t.loc[L] + ((int64_t)by * nside + bx) * p), x[i] - creal(c), y[i] - cimag(c), w);
        }
        /* stage 10: u - i v = w_far, plus the near field */
        u[k] = su + w[0];
        v[k] = sv - w[1];
    }
    if (npairs)
        *npairs = pairs;
    free_needed(need, L);
    free(qre);
    free(qim);
    tree_free(&t);
    return 0;
}

int oracle_fmm(int64_t n, const double *x, const double *y, const double *g, double sigma, int L, int p,
               const double *dom, int64_t nt, const int64_t *tidx, double *u, double *v, int64_t *npairs)
{
    return oracle_fmm_parts(n, x, y, g, sigma, L, p, dom, nt, tidx, u, v, npairs, 3);
}

/* The exact sum the FMM approximates (§2, last paragraph): K_sigma between particles whose leaves are
 * equal or adjacent, the point-vortex kernel between all other pairs. Same target convention as above. */
int oracle_split_direct(int64_t n, const double *x, const double *y, const double *g, double sigma, int L,
                        const double *dom, int64_t nt, const int64_t *tidx, double *u, double *v)
{
    if (n <= 0 || nt <= 0)
        return 0;
    tree_t t;
    int rc = tree_build(&t, n, x, y, L, 1, dom);
    if (rc != 0) {
        tree_free(&t);
        return rc;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < nt; ++k) {
        int64_t i = tidx ? tidx[k] : k;
        double su = 0.0, sv = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double ku, kv;
            if (abs(t.ix[i] - t.ix[j]) <= 1 && abs(t.iy[i] - t.iy[j]) <= 1)
                oracle_kernel(x[i] - x[j], y[i] - y[j], sigma, &ku, &kv);
            else
                point_vortex_kernel(x[i] - x[j], y[i] - y[j], &ku, &kv);
            su += g[j] * ku;
            sv += g[j] * kv;
        }
        u[k] = su;
        v[k] = sv;
    }
    tree_free(&t);
    return 0;
}

/* The regularised far-field correction (reading of §2, last paragraph, for leaves not much wider than sigma):
 * sum_j gamma_j (K_sigma - K_point)(z_i - z_j) over the particles j whose leaves are `rings` or fewer leaves
 * beyond the adjacent ones (Chebyshev leaf distance 2 .. 1 + rings), written out as the difference of the two
 * kernels. Added to the FMM, those pairs take the exact Eq. 6 kernel; the pairs still left to the point-vortex
 * kernel are at least (1 + rings) leaf widths w apart, so they miss at most exp(-(1 + rings)^2 w^2 / 2 sigma^2)
 * of theirs. Same target convention as oracle_split_direct. */
int oracle_far_tail(int64_t n, const double *x, const double *y, const double *g, double sigma, int L, int rings,
                    const double *dom, int64_t nt, const int64_t *tidx, double *u, double *v)
{
    if (n <= 0 || nt <= 0)
        return 0;
    tree_t t;
    int rc = tree_build(&t, n, x, y, L, 1, dom);
    if (rc != 0) {
        tree_free(&t);
        return rc;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < nt; ++k) {
        int64_t i = tidx ? tidx[k] : k;
        double su = 0.0, sv = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            int dx = abs(t.ix[i] - t.ix[j]), dy = abs(t.iy[i] - t.iy[j]);
            int dist = dx > dy ? dx : dy;
            if (dist < 2 || dist > 1 + rings)
                continue;
            double ku, kv, pu, pv;
            oracle_kernel(x[i] - x[j], y[i] - y[j], sigma, &ku, &kv);
            point_vortex_kernel(x[i] - x[j], y[i] - y[j], &pu, &pv);
            su += g[j] * (ku - pu);
            sv += g[j] * (kv - pv);
        }
        u[k] = su;
        v[k] = sv;
    }
    tree_free(&t);
    return 0;
}

/* ---------------------------------------------------------------- the adjoint of the FMM */

/* Derivatives of K_sigma at (a, b): J = [[dku/da, dku/db], [dkv/da, dkv/db]], with
 * K = (-b, a) f(s), s = a^2 + b^2, f(s) = (1 - exp(-s / 2 sigma^2)) / (2 pi s). */
static void kernel_jacobian(double a, double b, double sigma, double J[4])
{
    double s = a * a + b * b;
    if (s == 0.0) {
        J[0] = J[1] = J[2] = J[3] = 0.0;
        return;
    }
    double k = 1.0 / (2.0 * sigma * sigma);
    double om = -expm1(-s * k); /* 1 - e^{-ks} */
    double f = om / (2.0 * ORACLE_PI * s);
    /* f'(s) = (k e^{-ks} s - (1 - e^{-ks})) / (2 pi s^2) */
    double fp = (k * exp(-s * k) * s - om) / (2.0 * ORACLE_PI * s * s);
    J[0] = -b * fp * 2.0 * a;    /* d(-b f)/da */
    J[1] = -(f + 2.0 * b * b * fp); /* d(-b f)/db */
    J[2] = f + 2.0 * a * a * fp; /* d(a f)/da */
    J[3] = 2.0 * a * b * fp;     /* d(a f)/db */
}

/* Gradient of L = sum_i (gu_i u_i + gv_i v_i) with u, v from oracle_fmm (all particles, full tree), with
 * respect to gamma, x and y. The far field is back-propagated by applying the transpose of each stage in
 * reverse order (L2P^T, L2L^T, M2L^T, M2M^T, P2M^T); positions also act through the derivatives of the
 * P2M and L2P monomials. Any output pointer may be NULL. Returns as oracle_fmm. */
int oracle_fmm_adjoint(int64_t n, const double *x, const double *y, const double *g, double sigma, int L, int p,
                       const double *dom, const double *gu, const double *gv, double *dg, double *dx, double *dy)
{
    if (n <= 0)
        return 0;
    tree_t t;
    int rc = tree_build(&t, n, x, y, L, p, dom);
    if (rc != 0) {
        tree_free(&t);
        return rc;
    }
    size_t nn = (size_t)(n ? n : 1);
    double *qre = calloc(nn, sizeof(double)), *qim = malloc(nn * sizeof(double));
    double *rdg = calloc(nn, sizeof(double)), *rdx = calloc(nn, sizeof(double)), *rdy = calloc(nn, sizeof(double));
    for (int64_t j = 0; j < n; ++j)
        qim[j] = -g[j] / (2.0 * ORACLE_PI);
    int nside = 1 << L;

    /* near field: L_near = sum_i sum_{j near i, j != i} g_j (gu_i Ku + gv_i Kv)(z_i - z_j) */
    for (int64_t i = 0; i < n; ++i) {
        int bx = t.ix[i], by = t.iy[i];
        for (int ny = by - 1; ny <= by + 1; ++ny)
            for (int nx = bx - 1; nx <= bx + 1; ++nx) {
                if (nx < 0 || ny < 0 || nx >= nside || ny >= nside)
                    continue;
                int64_t b = (int64_t)ny * nside + nx;
                for (int64_t s = t.start[b]; s < t.start[b + 1]; ++s) {
                    int64_t j = t.list[s];
                    if (j == i)
                        continue;
                    double a = x[i] - x[j], bb = y[i] - y[j], ku, kv, J[4];
                    oracle_kernel(a, bb, sigma, &ku, &kv);
                    kernel_jacobian(a, bb, sigma, J);
                    rdg[j] += gu[i] * ku + gv[i] * kv;
                    double ga = g[j] * (gu[i] * J[0] + gv[i] * J[2]);
                    double gb = g[j] * (gu[i] * J[1] + gv[i] * J[3]);
                    rdx[i] += ga;
                    rdy[i] += gb;
                    rdx[j] -= ga;
                    rdy[j] -= gb;
                }
            }
    }

    if (L >= 2) {
        /* forward sweep for the local expansions b (needed for the target-side position derivative) */
        upward_downward(&t, x, y, qre, qim, NULL);
        int P = p;
        /* adjoint sweep: Bbar = adjoint of the local coefficients, Abar = adjoint of the multipoles */
        cplx **Bb = calloc((size_t)L + 1, sizeof(cplx *)), **Ab = calloc((size_t)L + 1, sizeof(cplx *));
        for (int l = 0; l <= L; ++l) {
            Bb[l] = calloc((size_t)P << (2 * l), sizeof(cplx));
            Ab[l] = calloc((size_t)P << (2 * l), sizeof(cplx));
        }
        /* dL = Re sum_i G_i dw_i with G_i = gu_i + i gv_i (since u = Re w, v = -Im w) */
        /* L2P^T: Bbar_l(leaf) += sum_i G_i (z_i - c)^l; also the target-side position derivative */
        for (int64_t i = 0; i < n; ++i) {
            int bx = t.ix[i], by = t.iy[i];
            int64_t b = (int64_t)by * nside + bx;
            cplx c = box_centre(&t, L, bx, by);
            cplx dz = (x[i] - creal(c)) + I * (y[i] - cimag(c));
            cplx G = gu[i] + I * gv[i];
            cplx pw = 1.0, dw = 0.0, pwm1 = 0.0;
            const cplx *bl = t.loc[L] + b * P;
            for (int l = 0; l < P; ++l) {
                Bb[L][b * P + l] += G * pw;
                if (l >= 1)
                    dw += (double)l * bl[l] * pwm1;
                pwm1 = pw;
                pw *= dz;
            }
            /* w depends on z_i through dz: dw/dx = w', dw/dy = i w' */
            rdx[i] += creal(G * dw);
            rdy[i] += creal(G * I * dw);
        }
        /* L2L^T: Bbar(parent)_l += sum_{k<=l} C(l, k) d^(l-k) Bbar(child)_k, levels L-1 .. 2 */
        for (int l = L - 1; l >= 2; --l) {
            int ns = 1 << l;
            for (int by = 0; by < ns; ++by)
                for (int bx = 0; bx < ns; ++bx) {
                    cplx cp = box_centre(&t, l, bx, by);
                    for (int cy = 0; cy < 2; ++cy)
                        for (int cx = 0; cx < 2; ++cx) {
                            int jx = 2 * bx + cx, jy = 2 * by + cy;
                            cplx d = box_centre(&t, l + 1, jx, jy) - cp;
                            const cplx *Bc = Bb[l + 1] + ((int64_t)jy * 2 * ns + jx) * P;
                            cplx *Bp = Bb[l] + ((int64_t)by * ns + bx) * P;
                            cplx dp[64];
                            dp[0] = 1.0;
                            for (int k = 1; k < P; ++k)
                                dp[k] = dp[k - 1] * d;
                            for (int k = 0; k < P; ++k)
                                for (int ll = k; ll < P; ++ll)
                                    Bp[ll] += binom(ll, k) * dp[ll - k] * Bc[k];
                        }
                }
        }
        /* M2L^T: Abar(S)_m += sum_l T_lm Bbar(T)_l for S in the list of T, T_lm = (-1)^(m+1) C(m+l, m) d^-(m+l+1) */
        for (int l = 2; l <= L; ++l) {
            int ns = 1 << l;
            for (int64_t b = 0; b < (int64_t)ns * ns; ++b) {
                int bx = (int)(b % ns), by = (int)(b / ns), sx[36], sy[36];
                cplx ct = box_centre(&t, l, bx, by);
                int cnt = interaction_list(l, bx, by, sx, sy);
                for (int s = 0; s < cnt; ++s) {
                    cplx d = box_centre(&t, l, sx[s], sy[s]) - ct, inv = 1.0 / d, ip[130];
                    ip[0] = 1.0;
                    for (int k = 1; k <= 2 * P; ++k)
                        ip[k] = ip[k - 1] * inv;
                    cplx *As = Ab[l] + ((int64_t)sy[s] * ns + sx[s]) * P;
                    const cplx *Bt = Bb[l] + b * P;
                    for (int m = 0; m < P; ++m) {
                        double sign = (m % 2 == 0) ? -1.0 : 1.0;
                        for (int ll = 0; ll < P; ++ll)
                            As[m] += (sign * binom(m + ll, m)) * ip[m + ll + 1] * Bt[ll];
                    }
                }
            }
        }
        /* M2M^T: Abar(child)_m += sum_{n>=m} C(n, m) d^(n-m) Abar(parent)_n, levels 2 .. L-1 */
        for (int l = 2; l < L; ++l) {
            int ns = 1 << l;
            for (int by = 0; by < ns; ++by)
                for (int bx = 0; bx < ns; ++bx) {
                    cplx cp = box_centre(&t, l, bx, by);
                    const cplx *Ap = Ab[l] + ((int64_t)by * ns + bx) * P;
                    for (int cy = 0; cy < 2; ++cy)
                        for (int cx = 0; cx < 2; ++cx) {
                            int jx = 2 * bx + cx, jy = 2 * by + cy;
                            cplx d = box_centre(&t, l + 1, jx, jy) - cp, dp[64];
                            dp[0] = 1.0;
                            for (int k = 1; k < P; ++k)
                                dp[k] = dp[k - 1] * d;
                            cplx *Ac = Ab[l + 1] + ((int64_t)jy * 2 * ns + jx) * P;
                            for (int m = 0; m < P; ++m)
                                for (int nn2 = m; nn2 < P; ++nn2)
                                    Ac[m] += binom(nn2, m) * dp[nn2 - m] * Ap[nn2];
                        }
                }
        }
        /* P2M^T: a_m = sum_j q_j (z_j - c)^m, q_j = -i gamma_j / (2 pi):
         * dL/dgamma_j += Re(sum_m Abar_m (-i / 2pi) dz^m); dL/dz_j via m q_j dz^(m-1) */
        for (int64_t j = 0; j < n; ++j) {
            int bx = t.ix[j], by = t.iy[j];
            int64_t b = (int64_t)by * nside + bx;
            cplx c = box_centre(&t, L, bx, by);
            cplx dz = (x[j] - creal(c)) + I * (y[j] - cimag(c));
            cplx q = qre[j] + I * qim[j];
            const cplx *A = Ab[L] + b * P;
            cplx pw = 1.0, pwm1 = 0.0, sg = 0.0, sd = 0.0;
            for (int m = 0; m < P; ++m) {
                sg += A[m] * pw;
                if (m >= 1)
                    sd += (double)m * A[m] * pwm1;
                pwm1 = pw;
                pw *= dz;
            }
            rdg[j] += creal(sg * (-I / (2.0 * ORACLE_PI)));
            rdx[j] += creal(q * sd);
            rdy[j] += creal(q * sd * I);
        }
        for (int l = 0; l <= L; ++l) {
            free(Bb[l]);
            free(Ab[l]);
        }
        free(Bb);
        free(Ab);
    }
    for (int64_t j = 0; j < n; ++j) {
        if (dg) dg[j] = rdg[j];
        if (dx) dx[j] = rdx[j];
        if (dy) dy[j] = rdy[j];
    }
    free(qre);
    free(qim);
    free(rdg);
    free(rdx);
    free(rdy);
    tree_free(&t);
    return 0;
}

/* ---------------------------------------------------------------- Eq. 3: advection of the particles */

/* In 2D ideal flow the vorticity is constant along particle paths (Eq. 3): the particles move with the local
 * velocity (Eq. 7, or the FMM approximation of it) and keep their circulation. The paper names no time
 * integrator; taken here: explicit Runge-Kutta of order 2 (the midpoint rule) or 4 (the classical scheme),
 *   stage s:   k_s = u(z + c_s dt k_{s-1}),     z <- z + dt sum_s b_s k_s,
 *   order 2:   c = (0, 1/2),          b = (0, 1)
 *   order 4:   c = (0, 1/2, 1/2, 1),  b = (1/6, 1/3, 1/3, 1/6)
 * with the stage velocity from the FMM (mode 0, at depth L and p terms, root square dom or the bounding-box
 * rule recomputed per stage) or from the direct sum (mode 1). x, y are updated in place.
 * Returns 0, -1 for a point outside an explicit square, -2 on allocation failure, -3 for bad arguments. */
int oracle_advect(int64_t n, double *x, double *y, const double *g, double sigma, int L, int p, const double *dom,
                  double dt, int nsteps, int order, int mode)
{
    static const double c2[2] = {0.0, 0.5}, b2[2] = {0.0, 1.0};
    static const double c4[4] = {0.0, 0.5, 0.5, 1.0}, b4[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    if ((order != 2 && order != 4) || (mode != 0 && mode != 1) || n < 0 || nsteps < 0)
        return -3;
    if (n == 0)
        return 0;
    const int S = order == 2 ? 2 : 4;
    const double *c = order == 2 ? c2 : c4, *b = order == 2 ? b2 : b4;
    double *tx = malloc((size_t)n * sizeof(double)), *ty = malloc((size_t)n * sizeof(double));
    double *ku = malloc((size_t)n * sizeof(double)), *kv = malloc((size_t)n * sizeof(double));
    double *au = malloc((size_t)n * sizeof(double)), *av = malloc((size_t)n * sizeof(double));
    int rc = 0;
    if (!tx || !ty || !ku || !kv || !au || !av)
        rc = -2;
    for (int step = 0; step < nsteps && rc == 0; ++step) {
        for (int64_t i = 0; i < n; ++i) {
            tx[i] = x[i];
            ty[i] = y[i];
            au[i] = 0.0;
            av[i] = 0.0;
        }
        for (int st = 0; st < S && rc == 0; ++st) {
            if (mode == 1) {
                oracle_direct(n, tx, ty, g, sigma, n, NULL, ku, kv);
            } else {
                int64_t npairs = 0;
                rc = oracle_fmm(n, tx, ty, g, sigma, L, p, dom, n, NULL, ku, kv, &npairs);
                if (rc != 0)
                    break;
            }
            for (int64_t i = 0; i < n; ++i) {
                au[i] += b[st] * ku[i];
                av[i] += b[st] * kv[i];
                if (st + 1 < S) {
                    tx[i] = x[i] + c[st + 1] * dt * ku[i];
                    ty[i] = y[i] + c[st + 1] * dt * kv[i];
                }
            }
        }
        if (rc == 0)
            for (int64_t i = 0; i < n; ++i) {
                x[i] += dt * au[i];
                y[i] += dt * av[i];
            }
    }
    free(tx);
    free(ty);
    free(ku);
    free(kv);
    free(au);
    free(av);
    return rc;
}

/* ================================================================ adaptive quadtree (§5: uneven densities)
 *
 * The paper's tree is uniform; its closing section names uneven particle distributions as the next step.
 * This is the standard adaptive quadtree of Carrier, Greengard and Rokhlin written out plainly:
 *   - a box is split into its four children while it holds more than B particles and its level is below
 *     Lmax; the boxes are the squares of the uniform tree (level l, column bx, row by), so a particle's box
 *     at level l is its depth-Lmax leaf coordinate shifted right by Lmax - l;
 *   - two boxes are adjacent when their closed squares touch or overlap;
 *   - U(a), leaf a: every leaf adjacent to a (a included)          -> exact K_sigma (stage 9)
 *   - V(a): boxes at a's level whose parents are adjacent to a's parent, not adjacent to a  -> M2L (stage 6)
 *   - W(a), leaf a: boxes below colleagues of a (same-level boxes adjacent to a) whose parent is adjacent
 *     to a but which are not adjacent to a                          -> multipole evaluated at a's particles
 *   - X(a): the boxes c with a in W(c) (all leaves)                -> local expansion of c's particles
 * Every list is found here by testing the definition on every pair of boxes (quadratic in the box count).
 * Locals exist on levels >= 2 (levels 0 and 1 have no well separated pairs) and multipoles likewise. */

typedef struct {
    int l, bx, by;
    int parent;
    int child[4]; /* -1 for a leaf */
    int64_t p0, np; /* particles ord[p0 .. p0 + np) */
    int64_t lo[2], hi[2]; /* closed range of depth-Lmax cells, x and y */
} abox_t;

typedef struct {
    int Lmax, B, nbox, cap;
    double x0, y0, S;
    abox_t *box;
    int64_t *ord;  /* particle indices grouped by box (children are sub-ranges of the parent) */
    int32_t *ix, *iy;
} atree_t;

static void atree_free(atree_t *t)
{
    free(t->box);
    free(t->ord);
    free(t->ix);
    free(t->iy);
}

static int atree_add(atree_t *t, int l, int bx, int by, int parent, int64_t p0, int64_t np)
{
    if (t->nbox == t->cap) {
        int nc = t->cap ? 2 * t->cap : 64;
        abox_t *nb = realloc(t->box, sizeof(abox_t) * (size_t)nc);
        if (!nb)
            return -1;
        t->box = nb;
        t->cap = nc;
    }
    abox_t *b = &t->box[t->nbox];
    b->l = l;
    b->bx = bx;
    b->by = by;
    b->parent = parent;
    b->child[0] = b->child[1] = b->child[2] = b->child[3] = -1;
    b->p0 = p0;
    b->np = np;
    int sh = t->Lmax - l;
    b->lo[0] = (int64_t)bx << sh;
    b->hi[0] = (((int64_t)bx + 1) << sh) - 1;
    b->lo[1] = (int64_t)by << sh;
    b->hi[1] = (((int64_t)by + 1) << sh) - 1;
    return t->nbox++;
}

/* Builds the tree breadth first, so boxes come in non-decreasing level order and a parent precedes its
 * children. Particles keep the input order inside every box. */
static int atree_build(atree_t *t, int64_t n, const double *x, const double *y, int Lmax, int B, const double *dom)
{
    memset(t, 0, sizeof(*t));
    t->Lmax = Lmax;
    t->B = B;
    double d[3];
    if (dom) {
        d[0] = dom[0];
        d[1] = dom[1];
        d[2] = dom[2];
    } else {
        oracle_default_domain(n, x, y, d);
    }
    t->x0 = d[0];
    t->y0 = d[1];
    t->S = d[2];
    size_t nn = (size_t)(n ? n : 1);
    t->ix = malloc(sizeof(int32_t) * nn);
    t->iy = malloc(sizeof(int32_t) * nn);
    t->ord = malloc(sizeof(int64_t) * nn);
    int64_t *tmp = malloc(sizeof(int64_t) * nn);
    if (!t->ix || !t->iy || !t->ord || !tmp) {
        free(tmp);
        return -2;
    }
    if (oracle_leaf_coords(n, x, y, Lmax, d, dom != NULL, t->ix, t->iy) != 0) {
        free(tmp);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i)
        t->ord[i] = i;
    if (atree_add(t, 0, 0, 0, -1, 0, n) < 0) {
        free(tmp);
        return -2;
    }
    for (int k = 0; k < t->nbox; ++k) {
        abox_t b = t->box[k];
        if (b.np <= B || b.l >= Lmax)
            continue;
        /* stable partition of the box's particles into its children (child index cy * 2 + cx) */
        int sh = Lmax - (b.l + 1);
        int64_t cnt[4] = {0, 0, 0, 0};
        for (int64_t e = 0; e < b.np; ++e) {
            int64_t i = t->ord[b.p0 + e];
            int c = (((t->iy[i] >> sh) & 1) << 1) | ((t->ix[i] >> sh) & 1);
            cnt[c]++;
        }
        int64_t off[4] = {0, cnt[0], cnt[0] + cnt[1], cnt[0] + cnt[1] + cnt[2]};
        int64_t fill[4] = {off[0], off[1], off[2], off[3]};
        for (int64_t e = 0; e < b.np; ++e) {
            int64_t i = t->ord[b.p0 + e];
            int c = (((t->iy[i] >> sh) & 1) << 1) | ((t->ix[i] >> sh) & 1);
            tmp[fill[c]++] = i;
        }
        memcpy(t->ord + b.p0, tmp, sizeof(int64_t) * (size_t)b.np);
        for (int c = 0; c < 4; ++c) {
            int id = atree_add(t, b.l + 1, 2 * b.bx + (c & 1), 2 * b.by + (c >> 1), k, b.p0 + off[c], cnt[c]);
            if (id < 0) {
                free(tmp);
                return -2;
            }
            t->box[k].child[c] = id;
        }
    }
    free(tmp);
    return 0;
}

static int a_adjacent(const abox_t *a, const abox_t *c)
{
    return a->lo[0] <= c->hi[0] + 1 && c->lo[0] <= a->hi[0] + 1 && a->lo[1] <= c->hi[1] + 1 &&
           c->lo[1] <= a->hi[1] + 1;
}

static int a_is_leaf(const abox_t *a) { return a->child[0] < 0; }

static int in_U(const atree_t *t, int a, int c)
{
    const abox_t *A = &t->box[a], *C = &t->box[c];
    return a_is_leaf(A) && a_is_leaf(C) && a_adjacent(A, C);
}

static int in_V(const atree_t *t, int a, int c)
{
    const abox_t *A = &t->box[a], *C = &t->box[c];
    if (A->l < 2 || C->l != A->l || a_adjacent(A, C))
        return 0;
    return a_adjacent(&t->box[A->parent], &t->box[C->parent]);
}

static int in_W(const atree_t *t, int a, int c)
{
    const abox_t *A = &t->box[a], *C = &t->box[c];
    if (!a_is_leaf(A) || C->l <= A->l || a_adjacent(A, C) || !a_adjacent(A, &t->box[C->parent]))
        return 0;
    int anc = c; /* c's ancestor at a's level must be a colleague of a */
    while (t->box[anc].l > A->l)
        anc = t->box[anc].parent;
    return a_adjacent(A, &t->box[anc]);
}

static int in_X(const atree_t *t, int a, int c) { return in_W(t, c, a); }

/* Structural check of the four lists: for every ordered pair of leaves (a, b) the number of ways the
 * pair's interaction is delivered -- b in U(a); beta in V(alpha); beta in W(a); b in X(alpha), with alpha
 * ranging over a and its ancestors and beta over b and its ancestors -- must be exactly one. Returns the
 * number of leaf pairs where it is not; sizes = {boxes, leaves, sum |U|, sum |V|, sum |W|, sum |X|,
 * max |V|, deepest leaf level, ordered particle pairs (i, j != i) whose leaves are in each other's U list}. */
int oracle_adaptive_lists_check(int64_t n, const double *x, const double *y, int Lmax, int B, const double *dom,
                                int64_t *sizes)
{
    atree_t t;
    int rc = atree_build(&t, n, x, y, Lmax, B, dom);
    if (rc != 0) {
        atree_free(&t);
        return rc;
    }
    int nb = t.nbox;
    int64_t su = 0, sv = 0, sw = 0, sx = 0, nleaf = 0, maxv = 0, deep = 0, pairs = 0;
    for (int a = 0; a < nb; ++a) {
        int64_t va = 0;
        for (int c = 0; c < nb; ++c) {
            su += in_U(&t, a, c);
            if (in_U(&t, a, c))
                pairs += t.box[a].np * t.box[c].np;
            va += in_V(&t, a, c);
            sw += in_W(&t, a, c);
            sx += in_X(&t, a, c);
        }
        sv += va;
        if (va > maxv)
            maxv = va;
        if (a_is_leaf(&t.box[a])) {
            nleaf++;
            if (t.box[a].l > deep)
                deep = t.box[a].l;
        }
    }
    int bad = 0;
    for (int a = 0; a < nb; ++a) {
        if (!a_is_leaf(&t.box[a]))
            continue;
        for (int b = 0; b < nb; ++b) {
            if (!a_is_leaf(&t.box[b]))
                continue;
            int count = in_U(&t, a, b);
            for (int al = a; al >= 0; al = t.box[al].parent) {
                for (int be = b; be >= 0; be = t.box[be].parent)
                    count += in_V(&t, al, be);
                count += in_X(&t, al, b);
            }
            for (int be = b; be >= 0; be = t.box[be].parent)
                count += in_W(&t, a, be);
            bad += count != 1;
        }
    }
    if (sizes) {
        int64_t s[9] = {nb, nleaf, su, sv, sw, sx, maxv, deep, pairs - n};
        memcpy(sizes, s, sizeof s);
    }
    atree_free(&t);
    return bad;
}

/* X list operator (P2L): the local expansion about c of point charges q_j at z_j outside its disc, from
 * 1/(z - z_j) = -sum_l (z - c)^l / (z_j - c)^(l+1):   b_l += -sum_j q_j / (z_j - c)^(l+1).   Accumulates. */
void oracle_p2l(int64_t np, const double *x, const double *y, const double *qre, const double *qim, double cx,
                double cy, int p, double *b_out)
{
    cplx *b = (cplx *)b_out;
    for (int64_t j = 0; j < np; ++j) {
        cplx q = qre[j] + I * qim[j];
        cplx inv = 1.0 / ((x[j] - cx) + I * (y[j] - cy)), pw = inv;
        for (int l = 0; l < p; ++l) {
            b[l] -= q * pw;
            pw *= inv;
        }
    }
}

static cplx a_centre(const atree_t *t, const abox_t *b)
{
    double w = t->S / ldexp(1.0, b->l);
    return (t->x0 + (b->bx + 0.5) * w) + I * (t->y0 + (b->by + 0.5) * w);
}

/* The adaptive FMM: P2M at the leaves, M2M up, then level by level M2L (V), P2L (X) and L2L down; at every
 * leaf L2P, the W multipoles evaluated at its particles, and the exact K_sigma over U. parts: 1 near, 2 far,
 * 3 both. Output in input order. Returns 0, -1 for a point outside an explicit square, -2 on allocation
 * failure. */
int oracle_adaptive_fmm(int64_t n, const double *x, const double *y, const double *g, double sigma, int Lmax,
                        int B, int p, const double *dom, double *u, double *v, int parts)
{
    if (n <= 0)
        return 0;
    atree_t t;
    int rc = atree_build(&t, n, x, y, Lmax, B, dom);
    if (rc != 0) {
        atree_free(&t);
        return rc;
    }
    int nb = t.nbox;
    cplx *mp = calloc((size_t)nb * (size_t)p, sizeof(cplx)), *loc = calloc((size_t)nb * (size_t)p, sizeof(cplx));
    double *qre = calloc((size_t)n, sizeof(double)), *qim = malloc(sizeof(double) * (size_t)n);
    double *bx = malloc(sizeof(double) * (size_t)n), *by = malloc(sizeof(double) * (size_t)n);
    if (!mp || !loc || !qre || !qim || !bx || !by) {
        rc = -2;
        goto done;
    }
    /* particles in box order, so a box's particles are one contiguous run */
    for (int64_t e = 0; e < n; ++e) {
        int64_t i = t.ord[e];
        bx[e] = x[i];
        by[e] = y[i];
        qim[e] = -g[i] / (2.0 * ORACLE_PI); /* q = -i gamma / 2 pi */
    }
    /* upward: P2M at leaves on levels >= 2, then M2M from the deepest level up (reverse breadth-first order) */
    for (int k = nb - 1; k >= 0; --k) {
        abox_t *b = &t.box[k];
        if (b->l < 2)
            continue;
        cplx c = a_centre(&t, b);
        if (a_is_leaf(b)) {
            oracle_p2m(b->np, bx + b->p0, by + b->p0, qre + b->p0, qim + b->p0, creal(c), cimag(c), p,
                       (double *)(mp + (size_t)k * p));
        } else {
            for (int q = 0; q < 4; ++q) {
                int ch = b->child[q];
                cplx d = a_centre(&t, &t.box[ch]) - c;
                oracle_m2m(p, (const double *)(mp + (size_t)ch * p), creal(d), cimag(d), (double *)(mp + (size_t)k * p));
            }
        }
    }
    /* downward in breadth-first order: a parent's local is complete before its children read it */
    for (int k = 0; k < nb; ++k) {
        abox_t *b = &t.box[k];
        if (b->l < 2)
            continue;
        cplx c = a_centre(&t, b);
        double *lk = (double *)(loc + (size_t)k * p);
        if (b->l >= 3) {
            cplx d = c - a_centre(&t, &t.box[b->parent]);
            oracle_l2l(p, (const double *)(loc + (size_t)b->parent * p), creal(d), cimag(d), lk);
        }
        for (int s = 0; s < nb; ++s) {
            if (in_V(&t, k, s)) {
                cplx d = a_centre(&t, &t.box[s]) - c;
                oracle_m2l(p, (const double *)(mp + (size_t)s * p), creal(d), cimag(d), lk);
            } else if (in_X(&t, k, s)) {
                const abox_t *S = &t.box[s];
                oracle_p2l(S->np, bx + S->p0, by + S->p0, qre + S->p0, qim + S->p0, creal(c), cimag(c), p, lk);
            }
        }
    }
    /* leaves: far (L2P + W) and near (U) */
    for (int k = 0; k < nb; ++k) {
        abox_t *b = &t.box[k];
        if (!a_is_leaf(b) || b->np == 0)
            continue;
        cplx c = a_centre(&t, b);
        for (int64_t e = b->p0; e < b->p0 + b->np; ++e) {
            int64_t i = t.ord[e];
            double su = 0.0, sv = 0.0;
            if (parts & 2) {
                cplx w = 0.0;
                double wv[2];
                if (b->l >= 2) {
                    oracle_l2p(p, (const double *)(loc + (size_t)k * p), bx[e] - creal(c), by[e] - cimag(c), wv);
                    w += wv[0] + I * wv[1];
                }
                for (int s = 0; s < nb; ++s)
                    if (in_W(&t, k, s)) {
                        cplx cs = a_centre(&t, &t.box[s]);
                        oracle_multipole_eval(p, (const double *)(mp + (size_t)s * p), bx[e] - creal(cs),
                                              by[e] - cimag(cs), wv);
                        w += wv[0] + I * wv[1];
                    }
                su += creal(w);
                sv -= cimag(w);
            }
            if (parts & 1)
                for (int s = 0; s < nb; ++s) {
                    if (!in_U(&t, k, s))
                        continue;
                    const abox_t *S = &t.box[s];
                    for (int64_t f = S->p0; f < S->p0 + S->np; ++f) {
                        if (f == e)
                            continue;
                        double ku, kv;
                        oracle_kernel(bx[e] - bx[f], by[e] - by[f], sigma, &ku, &kv);
                        int64_t j = t.ord[f];
                        su += g[j] * ku;
                        sv += g[j] * kv;
                    }
                }
            u[i] = su;
            v[i] = sv;
        }
    }
done:
    free(mp);
    free(loc);
    free(qre);
    free(qim);
    free(bx);
    free(by);
    atree_free(&t);
    return rc;
}

/* The exact sum the adaptive FMM approaches as p grows: K_sigma between particles whose leaves are
 * adjacent (or equal), the point-vortex kernel between all other pairs. Output in input order. */
int oracle_adaptive_split_direct(int64_t n, const double *x, const double *y, const double *g, double sigma,
                                 int Lmax, int B, const double *dom, double *u, double *v)
{
    if (n <= 0)
        return 0;
    atree_t t;
    int rc = atree_build(&t, n, x, y, Lmax, B, dom);
    int *leaf = malloc(sizeof(int) * (size_t)n);
    if (rc != 0 || !leaf) {
        free(leaf);
        atree_free(&t);
        return rc ? rc : -2;
    }
    for (int k = 0; k < t.nbox; ++k)
        if (a_is_leaf(&t.box[k]))
            for (int64_t e = t.box[k].p0; e < t.box[k].p0 + t.box[k].np; ++e)
                leaf[t.ord[e]] = k;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double su = 0.0, sv = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double ku, kv;
            if (a_adjacent(&t.box[leaf[i]], &t.box[leaf[j]]))
                oracle_kernel(x[i] - x[j], y[i] - y[j], sigma, &ku, &kv);
            else
                point_vortex_kernel(x[i] - x[j], y[i] - y[j], &ku, &kv);
            su += g[j] * ku;
            sv += g[j] * kv;
        }
        u[i] = su;
        v[i] = sv;
    }
    free(leaf);
    atree_free(&t);
    return 0;
}
