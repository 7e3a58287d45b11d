// fmm_internal.cuh -- data layout and kernel entry points shared by the library's translation units.
//
// Layout in HBM (one workspace allocation per handle, carved into 256-byte aligned arrays):
//   particles in the caller's order : key[n] (global leaf of each particle)
//   particles in leaf order         : perm[n] (sorted position -> caller index), sleaf[n] (global leaf),
//                                     FP64 form: sx, sy, sg (absolute coordinates, circulation),
//                                     precision form: leaf-relative split coordinates (hi + lo floats) in
//                                     units of w_L / s (see SysDev::s_unit), each value stored twice so that
//                                     one 64-bit register pair feeds a packed f32x2 operation on two targets:
//                                     eh = (xh, xh, yh, yh), el = (xl, xl, yl, yl), eg = (g, g, -g, -g)
//   leaves                          : cnt[nleaf] (histogram), start[nleaf + 1] (first sorted position)
//   boxes (levels 2..L of every system, row-major per level): bcount[nbox] (particles in the box),
//                                     multipoles and locals, p complex coefficients per box, FP64 and/or FP32
// Expansions are stored radius-scaled so every translation matrix is level independent:
//   multipole  a~_m = sum_j q'_j zeta_j^m, zeta = (z - c) / w_l, q' = -i gamma (the 1/2pi is applied at the end)
//   local      b^_l = w_l^(l+1) b_l, so that the far field at z is (1 / (2 pi w_L)) sum_l b^_l zeta^l.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define FMM_MAXL 12
#define FMM_PMAX 32
#define FMM_MAXSYS 4096
#define FMM_NOFF 49  // M2L offsets (dx, dy) in [-3, 3]^2, indexed (dy + 3) * 7 + (dx + 3)

// device status bits (OR-ed into the status word)
#define FMM_DEV_OUTSIDE 1u
#define FMM_DEV_BOUNDS 2u
#define FMM_DEV_TIMEOUT 4u

// Largest s (leaf width w_L in units of sqrt(2 / log2 e) sigma) at which the near field keeps one float per
// coordinate in the leaf frame: the rounding of a source coordinate, |x| <= 3 s / 2, relative to sigma grows
// with s; at s = 13.6 (64 uniform particles per leaf, sigma = h / 2) it costs 7e-8 relative L2 of the near
// field, so up to s = 32 it stays below 2e-7. Wider leaves take the hi + lo split form.
#define P2P_SPLIT_S 32.0f

namespace fmm {

// Per-system descriptor, device resident (one per system of a batch; a plain evaluation is a batch of one).
struct SysDev {
    int64_t p0, np;                 // particle range [p0, p0 + np) in caller and in sorted order
    int64_t leaf0;                  // first global leaf of this system
    int64_t box0[FMM_MAXL + 1];     // first global box of level l (2 <= l <= depth), else -1
    double x0, y0, S;               // root square (explicit, or written by the bounding-box kernel)
    double sigma;
    int depth;
    int explicit_domain;
    int pad[2];
    // derived once per evaluation by k_domain_finalize (so no per-particle kernel divides in FP64)
    double scale;                   // 2^L / S
    double xe, ye;                  // x0 + S, y0 + S
    double wl;                      // S / 2^L, leaf width
    double far_scale;               // 1 / (2 pi w_L)
    float s_unit;                   // precision form length unit: s = fl32(sqrt(log2(e) w_L^2 / 2 sigma^2)) per leaf
                                    // width, so that exp(-r^2 / 2 sigma^2) = 2^-(r')^2 with r' = s r / w_L
    float inv_s;                    // 1 / s
    float snear;                    // s / (2 pi w_L): scale of the near-field sum in these units
    float pad_f;
    double iu;                      // adaptive tree's precision form: 1 / u, u = sigma sqrt(2 / log2 e)
    // boundary bands of the precision form's near field: a particle whose leaf-relative position zeta (in leaf
    // widths, |zeta| <= 1/2) has |zeta_x| * 2^52 > fbnd lies within delta = sigma (1 + 2^-8) of its leaf's left or
    // right side (likewise y); bnd_ok = 0 when the bands would overlap (leaf narrower than 2 delta)
    long long fbnd;
    int bnd_ok;
    int pad_b;
};

// Per-level work lists for the tree sweeps, computed on the host and passed by value. The systems that have
// level l (depth >= l) are sys_list[first_at[l] .. first_at[l] + nsys_at[l]) (device array, ascending).
struct LevelInfo {
    int nsys_at[FMM_MAXL + 2];
    int first_at[FMM_MAXL + 2];
    int64_t m2l_item0[FMM_MAXL + 2];  // prefix over levels 2..maxdepth of (systems at l) * 4^l boxes
    int maxdepth;
    int mindepth2;                     // smallest depth >= 2 among the systems (0 if none)
};

// Read-only tables that depend on p only.
struct Tables {
    double2 *m2m64, *l2l64;   // [4][PMAX][PMAX]  (child position c = cy * 2 + cx; [c][input][output])
    float2 *m2m32, *l2l32;
    double2 *rho64;           // [FMM_NOFF][2 PMAX + 2]  (1/delta)^k
    float2 *rho32;
    double *binom64;          // [PMAX][PMAX]  C(m + l, m)
    float *binom32;
    unsigned char *m2l_tc;    // tensor-core M2L operands B_delta (m2l_tc.cu)
};

// One particle's FP64 inputs in the caller's order, written by the key kernel so that the leaf-order kernel's
// random gather reads one 32-byte sector per particle instead of three.
struct __align__(32) Rec64 {
    double x, y, g, pad;
};

struct Work {
    int n;
    int nleaf;
    int64_t nbox;
    int p;
    int mixed;
    int coarse_level;         // levels <= this run in FP64 in the precision form
    int m2l_tc;               // FP32 M2L levels on the tensor cores (1) or on the CUDA cores (0)
    float2 *far32;            // [n] leaf order: FP32 far field (L2P) of the precision form, or null (fused)
    int nf_stride;            // float2 stride of near32 / far32: 2 where they interleave (near, far) per particle so
                              // that the final sum gathers one 16-byte record, else 1
    int *iperm;               // [n] caller index -> leaf-order position (inverse of perm)
    unsigned int *status_host;  // page-locked copy of *status written by the final sum kernel, or null
    float2 *nearp;            // [4][n] leaf order: symmetric near field, reactions from the leaf at -P2P
                              // forward offset d (d = 0..3: (1,0), (1,1), (0,1), (-1,1)), or null
    int p2p_all_plain;        // host knows every system takes one-float near-field coordinates
    int p2p_sym;              // this evaluation's near field is the symmetric kernel (nearp holds reactions)
    int p2p_rows;             // this evaluation's near field comes per source row (nearp[0..2] hold the parts)
    int nsys;
    int maxdepth;
    int morton;               // leaf keys in Morton order (adaptive tree) instead of row-major
    int adapt_cap;            // adaptive tree: a box holding more than this many particles is split (0: uniform)
    int ad_mixed;             // adaptive tree in the precision form (FP32 expansions and near field)
    int *ad_list;             // adaptive tree: Morton indices of the existing boxes of level l at [box0[l], ...)
    int *ad_cnt;              // [FMM_MAXL + 2] adaptive tree: number of existing boxes per level
    // arrays
    int *key, *slot, *cnt, *start, *scan_tmp, *perm, *sleaf;
    int2 *tmp;                // [n] leaf order before the in-leaf ranking: (caller index, leaf) at the arrival slot;
                              // the uniform precision form stores (caller index, boundary class) instead
    int *cls_off;             // uniform precision form: [nleaf][8] first sorted position of boundary classes 1..8
                              // of each leaf (class 0 starts at start[leaf]), or null
    unsigned char *cls8;      // with cls_off: [n] caller order, boundary class of each particle (key kernel)
    int2 *bkt;                // uniform tree: [nleaf][bkt_cap] each leaf's entries (caller index, class) at their
                              // arrival slots, written by the key kernel; cnt[nleaf] != 0 marks a leaf that
                              // overflowed, and the evaluation then takes the scatter into tmp instead; or null
    int bkt_cap;
    int *big, *big_cnt;       // leaves too large for the per-position ranking, and their number
    double *sx, *sy, *sg;
    float4 *eh, *el, *eg;     // precision form, leaf order: (xh, xh, yh, yh), (xl, xl, yl, yl), (g, g, -g, -g)
    float4 *pos4u;            // precision form, caller order (made while binning), two float4 per particle in one
                              // 32-byte sector: (xh, yh, xl, yl), (gamma, 0, 0, 0)
    Rec64 *rec64;             // FP64 form and adaptive tree, caller order: (x, y, gamma)
    double2 *near64;
    float2 *near32;
    int *bcount;
    double2 *M64, *L64;
    float2 *M32, *L32;
    float4 *mtc;              // precision form, levels 2 .. 7: the tensor-core M2L's window source layout (TF32 hi and
                              // lo planes of the multipoles per class, m2l_tc.cu), or null
    float2 *m2l_part;         // with mtc: the tensor-core M2L's partial locals, four per box (one per source class)
    int *m2l_cnt;             // with mtc: completion counters of its tiles
    // adjoint extras
    double *sgu, *sgv;
    double2 *AM64, *AL64;     // expansions of the adjoint charges G = gu + i gv
    double2 *wprime;          // derivative of the forward far field at each sorted particle
    unsigned long long *minmax;  // [4 * nsys] bounding-box reduction
    unsigned int *status;
    unsigned long long *pair_count;
    double *adj_far;          // [3 n] far-field part of (dgamma, dx, dy) in leaf order
    SysDev *sys;
    int *sys_list;
    LevelInfo lv;
};

// Morton index of cell (x, y): bits of x on the even positions, bits of y on the odd ones (x, y < 2^16).
__host__ __device__ inline unsigned spread1(unsigned v)
{
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
__host__ __device__ inline unsigned morton2(unsigned x, unsigned y) { return spread1(x) | (spread1(y) << 1); }
__host__ __device__ inline unsigned compact1(unsigned v)  // inverse of spread1 on the even bits
{
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0f0f0f0fu;
    v = (v | (v >> 4)) & 0x00ff00ffu;
    v = (v | (v >> 8)) & 0x0000ffffu;
    return v;
}

// System of the sidx-th system that has level l.
__device__ __forceinline__ int sys_at_level(const Work &w, int l, int sidx)
{
    return w.sys_list[w.lv.first_at[l] + sidx];
}

// Level precision in the precision form: FP64 for l <= coarse_level.
__host__ __device__ inline bool level_fp64(const Work &w, int l) { return !w.mixed || l <= w.coarse_level; }

// System of a particle / leaf: the last system whose first particle / leaf is <= the index (systems are
// contiguous and ordered; empty systems share their first index with the next system).
__device__ inline int find_sys_by_particle(const SysDev *sys, int nsys, int64_t i)
{
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sys[mid].p0 <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ inline int find_sys_by_leaf(const SysDev *sys, int nsys, int64_t leaf)
{
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sys[mid].leaf0 <= leaf)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ---- launchers (each returns the number of kernels launched) ----
int launch_bbox(const Work &w, const double *x, const double *y, cudaStream_t s);
int launch_domain_finalize(const Work &w, cudaStream_t s);
__host__ __device__ void derive_constants(SysDev &d);  // binning.cu: per-system constants from square, depth, sigma
int launch_keys(const Work &w, const double *x, const double *y, const double *g, cudaStream_t s);
int launch_scan(const Work &w, cudaStream_t s);  // cnt -> start
int launch_scatter_sort(const Work &w, cudaStream_t s);
int launch_gather(const Work &w, const double *x, const double *y, const double *g, const double *gu,
                  const double *gv, cudaStream_t s);
int launch_pair_count(const Work &w, cudaStream_t s);
int launch_p2m(const Work &w, const Tables &t, int adjoint_charges, cudaStream_t s);
int launch_m2m(const Work &w, const Tables &t, int level, int adjoint_charges, cudaStream_t s, int prio);
int launch_m2l(const Work &w, const Tables &t, int adjoint_charges, cudaStream_t s, int prio);
int launch_l2l(const Work &w, const Tables &t, int level, int adjoint_charges, cudaStream_t s, int prio);
int launch_wait_timeout_selftest(const Work &w, int polls, cudaStream_t s);  // one bounded wait that runs out
int launch_p2p(const Work &w, int threads, int kt, cudaStream_t s);  // threads 32: 1 leaf per block, 64: 2,
                                                                     // 128: symmetric, 192: per source row
int launch_rk_stage(int64_t n, double *x, double *y, double *tx, double *ty, const double *u, const double *v,
                    double *au, double *av, double b, double c_next, double dt, int first, int last, cudaStream_t s);
// Sharded evaluations: level l's multipoles (double2, 4^l * p, boxes row-major) and box counts of the first system
// out of / into the tree.
int launch_level_export(const Work &w, int l, double2 *dst, long long *cnt, cudaStream_t s);
int launch_level_import(const Work &w, int l, const double2 *src, const long long *cnt, cudaStream_t s);
int launch_l2p(const Work &w, cudaStream_t s);  // precision form with far32: far field into far32 (stage 8)
int launch_combine(const Work &w, int use_near, int use_far, double *u, double *v, cudaStream_t s);
int launch_adjoint_far(const Work &w, cudaStream_t s);  // far part of (dgamma, dx, dy) into adj_far
int launch_adjoint_combine(const Work &w, double *dg, double *dx, double *dy, cudaStream_t s);  // adds it
int launch_adjoint_p2p(const Work &w, double *dg, double *dx, double *dy, int fp32, cudaStream_t s);
// Regularised far-field correction of the uniform tree (far_tail.cu): adds (K_sigma - K_point) over the sources whose
// leaves are 2 .. 1 + rings leaves from each target's leaf to the near field (after the near-field kernel).
int launch_far_tail(const Work &w, int rings, cudaStream_t s);

// Adaptive tree (adaptive.cu, single system, keys in Morton order, sorted FP64 particles and, in the precision form,
// the split records written by the leaf-order kernel). Side stream: the upward pass (box lists, P2L over X, P2M,
// M2M), then the downward pass (per level L2L + M2L over V). Main stream, after the sweep, one kernel per target:
// a walk of U and W, exact K_sigma over U if use_near, the multipoles of W and the leaf's local if use_far,
// written in the caller's order.
int launch_adaptive_up(const Work &w, const Tables &t, cudaStream_t s);
int launch_adaptive_down(const Work &w, const Tables &t, cudaStream_t s);
int launch_adaptive_near(const Work &w, unsigned long long *pairs, int use_near, int use_far, double *u, double *v,
                         cudaStream_t s);

void build_tables_host(int p, double2 *m2m, double2 *l2l, double2 *rho, double *binom);

// Tensor-core M2L (m2l_tc.cu): its operand table for p (the 40 offsets' translation matrices, TF32 hi and lo),
// the table's size, the p and levels it covers, the per-device kernel attributes (before any stream capture;
// 0 on success) and the launch over levels l_lo .. l_hi (<= m2l_tc_max_level()); returns the launches made.
size_t m2l_tc_table_bytes(int p);
size_t m2l_tc_layout_bytes(const LevelInfo &lv, int p);  // Work::mtc for these levels and p (0: not used)
size_t m2l_tc_part_bytes(const LevelInfo &lv, int p);    // Work::m2l_part
size_t m2l_tc_count_bytes(const LevelInfo &lv, int p);   // Work::m2l_cnt
void build_m2l_tc_table_host(int p, unsigned char *out);
bool m2l_tc_supported(int p);
int m2l_tc_max_level();
int prepare_m2l_tc();
int prepare_p2p();  // near-field kernel attributes, once per device before any stream capture; 0 on success
int launch_m2l_tc(const Work &w, const Tables &t, int l_lo, int l_hi, cudaStream_t s);
int upload_m2l_constants(cudaStream_t s);  // once per device, before any stream capture; 0 on success

}  // namespace fmm
