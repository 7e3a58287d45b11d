// capi.cu -- the C ABI declared in include/fmm2d.h: handle, workspace, the two-stream stage DAG of Fig. 1,
// CUDA-graph capture and replay, device status, timing, and the autotuner.
//
// Schedule of one evaluation (Fig. 1; {4,5,6,7} has no dependency on {9}):
//   caller stream : [1-2] bbox, keys, scan, scatter, in-leaf order, gather --fork-->  [9] P2P  --join--> [8+10]
//   side stream   :                                                          [4] P2M [5] M2M [6] M2L [7] L2L
// The side stream has the highest priority, so whenever near-field blocks retire the block scheduler issues
// the (small, latency-bound) coarse-level sweep kernels first; the near-field work fills the rest of the GPU.
#include <algorithm>
#include <cerrno>
#include <cmath>
#include <new>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "fmm2d.h"
#include "fmm_internal.cuh"

using namespace fmm;

namespace {

enum Mode { MODE_FULL = 0, MODE_NEAR = 1, MODE_FAR = 2 };

struct SysHost {
    int64_t p0, np;
    int depth;
    double sigma;
    int explicit_domain;
    double dom[3];
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// fixed workspace header: status word and pair count, bounding boxes, system descriptors, per-level lists
const size_t HDR_MINMAX = 256;
const size_t HDR_SYS = HDR_MINMAX + align256((size_t)FMM_MAXSYS * 32);
const size_t HDR_LIST = HDR_SYS + align256((size_t)FMM_MAXSYS * sizeof(SysDev));
const size_t HDR_BYTES = HDR_LIST + align256((size_t)(FMM_MAXL + 2) * FMM_MAXSYS * sizeof(int));

}  // namespace

struct fmm_ctx {
    int depth = 0, p = 0;
    double sigma = 0.0;
    int has_domain = 0;
    double dom[3] = {0, 0, 1};
    int mixed = 0;
    int coarse = -1;  // precision form: FP32 on every level (radius-scaled translations stay bounded)
    int tail_rings = 0;  // uniform tree: rings of leaves beyond the adjacent ones that get the far-field correction
    int m2l_engine = FMM_M2L_CUDA_CORES;  // the faster engine at the measured configurations; fmm_autotune re-times both
    int adaptive_cap = 0;  // > 0: adaptive tree (depth = maximum depth), split boxes holding more particles
    int adj_fp32 = 0;      // near-field part of the adjoint in FP32 (fmm_set_adjoint_precision)
    // sharded evaluations: level whose multipoles and counts come from outside (0: none), and the arrays
    int ext_level = 0;
    const double2 *ext_M = nullptr;
    const long long *ext_cnt = nullptr;
    cudaStream_t stream = nullptr;  // caller's stream
    cudaStream_t exec = nullptr;    // internal stream used for graph capture / replay
    cudaStream_t side = nullptr;    // high-priority stream of the multipole sweep
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_status = nullptr, ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t ev_t[8] = {};
    int timing = 0, count_pairs = 0, use_graph = 0;
    int p2p_threads = 64, p2p_kt = 4;
    int device = 0;
    // workspace: a fixed header (status, pair count, bounding boxes, system table and lists) that never moves,
    // and the per-size arrays carved from `ws`
    void *hdr = nullptr;
    void *ws = nullptr;
    size_t ws_cap = 0;
    Work w{};
    // tables (depend on p only)
    void *tab = nullptr;
    void *tab_tc = nullptr;  // tensor-core M2L operand table
    size_t tab_tc_cap = 0;
    double *adv = nullptr;  // advection scratch: stage positions, stage velocity, accumulated increment (6 n)
    size_t adv_cap = 0;
    Tables t{};
    int tab_p = -1;
    // host-visible status
    unsigned int *h_status = nullptr;
    unsigned long long *h_pairs = nullptr;
    int status_pending = 0;
    int pairs_valid = 0;
    // system table cache
    std::vector<SysHost> sys_cfg;
    std::vector<SysDev> sys_dev;
    std::vector<int> sys_list;
    LevelInfo lv{};
    uint64_t cfg_version = 1;
    uint64_t uploaded_version = 0;
    // graph
    cudaGraphExec_t gexec = nullptr;
    int g_nodes = 0;
    uint64_t layout_version = 1;
    size_t layout_sig[6] = {};
    struct GKey {
        int mode, n, nsys, mixed, coarse, m2l_engine, threads, kt, count_pairs, p, timing, adaptive, ext_level, tail;
        uint64_t layout;
        const void *ptr[7];
        uint64_t version;
        void *ws;
    } gkey{};
    // host-buffer staging
    double *d_io = nullptr;
    size_t d_io_cap = 0;
    int64_t launches = 0;
    int last_timed = 0;
    unsigned timed_mask = 0;  // which ev_t[] the last timed evaluation recorded
    std::string err;
};

static fmm_status set_err(fmm_handle h, fmm_status s, const char *fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return s;
}

#define CU(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return set_err(h, e_ == cudaErrorMemoryAllocation ? FMM_ENOMEM : FMM_ECUDA, "%s: %s (%s:%d)", \
                           #call, cudaGetErrorString(e_), __FILE__, __LINE__);                            \
    } while (0)

static fmm_status device_status_to_fmm(unsigned int st)
{
    if (st & FMM_DEV_BOUNDS)
        return FMM_EINTERNAL;
    if (st & FMM_DEV_TIMEOUT)
        return FMM_ETIMEOUT;
    if (st & FMM_DEV_OUTSIDE)
        return FMM_EINVAL;
    return FMM_OK;
}

// Reports (once) a device-side error of an earlier evaluation, without blocking.
static fmm_status poll_status(fmm_handle h, bool block)
{
    if (!h->status_pending)
        return FMM_OK;
    if (block) {
        CU(cudaEventSynchronize(h->ev_status));
    } else {
        cudaError_t q = cudaEventQuery(h->ev_status);
        if (q == cudaErrorNotReady)
            return FMM_OK;
        if (q != cudaSuccess)
            return set_err(h, FMM_ECUDA, "evaluation failed: %s", cudaGetErrorString(q));
    }
    h->status_pending = 0;
    unsigned int st = *h->h_status;
    if (st) {
        *h->h_status = 0;
        CU(cudaMemsetAsync(h->hdr, 0, sizeof(unsigned int), h->stream));  // the status word heads the header
        fmm_status s = device_status_to_fmm(st);
        const char *what = s == FMM_EINVAL     ? "a particle lies outside the root square or is not finite"
                           : s == FMM_ETIMEOUT ? "a bounded wait for a shared-memory copy ran out"
                                               : "a device bounds check failed";
        return set_err(h, s, "device reported: %s (status 0x%x)", what, st);
    }
    return FMM_OK;
}

// ------------------------------------------------------------------ tables

static fmm_status ensure_tables(fmm_handle h)
{
    if (upload_m2l_constants(h->stream) != 0)
        return set_err(h, FMM_ECUDA, "constant-table upload failed");
    if (prepare_m2l_tc() != 0)
        return set_err(h, FMM_ECUDA, "tensor-core M2L kernel attributes could not be set");
    if (prepare_p2p() != 0)
        return set_err(h, FMM_ECUDA, "near-field kernel attributes could not be set");
    if (h->tab_p == h->p)
        return FMM_OK;
    const int P = FMM_PMAX, RS = 2 * FMM_PMAX + 2;
    size_t n_mat = 4 * P * P, n_rho = FMM_NOFF * RS, n_bin = P * P;
    std::vector<double2> m2m(n_mat), l2l(n_mat), rho(n_rho);
    std::vector<double> bin(n_bin);
    build_tables_host(h->p, m2m.data(), l2l.data(), rho.data(), bin.data());
    std::vector<float2> m2m32(n_mat), l2l32(n_mat), rho32(n_rho);
    std::vector<float> bin32(n_bin);
    for (size_t i = 0; i < n_mat; ++i) {
        m2m32[i] = make_float2((float)m2m[i].x, (float)m2m[i].y);
        l2l32[i] = make_float2((float)l2l[i].x, (float)l2l[i].y);
    }
    for (size_t i = 0; i < n_rho; ++i)
        rho32[i] = make_float2((float)rho[i].x, (float)rho[i].y);
    for (size_t i = 0; i < n_bin; ++i)
        bin32[i] = (float)bin[i];
    size_t off[8], total = 0;
    size_t sz[8] = {n_mat * 16, n_mat * 16, n_mat * 8, n_mat * 8, n_rho * 16, n_rho * 8, n_bin * 8, n_bin * 4};
    for (int i = 0; i < 8; ++i) {
        off[i] = total;
        total += align256(sz[i]);
    }
    if (!h->tab) {
        CU(cudaMalloc(&h->tab, total));
    }
    char *b = (char *)h->tab;
    h->t.m2m64 = (double2 *)(b + off[0]);
    h->t.l2l64 = (double2 *)(b + off[1]);
    h->t.m2m32 = (float2 *)(b + off[2]);
    h->t.l2l32 = (float2 *)(b + off[3]);
    h->t.rho64 = (double2 *)(b + off[4]);
    h->t.rho32 = (float2 *)(b + off[5]);
    h->t.binom64 = (double *)(b + off[6]);
    h->t.binom32 = (float *)(b + off[7]);
    CU(cudaMemcpy(h->t.m2m64, m2m.data(), sz[0], cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->t.l2l64, l2l.data(), sz[1], cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->t.m2m32, m2m32.data(), sz[2], cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->t.l2l32, l2l32.data(), sz[3], cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->t.rho64, rho.data(), sz[4], cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->t.rho32, rho32.data(), sz[5], cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->t.binom64, bin.data(), sz[6], cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->t.binom32, bin32.data(), sz[7], cudaMemcpyHostToDevice));
    // tensor-core M2L operands (sized by p's bucket)
    const size_t tc_bytes = m2l_tc_table_bytes(h->p);
    if (tc_bytes > h->tab_tc_cap) {
        if (h->tab_tc)
            CU(cudaFree(h->tab_tc));
        h->tab_tc = nullptr;
        h->tab_tc_cap = 0;
        CU(cudaMalloc(&h->tab_tc, tc_bytes));
        h->tab_tc_cap = tc_bytes;
    }
    std::vector<unsigned char> tc(tc_bytes);
    build_m2l_tc_table_host(h->p, tc.data());
    CU(cudaMemcpy(h->tab_tc, tc.data(), tc_bytes, cudaMemcpyHostToDevice));
    h->t.m2l_tc = (unsigned char *)h->tab_tc;
    h->tab_p = h->p;
    return FMM_OK;
}

// ------------------------------------------------------------------ system table and workspace

// Builds device descriptors, leaf / box offsets and per-level system lists for the configured systems.
static void build_system_layout(fmm_handle h, int64_t *nleaf_out, int64_t *nbox_out)
{
    int nsys = (int)h->sys_cfg.size();
    h->sys_dev.assign(nsys, SysDev{});
    int64_t leaf = 0, box = 0;
    int maxd = 0;
    for (int k = 0; k < nsys; ++k) {
        const SysHost &c = h->sys_cfg[k];
        SysDev &d = h->sys_dev[k];
        d.p0 = c.p0;
        d.np = c.np;
        d.depth = c.depth;
        d.sigma = c.sigma;
        d.explicit_domain = c.explicit_domain;
        d.x0 = c.dom[0];
        d.y0 = c.dom[1];
        d.S = c.dom[2];
        d.leaf0 = leaf;
        leaf += (int64_t)1 << (2 * c.depth);
        for (int l = 0; l <= FMM_MAXL; ++l)
            d.box0[l] = -1;
        if (c.explicit_domain)
            derive_constants(d);  // else the domain kernel derives them from the bounding box
        if (c.depth > maxd)
            maxd = c.depth;
    }
    // boxes grouped by level, then by system, so one level of all systems is one contiguous range
    for (int l = 2; l <= maxd; ++l)
        for (int k = 0; k < nsys; ++k)
            if (h->sys_cfg[k].depth >= l) {
                h->sys_dev[k].box0[l] = box;
                box += (int64_t)1 << (2 * l);
            }
    LevelInfo lv{};
    lv.maxdepth = maxd;
    h->sys_list.clear();
    for (int l = 0; l <= FMM_MAXL + 1; ++l) {
        lv.first_at[l] = (int)h->sys_list.size();
        int cnt = 0;
        for (int k = 0; k < nsys; ++k)
            if (l <= FMM_MAXL && h->sys_cfg[k].depth >= l) {
                h->sys_list.push_back(k);
                ++cnt;
            }
        lv.nsys_at[l] = cnt;
    }
    int64_t acc = 0;
    for (int l = 0; l <= FMM_MAXL + 1; ++l)
        lv.m2l_item0[l] = 0;
    for (int l = 2; l <= maxd; ++l) {
        lv.m2l_item0[l] = acc;
        acc += (int64_t)lv.nsys_at[l] << (2 * l);
    }
    lv.m2l_item0[maxd + 1 <= FMM_MAXL + 1 ? maxd + 1 : FMM_MAXL + 1] = acc;
    lv.mindepth2 = 0;
    for (int k = 0; k < nsys; ++k) {
        int dk = h->sys_cfg[k].depth;
        if (dk >= 2 && (lv.mindepth2 == 0 || dk < lv.mindepth2))
            lv.mindepth2 = dk;
    }
    h->lv = lv;
    *nleaf_out = leaf;
    *nbox_out = box;
}

struct Layout {
    size_t off[40];
    size_t total;
};

static fmm_status ensure_workspace(fmm_handle h, int64_t n, int adjoint)
{
    int64_t nleaf, nbox;
    build_system_layout(h, &nleaf, &nbox);
    if (n >= ((int64_t)1 << 31) - 64 || nleaf >= ((int64_t)1 << 31) - 2)
        return set_err(h, FMM_EINVAL, "too many particles (%lld) or leaves (%lld) for 32-bit indices",
                       (long long)n, (long long)nleaf);
    int nsys = (int)h->sys_cfg.size();
    int p = h->p;
    bool mixed = h->mixed && !adjoint && !h->adaptive_cap;  // the adaptive tree bins in the FP64 form
    bool ad_mixed = h->mixed && !adjoint && h->adaptive_cap;  // ... and keeps FP32 expansions / split positions
    bool f64 = !mixed || adjoint;
    size_t np = (size_t)n + 8;
    size_t sizes[40];
    int i = 0;
    sizes[i++] = np * 4;                                      // 0 key
    sizes[i++] = (size_t)nleaf * 4 + 16;                      // 1 cnt and the overflow flag
    sizes[i++] = (size_t)(nleaf + 1) * 4 + 16;                // 2 start
    sizes[i++] = (size_t)((nleaf + 1023) / 1024 + 2) * 4;     // 3 scan_tmp
    sizes[i++] = np * 8;                                      // 4 tmp (caller index, leaf)
    sizes[i++] = np * 4;                                      // 5 perm
    sizes[i++] = np * 4;                                      // 6 sleaf
    sizes[i++] = f64 ? np * 8 : 0;                            // 7 sx
    sizes[i++] = f64 ? np * 8 : 0;                            // 8 sy
    sizes[i++] = f64 ? np * 8 : 0;                            // 9 sg
    sizes[i++] = (mixed || ad_mixed) ? np * 48 : 0;           // 10 eh, el, eg
    sizes[i++] = 0;                                           // 11 (far32 lives in near32's records)
    sizes[i++] = (mixed || h->adaptive_cap) ? 0 : np * 16;    // 12 near64 (the adaptive walk writes u, v itself)
    sizes[i++] = mixed ? np * 16 : 0;                         // 13 near32 + far32, interleaved
    sizes[i++] = (size_t)nbox * 4 + 16;                       // 14 bcount
    sizes[i++] = ad_mixed ? 0 : (size_t)nbox * p * 16;        // 15 M64 (the adaptive precision form keeps FP32 only)
    sizes[i++] = ad_mixed ? 0 : (size_t)nbox * p * 16;        // 16 L64
    sizes[i++] = (mixed || ad_mixed) ? (size_t)nbox * p * 8 : 0;  // 17 M32
    sizes[i++] = (mixed || ad_mixed) ? (size_t)nbox * p * 8 : 0;  // 18 L32
    sizes[i++] = adjoint ? np * 8 : 0;                        // 19 sgu
    sizes[i++] = adjoint ? np * 8 : 0;                        // 20 sgv
    sizes[i++] = adjoint ? (size_t)nbox * p * 16 : 0;         // 21 AM64
    sizes[i++] = adjoint ? (size_t)nbox * p * 16 : 0;         // 22 AL64
    sizes[i++] = mixed ? np * 32 : 0;                         // 23 nearp [4][n]
    sizes[i++] = mixed ? np * 32 : 0;                         // 24 pos4u (two float4 per particle)
    sizes[i++] = mixed ? 0 : np * 32;                         // 25 rec64
    sizes[i++] = np * 4;                                      // 26 slot
    sizes[i++] = np * 4;                                      // 27 iperm
    sizes[i++] = adjoint ? np * 24 : 0;                       // 28 adj_far
    sizes[i++] = h->adaptive_cap ? (size_t)nbox * 4 + 16 : 0;   // 29 ad_list
    sizes[i++] = h->adaptive_cap ? (FMM_MAXL + 2) * 4 : 0;      // 30 ad_cnt
    sizes[i++] = (size_t)(n / 129 + 2) * 4;                    // 31 big (leaves of more than 128 particles)
    sizes[i++] = mixed ? (size_t)nleaf * 32 + 16 : 0;          // 32 cls_off (boundary classes of each leaf)
    sizes[i++] = mixed ? np : 0;                              // 33 cls8 (boundary class of each particle)
    // 34 leaf buckets of the uniform tree: four times the mean occupancy (at least 32) per leaf, so that only
    // strongly clustered inputs overflow into the scatter; none where that would take more than 64 B a particle
    int64_t bcap = 4 * ((n + nleaf - 1) / (nleaf > 0 ? nleaf : 1));
    bcap = bcap < 32 ? 32 : (bcap + 31) / 32 * 32;
    const bool use_bkt = !h->adaptive_cap && nleaf > 0 && (size_t)nleaf * (size_t)bcap * 8 <= 64 * np;
    sizes[i++] = use_bkt ? (size_t)nleaf * (size_t)bcap * 8 : 0;
    sizes[i++] = mixed ? m2l_tc_layout_bytes(h->lv, p) : 0;     // 35 mtc (tensor-core M2L windows)
    sizes[i++] = mixed ? m2l_tc_part_bytes(h->lv, p) : 0;       // 36 m2l_part (its partial locals)
    sizes[i++] = mixed ? m2l_tc_count_bytes(h->lv, p) : 0;      // 37 m2l_cnt (its tile counters)
    int count = i;
    Layout lay;
    size_t total = 0;
    for (int j = 0; j < count; ++j) {
        lay.off[j] = total;
        total += align256(sizes[j]);
    }
    if (total > h->ws_cap) {
        if (h->ws) {
            CU(cudaDeviceSynchronize());
            CU(cudaFree(h->ws));
            h->ws = nullptr;
            h->ws_cap = 0;
        }
        size_t cap = total + total / 8;
        CU(cudaMalloc(&h->ws, cap));
        h->ws_cap = cap;
        CU(cudaMemset(h->ws, 0, cap));
    }
    size_t sig[6] = {(size_t)n, (size_t)nleaf, (size_t)nbox, (size_t)p, (size_t)(mixed ? 1 : 0) + 2 * (size_t)adjoint + 4 * (size_t)ad_mixed,
                     (size_t)h->ws};
    if (memcmp(sig, h->layout_sig, sizeof sig) != 0) {
        memcpy(h->layout_sig, sig, sizeof sig);
        h->layout_version++;
    }
    char *b = (char *)h->ws;
    Work &w = h->w;
    w = Work{};
    w.n = (int)n;
    w.nleaf = (int)nleaf;
    w.nbox = nbox;
    w.p = p;
    w.mixed = mixed ? 1 : 0;
    w.coarse_level = h->coarse;
    w.m2l_tc = h->m2l_engine == FMM_M2L_TENSOR ? 1 : 0;
    w.nsys = nsys;
    w.maxdepth = h->lv.maxdepth;
    w.morton = h->adaptive_cap > 0 ? 1 : 0;
    w.adapt_cap = h->adaptive_cap;
    w.ad_mixed = ad_mixed ? 1 : 0;
    w.key = (int *)(b + lay.off[0]);
    w.cnt = (int *)(b + lay.off[1]);
    w.start = (int *)(b + lay.off[2]);
    w.scan_tmp = (int *)(b + lay.off[3]);
    w.tmp = (int2 *)(b + lay.off[4]);
    w.perm = (int *)(b + lay.off[5]);
    w.sleaf = (int *)(b + lay.off[6]);
    w.sx = sizes[7] ? (double *)(b + lay.off[7]) : nullptr;
    w.sy = sizes[8] ? (double *)(b + lay.off[8]) : nullptr;
    w.sg = sizes[9] ? (double *)(b + lay.off[9]) : nullptr;
    w.eh = sizes[10] ? (float4 *)(b + lay.off[10]) : nullptr;
    w.el = sizes[10] ? w.eh + np : nullptr;
    w.eg = sizes[10] ? w.el + np : nullptr;
    w.near64 = sizes[12] ? (double2 *)(b + lay.off[12]) : nullptr;
    // precision form: near and far field of each particle side by side in one 16-byte record
    w.near32 = sizes[13] ? (float2 *)(b + lay.off[13]) : nullptr;
    w.far32 = sizes[13] ? w.near32 + 1 : nullptr;
    w.nf_stride = sizes[13] ? 2 : 1;
    w.nearp = sizes[23] ? (float2 *)(b + lay.off[23]) : nullptr;
    w.bcount = (int *)(b + lay.off[14]);
    w.M64 = sizes[15] ? (double2 *)(b + lay.off[15]) : nullptr;
    w.L64 = sizes[16] ? (double2 *)(b + lay.off[16]) : nullptr;
    w.M32 = sizes[17] ? (float2 *)(b + lay.off[17]) : nullptr;
    w.L32 = sizes[18] ? (float2 *)(b + lay.off[18]) : nullptr;
    w.mtc = sizes[35] ? (float4 *)(b + lay.off[35]) : nullptr;
    w.m2l_part = sizes[36] ? (float2 *)(b + lay.off[36]) : nullptr;
    w.m2l_cnt = sizes[37] ? (int *)(b + lay.off[37]) : nullptr;
    w.sgu = sizes[19] ? (double *)(b + lay.off[19]) : nullptr;
    w.sgv = sizes[20] ? (double *)(b + lay.off[20]) : nullptr;
    w.AM64 = sizes[21] ? (double2 *)(b + lay.off[21]) : nullptr;
    w.AL64 = sizes[22] ? (double2 *)(b + lay.off[22]) : nullptr;
    w.slot = (int *)(b + lay.off[26]);
    w.iperm = (int *)(b + lay.off[27]);
    {
        void *dp = nullptr;  // device view of the page-locked status word (null: copy it instead)
        w.status_host = cudaHostGetDevicePointer(&dp, h->h_status, 0) == cudaSuccess ? (unsigned int *)dp : nullptr;
        (void)cudaGetLastError();
    }
    w.pos4u = sizes[24] ? (float4 *)(b + lay.off[24]) : nullptr;
    w.rec64 = sizes[25] ? (Rec64 *)(b + lay.off[25]) : nullptr;
    char *hd = (char *)h->hdr;
    w.status = (unsigned int *)hd;
    w.pair_count = (unsigned long long *)(hd + 32);
    w.big_cnt = (int *)(hd + 64);
    w.minmax = (unsigned long long *)(hd + HDR_MINMAX);
    w.sys = (SysDev *)(hd + HDR_SYS);
    w.sys_list = (int *)(hd + HDR_LIST);
    w.adj_far = sizes[28] ? (double *)(b + lay.off[28]) : nullptr;
    w.ad_list = sizes[29] ? (int *)(b + lay.off[29]) : nullptr;
    w.ad_cnt = sizes[30] ? (int *)(b + lay.off[30]) : nullptr;
    w.big = (int *)(b + lay.off[31]);
    w.cls_off = sizes[32] ? (int *)(b + lay.off[32]) : nullptr;
    w.cls8 = sizes[33] ? (unsigned char *)(b + lay.off[33]) : nullptr;
    w.bkt = sizes[34] ? (int2 *)(b + lay.off[34]) : nullptr;
    w.bkt_cap = sizes[34] ? (int)bcap : 0;
    w.lv = h->lv;
    return FMM_OK;
}

static fmm_status upload_systems(fmm_handle h)
{
    if (h->uploaded_version == h->cfg_version && h->w.sys)
        return FMM_OK;
    // the previous evaluation may still read the table: order the upload on the stream
    CU(cudaMemcpyAsync(h->w.sys, h->sys_dev.data(), h->sys_dev.size() * sizeof(SysDev), cudaMemcpyHostToDevice,
                       h->stream));
    CU(cudaMemcpyAsync(h->w.sys_list, h->sys_list.data(), h->sys_list.size() * sizeof(int),
                       cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    h->uploaded_version = h->cfg_version;
    return FMM_OK;
}

static void set_single_system(fmm_handle h, int64_t n)
{
    SysHost c{};
    c.p0 = 0;
    c.np = n;
    c.depth = h->depth;
    c.sigma = h->sigma;
    c.explicit_domain = h->has_domain;
    c.dom[0] = h->dom[0];
    c.dom[1] = h->dom[1];
    c.dom[2] = h->dom[2];
    if (h->sys_cfg.size() != 1 || memcmp(&h->sys_cfg[0], &c, sizeof c) != 0) {
        h->sys_cfg.assign(1, c);
        h->cfg_version++;
    }
}

// ------------------------------------------------------------------ the stage DAG

// Timing events: inside a stream capture they must be external event-record nodes to carry timestamps.
static cudaError_t record_timing(cudaEvent_t ev, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    return cudaEventRecordWithFlags(ev, s, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                                : cudaEventRecordDefault);
}

// The adaptive tree: the same binning (Morton keys at the maximum depth), the multipole sweep on the side stream
// (box lists, P2L, P2M, M2M, then the downward L2L + M2L levels), then after the join one walk per target that
// evaluates the U-list pairs, the W-list multipoles and the leaf's local and writes the sum in the caller's order
// (adaptive.cu). Running the U-list pairs at the fork instead, concurrently with the sweep, with the W list and
// L2P in a second walk on the sweep stream, was measured slower on GB300: both halves keep every SM's issue slots
// busy, so they add up, and the second walk costs what it walks.
static fmm_status enqueue_adaptive(fmm_handle h, cudaStream_t s, int mode, const double *x, const double *y,
                                   const double *g, double *u, double *v)
{
    Work &w = h->w;
    const bool near = mode != MODE_FAR;
    const bool sweep = mode != MODE_NEAR && w.maxdepth >= 2;  // below depth 2 every pair is in a U list
    const bool timed = h->timing != 0;
    int64_t nl = 0;
    (void)cudaGetLastError();
    if (timed)
        CU(record_timing(h->ev_t[0], s));
    CU(cudaMemsetAsync(w.cnt, 0, (size_t)(w.nleaf + 1) * sizeof(int), s));  // counts and overflow flag
    if (!h->has_domain) {
        nl += launch_bbox(w, x, y, s);
        nl += launch_domain_finalize(w, s);
    }
    nl += launch_keys(w, x, y, g, s);
    nl += launch_scan(w, s);
    nl += launch_scatter_sort(w, s);
    nl += launch_gather(w, x, y, g, nullptr, nullptr, s);
    const bool count = near && h->count_pairs;
    if (count)
        CU(cudaMemsetAsync(w.pair_count, 0, sizeof(unsigned long long), s));
    if (sweep)
        CU(cudaMemsetAsync(w.ad_cnt, 0, (FMM_MAXL + 2) * sizeof(int), s));
    if (timed)
        CU(record_timing(h->ev_t[1], s));
    if (sweep) {
        CU(cudaEventRecord(h->ev_fork, s));
        CU(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        nl += launch_adaptive_up(w, h->t, h->side);
        if (timed)
            CU(record_timing(h->ev_t[2], h->side));
        nl += launch_adaptive_down(w, h->t, h->side);
        if (timed)
            CU(record_timing(h->ev_t[3], h->side));
        CU(cudaEventRecord(h->ev_join, h->side));
        CU(cudaStreamWaitEvent(s, h->ev_join, 0));
    }
    if (timed)
        CU(record_timing(h->ev_t[6], s));
    // the walk reads the W multipoles and the leaf's local expansion
    nl += launch_adaptive_near(w, count ? w.pair_count : nullptr, near ? 1 : 0, sweep ? 1 : 0, u, v, s);
    if (timed)
        CU(record_timing(h->ev_t[5], s));
    if (count)
        CU(cudaMemcpyAsync(h->h_pairs, w.pair_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(h->h_status, w.status, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    if (timed)
        CU(record_timing(h->ev_t[7], s));
    CU(cudaGetLastError());
    h->launches += nl;
    h->last_timed = timed;
    // recorded: binning (0-1), sweep (1-2 up, 2-3 down; 1-6 fork to join), the walk (6-5), total (0-7)
    h->timed_mask = timed ? (sweep ? 0xefu : 0xe3u) : 0u;
    return FMM_OK;
}

static fmm_status enqueue_forward(fmm_handle h, cudaStream_t s, int mode, const double *x, const double *y,
                                  const double *g, double *u, double *v)
{
    if (h->adaptive_cap > 0)
        return enqueue_adaptive(h, s, mode, x, y, g, u, v);
    Work &w = h->w;
    bool far = mode != MODE_NEAR && w.lv.maxdepth >= 2;
    bool near = mode != MODE_FAR;
    bool timed = h->timing != 0;  // in a graph the event records become event-record nodes
    const bool all_ev = h->timing == 1;  // timing 2: the near field's two events only (each node costs ~3 us)
    int64_t nl = 0;
    // symmetric near field (tile 128): reactions land in nearp and the final sum adds them. The host knows a
    // system takes one-float coordinates only for an explicit square (s is computed here as the device does,
    // with a margin); otherwise the split-form kernel is launched as well and skips the one-float systems.
    w.p2p_sym = near && w.mixed && h->p2p_threads == 128 && w.nearp ? 1 : 0;
    w.p2p_rows = near && w.mixed && h->p2p_threads == 192 && w.nearp ? 1 : 0;
    w.p2p_all_plain = 1;
    for (auto &c : h->sys_cfg) {
        if (!c.explicit_domain) {
            w.p2p_all_plain = 0;
            continue;
        }
        const double wl = ldexp(c.dom[2], -c.depth), kap = wl * wl / (2.0 * c.sigma * c.sigma);
        if (!(sqrt(1.4426950408889634074 * kap) < (double)P2P_SPLIT_S * (1.0 - 1e-6)))
            w.p2p_all_plain = 0;
    }
    (void)cudaGetLastError();  // drop a stale, non-sticky error left by an unrelated runtime call
    if (timed && all_ev)
        CU(record_timing(h->ev_t[0], s));
    CU(cudaMemsetAsync(w.cnt, 0, (size_t)(w.nleaf + 1) * sizeof(int), s));  // counts and overflow flag
    bool any_bbox = false;
    for (auto &c : h->sys_cfg)
        any_bbox |= !c.explicit_domain;
    if (any_bbox) {  // explicit squares: the host derived the constants
        nl += launch_bbox(w, x, y, s);
        nl += launch_domain_finalize(w, s);
    }
    nl += launch_keys(w, x, y, g, s);
    nl += launch_scan(w, s);
    nl += launch_scatter_sort(w, s);
    nl += launch_gather(w, x, y, g, nullptr, nullptr, s);
    if (timed)
        CU(record_timing(h->ev_t[1], s));
    if (far) {
        CU(cudaEventRecord(h->ev_fork, s));
        CU(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        nl += launch_p2m(w, h->t, 0, h->side);
        if (h->ext_level == w.lv.maxdepth)
            nl += launch_level_import(w, h->ext_level, h->ext_M, h->ext_cnt, h->side);
        for (int l = w.lv.maxdepth - 1; l >= 2; --l) {
            nl += launch_m2m(w, h->t, l, 0, h->side, 1);
            if (l == h->ext_level)  // the coarse levels carry every particle the given level stands for
                nl += launch_level_import(w, l, h->ext_M, h->ext_cnt, h->side);
        }
        if (timed && all_ev)
            CU(record_timing(h->ev_t[2], h->side));
        nl += launch_m2l(w, h->t, 0, h->side, 1);
        if (timed && all_ev)
            CU(record_timing(h->ev_t[3], h->side));
        for (int l = 2; l < w.lv.maxdepth; ++l)
            nl += launch_l2l(w, h->t, l, 0, h->side, 1);
        nl += launch_l2p(w, h->side);  // precision form: the far field before the join
        if (timed && all_ev)
            CU(record_timing(h->ev_t[4], h->side));
        CU(cudaEventRecord(h->ev_join, h->side));
    }
    if (near) {
        nl += launch_p2p(w, h->p2p_threads, h->p2p_kt, s);
        nl += launch_far_tail(w, h->tail_rings, s);
    }
    if (timed)
        CU(record_timing(h->ev_t[5], s));
    if (far)
        CU(cudaStreamWaitEvent(s, h->ev_join, 0));
    if (timed && all_ev)
        CU(record_timing(h->ev_t[6], s));
    nl += launch_combine(w, near ? 1 : 0, far ? 1 : 0, u, v, s);
    if (h->count_pairs) {
        CU(cudaMemsetAsync(w.pair_count, 0, sizeof(unsigned long long), s));
        nl += launch_pair_count(w, s);
        CU(cudaMemcpyAsync(h->h_pairs, w.pair_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    }
    if (!w.status_host)  // the final sum kernel writes it otherwise
        CU(cudaMemcpyAsync(h->h_status, w.status, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    if (timed && all_ev)
        CU(record_timing(h->ev_t[7], s));
    CU(cudaGetLastError());
    h->launches += nl;
    h->last_timed = timed;
    h->timed_mask = timed ? (all_ev ? (far ? 0xffu : 0xe3u) : 0x22u) : 0u;
    return FMM_OK;
}

static int count_kernel_nodes(cudaGraph_t g)
{
    size_t nn = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess)
        return 0;
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    int k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
            ++k;
    }
    return k;
}

static fmm_status run_forward(fmm_handle h, int mode, int64_t n, const double *x, const double *y,
                              const double *g, double *u, double *v)
{
    fmm_status st;
    if (h->tail_rings && h->adaptive_cap)
        return set_err(h, FMM_EINVAL, "the far-field tail correction needs the uniform tree (fmm_set_far_tail(h, 0))");
    if ((st = ensure_tables(h)) != FMM_OK)
        return st;
    if ((st = ensure_workspace(h, n, 0)) != FMM_OK)
        return st;
    if ((st = upload_systems(h)) != FMM_OK)
        return st;
    if (h->count_pairs)
        h->pairs_valid = 1;
    if (!h->use_graph) {
        if ((st = enqueue_forward(h, h->stream, mode, x, y, g, u, v)) != FMM_OK)
            return st;
        CU(cudaEventRecord(h->ev_status, h->stream));
        h->status_pending = 1;
        return FMM_OK;
    }
    fmm_ctx::GKey key{};
    key.mode = mode;
    key.n = (int)n;
    key.nsys = (int)h->sys_cfg.size();
    key.mixed = h->w.mixed;
    key.coarse = h->coarse;
    key.m2l_engine = h->m2l_engine;
    key.threads = h->p2p_threads;
    key.kt = h->p2p_kt;
    key.count_pairs = h->count_pairs;
    key.p = h->p;
    key.timing = h->timing;
    key.tail = h->tail_rings;
    key.adaptive = h->adaptive_cap;
    key.layout = h->layout_version;
    key.ptr[0] = x;
    key.ptr[1] = y;
    key.ptr[2] = g;
    key.ptr[3] = u;
    key.ptr[4] = v;
    key.ext_level = h->ext_level;
    key.ptr[5] = h->ext_M;
    key.ptr[6] = h->ext_cnt;
    key.version = h->cfg_version;
    key.ws = h->ws;
    if (!h->gexec || memcmp(&key, &h->gkey, sizeof key) != 0) {
        if (h->gexec) {
            CU(cudaGraphExecDestroy(h->gexec));
            h->gexec = nullptr;
        }
        CU(cudaStreamBeginCapture(h->exec, cudaStreamCaptureModeThreadLocal));
        int64_t before = h->launches;
        st = enqueue_forward(h, h->exec, mode, x, y, g, u, v);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->exec, &graph);
        h->launches = before;
        if (st != FMM_OK) {
            if (graph)
                cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess)
            return set_err(h, FMM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
        h->g_nodes = count_kernel_nodes(graph);
        e = cudaGraphInstantiate(&h->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            h->gexec = nullptr;
            return set_err(h, FMM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
        }
        h->gkey = key;
    }
    CU(cudaEventRecord(h->ev_in, h->stream));
    CU(cudaStreamWaitEvent(h->exec, h->ev_in, 0));
    CU(cudaGraphLaunch(h->gexec, h->exec));
    CU(cudaEventRecord(h->ev_out, h->exec));
    CU(cudaStreamWaitEvent(h->stream, h->ev_out, 0));
    h->launches += h->g_nodes;
    CU(cudaEventRecord(h->ev_status, h->stream));
    h->status_pending = 1;
    return FMM_OK;
}

// Median of 5 timed evaluations (after 2 untimed ones) of the handle as configured, in ms; < 0 if one failed.
static float time_evaluation(fmm_handle h, int64_t n, const double *x, const double *y, const double *g, double *u,
                             double *v, cudaEvent_t e0, cudaEvent_t e1);

// Adaptive tree: the leaf capacity (and the maximum depth within [depth_lo, depth_hi]) of the fastest evaluation,
// timed as the handle runs (graph replays when it uses graphs); cached like the uniform tree's choice.
static fmm_status autotune_adaptive(fmm_handle h, int64_t n, const double *x, const double *y, const double *g,
                                    double *u, double *v, int depth_lo, int depth_hi)
{
    const char *cache = getenv("FMM2D_TUNE_CACHE");
    char keybuf[192];
    snprintf(keybuf, sizeof keybuf, "adaptive n=%lld p=%d mixed=%d sigma=%.17g lo=%d hi=%d", (long long)n, h->p,
             h->mixed, h->sigma, depth_lo, depth_hi);
    if (cache) {
        FILE *f = fopen(cache, "r");
        if (f) {
            char line[256];
            while (fgets(line, sizeof line, f)) {
                int d, cap;
                char *bar = strchr(line, '|');
                if (!bar)
                    continue;
                *bar = 0;
                if (strcmp(line, keybuf) == 0 && sscanf(bar + 1, "%d %d", &d, &cap) == 2 && cap > 0) {
                    fclose(f);
                    h->depth = d;
                    h->adaptive_cap = cap;
                    h->cfg_version++;
                    return FMM_OK;
                }
            }
            fclose(f);
        }
    }
    static const int caps[] = {16, 24, 32, 48, 64, 96, 128};
    const int save_timing = h->timing;
    h->timing = 0;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    int bd = h->depth, bcap = h->adaptive_cap;
    for (int d = depth_lo; d <= depth_hi; ++d)
        for (int cap : caps) {
            h->depth = d;
            h->adaptive_cap = cap;
            h->cfg_version++;
            const float t = time_evaluation(h, n, x, y, g, u, v, e0, e1);
            if (t >= 0.f && t < best) {
                best = t;
                bd = d;
                bcap = cap;
            }
        }
    h->depth = bd;
    h->adaptive_cap = bcap;
    h->cfg_version++;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->timing = save_timing;
    if (best >= 1e30f)
        return set_err(h, FMM_ECUDA, "no candidate ran");
    if (cache) {
        FILE *f = fopen(cache, "a");
        if (f) {
            fprintf(f, "%s|%d %d\n", keybuf, bd, bcap);
            fclose(f);
        }
    }
    return FMM_OK;
}

// Sum of (u - ur)^2 + (v - vr)^2 and of ur^2 + vr^2 over all particles (FP64, one atomic per block and sum).
__global__ void __launch_bounds__(256) k_rel_l2_parts(int64_t n, const double *__restrict__ u,
                                                      const double *__restrict__ v, const double *__restrict__ ur,
                                                      const double *__restrict__ vr, double *out)
{
    __shared__ double sd[8], sr[8];
    double d = 0.0, r = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double du = u[i] - ur[i], dv = v[i] - vr[i];
        d += du * du + dv * dv;
        r += ur[i] * ur[i] + vr[i] * vr[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, o);
        r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sd[threadIdx.x >> 5] = d;
        sr[threadIdx.x >> 5] = r;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        d = r = 0.0;
        for (int k = 0; k < 8; ++k) {
            d += sd[k];
            r += sr[k];
        }
        atomicAdd(out, d);
        atomicAdd(out + 1, r);
    }
}

// ------------------------------------------------------------------ C ABI

extern "C" {

fmm_status fmm_create(int tree_depth, int p, double sigma, fmm_handle *out)
{
    if (!out)
        return FMM_EINVAL;
    *out = nullptr;
    if (tree_depth < 0 || tree_depth > FMM_MAXL || p < 1 || p > FMM_PMAX || !(sigma > 0.0) || !(sigma < 1e300))
        return FMM_EINVAL;
    fmm_handle h = new (std::nothrow) fmm_ctx();
    if (!h)
        return FMM_ENOMEM;
    h->depth = tree_depth;
    h->p = p;
    h->sigma = sigma;
    cudaError_t e = cudaGetDevice(&h->device);
    int lo = 0, hi = 0;
    if (e == cudaSuccess)
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&h->exec, cudaStreamNonBlocking);
    cudaEvent_t *evs[] = {&h->ev_fork, &h->ev_join, &h->ev_status, &h->ev_in, &h->ev_out};
    for (auto ev : evs)
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    for (int i = 0; i < 8 && e == cudaSuccess; ++i)
        e = cudaEventCreate(&h->ev_t[i]);
    if (e == cudaSuccess)
        e = cudaMalloc(&h->hdr, HDR_BYTES);
    if (e == cudaSuccess)
        e = cudaMemset(h->hdr, 0, HDR_BYTES);
    if (e == cudaSuccess)
        e = cudaMallocHost(&h->h_status, 64);
    if (e == cudaSuccess) {
        h->h_pairs = (unsigned long long *)((char *)h->h_status + 32);
        *h->h_status = 0;
        *h->h_pairs = 0;
    }
    if (e != cudaSuccess) {
        fmm_destroy(h);
        return e == cudaErrorMemoryAllocation ? FMM_ENOMEM : FMM_ECUDA;
    }
    *out = h;
    return FMM_OK;
}

fmm_status fmm_destroy(fmm_handle h)
{
    if (!h)
        return FMM_OK;
    if (h->stream || h->side)
        cudaDeviceSynchronize();
    if (h->gexec)
        cudaGraphExecDestroy(h->gexec);
    cudaEvent_t evs[] = {h->ev_fork, h->ev_join, h->ev_status, h->ev_in, h->ev_out};
    for (auto ev : evs)
        if (ev)
            cudaEventDestroy(ev);
    for (int i = 0; i < 8; ++i)
        if (h->ev_t[i])
            cudaEventDestroy(h->ev_t[i]);
    if (h->side)
        cudaStreamDestroy(h->side);
    if (h->exec)
        cudaStreamDestroy(h->exec);
    if (h->ws)
        cudaFree(h->ws);
    if (h->hdr)
        cudaFree(h->hdr);
    if (h->tab)
        cudaFree(h->tab);
    if (h->tab_tc)
        cudaFree(h->tab_tc);
    if (h->adv)
        cudaFree(h->adv);
    if (h->d_io)
        cudaFree(h->d_io);
    if (h->h_status)
        cudaFreeHost(h->h_status);
    delete h;
    return FMM_OK;
}

fmm_status fmm_set_domain(fmm_handle h, double x0, double y0, double side)
{
    if (!h)
        return FMM_EINVAL;
    if (!(side > 0.0) || !std::isfinite(x0) || !std::isfinite(y0) || !std::isfinite(side))
        return set_err(h, FMM_EINVAL, "invalid root square");
    h->has_domain = 1;
    h->dom[0] = x0;
    h->dom[1] = y0;
    h->dom[2] = side;
    return FMM_OK;
}

fmm_status fmm_clear_domain(fmm_handle h)
{
    if (!h)
        return FMM_EINVAL;
    h->has_domain = 0;
    return FMM_OK;
}

fmm_status fmm_set_precision(fmm_handle h, fmm_precision mode)
{
    if (!h || (mode != FMM_FP64 && mode != FMM_MIXED))
        return FMM_EINVAL;
    h->mixed = mode == FMM_MIXED;
    return FMM_OK;
}

fmm_status fmm_set_coarse_level(fmm_handle h, int coarse_level)
{
    if (!h || coarse_level < -1 || coarse_level > FMM_MAXL)
        return FMM_EINVAL;
    h->coarse = coarse_level;
    return FMM_OK;
}

fmm_status fmm_set_far_tail(fmm_handle h, int rings)
{
    if (!h || rings < 0 || rings > 8)
        return FMM_EINVAL;
    h->tail_rings = rings;
    return FMM_OK;
}

fmm_status fmm_set_m2l_engine(fmm_handle h, int engine)
{
    if (!h || (engine != FMM_M2L_CUDA_CORES && engine != FMM_M2L_TENSOR))
        return FMM_EINVAL;
    h->m2l_engine = engine;
    return FMM_OK;
}

int fmm_get_m2l_engine(fmm_handle h) { return h ? h->m2l_engine : -1; }

fmm_status fmm_set_adaptive(fmm_handle h, int leaf_capacity)
{
    if (!h || leaf_capacity < 0)
        return FMM_EINVAL;
    if (leaf_capacity != h->adaptive_cap) {
        h->adaptive_cap = leaf_capacity;
        h->cfg_version++;
    }
    return FMM_OK;
}

int fmm_get_adaptive(fmm_handle h) { return h ? h->adaptive_cap : -1; }

int fmm_suggest_depth(int64_t n, double sigma, double side, double tail_tol, double leaf_target)
{
    if (n <= 0 || !(sigma > 0.0) || !(side > 0.0) || !(tail_tol > 0.0 && tail_tol < 1.0))
        return -1;
    if (!(leaf_target > 0.0))
        leaf_target = 64.0;
    // occupancy: about leaf_target particles per leaf for uniformly spread particles
    int L = (int)std::lround(std::log((double)n / leaf_target) / std::log(4.0));
    L = std::max(0, std::min(L, FMM_MAXL));
    // far-field tail (§2: the expansions use the point-vortex kernel beyond adjacent leaves, and the nearest such
    // pair is one leaf width w apart): exp(-w^2 / 2 sigma^2) <= tail_tol
    const double wmin = sigma * std::sqrt(2.0 * std::log(1.0 / tail_tol));
    while (L > 0 && std::ldexp(side, -L) < wmin)
        --L;
    return L;
}

fmm_status fmm_set_params(fmm_handle h, int tree_depth, int p, double sigma)
{
    if (!h || tree_depth < 0 || tree_depth > FMM_MAXL || p < 1 || p > FMM_PMAX || !(sigma > 0.0))
        return FMM_EINVAL;
    h->depth = tree_depth;
    h->p = p;
    h->sigma = sigma;
    return FMM_OK;
}

fmm_status fmm_set_stream(fmm_handle h, void *cuda_stream)
{
    if (!h)
        return FMM_EINVAL;
    h->stream = (cudaStream_t)cuda_stream;
    return FMM_OK;
}

fmm_status fmm_set_graph(fmm_handle h, int enable)
{
    if (!h)
        return FMM_EINVAL;
    h->use_graph = enable ? 1 : 0;
    return FMM_OK;
}

fmm_status fmm_set_p2p_tile(fmm_handle h, int threads, int targets_per_thread)
{
    if (!h)
        return FMM_EINVAL;
    if (threads == 0)
        threads = 64;
    if (targets_per_thread == 0)
        targets_per_thread = 4;
    if ((threads != 32 && threads != 64 && threads != 128 && threads != 192 && threads != 256) ||
        (targets_per_thread != 2 && targets_per_thread != 4))
        return set_err(h, FMM_EINVAL,
                       "tile: threads 32 (one leaf per block), 64 (two), 256 (four), 128 (symmetric) or 192 (per "
                       "source row), targets per thread 2 or 4");
    h->p2p_threads = threads;
    h->p2p_kt = targets_per_thread;
    return FMM_OK;
}

static fmm_status check_common(fmm_handle h, int64_t n, const void *x, const void *y, const void *g, const void *u,
                               const void *v)
{
    if (!h)
        return FMM_EINVAL;
    if (n < 0)
        return set_err(h, FMM_EINVAL, "n < 0");
    if (n > 0 && (!x || !y || !g || !u || !v))
        return set_err(h, FMM_EINVAL, "NULL array");
    return FMM_OK;
}

static fmm_status velocity_mode(fmm_handle h, int mode, int64_t n, const double *x, const double *y,
                                const double *g, double *u, double *v)
{
    fmm_status st = check_common(h, n, x, y, g, u, v);
    if (st != FMM_OK)
        return st;
    if ((st = poll_status(h, false)) != FMM_OK)
        return st;
    if (n == 0)
        return FMM_OK;
    set_single_system(h, n);
    return run_forward(h, mode, n, x, y, g, u, v);
}

fmm_status fmm_velocity(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma, double *u,
                        double *v)
{
    return velocity_mode(h, MODE_FULL, n, x, y, gamma, u, v);
}

fmm_status fmm_advect(fmm_handle h, int64_t n, double *x, double *y, const double *gamma, double dt, int nsteps,
                      int order)
{
    fmm_status st = check_common(h, n, x, y, gamma, x, y);
    if (st != FMM_OK)
        return st;
    if ((order != 2 && order != 4) || nsteps < 0 || !std::isfinite(dt))
        return set_err(h, FMM_EINVAL, "advect: order 2 or 4, nsteps >= 0, finite dt");
    if ((st = poll_status(h, false)) != FMM_OK)
        return st;
    if (n == 0 || nsteps == 0)
        return FMM_OK;
    const size_t need = (size_t)6 * (size_t)n;
    if (need > h->adv_cap) {
        if (h->adv)
            CU(cudaFree(h->adv));
        h->adv = nullptr;
        h->adv_cap = 0;
        if (cudaMalloc(&h->adv, need * sizeof(double)) != cudaSuccess)
            return set_err(h, FMM_ENOMEM, "advect scratch (%zu bytes)", need * sizeof(double));
        h->adv_cap = need;
    }
    double *tx = h->adv, *ty = tx + n, *su = ty + n, *sv = su + n, *au = sv + n, *av = au + n;
    static const double c2[2] = {0.0, 0.5}, b2[2] = {0.0, 1.0};
    static const double c4[4] = {0.0, 0.5, 0.5, 1.0}, b4[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const int S = order == 2 ? 2 : 4;
    const double *c = order == 2 ? c2 : c4, *b = order == 2 ? b2 : b4;
    for (int step = 0; step < nsteps; ++step) {
        // every stage evaluates at (tx, ty) -> (su, sv): the same pointers each time, so a graph replays
        CU(cudaMemcpyAsync(tx, x, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        CU(cudaMemcpyAsync(ty, y, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        for (int s = 0; s < S; ++s) {
            if ((st = velocity_mode(h, MODE_FULL, n, tx, ty, gamma, su, sv)) != FMM_OK)
                return st;
            h->launches += launch_rk_stage(n, x, y, tx, ty, su, sv, au, av, b[s], s + 1 < S ? c[s + 1] : 0.0, dt,
                                           s == 0, s + 1 == S, h->stream);
            CU(cudaGetLastError());
        }
    }
    return FMM_OK;
}

fmm_status fmm_velocity_near(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                             double *u, double *v)
{
    return velocity_mode(h, MODE_NEAR, n, x, y, gamma, u, v);
}

fmm_status fmm_velocity_far(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                            double *u, double *v)
{
    return velocity_mode(h, MODE_FAR, n, x, y, gamma, u, v);
}

fmm_status fmm_velocity_host(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                             double *u, double *v)
{
    fmm_status st = check_common(h, n, x, y, gamma, u, v);
    if (st != FMM_OK)
        return st;
    if ((st = poll_status(h, false)) != FMM_OK)
        return st;
    if (n == 0)
        return FMM_OK;
    size_t need = (size_t)n * 5 * sizeof(double);
    if (need > h->d_io_cap) {
        if (h->d_io) {
            CU(cudaDeviceSynchronize());
            CU(cudaFree(h->d_io));
            h->d_io = nullptr;
            h->d_io_cap = 0;
        }
        CU(cudaMalloc(&h->d_io, need));
        h->d_io_cap = need;
    }
    double *dx = h->d_io, *dy = dx + n, *dg = dy + n, *du = dg + n, *dv = du + n;
    size_t bytes = (size_t)n * sizeof(double);
    // Page-locked inputs in the precision form with an explicit square are read once, by the key kernel, so it
    // reads them in place over the host link (the same bytes cross it, without a copy in front of the kernel).
    const double *in[3] = {x, y, gamma};
    bool direct = h->mixed && h->has_domain && !h->adaptive_cap;
    for (int k = 0; k < 3 && direct; ++k) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, in[k]) != cudaSuccess || a.type != cudaMemoryTypeHost || !a.devicePointer)
            direct = false;
        else
            in[k] = (const double *)a.devicePointer;
    }
    (void)cudaGetLastError();  // a pageable pointer leaves no sticky error, but clear the attribute query's
    if (!direct) {
        CU(cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, h->stream));
        CU(cudaMemcpyAsync(dy, y, bytes, cudaMemcpyHostToDevice, h->stream));
        CU(cudaMemcpyAsync(dg, gamma, bytes, cudaMemcpyHostToDevice, h->stream));
        in[0] = dx;
        in[1] = dy;
        in[2] = dg;
    }
    // page-locked outputs are written in place by the uniform tree's final (caller-order, contiguous) sum kernel;
    // the adaptive tree's walk writes through the permutation (scattered), so its outputs take one copy each
    double *out[2] = {u, v};
    bool direct_out = h->adaptive_cap == 0;
    for (int k = 0; k < 2 && direct_out; ++k) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, out[k]) != cudaSuccess || a.type != cudaMemoryTypeHost || !a.devicePointer)
            direct_out = false;
        else
            out[k] = (double *)a.devicePointer;
    }
    (void)cudaGetLastError();
    if (!direct_out) {
        out[0] = du;
        out[1] = dv;
    }
    set_single_system(h, n);
    if ((st = run_forward(h, MODE_FULL, n, in[0], in[1], in[2], out[0], out[1])) != FMM_OK)
        return st;
    if (!direct_out) {
        CU(cudaMemcpyAsync(u, du, bytes, cudaMemcpyDeviceToHost, h->stream));
        CU(cudaMemcpyAsync(v, dv, bytes, cudaMemcpyDeviceToHost, h->stream));
    }
    CU(cudaStreamSynchronize(h->stream));
    return poll_status(h, true);
}

fmm_status fmm_velocity_batched(fmm_handle h, int nsys, const int64_t *offsets, const int *depths,
                                const double *sigmas, const double *domains, const double *x, const double *y,
                                const double *gamma, double *u, double *v)
{
    if (!h)
        return FMM_EINVAL;
    if (h->adaptive_cap)
        return set_err(h, FMM_EINVAL, "batched systems use the uniform tree (adaptive capacity is set)");
    if (nsys < 1 || nsys > FMM_MAXSYS || !offsets)
        return set_err(h, FMM_EINVAL, "nsys must be in [1, %d] and offsets given", FMM_MAXSYS);
    if (offsets[0] != 0)
        return set_err(h, FMM_EINVAL, "offsets[0] must be 0");
    for (int k = 0; k < nsys; ++k) {
        if (offsets[k + 1] < offsets[k])
            return set_err(h, FMM_EINVAL, "offsets must be non-decreasing");
        if (depths && (depths[k] < 0 || depths[k] > FMM_MAXL))
            return set_err(h, FMM_EINVAL, "depth of system %d out of range", k);
        if (sigmas && !(sigmas[k] > 0.0))
            return set_err(h, FMM_EINVAL, "sigma of system %d must be > 0", k);
        if (domains && !(domains[3 * k + 2] > 0.0))
            return set_err(h, FMM_EINVAL, "side of system %d must be > 0", k);
    }
    int64_t n = offsets[nsys];
    fmm_status st = check_common(h, n, x, y, gamma, u, v);
    if (st != FMM_OK)
        return st;
    if ((st = poll_status(h, false)) != FMM_OK)
        return st;
    if (n == 0)
        return FMM_OK;
    std::vector<SysHost> cfg(nsys);
    for (int k = 0; k < nsys; ++k) {
        SysHost &c = cfg[k];
        memset(&c, 0, sizeof c);
        c.p0 = offsets[k];
        c.np = offsets[k + 1] - offsets[k];
        c.depth = depths ? depths[k] : h->depth;
        c.sigma = sigmas ? sigmas[k] : h->sigma;
        c.explicit_domain = domains ? 1 : 0;
        if (domains) {
            c.dom[0] = domains[3 * k];
            c.dom[1] = domains[3 * k + 1];
            c.dom[2] = domains[3 * k + 2];
        }
    }
    if (h->sys_cfg.size() != cfg.size() || memcmp(h->sys_cfg.data(), cfg.data(), cfg.size() * sizeof(SysHost))) {
        h->sys_cfg = cfg;
        h->cfg_version++;
    }
    return run_forward(h, MODE_FULL, n, x, y, gamma, u, v);
}

fmm_status fmm_velocity_adjoint(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                                const double *gu, const double *gv, double *dgamma, double *dx, double *dy)
{
    fmm_status st = check_common(h, n, x, y, gamma, gu, gv);
    if (st != FMM_OK)
        return st;
    if (h->adaptive_cap)
        return set_err(h, FMM_EINVAL, "the adjoint uses the uniform tree (adaptive capacity is set)");
    if (h->tail_rings)
        return set_err(h, FMM_EINVAL, "the adjoint has no far-field tail correction (fmm_set_far_tail(h, 0))");
    if ((st = poll_status(h, false)) != FMM_OK)
        return st;
    if (n == 0)
        return FMM_OK;
    set_single_system(h, n);
    if ((st = ensure_tables(h)) != FMM_OK)
        return st;
    if ((st = ensure_workspace(h, n, 1)) != FMM_OK)
        return st;
    if ((st = upload_systems(h)) != FMM_OK)
        return st;
    Work &w = h->w;
    cudaStream_t s = h->stream;
    int64_t nl = 0;
    bool far = w.lv.maxdepth >= 2;
    CU(cudaMemsetAsync(w.cnt, 0, (size_t)(w.nleaf + 1) * sizeof(int), s));  // counts and overflow flag
    if (!h->has_domain) {
        nl += launch_bbox(w, x, y, s);
        nl += launch_domain_finalize(w, s);
    }
    nl += launch_keys(w, x, y, gamma, s);
    nl += launch_scan(w, s);
    nl += launch_scatter_sort(w, s);
    nl += launch_gather(w, x, y, gamma, gu, gv, s);
    if (far) {
        CU(cudaEventRecord(h->ev_fork, s));
        CU(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        for (int adj = 0; adj < 2; ++adj) {
            nl += launch_p2m(w, h->t, adj, h->side);
            for (int l = w.lv.maxdepth - 1; l >= 2; --l)
                nl += launch_m2m(w, h->t, l, adj, h->side, 1);
            nl += launch_m2l(w, h->t, adj, h->side, 1);
            for (int l = 2; l < w.lv.maxdepth; ++l)
                nl += launch_l2l(w, h->t, l, adj, h->side, 1);
        }
        nl += launch_adjoint_far(w, h->side);
        CU(cudaEventRecord(h->ev_join, h->side));
    }
    // near field written to the outputs first; the far part is added after the join
    nl += launch_adjoint_p2p(w, dgamma, dx, dy, h->adj_fp32, s);
    if (far) {
        CU(cudaStreamWaitEvent(s, h->ev_join, 0));
        nl += launch_adjoint_combine(w, dgamma, dx, dy, s);
    }
    CU(cudaMemcpyAsync(h->h_status, w.status, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CU(cudaEventRecord(h->ev_status, s));
    CU(cudaGetLastError());
    h->status_pending = 1;
    h->launches += nl;
    return FMM_OK;
}

static fmm_status check_level(fmm_handle h, int level)
{
    if (h->adaptive_cap)
        return set_err(h, FMM_EINVAL, "level exchange needs the uniform tree (adaptive capacity is set)");
    if (h->tail_rings)
        return set_err(h, FMM_EINVAL, "level exchange has no far-field tail correction (fmm_set_far_tail(h, 0))");
    if (!h->has_domain)
        return set_err(h, FMM_EINVAL, "level exchange needs an explicit root square shared by every part");
    if (level < 2 || level > h->depth)
        return set_err(h, FMM_EINVAL, "level must be in [2, depth = %d]", h->depth);
    return FMM_OK;
}

fmm_status fmm_level_multipoles(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                                int level, double *M_out, int64_t *count_out)
{
    fmm_status st = check_common(h, n, x, y, gamma, x, y);
    if (st != FMM_OK)
        return st;
    if ((st = check_level(h, level)) != FMM_OK)
        return st;
    if (!M_out || !count_out)
        return set_err(h, FMM_EINVAL, "NULL output");
    if ((st = poll_status(h, false)) != FMM_OK)
        return st;
    const size_t nb = (size_t)1 << (2 * level);
    if (n == 0) {
        CU(cudaMemsetAsync(M_out, 0, nb * h->p * 2 * sizeof(double), h->stream));
        CU(cudaMemsetAsync(count_out, 0, nb * sizeof(int64_t), h->stream));
        return FMM_OK;
    }
    set_single_system(h, n);
    if ((st = ensure_tables(h)) != FMM_OK || (st = ensure_workspace(h, n, 0)) != FMM_OK ||
        (st = upload_systems(h)) != FMM_OK)
        return st;
    Work &w = h->w;
    cudaStream_t s = h->stream;
    int64_t nl = 0;
    (void)cudaGetLastError();
    CU(cudaMemsetAsync(w.cnt, 0, (size_t)(w.nleaf + 1) * sizeof(int), s));  // counts and overflow flag
    nl += launch_keys(w, x, y, gamma, s);  // an explicit square: the host derived the constants
    nl += launch_scan(w, s);
    nl += launch_scatter_sort(w, s);
    nl += launch_gather(w, x, y, gamma, nullptr, nullptr, s);
    nl += launch_p2m(w, h->t, 0, s);
    for (int l = w.lv.maxdepth - 1; l >= level; --l)
        nl += launch_m2m(w, h->t, l, 0, s, 1);
    nl += launch_level_export(w, level, (double2 *)M_out, (long long *)count_out, s);
    CU(cudaMemcpyAsync(h->h_status, w.status, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CU(cudaEventRecord(h->ev_status, s));
    CU(cudaGetLastError());
    h->status_pending = 1;
    h->launches += nl;
    return FMM_OK;
}

fmm_status fmm_velocity_level(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                              int level, const double *M_in, const int64_t *count_in, double *u, double *v)
{
    fmm_status st = check_common(h, n, x, y, gamma, u, v);
    if (st != FMM_OK)
        return st;
    if ((st = check_level(h, level)) != FMM_OK)
        return st;
    if (!M_in || !count_in)
        return set_err(h, FMM_EINVAL, "NULL level arrays");
    h->ext_level = level;
    h->ext_M = (const double2 *)M_in;
    h->ext_cnt = (const long long *)count_in;
    st = velocity_mode(h, MODE_FULL, n, x, y, gamma, u, v);
    h->ext_level = 0;
    h->ext_M = nullptr;
    h->ext_cnt = nullptr;
    return st;
}

fmm_status fmm_selftest_timeout(fmm_handle h, int polls)
{
    if (!h || polls < 1 || polls > (1 << 20))
        return h ? set_err(h, FMM_EINVAL, "polls must be in [1, 2^20]") : FMM_EINVAL;
    fmm_status st;
    if ((st = poll_status(h, false)) != FMM_OK)
        return st;
    // the status word lives in the fixed header, which exists from fmm_create on
    Work w{};
    w.status = (unsigned int *)h->hdr;
    h->launches += launch_wait_timeout_selftest(w, polls, h->stream);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(h->h_status, w.status, sizeof(unsigned int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaEventRecord(h->ev_status, h->stream));
    h->status_pending = 1;
    return FMM_OK;
}

fmm_status fmm_set_adjoint_precision(fmm_handle h, fmm_precision mode)
{
    if (!h || (mode != FMM_FP64 && mode != FMM_MIXED))
        return FMM_EINVAL;
    h->adj_fp32 = mode == FMM_MIXED;
    return FMM_OK;
}

fmm_status fmm_sync(fmm_handle h)
{
    if (!h)
        return FMM_EINVAL;
    CU(cudaStreamSynchronize(h->stream));
    CU(cudaStreamSynchronize(h->side));
    CU(cudaStreamSynchronize(h->exec));
    return poll_status(h, true);
}

fmm_status fmm_set_timing(fmm_handle h, int enable)
{
    if (!h)
        return FMM_EINVAL;
    h->timing = enable == 2 ? 2 : (enable ? 1 : 0);
    return FMM_OK;
}

int fmm_stage_times(fmm_handle h, float *out, int cap)
{
    if (!h || !out || cap <= 0 || !h->last_timed)
        return 0;
    const unsigned m = h->timed_mask;
    if (cudaEventSynchronize(h->ev_t[(m >> 7) & 1u ? 7 : 5]) != cudaSuccess)  // the last event recorded
        return 0;
    auto el = [&](int a, int b) {
        float ms = 0.f;
        if (((m >> a) & 1u) && ((m >> b) & 1u) && cudaEventElapsedTime(&ms, h->ev_t[a], h->ev_t[b]) != cudaSuccess) {
            ms = 0.f;
            (void)cudaGetLastError();
        }
        return ms;
    };
    float v[8];
    v[0] = el(0, 1);
    v[1] = el(1, 5);
    v[2] = el(1, 2);
    v[3] = el(2, 3);
    v[4] = el(3, 4);
    v[5] = el(6, 7);
    v[6] = el(0, 7);
    v[7] = el(1, 6);
    int k = cap < 8 ? cap : 8;
    for (int i = 0; i < k; ++i)
        out[i] = v[i];
    return k;
}

fmm_status fmm_set_count_pairs(fmm_handle h, int enable)
{
    if (!h)
        return FMM_EINVAL;
    h->count_pairs = enable ? 1 : 0;
    return FMM_OK;
}

int64_t fmm_last_pair_count(fmm_handle h)
{
    if (!h || !h->pairs_valid)
        return -1;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess)
        return -1;
    return (int64_t)*h->h_pairs;
}

int64_t fmm_kernel_launches(fmm_handle h) { return h ? h->launches : -1; }

fmm_status fmm_get_params(fmm_handle h, int *tree_depth, int *p, double *sigma, int *p2p_threads,
                          int *p2p_targets_per_thread)
{
    if (!h)
        return FMM_EINVAL;
    if (tree_depth)
        *tree_depth = h->depth;
    if (p)
        *p = h->p;
    if (sigma)
        *sigma = h->sigma;
    if (p2p_threads)
        *p2p_threads = h->p2p_threads;
    if (p2p_targets_per_thread)
        *p2p_targets_per_thread = h->p2p_kt;
    return FMM_OK;
}

// Times fmm_velocity (median of 5 after 2 warm-up runs) for each candidate depth and tile and keeps the best.
fmm_status fmm_autotune(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma, double *u,
                        double *v, int depth_lo, int depth_hi)
{
    fmm_status st = check_common(h, n, x, y, gamma, u, v);
    if (st != FMM_OK)
        return st;
    if (depth_lo < 0 || depth_hi > FMM_MAXL || depth_lo > depth_hi)
        return set_err(h, FMM_EINVAL, "bad depth range");
    if (h->adaptive_cap)
        return autotune_adaptive(h, n, x, y, gamma, u, v, depth_lo, depth_hi);
    const char *cache = getenv("FMM2D_TUNE_CACHE");
    char keybuf[160];
    snprintf(keybuf, sizeof keybuf, "n=%lld p=%d mixed=%d sigma=%.17g lo=%d hi=%d", (long long)n, h->p, h->mixed,
             h->sigma, depth_lo, depth_hi);
    if (cache) {
        FILE *f = fopen(cache, "r");
        if (f) {
            char line[256];
            while (fgets(line, sizeof line, f)) {
                int d, th, kt, eng = h->m2l_engine;
                char *bar = strchr(line, '|');
                if (!bar)
                    continue;
                *bar = 0;
                if (strcmp(line, keybuf) == 0 && sscanf(bar + 1, "%d %d %d %d", &d, &th, &kt, &eng) >= 3) {
                    fclose(f);
                    h->depth = d;
                    if (eng == FMM_M2L_CUDA_CORES || eng == FMM_M2L_TENSOR)
                        h->m2l_engine = eng;
                    return fmm_set_p2p_tile(h, th, kt);
                }
            }
            fclose(f);
        }
    }
    int tiles[][2] = {{64, 4}, {128, 4}, {192, 4}, {128, 2}, {192, 2}, {64, 2}, {256, 2}, {256, 4}, {32, 4}, {32, 2}};
    int ntile = h->mixed ? 10 : 1;
    // candidates are timed the way the handle will run them: replayed graphs when the handle uses graphs (the
    // overlap of the near field with the sweep differs between eager launches and a graph)
    int save_timing = h->timing;
    h->timing = 0;
    float best = 1e30f;
    int bd = h->depth, bth = h->p2p_threads, bkt = h->p2p_kt;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    auto time_eval = [&]() -> float { return time_evaluation(h, n, x, y, gamma, u, v, e0, e1); };
    for (int d = depth_lo; d <= depth_hi; ++d) {
        for (int ti = 0; ti < ntile; ++ti) {
            h->depth = d;
            h->p2p_threads = tiles[ti][0];
            h->p2p_kt = tiles[ti][1];
            const float t = time_eval();
            if (t >= 0.f && t < best) {
                best = t;
                bd = d;
                bth = tiles[ti][0];
                bkt = tiles[ti][1];
            }
        }
    }
    h->depth = bd;
    h->p2p_threads = bth;
    h->p2p_kt = bkt;
    // M2L engine of the precision form's FP32 levels, at the chosen depth and tile
    int beng = h->m2l_engine;
    if (h->mixed && best < 1e30f) {
        float tb = 1e30f;
        for (int eng : {FMM_M2L_TENSOR, FMM_M2L_CUDA_CORES}) {
            h->m2l_engine = eng;
            const float t = time_eval();
            if (t >= 0.f && t < tb) {
                tb = t;
                beng = eng;
            }
        }
    }
    h->m2l_engine = beng;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->timing = save_timing;
    if (cache) {
        FILE *f = fopen(cache, "a");
        if (f) {
            fprintf(f, "%s|%d %d %d %d\n", keybuf, bd, bth, bkt, beng);
            fclose(f);
        }
    }
    if (best >= 1e30f)
        return set_err(h, FMM_ECUDA, "no candidate ran");
    return FMM_OK;
}

// Batched systems (config 4): the leaf occupancy (each system's depth from its particle count) and the near-field
// tile of the fastest fmm_velocity_batched, timed as the handle runs it (graph replays when it uses graphs).
fmm_status fmm_autotune_batched(fmm_handle h, int nsys, const int64_t *offsets, const double *sigmas,
                                const double *domains, const double *x, const double *y, const double *gamma,
                                double *u, double *v, int *depths_out)
{
    if (!h)
        return FMM_EINVAL;
    if (nsys < 1 || nsys > FMM_MAXSYS || !offsets || !depths_out)
        return set_err(h, FMM_EINVAL, "autotune_batched: nsys in [1, %d], offsets and depths_out given", FMM_MAXSYS);
    static const double targets[] = {16.0, 32.0, 48.0, 64.0, 96.0, 128.0};
    static const int tiles[][2] = {{64, 4}, {64, 2}, {256, 2}, {256, 4}, {128, 4}, {192, 4}, {192, 2}, {128, 2},
                                   {32, 4}, {32, 2}};
    const int ntile = h->mixed ? 10 : 1;
    std::vector<int> depths(nsys), best_depths(nsys);
    const int save_timing = h->timing;
    h->timing = 0;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    int bth = h->p2p_threads, bkt = h->p2p_kt;
    fmm_status st = FMM_OK;
    for (double tgt : targets) {
        for (int k = 0; k < nsys; ++k) {
            const double nk = (double)(offsets[k + 1] - offsets[k]);
            int d = nk > 0 ? (int)std::lround(std::log(nk / tgt) / std::log(4.0)) : 0;
            depths[k] = std::max(0, std::min(d, FMM_MAXL));
        }
        for (int ti = 0; ti < ntile; ++ti) {
            h->p2p_threads = tiles[ti][0];
            h->p2p_kt = tiles[ti][1];
            float ts[5];
            bool ok = true;
            for (int r = 0; r < 7 && ok; ++r) {
                ok = cudaEventRecord(e0, h->stream) == cudaSuccess &&
                     (st = fmm_velocity_batched(h, nsys, offsets, depths.data(), sigmas, domains, x, y, gamma, u, v)) ==
                         FMM_OK &&
                     cudaEventRecord(e1, h->stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
                if (ok && r >= 2)
                    cudaEventElapsedTime(&ts[r - 2], e0, e1);
            }
            if (!ok)
                break;
            std::sort(ts, ts + 5);
            if (ts[2] < best) {
                best = ts[2];
                best_depths = depths;
                bth = tiles[ti][0];
                bkt = tiles[ti][1];
            }
        }
        if (st != FMM_OK)
            break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->timing = save_timing;
    h->p2p_threads = bth;
    h->p2p_kt = bkt;
    if (st != FMM_OK)
        return st;
    if (best >= 1e30f)
        return set_err(h, FMM_ECUDA, "autotune_batched: no candidate ran");
    for (int k = 0; k < nsys; ++k)
        depths_out[k] = best_depths[k];
    return FMM_OK;
}

// Smallest p in [p_lo, p_hi] whose evaluation (the handle's form and tree) is within rel_tol of the FP64 form at
// p = FMM_PMAX on the same tree, in relative L2 over all particles. The truncation error of the expansions falls
// geometrically with p (§3's t-term expansions), so the first p that meets the target is the cheapest.
fmm_status fmm_autotune_p(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                          double rel_tol, int p_lo, int p_hi, double *achieved)
{
    fmm_status st = check_common(h, n, x, y, gamma, x, y);
    if (st != FMM_OK)
        return st;
    if (p_lo < 1 || p_hi > FMM_PMAX || p_lo > p_hi || !(rel_tol > 0.0))
        return set_err(h, FMM_EINVAL, "autotune_p: 1 <= p_lo <= p_hi <= %d and rel_tol > 0", FMM_PMAX);
    if (n == 0) {
        h->p = p_lo;
        if (achieved)
            *achieved = 0.0;
        return FMM_OK;
    }
    if ((st = poll_status(h, false)) != FMM_OK)
        return st;
    double *buf = nullptr, *sums = nullptr;
    CU(cudaMalloc(&buf, (size_t)4 * n * sizeof(double)));
    if (cudaMalloc(&sums, 2 * sizeof(double)) != cudaSuccess) {
        cudaFree(buf);
        return set_err(h, FMM_ENOMEM, "autotune_p: scratch");
    }
    double *ur = buf, *vr = buf + n, *u = buf + 2 * n, *v = buf + 3 * n;
    const int save_p = h->p, save_mixed = h->mixed, save_timing = h->timing;
    h->timing = 0;
    auto done = [&](fmm_status s) {
        cudaStreamSynchronize(h->stream);
        cudaFree(buf);
        cudaFree(sums);
        h->mixed = save_mixed;
        h->timing = save_timing;
        return s;
    };
    // reference: the plain FP64 form at the largest p
    h->mixed = 0;
    h->p = FMM_PMAX;
    if ((st = fmm_velocity(h, n, x, y, gamma, ur, vr)) != FMM_OK || (st = fmm_sync(h)) != FMM_OK) {
        h->p = save_p;
        return done(st);
    }
    h->mixed = save_mixed;
    int best = p_hi;
    double err = -1.0;
    for (int p = p_lo; p <= p_hi; ++p) {
        h->p = p;
        if ((st = fmm_velocity(h, n, x, y, gamma, u, v)) != FMM_OK) {
            h->p = save_p;
            return done(st);
        }
        double hs[2] = {0.0, 0.0};
        if (cudaMemsetAsync(sums, 0, 2 * sizeof(double), h->stream) != cudaSuccess) {
            h->p = save_p;
            return done(set_err(h, FMM_ECUDA, "autotune_p: memset"));
        }
        k_rel_l2_parts<<<152 * 4, 256, 0, h->stream>>>(n, u, v, ur, vr, sums);
        ++h->launches;
        if (cudaMemcpyAsync(hs, sums, sizeof hs, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            (st = fmm_sync(h)) != FMM_OK) {
            h->p = save_p;
            return done(st != FMM_OK ? st : set_err(h, FMM_ECUDA, "autotune_p: copy"));
        }
        err = hs[1] > 0.0 ? std::sqrt(hs[0] / hs[1]) : 0.0;
        if (err <= rel_tol) {
            best = p;
            break;
        }
    }
    h->p = best;
    if (achieved)
        *achieved = err;
    return done(FMM_OK);
}

const char *fmm_status_string(fmm_status s)
{
    switch (s) {
    case FMM_OK: return "ok";
    case FMM_EINVAL: return "invalid argument or particle outside the root square";
    case FMM_ENOMEM: return "out of memory";
    case FMM_ECUDA: return "CUDA error";
    case FMM_ETIMEOUT: return "device wait timed out";
    case FMM_EINTERNAL: return "device bounds check failed";
    }
    return "unknown status";
}

const char *fmm_last_error(fmm_handle h) { return h ? h->err.c_str() : "no handle"; }

}  // extern "C"

static float time_evaluation(fmm_handle h, int64_t n, const double *x, const double *y, const double *g, double *u,
                             double *v, cudaEvent_t e0, cudaEvent_t e1)
{
    float ts[5];
    for (int r = 0; r < 7; ++r) {
        if (cudaEventRecord(e0, h->stream) != cudaSuccess || fmm_velocity(h, n, x, y, g, u, v) != FMM_OK ||
            cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
            return -1.f;
        if (r >= 2)
            cudaEventElapsedTime(&ts[r - 2], e0, e1);
    }
    std::sort(ts, ts + 5);
    return ts[2];
}
