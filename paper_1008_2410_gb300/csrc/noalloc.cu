// noalloc.cu -- fmm_velocity_noalloc: one velocity evaluation that allocates no memory at all.
//
// Some callers cannot let a library call cudaMalloc: code running under another framework's memory manager
// (which owns the GPU's free memory and would see allocations it did not make), code inside a region where
// allocation is forbidden or would synchronise the device, or code with a fixed memory budget. For them this
// entry point keeps all of its scratch -- translation tables, system descriptor, status word, leaf histogram,
// leaf-ordered particle copies and expansion coefficients -- in one file-scope __device__ array of fixed size.
// The array exists on every GPU that loads the library, for the life of the process.
//
// Host code cannot use the array's name as a device address (on the host it is only a stand-in symbol), so
// the first call on each device looks the address up with cudaGetSymbolAddress, with that device current, and
// every later call on that device reuses it. That first call should therefore come before any stream capture.
//
// All calls share the array, so two calls whose work overlaps on the GPU (other streams, other host threads)
// race on it; what must start at zero (histogram, status word) is cleared by each call on its stream.
#include <cstring>
#include <mutex>
#include <vector>

#include "fmm2d.h"
#include "fmm_internal.cuh"

using namespace fmm;

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // 16 MiB per GPU
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceState {
    unsigned char *base = nullptr;  // device address of g_noalloc_scratch on this device
    int tables_p = -1;              // p the tables currently hold
};
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Fixed part at the start of the array: tables (p-dependent), then status, bounding box, system descriptor,
// per-level system list.
constexpr size_t kMat = 4 * FMM_PMAX * FMM_PMAX, kRho = FMM_NOFF * (2 * FMM_PMAX + 2), kBin = FMM_PMAX * FMM_PMAX;
constexpr size_t kTabSizes[8] = {kMat * 16, kMat * 16, kMat * 8, kMat * 8, kRho * 16, kRho * 8, kBin * 8, kBin * 4};

size_t tables_bytes()
{
    size_t t = 0;
    for (size_t s : kTabSizes)
        t += up256(s);
    return t;  // no tensor-core M2L operands: this entry runs the FP32 M2L levels on the CUDA cores
}

void carve_tables(unsigned char *b, Tables &t)
{
    size_t off = 0;
    void *p[8];
    for (int i = 0; i < 8; ++i) {
        p[i] = b + off;
        off += up256(kTabSizes[i]);
    }
    t.m2m64 = (double2 *)p[0];
    t.l2l64 = (double2 *)p[1];
    t.m2m32 = (float2 *)p[2];
    t.l2l32 = (float2 *)p[3];
    t.rho64 = (double2 *)p[4];
    t.rho32 = (float2 *)p[5];
    t.binom64 = (double *)p[6];
    t.binom32 = (float *)p[7];
    t.m2l_tc = nullptr;
}

// Host copies of the tables for one p; the copy into the device array is ordered on the caller's stream.
fmm_status upload_tables(const Tables &t, int p, cudaStream_t s)
{
    static std::vector<double2> m2m(kMat), l2l(kMat), rho(kRho);
    static std::vector<double> bin(kBin);
    static std::vector<float2> m2m32(kMat), l2l32(kMat), rho32(kRho);
    static std::vector<float> bin32(kBin);
    build_tables_host(p, m2m.data(), l2l.data(), rho.data(), bin.data());
    for (size_t i = 0; i < kMat; ++i) {
        m2m32[i] = make_float2((float)m2m[i].x, (float)m2m[i].y);
        l2l32[i] = make_float2((float)l2l[i].x, (float)l2l[i].y);
    }
    for (size_t i = 0; i < kRho; ++i)
        rho32[i] = make_float2((float)rho[i].x, (float)rho[i].y);
    for (size_t i = 0; i < kBin; ++i)
        bin32[i] = (float)bin[i];
    const void *src[8] = {m2m.data(), l2l.data(), m2m32.data(), l2l32.data(), rho.data(), rho32.data(), bin.data(),
                          bin32.data()};
    void *dst[8] = {t.m2m64, t.l2l64, t.m2m32, t.l2l32, t.rho64, t.rho32, t.binom64, t.binom32};
    for (int i = 0; i < 8; ++i)
        if (cudaMemcpyAsync(dst[i], src[i], kTabSizes[i], cudaMemcpyHostToDevice, s) != cudaSuccess)
            return FMM_ECUDA;
    // pageable sources: make sure the copies have read them before the static buffers are reused
    return cudaStreamSynchronize(s) == cudaSuccess ? FMM_OK : FMM_ECUDA;
}

// Carves the per-size arrays of one single-system evaluation out of `b`; returns the bytes used.
size_t carve_work(unsigned char *b, Work &w, int64_t n, int depth, int p, bool mixed)
{
    const int64_t nleaf = (int64_t)1 << (2 * depth);
    int64_t nbox = 0;
    for (int l = 2; l <= depth; ++l)
        nbox += (int64_t)1 << (2 * l);
    const size_t np = (size_t)n + 8;
    size_t off = 0;
    auto take = [&](size_t bytes) -> unsigned char * {
        unsigned char *q = bytes ? b + off : nullptr;
        off += up256(bytes);
        return q;
    };
    w.key = (int *)take(np * 4);
    w.slot = (int *)take(np * 4);
    w.cnt = (int *)take((size_t)nleaf * 4 + 16);
    w.start = (int *)take((size_t)(nleaf + 1) * 4 + 16);
    w.scan_tmp = (int *)take((size_t)((nleaf + 1023) / 1024 + 2) * 4);
    w.tmp = (int2 *)take(np * 8);
    w.big = (int *)take((size_t)(n / 129 + 2) * 4);
    w.perm = (int *)take(np * 4);
    w.iperm = (int *)take(np * 4);
    w.sleaf = (int *)take(np * 4);
    w.sx = (double *)take(mixed ? 0 : np * 8);
    w.sy = (double *)take(mixed ? 0 : np * 8);
    w.sg = (double *)take(mixed ? 0 : np * 8);
    unsigned char *e = take(mixed ? np * 48 : 0);
    w.eh = (float4 *)e;
    w.el = e ? w.eh + np : nullptr;
    w.eg = e ? w.el + np : nullptr;
    w.near64 = (double2 *)take(mixed ? 0 : np * 16);
    w.near32 = (float2 *)take(mixed ? np * 8 : 0);
    w.nf_stride = 1;
    w.bcount = (int *)take((size_t)nbox * 4 + 16);
    w.M64 = (double2 *)take((size_t)nbox * p * 16);
    w.L64 = (double2 *)take((size_t)nbox * p * 16);
    w.M32 = (float2 *)take(mixed ? (size_t)nbox * p * 8 : 0);
    w.L32 = (float2 *)take(mixed ? (size_t)nbox * p * 8 : 0);
    w.pos4u = (float4 *)take(mixed ? np * 32 : 0);
    w.rec64 = (Rec64 *)take(mixed ? 0 : np * 32);
    w.cls_off = (int *)take(mixed ? (size_t)nleaf * 32 + 16 : 0);
    w.cls8 = (unsigned char *)take(mixed ? np : 0);
    w.n = (int)n;
    w.nleaf = (int)nleaf;
    w.nbox = nbox;
    w.p = p;
    w.mixed = mixed ? 1 : 0;
    w.coarse_level = -1;
    w.nsys = 1;
    w.maxdepth = depth;
    return off;
}

}  // namespace

extern "C" fmm_status fmm_velocity_noalloc(int tree_depth, int p, double sigma, fmm_precision mode,
                                           const double *domain, int64_t n, const double *x, const double *y,
                                           const double *gamma, double *u, double *v, void *cuda_stream)
{
    if (tree_depth < 0 || tree_depth > FMM_MAXL || p < 1 || p > FMM_PMAX || !(sigma > 0.0) || n < 0 ||
        (mode != FMM_FP64 && mode != FMM_MIXED))
        return FMM_EINVAL;
    if (domain && !(domain[2] > 0.0))
        return FMM_EINVAL;
    if (n == 0)
        return FMM_OK;
    if (!x || !y || !gamma || !u || !v || n >= ((int64_t)1 << 31) - 64)
        return FMM_EINVAL;
    const bool mixed = mode == FMM_MIXED;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // sizes first (no device access): fixed part + per-size arrays must fit the array
    const size_t tab = up256(tables_bytes());
    const size_t hdr_status = 0, hdr_minmax = 256, hdr_sys = 512, hdr_list = hdr_sys + up256(sizeof(SysDev));
    const size_t hdr = hdr_list + up256((FMM_MAXL + 2) * sizeof(int));
    Work probe{};
    const size_t need = tab + hdr + carve_work(nullptr, probe, n, tree_depth, p, mixed);
    if (need > kScratchBytes)
        return FMM_EINVAL;  // larger than the fixed scratch: use fmm_velocity with a handle instead

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return FMM_ECUDA;
    unsigned char *base;
    Tables t{};
    {
        std::lock_guard<std::mutex> lk(g_mu);
        DeviceState &ds = g_dev[dev];
        if (!ds.base) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
                return FMM_ECUDA;
            ds.base = (unsigned char *)ptr;
        }
        base = ds.base;
        carve_tables(base, t);
        if (ds.tables_p != p) {
            // the tables are marked as holding p only once the upload has completed; a failed upload leaves
            // them marked stale, so the next call uploads again
            ds.tables_p = -1;
            if (upload_tables(t, p, s) != FMM_OK)
                return FMM_ECUDA;
            ds.tables_p = p;
        }
    }
    if (upload_m2l_constants(s) != 0)  // constant memory of the module, once per device (no allocation)
        return FMM_ECUDA;
    if (prepare_m2l_tc() != 0 || prepare_p2p() != 0)  // kernel attributes, once per device
        return FMM_ECUDA;

    unsigned char *h = base + tab;
    Work w{};
    carve_work(h + hdr, w, n, tree_depth, p, mixed);
    w.m2l_tc = 0;  // the default of a handle: FP32 M2L levels on the CUDA cores
    w.status = (unsigned int *)(h + hdr_status);
    w.pair_count = (unsigned long long *)(h + hdr_status + 32);
    w.big_cnt = (int *)(h + hdr_status + 64);
    w.minmax = (unsigned long long *)(h + hdr_minmax);
    w.sys = (SysDev *)(h + hdr_sys);
    w.sys_list = (int *)(h + hdr_list);
    LevelInfo lv{};
    lv.maxdepth = tree_depth;
    lv.mindepth2 = tree_depth >= 2 ? tree_depth : 0;
    int list[FMM_MAXL + 2];
    for (int l = 0; l <= FMM_MAXL + 1; ++l) {
        lv.first_at[l] = l;
        lv.nsys_at[l] = l <= tree_depth ? 1 : 0;
        list[l] = 0;
    }
    int64_t acc = 0;
    for (int l = 2; l <= tree_depth; ++l) {
        lv.m2l_item0[l] = acc;
        acc += (int64_t)1 << (2 * l);
    }
    if (tree_depth >= 2)
        lv.m2l_item0[tree_depth + 1] = acc;
    w.lv = lv;

    SysDev sd{};
    sd.p0 = 0;
    sd.np = n;
    sd.leaf0 = 0;
    for (int l = 0; l <= FMM_MAXL; ++l)
        sd.box0[l] = -1;
    int64_t box = 0;
    for (int l = 2; l <= tree_depth; ++l) {
        sd.box0[l] = box;
        box += (int64_t)1 << (2 * l);
    }
    sd.depth = tree_depth;
    sd.sigma = sigma;
    sd.explicit_domain = domain ? 1 : 0;
    sd.x0 = domain ? domain[0] : 0.0;
    sd.y0 = domain ? domain[1] : 0.0;
    sd.S = domain ? domain[2] : 1.0;

#define NA_CU(call)                         \
    do {                                    \
        if ((call) != cudaSuccess)          \
            return FMM_ECUDA;               \
    } while (0)
    NA_CU(cudaMemcpyAsync(w.sys, &sd, sizeof sd, cudaMemcpyHostToDevice, s));
    NA_CU(cudaMemcpyAsync(w.sys_list, list, sizeof list, cudaMemcpyHostToDevice, s));
    NA_CU(cudaMemsetAsync(w.status, 0, 64, s));
    NA_CU(cudaMemsetAsync(w.cnt, 0, (size_t)(w.nleaf + 1) * sizeof(int), s));
    // the same stages as fmm_velocity, in order on the caller's stream (no second stream, no events)
    if (!domain)
        launch_bbox(w, x, y, s);
    launch_domain_finalize(w, s);
    launch_keys(w, x, y, gamma, s);
    launch_scan(w, s);
    launch_scatter_sort(w, s);
    launch_gather(w, x, y, gamma, nullptr, nullptr, s);
    const bool far = tree_depth >= 2;
    if (far) {
        launch_p2m(w, t, 0, s);
        for (int l = tree_depth - 1; l >= 2; --l)
            launch_m2m(w, t, l, 0, s, 0);
        launch_m2l(w, t, 0, s, 0);
        for (int l = 2; l < tree_depth; ++l)
            launch_l2l(w, t, l, 0, s, 0);
    }
    launch_p2p(w, 64, 4, s);
    launch_combine(w, 1, far ? 1 : 0, u, v, s);
    NA_CU(cudaGetLastError());
    // wait, then report what the device found (a point outside the square, a timed-out copy, a bounds check)
    NA_CU(cudaStreamSynchronize(s));
    unsigned int st = 0;
    NA_CU(cudaMemcpy(&st, w.status, sizeof st, cudaMemcpyDeviceToHost));
#undef NA_CU
    if (st & FMM_DEV_BOUNDS)
        return FMM_EINTERNAL;
    if (st & FMM_DEV_TIMEOUT)
        return FMM_ETIMEOUT;
    if (st & FMM_DEV_OUTSIDE)
        return FMM_EINVAL;
    return FMM_OK;
}
