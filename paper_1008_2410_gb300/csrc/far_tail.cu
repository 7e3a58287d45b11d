// far_tail.cu -- the regularised far-field correction of the uniform tree (an option, off by default).
//
// The FMM's far field uses the point-vortex kernel (§2, last paragraph); for leaves only a few sigma wide the
// nearest far pairs miss the Gaussian tail of K_sigma. These kernels add, after the near field, the kernel
// difference over the sources a few leaves away (fmm_set_far_tail).
#include "fmm_internal.cuh"

namespace fmm {

#define TWO_PI 6.283185307179586476925

// Each target's near field gets the difference
// (K_sigma - K_point)(z) = (dy, -dx) exp(-r^2 / 2 sigma^2) / (2 pi r^2) over the sources whose leaves are 2 .. 1 +
// rings leaves away (Chebyshev distance); pairs farther apart are at least (1 + rings) leaf widths apart. A thread
// per target (the targets of a leaf share their source leaves, so a warp's loops agree).
__global__ void __launch_bounds__(128) k_far_tail64(Work w, int rings)
{
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= w.n)
        return;
    const int leaf = w.sleaf[pos];
    const int k = w.nsys == 1 ? 0 : find_sys_by_leaf(w.sys, w.nsys, leaf);
    const SysDev &d = w.sys[k];
    const int L = d.depth, ns = 1 << L, local = leaf - (int)d.leaf0, ix = local & (ns - 1), iy = local >> L;
    const double xt = w.sx[pos], yt = w.sy[pos], k2 = 1.0 / (2.0 * d.sigma * d.sigma);
    double au = 0.0, av = 0.0;
    for (int jy = max(iy - 1 - rings, 0); jy <= min(iy + 1 + rings, ns - 1); ++jy)
        for (int jx = max(ix - 1 - rings, 0); jx <= min(ix + 1 + rings, ns - 1); ++jx) {
            if (max(abs(jx - ix), abs(jy - iy)) < 2)
                continue;  // own and adjacent leaves: the near field's exact kernel already
            const int lf = (int)d.leaf0 + jy * ns + jx;
            for (int j = w.start[lf]; j < w.start[lf + 1]; ++j) {
                const double ax = xt - w.sx[j], ay = yt - w.sy[j], r2 = ax * ax + ay * ay;
                const double f = exp(-r2 * k2) / r2 * w.sg[j];
                au += ay * f;
                av -= ax * f;
            }
        }
    double2 &o = w.near64[pos];
    o.x += au / TWO_PI;
    o.y += av / TWO_PI;
}

// The precision form: leaf-relative split coordinates in units where exp(-r^2 / 2 sigma^2) = 2^-(r')^2, FP32
// (the correction is a small part of the velocity), added to the FP32 near field.
__global__ void __launch_bounds__(128) k_far_tail32(Work w, int rings)
{
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= w.n)
        return;
    const int leaf = w.sleaf[pos];
    const int k = w.nsys == 1 ? 0 : find_sys_by_leaf(w.sys, w.nsys, leaf);
    const SysDev &d = w.sys[k];
    const int L = d.depth, ns = 1 << L, local = leaf - (int)d.leaf0, ix = local & (ns - 1), iy = local >> L;
    const float s = d.s_unit;
    const float4 th = w.eh[pos], tl = w.el[pos];
    float au = 0.f, av = 0.f;
    for (int jy = max(iy - 1 - rings, 0); jy <= min(iy + 1 + rings, ns - 1); ++jy)
        for (int jx = max(ix - 1 - rings, 0); jx <= min(ix + 1 + rings, ns - 1); ++jx) {
            if (max(abs(jx - ix), abs(jy - iy)) < 2)
                continue;
            const int lf = (int)d.leaf0 + jy * ns + jx;
            const float ox = (float)(ix - jx) * s, oy = (float)(iy - jy) * s;  // between the two leaf centres
            for (int j = w.start[lf]; j < w.start[lf + 1]; ++j) {
                const float4 sh = w.eh[j], sl = w.el[j];
                const float dx = (th.x - sh.x + ox) + (tl.x - sl.x), dy = (th.z - sh.z + oy) + (tl.z - sl.z);
                const float r2 = dx * dx + dy * dy;
                const float f = w.eg[j].x * exp2f(-r2) / r2;
                au += dy * f;
                av -= dx * f;
            }
        }
    float2 *dst = w.p2p_rows ? w.nearp + pos : w.near32 + (int64_t)pos * w.nf_stride;  // rows: row 0's part
    dst->x += au * d.snear;
    dst->y += av * d.snear;
}

int launch_far_tail(const Work &w, int rings, cudaStream_t s)
{
    if (rings <= 0 || w.n == 0)
        return 0;
    if (w.mixed)
        k_far_tail32<<<(w.n + 127) / 128, 128, 0, s>>>(w, rings);
    else
        k_far_tail64<<<(w.n + 127) / 128, 128, 0, s>>>(w, rings);
    return 1;
}

}  // namespace fmm
