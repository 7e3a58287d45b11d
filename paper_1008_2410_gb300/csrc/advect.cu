// advect.cu -- Eq. 3 (2D Euler): the particles move with their velocity and keep their circulation. One
// explicit Runge-Kutta stage update after each velocity evaluation (order 2: the midpoint rule; order 4: the
// classical scheme), fused into one kernel over the particles in caller order:
//   A <- (first ? 0 : A) + b_s k_s;   last stage: z <- z + dt (A + b_s k_s);   else: t <- z + c_{s+1} dt k_s
#include "fmm_internal.cuh"

namespace fmm {

__global__ void k_rk_stage(int64_t n, double *__restrict__ x, double *__restrict__ y, double *__restrict__ tx,
                           double *__restrict__ ty, const double *__restrict__ u, const double *__restrict__ v,
                           double *__restrict__ au, double *__restrict__ av, double b, double c_next, double dt,
                           int first, int last)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const double ku = u[i], kv = v[i];
    const double su = (first ? 0.0 : au[i]) + b * ku, sv = (first ? 0.0 : av[i]) + b * kv;
    if (last) {
        x[i] += dt * su;
        y[i] += dt * sv;
    } else {
        au[i] = su;
        av[i] = sv;
        tx[i] = x[i] + c_next * dt * ku;
        ty[i] = y[i] + c_next * dt * kv;
    }
}

int launch_rk_stage(int64_t n, double *x, double *y, double *tx, double *ty, const double *u, const double *v,
                    double *au, double *av, double b, double c_next, double dt, int first, int last, cudaStream_t s)
{
    if (n <= 0)
        return 0;
    k_rk_stage<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, x, y, tx, ty, u, v, au, av, b, c_next, dt, first,
                                                           last);
    return 1;
}

}  // namespace fmm
