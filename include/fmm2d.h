/*
 * fmm2d.h -- C ABI of the GB300 (sm_103a) library for one Fast Multipole velocity evaluation of 2D
 * Gaussian vortex blobs (M. G. Knepley, "Removing the Barrier to Scalability in Parallel FMM").
 *
 * What one evaluation computes:
 *   u_i = sum_{j != i} gamma_j K_sigma(z_i - z_j)                                   (Eq. 7)
 *   K_sigma(z) = (-v, u) (1 - exp(-|z|^2 / 2 sigma^2)) / (2 pi |z|^2), z = (u, v)    (Eq. 6)
 * with the paper's FMM split (§2, last paragraph): the exact K_sigma between particles whose finest-level
 * leaves are equal or adjacent (stage 9 of Fig. 1), and the point-vortex kernel through p-term multipole
 * and local expansions (§3 coefficients, stages 4-8) for every other pair. Fig. 1's stages map to:
 *   1 root square (given, or the bounding-box rule below)  2 particle binning into leaves
 *   3 interaction lists (implicit on the uniform tree)     4 P2M  5 M2M  6 M2L  7 L2L  8 L2P
 *   9 near-field direct sum (P2P)                          10 sum of near and far parts
 * Stage 9 runs on the caller's stream while stages 4-7 run concurrently on a second, high-priority stream
 * (Fig. 1: no dependency between {4,5,6,7} and {9}). Stage 8 runs on that second stream too in the precision
 * form (the far field is ready at the join); in the plain FP64 form it is fused into stage 10 after the join.
 *
 * Conventions for every call:
 *   - Array arguments of fmm_velocity*, fmm_velocity_adjoint and fmm_velocity_batched are DEVICE pointers
 *     (cudaMalloc / torch CUDA tensors) of FP64 values, one value per particle, in the caller's order.
 *     fmm_velocity_host takes HOST pointers instead. The caller owns all arrays; the library never frees or
 *     keeps them past the call. Outputs are written in the caller's particle order.
 *   - The handle owns its scratch memory (grown on demand, freed by fmm_destroy), two CUDA streams' worth
 *     of events, and an optional CUDA graph of the whole evaluation.
 *   - Calls are asynchronous on the handle's stream (fmm_set_stream; default: the legacy default stream).
 *     Errors found on the host are returned at once. Errors found on the device (a point outside an explicit
 *     root square, a non-finite coordinate, an internal bounds check) are returned by fmm_sync or by the next
 *     call on the handle, as FMM_EINVAL or FMM_EINTERNAL.
 *   - n == 0 is a no-op that returns FMM_OK.
 *   - One handle must not be used by two host threads at once.
 *
 * Root square and leaves (the paper is silent; these are this library's rules, shared with its tests):
 *   - default square: centre of the particles' bounding box, side = extent * (1 + 2^-20) (at least 1e-300);
 *   - leaf column ix = floor((x - x0) * (2^L / S)) in IEEE double, clamped to [0, 2^L - 1] (likewise iy);
 *     a point on a leaf edge belongs to the upper leaf, x = x0 + S to the last leaf.
 */
#ifndef FMM2D_H
#define FMM2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_ctx *fmm_handle;

typedef enum {
    FMM_OK = 0,
    FMM_EINVAL = 1,    /* bad argument, or (device) a point outside the explicit square / non-finite */
    FMM_ENOMEM = 2,    /* device or pinned-host allocation failed */
    FMM_ECUDA = 3,     /* a CUDA runtime call failed; fmm_last_error has the CUDA message */
    FMM_ETIMEOUT = 4,  /* a bounded device-side wait (bulk-copy barrier) ran out */
    FMM_EINTERNAL = 5  /* a device-side bounds check failed */
} fmm_status;

typedef enum {
    FMM_FP64 = 0,  /* plain form: every stage in FP64 */
    FMM_MIXED = 1  /* precision form: FP32 near field (leaf-relative split coordinates, small-r series,
                      compensated sums), FP32 expansions; FP64 binning (bit-exact leaves) and, optionally,
                      FP64 coarse levels (fmm_set_coarse_level) */
} fmm_precision;

/* Creates a handle. tree_depth L in [0, 12] (4^L leaves; L <= 1 means every pair is near field),
 * p in [1, 32] expansion terms (§3's t), sigma > 0 the blob core (Eq. 2). *out is set on success. */
fmm_status fmm_create(int tree_depth, int p, double sigma, fmm_handle *out);

/* Frees the handle and everything it owns. NULL is accepted. Synchronises the handle's streams first. */
fmm_status fmm_destroy(fmm_handle h);

/* Fixes the root square [x0, x0 + side] x [y0, y0 + side] (side > 0). Points outside it make the
 * evaluation report FMM_EINVAL. fmm_clear_domain returns to the bounding-box rule. */
fmm_status fmm_set_domain(fmm_handle h, double x0, double y0, double side);
fmm_status fmm_clear_domain(fmm_handle h);

/* Chooses the plain FP64 form or the precision form (see fmm_precision). Default FMM_FP64. */
fmm_status fmm_set_precision(fmm_handle h, fmm_precision mode);

/* In the precision form, levels 2..coarse_level of M2M, M2L and L2L run in FP64 and finer levels in FP32.
 * Default -1: every level in FP32 (the radius-scaled translation matrices have entries bounded by 1/2, so the
 * coarse levels need no extra range; on GB300 an FP64 operation costs about 64 FP32 operations).
 * Ignored by FMM_FP64. */
fmm_status fmm_set_coarse_level(fmm_handle h, int coarse_level);

/* Where the FP32 levels of M2L (Fig. 1 stage 6, the translation b_l of §3) run in the precision form, on
 * radius-scaled coefficients: b_l = sum_m (-1)^(m+1) C(m+l, m) rho^(m+l+1) a_m, rho = 1/delta.
 * FMM_M2L_CUDA_CORES (default): one lane per (target, source) pair in FP32, the binomial contraction by prefix sums.
 * FMM_M2L_TENSOR: tcgen05 tensor-core MMAs (kind::tf32) with 256 target boxes per instruction: each offset's
 * 2p x 2p real translation matrix and the source multipoles both split into TF32 hi + lo (four products), the
 * sources of one child class read from a bulk-copied window of a per-class layout written by a first kernel;
 * levels up to 7 and p <= 20 (deeper levels and larger p take the CUDA-core kernel). Both agree with the FP64
 * form to below 1e-6 relative (a few 1e-7 on the CUDA cores, up to about 7e-7 on the tensor cores, whose FP32
 * accumulation runs over tens of MMAs). fmm_autotune times both and keeps the faster.
 * FP64 levels (the plain form, levels <= coarse_level) and the adjoint always use FP64 CUDA-core kernels.
 * Returns FMM_EINVAL for any other value. */
#define FMM_M2L_CUDA_CORES 0
#define FMM_M2L_TENSOR 1
fmm_status fmm_set_m2l_engine(fmm_handle h, int engine);

/* The handle's M2L engine (FMM_M2L_TENSOR or FMM_M2L_CUDA_CORES; fmm_autotune may change it), -1 for NULL. */
int fmm_get_m2l_engine(fmm_handle h);

/* Adaptive quadtree for uneven densities (the paper's closing section names them as the next step beyond its
 * uniform tree). leaf_capacity = 0 (default): the uniform tree of depth tree_depth. leaf_capacity = B > 0: the
 * tree is refined where the particles are: a box is split into its four children while it holds more than B
 * particles and its level is below tree_depth (now the maximum depth). Interactions follow the U, V, W, X
 * lists of Carrier, Greengard and Rokhlin: the exact K_sigma of Eq. 6 between particles of adjacent leaves
 * (U), M2L between same-level boxes whose parents are adjacent (V), multipoles of small boxes evaluated at the
 * particles of a larger adjacent-parent leaf (W) and the particles of a coarse leaf expanded into a small
 * box's local expansion (X). So the sum is Eq. 7 with K_sigma between adjacent leaves and the point-vortex
 * kernel elsewhere, as on the uniform tree. The adaptive evaluation has both forms: FMM_FP64 computes every
 * stage in FP64; FMM_MIXED keeps FP64 binning and sorted coordinates, evaluates the U-list pairs in FP32 on
 * split (hi + lo) coordinates (FP32 sums per source leaf, FP64 across leaves), and keeps the multipole and
 * local expansions (P2M, M2M, M2L, L2L, P2L, W-list and L2P evaluations) in FP32. It serves fmm_velocity,
 * fmm_velocity_near / _far, fmm_velocity_host and fmm_advect, and counts the ordered pairs of its U lists
 * when pair counting is on; fmm_autotune then picks the leaf capacity (and the
 * maximum depth within its range); fmm_velocity_batched and fmm_velocity_adjoint return FMM_EINVAL while it is set.
 * Returns FMM_EINVAL for NULL or a negative capacity. */
fmm_status fmm_set_adaptive(fmm_handle h, int leaf_capacity);

/* The handle's leaf capacity (0: uniform tree), -1 for NULL. */
int fmm_get_adaptive(fmm_handle h);

/* A tree depth for n particles in a root square of side `side` with blob core sigma (host only, no device
 * work): the occupancy depth round(log4(n / leaf_target)) (leaf_target <= 0: 64, the occupancy measured fastest
 * for the precision form on GB300), reduced until the leaf width w = side / 2^L keeps the Gaussian tail of the
 * nearest pair that goes through the expansions below tail_tol: exp(-w^2 / 2 sigma^2) <= tail_tol (§2: the far
 * field uses the point-vortex kernel, so that tail is left out of the sum). Returns the depth in [0, 12], or -1
 * for n <= 0, sigma <= 0, side <= 0 or tail_tol outside (0, 1). */
int fmm_suggest_depth(int64_t n, double sigma, double side, double tail_tol, double leaf_target);

/* Changes depth, p or sigma of an existing handle (same ranges as fmm_create). */
fmm_status fmm_set_params(fmm_handle h, int tree_depth, int p, double sigma);

/* Sets the stream every call is ordered on (a cudaStream_t; NULL = legacy default stream). */
fmm_status fmm_set_stream(fmm_handle h, void *cuda_stream);

/* Enables (1) or disables (0, default) capturing the evaluation into a CUDA graph that later calls with the
 * same sizes, pointers and parameters replay with one launch. */
fmm_status fmm_set_graph(fmm_handle h, int enable);

/* Near-field tile shape of the precision form: threads 32 (one leaf per thread block), 64 (two
 * horizontally adjacent leaves per block, sharing their source tiles), 256 (four such leaves, 128-thread
 * blocks; trees of depth >= 2, else as 64) or 128 (symmetric: each pair of
 * particles in adjacent leaves evaluated once and applied to both, one warp per leaf, four warps per block;
 * leaves wider than about 38 sigma still take the target-side kernel) or 192 (the 64-thread kernel with each
 * of the three source rows in its own block, summed at the end); targets_per_thread 2 or 4 (the most
 * targets one lane takes per pass; passes are balanced over the leaf). 0 = default (64, 4).
 * Set by fmm_autotune; exposed for experiments. */
fmm_status fmm_set_p2p_tile(fmm_handle h, int threads, int targets_per_thread);

/* Regularised far-field correction (§2, last paragraph: the FMM's far field uses the point-vortex kernel, which
 * misses the Gaussian tail of K_sigma for far pairs when the leaves are only a few sigma wide): adds
 * gamma_j (K_sigma - K_point)(z_i - z_j) = gamma_j (dy, -dx) exp(-r^2 / 2 sigma^2) / (2 pi r^2) over the sources
 * j whose leaves are 2 .. 1 + rings leaves from target i's leaf (Chebyshev leaf distance), after the near field;
 * the pairs still left to the point-vortex kernel are then at least (1 + rings) leaf widths w apart and miss at
 * most exp(-(1 + rings)^2 w^2 / 2 sigma^2) of their term. rings in [0, 8]; 0 (the default) turns it off. Uniform
 * tree only: an evaluation with it on an adaptive handle, the adjoint and the level exchange return FMM_EINVAL.
 * FP64 form in FP64 (exp), precision form in FP32 on the split coordinates. No counterpart in the paper's
 * kernels; the reading is the paper's kernel split made exact up to the stated tail. */
fmm_status fmm_set_far_tail(fmm_handle h, int rings);

/* Velocity of n particles (x, y, gamma device FP64 arrays) written to u, v (device FP64). Fig. 1 stages
 * 1-10 as described at the top of this file. */
fmm_status fmm_velocity(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                        double *u, double *v);

/* Same result from HOST arrays (pageable or pinned): copies the inputs into handle-owned device memory,
 * evaluates, copies u, v back and synchronises the stream before returning. Page-locked inputs of the
 * precision form with an explicit root square are not copied first: the key kernel, their only reader,
 * reads them in place over the host link; page-locked outputs are written in place by the final sum, which
 * writes in caller order. On the adaptive tree (fmm_set_adaptive) inputs and outputs are always copied. */
fmm_status fmm_velocity_host(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                             double *u, double *v);

/* The two halves of the FMM split on their own (same conventions as fmm_velocity):
 *   fmm_velocity_near -- stage 9 only: sum over particles in the same or adjacent leaves, exact K_sigma;
 *   fmm_velocity_far  -- stages 4-8 only: the expansions' point-vortex field of all other particles.
 * fmm_velocity == near + far, up to rounding. */
fmm_status fmm_velocity_near(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                             double *u, double *v);
fmm_status fmm_velocity_far(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                            double *u, double *v);

/* Adjoint (reverse-mode derivative) of fmm_velocity for a loss L with dL/du = gu, dL/dv = gv (device FP64):
 * writes dL/dgamma, dL/dx, dL/dy (device FP64; any output may be NULL to skip it). The far field's
 * transpose is evaluated exactly (the truncated far-field operator of this tree is antisymmetric), so finite
 * differences of fmm_velocity agree to rounding as long as no particle changes leaf. FP64 unless
 * fmm_set_adjoint_precision chose FP32 for the near-field part. */
fmm_status fmm_velocity_adjoint(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                                const double *gu, const double *gv, double *dgamma, double *dx, double *dy);

/* Precision of the adjoint's near-field part (its dominant cost: every adjacent pair with K_sigma's Jacobian).
 * FMM_FP64 (default): FP64 throughout, the exact transpose to rounding (finite differences of fmm_velocity agree
 * to rounding). FMM_MIXED: that part in FP32 on leaf-relative coordinates (the forward precision form's units; the
 * small-r factors of K_sigma and of its derivative from their series), FP64 sums across rows of leaves; systems
 * whose leaves are wider than about 38 sigma keep FP64; the far-field part stays FP64. Agrees with the FP64 adjoint
 * to about 1e-6 relative. */
fmm_status fmm_set_adjoint_precision(fmm_handle h, fmm_precision mode);

/* nsys independent systems in one evaluation (one launch per stage across all systems). offsets (HOST,
 * nsys + 1 entries, non-decreasing, offsets[0] = 0) delimit each system's particles in the device arrays.
 * depths (HOST, nsys entries, each in [0, 12]) and sigmas (HOST, nsys entries > 0) may be NULL to use the
 * handle's depth / sigma for every system. domains (HOST, 3 * nsys: x0, y0, side) may be NULL for the
 * bounding-box rule per system. p and the precision form are the handle's. */
fmm_status fmm_velocity_batched(fmm_handle h, int nsys, const int64_t *offsets, const int *depths,
                                const double *sigmas, const double *domains, const double *x, const double *y,
                                const double *gamma, double *u, double *v);

/* Particle advection, §2 Eq. 3: in 2D ideal flow the particles move with their velocity (Eq. 7, evaluated by
 * this handle's FMM in its current configuration) and keep their circulation. Runs nsteps explicit
 * Runge-Kutta steps of size dt, order 2 (the midpoint rule) or 4 (the classical scheme; the paper names no
 * integrator), each stage one evaluation. x, y: device arrays of n doubles in any order, updated in place;
 * gamma: device, unchanged. Scratch of 6 n doubles is owned by the handle and reused. With an explicit root
 * square, a particle that leaves it makes the next evaluation report FMM_EINVAL (device flag, seen by the
 * next call or fmm_sync). Asynchronous on the handle's stream. FMM_EINVAL for order other than 2 or 4,
 * nsteps < 0 or a non-finite dt. */
fmm_status fmm_advect(fmm_handle h, int64_t n, double *x, double *y, const double *gamma, double dt, int nsteps,
                      int order);

/* Waits for all work of the handle and returns the first device-side error since the last check. */
fmm_status fmm_sync(fmm_handle h);

/* Sharded evaluation (§3-§4: P processes each own the subtrees below a level k of the tree; the levels above k,
 * the "root tree", are formed from every process's level-k multipoles; each process's near field needs the
 * particles of the leaves next to its own). Both calls need the uniform tree, an explicit root square shared by
 * all parts (fmm_set_domain) and 2 <= level <= the handle's depth; FMM_EINVAL otherwise.
 *
 * fmm_level_multipoles: bins the given particles (device arrays, as fmm_velocity) and forms their multipoles
 * (P2M, then M2M up to `level`); writes the 4^level boxes of that level, row-major (box = iy 2^level + ix), p
 * complex coefficients each in the library's radius-scaled form (a_m scaled by w_level^-m, charges -i gamma) as
 * (re, im) doubles to M_out (DEVICE, 4^level * p * 2 doubles) and the boxes' particle counts to count_out (DEVICE,
 * 4^level int64). Boxes without particles give zeros. Asynchronous on the handle's stream.
 *
 * fmm_velocity_level: fmm_velocity of the given particles in which, once the upward pass has reached `level`, that
 * level's multipoles and counts are replaced by M_in and count_in (same layout, DEVICE): levels `level` and
 * coarser then stand for every particle those arrays sum (e.g. the sum over all parts of fmm_level_multipoles),
 * while finer levels and the near field use the given particles. A part that passes its own particles plus every
 * particle in the level-`level` boxes adjacent to its own gets, at its own particles, the velocity of the whole
 * system (the finer levels' interaction lists and the adjacent leaves of its boxes all lie in that neighbourhood);
 * results at the other particles are not meaningful. */
fmm_status fmm_level_multipoles(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                                int level, double *M_out, int64_t *count_out);
fmm_status fmm_velocity_level(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                              int level, const double *M_in, const int64_t *count_in, double *u, double *v);

/* Test of the device-side timeout path (the paper has no counterpart; it checks this library's failure
 * reporting). Launches, on the handle's stream, one thread that waits with the library's bounded mbarrier wait on
 * a barrier that nothing arrives on and no copy targets, giving up after `polls` polls (1 .. 2^20; each poll may
 * suspend the thread for a short hardware-defined time). The wait runs out, the status word gets the timeout bit,
 * and the next fmm_sync (or call on the handle) returns FMM_ETIMEOUT; the handle stays usable afterwards.
 * FMM_EINVAL for polls outside the range. */
fmm_status fmm_selftest_timeout(fmm_handle h, int polls);

/* Per-stage device times (ms) of the last evaluation when timing is on (fmm_set_timing(h, 1)); with graphs
 * (fmm_set_graph) the events are nodes of the graph, so every replay records them (each event node costs a few
 * microseconds of the evaluation). fmm_set_timing(h, 2), uniform tree: only the near field's two events, out[1]
 * (every other stage reads 0). Uniform tree: out[0]
 * binning, [1] near field, [2] up sweep (P2M+M2M), [3] M2L, [4] L2L (and L2P in the precision form, which
 * evaluates the far field on the sweep stream), [5] the final sum and scatter to input order (with L2P in the
 * plain form), [6] whole evaluation, [7] from the fork to the join (near field and sweep overlapped; in a
 * far-only evaluation the sweep alone). Adaptive tree: [0] binning, [1] from the fork to the end of the walk
 * (U, W, L2P) that follows the sweep, [2] box lists + P2L + P2M + M2M, [3] the downward L2L + M2L levels,
 * [5] the walk, [6] whole evaluation, [7] the sweep (fork to join). Stages an evaluation does not run read 0.
 * Returns the number of values written (at most cap). */
fmm_status fmm_set_timing(fmm_handle h, int enable);
int fmm_stage_times(fmm_handle h, float *out, int cap);

/* Number of ordered near-field pairs (i != j) of the last evaluation's tree (computed on the device when
 * counting is on: fmm_set_count_pairs(h, 1)). */
fmm_status fmm_set_count_pairs(fmm_handle h, int enable);
int64_t fmm_last_pair_count(fmm_handle h);

/* Number of kernels the library launched since the handle was created (graph replays count each kernel
 * node once per replay). */
int64_t fmm_kernel_launches(fmm_handle h);

/* Picks depth and near-field tile for the handle's p, sigma and precision by timing fmm_velocity on the given
 * particles (device arrays, left unchanged; u, v are scratch outputs). Tries depths depth_lo..depth_hi; in
 * the precision form it then times both M2L engines (fmm_set_m2l_engine) and keeps the faster. With a leaf
 * capacity set (fmm_set_adaptive) it instead times the adaptive tree with capacities 16, 24, 32, 48, 64, 96 and
 * 128 at each maximum depth depth_lo..depth_hi and keeps the fastest pair.
 * The choice is stored in the handle and, when the environment variable FMM2D_TUNE_CACHE names a file,
 * cached there keyed by (n, p, precision, tree kind). */
fmm_status fmm_autotune(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                        double *u, double *v, int depth_lo, int depth_hi);
fmm_status fmm_get_params(fmm_handle h, int *tree_depth, int *p, double *sigma, int *p2p_threads,
                          int *p2p_targets_per_thread);

/* Autotuner of batched evaluations (fmm_velocity_batched's arguments, depths excepted): times the batch with each
 * system's depth set for a leaf occupancy of 16, 32, 48, 64, 96 or 128 particles (depth = round(log4(N_k /
 * occupancy)), clamped to [0, 12]) and, in the precision form, each near-field tile of fmm_set_p2p_tile; keeps
 * the fastest. The tile is stored in the handle; the chosen depths are written to depths_out (HOST, nsys ints)
 * for the caller's later fmm_velocity_batched calls. u, v are scratch outputs. */
fmm_status fmm_autotune_batched(fmm_handle h, int nsys, const int64_t *offsets, const double *sigmas,
                                const double *domains, const double *x, const double *y, const double *gamma,
                                double *u, double *v, int *depths_out);

/* Picks the expansion order for an accuracy target (§3: the t-term expansions' truncation error falls
 * geometrically with t): evaluates the given particles (device arrays, left unchanged) once in the plain FP64
 * form at p = 32 as the reference, then in the handle's own form and tree at p = p_lo, p_lo + 1, ... and keeps
 * the first p whose result is within rel_tol of the reference in relative L2 over all particles (in the
 * precision form the FP32 rounding, a few 1e-7, is part of that error). Sets the handle's p (p_hi if no p in
 * [p_lo, p_hi] meets rel_tol) and writes the error of the chosen p to *achieved (may be NULL). Allocates and
 * frees 4 n doubles of device scratch; synchronises the handle's stream. FMM_EINVAL unless
 * 1 <= p_lo <= p_hi <= 32 and rel_tol > 0. */
fmm_status fmm_autotune_p(fmm_handle h, int64_t n, const double *x, const double *y, const double *gamma,
                          double rel_tol, int p_lo, int p_hi, double *achieved);

/* Measured throughput of the units the kernels are bound by, on the current device (a few hundred ms):
 * out[0] FP32 FMA TFLOP/s, out[1] FP64 FMA TFLOP/s, out[2] SFU ex2+rcp results per second / 1e12,
 * out[3] SM count; with cap >= 6 also out[4], out[5] clock cycles per tcgen05.mma kind::tf32 (M = 128, K = 8)
 * at N = 48 and N = 256, issued back to back by one thread per SM. cap >= 4. Allocates and frees 1 MiB of
 * device memory. */
fmm_status fmm_probe_peaks(double *out, int cap);

/* Allocation-free evaluation, for callers that cannot let a library allocate device memory (code running under
 * another framework's memory manager, inside an allocation-free region, or on a fixed memory budget). The paper
 * has no counterpart: this is a deployment variant of fmm_velocity. It needs no handle: depth, p, sigma, the form
 * (FMM_FP64 / FMM_MIXED) and the root square (domain = {x0, y0, side}, or NULL for the bounding-box rule) are
 * arguments; x, y, gamma, u, v are device arrays as for fmm_velocity; cuda_stream orders the work (NULL = legacy
 * default stream). All scratch lives in one fixed 16 MiB __device__ array that every GPU loading the library
 * holds until the process exits; it fits, for example, 65,536 particles at depth <= 6 with p <= 20 in either
 * form. Sizes that do not fit return FMM_EINVAL before any device work. Calls no cudaMalloc, cudaFree or other
 * allocating routine. The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current, so make that first call before any stream capture. Calls share the array: calls
 * whose work overlaps on the GPU race on it. Runs the stages one after another on the stream (no second stream),
 * waits for them, and returns device-detected errors (FMM_EINVAL for a point outside the square) directly. */
fmm_status fmm_velocity_noalloc(int tree_depth, int p, double sigma, fmm_precision mode, const double *domain,
                                int64_t n, const double *x, const double *y, const double *gamma, double *u,
                                double *v, void *cuda_stream);

/* Human-readable text of a status, and the last error message recorded on the handle. */
const char *fmm_status_string(fmm_status s);
const char *fmm_last_error(fmm_handle h);

#ifdef __cplusplus
}
#endif

#endif /* FMM2D_H */
