/*
 * steinicp.h -- C ABI of the GB300 Stein ICP library (libsteinicp.so).
 *
 * Stein ICP (Afzal Maken, Ramos, Ott, "Stein ICP for Uncertainty Estimation
 * in Point Cloud Matching") approximates the posterior over a 6-DoF rigid
 * pose theta = (x, y, z, roll, pitch, yaw) that maps a source cloud S into a
 * reference cloud R by K particles moved with Stein variational gradient
 * descent.  Each iteration (Sec. IV, summary paragraph):
 *   1. draws one minibatch of m source points (Sec. III-B),
 *   2. transforms it by every particle, s' = R(theta) s + u (Sec. III-A),
 *   3. finds each transformed point's nearest reference point
 *      (Eq. correspondences),
 *   4. averages the point-to-point cost gradient per particle
 *      (Eqs. trans_gradient, rotation_gradient),
 *   5. forms the Stein direction with RBF kernels whose bandwidths follow the
 *      median heuristic (Eq. stein_icp_phi and the kernels after it),
 *   6. moves the particles with Adam (Sec. V).
 *
 * Conventions shared by every call:
 *  - Points are float32, row-major [n][3], metres.
 *  - Particles are float32 [K][6] in the order (x, y, z, roll, pitch, yaw),
 *    metres and radians; R = Rz(yaw) Ry(pitch) Rx(roll).
 *  - `on_device` = 1: every array argument is a CUDA device pointer on the
 *    context's device; 0: every array argument is a host pointer.  Either way
 *    the call returns after its GPU work has finished (it synchronises the
 *    context's stream), so outputs are ready on return.
 *  - The caller owns every buffer it passes; the library only reads inputs and
 *    writes outputs, and keeps no pointer to them after the call returns.  The
 *    context owns its own device memory (reference structures, per-problem
 *    state, scratch), released by sicp_destroy.
 *  - Return value: SICP_OK (0) or a negative SICP_E* code.  On error the
 *    outputs are left untouched where the error is found before any output is
 *    written (all argument checks), and sicp_last_error() describes it.  No
 *    error path traps the GPU.
 *  - A context is not thread-safe: one host thread at a time per context.
 *  - Environment (for diagnosis; results do not change):
 *    SICP_NO_GRAPH runs the registration loop as plain launches instead of a
 *    captured CUDA graph; SICP_NO_PDL launches its kernels in plain stream
 *    order instead of with programmatic dependent launch (read once per
 *    process).
 */
#ifndef STEINICP_H
#define STEINICP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SICP_OK 0
#define SICP_EINVAL (-1)        /* bad size, pointer, mode or non-finite input */
#define SICP_ENOREF (-2)        /* no reference cloud set on the context (or no normals for
                                   SICP_POINT_TO_PLANE) */
#define SICP_ENOMEM (-3)        /* device allocation failed */
#define SICP_ECUDA (-4)         /* a CUDA runtime call failed */
#define SICP_ETIMEOUT (-5)      /* a bounded device wait gave up */
#define SICP_ENOSURROGATE (-6)  /* surrogate mode without a trained surrogate */

/* Nearest-neighbour search used for step 3. */
#define SICP_NN_BRUTE_FP32 0    /* exhaustive FP32 scan of the whole reference */
#define SICP_NN_BRUTE_BF16 1    /* exhaustive, BF16 tensor-core distance tiles + exact FP32 re-check;
                                   same results as SICP_NN_BRUTE_FP32 */
#define SICP_NN_GRID 2          /* uniform voxel grid, exact */
#define SICP_NN_SURROGATE 3     /* learned closest-point field, then exact grid */
/* Metric flag, OR-ed into the search mode of sicp_register (nn_mode) and
 * sicp_icp_grad (mode), with SICP_NN_GRID, SICP_NN_BRUTE_FP32 or
 * SICP_NN_BRUTE_BF16 (not with the learned field): the
 * point-to-plane error, which the paper uses for its method comparison and
 * trajectory errors without printing it.  Correspondences stay the nearest
 * reference point r (Eq. correspondences); the residual becomes
 * e = n . (R s + u - r) with n the unit normal at r, and gbar the gradient of
 * (1/2m) sum e^2 with r and n held fixed (the terms of Eqs. trans_gradient /
 * rotation_gradient with the residual vector replaced by e n).  Needs
 * sicp_reference_normals on the current reference. */
#define SICP_POINT_TO_PLANE 0x100
/* Flag for sicp_register (nn_mode), with an exact search: every particle j is
 * an independent SGD-ICP run (Sec. III-B) with its own minibatch stream (that
 * of seed + j) and Adam on its own log-posterior gradient, phi_j = G_j,
 * instead of the Stein coupling; particle j then evolves exactly as the
 * K = 1 run with seed + j.  This is the Monte Carlo reference distribution of
 * the paper's experiments: many SGD-ICP runs from spread initial poses.
 * Needs 4 K T m bytes of minibatch indices. */
#define SICP_INDEPENDENT 0x200

typedef struct sicp_ctx sicp_ctx;

/* Parameters of one registration run. */
typedef struct sicp_params {
    int32_t T;                 /* SVGD iterations (>= 0) */
    int32_t m;                 /* minibatch size, 1 <= m <= N (Sec. III-B) */
    float lr;                  /* Adam step size (Sec. V: 0.01 laser, 0.03 RGB-D) */
    float beta1, beta2, eps;   /* Adam constants (0.9, 0.999, 1e-8 when zero) */
    uint64_t seed;             /* minibatch stream seed */
    int32_t nn_mode;           /* SICP_NN_* */
    int32_t surrogate_iters;   /* SICP_NN_SURROGATE: iterations served by the surrogate */
    int32_t prior;             /* 0 uniform; 1 Gaussian translation + von Mises rotation */
    float prior_mu[6];         /* prior means (Eqs. trans_prior, rot_prior) */
    float prior_sigma[3];      /* translation prior divisor, printed as a variance */
    float prior_kappa[3];      /* von Mises concentrations */
    float surrogate_min_conf;  /* SICP_NN_SURROGATE: queries whose confidence is below this use the exact search */
} sicp_params;

/* Fill `p` with the defaults: T 100, m 100, lr 0.01, Adam (0.9, 0.999, 1e-8),
 * seed 0, SICP_NN_GRID, surrogate_iters 0, surrogate_min_conf 0.5, uniform
 * prior. */
void sicp_default_params(sicp_params* p);

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to run on (NULL: the library creates its own non-blocking stream). */
int sicp_create(sicp_ctx** out, int device, void* cuda_stream);

/* Release the context and all device memory it owns.  NULL is ignored. */
void sicp_destroy(sicp_ctx* ctx);

/* Message describing the last error on this context ("" if none). */
const char* sicp_last_error(const sicp_ctx* ctx);

/* Set the reference cloud R (Sec. III-A): xyz [M][3], M >= 1.  The library
 * copies it and builds its search structures (the voxel grid of
 * SICP_NN_GRID and the tile layout of the brute-force modes).
 * cell_size > 0 fixes the grid cell edge in metres; 0 picks it from the
 * cloud's extent and size.  Errors: SICP_EINVAL (M < 1, NULL, non-finite
 * coordinate, cell_size < 0), SICP_ENOMEM, SICP_ECUDA. */
int sicp_set_reference(sicp_ctx* ctx, const float* xyz, int64_t M, float cell_size, int on_device);

/* One full Stein ICP run (Sec. IV summary): source S = src_xyz [N][3],
 * initial particles particles_in [K][6], parameters `p`.  Outputs:
 * particles_out [K][6] after T iterations; mean6 [6] and cov36 [6][6]
 * (row-major, divisor K-1, zero for K = 1) of the final particles, both
 * float64 (may be NULL).  T = 0 returns the input particles and their
 * moments.  1 <= K <= 2048.  With SICP_NN_SURROGATE the first
 * min(surrogate_iters, T) iterations take their correspondences from the
 * trained surrogate (sicp_surrogate_train), each query falling back to the
 * exact grid search where the surrogate's confidence is below
 * surrogate_min_conf or the query lies outside the cube it was trained on;
 * the remaining iterations use the exact grid search.  Errors: SICP_EINVAL
 * (N < 1, K outside [1, 2048], m outside [1, N], T < 0, surrogate_iters < 0,
 * surrogate_min_conf outside [0, 1], bad mode, non-finite input),
 * SICP_ENOREF, SICP_ENOSURROGATE, SICP_ENOMEM, SICP_ECUDA, SICP_ETIMEOUT. */
int sicp_register(sicp_ctx* ctx, const float* src_xyz, int64_t N, const float* particles_in,
                  int32_t K, const sicp_params* p, float* particles_out, double* mean6,
                  double* cov36, int on_device);

/* Checkpoint / resume: T = p->T more iterations of a run that has done t0
 * iterations.  state [3][K][6] float32 (in/out) holds the particles, then the
 * Adam first and second moments; a new run starts from its initial particles
 * and zero moments with t0 = 0.  Iteration t of a run draws minibatch t of
 * p->seed and takes Adam step t + 1 whether the run is done in one call or
 * several, so continuing with t0 += T gives the particles of one longer call.
 * mean6, cov36 as sicp_register.  Errors as sicp_register, plus SICP_EINVAL
 * for t0 < 0 or t0 > 2^40 or a negative second moment.  A call rejected by
 * its argument checks leaves the context's run state (sicp_export_state)
 * as it was. */
int sicp_register_continue(sicp_ctx* ctx, const float* src_xyz, int64_t N, float* state, int32_t K,
                           int64_t t0, const sicp_params* p, double* mean6, double* cov36, int on_device);

/* The context's run state as bytes, for checkpoints that outlive the
 * context or the process.  After a finished sicp_register,
 * sicp_register_continue or sicp_resume, the context holds that run's K,
 * iterations done t, minibatch seed, particles and Adam moments.
 * sicp_export_state writes them to buf (host memory): "SICPRUN1", u32
 * version 1, i32 K, i64 t, u64 seed, float32 state [3][K][6] (particles,
 * first moments, second moments), u32 CRC-32 (IEEE polynomial, reflected)
 * of all bytes before it; host byte order; 36 + 72 K bytes.  With buf NULL
 * only *len is set to that size.  Errors: SICP_EINVAL (no finished run in
 * the context; *len smaller than needed, then *len is set to the size),
 * SICP_ECUDA.
 * sicp_import_state makes such bytes the context's run state (checked:
 * magic, version, size, checksum, 1 <= K <= 2048, finite values, second
 * moments >= 0); errors
 * SICP_EINVAL, SICP_ENOMEM, SICP_ECUDA.  A failed call leaves the context
 * without a run state. */
int sicp_export_state(sicp_ctx* ctx, void* buf, size_t* len);
int sicp_import_state(sicp_ctx* ctx, const void* buf, size_t len);

/* T = p->T more iterations of the context's run state (previous run, or
 * sicp_import_state): the same as sicp_register_continue with that state
 * and t0.  p->seed must be the run's seed.  particles_out [K][6] (may be
 * NULL), mean6, cov36 as sicp_register; the context's state moves on to
 * t0 + T.  Errors as sicp_register, plus SICP_EINVAL when the context has
 * no run state or the seed differs. */
int sicp_resume(sicp_ctx* ctx, const float* src_xyz, int64_t N, const sicp_params* p, float* particles_out,
                double* mean6, double* cov36, int on_device);

/* ---- many problems at once ---- */

/* P independent runs of sicp_register (Sec. IV summary) in one persistent
 * GPU launch, for serving many registrations at once.  Problem p has
 * reference points ref_xyz[ref_off[p] .. ref_off[p+1]) [3], source points
 * src_xyz[src_off[p] .. src_off[p+1]) [3] and particles
 * particles_in[part_off[p] .. part_off[p+1]) [6]; the offset arrays have
 * P+1 entries starting at 0 and are always host arrays.  All problems share
 * the parameters `p` (T, m, lr, Adam constants, prior) except the
 * minibatch stream: problem p uses seed p->seed + p.  p->nn_mode must be
 * SICP_NN_GRID.  Outputs: particles_out laid out like particles_in; mean6
 * [P][6] and cov36 [P][36] (may be NULL).  Each problem needs M >= 1,
 * N >= m and 1 <= K <= 2048.  Uses the grid cell-size factor and work-item
 * size set by sicp_autotune_batched (defaults 0.5 and 4).  Errors:
 * SICP_EINVAL, SICP_ENOMEM, SICP_ECUDA, SICP_ETIMEOUT (a bounded grid
 * barrier of the persistent kernel gave up). */
int sicp_register_batched(sicp_ctx* ctx, int32_t P, const int64_t* ref_off, const float* ref_xyz,
                          const int64_t* src_off, const float* src_xyz, const int32_t* part_off,
                          const float* particles_in, const sicp_params* p, float* particles_out,
                          double* mean6, double* cov36, int on_device);

/* Autotuner of the batched path (no counterpart in the paper): times
 * trial_iters iterations of the persistent kernel for each candidate grid
 * cell-size factor (0.35, 0.5, 0.7, 1.0 times the volumetric point spacing),
 * minibatch entries per work item (2, 4, 8) and CTA shape (1024 threads per
 * CTA, one CTA per SM, with the Stein phase's pair distances kept in shared
 * memory; or 512 or 256 threads, three or six CTAs per SM, without that
 * cache) on the given batch, keeps the fastest on the context for later
 * sicp_register_batched calls, and returns it (out_cta_threads: threads per
 * CTA; any out pointer may be NULL).  With cache_path (may be NULL) the
 * choice is read from / written to a small JSON file keyed by GPU name,
 * problem count, mean reference size and m.  Arguments otherwise as
 * sicp_register_batched. */
int sicp_autotune_batched(sicp_ctx* ctx, int32_t P, const int64_t* ref_off, const float* ref_xyz,
                          const int64_t* src_off, const float* src_xyz, const int32_t* part_off,
                          const float* particles_in, const sicp_params* p, int32_t trial_iters,
                          const char* cache_path, float* out_cell_factor, int32_t* out_points_per_item,
                          int32_t* out_cta_threads, int on_device);

/* Trace of one iteration of a batched run, for checking the persistent
 * kernel step by step against a plain implementation (no counterpart in the
 * paper).  sicp_trace_batched(ctx, t) arms the next sicp_register_batched
 * call on this context to record iteration t (0-based; t < 0 disarms; the
 * arming lasts one run): the particles and Adam moments the iteration starts
 * from, its correspondences, and the mean gradients and Stein directions of
 * its update.  sicp_read_batched_trace copies them to host arrays, all
 * problems' particles back to back as in particles_in: theta, adam_m,
 * adam_v, gbar, phi [sum K][6] float32 and nn [sum K][m] int32 (reference
 * indices within the problem, -1 for none); any may be NULL.  Errors:
 * SICP_EINVAL (no trace recorded since the last arming: the run failed, had
 * T <= t, or was an autotuning trial), SICP_ECUDA. */
int sicp_trace_batched(sicp_ctx* ctx, int32_t t);
int sicp_read_batched_trace(sicp_ctx* ctx, float* theta, float* adam_m, float* adam_v, int32_t* nn, float* gbar,
                            float* phi);

/* ---- single steps of the iteration, for users who drive the loop ---- */

/* Step 1 (Sec. III-B): the minibatches of iterations t0 .. t0+T-1 of the
 * stream `seed`: out_idx [T][m] int32, each row the m source indices in
 * [0, N) whose splitmix64 keys are smallest, in ascending index order.  The
 * key of index i at iteration t is output i+1 of a splitmix64 stream whose
 * state is output t+1 of a splitmix64 stream started at `seed`.
 * Errors: SICP_EINVAL (N < 1, m outside [1, N], T < 1, t0 < 0). */
int sicp_minibatch(sicp_ctx* ctx, uint64_t seed, int64_t t0, int32_t T, int64_t N, int32_t m,
                   int32_t* out_idx, int on_device);

/* Step 3 (Eq. correspondences): nearest reference point of each query
 * q [n][3] (float32) by search `mode` (SICP_NN_BRUTE_FP32, _BRUTE_BF16 or
 * _GRID).  out_idx [n] int32 reference indices (ties: lowest index), out_d2
 * [n] float32 squared distances (may be NULL).  All three modes return the
 * minimiser of the same float32 squared distance |q - r|^2.  SICP_NN_BRUTE_BF16
 * computes every query-point distance bound on the tensor cores from bf16
 * splits of the coordinates (about 16 significant bits) and re-checks in
 * float32 the points it cannot rule out.  n = 0 is a no-op.
 * Errors: SICP_EINVAL, SICP_ENOREF, SICP_ECUDA, SICP_ETIMEOUT. */
int sicp_nn(sicp_ctx* ctx, const float* q, int64_t n, int32_t mode, int32_t* out_idx,
            float* out_d2, int on_device);

/* Steps 2-4 (Eqs. trans_gradient, rotation_gradient): for K particles
 * [K][6] and one minibatch mb [m] of indices into src_xyz [N][3], the mean
 * gradient of L/2 per particle, out_gbar [K][6] float32, and optionally the
 * correspondences out_nn [K][m] int32 (may be NULL).  `mode` is
 * SICP_NN_BRUTE_FP32, SICP_NN_BRUTE_BF16 (K * m <= 2^26), SICP_NN_GRID or
 * SICP_NN_SURROGATE; the last takes each
 * correspondence from the trained surrogate (predicted nearest point
 * q + d) where its confidence is at least 0.5 and the query lies in the
 * trained cube, from the exact grid search otherwise, and needs
 * out_nn = NULL and K * m <= 2^24.  Errors as sicp_nn, plus
 * SICP_ENOSURROGATE and SICP_ETIMEOUT in surrogate mode. */
int sicp_icp_grad(sicp_ctx* ctx, const float* src_xyz, int64_t N, const int32_t* mb, int32_t m,
                  const float* particles, int32_t K, int32_t mode, float* out_gbar,
                  int32_t* out_nn, int on_device);

/* Steps 5-6 (Eq. stein_icp_phi, Sec. V): one Stein + Adam update in place.
 * particles, adam_m, adam_v: [K][6] float32 (in/out; Adam moments start at
 * zero); gbar [K][6] the mean gradients of this iteration; N the source
 * size that scales them (G = -N gbar + grad log prior); t the 1-based Adam
 * step; p supplies lr, Adam constants and the prior.  Optional outputs:
 * out_phi [K][6] the Stein direction, out_h [2] the translation and rotation
 * bandwidths.  Errors: SICP_EINVAL (K < 1, t < 1, N < 1), SICP_ETIMEOUT (the
 * CTAs that share one block's update wait for one another with a bounded
 * wait; nothing is written when it gives up). */
int sicp_stein_adam(sicp_ctx* ctx, float* particles, float* adam_m, float* adam_v,
                    const float* gbar, int32_t K, int64_t N, int64_t t, const sicp_params* p,
                    float* out_phi, float* out_h, int on_device);

/* Mean [6] and covariance [6][6] (divisor K-1; zero for K = 1) of K particles
 * [K][6], accumulated in float64.  Errors: SICP_EINVAL (K < 1). */
int sicp_moments(sicp_ctx* ctx, const float* particles, int32_t K, double* mean6, double* cov36,
                 int on_device);

/* Unit normals of the current reference for the point-to-plane metric: the
 * eigenvector of the smallest eigenvalue of the float64 covariance (divisor
 * k) of each point's k nearest reference points (itself included; ranked by
 * the library's fp32 squared distance, ties to the lower index).  The context
 * keeps them for SICP_POINT_TO_PLANE until the next sicp_set_reference.
 * out_normals ([M][3] float32, original order, may be NULL) receives a copy;
 * a normal's sign is arbitrary (the metric does not depend on it).  Errors:
 * SICP_ENOREF (no reference), SICP_EINVAL (k outside [3, min(32, M)]),
 * SICP_ENOMEM, SICP_ECUDA. */
int sicp_reference_normals(sicp_ctx* ctx, int32_t k, float* out_normals, int on_device);

/* Distribution quality (no context; float64).  The paper scores a pose
 * distribution against its Monte Carlo reference (SICP_INDEPENDENT runs from
 * spread initial poses) by the KL divergence, computed from the samples'
 * covariances, and by the overlapping coefficient (OVL).  Both act on the
 * Gaussians N(mean0, cov0) and N(mean1, cov1) of dimension d (1..64;
 * covariances row-major d x d, symmetric positive definite).
 * sicp_gaussian_kl: *out = KL(N0 || N1) = 1/2 [tr(S1^-1 S0) + (m1 - m0)^T
 * S1^-1 (m1 - m0) - d + ln det S1 - ln det S0].
 * sicp_gaussian_ovl: *out = the integral of min(p0, p1), estimated from the
 * caller's standard-normal draws z0, z1 ([n][d] each, n >= 1) as 1/2 [mean
 * over x = m0 + L0 z0 of min(1, p1(x)/p0(x)) + mean over x = m1 + L1 z1 of
 * min(1, p0(x)/p1(x))], L the Cholesky factors; 1 for identical Gaussians.
 * Errors: SICP_EINVAL (null pointer, d or n out of range, a non-finite value,
 * a covariance that is not positive definite). */
int sicp_gaussian_kl(const double* mean0, const double* cov0, const double* mean1, const double* cov1,
                     int32_t d, double* out);
int sicp_gaussian_ovl(const double* mean0, const double* cov0, const double* mean1, const double* cov1,
                      int32_t d, const double* z0, const double* z1, int64_t n, double* out);

/* Odometry chaining (no context; host arrays; float64).  The paper's odometry
 * experiment multiplies consecutive scan-to-scan mean transforms, T_E =
 * T^1_0 T^2_1 ... T^l_(l-1), and combines their covariances to fourth order
 * (an approximation it cites, not prints).  A pose distribution is a mean
 * pose T (4 x 4 row-major, [C r; 0 1]) and the 6 x 6 row-major covariance of
 * the left perturbation xi = [rho; phi] in exp(xi^) T.
 * sicp_pose_distribution: the distribution of K particles [K][6] (x, y, z,
 * roll, pitch, yaw; C = Rz Ry Rx): the mean pose where their perturbations
 * average to zero (fixed-point iteration from the pose of the mean
 * parameters, angles by circular mean) and the sample covariance of the
 * perturbations (divisor K - 1; zero for K = 1).
 * sicp_compound: the distribution of T1 T2 for independent distributions 1
 * and 2: mean T1 T2; covariance S1 + Ad(T1) S2 Ad(T1)^T (order 2) plus the
 * fourth-order terms (order 4).
 * Errors: SICP_EINVAL (null pointer, K outside [1, 2^20], order not 2 or 4,
 * a non-finite value, a T that is not a rigid transform to 1e-6). */
int sicp_pose_distribution(const float* particles, int32_t K, double* T_mean, double* cov);
int sicp_compound(const double* T1, const double* cov1, const double* T2, const double* cov2, int32_t order,
                  double* T_out, double* cov_out);

/* The same moments with circular statistics for the three angles, for
 * particle sets whose rotations straddle +-pi (the plain mean of angles near
 * pi and -pi lands near 0).  Mean of angle a: atan2(sum_j sin theta_j,a,
 * sum_j cos theta_j,a), 0 when both sums vanish; covariance [6][6] of the
 * deviations [theta_t - mean_t ; wrap(theta_r - mean_r)], wrap(x) =
 * atan2(sin x, cos x), divisor K-1 (zero for K = 1); translations as
 * sicp_moments.  The paper uses the particles' mean and covariance
 * downstream (the odometry subsection of the experiments) and gives no
 * formula for angles; this is the standard circular mean.  Float64
 * throughout.  Errors: SICP_EINVAL (K < 1). */
int sicp_moments_circular(sicp_ctx* ctx, const float* particles, int32_t K, double* mean6, double* cov36,
                          int on_device);

/* ---- allocation-free variant ---- */

/* The mean ICP gradient of sicp_icp_grad with SICP_NN_BRUTE_FP32, for
 * callers that cannot allocate device memory.  Examples are code that runs
 * inside a fixed pre-allocated memory budget, a real-time loop where any
 * cudaMalloc/cudaFree would stall or is forbidden, and a host process whose
 * allocator belongs to another framework.  There is no counterpart in the
 * paper: this is a deployment variant of the same computation.
 *
 * No context is needed and nothing is allocated.  All array arguments are
 * device pointers on the current device: reference ref_xyz [M][3], source
 * src_xyz [N][3], minibatch mb [m] (indices into the source; the device
 * values are not checked on the host, and an entry outside [0, N) reads
 * nothing and adds nothing to the sum, which is still divided by m),
 * particles [K][6]; the result goes to out_gbar [K][6].  The work is queued
 * on `cuda_stream` (NULL: the legacy default stream) and the call returns
 * without waiting.
 *
 * Scratch: the kernel's partial sums and arrival counters live in one
 * file-scope device array of 25,600 bytes that every GPU loading this library
 * holds until the process exits.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) for that device and keeps it
 * for the life of the process; make that first call before any stream
 * capture.  A device reset (cudaDeviceReset, or the primary context torn
 * down and created again) invalidates the kept address and is not supported
 * while the library is loaded.  Each call clears the counters itself.
 * Calls share the array, so calls that overlap on the GPU (on two streams,
 * or from two threads) race and must be serialised by the caller.
 *
 * Limits: K <= 256, m <= 1024, M <= 2^30, N <= 2^31 - 1.  Returns SICP_OK,
 * SICP_EINVAL (a NULL pointer or a size outside these limits; nothing is
 * launched), or SICP_ECUDA (no current device, or a failed launch). */
int sicp_icp_grad_noalloc(const float* ref_xyz, int64_t M, const float* src_xyz, int64_t N,
                          const int32_t* mb, int32_t m, const float* particles, int32_t K,
                          float* out_gbar, void* cuda_stream);

/* ---- learned closest-point field (no counterpart in the paper) ----
 *
 * A small network that stands in for step 3 during the early iterations:
 * for a query q it predicts the displacement d from q to its nearest
 * reference point and a confidence c in (0, 1).  With c = (cx, cy, cz) the
 * centre of the reference bounding box and s = 0.6 x its largest extent,
 * q~ = (q - c) / s; the input features (112) are q~, then sin and cos of
 * w_f q~_a for w_f = pi 2^(8f/15), f = 0..15, a = x, y, z (feature
 * 3 + 6f + 2a is the sine, the next one the cosine), then zeros.  Layers:
 * x -> h1 = relu(W1 x + b1) (128) -> h2 = relu(W2 h1 + b2) (128) ->
 * o = W3 h2 + b3 (16); d = s (o0, o1, o2), c = sigmoid(o3); outputs 4..15
 * are unused.  Parameters are float32, flat, in the order W1 [128][112],
 * b1 [128], W2 [128][128], b2 [128], W3 [16][128], b3 [16]: 33,040 values.
 * The GPU computes with bf16 weights, features and activations and float32
 * accumulation (fifth-generation tensor cores).
 *
 * Training loss per sample (normalised units, targets d~* = (r - q) / s of
 * the exact nearest reference point r):
 *   |d~ - d~*|^2 + lam (softplus(o3) - c* o3),  c* = exp(-|d~ - d~*|^2 / delta^2)
 * with c* held constant in the gradient; lam = 0.1 and delta = 0.01 in
 * sicp_surrogate_train. */

/* Train the surrogate of the context's reference cloud.  Draws n_queries
 * (rounded down to a multiple of batch) queries from the counter-based stream
 * `seed`: even ones are reference points plus normal offsets whose standard
 * deviation per axis is log-uniform in [0.002 s, 0.1 s], odd ones uniform in
 * the cube |q~| <= 1; labels them with the exact
 * grid search; initialises the weights (He-normal from the same seed) and
 * runs `epochs` passes of Adam (lr, 0.9, 0.999, 1e-8) over batches of `batch`
 * samples in a fixed order.  out_loss (may be NULL): mean batch loss of the
 * last epoch.  The surrogate stays valid until the next sicp_set_reference.
 * Errors: SICP_EINVAL (n_queries outside [128, 2^26], epochs outside
 * [1, 1e5], batch not a multiple of 128 in [128, 65536], lr <= 0),
 * SICP_ENOREF, SICP_ENOMEM, SICP_ECUDA, SICP_ETIMEOUT. */
int sicp_surrogate_train(sicp_ctx* ctx, int64_t n_queries, uint64_t seed, int32_t epochs, int32_t batch,
                         float lr, float* out_loss);

/* sicp_surrogate_train with the training queries that a registration run
 * puts to the search: n_queries source points s drawn uniformly from
 * src_xyz [N][3], each moved by a pose theta drawn uniformly from the
 * axis-aligned box that the run's initial particles [K][6] span,
 * q = R(theta) s + u, labelled by the exact grid search.  The particles of
 * the early iterations, where the surrogate stands in for the search, move
 * inside that box towards the answer.  Everything else (normalisation,
 * initial weights from `seed`, epochs, batches, Adam, out_loss) as
 * sicp_surrogate_train.  on_device as everywhere.  Errors as
 * sicp_surrogate_train, plus SICP_EINVAL for N outside [1, 2^31 - 1], K
 * outside [1, 2048] or a non-finite input. */
int sicp_surrogate_train_run(sicp_ctx* ctx, const float* src_xyz, int64_t N, const float* particles, int32_t K,
                             int64_t n_queries, uint64_t seed, int32_t epochs, int32_t batch, float lr,
                             float* out_loss, int on_device);

/* Read (set = 0) or replace (set = 1) the surrogate's parameters: params
 * [33040] float32 in the layout above, norm4 = (cx, cy, cz, s); host arrays.
 * Setting marks the surrogate trained.  Errors: SICP_EINVAL (NULL,
 * non-finite value, s <= 0), SICP_ENOSURROGATE (reading before any
 * surrogate exists), SICP_ENOMEM, SICP_ECUDA. */
int sicp_surrogate_params(sicp_ctx* ctx, int set, float* params, float* norm4);

/* The training kernels' loss and gradient for given parameters [33040] on
 * n normalised queries qn [n][3] with targets dstar [n][3] (host arrays):
 * out_loss (may be NULL) the mean loss, out_grad [33040] its gradient with
 * respect to the parameters.  The context's own surrogate is left unchanged.
 * n a multiple of 128 in [128, 65536].  Errors: SICP_EINVAL, SICP_ENOMEM,
 * SICP_ECUDA, SICP_ETIMEOUT. */
int sicp_surrogate_loss_grad(sicp_ctx* ctx, const float* params, const float* qn, const float* dstar,
                             int64_t n, float lam, float delta, float* out_loss, float* out_grad);

/* Save the context's surrogate (parameters and normalisation) to `path`, or
 * load one saved there (which marks it trained on this context).  The file is
 * "SICPSURR", u32 version 1, u32 parameter count 33040, float norm4[4], float
 * params[33040], u32 FNV-1a checksum of the bytes between the magic and the
 * checksum, all little-endian.  Loading checks size, magic, version, count,
 * checksum and finiteness.  Errors: SICP_EINVAL (unreadable or corrupt file),
 * SICP_ENOSURROGATE (saving without a surrogate), SICP_ECUDA. */
int sicp_surrogate_save(sicp_ctx* ctx, const char* path);
int sicp_surrogate_load(sicp_ctx* ctx, const char* path);

/* Surrogate inference: for queries q [n][3] (metres) the predicted
 * displacement out_disp [n][3] (metres; the predicted nearest point is
 * q + d) and confidence out_conf [n].  n = 0 is a no-op.  Errors:
 * SICP_EINVAL, SICP_ENOSURROGATE, SICP_ECUDA, SICP_ETIMEOUT. */
int sicp_surrogate_infer(sicp_ctx* ctx, const float* q, int64_t n, float* out_disp, float* out_conf,
                         int on_device);

/* ---- measurement ---- */

/* Work counters of the searches (no counterpart in the paper; they state
 * the algorithmic bytes a search moved).  Copies the counters accumulated
 * since the previous call into out10 (may be NULL): grid search queries, rows
 * examined (one row span each), row segments read (two cell offsets each),
 * candidate points read (16 bytes each), queries that went on to the coarse
 * level, queries that went on to the exhaustive scan, queries put to the
 * surrogate, surrogate queries sent on to the exact search, query tiles of
 * the tensor-core search (128 queries each), reference tiles those query
 * tiles swept (256 points each; the others were ruled out by their bounding
 * boxes); then zeroes them and turns counting on (enable = 1) or off.
 * Counting adds a few warp-aggregated atomics per 32 lanes. */
int sicp_stats(sicp_ctx* ctx, int enable, uint64_t* out10);

/* Kernel timing inside sicp_register (no counterpart in the paper).  With
 * stride s > 0 the captured loop records CUDA events around the gradient and
 * Stein kernels of every s-th iteration; their durations are summed on the
 * host while the next run executes.  Copies the totals since the previous
 * call into out4 (may be NULL): gradient-kernel ms, gradient launches timed,
 * Stein-kernel ms, Stein launches timed; then zeroes them and sets the
 * stride (0 = off).  While the stride is > 0, each sicp_register_batched call
 * adds its one persistent launch (all T iterations, with the minibatch draw
 * before it and the moments after it) to the gradient-kernel totals.
 * Synchronises the context's stream. */
int sicp_profile(sicp_ctx* ctx, int stride, double* out4);

/* Per-iteration telemetry (no counterpart in the paper).  With on = 1 every
 * later registration run of the context (sicp_register,
 * sicp_register_continue, sicp_resume; not the batched path) records one row
 * of 16 float32 per iteration t, kept on the device until the next run:
 *   [0..5]   mean of the six pose parameters of the particles the iteration
 *            starts from (the arithmetic mean, as sicp_moments),
 *   [6..11]  their standard deviations (divisor K-1; 0 for K = 1),
 *   [12]     mean Euclidean distance from the iteration's K m transformed
 *            minibatch points to their correspondences (Eq.
 *            correspondences; in iterations on the learned field, the
 *            residual the field or its exact fallback gave),
 *   [13]     share of the iteration's queries the learned field answered
 *            (0 in exact iterations),
 *   [14]     the iteration's absolute index (t0 + t),
 *   [15]     share of the queries that had a correspondence (1 unless a
 *            transformed point was non-finite).
 * It adds two small launches per iteration (sicp_profile's Stein times
 * include them) and the exact searches' correspondence writes; the run's
 * results are unchanged, bit for bit.  on = 0 turns it off.  Errors:
 * SICP_EINVAL (null ctx). */
int sicp_set_telemetry(sicp_ctx* ctx, int on);

/* Copies at most max_rows rows of the last run's telemetry to out
 * [rows][16] float32 (host memory); *rows (may be NULL) receives the number
 * of rows that run recorded: its T, or 0 when telemetry was off or the run
 * did not finish.  Errors: SICP_EINVAL (max_rows < 0, or out NULL with
 * max_rows > 0). */
int sicp_read_telemetry(sicp_ctx* ctx, float* out, int32_t max_rows, int32_t* rows);

/* ---- resource limits and failure detection (no counterpart in the paper) ---- */

/* Device memory budget of a context: from now on an allocation that would
 * take the bytes the context holds in its growable buffers (reference and
 * its search structures, per-run state, scratch of every path) above `bytes`
 * fails, and the call that needed it returns SICP_ENOMEM before it launches
 * anything or writes any output.  0 removes the budget.  Buffers already
 * held are kept and counted.  *held (may be NULL) receives the bytes held
 * now.  A failed allocation can leave the context without its reference or
 * run state (it frees the smaller buffer it was replacing first); set the
 * reference again.  Never fails for a valid context. */
int sicp_set_memory_limit(sicp_ctx* ctx, size_t bytes, size_t* held);

/* Failure-detection check of the device waits.  Several kernels wait on the
 * GPU for other CTAs (the CTAs of one Stein update, the grid barrier of the
 * persistent batched kernel) or for the tensor cores (the mbarrier of the
 * tensor-core search), and every such wait is bounded: it gives up after a
 * number of polls, sets an error flag that the host reads, and the call
 * returns SICP_ETIMEOUT with its outputs untouched, the GPU still usable.
 * With on = 1 every such wait of the context's later calls waits for an
 * event that never happens (one arrival more than there are CTAs; an
 * mbarrier nothing arrives on, before any copy or MMA is issued) and gives
 * up after `polls` polls (0: each wait's default limit, up to seconds), so
 * the give-up path can be exercised on purpose.  on = 0 restores normal
 * operation; polls then still caps the waits (0: the defaults).  Errors:
 * SICP_EINVAL (polls outside [0, 2^30]). */
int sicp_set_wait_check(sicp_ctx* ctx, int on, int64_t polls);

/* Index checks of the bounds-checked build (no counterpart in the paper).
 * The library built with SICP_CHECKED checks every index that comes from
 * data (cell coordinates, the seed map, cell bounds, the row table, minibatch
 * entries, search results, fallback lists, batched work items) before its
 * access; an index outside its buffer is recorded and replaced by 0, so the
 * access stays inside the buffer.  *checked (may be NULL) receives 1 for
 * that build and 0 for the normal one; *first (may be NULL) the first failed
 * check since the last call, 0 if none, else bit 63 | site << 40 | the low
 * 40 bits of the index (sites: 1 query cell, 2 seed point, 3 cell bounds,
 * 4 candidate point, 5 row table, 6 source point, 7 reference point or
 * normal, 8 fallback query, 9 batched problem); *count (may be NULL) how many
 * checks failed.  Clears both.  Synchronises the device (all streams) first.
 * Errors: SICP_ECUDA (the synchronisation failed). */
int sicp_check_status(int32_t* checked, uint64_t* first, uint64_t* count);

#ifdef __cplusplus
}
#endif

#endif /* STEINICP_H */
