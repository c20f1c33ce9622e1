/*
 * wke.h -- C ABI of the GB300 (sm_103a) collision-operator library.
 *
 * The library evaluates the collision operator of the 4-wave kinetic equation
 * with omega(k) = |k|^2/2 (or |k|^2, see dispersion) and beta = 0, in the
 * Boltzmann-type spherical form of Qi, Shen and Wang, "A fast Fourier
 * spectral method for wave kinetic equation" (arXiv 2503.12805),
 * Eq. (2.7)-(2.8), discretised as in Sec. 3:
 *
 *   Q(k_i) = 2^{1-d} sum_p W_p [ A B (C + F) - C F (A + B) ](k_i)
 *
 * on the periodic grid k_i = -L + i 2L/N of D_L = [-L, L]^d (Sec. 3.2,
 * Step 1), where for every quadrature node p = (p1, p2, p3) of Eq. (3.8)
 *   F = f(k_i), C = f_N(k_i - q), A = f_N(k_i - a), B = f_N(k_i - b),
 *   q = |q|_{p1} qhat_{p2}, a = (q - |q| sigma_{p3})/2, b = (q + |q| sigma_{p3})/2,
 *   W_p = w_r |q|_{p1}^{2d-3} w_s w_sig,
 * f_N the truncated Fourier series of Eq. (3.1) with modes [-N/2, N/2-1]^d.
 * The four products are the terms K1 = ABC, K2 = FCB, K3 = AFB, K4 = ACF of
 * Eq. (2.7); Algorithm 1 (Sec. 3.4) computes the same sum with its forward
 * and inverse transforms of each product cancelled by linearity.  The
 * Nyquist modes -N/2 are kept by default, so shifted fields are complex:
 * Q is returned as its real part, the imaginary part on request.
 *
 * Conventions for every call below:
 *   - Grids are N^d arrays in row-major order (last axis fastest), in the
 *     plan's precision: double for WKE_FP64, float for WKE_FP32.
 *   - Pointers named *_dev are device pointers (cudaMalloc or torch CUDA
 *     memory) owned by the caller; *_host are host pointers owned by the
 *     caller.  The library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls taking a stream are asynchronous on it and do not
 *     synchronise the host unless stated.
 *   - Every call returns WKE_OK (0) or a negative WKE_ERR_* code; it never
 *     aborts or throws.  wke_last_error_string() describes the last failure
 *     on the calling thread.
 *   - A plan may be used by one host thread at a time.
 */
#ifndef WKE_H
#define WKE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ return codes */
#define WKE_OK                 0
#define WKE_ERR_INVALID       -1   /* bad argument (sizes, rule, pointers)   */
#define WKE_ERR_OOM           -2   /* device or host allocation failed        */
#define WKE_ERR_CUDA          -3   /* a CUDA runtime call or launch failed    */
#define WKE_ERR_UNSUPPORTED   -4   /* valid request the library has no kernel for */
#define WKE_CANCELLED         -5   /* a served request was cancelled before it ran */

/* ------------------------------------------------------------ enumerations */
/* Sphere rules (Sec. 3.3: mid-point in 2D, spherical designs in 3D). */
#define WKE_SPHERE_MIDPOINT_2D  0  /* theta_p = (p + 1/2) 2pi/n, weight 2pi/n  */
#define WKE_SPHERE_PLATONIC_3D  1  /* n = 6, 8, 12, 20 vertex designs, 4pi/n   */
#define WKE_SPHERE_PRODUCT_3D   2  /* Gauss-Legendre in cos(theta) x mid-point
                                      in phi; n_theta = *_param, n_phi = n/n_theta */
#define WKE_SPHERE_USER         3  /* caller's directions and weights          */

#define WKE_FP64  0   /* every step in double                                 */
#define WKE_FP32  1   /* transforms and products in float, tables computed in
                         double and rounded, forward transform in double; the
                         sum over chunks of quadrature groups in a compensated
                         float pair (hi + lo, about twice the float
                         significand) in the fused kernels, in double
                         otherwise                                             */
#define WKE_SPLIT 2   /* WKE_FP32 (float data) whose axis-0 transforms run on
                         the tensor cores: each N-point DFT as a real GEMM in
                         TF32 with both operands split into a TF32 high part
                         and a TF32 low part (three products, FP32
                         accumulation).  Needs the shared-field layout and a
                         3D transform grid of N = 32 or 64.                    */

#define WKE_NYQ_KEEP  0   /* modes [-N/2, N/2-1]^d as in Eq. (3.1) (default)  */
#define WKE_NYQ_ZERO  1   /* zero every mode with a component equal to -N/2   */

/* Index sums of the cubic products (Sec. 3.2).  Circular: the N-point
 * transforms of Algorithm 1, l + m + n = j (mod N).  De-aliased: the linear
 * sums l + m + n = j of Eqs. (3.3)-(3.6), computed on a 2N grid over the same
 * domain (zero padding, the classical de-aliasing of the Sec. 3.2 remark);
 * needs WKE_NYQ_ZERO (the kept -N/2 modes have no partner on the 2N grid, so
 * its fields would not be real), costs 2^d times the transform work, and
 * conserves mass exactly for the same antipodal rule on qhat and sigma. */
#define WKE_ALIAS_CIRCULAR  0
#define WKE_DEALIAS_PAD2    1

/* Evaluation layout (results agree to rounding).  Per group: each
 * quadrature group (radius, direction) transforms its own C and product
 * fields and pass 2 forms the products as it transforms them.  Shared: a
 * chunk of groups transforms each distinct shifted field once (with
 * symmetric rules many coincide: 26 instead of 56 per radius for the cube
 * rule), then a product pass reads them.  Auto picks shared when it saves
 * at least 15% of the transforms. */
#define WKE_LAYOUT_AUTO       0
#define WKE_LAYOUT_PER_GROUP  1
#define WKE_LAYOUT_SHARED     2
/* Shared fields with separable transforms (3D): the phase of a shift x
 * factors per axis, so the inverse transform over axes 2 and 1 depends only
 * on (x1, x2); each distinct x2 is transformed along axis 2 once and each
 * distinct (x1, x2) along axis 1 once per plane, and only the axis-0
 * transform is per field (the cube rule: 3 + 9 plane transforms per radius
 * instead of 26).  Auto picks it in 3D when it saves at least 15% of the
 * trailing-axis transforms; not with WKE_SPLIT. */
#define WKE_LAYOUT_SEPARABLE  3

#define WKE_OMEGA_HALF_K2  0   /* omega = |k|^2/2, the paper's numerics (Sec. 2) */
#define WKE_OMEGA_K2       1   /* omega = |k|^2: the frequency delta halves Q    */

/* Quadrature and numerics of a plan (Eq. (3.8)).  Fill with
 * wke_quadrature_default() and then override fields. */
typedef struct wke_quadrature {
    int n_r;                 /* radial Gauss-Legendre nodes on [0, R]          */
    int n_s;                 /* directions qhat                                */
    int n_sig;               /* collision angles sigma                         */
    int sphere_rule;         /* rule for qhat (WKE_SPHERE_*)                   */
    int sphere_rule_sig;     /* rule for sigma; -1 = same as sphere_rule       */
    int sphere_param;        /* n_theta of WKE_SPHERE_PRODUCT_3D for qhat      */
    int sphere_param_sig;    /* n_theta for sigma                              */
    const double *user_s;    /* WKE_SPHERE_USER: n_s rows of (d coords, weight)
                                for qhat, host memory, read at plan creation   */
    const double *user_sig;  /* same for sigma                                 */
    double R;                /* radial cut-off; 0 => R = 4L/(3 + sqrt 2), i.e.
                                R = 2S with L = (3 + sqrt 2) S / 2 (Step 1)     */
    int precision;           /* WKE_FP64, WKE_FP32 or WKE_SPLIT                */
    int nyquist;             /* WKE_NYQ_KEEP or WKE_NYQ_ZERO                   */
    int dispersion;          /* WKE_OMEGA_HALF_K2 or WKE_OMEGA_K2              */
    int pair_antipodal;      /* 1 (default): when the sigma rule is antipodal
                                with equal weights, evaluate the identical
                                fields f_N(k - b(sigma)) = f_N(k - a(-sigma))
                                and the identical node products once, and
                                skip the nodes with sigma = +-qhat, whose
                                bracket is identically zero when F = f_N on
                                the transform grid (Nyquist kept, or
                                de-aliased); 0: every node separately, as
                                Algorithm 1 loops                              */
    size_t chunk_bytes;      /* budget for the per-chunk intermediate fields;
                                0 => 48 MiB in FP32 (sized to stay resident in
                                L2), 64 MiB in FP64                            */
    int alias;               /* WKE_ALIAS_CIRCULAR (default) or
                                WKE_DEALIAS_PAD2                               */
    int layout;              /* WKE_LAYOUT_AUTO (default), _PER_GROUP, _SHARED or
                                _SEPARABLE                                     */
} wke_quadrature;

typedef struct wke_plan wke_plan;   /* opaque */

/* Counts describing a plan (for tests, benchmarks and admission). */
typedef struct wke_plan_info {
    int d, N, M, precision;
    int n_groups;            /* n_r * n_s: nodes sharing C = f_N(k - q)       */
    int fields_per_group;    /* distinct shifted fields per group             */
    int products_per_group;  /* distinct node products per group              */
    int groups_per_chunk;
    int n_chunks;
    int launches_per_collision;  /* kernels one wke_collision launches        */
    double flops_per_collision;  /* arithmetic of the transforms, phases and
                                    products actually executed (5 n log2 n per
                                    complex transform of n points)            */
    double l2_bytes_per_collision; /* intermediate-field traffic (write + read)*/
    size_t device_bytes;     /* device memory the plan owns                    */
    int N_compute;           /* grid of the transforms: N, or 2N de-aliased    */
    int shared_fields;       /* 1 when the plan uses WKE_LAYOUT_SHARED         */
    int units_per_collision; /* packed transforms (two fields each) per
                                evaluation                                     */
    int separable;           /* 1 when the plan uses WKE_LAYOUT_SEPARABLE      */
    int pair_planes_per_collision; /* separable plans: (x1, x2) pairs transformed
                                along axes 2 and 1 per evaluation              */
    int fused_products;      /* 1 when the axis-0 transform and the products
                                run in one kernel per chunk (3D FP32 shared
                                layouts)                                       */
    int row_values_per_collision; /* separable plans: distinct x2 values
                                transformed along axis 2 per evaluation        */
    int rule_products_available; /* 1 when the plan has the cube rule's own
                                product schedule (wke_tuning.rule_products)    */
} wke_plan_info;

/* ------------------------------------------------------------ calls */

/* Defaults: 2D mid-point / 3D cube rules, R = 0 (automatic), FP64, Nyquist
 * kept, omega = |k|^2/2, antipodal pairing on, automatic chunk budget.  n_r, n_s,
 * n_sig are set to 0 and must be filled in.  Returns WKE_ERR_INVALID if q is
 * NULL. */
int wke_quadrature_default(wke_quadrature *q);

/* Create a plan for d in {2, 3}, N in {16, 32, 48, 64, 96, 128, 256} (2D) or
 * {16, 32, 48, 64} (3D) (lengths 3 * 2^a use radix-12 stages; de-aliased
 * plans need 2N in that set too), half-width L > 0, and M = n_r * n_s * n_sig
 * quadrature nodes
 * (Algorithm 1 inputs: grid size, N_r, N_s, N_sig, nodes and weights).
 * Builds the nodes, weights and shift vectors, the per-axis phase tables
 * exp(-i pi j x / L) and transform twiddles in double precision on the host
 * and uploads them, and allocates all device workspace on the current CUDA
 * device.  *out receives the plan (NULL on failure).
 * Errors: WKE_ERR_INVALID (d, N, L, M or the rule out of range, M !=
 * n_r n_s n_sig, unknown Platonic size, user rule with zero-length
 * direction, WKE_DEALIAS_PAD2 without WKE_NYQ_ZERO), WKE_ERR_UNSUPPORTED
 * (valid N without a compiled kernel),
 * WKE_ERR_OOM, WKE_ERR_CUDA. */
int wke_plan_create(int d, int N, double L, int M, const wke_quadrature *quad,
                    wke_plan **out);

/* Release the plan's device memory and host state.  NULL is accepted.  The
 * caller must ensure no work using the plan is still running. */
int wke_plan_destroy(wke_plan *plan);

/* Device bytes a plan with these parameters would own, without creating it
 * (admission control).  Errors as wke_plan_create, minus OOM/CUDA. */
int wke_plan_footprint_bytes(int d, int N, double L, int M,
                             const wke_quadrature *quad, size_t *bytes);

/* Fill *info for an existing plan. */
int wke_plan_get_info(const wke_plan *plan, wke_plan_info *info);

/* Fill *info for the plan wke_plan_create would build from these arguments,
 * without creating it: host work only, no device memory or CUDA call
 * (device_bytes is the footprint of wke_plan_footprint_bytes).  For
 * planning and admission; errors as wke_plan_create's argument checks. */
int wke_plan_describe(int d, int N, double L, int M, const wke_quadrature *quad,
                      wke_plan_info *info);

/* Copy the node table to host memory: M rows, in (p1, p2, p3) lexicographic
 * order, of 1 + 3d doubles: W_p, q (d), a (d), b (d).  `out_host` must hold
 * M * (1 + 3d) doubles. */
int wke_plan_node_table(const wke_plan *plan, double *out_host);

/* Q = Re K(f) on the grid (Eq. (2.7) discretised as above; Algorithm 1's
 * output).  f_dev: N^d values, read only.  Q_dev: N^d values, written.  They
 * must not overlap.  Asynchronous on `stream`; the plan's workspace is in use
 * until the stream reaches the end of the call, so calls with one plan on
 * different streams must be ordered by the caller. */
int wke_collision(wke_plan *plan, const void *f_dev, void *Q_dev, void *stream);

/* As wke_collision and, if Qim_dev is not NULL, also Im K(f) into Qim_dev
 * (N^d values, plan precision): nonzero only through the kept Nyquist modes. */
int wke_collision_ex(wke_plan *plan, const void *f_dev, void *Q_dev, void *Qim_dev,
                     void *stream);

/* As wke_collision, then the Fourier coefficients of Q (Algorithm 1's Q-hat
 * before its final inverse transform; Eq. (3.1) applied to Q):
 *   Qhat_j = N^{-d} sum_i Q_i exp(-i pi j.k_i / L),  j in [-N/2, N/2-1]^d,
 * one forward transform of the grid values (computed in double), stored in
 * DFT order (mode j at position j mod N per axis) as N^d interleaved
 * (re, im) pairs of the plan's precision.  Q_dev (N^d values) and Qhat_dev
 * (2 N^d values) are device buffers owned by the caller and must not
 * overlap f_dev or each other.  Stream-ordered like wke_collision.
 * Errors: WKE_ERR_INVALID for NULL or overlapping buffers, WKE_ERR_CUDA. */
int wke_collision_spectrum(wke_plan *plan, const void *f_dev, void *Q_dev, void *Qhat_dev, void *stream);

/* End-to-end variant with host buffers: copies f_host to plan-owned device
 * memory, evaluates, copies Q back to Q_host and synchronises the plan's
 * stream before returning.  Pinned host memory gives full copy bandwidth. */
int wke_collision_host(wke_plan *plan, const void *f_host, void *Q_host);

/* Stream used by wke_step and wke_collision_host (default: NULL). */
int wke_plan_set_stream(wke_plan *plan, void *stream);

/* One explicit Runge-Kutta step of df/dt = Q(f) on the grid values (the
 * paper integrates with RK4, Sec. 4): rk_stages 1 = forward Euler, 2 = Heun,
 * 4 = classical RK4.  f_dev is updated in place on the plan's stream;
 * asynchronous.  With graphs on (the default) the whole step - every
 * stage's evaluation and stage update - is captured once per (f_dev, dt,
 * rk_stages) and replayed as one graph launch.  Errors: WKE_ERR_INVALID for
 * other rk_stages or dt not finite. */
int wke_step(wke_plan *plan, void *f_dev, double dt, int rk_stages);

/* Macroscopic moments of a grid function g (Sec. 2): out_dev[0] = h^d sum g
 * (mass), out_dev[1..d] = h^d sum k g (momentum), out_dev[d+1] = h^d sum
 * |k|^2 g (energy), h = 2L/N, summed in double in a fixed order.  out_dev is
 * a device pointer to d + 2 doubles.  Asynchronous on `stream`. */
int wke_moments(wke_plan *plan, const void *g_dev, double *out_dev, void *stream);

/* Launch layout of a plan's kernels.  Layouts change speed, not results
 * beyond rounding. */
typedef struct wke_tuning {
    int pass2_points_per_thread;   /* axis-0 transform in pass 2: 4 (radices
                                      4,4,4 at N = 64: fewer registers, more
                                      blocks per SM) or 8 (radices 8,8: fewer
                                      instructions); N >= 128 always uses 8,
                                      N = 48, 96 always 12 (get reports the
                                      value in use; set accepts 12 there) */
    int pass1_units_per_block;     /* units each pass-1 block transforms for its
                                      plane (reuses the plane's coefficients);
                                      0 = automatic */
    int fuse_products;             /* 3D FP32 shared layouts: 1 = the axis-0
                                      transform runs inside the product kernel
                                      (the default where the plan supports
                                      it), 0 = separate axis-0 and product
                                      kernels with a unit buffer between them
                                      (allocated on first use: the call may
                                      return WKE_ERR_OOM); other plans: 0 */
    int forward_fp32;              /* WKE_FP32 plans that are not de-aliased:
                                      1 = the forward transform of f computes in
                                      float, 0 = in double (default); other
                                      plans: 0 */
    int rule_products;             /* fused plans of the cube rule (cube q-hat
                                      and sigma rules, antipodal pairing): 1 =
                                      the products follow the rule's own
                                      schedule, which reads every field once
                                      per point (the default), 0 = the generic
                                      product table; other plans: 0 */
} wke_tuning;

int wke_plan_get_tuning(const wke_plan *plan, wke_tuning *out);

/* Set the layout; WKE_ERR_INVALID for values out of range.  Drops the plan's
 * cached graphs (the next call re-captures). */
int wke_plan_set_tuning(wke_plan *plan, const wke_tuning *tuning);

/* Autotuner: times every candidate layout on this plan's own workload
 * (f_dev in, Q_dev out, both device buffers of the plan's grid), `reps`
 * evaluations each after one warm-up, with CUDA events on the plan's stream,
 * and keeps the fastest.  chosen (may be NULL) receives it and best_ms (may
 * be NULL) its milliseconds per evaluation.  Synchronises the plan's stream. */
int wke_plan_autotune(wke_plan *plan, const void *f_dev, void *Q_dev, int reps, wke_tuning *chosen,
                      double *best_ms);

/* Plan creation with the autotuner over pencil layouts as well: the same
 * evaluation as wke_plan_create (Algorithm 1, Sec. 3.4) for the same
 * arguments, with the layout chosen by timing.  With quad->layout =
 * WKE_LAYOUT_AUTO the candidates are WKE_LAYOUT_SEPARABLE (3D, not
 * WKE_SPLIT), _SHARED and _PER_GROUP (not WKE_SPLIT): which axes every
 * distinct shifted field is transformed along on its own, and so the
 * shape of the line batches each transform kernel works on.  A candidate
 * whose plan cannot be built for this rule (or does not fit in memory) is
 * skipped; each other one is created, tuned by wke_plan_autotune on f_dev
 * (device buffer of the plan's grid and precision; Q_dev receives its
 * results) with `reps` timed evaluations per launch layout on `stream` (NULL:
 * the plan's own stream), and all but the fastest are destroyed again.  Any
 * other layout value tunes that layout alone.  *out receives the plan (owned
 * by the caller, freed with wke_plan_destroy; a non-NULL `stream` stays its
 * stream, as after wke_plan_set_stream), layout_out (may be NULL) the layout
 * it uses and best_ms (may be NULL) its milliseconds per evaluation.
 * Holds at most two plans at a time; synchronises `stream`.  Errors: those of
 * wke_plan_create when no candidate can be built, else those of
 * wke_plan_autotune; *out is NULL after an error. */
int wke_plan_create_autotuned(int d, int N, double L, int M, const wke_quadrature *quad, const void *f_dev,
                              void *Q_dev, void *stream, int reps, wke_plan **out, int *layout_out,
                              double *best_ms);

/* Evaluations are captured into a CUDA graph per distinct (f, Q, Qim)
 * pointer set on first use and replayed afterwards (default on; at most 8
 * graphs per plan).  enable = 0 launches every kernel directly instead.  A
 * capture runs on the plan's own streams, so the first call with a new
 * pointer set must not itself be inside a caller's stream capture. */
int wke_plan_use_graphs(wke_plan *plan, int enable);

/* Kernel timing.  While enabled, every wke_collision records CUDA events
 * around its launches on the call's stream (no host synchronisation).
 * wke_plan_profile_read() must be called after that stream is idle: it adds
 * up the recorded intervals per kernel class into out_host[2 * WKE_PROF_CLASSES]
 * as (total milliseconds, number of launches) pairs, in the order forward,
 * pass 1, pass 2 (the product pass in the shared-field layout), finalize,
 * Nyquist tables, axis-0 transform (shared-field layout), and forgets them.
 * Enabling resets the record.
 * While enabled, evaluations launch directly (no graph replay) and the two
 * passes of consecutive chunks do not overlap, so each interval is one
 * kernel's own duration. */
#define WKE_PROF_CLASSES 6
int wke_plan_profile(wke_plan *plan, int enable);
int wke_plan_profile_read(wke_plan *plan, double *out_host);

/* The same sums as wke_moments for callers that cannot allocate device
 * memory where they need them (a caller living inside another allocator's
 * fixed budget, or one that must not allocate while a stream capture is
 * open): no plan, no cudaMalloc, no cudaFree.  The paper has no counterpart;
 * this is a service of the library.  d in {2, 3}, grid N^d on [-L, L]^d as
 * above, precision WKE_FP64 (g is double) or WKE_FP32 (g is float);
 * out_dev receives d + 2 doubles; asynchronous on `stream`.
 * The per-block partial sums live in a fixed 40 KiB array in the library's
 * device image, so grids above 4,194,304 points (1024 blocks of 4096) are
 * rejected with WKE_ERR_INVALID.  A call outside a stream capture resolves
 * the array's address on the current device with cudaGetSymbolAddress (so
 * it follows the device image across a cudaDeviceReset); a call inside a
 * capture uses the address of the last call outside one, so make the first
 * call on each device before any stream capture.  All calls share the
 * array: calls whose kernels overlap on the GPU race, so order them (one
 * stream, or events). */
int wke_moments_noalloc(int d, int N, double L, int precision, const void *g_dev, double *out_dev,
                        void *stream);

/* Arithmetic roofs of the current device (a measurement service of the
 * library; the paper has no counterpart).  Launches register-resident chains
 * of fused multiply-adds on every SM (4 blocks of 256 threads per SM, 8
 * independent chains per thread), times `reps` launches after one warm-up
 * with CUDA events on a private stream, and returns the best rate in
 * *tflops (2 flops per multiply-add).  precision WKE_FP32 times both the
 * scalar FMA and the packed two-lane f32x2 FMA and keeps the faster;
 * WKE_FP64 times the double FMA.  *best_ms (may be NULL) receives the
 * duration of the best launch.  Allocates and frees a small scratch buffer;
 * synchronises.  Errors: WKE_ERR_INVALID (precision, reps outside
 * [1, 1000], tflops NULL), WKE_ERR_OOM, WKE_ERR_CUDA. */
int wke_alu_peak(int precision, int reps, double *tflops, double *best_ms);

/* ------------------------------------------------------------ serving */
/* A serving loop runs time-stepping requests of mixed sizes from concurrent
 * simulations with continuous batching: a worker thread admits the oldest
 * pending request as soon as fewer than `max_active` requests run and its
 * device footprint (wke_plan_footprint_bytes plus its grid) fits within
 * `device_budget_bytes`, then enqueues all of its steps on its own stream,
 * so requests overlap on the GPU.  Plans of finished requests stay resident
 * and are reused by later requests of the same shape; idle plans are evicted
 * least recently used first when memory is needed.  Results are identical to
 * running the same steps alone (the kernels sum in a fixed order). */
typedef struct wke_server wke_server;

typedef struct wke_request {
    int d, N;              /* grid (see wke_plan_create)                      */
    double L;
    int n_r, n_s, n_sig;   /* quadrature counts, default rules                */
    int precision;         /* WKE_FP32 or WKE_FP64                            */
    int rk_stages;         /* 1, 2 or 4 (see wke_step)                        */
    int steps;             /* number of time steps                            */
    double dt;             /* step size                                       */
    const void *f_host;    /* initial grid, read when the request is admitted  */
    void *out_host;        /* final grid, written when the request completes   */
} wke_request;

typedef struct wke_request_stats {
    long long id;
    int status;            /* WKE_OK, WKE_CANCELLED or a WKE_ERR_* code       */
    double t_submit, t_admit, t_done;   /* seconds on the server's clock      */
} wke_request_stats;

/* Start a server on the current device.  The worker thread makes every CUDA
 * call of the server. */
int wke_server_create(size_t device_budget_bytes, int max_active, wke_server **out);

/* Queue a request (any thread); the descriptor is copied, the host buffers
 * must stay valid until the request completes.  *id receives its id.  A
 * request whose footprint exceeds the whole budget completes with
 * WKE_ERR_OOM. */
int wke_server_submit(wke_server *server, const wke_request *request, long long *id);

/* Cancel a request that has not been admitted yet (WKE_ERR_INVALID otherwise). */
int wke_server_cancel(wke_server *server, long long id);

/* Block until request `id` completes (timeout_s < 0: no limit) and fill
 * *stats.  WKE_ERR_INVALID on an unknown id or a timeout. */
int wke_server_wait(wke_server *server, long long id, double timeout_s, wke_request_stats *stats);

/* Finish every queued request, stop the worker and release all memory. */
int wke_server_destroy(wke_server *server);

/* Bounds-checked debug build (the library compiled with -DWKE_CHECK,
 * libwke_check.so): the hot kernels test the indices they take from the
 * plan's tables against the extents of the buffers they address, record a
 * bit per failing check site in a device word and skip the access (nothing
 * traps).  wke_check_status synchronises the device, returns the bits in
 * *flags, clears them, and returns WKE_ERR_CUDA when any is set (the message
 * names the sites), WKE_OK otherwise.  In the default build it sets *flags to
 * 0 and returns WKE_OK.  A debugging aid of the library; the paper has no
 * counterpart. */
int wke_check_status(unsigned *flags);

/* Message for the last failed call on this thread ("" if none). */
const char *wke_last_error_string(void);

/* Library version string. */
const char *wke_version(void);

#ifdef __cplusplus
}
#endif
#endif /* WKE_H */
