/*
 * l1alm.h -- C ABI of the GB300 (sm_103a) augmented Lagrangian l1 solvers.
 *
 * Method: A. Y. Yang, Z. Zhou, A. Ganesh, S. S. Sastry, Y. Ma, "Fast
 * l1-Minimization Algorithms for Robust Face Recognition":
 *   - primal ALM (PALM): Algorithm 1 (§V-A) for the cross-and-bouquet
 *     problem of Eq. 5, and the method of multipliers of Eq. 33 with FISTA
 *     inner solves (§V-A) for basis pursuit (P1, Eq. 1);
 *   - dual ALM (DALM): Algorithm 2 (§V-B, Eqs. 36-39);
 *   - FISTA (Eq. 18, §IV-A) for unconstrained BPDN (QP_lambda, Eq. 3);
 *   - the per-class residual and SCI classifiers (§II-A, Eq. 40).
 * Equation numbers are the paper's in source order.
 *
 * Conventions for every entry point
 *   - Matrices are column-major FP32: element (i, j) of an m x n matrix with
 *     leading dimension ld sits at p[i + j*ld], ld >= m.
 *   - Pointers may be host or device memory; the library detects which with
 *     cudaPointerGetAttributes and copies host data in and out itself (these
 *     copies are enqueued on the handle's stream).  Caller-owned buffers stay
 *     caller-owned; the handle owns everything it derives from A.
 *   - A negative return value means the call failed and wrote no output;
 *     l1_status_string() names it.  Calls never abort the process.
 *   - All device work is enqueued on the handle's stream (l1_options.stream
 *     at setup, or l1_set_stream).  l1_solve_batch returns after the results
 *     are on the host (it synchronises that stream).
 *   - Handles are not thread-safe: one host thread at a time per handle.
 */
#ifndef L1ALM_H
#define L1ALM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define L1_API __attribute__((visibility("default")))
#else
#define L1_API
#endif

/* ------------------------------------------------------------ return codes */
#define L1_OK 0
#define L1_ERR_INVALID_ARG (-1) /* bad pointer, size, mode or option */
#define L1_ERR_NOT_SPD (-2)     /* DALM needs A A^T invertible (§V-B); P1 with rank-deficient A */
#define L1_ERR_OOM (-3)         /* device allocation failed */
#define L1_ERR_CUDA (-4)        /* a CUDA runtime call failed (message: l1_last_error) */
#define L1_ERR_TIMEOUT (-5)     /* a bounded device wait expired; the context stays usable */
#define L1_ERR_NO_TAPE (-6)     /* l1_backward without an unrolled forward */
#define L1_ERR_UNSUPPORTED (-7) /* valid request the library does not implement */

/* --------------------------------------------------- per-instance status */
#define L1_CONVERGED 0 /* stopping rule met: ||w_{k+1}-w_k|| / ||w_k|| < tol (§VI-C) */
#define L1_MAX_ITER 1  /* max_iter reached first */
#define L1_NONFINITE 2 /* an iterate became NaN/Inf; the instance was frozen */

/* ------------------------------------------------------------------ enums */
typedef enum {
    L1_P1 = 0,        /* min ||x||_1  s.t. b = A x                      (Eq. 1) */
    L1_P1_2 = 1,      /* min ||x||_1  s.t. ||b - A x||_2 <= epsilon     (Eq. 2) */
    L1_QP_LAMBDA = 2, /* min 1/2||b - A x||^2 + lambda ||x||_1          (Eq. 3) */
    L1_CAB = 3        /* min ||x||_1 + ||e||_1 s.t. b = A x + e, B=[A I] (Eq. 5) */
} l1_mode;

typedef enum {
    L1_PALM = 0, /* primal ALM, Algorithm 1 (§V-A) */
    L1_DALM = 1, /* dual ALM, Algorithm 2 (§V-B) */
    L1_AMP = 2   /* approximate message passing (§IV, reading R18), mode L1_P1 only, FP32
                  * dictionary, either engine: x_{k+1} = soft(A^T z_k + x_k, tau_k),
                  * z_{k+1} = b - A x_{k+1} + (n/m) <eta'> z_k, tau_{k+1} = (n/m) <eta'> tau_k
                  * with <eta'> the fraction of entries above the threshold; x_0 = 0,
                  * z_0 = b.  A comparison solver: §VI-B reports that it diverges on face
                  * dictionaries (status L1_NONFINITE) */
} l1_solver;

typedef enum {
    L1_A_FP32 = 0, /* A held in FP32 */
    L1_A_BF16 = 1, /* A held in BF16 (round to nearest even), FP32 accumulate */
    L1_A_FP8E4M3 = 2 /* A held in FP8 e4m3 (nearest, saturating) with one FP32 scale
                      * per row of each stored layout (per row of A for A u, per
                      * column of A for A^T y), FP32 accumulate */
} l1_precision;

typedef enum {
    L1_ENGINE_AUTO = 0,  /* DALM (P1, CAB) with an FP32 or BF16 dictionary, and AMP:
                          * L1_ENGINE_TC; everything else: L1_ENGINE_SIMT */
    L1_ENGINE_SIMT = 1,  /* CUDA-core FP32 kernels (GEMV for N <= 8, tiled GEMM above) */
    L1_ENGINE_TC = 2     /* tcgen05 BF16 tensor-core sweeps for batched DALM and AMP: A and the
                          * panels as aligned BF16 pieces, the leading product summed
                          * exactly, FP32 accumulation; narrow batches (tc_min_cols)
                          * fall back to the CUDA-core sweeps */
} l1_engine;

/* ---------------------------------------------------------------- options
 * Zero in a field means "default"; l1_options_init fills the defaults. */
typedef struct {
    int32_t solver;     /* l1_solver; QP_LAMBDA always runs FISTA */
    int32_t precision;  /* l1_precision */
    int32_t engine;     /* l1_engine */
    int32_t inner_max;  /* PALM inner FISTA cap per outer step; default 50 */
    double lambda;      /* QP_LAMBDA weight (> 0) */
    double epsilon;     /* P1_2 radius (> 0) */
    double xi0;         /* PALM penalty; 0 -> 2m/||b||_1 per instance (§V-A) */
    double xi_growth;   /* P1/P1_2 PALM: xi_{k+1} = min(growth xi_k, xi_max xi_0); 0 -> 1.2 */
    double xi_max;      /* cap factor; 0 -> 1e4.  CAB keeps xi fixed (§V-A). */
    double beta;        /* DALM penalty; 0 -> ||b||_1 / m per instance */
    double lipschitz;   /* L of Algorithm 1 step 6; 0 -> power iteration x 1.01 */
    double inner_tol;   /* PALM inner tolerance; 0 -> 0.1 * tol */
    int32_t check_every; /* host polls the active count every this many iterations; 0 -> 16 */
    int32_t class_count; /* CAB classification: number of classes C (0: off) */
    const int32_t* class_offsets; /* host, C+1 entries; class c owns columns [off[c], off[c+1]) */
    void* stream;        /* cudaStream_t for all work; NULL = legacy default stream */
    int32_t unroll_K;    /* > 0: l1_solve_batch runs K unrolled PALM steps (P1) and keeps a tape */
    int32_t unroll_J;    /* multiplier update every J inner steps; 0 -> 10 */
    int32_t ckpt_every;  /* checkpoint interval of the tape; 0 -> 20 */
    int32_t profile;     /* 1: time every sweep with CUDA events (l1_info.sweep_*) */
    int32_t tc_pieces;   /* L1_ENGINE_TC: BF16 pieces of A and of the panels in the A u and
                          * A^T y sweeps, 2 (three terms, about 16 bits) or 3 (six terms,
                          * FP32-level products); 0 -> 3.
                          * Precision BF16 runs its first phase with one piece of A
                          * whatever this says. */
    int32_t refine;      /* precision BF16 / FP8: 0 -> after every column has met the
                          * stopping rule on the low-precision A, resume each one from
                          * its iterate on the FP32 A until the rule is met again
                          * (results and iters cover both phases); -1 -> return the
                          * low-precision answer */
    int32_t tc_pieces_y; /* L1_ENGINE_TC: BF16 pieces of (B B^T)^{-1} and of the y-step's
                          * right-hand side, 2 or 3; 0 -> 3 */
    int32_t tc_min_cols; /* L1_ENGINE_TC: the tensor-core sweeps run while at least this
                          * many columns are active, the CUDA-core sweeps below; 0 -> 1
                          * (the tensor-core products track the FP64 iteration more
                          * closely than the CUDA-core FP32 ones, so by default they
                          * run to the last column) */
    int32_t tune;        /* L1_ENGINE_TC: 0 -> l1_setup times the tile strategies of
                          * the tensor-core sweeps (fused or deferred epilogue,
                          * split-K slices) at batch widths up to 4096 for each sweep
                          * shape and keeps the fastest (l1_tuning); -1 -> a fixed
                          * rule from the tile and multiprocessor counts (deferred
                          * epilogue; split-K when a quarter of the SMs would hold
                          * every tile), e.g. under a profiler, whose per-launch
                          * overhead distorts the tuner's timings.  The slice
                          * count sets the order in which K slices are added, so two
                          * handles whose timings chose differently can differ in the
                          * last bits. */
    int32_t cg_steps;    /* DALM: 0 -> the exact y-step of Eq. 39 through the FP64 factor
                          * of B B^T; 1 -> one conjugate-gradient step on that system
                          * from the previous y per iteration instead (§V-B, reading
                          * R15): no m x m factor is formed, so setup needs no O(m^2)
                          * memory or Cholesky.  §V-B reports that this variant fails
                          * on face images; on the cross-and-bouquet model it stalls
                          * far from the constraint.  FP32 dictionary and the
                          * tensor-core engine only (L1_ERR_UNSUPPORTED otherwise). */
    double lambda0;      /* QP_LAMBDA: > lambda -> FISTA with fixed-point continuation
                          * (the FISTA setup of the §VI-A comparison, reading R17):
                          * step k of Eq. 18 thresholds at lambda_k / L with
                          * lambda_1 = lambda0, lambda_{k+1} = max(rho lambda_k,
                          * lambda), and the stopping rule applies once lambda_k has
                          * reached lambda; 0 -> plain FISTA at lambda */
    double cont_rho;     /* continuation factor rho in (0, 1]; 0 -> 0.95 */
    double tau0;         /* L1_AMP: initial threshold tau_0 for every column; 0 ->
                          * 1.5 ||b||_2 / sqrt(m) per column (reading R18) */
} l1_options;

/* Per-instance results (host memory). */
typedef struct {
    int32_t status;      /* L1_CONVERGED / L1_MAX_ITER / L1_NONFINITE */
    int32_t iters;       /* outer iterations (PALM), iterations (DALM, FISTA) */
    int32_t inner_iters; /* total inner FISTA steps (PALM); = iters otherwise */
    int32_t label;       /* CAB: argmin_c ||b - e - A delta_c(x)||_2 (lowest index on ties), else -1 */
    int32_t sci_label;   /* CAB: SCI argmax of Eq. 40, else -1 */
    int32_t reserved;
    double rel_change;   /* last ||w_{k+1}-w_k|| / ||w_k|| */
    double primal_obj;   /* ||x||_1 (+||e||_1); QP: 1/2||b-Ax||^2 + lambda ||x||_1 */
    double dual_obj;     /* b^T y / max(1, ||B^T y||_inf); QP: b^T u - 1/2||u||^2 */
    double gap;          /* primal_obj - dual_obj (>= 0 up to rounding) */
    double resid;        /* ||b - B w||_2 */
    double param;        /* xi_0 (PALM), beta (DALM), lambda / L (FISTA) used, or the
                          * last threshold tau_k (AMP) */
} l1_result;

typedef struct l1_handle_s* l1_handle;

/* Handle information. */
typedef struct {
    int64_t m, n;
    int32_t mode, solver, precision, engine;
    double lipschitz;        /* L used by PALM / FISTA (0 if not computed) */
    double setup_ms;         /* device time of l1_setup */
    int64_t device_bytes;    /* bytes the handle holds on the device */
    int64_t gpu_launches;    /* kernels launched by this handle so far */
    /* with l1_options.profile = 1, per sweep kind (0: A u, 1: (B B^T)^{-1} r,
     * 2: A^T y, 3: other): launches, summed CUDA-event time, and algorithmic
     * FLOPs 2*M*K*(columns active at the last host poll), since setup */
    int64_t sweep_launches[4];
    double sweep_ms[4];
    double sweep_flop[4];
} l1_info;

/* Fill *opt with the defaults. */
L1_API void l1_options_init(l1_options* opt);

/*
 * l1_setup -- build a solver handle for the dictionary A (m x n, column-major,
 * leading dimension lda >= m; host or device FP32).  A is copied; the caller
 * keeps ownership.  One-time work (§V): the Lipschitz constant L = ||A||_2^2
 * by power iteration (PALM, FISTA), and for DALM the FP64 Cholesky factor of
 * B B^T = A A^T (+ I for CAB) and its explicit inverse (Eq. 39), stored FP32.
 * Errors: L1_ERR_INVALID_ARG (null pointer, m or n <= 0, lda < m, P1 with
 * m > n, unknown mode/solver/precision), L1_ERR_NOT_SPD (DALM on P1 with
 * singular A A^T), L1_ERR_OOM, L1_ERR_CUDA, L1_ERR_UNSUPPORTED.
 */
L1_API int l1_setup(const float* A, int64_t m, int64_t n, int64_t lda, int32_t mode,
                    const l1_options* opt, l1_handle* out);

/*
 * l1_setup_group -- a batch of `count` independent (QP_lambda) problems
 * (Eq. 3) whose dictionaries differ in size: instance i has A[i], m[i] x n[i],
 * column-major FP32 with leading dimension m[i] (host or device).  The group
 * is solved by FISTA (Eq. 18, §IV-A) in one persistent launch per solve with
 * per-instance stopping (§VI-C rule) and an active-instance work list.
 * opt->precision selects the storage of the dictionaries: L1_A_FP32 or
 * L1_A_BF16 (round to nearest even; FP32 arithmetic).  L = ||A_i||_2^2 of
 * each instance comes from a batched power iteration (x 1.01).  A == NULL
 * allocates the group and leaves the dictionaries to l1_group_load.
 * Sizes: 1 <= m[i] <= 4096 (an instance's rows stay in the registers of one
 * CTA), 1 <= n[i] <= 2^24.
 * Errors: L1_ERR_INVALID_ARG (mode other than QP_LAMBDA, lambda <= 0, count
 * or a size out of range), L1_ERR_OOM, L1_ERR_CUDA, L1_ERR_UNSUPPORTED.
 */
L1_API int l1_setup_group(const float* const* A, const int64_t* m, const int64_t* n, int64_t count,
                          int32_t mode, const l1_options* opt, l1_handle* out);

/*
 * l1_group_load -- copy (and quantise) the dictionaries of instances
 * first .. first+k-1 of a group handle from A[0..k-1] (layout as in
 * l1_setup_group), then (re)compute their Lipschitz constants.  Lets a
 * caller stream a group that does not fit in host or device memory in FP32.
 */
L1_API int l1_group_load(l1_handle h, int64_t first, int64_t k, const float* const* A);

/*
 * l1_solve_batch on a group handle: b packs the right-hand sides (instance i
 * at offset sum_{k<i} m[k]), x packs the solutions (offset sum_{k<i} n[k]);
 * N must equal count, ldb and ldx are ignored, y must be NULL.  res[i].resid
 * is ||b - A x||_2 and primal_obj 1/2||b - A x||^2 + lambda ||x||_1;
 * dual_obj and gap are NaN (not computed for groups).  x_init and y_init must
 * be NULL.
 */

/*
 * l1_solve_batch -- solve N independent problems that share A, one per
 * column of b (m x N, leading dimension ldb >= m), 1 <= N <= 65535.
 *   tol       stopping tolerance of the relative-change rule (§VI-C); 0 runs
 *             exactly max_iter iterations.
 *   max_iter  cap on outer iterations (PALM) or iterations (DALM, FISTA, AMP).
 *   x         output, (n + m) x N for CAB ([x; e] per column), n x N otherwise,
 *             leading dimension ldx.
 *   y         optional (NULL) output of the dual iterate, m x N, leading
 *             dimension ldy: DALM's y, PALM's multiplier theta, AMP's z_k
 *             (of the last x-step; the dual_obj and gap results computed
 *             from it do not certify AMP's answer).
 *   res       host array of N results.
 *   x_init    optional (NULL) warm start, laid out like x (leading dimension
 *             ldxi): DALM's w_1 = [x; e] (Algorithm 2 starts from w_1 = 0
 *             otherwise), PALM's x_1 and, for CAB, e_1 (Algorithm 1 takes
 *             e_1 = b otherwise; the first e-step recomputes e from x_1),
 *             FISTA's x_0 (Eq. 18), AMP's x_0 (0 otherwise).
 *   y_init    optional (NULL) warm start of the dual iterate, laid out like y
 *             (leading dimension ldyi): DALM's y_1, PALM's theta_1, AMP's z_0
 *             (b otherwise); zero otherwise.  A DALM solve resumed from the x and y another solve
 *             returned continues that solve's iteration: its first z-step
 *             (Eq. 38) is recomputed from (w, y).
 * Each column stops on its own rule and is frozen from then on (per-instance
 * convergence masking).  Host pointers are copied in and out on the handle's
 * stream.  Errors: L1_ERR_INVALID_ARG, L1_ERR_OOM, L1_ERR_CUDA,
 * L1_ERR_TIMEOUT.
 */
L1_API int l1_solve_batch(l1_handle h, const float* b, int64_t ldb, int64_t N, double tol,
                          int32_t max_iter, float* x, int64_t ldx, float* y, int64_t ldy,
                          l1_result* res, const float* x_init, int64_t ldxi, const float* y_init,
                          int64_t ldyi);

/*
 * l1_solve_batch on a handle set up with unroll_K > 0 (mode L1_P1, solver
 * L1_PALM): runs exactly K inner FISTA steps of Algorithm 1 in total, with the
 * multiplier step theta += xi (b - A x) after every unroll_J inner steps and
 * FISTA restarted (t = 1, z = w = x) at each block start (reading R11).  xi is
 * xi0, or 2m/||b||_1 per column when xi0 = 0, and stays constant; L is the
 * handle's.  tol and max_iter are ignored; y must be NULL.  Every column
 * reports L1_MAX_ITER with iters = ceil(K / J) and inner_iters = K,
 * primal_obj = ||x||_1, resid = ||b - A x||, param = xi; rel_change, dual_obj
 * and gap are NaN.  The call keeps a tape for l1_backward: (z, w, theta) every
 * ckpt_every steps and x at the end of every block.
 */

/*
 * l1_backward -- reverse-mode derivative of that unrolled forward (R11: xi and
 * L held constant; the soft-threshold derivative is 1 where |v| > 1/(xi L),
 * else 0).  grad_x (n x N, leading dimension n, host or device) is the
 * adjoint of the x the forward returned; N must equal the forward's N.  Each
 * checkpointed segment is recomputed once and then reversed.  Outputs (host
 * or device, nullable): grad_b (m x N, leading dimension m) and grad_A
 * (m x n, leading dimension m, the sum over the N columns); both are
 * overwritten.  Returns after the outputs are written.  Errors:
 * L1_ERR_NO_TAPE (no unrolled forward yet), L1_ERR_INVALID_ARG (N differs,
 * null grad_x), L1_ERR_OOM, L1_ERR_CUDA.
 */
L1_API int l1_backward(l1_handle h, const float* grad_x, int64_t N, float* grad_b,
                       float* grad_A);

/*
 * l1_lipschitz_static -- the power-iteration estimate of ||A||_2^2 that
 * l1_setup makes (start vector 1/sqrt(n), Rayleigh quotient ||A v||^2, stop
 * when it changes by at most rtol relative or after max_iter iterations;
 * l1_setup takes L = 1.01 x this), computed without allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that may
 * not call cudaMalloc or cudaFree -- a process whose device memory is owned by
 * its own pool allocator, or a loop that must not stall the device while
 * memory is allocated or freed.
 *   A          device (or managed) memory, m x n, column-major, leading
 *              dimension lda >= m; on the current device; read only.
 *   stream     the work is enqueued there (NULL: the legacy default stream).
 *              The call copies its state to the host and synchronises this
 *              stream before it returns, so it must not be called while the
 *              stream is being captured into a CUDA graph (it returns
 *              L1_ERR_INVALID_ARG then, before enqueuing anything).
 *   rho_out    host pointer; receives the estimate.
 *   status_out nullable host pointer; receives L1_CONVERGED when the stopping
 *              rule fired, L1_MAX_ITER when max_iter ran out first (rho_out
 *              then holds the last, unconverged estimate, which is below
 *              ||A||_2^2; close top singular values make this likely).
 *   iters_out  nullable host pointer; receives the iterations run.
 * Scratch: one static device array of 1.34 MiB per GPU that loads this
 * library, held until the process exits; hence m <= 8192 and n <= 65536.
 * Larger sizes return L1_ERR_INVALID_ARG with a message in l1_last_error.
 * The first call on a device looks up that array's device address (once,
 * with that device current).  Each call initialises the scratch it reads,
 * but every call on a device shares the one array: calls that can overlap on
 * the GPU (other streams, other host threads) race and must be serialised by
 * the caller.
 * Errors: L1_ERR_INVALID_ARG (null pointer, a size <= 0 or above the limits,
 * lda < m, max_iter <= 0, rtol < 0, A not device memory or on a device other
 * than the current one, the stream being captured), L1_ERR_CUDA.
 */
L1_API int l1_lipschitz_static(const float* A, int64_t m, int64_t n, int64_t lda, int32_t max_iter,
                               double rtol, void* stream, double* rho_out, int32_t* status_out,
                               int32_t* iters_out);

/*
 * l1_solve_plain -- DALM (Algorithm 2, reading R1) for ONE right-hand side b
 * (m floats, host or device) on a DALM handle (modes P1 and CAB), in plain
 * FP32: one simple kernel per step of the iteration (z-step of Eq. 38, the
 * products A u, (B B^T)^{-1} r with the FP32 inverse, A^T y, the w-step), and
 * the relative-change rule of §VI-C read on the host after every iteration.
 * It is the unbatched, unfused baseline the batched solver is measured
 * against.  x (n + m floats for CAB, n for P1, host or device) receives w;
 * res gets status, iters, rel_change, primal_obj = ||w||_1 and param = beta
 * (dual_obj, gap and resid are NaN, labels -1).  The call allocates its
 * work buffers and synchronises the handle's stream.
 * Errors: L1_ERR_INVALID_ARG, L1_ERR_UNSUPPORTED (not a DALM handle in P1 or
 * CAB mode, a group or an unrolled handle), L1_ERR_OOM, L1_ERR_CUDA.
 */
L1_API int l1_solve_plain(l1_handle h, const float* b, double tol, int32_t max_iter, float* x,
                          l1_result* res);

/*
 * l1_tuning -- the tile shapes and strategies l1_setup's autotuner chose for
 * the batched tensor-core sweeps (L1_ENGINE_TC, tune = 0).  No counterpart in
 * the paper: it concerns how the products of Algorithm 2's batched iteration
 * are tiled.  For each sweep shape and timed batch width it tried 128-wide
 * output tiles with the epilogue fused into the sweep or deferred to a second
 * kernel that reads the tile's FP32 sums, split-K with every slice count that
 * fills at most four waves of one CTA per multiprocessor, and 64-wide tiles
 * (deferred, split-K),
 * and kept the fastest (the simplest within 2 %).  Writes up to cap entries
 * of 7 int32 each to out (host): the sweep's output rows M, its depth K, the
 * batch width as a count of 128 x 128 output tiles, the number of K slices, 1
 * if the epilogue is deferred, the tile width (128 or 64), and the chosen
 * launch's measured time in microseconds (rounded); returns the number of
 * entries written (0: no tuning was done), or L1_ERR_INVALID_ARG for a null
 * handle, or for out == NULL with cap > 0.
 */
L1_API int l1_tuning(l1_handle h, int32_t* out, int32_t cap);

/*
 * l1_align_batch -- the convex step of the face-alignment loop (§II-B, the
 * last problem displayed there): for k < count, min ||e||_1 s.t.
 * b_k = B_k w + e with B_k tall (m x p, p <= 32, p < m; in the paper the
 * training images of one subject beside the negated Jacobian of the
 * transformation) and w not penalised.  Reading R16: Algorithm 1 with its
 * x-step replaced by the exact least-squares minimiser over w (B_k^T B_k
 * inverted once per problem in FP64), e-step and multiplier step as in
 * Algorithm 1, xi = 2m/||b_k||_1 (or xi0 > 0) held fixed, from w = 0,
 * e = b_k, theta = 0; each problem stops on the relative change of [w; e]
 * (§VI-C) below tol, or after max_outer iterations.
 *   B      device, problem k at B + k strideB, column-major with leading
 *          dimension ldB >= m (strideB >= ldB p)
 *   b      device, problem k at b + k strideb (strideb >= m)
 *   w, e   device outputs: w of problem k at w + k p, e at e + k m
 *   res    host, count results: status (L1_NONFINITE also for a B_k^T B_k
 *          that is singular to working precision), iters, rel_change,
 *          primal_obj = ||e||_1, param = xi; dual_obj, gap, resid NaN
 * One CTA per problem holds B_k and the m-vectors in shared memory, so
 * 4 (m p + 4 m) bytes + 17 KB must fit 200 KB.  The call allocates a small
 * result buffer and synchronises the stream.  Needs no handle.
 * Errors: L1_ERR_INVALID_ARG (sizes, strides, null pointers, a problem too
 * large), L1_ERR_OOM, L1_ERR_CUDA.
 */
L1_API int l1_align_batch(const float* B, int64_t m, int64_t p, int64_t ldB, int64_t strideB, const float* b,
                          int64_t strideb, int64_t count, double tol, int32_t max_outer, double xi0, void* stream,
                          float* w, float* e, l1_result* res);

/*
 * l1_align_warp -- the image side of the alignment loop (§II-B, reading R19):
 * for each task k < count, the warped query b_k = y_k o tau_k and the negated
 * Jacobian -d(y_k o tau_k)/d tau_k on the rows x cols canonical frame.
 * tau_k = (a, b, tx, ty) is a similarity: canonical pixel (u, v) (column u,
 * row v, vector index v cols + u) lies at x = a u - b v + tx, y = b u + a v
 * + ty of the query image.  y o tau is the bilinear interpolant of the query
 * at that point clamped to [0, W-1] x [0, H-1] (cell with lower corner
 * (min(floor x, W-2), min(floor y, H-2))); its derivative in x (in y) is the
 * interpolant's slope in that cell, 0 where x (y) was clamped.  Coordinates
 * and weights FP64, pixels and outputs FP32.
 *   img     device, query k at img + k img_stride, row-major H x W (H, W >= 2)
 *   tau     device, 4 doubles per task
 *   B       device, task k at B + k strideB, column-major with leading
 *           dimension ldB >= rows cols; columns col0 .. col0 + 3 receive -J
 *           (strideB >= ldB (col0 + 4))
 *   b       device, task k at b + k strideb (strideb >= rows cols)
 *   active  device, count flags, or NULL: tasks with a zero flag are skipped
 * Enqueued on stream, no synchronisation.  count <= 65535.
 * Errors: L1_ERR_INVALID_ARG (null pointers, sizes, strides), L1_ERR_CUDA.
 */
L1_API int l1_align_warp(const float* img, int64_t H, int64_t W, int64_t img_stride, const double* tau,
                         int64_t count, int32_t rows, int32_t cols, int32_t col0, void* stream, float* B, int64_t ldB,
                         int64_t strideB, float* b, int64_t strideb, const int32_t* active);

/*
 * l1_align_images -- the face-alignment loop of §II-B (reading R19) for count
 * tasks: task k aligns its query image to its subject's n training images
 * by repeating b = y o tau, J = d(y o tau)/d tau (l1_align_warp), the convex
 * step min ||e||_1 s.t. b = [A_k, -J] w + e (l1_align_batch to the relative
 * change tol, at most max_outer iterations), tau <- tau + dtau with dtau the
 * last four entries of w, until dtau moves no corner of the canonical frame
 * by tau_tol pixels or more (status L1_CONVERGED), after max_align steps
 * (L1_MAX_ITER), or when a step is not finite or its B^T B is singular
 * (L1_NONFINITE).
 *   img     device, query k at img + k img_stride, row-major H x W
 *   A       device, task k's training images at A + k A_stride, column-major
 *           (rows cols) x n, pixel (u, v) at row v cols + u; n + 4 <= 32 and
 *           n + 4 < rows cols
 *   tau     device, 4 doubles per task: the starting transformation in, the
 *           final one out
 *   iters, status  host, count each: alignment steps taken, final status
 * Allocates its work buffers (count ((n + 6) rows cols + n + 4) floats) and
 * synchronises the stream once per step.
 * Errors: L1_ERR_INVALID_ARG, L1_ERR_OOM, L1_ERR_CUDA.
 */
L1_API int l1_align_images(const float* img, int64_t H, int64_t W, int64_t img_stride, const float* A, int32_t n,
                           int64_t A_stride, int32_t rows, int32_t cols, int64_t count, double* tau, double tol,
                           int32_t max_outer, double tau_tol, int32_t max_align, void* stream, int32_t* iters,
                           int32_t* status);

/* Set the stream later calls enqueue on. */
L1_API int l1_set_stream(l1_handle h, void* stream);

/* Fill *info. */
L1_API int l1_get_info(l1_handle h, l1_info* info);

/* Release every device allocation of h.  NULL is a no-op. */
L1_API int l1_destroy(l1_handle h);

/* Static string naming a return code or status. */
L1_API const char* l1_status_string(int code);

/* Message of the last L1_ERR_CUDA (or of a rejected size) on this thread
 * (static storage). */
L1_API const char* l1_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* L1ALM_H */
