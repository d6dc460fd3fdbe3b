/*
 * ssm.h -- C ABI of the GB300 (sm_103a) split-step-method library.
 *
 * The library advances the N-particle system of a McKean-Vlasov SDE
 * (Chen & dos Reis, arXiv:2105.09688, §1 Eq. (MV-SDE Propagation))
 *
 *   dX^i = ( v(X^i, mu^N) + b(X^i, mu^N) ) dt + sigma(X^i, mu^N) dW^i,
 *   mu^N = (1/N) sum_j delta_{X^j}    (self term included, weight 1/N)
 *
 * with the split-step method (SSM) of §2.3 (eq. SSTM:scheme 1, SSTM:scheme 2)
 * on the uniform grid t_n = n h, h = T/M:
 *
 *   step 1 (implicit):  Y_i  = X_i + h v(Y_i, mu^X_n)          (mu^X_n frozen)
 *   step 2 (explicit):  X'_i = Y_i + h b(Y_i, mu^Y_n) + sigma(Y_i, mu^Y_n) dW_n^i
 *
 * Every step of that path runs in this library's CUDA kernels on one GPU.
 *
 * Conventions shared by all entry points
 *  - Every function returns ssm_status and never aborts the process.
 *  - Host arrays are owned by the caller and copied; particle arrays on the host
 *    are particle-major, x[d*i + c], i < N, c < d, IEEE double.
 *  - Device memory of a context is owned by the context (allocated in
 *    ssm_create, or carved from a caller-owned workspace given in ssm_opts).
 *  - The CUDA stream in ssm_opts is borrowed: work is enqueued on it and the
 *    functions that return host data synchronise it.
 *  - Errors detected on the device (non-finite state, implicit solve not
 *    converged, a bounded wait that gave up) are sticky: once seen, every later
 *    call on that context returns the same status until ssm_destroy.
 *  - Functions are not thread-safe on one context; distinct contexts are
 *    independent.
 */
#ifndef SSM_H
#define SSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SSM_OK = 0,
    SSM_EINVAL = 1,      /* bad argument (size, step size beyond Theorem 2.3's bound, ...) */
    SSM_ENOMEM = 2,      /* device allocation failed or workspace too small */
    SSM_ECUDA = 3,       /* a CUDA runtime call failed */
    SSM_ENOCONV = 4,     /* an implicit solve missed its tolerance within newton_kmax passes */
    SSM_ENONFINITE = 5,  /* a particle state became NaN or infinite */
    SSM_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
    SSM_ESTATE = 7,      /* call not valid in the context's state (e.g. past t = T) */
    SSM_EBOUNDS = 8      /* debug build only (ssm_build_flags): a kernel index fell outside the
                            array it addresses; the access was skipped (results of that call
                            are not valid) */
} ssm_status;

/* Coefficient sets (v, b, sigma) built into the library.
 *  SSM_COEF_CUBIC1D_GAUSS (d = 1): v(x) = x - x^3;
 *      b(y, mu) = 0.5 int (z - y) exp(-(y - z)^2) mu(dz);  sigma(y) = 0.4 y + 0.1.
 *      Step 1 is a scalar cubic, solved in closed form (Cardano).
 *  SSM_COEF_COUPLED3D (d = 3): v(y, mu) = -y|y|^2 + 0.5 int (z - y)/(1 + |y - z|^2) mu(dz);
 *      b(y, mu) = int (z - y) exp(-|y - z|^2 / 2) mu(dz);  sigma(y) = diag(0.3 y_k + 0.2).
 *      Step 1 couples every particle to mu^X through an O(N) sum per particle,
 *      solved by Newton-type iterations whose N^2 pair sums run on the GPU.
 *  SSM_COEF_OU (any d, componentwise; §3.4.1 Eq. (stablity:OU)): v(x) = rho x,
 *      b(mu) = lambda int z mu(dz), sigma = eta, with (rho, lambda, eta) taken
 *      from ssm_opts.coef_params[0..2].
 *  SSM_COEF_COUPLED1D (d = 1): the three formulas of SSM_COEF_COUPLED3D at d = 1.
 * The paper's examples whose measure enters through means (step 1 per particle,
 * no pair sums; the parameters come from ssm_opts.coef_params):
 *  SSM_COEF_GL1 (d = 1; §3.2 Eq. (MV-GL-SDE-veresion1)), params (s, c): v(x) = -x^3,
 *      b(y, mu) = s^2/2 y + c int z mu(dz), sigma(y) = s y.  Step 1: y + h y^3 = x.
 *  SSM_COEF_GL2 (d = 1; §3.2 Eq. (MV-GL-SDE-veresion2)), params (s, c):
 *      v(x, mu) = -x^3 + c int z mu(dz), b(y) = s^2/2 y, sigma(y) = s y.
 *  SSM_COEF_POLY (d = 1; §3.3 Eq. (poly1)), params (gamma): v(x, mu) = gamma x
 *      - x int z^2 mu(dz), b(mu) = int z mu(dz), sigma(y) = y.  Step 1 is linear.
 *  SSM_COEF_CS (d = 2, x = (V, X); §3.4 Cucker-Smale), params (lambda, s):
 *      v = (-V^3, 0), b = (1 + lambda int (z - V) mu^V(dz), V),
 *      sigma = diag(s int (z - V) mu^V(dz), 0) -- the sign of the paper's particle
 *      system (a pull towards the mean velocity), not of its coefficient display.
 *  SSM_COEF_GLSTAB (d = 1; §3.4.2 Eq. (satblity:MV-GL-SDE)), params (gamma): the
 *      stability example with gamma x moved from v to b (Remark on the L_v constraint):
 *      v(x) = -(5/2 + gamma) x - x^3/4, b(y, mu) = int z mu(dz) + gamma y, sigma(y) = y.
 *      Accepted for any h with 1 + h (5/2 + gamma) > 0 (a unique step-1 root): the
 *      paper's study runs it outside Theorem 2.3's step bound on purpose. */
typedef enum { SSM_COEF_CUBIC1D_GAUSS = 0, SSM_COEF_COUPLED3D = 1, SSM_COEF_OU = 2, SSM_COEF_COUPLED1D = 3,
               SSM_COEF_GL1 = 4, SSM_COEF_GL2 = 5, SSM_COEF_POLY = 6, SSM_COEF_CS = 7,
               SSM_COEF_GLSTAB = 8 } ssm_coef;

/* Arithmetic of a step.
 *  SSM_FP64: IEEE double throughout.
 *  SSM_FP32C: pair terms in FP32, summed in FP32 over blocks of 256 sources whose
 *      block sums are combined with error-free (two-sum) compensation and then in
 *      double; the Newton residual, the per-particle solves and the state stay in
 *      double.  Step 2 draws the same Philox words but evaluates the Box-Muller
 *      transform in FP32 (|z error| < 5e-6) and forms the increment h b + sigma dW
 *      in FP32 before adding it to the FP64 state; the moments are FP32 powers
 *      summed in FP32 over 32 particles and in double beyond.
 *      X_0 is drawn in FP64 in both forms.
 *  SSM_FP32C_LEARNED: SSM_FP32C with a learned initial guess for step 1
 *      (SSM_COEF_COUPLED3D only; load weights with ssm_ws_load). */
typedef enum { SSM_FP64 = 0, SSM_FP32C = 1, SSM_FP32C_LEARNED = 2 } ssm_precision;

typedef struct {
    int precision;          /* ssm_precision; default SSM_FP64 */
    double newton_tol;      /* step 1 stops when max_c |r_c| <= newton_tol, with
                               r = Y - X - h v(Y, mu^X); 0 = default: 1e-13 (FP64);
                               FP32 forms: max(1e-10, 2^-27 h (1 + 64/sqrt(N))), i.e. 1e-10
                               at h <= 2^-8, N >= 2^14, and the FP32 evaluation floor of
                               the residual at larger h or small N */
    int newton_kmax;        /* maximum N-body passes of one implicit step; default 12 */
    int fine_log2;          /* 0: dW on the step's own grid.  L > 0: the Brownian path
                               lives on the grid T 2^-L (h must be a multiple of it) and
                               dW over a step is the sum of its fine increments, so runs
                               at different h share one path (§3). */
    double x0_mean;         /* X_0 = x0_mean + x0_std Z, Z ~ N(0, I_d); default 0 */
    double x0_std;          /* default 1 */
    double coef_params[4];  /* OU: rho, lambda, eta; GL1/GL2: s, c; POLY: gamma; CS: lambda, s;
                               GLSTAB: gamma */
    void *stream;           /* cudaStream_t to enqueue on (borrowed); NULL = default stream */
    void *workspace;        /* optional caller-owned device memory, >= ssm_workspace_bytes(),
                               256-byte aligned; NULL = the context allocates */
    size_t workspace_bytes;
    int tile_chunks;        /* 0 = tuned; else number of source chunks per pair pass */
    int ws_passes;          /* learned form: passes from the learned start before the
                               plain restart; default 4 */
    int measure_y;          /* coupled sets: 0 (default) = step 1 against mu^X, the SSM of
                               §2.3; 1 = step 1 against mu^Y, the joint R^{dN} system
                               Y_i = X_i + h v(Y_i, mu^Y) of the earlier implicit scheme that
                               §1 contrasts with the SSM, solved by block-Jacobi passes (each
                               an O(N^2) pair pass at the common iterate) to newton_tol.
                               Not with SSM_FP32C_LEARNED. */
    int ws_forward;         /* learned form: the network's forward in the start of step 1 on
                               0 (default) the tensor cores (mma.sync m16n8k16, BF16 operands,
                               FP32 accumulation) or 1 the CUDA cores (FFMA, FP32 activations);
                               the default is the faster one measured (ssm_pair_pass(ctx, 2)
                               times it) */
    int fixed_pass_launches; /* 0 (default): the passes of step 1 (coupled sets against mu^X)
                               run as a device-driven loop, a conditional node of the step's
                               CUDA graph that launches only passes with work.  1: the step
                               graph holds newton_kmax pass launches, those past the last
                               working pass exit at once -- for profilers that do not follow
                               conditional graph nodes.  Same arithmetic, same results. */
    int inject;             /* test hook of the debug build (ssm_build_flags() has
                               SSM_BUILD_CHECK_BOUNDS): 1 = every step-1 start plants particle
                               index N in entry 0 of the active list (coupled sets against mu^X,
                               N not a multiple of 128, so the index lies inside the padded
                               arrays) for the bounds checks to report as SSM_EBOUNDS.  Must be 0
                               otherwise (SSM_EINVAL). */
    int carry_start;        /* coupled sets (single contexts and batches), SSM_FP64 and
                               SSM_FP32C, step 1 against mu^X: 0
                               (default) = step 1 starts at Y = X; 1 = from the second step of
                               a run on (and after ssm_set_state at the same step index) it
                               starts at the root of u = X + h(-u|u|^2 + S* / 2), S* the
                               particle's converged pair sum of the previous step: a warm start
                               of the same solve (no counterpart in the paper), the roots are
                               certified to newton_tol as before, about one pass fewer.
                               SSM_EINVAL with other sets, forms or measure_y. */
} ssm_opts;

typedef struct {
    int64_t steps;           /* SSM steps taken by this context */
    int64_t newton_passes;   /* N-body passes of step 1, summed over steps */
    int64_t newton_rows;     /* targets evaluated in those passes (pairs = rows * N) */
    int64_t drift_rows;      /* targets evaluated by the step-2 pair sums */
    int64_t fallbacks;       /* learned starts that missed the tolerance and restarted */
    int64_t max_passes;      /* largest pass count of one implicit step */
    int64_t hist[16];        /* particles that converged after k passes (last step), k < 16 */
    int64_t floor_accepts;   /* FP32 forms: particles whose step-1 residual was still above
                                newton_tol (at most 64 newton_tol) when its decrease from the
                                previous pass fell below tenfold, the evaluation floor of FP32
                                pair sums, and that were accepted there (0 in SSM_FP64).  With
                                step 1 against mu^Y: those of each step's last pass. */
} ssm_stats_t;

typedef struct ssm_ctx ssm_ctx;

/* Fill *opts with the defaults listed above. */
void ssm_opts_default(ssm_opts *opts);

/* Bytes of device memory a context of this shape needs (for ssm_opts.workspace). */
size_t ssm_workspace_bytes(int d, int64_t N, int coef, const ssm_opts *opts);

/* Create a context for N particles in R^d on [0, T] with step h (§2.3: M = T/h
 * steps; h must divide T to 1e-12 relative).  Draws X_0 on the device from the
 * Philox4x32-10 stream of `seed` (stream 0).  Rejects with SSM_EINVAL: d not
 * supported by `coef` (CUBIC1D, COUPLED1D, GL1, GL2, POLY: 1; COUPLED3D: 3; CS: 2;
 * OU: 1..3), a precision the set
 * has no form for (SSM_FP32C_LEARNED is COUPLED3D only), N < 1 or N > 2^26,
 * h <= 0, T <= 0, or h above the step-size bound of Theorem 2.3,
 * h <= 1/(1 + 2 L_v) when L_v > -1/2 (L_v = 1 for CUBIC1D, 1/16 for COUPLED3D,
 * rho for OU, 0 for GL1, GL2 and CS, gamma for POLY).  *out receives the context,
 * or NULL on error. */
ssm_status ssm_create(int d, int64_t N, double h, double T, int coef, uint64_t seed,
                      const ssm_opts *opts, ssm_ctx **out);

/* Enqueue one SSM step n -> n+1 (steps 1 and 2 above).  Asynchronous.
 * SSM_ESTATE if the context is already at n = M. */
ssm_status ssm_step(ssm_ctx *ctx);

/* Enqueue k steps (k >= 0, n + k <= M), replayed from a CUDA graph of one step. */
ssm_status ssm_run_steps(ssm_ctx *ctx, int64_t k);

/* Enqueue the remaining steps up to n = M. */
ssm_status ssm_run(ssm_ctx *ctx);

/* Wait for enqueued work and report any device-detected error. */
ssm_status ssm_sync(ssm_ctx *ctx);

/* Raw empirical moments of the current state, out[k*d + c] = (1/N) sum_i x_{i,c}^(k+1),
 * k = 0..3 (caller-owned host array of 4*d doubles).  Synchronising. */
ssm_status ssm_moments(ssm_ctx *ctx, double *out);

/* Copy the current state X_n to the caller's host array x[N*d] and the step
 * index to *n (either may be NULL).  Synchronising. */
ssm_status ssm_get_state(ssm_ctx *ctx, double *x, int64_t *n);

/* Replace the state by x[N*d] (host, particle-major) at step index n (0 <= n <= M).
 * Brownian increments are a pure function of (seed, particle, step), so a run
 * resumed from (X_n, n) continues bit for bit.  Asynchronous w.r.t. the device. */
ssm_status ssm_set_state(ssm_ctx *ctx, const double *x, int64_t n);

/* Stages of the last step, copied to a host array [N*d] (particle-major). */
enum { SSM_STAGE_Y = 0, SSM_STAGE_B = 1 };
ssm_status ssm_get_stage(ssm_ctx *ctx, int which, double *out);

/* Counters of the work done (synchronising). */
ssm_status ssm_stats(ssm_ctx *ctx, ssm_stats_t *out);

/* Release the context and its device memory (not a caller workspace).  NULL-safe. */
void ssm_destroy(ssm_ctx *ctx);

/* Human-readable name of a status code. */
const char *ssm_status_str(int status);

/* Measured throughput of the FP32 pipes on the current device (no counterpart in the
 * paper; a roofline basis for the pair sums): out[0..3] = FP32 lane operations per
 * clock per SM of a sustained stream of FFMA, packed FFMA2, MUFU reciprocal
 * (rcp.approx) and MUFU base-2 exponential (ex2.approx), each on eight independent
 * register chains per thread over eight 256-thread blocks per SM; out[4] = the SM
 * clock in GHz during the runs (clock64 against the global timer).  Synchronous,
 * on the default stream, a few milliseconds; allocates and frees a small buffer.
 * out: caller-owned host array of 5 doubles. */
ssm_status ssm_pipe_probe(double *out);

/* Build variant of the loaded library: a bit set of SSM_BUILD_* (0 = release).
 * SSM_BUILD_CHECK_BOUNDS: compiled with SSM_CHECK_BOUNDS, the debug build whose
 * kernels check the indices they take from data (active lists, counts, ensemble
 * lookups) against the arrays they address, skip an access that falls outside and
 * report it as SSM_EBOUNDS at the next synchronising call, without trapping (a
 * stand-in for a memory checker).  Its words are per process, so a hit is
 * reported by the next synchronising call of any context or batch. */
enum { SSM_BUILD_CHECK_BOUNDS = 1 };
int ssm_build_flags(void);

/* ---- component entry points (the same device code as the step, for checks) ---- */

/* Philox4x32-10 (Salmon et al., SC'11) of n counters ctr[4*k .. 4*k+3] under the key
 * (seed mod 2^32, seed >> 32), computed on the device; out[4*n] (host arrays).
 * The paper leaves the random source open; this is the library's. */
ssm_status ssm_philox(uint64_t seed, const uint32_t *ctr, int64_t n, uint32_t *out);

/* The d standard normals of particles 0..N-1 at counter (i, step, stream) that the
 * step uses (Box-Muller of Philox uniforms), out[N*d] on the host. */
ssm_status ssm_normals(uint64_t seed, int d, int64_t N, int64_t step, int stream, double *out);

/* The same normals as the FP32C forms evaluate them (FP32 Box-Muller of the same
 * Philox uniforms, with the library's own FP32 log and cos/sin of pi a; |error| <
 * 5e-6 against ssm_normals), out[N*d] on the host. */
ssm_status ssm_normals_fp32(uint64_t seed, int d, int64_t N, int64_t step, int stream, float *out);

/* The binary64 -> binary32 (round to nearest even) and binary32 -> binary64
 * conversions that the FP32C kernels perform with integer instructions, run on
 * the host on the same source: out32[k] = (float)in[k], out64[k] = (double)out32[k]
 * for k < n (host arrays), except that inputs of magnitude below 2^-126 (the
 * binary32 subnormal range and below) give a zero of the same sign.  Overflow
 * gives infinity, NaN stays NaN.  For checking them against another
 * implementation. */
ssm_status ssm_convert_check(const double *in, int64_t n, float *out32, double *out64);

/* The constant beta of the mean-square stability theorem of §2 (label
 * SSTM:stabilty, eq. (SSTM:beta formula)): for two SSM runs X, Z driven by the same
 * noise, sup_i E|X_n^i - Z_n^i|^2 <= (1 + beta h)^n sup_i E|X_0^i - Z_0^i|^2, with
 *   beta = ((2 L_v + A + 1 + L_vt) + h (L_vt A + B) + h^2 B L_vt) / (1 - h (2 L_v + 1)),
 *   A = 2 sqrt(L_b) + 2 sqrt(L_bt) + L_s + L_st,  B = L_b + L_bt,
 * from the one-sided Lipschitz constant L_v of v, the measure-Lipschitz constant
 * L_vt of v and the squared Lipschitz constants (L_b, L_bt) and (L_s, L_st) of b and
 * sigma in space and measure.  Host arithmetic, no device.  The bound needs
 * 1 - h (2 L_v + 1) > 0 (the theorem's choice of h); beta is returned whenever the
 * denominator is nonzero.  SSM_EINVAL for a negative constant (other than L_v), a
 * non-finite input or a zero denominator. */
ssm_status ssm_stability_beta(double Lv, double Lvt, double Lb, double Lbt, double Ls, double Lst, double h,
                              double *beta);

/* Step 1 for SSM_COEF_CUBIC1D_GAUSS alone: y[k] = the real root of
 * h y^3 + (1 - h) y - x[k] = 0 (Lemma 4.1's F_h for v = x - x^3), 0 < h < 1/3. */
ssm_status ssm_cardano(const double *x, int64_t n, double h, double *y);

/* Enqueue one full O(N^2) pair-sum pass of the context's current state on its
 * stream, for timing and profiling the dominant kernel in isolation:
 *   which = 0: the step-1 pair sums of SSM_COEF_COUPLED3D, (1/N) sum_j (X_j - Y_i) w_ij
 *              and (1/N) sum_j w_ij, w_ij = 1/(1 + |X_j - Y_i|^2), for all N targets
 *              at the current Y (§2.3 eq. SSTM:scheme 1);
 *   which = 1: the step-2 drift pair sums b(Y_i, mu^Y) of the context's
 *              coefficient set (§2.3 eq. SSTM:scheme 2);
 *   which = 2: the learned start of step 1 alone (SSM_FP32C_LEARNED with weights
 *              loaded; no counterpart in the paper), from the current X into Y.
 * Overwrites only the context's partial-sum scratch, or for which = 2 the stage Y
 * (the state X is untouched).  *pairs receives the number of pair evaluations
 * enqueued, 0 for which = 2 (may be NULL). */
ssm_status ssm_pair_pass(ssm_ctx *ctx, int which, int64_t *pairs);

/* Autotuner of the pair-sum launch shapes (no counterpart in the paper, whose
 * runs are on 4 CPU cores): times every compiled shape (scalar or packed-FP32
 * kernel, threads per block, targets per thread; source chunks chosen to fill
 * whole waves of the device's resident-block slots) of each pair kind the
 * context uses, on its current state and stream, then 1.5, 2 and 2.5 times the
 * chunk count of the fastest (unless ssm_opts.tile_chunks fixes it), and keeps
 * the fastest for later steps.  best_ms (may be NULL) receives the best per-pass
 * times [step-1 sums, drift].  Synchronising; overwrites only the partial-sum
 * scratch. */
ssm_status ssm_autotune(ssm_ctx *ctx, double *best_ms);

/* The launch shape in use for which = 0 (step-1 sums) or 1 (drift):
 * out[5] = {form, threads per block, targets per thread, chunks, sources per chunk},
 * form 0 = scalar kernel, 1 = packed-FP32 difference form, 2 = packed-FP32 centred
 * expansion (d = 3 FP32 forms only; same sums, fewer instructions per pair; a block
 * whose targets lie far from the ensemble mean falls back to the difference form). */
ssm_status ssm_get_plan(ssm_ctx *ctx, int which, int *out);

/* Select a launch shape explicitly: in[3] = {form (0/1/2 as in ssm_get_plan),
 * threads per block, targets per thread}; the chunk count is planned (or fixed by
 * ssm_opts.tile_chunks), not tuned.
 * SSM_EINVAL if that shape is not compiled for the context's pair kind/precision. */
ssm_status ssm_set_plan(ssm_ctx *ctx, int which, const int *in);

/* The same with the source chunk count fixed: in[4] = {form, threads per block,
 * targets per thread, chunks >= 1 (at most the context's cap: one chunk per 256
 * sources, at most 32, and the partial-sum scratch)}.  ssm_get_plan's out[0..3] of a
 * tuned context, given back here, restore its plan exactly (the chunk length is a
 * function of N, the shape and the chunk count), which is how a tuning cache skips
 * the autotuner.  SSM_EINVAL for an unknown shape or a chunk count out of range. */
ssm_status ssm_set_plan_chunks(ssm_ctx *ctx, int which, const int *in);

/* ---- batched form: many independent ensembles in one graph launch ----
 * Each ensemble is the coupled coefficient set (SSM_COEF_COUPLED3D formulas) at
 * d = 1 or d = 3, with its own N, h, T, seed and Brownian grid, stepped by the SSM
 * of §2.3 exactly as a single context would step it (same kernels' device code,
 * same Philox streams): results match ssm_create/ssm_run of each ensemble alone to
 * rounding of the pair-sum grouping.  One batch step advances every unfinished
 * ensemble by one step; ensembles with fewer steps (larger h) stop early.  The
 * whole run is one CUDA graph with device-side loops over steps and over the
 * passes of step 1 (graph conditional nodes), so ssm_batch_run is a single
 * graph launch.  Precision SSM_FP64 or SSM_FP32C (ssm_opts.precision); the other
 * ssm_opts fields used are newton_tol, newton_kmax, x0_mean, x0_std, stream. */
typedef struct {
    int d;              /* 1 or 3 */
    int64_t N;          /* particles, 1 .. 2^24 */
    double h, T;        /* step size and horizon (M = T/h steps; h <= 1/(1 + 2/16)) */
    uint64_t seed;      /* Philox key of X_0 and dW */
    int fine_log2;      /* 0: dW on the ensemble's own grid; L > 0: Brownian path on the grid T 2^-L */
} ssm_ens_desc;

typedef struct ssm_batch ssm_batch;

/* Create n <= 1024 ensembles (descriptors desc[n], host) and draw their X_0.
 * SSM_EINVAL for a bad descriptor (same rules as ssm_create).  Synchronous. */
ssm_status ssm_batch_create(int n, const ssm_ens_desc *desc, const ssm_opts *opts, ssm_batch **out);

/* Enqueue up to k batch steps (one graph launch; stops early when every ensemble
 * has reached its horizon).  Asynchronous. */
ssm_status ssm_batch_run_steps(ssm_batch *b, int64_t k);

/* Enqueue the whole run: every ensemble to its horizon, one graph launch. */
ssm_status ssm_batch_run(ssm_batch *b);

/* Wait and report device-detected errors (sticky, as for contexts). */
ssm_status ssm_batch_sync(ssm_batch *b);

/* State of ensemble e (host x[N*d], particle-major) and its step index. Synchronising. */
ssm_status ssm_batch_get_state(ssm_batch *b, int e, double *x, int64_t *n);

/* Raw moments of ensemble e, out[k*d + c], k = 0..3.  Synchronising. */
ssm_status ssm_batch_moments(ssm_batch *b, int e, double *out);

/* Work counters summed over ensembles (steps = ensemble-steps; max_passes holds
 * the number of batch steps taken).  Synchronising. */
ssm_status ssm_batch_stats(ssm_batch *b, ssm_stats_t *out);

/* Autotuner (no counterpart in the paper): times each compiled launch shape and
 * source-chunk length on the batch's pair-sum phases and rebuilds the graph with
 * the fastest; *best_ms = the best time of one step-1 pass plus one drift pass
 * over all ensembles.  Leaves the state unchanged.  Synchronising. */
ssm_status ssm_batch_autotune(ssm_batch *b, double *best_ms);

/* Launch shape in use: out[5] = {d=3 form (0 scalar, 1 packed difference form,
 * 2 packed centred expansion), threads, targets/thread d=1, targets/thread d=3,
 * sources per chunk}. */
ssm_status ssm_batch_get_plan(ssm_batch *b, int *out);

/* Select the launch shape explicitly: in[4] = {d=3 form (0/1/2 as in
 * ssm_batch_get_plan), targets/thread d=1, targets/thread d=3, sources per chunk
 * (4096, 8192 or 16384)}; rebuilds the graph.  The state is unchanged.
 * SSM_EINVAL if that shape is not compiled for the batch's precision.  Synchronising. */
ssm_status ssm_batch_set_plan(ssm_batch *b, const int *in);

/* Release the batch and its device memory.  NULL-safe. */
void ssm_batch_destroy(ssm_batch *b);

/* ---- learned initial guess of step 1 (SSM_FP32C_LEARNED, SSM_COEF_COUPLED3D) ----
 * The paper has no counterpart; its step 1 (§2.3, eq. SSTM:scheme 1) only needs
 * some convergent solver.  A network 16 -> 64 -> 64 -> 64 -> 3 (SiLU, BF16
 * weights, FP32 arithmetic) maps the features f = (x_i (3), the raw moments
 * m_k = (1/N) sum_j x_j^k, k = 1..4, per coordinate (12, k-major), h) of particle i
 * to the converged pair sum S(Y*_i) = (1/N) sum_j (X_j - Y*_i)/(1 + |X_j - Y*_i|^2);
 * step 1 then starts from the root of u = x_i + h(-u|u|^2 + S_start/2) and runs the
 * usual passes, where S_start = S_pred plus, from the second step of a run on, the
 * previous step's error S(Y*_i) - S_pred of the same particle (the part of S that
 * the network cannot see -- the fluctuation of the particular sample of N particles
 * about its law -- changes little in one step; ssm_ws_load, ssm_pair_pass(ctx, 2)
 * and ssm_set_state to another step index than the current one drop the carried
 * error for the next step).  A particle whose residual still exceeds newton_tol after
 * ssm_opts.ws_passes passes restarts from the plain start Y = X (plain Newton is
 * the judge); ssm_stats reports those restarts as fallbacks.
 *
 * Network parameters travel as one "blob" of ssm_ws_blob_bytes() bytes: header
 * (magic 0x57534D53, version 1, 16, 64, 3), feature mean/std [16]/[16], label
 * mean/std [4]/[4], biases b1, b2, b3 [64] and b4 [4] in FP32, then BF16 weights
 * W1 [64][16], W2 [64][64], W3 [64][64], W4 [4][64] (row-major, row 3 of W4 zero).
 * All arrays of these functions are host arrays owned by the caller. */
size_t ssm_ws_blob_bytes(void);

/* Number of trainable parameters (order W1, b1, W2, b2, W3, b3, W4 [3][64], b4). */
int ssm_ws_num_params(void);

/* Load a blob into a SSM_COEF_COUPLED3D context; with precision
 * SSM_FP32C_LEARNED the following steps use the learned start. */
ssm_status ssm_ws_load(ssm_ctx *ctx, const void *blob, size_t bytes);

/* Training rows from the context's last step, for particles i = offset,
 * offset + stride, ... < N: feat[r*16 + ...] = (X_n,i, moments of X_n, h) and
 * label[r*3 + c] = S(Y*_n,i); *rows receives the count.  X_n,i is rebuilt as
 * Y* - h v(Y*), exact up to the residual tolerance.  SSM_ESTATE before any step. */
ssm_status ssm_ws_collect(ssm_ctx *ctx, int64_t stride, int64_t offset, float *feat, float *label, int64_t *rows);

/* Network outputs (S_pred, unstandardised) for n feature rows: out[n*3]. */
ssm_status ssm_ws_predict(const void *blob, size_t bytes, const float *feat, int64_t n, float *out);

/* One forward + backward pass over n <= 2^20 rows: grad[num_params] = gradient of
 * the mean over rows and outputs of (net(f) - (label - mean)/std)^2 w.r.t. the
 * parameters (weights at their BF16 values); *loss = that mean (may be NULL). */
ssm_status ssm_ws_grad(const void *blob, size_t bytes, const float *feat, const float *label, int64_t n,
                       float *grad, double *loss);

/* Train a network on n rows: minibatch Adam (batch <= 65536), `epochs` shuffled
 * passes, learning rate lr with cosine decay to lr/20, weights initialised
 * N(0, 1/fan_in) from `seed`, feature and label statistics from the data.  Writes
 * the blob to blob_out (bytes >= ssm_ws_blob_bytes()) and the mean loss of each
 * epoch to loss_curve[epochs] (may be NULL).  Synchronous; uses its own device
 * buffers on the default stream. */
ssm_status ssm_ws_train(const float *feat, const float *label, int64_t n, int epochs, int batch, float lr,
                        uint64_t seed, void *blob_out, size_t bytes, double *loss_curve);

/* The parameter vector of a blob (weights at their BF16 values): params[num_params]. */
ssm_status ssm_ws_params(const void *blob, size_t bytes, float *params);

/* Step-2 pair drift without any allocation (the paper has no counterpart; this
 * is a convenience for callers that cannot allocate device memory when they need
 * it -- code in host callbacks or real-time loops that must not block on the
 * allocator, or runtimes that hand out one pre-reserved memory pool).
 *
 * Computes, for coef = SSM_COEF_CUBIC1D_GAUSS (d = 1) or SSM_COEF_COUPLED3D
 * (d = 3) and precision SSM_FP64 or SSM_FP32C, the drift b(y_i, mu^y) of that
 * coefficient set for the N particles y (device array, SoA: component c of
 * particle i at y[c*ld + i], ld >= N) into b (device array, same layout), on
 * `stream` (cudaStream_t, NULL = default stream).  Asynchronous.  The result is
 * the drift ssm_get_stage(SSM_STAGE_B) reports after a step whose Y is y, up to
 * rounding: this entry point splits the sources into its own chunks, so the
 * partial sums are grouped differently (SSM_FP64: to the rounding of the
 * regrouped double sums; SSM_FP32C: within ~1e-9 absolute, from the FP32
 * sub-tile sums).
 *
 * Its scratch is a fixed 8 MiB static device array inside the library (held by
 * every GPU that loads the library until the process exits), so d * ld must be
 * at most 2^20 (ld <= 349,525 for d = 3, <= 1,048,576 for d = 1); larger sizes
 * return SSM_ENOMEM and launch nothing.  The call allocates and frees nothing.
 * The first call on a device looks up the scratch array's device address on
 * that device (it must be current); make that first call before any stream
 * capture.  After cudaDeviceReset the device has a new context and the next
 * call looks the address up again: make it before any capture as well.  All calls share the scratch: calls that overlap on the GPU (other
 * streams, unordered threads) race; calls on one stream are safe.  Nothing in
 * the scratch needs to start at zero.  SSM_EINVAL for null pointers, N < 1,
 * ld < N or an unsupported coef/precision. */
ssm_status ssm_drift_noalloc(int coef, int precision, int64_t N, const double *y, int64_t ld, double *b,
                             void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SSM_H */
