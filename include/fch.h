/*
 * fch.h -- C ABI of the GB300 (sm_103a) Fourier pseudo-spectral steppers for the
 * functionalized Cahn-Hilliard (FCH) gradient flow of
 *   A. Christlieb, K. Promislow, Z. Tan, S. Wang, B. Wetton, S. Wise,
 *   "Benchmark computation of morphological complexity in the functionalized
 *    Cahn-Hilliard gradient flow", arXiv 2006.04784.
 *
 * Conventions (all entry points):
 *  - Every function returns an fch_status; nothing throws across the ABI.
 *  - Grid: N x N points on the periodic square [x0, x0+L)^2, N a power of two,
 *    16 <= N <= 2048. A real field is a row-major N x N array, row index y,
 *    column index x: u[y*N + x] is the value at (x0 + x h, x0 + y h), h = L/N.
 *  - Spectra (the standalone transforms) are half spectra stored kx-major:
 *    X[kx*N + ky], kx = 0..N/2, ky = 0..N-1, interleaved complex (re, im),
 *    X(kx,ky) = sum_{x,y} u[y*N+x] exp(-2 pi i (kx x + ky y)/N)  (unnormalised);
 *    the inverse transform divides by N^2.
 *  - Host pointers are read or written during the call only and stay owned by the
 *    caller. Device pointers passed in must be device memory of the context's
 *    device; they are used in stream order on the context's stream (the caller
 *    makes their contents ready with respect to that stream) and are not
 *    retained after the work of the call has run.
 *  - Calls on one context are not thread safe; different contexts are independent.
 *  - Work is enqueued on the context's stream. fch_step, fch_set_state_device and
 *    fch_get_state_device return without waiting; an error raised on the device
 *    inside them (non-convergence, non-finite values) is reported by the next call
 *    that waits for the stream (fch_get_state, fch_energy, fch_mass,
 *    fch_get_stats, fch_run_adaptive, fch_synchronize). After a failed step every
 *    stepping call returns FCH_ESTATE until a new state is set.
 */
#ifndef FCH_H
#define FCH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FCH_OK = 0,
    FCH_EINVAL = 1,      /* bad argument (N not a power of two, dt <= 0, NULL ...) */
    FCH_ENOMEM = 2,      /* device or host allocation failed */
    FCH_ECUDA = 3,       /* a CUDA runtime call failed (see fch_last_cuda_error) */
    FCH_ENOCONV = 4,     /* PSD iteration reached psd_max_iter without meeting i_tol */
    FCH_ENONFINITE = 5,  /* a norm, energy or error estimate was not finite */
    FCH_ETIMEOUT = 6,    /* an attempt budget (max_attempts) ran out before t_final */
    FCH_ESTATE = 7       /* stepping after a failure, or before a state was set */
} fch_status;

/* The time integrators of Secs. 3.3-3.6 of the paper. */
typedef enum { FCH_IMEX = 0, FCH_SAV = 1, FCH_PSD = 2, FCH_ETD = 3 } fch_scheme;

/* FCH_FP64: every stage in double precision.
 * FCH_MIXED: transforms and pointwise stages in single precision; the mass,
 * energy, SAV inner products and auxiliary scalar, the LTE norms and the
 * step-size controller stay in double precision. At large N the single-precision
 * rounding of the transforms, amplified by the sixth-order operator in F(u),
 * dominates the AM3 error estimate; use it for fixed steps.
 * FCH_FP32X2: transforms and pointwise stages in double-float arithmetic (each
 * value an unevaluated sum of two floats, about 48 bits) on the single-precision
 * pipe; reductions and controller in double. Accuracy of the FP64 mode to ~1e-13
 * per step. */
typedef enum { FCH_FP64 = 0, FCH_MIXED = 1, FCH_FP32X2 = 2 } fch_precision;

typedef struct {
    int n;       /* grid points per side, power of two in [16, 2048] */
    double L;    /* period (paper: 4 pi) */
    double x0;   /* origin of the square (only used to document the input grid) */
} fch_grid;

typedef struct {
    /* model: regularised well W_q, eq. (e:Wq-def); energy, eq. (Functional) */
    double eps, q, gamma, b_minus, b_plus, eta1, eta2;
    /* SAV, eqs. (4.1)-(4.8): stabilisers beta1, beta2; zeta; energy shift D0 */
    double beta1, beta2, zeta, D0;
    /* ETDRK2 stabilisers, eq. (ETD-L) */
    double kappa0, kappa2;
    /* step-size controller, Sec. 3.2: safety rho_s, bounds k_min, k_max
     * (k_max applies to IMEX, SAV, ETD; PSD uses min(k_max, psd_k_max)) */
    double rho_s, k_min, k_max;
    int zero_stab_cap;   /* 1: cap A_dp at (1 + sqrt 2) k (Sec. 3.2) */
    /* PSD, Sec. 3.3: i_tol = psd_nu * sigma_tol in adaptive runs, psd_itol for
     * fixed steps; lambda from Table SearchSize unless psd_lambda > 0 */
    double psd_nu, psd_itol, psd_lambda, psd_k_max;
    int psd_max_iter;
    int prec;            /* fch_precision */
    int sync_every;      /* adaptive runs: trial steps enqueued between host checks */
    int fft_path;        /* 0: automatic; 1: shared-memory Stockham passes for every N;
                          * 2: warp-transform passes where available (FCH_MIXED, N = 1024) */
    int autotune;        /* 1: fch_create takes the tiles fch_autotune picks for (n, prec)
                          * (timing them on first use in the process); 2: the tiles
                          * fch_autotune_step picks; 0: tile_row/tile_col */
    int tile_row, tile_col; /* pass tiles: 0 default (at n = 1024 two-block-cluster
                          * column passes for FCH_FP64 / FCH_FP32X2, warp-level row passes
                          * for FCH_MIXED; in FCH_FP64 and FCH_FP32X2 at n = 128 / 256 the
                          * generic kernels with 2 / 1 rows a block and columns as -3, and
                          * in FCH_FP32X2 at n = 512 columns as -3; else the kernel built
                          * for the grid size); -1 the shared-memory kernels built for the
                          * size, without clusters or warp-level rows; -2 (tile_col,
                          * FCH_MIXED at n = 1024) the warp-level column passes; r > 0 the
                          * generic row kernel with r rows per block / the generic column
                          * kernel with r column pairs per block; tile_col = -2 - P
                          * (-3, -4, -6, ...) the generic column kernel with P pairs per
                          * block at four points a thread (radix-4 stages, twice the
                          * threads), tile_row = -2 - R the generic row kernel with R
                          * rows per block at four points a thread. Generic tiles are powers of two that fit whole
                          * warps, the row kernel's 256 threads or the column kernel's
                          * 1024 threads a block and a block's shared memory; else
                          * FCH_EINVAL */
} fch_params;

typedef struct {
    long long n_steps;     /* accepted steps since the state was set */
    long long n_rejects;   /* rejected trial steps */
    long long n_attempts;  /* trial steps */
    long long n_psd_iter;  /* PSD iterations */
    long long n_fft;       /* 2D real transforms (one field, R2C or C2R) */
    double t;              /* current time */
    double k_last;         /* last accepted step size */
    double e_last;         /* last relative LTE estimate */
    int last_psd_iter;     /* PSD iterations of the last solve */
} fch_stats;

typedef struct fch_ctx fch_ctx;
typedef struct fch_fft_plan fch_fft_plan;

/* Human-readable name of a status code (static string). */
const char *fch_status_string(fch_status s);

/* Text of the last CUDA error seen by this context; with ctx = NULL, the last
 * error of a standalone-transform call on the calling thread. */
const char *fch_last_cuda_error(const fch_ctx *ctx);

/* Fill *p with the paper's constants for well parameter q (Table t:Benchmark,
 * sub-critical row: eps = 0.1, gamma = 0.3, b_-/+ = -1/+1, eta1 = 1.45 eps,
 * eta2 = 3 eps; beta1 = 2, beta2 = 1 (Sec. 3.5); kappa0 = 1e-2, kappa2 = 15
 * (Sec. 3.6); rho_s = 0.9, k_min = 1e-9, k_max = infinity (Sec. 3.2);
 * psd_nu and psd_k_max from Table tolPSD for q = 0, 0.2, 0.5). zeta exceeds
 * -min W_q'' and D0 bounds -E1 from below as Sec. 3.5 requires; both are
 * computed here by sampling W_q. prec = FCH_FP64. */
fch_status fch_params_default(fch_params *p, double q);

/* Create a context: allocates all device buffers for grid g on the current
 * device. stream: a cudaStream_t to run on, or NULL for a stream the context
 * creates and owns. The grid and params are copied. */
fch_status fch_create(const fch_grid *g, const fch_params *p, void *stream, fch_ctx **out);
fch_status fch_destroy(fch_ctx *ctx);

/* Wait for all work enqueued on the context's stream; report device errors. */
fch_status fch_synchronize(fch_ctx *ctx);

/* Set u^0 from a host array of n_elems = N*N doubles. Clears the step history:
 * the next step is a backward-Euler start (the k_{n-1} -> infinity limit of the
 * variable-step BDF2, eq. (BDF2Coef)); SAV r^0 = sqrt(E1(u^0) + D0). */
fch_status fch_set_state(fch_ctx *ctx, const double *u_host, size_t n_elems);

/* Same from device memory; dtype 0 = float64, 1 = float32. */
fch_status fch_set_state_device(fch_ctx *ctx, const void *u_dev, int dtype);

/* Set (u^n, u^{n-1}, k_n): the next step is a full variable-step BDF2 step.
 * SAV takes r^n = sqrt(E1(u^n)+D0), r^{n-1} = sqrt(E1(u^{n-1})+D0). */
fch_status fch_set_history(fch_ctx *ctx, const double *un_host, const double *unm1_host,
                           size_t n_elems, double kn);

/* Copy u^n to the host (N*N doubles) / to device memory (dtype as above). */
fch_status fch_get_state(fch_ctx *ctx, double *u_host, size_t n_elems);
fch_status fch_get_state_device(fch_ctx *ctx, void *u_dev, int dtype);

/* One step of size dt with the given scheme (Secs. 3.3-3.6):
 * IMEX eq. (IMEX-eq); SAV eqs. (4.7)-(4.8); PSD eqs. (residual), (recurrence)
 * with i_tol = psd_itol; ETDRK2 eqs. (ETDRK2), (ETD-L). Enqueued without waiting;
 * PSD enqueues its iterations in chunks of four (as many chunks as the previous
 * solve took, then one at a time) and waits after each batch to read the stopping
 * test; chunks after convergence return at once on the device. (Captured steps --
 * fch_run_fixed, fch_run_adaptive, ensembles -- iterate PSD on the device instead.) */
fch_status fch_step(fch_ctx *ctx, fch_scheme scheme, double dt);

/* nsteps fixed steps of size dt, as nsteps fch_step calls, without host work
 * between them: after the first step, one step captured as a CUDA graph is replayed
 * (contexts with per-pass timing on take fch_step calls). In the graph, PSD's
 * iterations run in a conditional while node: a one-thread launch after each chunk
 * of four iterations reads the stopping test on the device and ends the loop once
 * it holds, the run has failed, or psd_max_iter / 4 + 3 chunks have run. Enqueued; a
 * failure inside the steps (non-finite values, PSD not converged) shows at the next
 * call that reads the control block (fch_synchronize, fch_get_stats,
 * fch_get_state). */
fch_status fch_run_fixed(fch_ctx *ctx, fch_scheme scheme, double dt, long long nsteps);

/* E(u^n) of eq. (Functional), FP64 accumulation (waits for the stream). */
fch_status fch_energy(fch_ctx *ctx, double *E);

/* m(u^n) = 1/2 int (u+1) dx (Sec. 2.3), read from the k = 0 mode. */
fch_status fch_mass(fch_ctx *ctx, double *m);

/* F(u) = Lap dE/du (eq. sFCH) of a device field u (dtype as above) into F. */
fch_status fch_rhs_device(fch_ctx *ctx, const void *u_dev, void *F_dev, int dtype);

/* SAV auxiliary variables r^n, r^{n-1} (waits for the stream). */
fch_status fch_get_sav_r(fch_ctx *ctx, double *r_n, double *r_nm1);

/* Adaptive integration to t_final with the algorithm of Sec. 3.2 (AM3
 * predictor, eq. (Predictor); relative L2 error; A_dp controller). The
 * controller runs on the device; the host waits every sync_every trial steps.
 * max_attempts bounds the number of trial steps of this call (<= 0: no bound);
 * running out returns FCH_ETIMEOUT with the state valid at the time reached.
 * stats may be NULL. */
fch_status fch_run_adaptive(fch_ctx *ctx, fch_scheme scheme, double sigma_tol, double t_final,
                            long long max_attempts, fch_stats *stats);

fch_status fch_get_stats(fch_ctx *ctx, fch_stats *stats);

/* fch_run_adaptive in three parts, for callers that enqueue trial steps without
 * waiting (the controller of Sec. 3.2 runs on the device, so no host decision
 * is needed between trials):
 *  begin   -- sets sigma_tol and t_final, takes the backward-Euler start if the
 *             history is empty and evaluates the F history; does not wait;
 *  enqueue -- enqueues n trial steps without waiting: the first trial of a run
 *             launches pass by pass (PSD waits inside it to test convergence),
 *             later ones replay one captured trial (PSD's iterations in a
 *             conditional while node, as in fch_run_fixed); trials past t_final do
 *             nothing;
 *  end     -- waits, reports device errors, fills stats (may be NULL). */
fch_status fch_adaptive_begin(fch_ctx *ctx, fch_scheme scheme, double sigma_tol, double t_final);
fch_status fch_adaptive_enqueue(fch_ctx *ctx, int n_trials);
fch_status fch_adaptive_end(fch_ctx *ctx, fch_stats *stats);

/* Device timing of the passes: with on = 1 every pass launch of this context is
 * bracketed by CUDA events recorded on the context's stream. fch_pass_times waits
 * for the stream, then returns and clears the accumulated milliseconds and launch
 * counts per pass kind: index m < FCH_NCOL is the column pass in mode m, then
 * FCH_NROW row-pass modes, then the control kernel (n >= FCH_NPASS entries). */
#define FCH_NCOL 10
#define FCH_NROW 8
#define FCH_NPASS (FCH_NCOL + FCH_NROW + 1)
fch_status fch_pass_timing(fch_ctx *ctx, int on);
fch_status fch_pass_times(fch_ctx *ctx, double *ms, long long *launches, int n);

/* ---- ensembles of independent instances ----
 * The paper integrates one instance at a time; an ensemble advances m independent
 * contexts (each its own grid size, parameters and initial data) together, for
 * parameter sweeps and seeds. fch_ensemble_create makes m contexts as fch_create
 * would (grids[i], params[i]), each on a stream of its own; the graphs of
 * fch_ensemble_run_adaptive launch on `stream` (NULL: one the ensemble creates).
 * The ensemble owns the members: use fch_ensemble_member to reach member i through
 * the single-instance API (set_state, get_state, energy, mass, stats, ...), never
 * fch_destroy it. Errors: FCH_EINVAL (m outside [1, FCH_ENSEMBLE_MAX], NULL
 * arrays), a member's fch_create status (message in fch_last_cuda_error(NULL)).
 *
 * fch_ensemble_run_adaptive runs the adaptive algorithm of Sec. 3.2 on every
 * member, from its current state, to t_final at the same sigma_tol: each member
 * begins as fch_adaptive_begin and takes one trial on its own stream; then one CUDA
 * graph, holding `rounds` trials of every member as one branch per member (the
 * branches run concurrently), is launched until every member has reached t_final,
 * or a member has failed, or max_launches launches (> 0) have run (FCH_ETIMEOUT).
 * A member that has reached t_final skips its passes in later launches. stats
 * (m entries, may be NULL) receive every member's fch_stats. Every scheme; a PSD
 * member iterates in a conditional while node of its branch (as fch_run_fixed), so
 * members with different iteration counts do not wait for one another. Members
 * with per-pass timing on: FCH_ESTATE. Returns after the members' streams are idle. */
typedef struct fch_ensemble fch_ensemble;
#define FCH_ENSEMBLE_MAX 4096
fch_status fch_ensemble_create(int m, const fch_grid *grids, const fch_params *params, void *stream,
                               fch_ensemble **out);
fch_status fch_ensemble_destroy(fch_ensemble *e);
fch_status fch_ensemble_member(fch_ensemble *e, int i, fch_ctx **ctx);
fch_status fch_ensemble_run_adaptive(fch_ensemble *e, fch_scheme scheme, double sigma, double t_final, int rounds,
                                     long long max_launches, fch_stats *stats);
/* fch_ensemble_run_adaptive_each is the same run with a scheme and a sigma_tol per
 * member (schemes[i], sigmas[i]; host arrays of m entries, read during the call):
 * the sigma_tol sweeps of Sec. 5.2 (global error and cost against sigma_tol) as one
 * ensemble. fch_ensemble_run_adaptive(e, s, sigma, ...) is this call with every
 * entry s, sigma. Errors as above; FCH_EINVAL also for NULL arrays. */
fch_status fch_ensemble_run_adaptive_each(fch_ensemble *e, const fch_scheme *schemes, const double *sigmas,
                                          double t_final, int rounds, long long max_launches, fch_stats *stats);

/* ---- learned initial iterate for the PSD iteration (a Fourier neural operator) ----
 * Sec. 3.3 starts the PSD iteration, eqs. (residual), (recurrence), from any v_0
 * (the scheme uses u*); the network predicts a better one. Inputs per sample: two
 * channels a = (u^n, (u* - u^n)/s), u* the extrapolation of eq. (Richardson), s the
 * RMS of u* - u^n; output y, the predicted (u^{n+1} - u*)/s, so v_0 = u* + s y.
 * Network: lifting to `width` channels (8, 16 or 32), `layers` Fourier layers
 * (GELU after all but the last) keeping `modes` x (2 modes - 1) Fourier modes,
 * projection through `proj` hidden channels (<= 128, proj x width <= 2048); FP32
 * throughout, on this library's kernels and real transforms. Parameters are one
 * flat float vector (order P, bP, {W_l, b_l, R_l}, Q1, bQ1, Q2, bQ2; R_l as
 * [modes (2 modes - 1)][width][width] complex, re/im interleaved); they start at 0.
 * fch_fno_forward(batch B, grid n, a [B][2][n][n], y [B][n][n], device float) keeps
 * what the backward pass needs; fch_fno_backward(target [B][n][n]) then writes the
 * gradient of mean((y - target)^2) over all B n^2 points (read with
 * fch_fno_get_grads) and that mean in *loss (may be NULL); fch_fno_adam takes one
 * Adam step with that gradient. n: power of two in [16, 2048], n >= 2 modes.
 * Errors: FCH_EINVAL (arguments), FCH_ESTATE (backward without a forward pass),
 * FCH_ENOMEM / FCH_ECUDA (reason in fch_last_cuda_error(NULL)). Work runs on
 * `stream`; the get/set calls synchronize it. */
typedef struct fch_fno fch_fno;
fch_status fch_fno_create(int width, int layers, int modes, int proj, void *stream, fch_fno **out);
fch_status fch_fno_destroy(fch_fno *f);
fch_status fch_fno_num_params(const fch_fno *f, size_t *count);
fch_status fch_fno_set_params(fch_fno *f, const float *host, size_t count);
fch_status fch_fno_get_params(fch_fno *f, float *host, size_t count);
fch_status fch_fno_get_grads(fch_fno *f, float *host, size_t count);
fch_status fch_fno_forward(fch_fno *f, int batch, int n, const float *a_dev, float *y_dev);
fch_status fch_fno_backward(fch_fno *f, const float *target_dev, double *loss);
fch_status fch_fno_adam(fch_fno *f, float lr, float beta1, float beta2, float eps);
/* fch_fno_set_bf16(f, 1): later forward passes read a bfloat16 copy of the
 * parameters (rounded to nearest even; refreshed by set_params and every Adam step),
 * products and sums staying in FP32: BF16 weights with FP32 accumulation for
 * inference. Training keeps the FP32 weights: fch_fno_backward after a forward pass
 * on the bfloat16 copy returns FCH_ESTATE. fch_fno_set_bf16(f, 0) frees the copy.
 * fch_fno_set_bf16(f, 2): as 1, and the forward pass runs its dense contractions on
 * the tensor cores (tcgen05 GEMMs, bfloat16 operands rounded to nearest even, FP32
 * sums): each spectral convolution as truncated DFTs over the retained modes instead
 * of full transforms of every channel (the DFT along x, a GEMM with K = n whose input
 * tiles arrive by TMA; the DFTs along y, the mode mixing and the inverse DFT along y
 * in FP32 kernels), the channel mixing W h fused with the inverse DFT along x, and
 * the projection Q1 h. Needs modes = 16, width 16 or 32, proj a multiple of 16 and n a
 * multiple of 128 at forward time (else FCH_EINVAL); the forward pass then
 * synchronizes its stream once to read the tensor-core kernels' status (FCH_ECUDA if
 * one of their bounded waits ran out). */
fch_status fch_fno_set_bf16(fch_fno *f, int on);

/* One PSD-BDF2 step of size dt (as fch_step with FCH_PSD) whose iteration starts
 * from the real field v0 (device, n x n, dtype 0 double / 1 float) instead of u*.
 * v0 must carry the mass of u*: the residual acts on the k != 0 modes only, so the
 * iteration keeps the k = 0 mode of its start; pass u* plus a correction of zero
 * mean. The converged iterate agrees with the plain step's to within the PSD
 * tolerance. */
fch_status fch_step_psd_from(fch_ctx *ctx, double dt, const void *v0_dev, int dtype);

/* One fixed IMEX-BDF2 (eq. IMEX-eq) or SAV-BDF2 (eqs. 4.7-4.8) step of size dt whose
 * extrapolation u* is the real field ustar (device, n x n, dtype 0 double / 1 float)
 * instead of eq. (Richardson): the explicit part is evaluated at the caller's
 * prediction of u^{n+1}, e.g. a learned one. Given the fully implicit BDF2 solution,
 * the IMEX step returns it. Mass does not depend on ustar (the k = 0 mode of either
 * solve involves u^n and u^{n-1} only). Otherwise as fch_step: FCH_EINVAL for another
 * scheme, dt <= 0, a NULL field or another dtype; FCH_ESTATE without a state. */
fch_status fch_step_from(fch_ctx *ctx, fch_scheme scheme, double dt, const void *ustar_dev, int dtype);

/* Adaptive PSD runs with a caller-given first iterate per trial (the same trial as
 * fch_adaptive_enqueue: PSD iteration, F of the trial, AM3 estimate, decision):
 *  - fch_adaptive_trial_info: after fch_adaptive_begin or a trial, the next trial's
 *    step size k and gamma = k/k_n (0 for a backward-Euler start), and whether the run
 *    is done (t_final reached or a failure); synchronizes the context's stream;
 *  - fch_get_history_device: u^n and u^{n-1} as real n x n fields (dtype as
 *    fch_get_state_device), from which the caller forms u* = u^n + gamma (u^n - u^{n-1});
 *  - fch_adaptive_enqueue_psd_from: one trial whose PSD iteration starts from v0 (a
 *    real field with the mass of u*, as fch_step_psd_from). FCH_ESTATE unless an
 *    adaptive PSD run is open. */
fch_status fch_adaptive_trial_info(fch_ctx *ctx, double *k_trial, double *gamma, int *done);
fch_status fch_get_history_device(fch_ctx *ctx, void *un_dev, void *unm1_dev, int dtype);
fch_status fch_adaptive_enqueue_psd_from(fch_ctx *ctx, const void *v0_dev, int dtype);

/* One trial of the open adaptive IMEX or SAV run (as fch_adaptive_enqueue: trial, F of
 * the trial, AM3 estimate, decision on the device) whose explicit part is evaluated at
 * the caller's u* (device, n x n, dtype 0 double / 1 float) instead of eq.
 * (Richardson), as fch_step_from does for a fixed step: the learned extrapolation
 * inside adaptive runs. FCH_EINVAL for NULL or another dtype; FCH_ESTATE unless an
 * adaptive IMEX or SAV run is open. */
fch_status fch_adaptive_enqueue_from(fch_ctx *ctx, const void *ustar_dev, int dtype);

/* The learned first iterate itself, on the device (Sec. 3.3: the PSD iteration of
 * eqs. (residual), (recurrence) may start from any v_0; eq. (Richardson) gives u*):
 * from the context's history u^n, u^{n-1} and the step ratio gam of the next step
 * (dt = 0: the next trial of the open adaptive run, gam from the control block;
 * dt > 0: a fixed step of size dt, gam = dt / k_n), it forms
 *   u* = u^n + gam (u^n - u^{n-1}),  s = RMS(u* - u^n),  a = (u^n, (u* - u^n)/s),
 *   y = net(a) (fch_fno_forward, batch 1),  v_0 = u* + s (y - mean y)
 * and writes v_0 (n x n doubles, device, caller-owned) for fch_step_psd_from or
 * fch_adaptive_enqueue_psd_from, or as the u* of fch_step_from. Sums are FP64 in a
 * fixed order; with no history (gam = 0) or u^n = u^{n-1}, s = 0 and v_0 = u*. The
 * network's forward pass runs on its own stream, ordered after the input kernels
 * and before the output kernel by events; nothing is read back to the host. The
 * first call allocates the network's input and output arrays for the grid (kept by
 * the context). Errors: FCH_EINVAL (NULL arguments, dt < 0), FCH_ESTATE (no state, a
 * failed context, or dt = 0 without an open adaptive run), the network's status. */
fch_status fch_fno_learned_start(fch_ctx *ctx, fch_fno *net, double dt, void *v0_dev);

/* ---- pass tiles (the paper has no counterpart: a GPU launch choice) ----
 * fch_autotune times the forward row pass (real fields -> pair-layout work array)
 * and the forward column pass (work array -> half spectra) at n x n in precision
 * prec as a standalone transform plan launches them (as many field pairs per launch
 * as a plan's work array holds; one pair for FCH_FP32X2), for each candidate tile: the default, the
 * plain shared-memory kernels at n = 1024 (where the default is the warp-level path
 * or the two-block clusters), the warp-level column passes (FCH_MIXED, n = 1024), and
 * the generic kernels at 1, 2, 4, 8, 16 rows (column pairs) per
 * block that fit. It allocates and frees its own scratch arrays on the given
 * stream (NULL: the legacy default stream), synchronizes it, and keeps the fastest
 * tiles per (n, prec) for the process: later calls return them without timing,
 * contexts created with params.autotune = 1 and plans created afterwards use them.
 * Tiles change launch shapes only; every tile computes the same transform (results
 * may differ in rounding where the warp-level and shared-memory paths differ).
 * Errors: FCH_EINVAL (n not a power of two in [16, 2048], prec not 0..2, out NULL),
 * FCH_ECUDA (reason in fch_last_cuda_error(NULL)). fch_autotune_reset forgets the
 * kept choices. */
typedef struct {
    int tile_row, tile_col;               /* chosen tiles (meaning as in fch_params) */
    double row_us, col_us;                /* mean time of one launch with them */
    double row_default_us, col_default_us; /* the same with the default tiles */
    int candidates;                       /* tiles timed */
} fch_tile;
fch_status fch_autotune(int n, int prec, void *stream, fch_tile *out);
fch_status fch_autotune_reset(void);
/* fch_autotune_step picks the tiles by timing what a context runs: adaptive IMEX
 * trials (sigma_tol 1e-5, default parameters at q = 0, a circular bilayer) of a
 * scratch context per candidate, the row tiles first (default columns), then the
 * column tiles with the chosen rows; a tile replaces the default only if 3 % faster.
 * At small n the transform-only timing of fch_autotune can mislead: fewer rows a
 * block speed up the bare transform but slow the fused passes. out: the chosen tiles;
 * row_us / col_us the mean trial time after each search, *_default_us the same with
 * the default tiles of that search, candidates the contexts timed. Kept per
 * (n, prec) for the process (reset by fch_autotune_reset); contexts created with
 * params.autotune = 2 use them. Errors as fch_autotune, and any status of fch_create
 * for the scratch contexts (FCH_ENOMEM). */
fch_status fch_autotune_step(int n, int prec, void *stream, fch_tile *out);

/* ---- measured arithmetic peaks (the paper has no counterpart) ----
 * fch_alu_peak times a kernel of independent fused multiply-add chains (eight per
 * thread, 256 threads a block, eight blocks per SM, no memory traffic) on the
 * current device and returns the best of five timed launches (after one warm-up)
 * as floating-point operations per second (an FMA counts as two): the peak of the
 * FP32 pipe for prec = FCH_MIXED, of the FP64 pipe for prec = FCH_FP64. These are
 * the denominators of the passes' arithmetic roofline (double-float passes run on
 * the FP32 pipe). sm_count (may be NULL) receives the device's SM count. Allocates
 * and frees an 8-byte device word; runs on `stream` (NULL: the legacy default
 * stream) and synchronizes it. Errors: FCH_EINVAL (another prec, flops_per_s NULL),
 * FCH_ENOMEM, FCH_ECUDA (reason in fch_last_cuda_error(NULL)). */
fch_status fch_alu_peak(int prec, void *stream, double *flops_per_s, int *sm_count);

/* ---- standalone 2D real transforms (the paper's cost unit, Sec. 1) ---- */

/* Plan for N x N real transforms in precision prec on the given stream (NULL:
 * the legacy default stream). Allocates a work array of c N x N complex elements,
 * c = min(64, max(1, 64 MiB / (N^2 x element size))): the field pairs one launch
 * transforms. The plan must not be used from two streams at once. */
fch_status fch_fft_plan_create(int n, int prec, void *stream, fch_fft_plan **out);
fch_status fch_fft_plan_destroy(fch_fft_plan *plan);

/* batch real fields x[b][N][N] -> half spectra X[b][N/2+1][N] (layout above);
 * elements are double (FCH_FP64) or float (FCH_MIXED). Fields 2j, 2j+1 share one
 * complex transform; up to c such pairs go in one row and one column launch (the
 * odd last field alone). Enqueued, no wait. */
fch_status fch_fft_r2c(fch_fft_plan *plan, const void *x_dev, void *X_dev, int batch);

/* inverse of fch_fft_r2c (divides by N^2); X is not modified. */
fch_status fch_fft_c2r(fch_fft_plan *plan, const void *X_dev, void *x_dev, int batch);

/* Synchronizes the plan's stream and reports whether the plan's transforms since its
 * creation (or the previous call) ran into a device-side timeout: the single-precision
 * column passes at N = 1024 fetch their input by bulk copies (the TMA engine) and wait
 * for each at most 1 s; a wait that runs out (not expected) leaves the rest of that
 * pass's work unwritten and sets the plan's error word. FCH_OK, or FCH_ECUDA (the word
 * was set, and is cleared; or the stream reports an error) with the reason in
 * fch_last_cuda_error(NULL); FCH_EINVAL for a NULL plan. */
fch_status fch_fft_plan_status(fch_fft_plan *plan);

/* ---- standalone R2C transform without device allocation ----
 * The paper has no counterpart to this entry point; it serves callers that must
 * not allocate device memory once running (another component owns the device's
 * memory budget, cudaMalloc/cudaFree could synchronize the device and stall other
 * work, or the caller's rules forbid dynamic allocation after start-up).
 * Same transform, layouts and precisions as fch_fft_r2c, for n <= FCH_NOALLOC_MAX_N;
 * the work array and twiddle table live in a fixed array inside the library
 * (n^2 + n complex doubles at the maximum n, about 4 MiB), which every GPU that
 * loads the library holds until the process exits. Nothing is allocated, freed or
 * created: no cudaMalloc, cudaFree, plan or library allocation.
 *  - n > FCH_NOALLOC_MAX_N, n not a power of two >= 16, prec not 0/1, NULL
 *    pointers: FCH_EINVAL, with the reason in fch_last_cuda_error(NULL).
 *  - The first call on a device looks up that array's device address with the
 *    device current and caches it; make that first call before any stream capture.
 *    The cached address belongs to the device's context of that moment: after
 *    cudaDeviceReset, do not call this entry point again in the process.
 *  - All calls share the array and it keeps the last call's contents; nothing in it
 *    needs clearing (each call rewrites the twiddles and writes each work element
 *    before reading it). Calls whose GPU work overlaps (different streams or host
 *    threads) race on the array and must be ordered by the caller.
 *  - stream: a cudaStream_t, or NULL for the legacy default stream. Enqueued, no wait. */
#define FCH_NOALLOC_MAX_N 512
fch_status fch_fft_r2c_noalloc(int n, int prec, const void *x_dev, void *X_dev, int batch, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FCH_H */
