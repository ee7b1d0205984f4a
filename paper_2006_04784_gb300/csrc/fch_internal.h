// fch_internal.h -- types shared by the host API and the CUDA kernels of libfch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fch_df.cuh"

#define FCH_MIN_N 16
#define FCH_MAX_N 2048
#define FCH_NRED 4        // reduction slots per pass
#define FCH_MAXBLK 4096   // partial sums per slot (>= the largest grid of a pass)

// Model and grid constants in the precision of a pass (filled on the host, so a
// single-precision pass does no double-precision arithmetic per element).
template <typename T> struct fch_consts {
    T kf2;            // (2 pi / L)^2
    T e2, e4;         // eps^2, eps^4
    T am, am2;        // alpha_m, alpha_m^2
    T eta1, eta2, zeta;
    T b1am_e2, b2am2; // beta1 alpha_m eps^2, beta2 alpha_m^2 (SAV L0, L1)
    T l1c;            // eps^2 (eta1 + 2 zeta) (SAV L1)
    T kappa0, k2e2;   // kappa0, kappa2 eps^2 (ETD)
    T inv_n2;         // 1 / N^2
    T bm, bp, eps, q, qeps, qoe, g3, c3; // well: b_-, b_+, eps, q, q eps, q/eps, gamma/3, (3 b_+ - b_-)/2
    // q = 0: W, W' and W'' as polynomials in u, coefficients of u^0, u^1, ...
    T wp[5], w1p[4], w2p[3];
};

// Per-trial coefficients, mirrored in both precisions by the control kernel.
template <typename T> struct fch_coef {
    T a, b, c, gam;   // eq. (BDF2Coef) and k_{n+1}/k_n
    T w1, w2, w3;     // eq. (Predictor) weights
    T lam, k1;        // PSD search step, trial step
    T r_new, isq;     // SAV r^{n+1}, 1/sqrt(E1 + D0)
};

// Device-resident stepping state: step sizes, BDF2/AM3 coefficients, SAV
// scalars, controller decisions and counters. Written only by fch_ctrl_kernel
// (one thread) and by the host between runs; read by every pass.
struct fch_ctrl {
    double t, kn, ktrial, t_final, sigma, k1;
    double a, b, c, gam;            // eq. (BDF2Coef) for the current trial, gam = k1/kn
    double w1, w2, w3;              // eq. (Predictor) weights (include k1)
    double lam, itol;               // PSD search step and stopping tolerance
    double r_n, r_m, r_new;         // SAV auxiliary variable history
    double e1, inv_sqrt_e1;         // SAV E1(u*) and 1/sqrt(E1 + D0)
    double e_last, psd_ratio, energy;
    double kmin, kmax, rho_s;
    int cap;                        // zero-stability cap on A_dp
    int iu_n, iu_m, iu_new;         // which of the three state spectra hold u^n, u^{n-1}, trial
    int if_n, if_m, if_new;         // same for F(u^n), F(u^{n-1}), F(trial)
    int done;                       // 1: t_final reached or a failure: all passes return at once
    int status;                     // fch_status of the first device-side failure
    int psd_conv, psd_iter, psd_max_iter, last_psd_iter;
    int accepted_last, adaptive, first_step;
    long long n_steps, n_rejects, n_attempts, n_psd_iter;
    double lam_tab[10], lam_k[10];  // PSD search step table row for q
    double lam_slope[10];           // (lam_tab[j+1] - lam_tab[j]) / (lam_k[j+1] - lam_k[j])
    double sigma2, lte_num, lte_den; // sigma_tol^2; last ||u~ - u_p||^2, ||u_p||^2 (Parseval sums)
    fch_coef<float> cof;            // float mirror of the coefficients above
    fch_coef<double> cod;           // double copy, read by the double-precision passes
    fch_coef<fch::df> codf;         // double-float copy, read by the FP32x2 passes
};
static_assert(sizeof(fch_ctrl) % 8 == 0, "the control kernel copies fch_ctrl as 8-byte words");

// Everything a pass needs, passed by value.
struct fch_kparams {
    int N, logN, P;                 // grid size, log2 N, column pairs per block
    int pdl;                        // launch with programmatic stream serialization
    double L, kf, inv_n2, h2;       // period, 2 pi / L, 1/N^2, (L/N)^2
    double eps, eps2, q, gamma, bm, bp, eta1, eta2, am, beta1, beta2, zeta, D0, kappa0, kappa2;
    void *U[3], *F[3];              // state spectra and F spectra (rotated through fch_ctrl)
    void *Pb, *Qb, *Vb, *Nb;        // SAV p/q, PSD iterate, ETD N(u^n)
    void *Rs[3];                    // real-space (u, Lap u) of the three state slots, N x N complex
    void *Z;                        // N x N complex pair-layout work array
    const void *tw;                 // per-stage Stockham twiddles of radix-8 stages (see fft_smem)
    const void *tw4;                // the same for radix-4 stages (contexts; null in plans)
    const void *tw2;                // N = 1024 warp transform: [k2][n1] exp(-2 pi i n1 k2 / 1024), float
    double *part;                   // [FCH_NRED][FCH_MAXBLK] per-block partial sums
    fch_ctrl *ctrl;
    unsigned long long *nfft;       // 2D real-transform counter (may be null)
    const void *in0, *in1;          // explicit inputs (standalone transforms, device fields)
    void *out0, *out1;              // explicit outputs
    int tile_row, tile_col;         // pass tiles: 0 default; -1 shared-memory kernel without the
                                    // warp-level path; > 0 generic kernel with that many rows
                                    // (column pairs) per block
    int npairs;                     // standalone transforms: field pairs of one launch (grid y; 0 = 1)
    long long pstride_in, pstride_out; // bytes from one pair's in0/in1 (out0/out1) to the next's
    int src;                        // spectrum a start pass reads (FCH_SRC_*)
    int flags;                      // FCH_FL_*
    int tail_op;                    // < 0: none; else the control op the pass's last block runs
    double tail_arg;
    unsigned int *ticket;           // arrival counter of the blocks of a pass (reset by the last)
    int *err;                       // set to 1 by a pass whose bounded wait on a bulk copy ran out (may be null)
    fch_consts<float> cf;
    fch_consts<double> cd;
    fch_consts<fch::df> cdf;
};

enum { FCH_SRC_UN = 0, FCH_SRC_UNEW = 1, FCH_SRC_V = 2, FCH_SRC_IN0 = 3 };
enum {
    FCH_FL_AM3 = 1,        // F finish: also form the AM3 predictor and the LTE norms
    FCH_FL_PACK_F = 2,     // solve passes: pack (u_new, Lap u_new) for F(u_new)
    FCH_FL_ENERGY = 4,     // F row pass: also accumulate the energy density
    FCH_FL_NOSKIP = 8,     // ignore ctrl->done (host-driven single evaluations)
    FCH_FL_COPYV = 16,     // F start from the PSD iterate: copy it into the trial slot
    FCH_FL_PSDSKIP = 32,   // pass belongs to a PSD iteration: return if converged
    FCH_FL_F64IO = 64,     // explicit real-space io in float64 (else the pass precision)
    FCH_FL_STORE_REAL = 256, // F row pass: also store (u, Lap u) into the real-space slot of src
    FCH_FL_GAMMA0 = 512,     // direct row passes: use u^n itself (gamma = 0, the ETD first stage)
    FCH_FL_USTAR_V = 1024    // SAV p/q pass: u* is the caller's field in Vb, not eq. (Richardson)
};

// column-pass modes (the fused spectral stage between the column transforms)
enum {
    CM_FWD_STORE = 0,  // forward columns -> two half spectra (standalone R2C)
    CM_INV_LOAD,       // two half spectra -> inverse columns (standalone C2R)
    CM_START,          // pack (v, Lap v) for v = u*, u^n, u_new, PSD iterate or in0
    CM_IMEX_SOLVE,     // eq. (IMEX-eq)
    CM_F_FINISH,       // F = Lap mu; AM3 predictor + norms (flag)
    CM_SAV_PQ,         // SAV p, q and their inner products
    CM_SAV_COMBINE,    // u_new = p + r q
    CM_PSD_ITER,       // one preconditioned steepest-descent update
    CM_ETD_STAGE1,     // ETDRK2 first stage
    CM_ETD_STAGE2,     // ETDRK2 second stage
    CM_NMODES
};

// row-pass modes (the fused pointwise stage between the row transforms)
enum {
    RM_R2C_LOAD = 0,   // real fields -> forward rows (standalone R2C, device fields)
    RM_C2R_STORE,      // inverse rows -> real fields
    RM_NIMEX,          // (u, Lap u) -> pieces of N_IMEX(u)
    RM_F,              // (u, Lap u) -> pieces of mu(u) (+ energy density)
    RM_SAV,            // (u, Lap u) -> pieces of V[u] (+ G(u) density)
    RM_ENERGY,         // (u, Lap u) -> energy density only
    RM_NIMEX_DIRECT,   // (u*, Lap u*) from the stored real-space slots -> pieces of N_IMEX(u*)
    RM_SAV_DIRECT,     // same -> pieces of V[u*]
    RM_NMODES
};

// control-kernel operations
enum {
    OP_INIT_TRIAL = 0, // arg0 = dt (fixed step) or < 0 (adaptive: ktrial clipped to t_final)
    OP_SAV_E1,         // E1 from partials -> 1/sqrt(E1 + D0); arg0 = 1: also r_n (set_state)
    OP_SAV_R,          // r_new from the two inner products
    OP_PSD_CHECK,      // stopping test ||d|| / ||v|| < i_tol
    OP_DECIDE,         // adaptive accept / reject and next trial size
    OP_ACCEPT,         // fixed step: accept unconditionally
    OP_ENERGY,         // energy from partials
    OP_DECIDE_INIT,    // OP_DECIDE, then OP_INIT_TRIAL (adaptive) for the next trial
    OP_ACCEPT_INIT     // OP_ACCEPT of a fixed step, then OP_INIT_TRIAL with step size arg0
};

// pass geometry for grid N and precision (0 = f64, 1 = f32)
struct fch_geom {
    int col_blocks, col_threads, col_smem;
    int row_blocks, row_threads, row_smem, rpb;
    int P;
};
fch_geom fch_geometry(int N, int prec);
// the geometry of tiles tile_row / tile_col (as in fch_kparams) at grid size N
fch_geom fch_geometry_tiled(int N, int prec, int tile_row, int tile_col);
// whether tiles tile_row / tile_col launch at grid size N (threads, shared memory)
bool fch_tile_valid(int N, int prec, int tile_row, int tile_col);

cudaError_t fch_launch_col_f64(int mode, const fch_kparams &kp, cudaStream_t s);
cudaError_t fch_launch_row_f64(int mode, const fch_kparams &kp, cudaStream_t s);
cudaError_t fch_launch_col_f32(int mode, const fch_kparams &kp, cudaStream_t s);
cudaError_t fch_launch_row_f32(int mode, const fch_kparams &kp, cudaStream_t s);
cudaError_t fch_launch_col_dfl(int mode, const fch_kparams &kp, cudaStream_t s);
cudaError_t fch_launch_row_dfl(int mode, const fch_kparams &kp, cudaStream_t s);
// launch configuration with programmatic stream serialization (when enabled)
bool fch_pdl_enabled();
void fch_pdl_config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *at, dim3 grid, dim3 block, size_t smem,
                    cudaStream_t s, bool pdl);
cudaError_t fch_launch_ctrl(int op, const fch_kparams &kp, int nblk_a, int nblk_b, double arg0,
                            cudaStream_t s);

// sets the per-thread message returned by fch_last_cuda_error(NULL)
void fch_set_thread_error(const char *msg);

// the stream a network's work runs on (fch_fno.cu)
struct fch_fno;
cudaStream_t fch_fno_stream_of(const fch_fno *f);
