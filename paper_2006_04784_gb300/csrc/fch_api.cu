// fch_api.cu -- host side of libfch: contexts, the scheme pipelines, the adaptive
// driver, the control kernel (FP64 reductions and the step-size controller) and
// the standalone transforms. The C ABI is declared in include/fch.h.
#include <math.h>
#include <mutex>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <vector>

#include "../../include/fch.h"
#include "fch_ctrl.cuh"
#include "fch_internal.h"

// ---------------------------------------------------------------------------
// geometry
fch_geom fch_geometry(int N, int prec)
{
    fch_geom g;
    const int csz = prec == 1 ? 8 : 16; // bytes per complex element (single: 8; double, double-float: 16)
    // column pairs per block: enough that a block reads whole 32-byte sectors of
    // each row (2 pairs of 8-byte or 1 pair of 16-byte elements) and has >= 256 threads
    const int pmin = csz == 8 ? 2 : 1;
    int P = 1024 / N;
    if (P < pmin) P = pmin;
    if (P > N / 2) P = N / 2;
    g.P = P;
    g.col_threads = P * N / 4; // 2P sequences x N/8 threads
    g.col_blocks = N / (2 * P);
    const int SL = N + N / 8; // skewed sequence length in shared memory
    g.col_smem = (N + 2 * P * SL) * csz;
    if (N == 1024 && csz == 16) {
        // two-block clusters, one column of a pair per block, twiddles in global memory
        g.col_threads = N / 8;
        g.col_blocks = N;
        g.col_smem = SL * csz;
    }
    // rows per block: one at N = 1024 (the compile-time kernel's 128 threads), else
    // 256 threads' worth; the row pass keeps its twiddles in global memory
    const int tps = N / 8;
    int rpb = N == 1024 ? 1 : 256 / tps;
    if (rpb < 1) rpb = 1;
    if (rpb > N) rpb = N;
    g.rpb = rpb;
    g.row_threads = rpb * tps;
    g.row_blocks = N / rpb;
    g.row_smem = rpb * SL * csz;
    return g;
}

fch_geom fch_geometry_tiled(int N, int prec, int tile_row, int tile_col)
{
    fch_geom g = fch_geometry(N, prec);
    const int csz = prec == 1 ? 8 : 16, SL = N + N / 8;
    if ((tile_col == -1 || tile_col == -2) && N == 1024) {
        // without clusters: the compile-time kernel (-1) with 1 (16-byte) or 2 (8-byte)
        // column pairs per block, or the warp-level kernel (-2, single precision) with
        // two pairs per block
        const int P = csz == 16 ? 1 : 2;
        g.P = P;
        g.col_threads = tile_col == -2 ? 128 : P * N / 4;
        g.col_blocks = N / (2 * P);
        g.col_smem = tile_col == -2 ? (N * 5 + 4 * 33 * 32) * csz : (N + 2 * P * SL) * csz;
    }
    if (tile_col > 0) {
        g.P = tile_col;
        g.col_threads = tile_col * N / 4;
        g.col_blocks = N / (2 * tile_col);
        g.col_smem = (N + 2 * tile_col * SL) * csz;
    }
    if (tile_col <= -3) {
        // the generic kernel with P = -2 - tile_col pairs a block and four points a
        // thread (radix-4 stages): twice the threads of the tile P
        const int P = -2 - tile_col;
        g.P = P;
        g.col_threads = P * N / 2;
        g.col_blocks = N / (2 * P);
        g.col_smem = (N + 2 * P * SL) * csz;
    }
    if (tile_row > 0) {
        g.rpb = tile_row;
        g.row_threads = tile_row * (N / 8);
        g.row_blocks = N / tile_row;
        g.row_smem = tile_row * SL * csz;
    }
    if (tile_row <= -3) {
        // the generic row kernel with R = -2 - tile_row rows a block at four points a thread
        const int R = -2 - tile_row;
        g.rpb = R;
        g.row_threads = R * (N / 4);
        g.row_blocks = N / R;
        g.row_smem = R * SL * csz;
    }
    return g;
}

// generic-kernel tiles: powers of two, whole blocks, whole warps (the block sums
// shuffle across all 32 lanes), at most 256 threads for the row kernel (its launch
// bound) and 1024 for the column kernel, and the opt-in shared memory of a block
// (227 KiB, less the kernels' 1 KiB of static arrays)
bool fch_tile_valid(int N, int prec, int tile_row, int tile_col)
{
    const int smem_max = 227 * 1024 - 1024;
    const int pmin = prec == 1 ? 2 : 1;
    if (tile_row > 0 || tile_row <= -3) {
        const int R = tile_row > 0 ? tile_row : -2 - tile_row;
        if ((R & (R - 1)) || R > N) return false;
        const fch_geom g = fch_geometry_tiled(N, prec, tile_row, 0);
        if (g.row_threads > 256 || (g.row_threads & 31) || g.row_smem > smem_max) return false;
    } else if (tile_row == -2) {
        return false;
    }
    if (tile_col > 0 || tile_col <= -3) {
        const int P = tile_col > 0 ? tile_col : -2 - tile_col;
        if ((P & (P - 1)) || P < pmin || P > N / 2) return false;
        const fch_geom g = fch_geometry_tiled(N, prec, 0, tile_col);
        if (g.col_threads > 1024 || (g.col_threads & 31) || g.col_smem > smem_max) return false;
    } else if (tile_col == -2 && !(prec == 1 && N == 1024)) {
        return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// control kernel: one block of 256 threads running ctrl_block
__global__ void __launch_bounds__(256) fch_ctrl_kernel(const fch_kparams kp, int op, int na, double arg0)
{
    pdl_begin();
    ctrl_block(kp, op, na, arg0);
}

cudaError_t fch_launch_ctrl(int op, const fch_kparams &kp, int na, int, double arg0, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    fch_pdl_config(cfg, at, dim3(1), dim3(256), 0, s, kp.pdl != 0);
    return cudaLaunchKernelEx(&cfg, fch_ctrl_kernel, kp, op, na, arg0);
}

// launch configuration of a pass or control kernel: programmatic stream
// serialization (see pdl_begin) where the launch asks for it (fch_kparams::pdl),
// unless FCH_NO_PDL is set in the environment
bool fch_pdl_enabled()
{
    static const bool on = getenv("FCH_NO_PDL") == nullptr;
    return on;
}

void fch_pdl_config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *at, dim3 grid, dim3 block, size_t smem,
                    cudaStream_t s, bool pdl)
{
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl && fch_pdl_enabled() ? 1 : 0;
}

// ---------------------------------------------------------------------------
// host-side model constants (product side; the test oracle has its own)
static void host_well(const fch_params &p, double u, double *W, double *W1, double *W2)
{
    const double v = u - p.b_minus;
    double A = 0.5 * v * v, A1 = v, A2 = 1.0;
    if (p.q != 0.0) {
        const double x = v / p.eps;
        const double e = exp(-fabs(x));
        const double sech = 2.0 * e / (1.0 + e * e);
        const double th = copysign((1.0 - e * e) / (1.0 + e * e), x);
        A += p.q * p.eps * (1.0 - sech);
        A1 += p.q * sech * th;
        A2 += (p.q / p.eps) * sech * (2.0 * sech * sech - 1.0);
    }
    const double w = u - p.b_plus;
    const double B = 0.5 * w * w + p.gamma / 3.0 * (u - 0.5 * (3.0 * p.b_plus - p.b_minus));
    const double B1 = w + p.gamma / 3.0;
    *W = A * B;
    *W1 = A1 * B + A * B1;
    *W2 = A2 * B + 2.0 * A1 * B1 + A;
}

// zeta > -min W_q'' and D0 >= -|Omega| min (W'^2/2 - eta2 W) + |Omega|, Sec. 3.5
static void sav_constants(const fch_params &p, double area, double *zeta, double *D0)
{
    double minW2 = 1e300, minG = 1e300;
    for (int i = 0; i <= 600000; i++) {
        const double u = -4.0 + 8.0 * i / 600000.0;
        double W, W1, W2;
        host_well(p, u, &W, &W1, &W2);
        if (W2 < minW2) minW2 = W2;
        const double g = 0.5 * W1 * W1 - p.eta2 * W;
        if (g < minG) minG = g;
    }
    *zeta = -minW2 + 0.1;
    *D0 = area * (fmax(0.0, -minG) + 1.0);
}

static int psd_row(double q) { return q < 0.1 ? 0 : (q < 0.35 ? 1 : 2); }

static const double kLamK[10] = {1e-6, 1e-5, 5e-5, 1e-4, 5e-4, 1e-3, 5e-3, 1e-2, 2e-2, 3e-2};
static const double kLamTab[3][10] = { // Table SearchSize
    {1, 1.07, 1.11, 1.14, 1.24, 1.34, 1.60, 1.738, 1.804, 1.855},
    {1, 1.04, 1.15, 1.28, 1.50, 1.70, 1.87, 1.92, 1.95, 1.97},
    {1, 1.20, 1.32, 1.45, 1.72, 1.83, 1.965, 1.97, 1.985, 1.99},
};

extern "C" fch_status fch_params_default(fch_params *p, double q)
{
    if (!p) return FCH_EINVAL;
    memset(p, 0, sizeof(*p));
    p->eps = 0.1;
    p->q = q;
    p->gamma = 0.3;
    p->b_minus = -1.0;
    p->b_plus = 1.0;
    p->eta1 = 1.45 * p->eps;
    p->eta2 = 3.0 * p->eps;
    p->beta1 = 2.0;
    p->beta2 = 1.0;
    p->zeta = 0.0; // 0: computed at fch_create from the well
    p->D0 = 0.0;   // 0: computed at fch_create for the grid's area
    p->kappa0 = 1e-2;
    p->kappa2 = 15.0;
    p->rho_s = 0.9;
    p->k_min = 1e-9;
    p->k_max = INFINITY;
    p->zero_stab_cap = 0;
    const int row = psd_row(q); // Table tolPSD: nu(q) and the optimal k_max
    const double nu[3] = {1e-3, 2e-5, 1e-6}, km[3] = {0.05, 0.02, 0.01};
    p->psd_nu = nu[row];
    p->psd_k_max = km[row];
    p->psd_itol = 1e-10;
    p->psd_lambda = 0.0;
    p->psd_max_iter = 1000;
    p->prec = FCH_FP64;
    p->sync_every = 16;
    return FCH_OK;
}

extern "C" const char *fch_status_string(fch_status s)
{
    switch (s) {
    case FCH_OK: return "ok";
    case FCH_EINVAL: return "invalid argument";
    case FCH_ENOMEM: return "out of memory";
    case FCH_ECUDA: return "CUDA error";
    case FCH_ENOCONV: return "PSD iteration did not converge";
    case FCH_ENONFINITE: return "non-finite value";
    case FCH_ETIMEOUT: return "attempt budget exhausted";
    case FCH_ESTATE: return "invalid state (failed step or no state set)";
    }
    return "unknown status";
}

// ---------------------------------------------------------------------------
// context
struct fch_ctx {
    int N, prec;
    fch_grid grid;
    fch_params p;
    cudaStream_t stream;
    bool own_stream;
    fch_geom geom;
    fch_kparams kp;      // base parameters; passes copy and adjust
    fch_ctrl hc;         // host mirror of the control block
    bool hc_fresh;       // hc equals the device's block: no launch since the last copy
    fch_ctrl *dctrl;
    double *part;
    void *U[3], *F[3], *Pb, *Qb, *Vb, *Nb, *Z, *tw, *tw4, *tw2;
    void *Rs[3];         // real-space (u, Lap u) of the state slots, kept by adaptive trials
    bool rvalid;         // Rs holds u^n (and u^{n-1} when k_n > 0)
    double *staging;     // N*N doubles for host io
    // learned first iterate (fch_fno_learned_start): network input [2][N][N] and
    // output [N][N] floats, per-block partial sums, two events; made on first use
    float *ls_a, *ls_y;
    double *ls_part;
    cudaEvent_t ls_ev[2];
    long long *nfft_dev;
    unsigned int *ticket; // [0] the pass-tail ticket, [1] the PSD loop's chunk count
    long long nfft_base;
    bool have_state, failed, have_F;
    fch_scheme ad_scheme;           // scheme of the adaptive run begun last
    bool ad_open;
    // one trial step (trial + F + decide) of each scheme captured as a CUDA graph:
    // every launch reads its per-trial state from the control block, so the same
    // graph replays any trial; PSD's iterations run in a conditional while node
    cudaGraphExec_t trial_graph[4];
    bool trial_warm[4], trial_nograph[4];
    bool capturing;            // the stream is being captured: PSD loops on the device
    cudaStream_t bstream;      // captures the body of the PSD while node (made on first use)
    cudaGraphExec_t psd_graph; // one chunk of PSD iterations (eager trials)
    bool psd_warm, psd_nograph;
    int psd_hint;              // iterations the last PSD solve took
    // one fixed step (step size fixed_dt[s]) of IMEX, SAV, ETD captured as a CUDA graph
    cudaGraphExec_t fixed_graph[4];
    double fixed_dt[4];
    // per-pass event timing
    bool timing;
    int nev;
    cudaEvent_t ev[2 * 2048];
    int ev_kind[2048];
    double t_ms[FCH_NPASS];
    long long t_n[FCH_NPASS];
    char errbuf[256];
};

static void timing_flush(fch_ctx *ctx)
{
    if (!ctx->nev) return;
    cudaStreamSynchronize(ctx->stream);
    for (int i = 0; i < ctx->nev; i++) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ctx->ev[2 * i], ctx->ev[2 * i + 1]);
        ctx->t_ms[ctx->ev_kind[i]] += ms;
        ctx->t_n[ctx->ev_kind[i]]++;
    }
    ctx->nev = 0;
}

static void timing_begin(fch_ctx *ctx)
{
    if (!ctx->timing) return;
    if (ctx->nev == 2048) timing_flush(ctx);
    cudaEventRecord(ctx->ev[2 * ctx->nev], ctx->stream);
}

static void timing_end(fch_ctx *ctx, int kind)
{
    if (!ctx->timing) return;
    cudaEventRecord(ctx->ev[2 * ctx->nev + 1], ctx->stream);
    ctx->ev_kind[ctx->nev++] = kind;
}

#define CKC(ctx, call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            snprintf((ctx)->errbuf, sizeof((ctx)->errbuf), "%s: %s", #call,               \
                     cudaGetErrorString(e_));                                             \
            return FCH_ECUDA;                                                             \
        }                                                                                 \
    } while (0)

static thread_local char g_plan_err[256];

extern "C" const char *fch_last_cuda_error(const fch_ctx *ctx) { return ctx ? ctx->errbuf : g_plan_err; }

void fch_set_thread_error(const char *msg) { snprintf(g_plan_err, sizeof(g_plan_err), "%s", msg); }

static bool pow2_in_range(int n) { return n >= FCH_MIN_N && n <= FCH_MAX_N && (n & (n - 1)) == 0; }

static int ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n) l++;
    return l;
}

// Forward twiddles of every Stockham stage with Ns > 1, in the order the passes
// read them: the stage with sub-transform length Ns and radix R holds
// exp(-2 pi i r j / (Ns R)) at Ns - 8 + (r-1) Ns + j, r = 1..R-1, j < Ns.
// Stages: radix 8 while >= 3 bits remain, then one radix-4 or radix-2 stage.
// per-stage twiddles of the shared-memory transforms (fft_smem) whose stages have
// radix 2^lp but the last: lp = 3 (eight points a thread) or 2 (four)
template <typename T> static void make_twiddles(int N, T *out, int lp = 3)
{
    for (int m = 0; m < 2 * N; m++) out[m] = 0;
    int Ns = 1, rem = ilog2(N);
    while (rem > 0) {
        const int lr = rem >= lp ? lp : rem, R = 1 << lr;
        if (Ns > 1)
            for (int r = 1; r < R; r++)
                for (int j = 0; j < Ns; j++) {
                    const int m = Ns - (1 << lp) + (r - 1) * Ns + j;
                    const double a = -2.0 * M_PI * (double)(r * j) / (double)(Ns * R);
                    out[2 * m] = (T)cos(a);
                    out[2 * m + 1] = (T)sin(a);
                }
        Ns <<= lr;
        rem -= lr;
    }
}

// the 32 x 32 twiddles of the warp transform for N = 1024: [k2][n1] = exp(-2 pi i n1 k2 / 1024)
static cudaError_t upload_tw2(void **dst, cudaStream_t s)
{
    float h[2 * 1024];
    for (int k2 = 0; k2 < 32; k2++)
        for (int n1 = 0; n1 < 32; n1++) {
            const double a = -2.0 * M_PI * (double)(n1 * k2) / 1024.0;
            h[2 * (k2 * 32 + n1)] = (float)cos(a);
            h[2 * (k2 * 32 + n1) + 1] = (float)sin(a);
        }
    cudaError_t e = cudaMalloc(dst, sizeof(h));
    if (e == cudaSuccess) e = cudaMemcpyAsync(*dst, h, sizeof(h), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

static fch_status upload_twiddles(fch_ctx *ctx, int N, int prec, void *dst, cudaStream_t s, int lp = 3)
{
    if (prec == FCH_FP32X2) {
        fch::df *h = (fch::df *)malloc(sizeof(fch::df) * 2 * N);
        make_twiddles(N, h, lp);
        cudaError_t e = cudaMemcpyAsync(dst, h, sizeof(fch::df) * 2 * N, cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
        free(h);
        if (e != cudaSuccess) return FCH_ECUDA;
    } else if (prec) {
        float *h = (float *)malloc(sizeof(float) * 2 * N);
        make_twiddles(N, h, lp);
        cudaError_t e = cudaMemcpyAsync(dst, h, sizeof(float) * 2 * N, cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
        free(h);
        if (e != cudaSuccess) return FCH_ECUDA;
    } else {
        double *h = (double *)malloc(sizeof(double) * 2 * N);
        make_twiddles(N, h, lp);
        cudaError_t e = cudaMemcpyAsync(dst, h, sizeof(double) * 2 * N, cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
        free(h);
        if (e != cudaSuccess) return FCH_ECUDA;
    }
    (void)ctx;
    return FCH_OK;
}

// products and sums of polynomials in u (coefficient of u^i at index i)
static void poly_mul(const double *a, int na, const double *b, int nb, double *c)
{
    for (int i = 0; i < na + nb - 1; i++) c[i] = 0.0;
    for (int i = 0; i < na; i++)
        for (int j = 0; j < nb; j++) c[i + j] += a[i] * b[j];
}

// the q = 0 well W(u) = A(u) B(u) and its first two derivatives as polynomials
static void well_polynomials(double bm, double bp, double g3, double c3, double *wp, double *w1p, double *w2p)
{
    const double v[2] = {-bm, 1.0}, w[2] = {-bp, 1.0};
    double v2[3], w2[3];
    poly_mul(v, 2, v, 2, v2);
    poly_mul(w, 2, w, 2, w2);
    const double A[3] = {0.5 * v2[0], 0.5 * v2[1], 0.5 * v2[2]};
    const double B[3] = {0.5 * w2[0] - g3 * c3, 0.5 * w2[1] + g3, 0.5 * w2[2]};
    const double B1[2] = {w[0] + g3, 1.0};
    poly_mul(A, 3, B, 3, wp);
    double vB[4], AB1[4], vB1[3];
    poly_mul(v, 2, B, 3, vB);
    poly_mul(A, 3, B1, 2, AB1);
    for (int i = 0; i < 4; i++) w1p[i] = vB[i] + AB1[i];
    poly_mul(v, 2, B1, 2, vB1);
    for (int i = 0; i < 3; i++) w2p[i] = B[i] + 2.0 * vB1[i] + A[i];
}

template <typename T>
static void fill_consts(fch_consts<T> &k, const fch_params &p, double kf, double am, double inv_n2)
{
    const double e2 = p.eps * p.eps;
    k.kf2 = (T)(kf * kf);
    k.e2 = (T)e2;
    k.e4 = (T)(e2 * e2);
    k.am = (T)am;
    k.am2 = (T)(am * am);
    k.eta1 = (T)p.eta1;
    k.eta2 = (T)p.eta2;
    k.zeta = (T)p.zeta;
    k.b1am_e2 = (T)(p.beta1 * am * e2);
    k.b2am2 = (T)(p.beta2 * am * am);
    k.l1c = (T)(e2 * (p.eta1 + 2.0 * p.zeta));
    k.kappa0 = (T)p.kappa0;
    k.k2e2 = (T)(p.kappa2 * e2);
    k.inv_n2 = (T)inv_n2;
    k.bm = (T)p.b_minus;
    k.bp = (T)p.b_plus;
    k.eps = (T)p.eps;
    k.q = (T)p.q;
    k.qeps = (T)(p.q * p.eps);
    k.qoe = (T)(p.q / p.eps);
    k.g3 = (T)(p.gamma / 3.0);
    k.c3 = (T)(0.5 * (3.0 * p.b_plus - p.b_minus));
    // q = 0: W = A B with A = v^2/2, v = u - b_-, and B = w^2/2 + gamma/3 (u - c3),
    // w = u - b_+ (eq. e:Wq-def), expanded: W' = v B + A B', W'' = B + 2 v B' + A,
    // B' = w + gamma/3
    double wp[5], w1p[4], w2p[3];
    well_polynomials(p.b_minus, p.b_plus, p.gamma / 3.0, 0.5 * (3.0 * p.b_plus - p.b_minus), wp, w1p, w2p);
    for (int i = 0; i < 5; i++) k.wp[i] = (T)wp[i];
    for (int i = 0; i < 4; i++) k.w1p[i] = (T)w1p[i];
    for (int i = 0; i < 3; i++) k.w2p[i] = (T)w2p[i];
}

static void fill_kparams_model(fch_kparams &kp, const fch_params &p, int N, double L)
{
    kp.N = N;
    kp.logN = ilog2(N);
    kp.L = L;
    kp.kf = 2.0 * M_PI / L;
    kp.inv_n2 = 1.0 / ((double)N * N);
    kp.h2 = (L / N) * (L / N);
    kp.eps = p.eps;
    kp.eps2 = p.eps * p.eps;
    kp.q = p.q;
    kp.gamma = p.gamma;
    kp.bm = p.b_minus;
    kp.bp = p.b_plus;
    kp.eta1 = p.eta1;
    kp.eta2 = p.eta2;
    double W, W1, W2;
    host_well(p, p.b_minus, &W, &W1, &W2);
    kp.am = W2; // alpha_m = W_q''(b_-)
    kp.beta1 = p.beta1;
    kp.beta2 = p.beta2;
    kp.zeta = p.zeta;
    kp.D0 = p.D0;
    kp.kappa0 = p.kappa0;
    kp.kappa2 = p.kappa2;
    fill_consts(kp.cf, p, kp.kf, kp.am, kp.inv_n2);
    fill_consts(kp.cd, p, kp.kf, kp.am, kp.inv_n2);
    fill_consts(kp.cdf, p, kp.kf, kp.am, kp.inv_n2);
}

static void reset_ctrl(fch_ctx *ctx)
{
    fch_ctrl &c = ctx->hc;
    memset(&c, 0, sizeof(c));
    c.iu_n = 0;
    c.iu_m = 1;
    c.iu_new = 2;
    c.if_n = 0;
    c.if_m = 1;
    c.if_new = 2;
    c.rho_s = ctx->p.rho_s;
    c.kmin = ctx->p.k_min;
    c.kmax = ctx->p.k_max;
    c.cap = ctx->p.zero_stab_cap;
    c.psd_max_iter = ctx->p.psd_max_iter;
    c.itol = ctx->p.psd_itol;
    if (ctx->p.psd_lambda > 0) {
        c.lam_k[0] = -1.0;
        c.lam_tab[0] = ctx->p.psd_lambda;
    } else {
        const int row = psd_row(ctx->p.q);
        for (int j = 0; j < 10; j++) {
            c.lam_k[j] = kLamK[j];
            c.lam_tab[j] = kLamTab[row][j];
        }
        for (int j = 0; j < 9; j++)
            c.lam_slope[j] = (kLamTab[row][j + 1] - kLamTab[row][j]) / (kLamK[j + 1] - kLamK[j]);
    }
}

static fch_status push_ctrl(fch_ctx *ctx)
{
    CKC(ctx, cudaMemcpyAsync(ctx->dctrl, &ctx->hc, sizeof(fch_ctrl), cudaMemcpyHostToDevice, ctx->stream));
    ctx->hc_fresh = true;
    return FCH_OK;
}

static fch_status pull_ctrl(fch_ctx *ctx)
{
    CKC(ctx, cudaMemcpyAsync(&ctx->hc, ctx->dctrl, sizeof(fch_ctrl), cudaMemcpyDeviceToHost, ctx->stream));
    CKC(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->hc_fresh = true;
    return FCH_OK;
}

// pass launchers
static fch_status col(fch_ctx *ctx, int mode, int src = 0, int flags = 0, const void *in0 = nullptr,
                      const void *in1 = nullptr, void *out0 = nullptr, void *out1 = nullptr,
                      int tail = -1, double tail_arg = 0.0)
{
    fch_kparams kp = ctx->kp;
    kp.tail_op = tail;
    kp.tail_arg = tail_arg;
    kp.src = src;
    kp.flags = flags;
    kp.in0 = in0;
    kp.in1 = in1;
    kp.out0 = out0;
    kp.out1 = out1;
    ctx->hc_fresh = false;
    timing_begin(ctx);
    cudaError_t e = ctx->prec == FCH_MIXED    ? fch_launch_col_f32(mode, kp, ctx->stream)
                    : ctx->prec == FCH_FP32X2 ? fch_launch_col_dfl(mode, kp, ctx->stream)
                                              : fch_launch_col_f64(mode, kp, ctx->stream);
    timing_end(ctx, mode);
    CKC(ctx, e);
    return FCH_OK;
}

static fch_status row(fch_ctx *ctx, int mode, int flags = 0, const void *in0 = nullptr,
                      void *out0 = nullptr, int tail = -1, double tail_arg = 0.0, int src = 0)
{
    fch_kparams kp = ctx->kp;
    kp.src = src;
    kp.tail_op = tail;
    kp.tail_arg = tail_arg;
    kp.flags = flags;
    kp.in0 = in0;
    kp.out0 = out0;
    ctx->hc_fresh = false;
    timing_begin(ctx);
    cudaError_t e = ctx->prec == FCH_MIXED    ? fch_launch_row_f32(mode, kp, ctx->stream)
                    : ctx->prec == FCH_FP32X2 ? fch_launch_row_dfl(mode, kp, ctx->stream)
                                              : fch_launch_row_f64(mode, kp, ctx->stream);
    timing_end(ctx, FCH_NCOL + mode);
    CKC(ctx, e);
    return FCH_OK;
}

static fch_status ctl(fch_ctx *ctx, int op, int na, double arg0 = 0.0, int flags = 0)
{
    fch_kparams kp = ctx->kp;
    kp.flags = flags;
    ctx->hc_fresh = false;
    timing_begin(ctx);
    cudaError_t e = fch_launch_ctrl(op, kp, na, 0, arg0, ctx->stream);
    timing_end(ctx, FCH_NCOL + FCH_NROW);
    CKC(ctx, e);
    return FCH_OK;
}

// a column / row pass whose last block then runs control op `op` on its partial sums
static fch_status colt(fch_ctx *ctx, int mode, int src, int flags, int op, double arg = 0.0)
{
    return col(ctx, mode, src, flags, nullptr, nullptr, nullptr, nullptr, op, arg);
}

static fch_status rowt(fch_ctx *ctx, int mode, int flags, int op, double arg = 0.0)
{
    return row(ctx, mode, flags, nullptr, nullptr, op, arg);
}

#define TRY(x)                                                                            \
    do {                                                                                  \
        fch_status s_ = (x);                                                              \
        if (s_ != FCH_OK) return s_;                                                      \
    } while (0)

extern "C" fch_status fch_create(const fch_grid *g, const fch_params *p, void *stream, fch_ctx **out)
{
    if (!g || !p || !out) return FCH_EINVAL;
    *out = nullptr;
    if (!pow2_in_range(g->n) || !(g->L > 0) || !(p->eps > 0) || p->prec < 0 || p->prec > 2 ||
        p->fft_path < 0 || p->fft_path > 2 || p->autotune < 0 || p->autotune > 2 ||
        !fch_tile_valid(g->n, p->prec == FCH_MIXED, p->tile_row, p->tile_col) ||
        !(p->k_min > 0) || !(p->rho_s > 0) || p->psd_max_iter < 1)
        return FCH_EINVAL;
    fch_ctx *ctx = (fch_ctx *)calloc(1, sizeof(fch_ctx));
    if (!ctx) return FCH_ENOMEM;
    ctx->N = g->n;
    ctx->prec = p->prec;
    ctx->grid = *g;
    ctx->p = *p;
    if (ctx->p.sync_every < 1) ctx->p.sync_every = 16;
    if (ctx->p.zeta <= 0 || ctx->p.D0 <= 0) {
        double z, d;
        sav_constants(ctx->p, g->L * g->L, &z, &d);
        if (ctx->p.zeta <= 0) ctx->p.zeta = z;
        if (ctx->p.D0 <= 0) ctx->p.D0 = d;
    }
    const int N = ctx->N;
    const size_t csz = ctx->prec == FCH_MIXED ? 8 : 16;
    const size_t hs = (size_t)(N / 2 + 1) * N * csz;
    cudaError_t e = cudaSuccess;
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        ctx->own_stream = true;
    }
    int trow = p->tile_row, tcol = p->tile_col;
    // fft_path 2 asks for the warp-level passes where they exist (single precision, 1024^2)
    if (p->fft_path == 2 && p->prec == FCH_MIXED && g->n == 1024 && tcol == 0) tcol = -2;
    if (e == cudaSuccess && p->autotune) {
        fch_tile t;
        const fch_status ts = p->autotune == 2 ? fch_autotune_step(N, ctx->prec, ctx->stream, &t)
                                               : fch_autotune(N, ctx->prec, ctx->stream, &t);
        if (ts != FCH_OK) {
            snprintf(ctx->errbuf, sizeof(ctx->errbuf), "fch_create: autotune: %.200s", g_plan_err);
            fch_destroy(ctx);
            return ts;
        }
        trow = t.tile_row;
        tcol = t.tile_col;
    }
    // At 128^2 and 256^2 in double and double-float the compile-time kernels give a
    // block several rows (column pairs): 8 to 32 blocks for 152 SMs, each pair's chain
    // of dependent work long. There the default (tile 0, asked for or tuned) is the
    // row tile the step tuner (fch_autotune_step, adaptive IMEX trials) picked on GB300
    // and one column pair a block at four points a thread (tile_col -3), and in
    // double-float at 512^2 the same columns; -1 still asks for the compile-time
    // kernels. Against those: 2.0x the trials per second in double, 1.3-1.4x in
    // double-float; 1.09x at 512^2.
    if (ctx->prec != FCH_MIXED) {
        if (trow == 0 && (N == 128 || N == 256)) trow = N == 128 ? 2 : 1;
        if (tcol == 0 && (N == 128 || N == 256 || (N == 512 && ctx->prec == FCH_FP32X2))) tcol = -3;
    }
    ctx->geom = fch_geometry_tiled(N, ctx->prec == FCH_MIXED, trow, tcol);
    void **bufs[] = {&ctx->U[0], &ctx->U[1], &ctx->U[2], &ctx->F[0], &ctx->F[1], &ctx->F[2],
                     &ctx->Pb, &ctx->Qb, &ctx->Vb, &ctx->Nb};
    for (void **b : bufs)
        if (e == cudaSuccess) e = cudaMalloc(b, hs);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->Z, (size_t)N * N * csz);
    for (int i = 0; i < 3 && e == cudaSuccess; i++) e = cudaMalloc(&ctx->Rs[i], (size_t)N * N * csz);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->tw, (size_t)N * csz);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->tw4, (size_t)N * csz);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->part, sizeof(double) * FCH_NRED * FCH_MAXBLK);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->dctrl, sizeof(fch_ctrl));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->staging, sizeof(double) * N * N * 2);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->nfft_dev, sizeof(long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->nfft_dev, 0, sizeof(long long), ctx->stream);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->ticket, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ticket, 0, 2 * sizeof(unsigned int), ctx->stream);
    // every state array starts at zero: a backward-Euler start multiplies u^{n-1} by
    // c = 0, which must not meet whatever the memory held before (0 x NaN = NaN)
    for (void **b : bufs)
        if (e == cudaSuccess) e = cudaMemsetAsync(*b, 0, hs, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->Z, 0, (size_t)N * N * csz, ctx->stream);
    for (int i = 0; i < 3 && e == cudaSuccess; i++) e = cudaMemsetAsync(ctx->Rs[i], 0, (size_t)N * N * csz, ctx->stream);
    if (e != cudaSuccess) {
        snprintf(ctx->errbuf, sizeof(ctx->errbuf), "fch_create: %s", cudaGetErrorString(e));
        fch_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? FCH_ENOMEM : FCH_ECUDA;
    }
    fill_kparams_model(ctx->kp, ctx->p, N, g->L);
    ctx->kp.P = ctx->geom.P;
    ctx->kp.tile_row = trow;
    ctx->kp.tile_col = tcol;
    // Programmatic dependent launch pays where every pass is one full wave: the default
    // tiles at 1024^2 in double and double-float (1024 blocks of 128 threads, seven a
    // SM), where a successor's blocks can only take the slots the tail frees. Where a
    // pass leaves SMs free (smaller grids) the successor's waiting blocks take them
    // early and the running pass ends up packed onto fewer SMs (512^2: 2.3x slower
    // trials in double); where it has several waves (2048^2) they take later waves'
    // slots.
    ctx->kp.pdl = N == 1024 && ctx->prec != FCH_MIXED && trow == 0 && tcol == 0;
    for (int i = 0; i < 3; i++) {
        ctx->kp.U[i] = ctx->U[i];
        ctx->kp.F[i] = ctx->F[i];
    }
    ctx->kp.Pb = ctx->Pb;
    ctx->kp.Qb = ctx->Qb;
    ctx->kp.Vb = ctx->Vb;
    ctx->kp.Nb = ctx->Nb;
    ctx->kp.Z = ctx->Z;
    for (int i = 0; i < 3; i++) ctx->kp.Rs[i] = ctx->Rs[i];
    ctx->kp.tw = ctx->tw;
    ctx->kp.tw4 = ctx->tw4;
    ctx->kp.part = ctx->part;
    ctx->kp.ctrl = ctx->dctrl;
    ctx->kp.nfft = (unsigned long long *)ctx->nfft_dev;
    ctx->kp.ticket = ctx->ticket;
    ctx->kp.tail_op = -1;
    fch_status s = upload_twiddles(ctx, N, ctx->prec, ctx->tw, ctx->stream);
    if (s == FCH_OK) s = upload_twiddles(ctx, N, ctx->prec, ctx->tw4, ctx->stream, 2);
    if (s == FCH_OK && ctx->prec == FCH_MIXED && N == 1024 && ctx->p.fft_path != 1) {
        if (upload_tw2(&ctx->tw2, ctx->stream) != cudaSuccess) s = FCH_ECUDA;
        ctx->kp.tw2 = ctx->tw2;
    }
    if (s != FCH_OK) {
        fch_destroy(ctx);
        return s;
    }
    reset_ctrl(ctx);
    s = push_ctrl(ctx);
    if (s != FCH_OK) {
        fch_destroy(ctx);
        return s;
    }
    *out = ctx;
    return FCH_OK;
}

extern "C" fch_status fch_destroy(fch_ctx *ctx)
{
    if (!ctx) return FCH_OK;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    void *bufs[] = {ctx->U[0], ctx->U[1], ctx->U[2], ctx->F[0], ctx->F[1], ctx->F[2], ctx->Pb,
                    ctx->Qb, ctx->Vb, ctx->Nb, ctx->Z, ctx->tw, ctx->tw4, ctx->part, ctx->dctrl,
                    ctx->staging, ctx->nfft_dev, ctx->ticket, ctx->tw2, ctx->Rs[0],
                    ctx->Rs[1], ctx->Rs[2], ctx->ls_a, ctx->ls_y, ctx->ls_part};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (int i = 0; i < 2; i++)
        if (ctx->ls_ev[i]) cudaEventDestroy(ctx->ls_ev[i]);
    if (ctx->timing)
        for (int i = 0; i < 2 * 2048; i++) cudaEventDestroy(ctx->ev[i]);
    for (int i = 0; i < 4; i++) {
        if (ctx->trial_graph[i]) cudaGraphExecDestroy(ctx->trial_graph[i]);
        if (ctx->fixed_graph[i]) cudaGraphExecDestroy(ctx->fixed_graph[i]);
    }
    if (ctx->psd_graph) cudaGraphExecDestroy(ctx->psd_graph);
    if (ctx->bstream) cudaStreamDestroy(ctx->bstream);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    free(ctx);
    return FCH_OK;
}

extern "C" fch_status fch_synchronize(fch_ctx *ctx)
{
    if (!ctx) return FCH_EINVAL;
    TRY(pull_ctrl(ctx));
    if (ctx->hc.status) {
        ctx->failed = true;
        return (fch_status)ctx->hc.status;
    }
    return FCH_OK;
}

// real field (device; f64 when io64) -> U[slot]
static fch_status load_field(fch_ctx *ctx, const void *u_dev, bool io64, void *dst)
{
    TRY(row(ctx, RM_R2C_LOAD, FCH_FL_NOSKIP | (io64 ? FCH_FL_F64IO : 0), u_dev));
    TRY(col(ctx, CM_FWD_STORE, 0, FCH_FL_NOSKIP, nullptr, nullptr, dst, nullptr));
    return FCH_OK;
}

// SAV r from E1 of the state in slot src (4 = u^n via USTAR with gam 0? use explicit srcs)
static fch_status sav_r_init(fch_ctx *ctx, int src, double which)
{
    TRY(col(ctx, CM_START, src, FCH_FL_NOSKIP));
    TRY(rowt(ctx, RM_SAV, FCH_FL_NOSKIP, OP_SAV_E1, which));
    return FCH_OK;
}

static fch_status set_state_common(fch_ctx *ctx, const void *u_dev, bool io64)
{
    reset_ctrl(ctx);
    TRY(push_ctrl(ctx));
    // u^{n-1} (slot 1) enters the start step with the coefficient c = 0: keep it finite
    CKC(ctx, cudaMemsetAsync(ctx->U[1], 0, (size_t)(ctx->N / 2 + 1) * ctx->N * (ctx->prec == FCH_MIXED ? 8 : 16),
                             ctx->stream));
    TRY(load_field(ctx, u_dev, io64, ctx->U[0]));
    TRY(sav_r_init(ctx, FCH_SRC_UN, 1.0));
    ctx->have_state = true;
    ctx->failed = false;
    ctx->have_F = false;
    ctx->rvalid = false;
    return FCH_OK;
}

extern "C" fch_status fch_set_state(fch_ctx *ctx, const double *u_host, size_t n)
{
    if (!ctx || !u_host || n != (size_t)ctx->N * ctx->N) return FCH_EINVAL;
    CKC(ctx, cudaMemcpyAsync(ctx->staging, u_host, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    TRY(set_state_common(ctx, ctx->staging, true));
    return fch_synchronize(ctx);
}

extern "C" fch_status fch_set_state_device(fch_ctx *ctx, const void *u_dev, int dtype)
{
    if (!ctx || !u_dev || (dtype != 0 && dtype != 1)) return FCH_EINVAL;
    return set_state_common(ctx, u_dev, dtype == 0);
}

extern "C" fch_status fch_set_history(fch_ctx *ctx, const double *un, const double *unm1, size_t n,
                                      double kn)
{
    if (!ctx || !un || !unm1 || n != (size_t)ctx->N * ctx->N || !(kn > 0)) return FCH_EINVAL;
    reset_ctrl(ctx);
    ctx->hc.kn = kn;
    ctx->hc.ktrial = kn;
    TRY(push_ctrl(ctx));
    CKC(ctx, cudaMemcpyAsync(ctx->staging, un, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    CKC(ctx, cudaMemcpyAsync(ctx->staging + n, unm1, sizeof(double) * n, cudaMemcpyHostToDevice,
                             ctx->stream));
    TRY(load_field(ctx, ctx->staging, true, ctx->U[0]));
    TRY(load_field(ctx, ctx->staging + n, true, ctx->U[1]));
    TRY(sav_r_init(ctx, FCH_SRC_UN, 1.0));
    TRY(sav_r_init(ctx, 5, 2.0));
    ctx->have_state = true;
    ctx->failed = false;
    ctx->have_F = false;
    ctx->rvalid = false;
    return fch_synchronize(ctx);
}

// u^n -> real field (device; f64 when io64)
static fch_status store_state(fch_ctx *ctx, void *u_dev, bool io64)
{
    TRY(col(ctx, CM_START, FCH_SRC_UN, FCH_FL_NOSKIP));
    TRY(row(ctx, RM_C2R_STORE, FCH_FL_NOSKIP | (io64 ? FCH_FL_F64IO : 0), nullptr, u_dev));
    return FCH_OK;
}

extern "C" fch_status fch_get_state(fch_ctx *ctx, double *u_host, size_t n)
{
    if (!ctx || !u_host || n != (size_t)ctx->N * ctx->N) return FCH_EINVAL;
    if (!ctx->have_state) return FCH_ESTATE;
    TRY(store_state(ctx, ctx->staging, true));
    CKC(ctx, cudaMemcpyAsync(u_host, ctx->staging, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    return fch_synchronize(ctx);
}

extern "C" fch_status fch_get_state_device(fch_ctx *ctx, void *u_dev, int dtype)
{
    if (!ctx || !u_dev || (dtype != 0 && dtype != 1)) return FCH_EINVAL;
    if (!ctx->have_state) return FCH_ESTATE;
    return store_state(ctx, u_dev, dtype == 0);
}

// one trial step from the current history into the trial slot (parameters already
// in the control block). pack_f: leave (u_new, Lap u_new) packed for F(u_new).
// PSD iterations, eqs. (residual), (recurrence), from the iterate in Vb (packed in Z
// by the pass before) until the stopping test holds; the trial slot then receives
// the converged iterate
static const int kPsdChunk = 4;

static fch_status psd_chunk_eager(fch_ctx *ctx)
{
    for (int i = 0; i < kPsdChunk; i++) {
        TRY(row(ctx, RM_F, FCH_FL_PSDSKIP));
        TRY(colt(ctx, CM_PSD_ITER, 0, FCH_FL_PSDSKIP, OP_PSD_CHECK));
    }
    return FCH_OK;
}

// kPsdChunk iterations: the first chunk of a context runs eagerly (it also sets the
// kernels' attributes), later ones replay a captured graph unless per-pass timing is
// on. Once the stopping test holds, the remaining passes of a chunk return at once.
static fch_status psd_chunk(fch_ctx *ctx)
{
    const bool graph_ok = !ctx->timing && ctx->psd_warm && !ctx->psd_nograph;
    if (graph_ok && !ctx->psd_graph) {
        bool ok = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
        if (ok) {
            const fch_status st = psd_chunk_eager(ctx);
            cudaGraph_t g = nullptr;
            ok = cudaStreamEndCapture(ctx->stream, &g) == cudaSuccess && g && st == FCH_OK;
            if (ok) ok = cudaGraphInstantiate(&ctx->psd_graph, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
        }
        if (!ok) {
            ctx->psd_graph = nullptr;
            ctx->psd_nograph = true;
            cudaGetLastError();
        }
    }
    if (graph_ok && ctx->psd_graph) {
        ctx->hc_fresh = false;
        CKC(ctx, cudaGraphLaunch(ctx->psd_graph, ctx->stream));
        return FCH_OK;
    }
    TRY(psd_chunk_eager(ctx));
    ctx->psd_warm = true;
    return FCH_OK;
}

// The host reads the control block after each batch of chunks; the first batch
// covers as many iterations as the previous solve took (rounded down to chunks),
// later ones one chunk each.
static fch_status psd_iterate(fch_ctx *ctx)
{
    int chunks = ctx->psd_hint >= kPsdChunk ? ctx->psd_hint / kPsdChunk : 1;
    for (long long launched = 0;; chunks = 1) {
        if (launched > ctx->p.psd_max_iter + 2 * kPsdChunk) return FCH_ENOCONV;
        for (int c = 0; c < chunks; c++) TRY(psd_chunk(ctx));
        launched += (long long)chunks * kPsdChunk;
        TRY(pull_ctrl(ctx));
        if (ctx->hc.status || ctx->hc.done || ctx->hc.psd_conv) break;
    }
    if (ctx->hc.status) return (fch_status)ctx->hc.status;
    ctx->psd_hint = ctx->hc.last_psd_iter;
    TRY(col(ctx, CM_START, FCH_SRC_V, FCH_FL_COPYV));
    return FCH_OK;
}

// The condition of the captured PSD loop (one thread): arm (before the while node)
// zeroes the chunk count, the body's last launch counts its chunk. The loop goes on
// while the stopping test has not held, the run has not stopped (done or a failure:
// OP_PSD_CHECK stops it at psd_max_iter iterations) and fewer than `limit` chunks ran,
// so it ends after at most `limit` chunks whatever the control block holds.
__global__ void fch_psd_loop_kernel(cudaGraphConditionalHandle h, const fch_ctrl *c, unsigned int *count, int arm,
                                    unsigned int limit)
{
    const unsigned int n = arm ? 0u : *count + 1u;
    *count = n;
    const bool more = !c->done && !c->status && !c->psd_conv && n < limit;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// PSD iterations inside a stream capture: a while node whose body is one chunk of
// iterations and the condition launch, then the copy of the converged iterate. The
// launches next to the node go without programmatic serialization (a programmatic
// edge joins two kernel nodes only), and so do the body's.
static fch_status psd_loop_captured(fch_ctx *ctx)
{
    if (!ctx->bstream) CKC(ctx, cudaStreamCreateWithFlags(&ctx->bstream, cudaStreamNonBlocking));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edata = nullptr;
    size_t nd = 0;
    CKC(ctx, cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &g, &deps, &edata, &nd));
    if (cs != cudaStreamCaptureStatusActive || !g) return FCH_ESTATE;
    cudaGraphConditionalHandle h;
    CKC(ctx, cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    const unsigned int limit = (unsigned int)(ctx->p.psd_max_iter / kPsdChunk + 3);
    unsigned int *count = ctx->ticket + 1;
    fch_psd_loop_kernel<<<1, 1, 0, ctx->stream>>>(h, ctx->dctrl, count, 1, limit);
    CKC(ctx, cudaGetLastError());
    CKC(ctx, cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &g, &deps, &edata, &nd));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CKC(ctx, cudaGraphAddNode(&node, g, deps, edata, nd, &np));
    const cudaGraph_t body = np.conditional.phGraph_out[0];
    CKC(ctx, cudaStreamBeginCaptureToGraph(ctx->bstream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    const cudaStream_t outer = ctx->stream;
    const int pdl = ctx->kp.pdl;
    ctx->stream = ctx->bstream;
    ctx->kp.pdl = 0;
    fch_status s = psd_chunk_eager(ctx);
    if (s == FCH_OK) {
        fch_psd_loop_kernel<<<1, 1, 0, ctx->stream>>>(h, ctx->dctrl, count, 0, limit);
        if (cudaGetLastError() != cudaSuccess) s = FCH_ECUDA;
    }
    ctx->stream = outer;
    cudaGraph_t bg = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->bstream, &bg);
    if (s == FCH_OK && e != cudaSuccess) s = FCH_ECUDA;
    if (s == FCH_OK && cudaStreamUpdateCaptureDependencies(ctx->stream, &node, nullptr, 1,
                                                           cudaStreamSetCaptureDependencies) != cudaSuccess)
        s = FCH_ECUDA;
    if (s == FCH_OK) s = col(ctx, CM_START, FCH_SRC_V, FCH_FL_COPYV);
    ctx->kp.pdl = pdl;
    return s;
}

static fch_status enqueue_trial(fch_ctx *ctx, fch_scheme scheme, bool pack_f)
{
    const int pf = pack_f ? FCH_FL_PACK_F : 0;
    // with (u, Lap u) of u^n and u^{n-1} kept in real space (adaptive runs), the
    // extrapolation u* and its Laplacian are formed pointwise by the first row pass
    // instead of by an inverse column pass and inverse row transforms
    const bool direct = ctx->rvalid;
    switch (scheme) {
    case FCH_IMEX:
        if (direct) {
            TRY(row(ctx, RM_NIMEX_DIRECT));
        } else {
            TRY(col(ctx, CM_START, 4));
            TRY(row(ctx, RM_NIMEX));
        }
        TRY(col(ctx, CM_IMEX_SOLVE, 0, pf));
        return FCH_OK;
    case FCH_SAV:
        if (direct) {
            TRY(rowt(ctx, RM_SAV_DIRECT, 0, OP_SAV_E1, 0.0));
        } else {
            TRY(col(ctx, CM_START, 4));
            TRY(rowt(ctx, RM_SAV, 0, OP_SAV_E1, 0.0));
        }
        TRY(colt(ctx, CM_SAV_PQ, 0, 0, OP_SAV_R));
        TRY(col(ctx, CM_SAV_COMBINE, 0, pf));
        return FCH_OK;
    case FCH_ETD:
        if (direct) {
            TRY(row(ctx, RM_NIMEX_DIRECT, FCH_FL_GAMMA0));
        } else {
            TRY(col(ctx, CM_START, FCH_SRC_UN));
            TRY(row(ctx, RM_NIMEX));
        }
        TRY(col(ctx, CM_ETD_STAGE1));
        TRY(row(ctx, RM_NIMEX));
        TRY(col(ctx, CM_ETD_STAGE2, 0, pf));
        return FCH_OK;
    case FCH_PSD:
        TRY(col(ctx, CM_START, 4, 128));
        return ctx->capturing ? psd_loop_captured(ctx) : psd_iterate(ctx);
    }
    return FCH_EINVAL;
}

extern "C" fch_status fch_step(fch_ctx *ctx, fch_scheme scheme, double dt)
{
    if (!ctx || !(dt > 0) || scheme < FCH_IMEX || scheme > FCH_ETD) return FCH_EINVAL;
    if (!ctx->have_state || ctx->failed) return FCH_ESTATE;
    ctx->rvalid = false; // fixed steps do not keep the real-space fields
    TRY(ctl(ctx, OP_INIT_TRIAL, 0, dt));
    fch_status s = enqueue_trial(ctx, scheme, false);
    if (s != FCH_OK) {
        ctx->failed = true;
        return s;
    }
    TRY(ctl(ctx, OP_ACCEPT, 0, 0.0));
    ctx->have_F = false;
    return FCH_OK;
}

// F of the state in slot src into its F slot (src: FCH_SRC_UN -> F(u^n), 5 -> F(u^{n-1}))
// one fixed step without host checks, its control set-up already done: the scheme's
// step, then one control launch that accepts it and sets up the next step of size dt
// (the set-up after the last step is left unused)
static fch_status enqueue_fixed_step(fch_ctx *ctx, fch_scheme scheme, double dt)
{
    TRY(enqueue_trial(ctx, scheme, false));
    TRY(ctl(ctx, OP_ACCEPT_INIT, 0, dt));
    return FCH_OK;
}

extern "C" fch_status fch_run_fixed(fch_ctx *ctx, fch_scheme scheme, double dt, long long nsteps)
{
    if (!ctx || !(dt > 0) || nsteps < 0 || scheme < FCH_IMEX || scheme > FCH_ETD) return FCH_EINVAL;
    if (!ctx->have_state || ctx->failed) return FCH_ESTATE;
    if (nsteps == 0) return FCH_OK;
    // with per-pass timing every launch is timed
    if (ctx->timing) {
        for (long long i = 0; i < nsteps; i++) TRY(fch_step(ctx, scheme, dt));
        return FCH_OK;
    }
    ctx->rvalid = false;
    ctx->have_F = false;
    // the first step runs eagerly (it also sets the kernels' attributes)
    TRY(ctl(ctx, OP_INIT_TRIAL, 0, dt));
    fch_status s = enqueue_fixed_step(ctx, scheme, dt);
    if (s != FCH_OK) {
        ctx->failed = true;
        return s;
    }
    if (nsteps == 1) return FCH_OK;
    if (ctx->fixed_graph[scheme] && ctx->fixed_dt[scheme] != dt) {
        cudaGraphExecDestroy(ctx->fixed_graph[scheme]);
        ctx->fixed_graph[scheme] = nullptr;
    }
    if (!ctx->fixed_graph[scheme]) {
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
        if (ok) {
            ctx->capturing = true;
            s = enqueue_fixed_step(ctx, scheme, dt);
            ctx->capturing = false;
            ok = cudaStreamEndCapture(ctx->stream, &g) == cudaSuccess && g && s == FCH_OK;
        }
        if (ok) ok = cudaGraphInstantiate(&ctx->fixed_graph[scheme], g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (!ok) {
            // no graph: the remaining steps launch one kernel at a time
            cudaGetLastError();
            ctx->fixed_graph[scheme] = nullptr;
            for (long long i = 1; i < nsteps; i++) TRY(enqueue_fixed_step(ctx, scheme, dt));
            return FCH_OK;
        }
        ctx->fixed_dt[scheme] = dt;
    }
    if (nsteps > 1) ctx->hc_fresh = false;
    for (long long i = 1; i < nsteps; i++) CKC(ctx, cudaGraphLaunch(ctx->fixed_graph[scheme], ctx->stream));
    return FCH_OK;
}

extern "C" fch_status fch_get_history_device(fch_ctx *ctx, void *un_dev, void *unm1_dev, int dtype)
{
    if (!ctx || !un_dev || !unm1_dev || (dtype != 0 && dtype != 1)) return FCH_EINVAL;
    if (!ctx->have_state) return FCH_ESTATE;
    TRY(col(ctx, CM_START, FCH_SRC_UN, FCH_FL_NOSKIP));
    TRY(row(ctx, RM_C2R_STORE, FCH_FL_NOSKIP | (dtype == 0 ? FCH_FL_F64IO : 0), nullptr, un_dev));
    TRY(col(ctx, CM_START, 5, FCH_FL_NOSKIP)); // u^{n-1}
    TRY(row(ctx, RM_C2R_STORE, FCH_FL_NOSKIP | (dtype == 0 ? FCH_FL_F64IO : 0), nullptr, unm1_dev));
    return FCH_OK;
}

extern "C" fch_status fch_adaptive_trial_info(fch_ctx *ctx, double *k_trial, double *gamma, int *done)
{
    if (!ctx || !k_trial || !gamma || !done) return FCH_EINVAL;
    if (!ctx->ad_open) return FCH_ESTATE;
    TRY(pull_ctrl(ctx));
    *done = ctx->hc.done || ctx->hc.status;
    *k_trial = ctx->hc.k1;
    *gamma = ctx->hc.kn > 0 ? ctx->hc.gam : 0.0;
    return ctx->hc.status ? (fch_status)ctx->hc.status : FCH_OK;
}

extern "C" fch_status fch_adaptive_enqueue_psd_from(fch_ctx *ctx, const void *v0, int dtype)
{
    if (!ctx || !v0 || (dtype != 0 && dtype != 1)) return FCH_EINVAL;
    if (!ctx->ad_open || ctx->failed || ctx->ad_scheme != FCH_PSD) return FCH_ESTATE;
    TRY(load_field(ctx, v0, dtype == 0, ctx->Vb));
    TRY(col(ctx, CM_START, FCH_SRC_V));
    fch_status s = psd_iterate(ctx);
    if (s == FCH_OK) s = row(ctx, RM_F, FCH_FL_STORE_REAL, nullptr, nullptr, -1, 0.0, FCH_SRC_UNEW);
    if (s == FCH_OK) s = col(ctx, CM_F_FINISH, FCH_SRC_UNEW, FCH_FL_AM3);
    if (s == FCH_OK) s = ctl(ctx, OP_DECIDE_INIT, ctx->geom.col_blocks);
    if (s != FCH_OK) ctx->failed = true;
    return s;
}

// one adaptive IMEX or SAV trial (as fch_adaptive_enqueue) whose explicit part is
// evaluated at the caller's u* instead of eq. (Richardson)
extern "C" fch_status fch_adaptive_enqueue_from(fch_ctx *ctx, const void *ustar, int dtype)
{
    if (!ctx || !ustar || (dtype != 0 && dtype != 1)) return FCH_EINVAL;
    if (!ctx->ad_open || ctx->failed || (ctx->ad_scheme != FCH_IMEX && ctx->ad_scheme != FCH_SAV))
        return FCH_ESTATE;
    // the given u*: its spectrum in Vb, (u*, Lap u*) packed for the row pass
    TRY(load_field(ctx, ustar, dtype == 0, ctx->Vb));
    TRY(col(ctx, CM_START, FCH_SRC_V));
    fch_status s;
    if (ctx->ad_scheme == FCH_IMEX) {
        s = row(ctx, RM_NIMEX);
        if (s == FCH_OK) s = col(ctx, CM_IMEX_SOLVE, 0, FCH_FL_PACK_F);
    } else {
        s = rowt(ctx, RM_SAV, 0, OP_SAV_E1, 0.0);
        if (s == FCH_OK) s = colt(ctx, CM_SAV_PQ, 0, FCH_FL_USTAR_V, OP_SAV_R);
        if (s == FCH_OK) s = col(ctx, CM_SAV_COMBINE, 0, FCH_FL_PACK_F);
    }
    if (s == FCH_OK) s = row(ctx, RM_F, FCH_FL_STORE_REAL, nullptr, nullptr, -1, 0.0, FCH_SRC_UNEW);
    if (s == FCH_OK) s = col(ctx, CM_F_FINISH, FCH_SRC_UNEW, FCH_FL_AM3);
    if (s == FCH_OK) s = ctl(ctx, OP_DECIDE_INIT, ctx->geom.col_blocks);
    if (s != FCH_OK) ctx->failed = true;
    return s;
}

extern "C" fch_status fch_step_from(fch_ctx *ctx, fch_scheme scheme, double dt, const void *ustar, int dtype)
{
    if (!ctx || !(dt > 0) || !ustar || (dtype != 0 && dtype != 1) || (scheme != FCH_IMEX && scheme != FCH_SAV))
        return FCH_EINVAL;
    if (!ctx->have_state || ctx->failed) return FCH_ESTATE;
    ctx->rvalid = false;
    TRY(ctl(ctx, OP_INIT_TRIAL, 0, dt));
    // the given u*: its spectrum in Vb, (u*, Lap u*) packed for the row pass
    TRY(load_field(ctx, ustar, dtype == 0, ctx->Vb));
    TRY(col(ctx, CM_START, FCH_SRC_V));
    fch_status s;
    if (scheme == FCH_IMEX) {
        s = row(ctx, RM_NIMEX);
        if (s == FCH_OK) s = col(ctx, CM_IMEX_SOLVE, 0, 0);
    } else {
        s = rowt(ctx, RM_SAV, 0, OP_SAV_E1, 0.0);
        if (s == FCH_OK) s = colt(ctx, CM_SAV_PQ, 0, FCH_FL_USTAR_V, OP_SAV_R);
        if (s == FCH_OK) s = col(ctx, CM_SAV_COMBINE, 0, 0);
    }
    if (s != FCH_OK) {
        ctx->failed = true;
        return s;
    }
    TRY(ctl(ctx, OP_ACCEPT, 0, 0.0));
    ctx->have_F = false;
    return FCH_OK;
}

extern "C" fch_status fch_step_psd_from(fch_ctx *ctx, double dt, const void *v0, int dtype)
{
    if (!ctx || !(dt > 0) || !v0 || (dtype != 0 && dtype != 1)) return FCH_EINVAL;
    if (!ctx->have_state || ctx->failed) return FCH_ESTATE;
    ctx->rvalid = false;
    TRY(ctl(ctx, OP_INIT_TRIAL, 0, dt));
    // v_0: the given field's spectrum is the first iterate; packed into Z for the
    // first F pass of the iteration
    TRY(load_field(ctx, v0, dtype == 0, ctx->Vb));
    TRY(col(ctx, CM_START, FCH_SRC_V));
    fch_status s = psd_iterate(ctx);
    if (s != FCH_OK) {
        ctx->failed = true;
        return s;
    }
    TRY(ctl(ctx, OP_ACCEPT, 0, 0.0));
    ctx->have_F = false;
    return FCH_OK;
}

// ---------------------------------------------------------------------------
// Learned first iterate of the PSD iteration (Sec. 3.3: eqs. (residual),
// (recurrence) start from any v_0). From the context's history u^n, u^{n-1} and the
// step ratio gam of the next step (the open adaptive run's next trial from the
// control block, or dt / k_n for a fixed step of size dt):
//   u* = u^n + gam (u^n - u^{n-1})                   (eq. Richardson)
//   s  = RMS(u* - u^n) = gam RMS(u^n - u^{n-1})
//   a  = (u^n, (u* - u^n) / s)                        (network input, float)
//   y  = network(a)                                   (predicts (u^{n+1} - u*) / s)
//   v_0 = u* + s (y - mean y)                         (mass of u*)
// All of it on the device: FP64 sums over per-block partials in a fixed order
// (every block re-adds the partials itself, so no single-block pass is needed), the
// network's forward pass ordered between the kernels by events. With gam = 0 (no
// history) or u^n = u^{n-1}, s = 0 and v_0 = u*.
static const int kLsBlocks = 256, kLsThreads = 256;

__device__ inline double ls_block_sum(double v)
{
    __shared__ double sh[kLsThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kLsThreads / 32; w++) t += sh[w];
    __syncthreads();
    return t; // valid in thread 0
}

// the total of the nb partials, in index order, by one warp (valid in every lane)
__device__ inline double ls_total(const double *part, int nb)
{
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    for (int i = lane; i < nb; i += 32) v += part[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ inline double ls_gam(const fch_ctrl *c, double dt)
{
    if (dt > 0) return c->kn > 0 ? dt / c->kn : 0.0;
    return c->kn > 0 ? c->gam : 0.0;
}

// part[b] = sum over the block's points of (u^n - u^{n-1})^2
__global__ void __launch_bounds__(kLsThreads) ls_diff_sums(const double *__restrict__ un,
                                                           const double *__restrict__ um, long cnt,
                                                           double *__restrict__ part)
{
    double v = 0.0;
    for (long i = blockIdx.x * (long)kLsThreads + threadIdx.x; i < cnt; i += (long)gridDim.x * kLsThreads) {
        const double d = un[i] - um[i];
        v += d * d;
    }
    const double t = ls_block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// a[0] = u^n, a[1] = (u* - u^n) / s as floats
__global__ void __launch_bounds__(kLsThreads) ls_inputs(const double *__restrict__ un, const double *__restrict__ um,
                                                        long cnt, const fch_ctrl *__restrict__ c, double dt,
                                                        const double *__restrict__ part, int nb,
                                                        float *__restrict__ a)
{
    const double g = ls_gam(c, dt);
    const double r = sqrt(ls_total(part, nb) / (double)cnt); // RMS(u^n - u^{n-1})
    const double s = g * r;
    const double inv = s > 0 ? 1.0 / s : 0.0;
    for (long i = blockIdx.x * (long)kLsThreads + threadIdx.x; i < cnt; i += (long)gridDim.x * kLsThreads) {
        const double d = g * (un[i] - um[i]);
        a[i] = (float)un[i];
        a[cnt + i] = (float)(d * inv);
    }
}

// part[b] = sum over the block's points of y
__global__ void __launch_bounds__(kLsThreads) ls_y_sums(const float *__restrict__ y, long cnt,
                                                        double *__restrict__ part)
{
    double v = 0.0;
    for (long i = blockIdx.x * (long)kLsThreads + threadIdx.x; i < cnt; i += (long)gridDim.x * kLsThreads)
        v += (double)y[i];
    const double t = ls_block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// v_0 = u* + s (y - mean y)
__global__ void __launch_bounds__(kLsThreads) ls_v0(const double *__restrict__ un, const double *__restrict__ um,
                                                    const float *__restrict__ y, long cnt,
                                                    const fch_ctrl *__restrict__ c, double dt,
                                                    const double *__restrict__ part_d,
                                                    const double *__restrict__ part_y, int nb,
                                                    double *__restrict__ v0)
{
    const double g = ls_gam(c, dt);
    const double s = g * sqrt(ls_total(part_d, nb) / (double)cnt);
    const double ym = ls_total(part_y, nb) / (double)cnt;
    for (long i = blockIdx.x * (long)kLsThreads + threadIdx.x; i < cnt; i += (long)gridDim.x * kLsThreads) {
        const double ustar = un[i] + g * (un[i] - um[i]);
        v0[i] = s > 0 ? ustar + s * ((double)y[i] - ym) : ustar;
    }
}

extern "C" fch_status fch_fno_learned_start(fch_ctx *ctx, fch_fno *net, double dt, void *v0_dev)
{
    if (!ctx || !net || !v0_dev || !(dt >= 0)) return FCH_EINVAL;
    if (!ctx->have_state || ctx->failed) return FCH_ESTATE;
    if (dt == 0 && !ctx->ad_open) return FCH_ESTATE;
    const long cnt = (long)ctx->N * ctx->N;
    if (!ctx->ls_a) {
        CKC(ctx, cudaMalloc((void **)&ctx->ls_a, sizeof(float) * 2 * cnt));
        CKC(ctx, cudaMalloc((void **)&ctx->ls_y, sizeof(float) * cnt));
        CKC(ctx, cudaMalloc((void **)&ctx->ls_part, sizeof(double) * 2 * kLsBlocks));
        for (int i = 0; i < 2; i++) CKC(ctx, cudaEventCreateWithFlags(&ctx->ls_ev[i], cudaEventDisableTiming));
    }
    // u^n, u^{n-1} as real fields in the staging buffer (2 N^2 doubles)
    double *un = ctx->staging, *um = ctx->staging + cnt;
    TRY(col(ctx, CM_START, FCH_SRC_UN, FCH_FL_NOSKIP));
    TRY(row(ctx, RM_C2R_STORE, FCH_FL_NOSKIP | FCH_FL_F64IO, nullptr, un));
    TRY(col(ctx, CM_START, 5, FCH_FL_NOSKIP));
    TRY(row(ctx, RM_C2R_STORE, FCH_FL_NOSKIP | FCH_FL_F64IO, nullptr, um));
    cudaStream_t s = ctx->stream, fs = fch_fno_stream_of(net);
    double *pd = ctx->ls_part, *py = ctx->ls_part + kLsBlocks;
    ls_diff_sums<<<kLsBlocks, kLsThreads, 0, s>>>(un, um, cnt, pd);
    ls_inputs<<<kLsBlocks, kLsThreads, 0, s>>>(un, um, cnt, ctx->dctrl, dt, pd, kLsBlocks, ctx->ls_a);
    CKC(ctx, cudaGetLastError());
    // the network's forward pass on its own stream, between the kernels above and below
    CKC(ctx, cudaEventRecord(ctx->ls_ev[0], s));
    CKC(ctx, cudaStreamWaitEvent(fs, ctx->ls_ev[0], 0));
    const fch_status fst = fch_fno_forward(net, 1, ctx->N, ctx->ls_a, ctx->ls_y);
    if (fst != FCH_OK) {
        snprintf(ctx->errbuf, sizeof(ctx->errbuf), "fch_fno_learned_start: %s", fch_last_cuda_error(nullptr));
        return fst;
    }
    CKC(ctx, cudaEventRecord(ctx->ls_ev[1], fs));
    CKC(ctx, cudaStreamWaitEvent(s, ctx->ls_ev[1], 0));
    ls_y_sums<<<kLsBlocks, kLsThreads, 0, s>>>(ctx->ls_y, cnt, py);
    ls_v0<<<kLsBlocks, kLsThreads, 0, s>>>(un, um, ctx->ls_y, cnt, ctx->dctrl, dt, pd, py, kLsBlocks,
                                           (double *)v0_dev);
    CKC(ctx, cudaGetLastError());
    return FCH_OK;
}

static fch_status eval_F(fch_ctx *ctx, int src)
{
    TRY(col(ctx, CM_START, src));
    TRY(row(ctx, RM_F, FCH_FL_STORE_REAL, nullptr, nullptr, -1, 0.0, src));
    TRY(col(ctx, CM_F_FINISH, src));
    return FCH_OK;
}

static void fill_stats(fch_ctx *ctx, fch_stats *st)
{
    st->n_steps = ctx->hc.n_steps;
    st->n_rejects = ctx->hc.n_rejects;
    st->n_attempts = ctx->hc.n_attempts;
    st->n_psd_iter = ctx->hc.n_psd_iter;
    long long nf = 0;
    cudaMemcpy(&nf, ctx->nfft_dev, sizeof(long long), cudaMemcpyDeviceToHost);
    st->n_fft = nf;
    st->t = ctx->hc.t;
    st->k_last = ctx->hc.kn;
    st->e_last = ctx->hc.lte_den > 0 ? sqrt(ctx->hc.lte_num / ctx->hc.lte_den) : 0.0;
    st->last_psd_iter = ctx->hc.last_psd_iter;
}

// att0 (may be NULL): the attempts counted before this run; started (may be NULL):
// whether the run began with the backward-Euler start (one attempt)
static fch_status adaptive_begin(fch_ctx *ctx, fch_scheme scheme, double sigma, double t_final,
                                 long long *att0, bool *started)
{
    if (!ctx || !(sigma > 0) || scheme < FCH_IMEX || scheme > FCH_ETD) return FCH_EINVAL;
    if (!ctx->have_state || ctx->failed) return FCH_ESTATE;
    // the host mirror is read back only if something ran since it was last copied
    // (a run resumed right after the end of the last one needs no device read)
    if (!ctx->hc_fresh) TRY(pull_ctrl(ctx));
    if (ctx->hc.status) {
        ctx->failed = true;
        return (fch_status)ctx->hc.status;
    }
    if (!(t_final >= ctx->hc.t)) return FCH_EINVAL;
    fch_ctrl &c = ctx->hc;
    if (att0) *att0 = c.n_attempts;
    if (started) *started = c.kn <= 0;
    c.sigma = sigma;
    c.sigma2 = sigma * sigma;
    c.t_final = t_final;
    c.kmax = scheme == FCH_PSD ? fmin(ctx->p.k_max, ctx->p.psd_k_max) : ctx->p.k_max;
    c.itol = ctx->p.psd_nu * sigma;
    c.done = 0;
    c.adaptive = 1;
    TRY(push_ctrl(ctx));
    ctx->ad_scheme = scheme;
    ctx->ad_open = true;
    if (c.kn <= 0) {
        // first step k_1 = k_min by the backward-Euler start (Sec. 3.2)
        TRY(eval_F(ctx, FCH_SRC_UN));
        ctx->rvalid = true; // u^n in real space (the start uses gam = 0: u^{n-1} not read)
        TRY(ctl(ctx, OP_INIT_TRIAL, 0, ctx->p.k_min));
        fch_status s = enqueue_trial(ctx, scheme, true);
        if (s != FCH_OK) {
            ctx->failed = true;
            return s;
        }
        TRY(row(ctx, RM_F, FCH_FL_STORE_REAL, nullptr, nullptr, -1, 0.0, FCH_SRC_UNEW));
        TRY(col(ctx, CM_F_FINISH, FCH_SRC_UNEW));
        TRY(ctl(ctx, OP_ACCEPT, 0, 1.0));
    } else if (!ctx->have_F) {
        TRY(eval_F(ctx, FCH_SRC_UN));
        TRY(eval_F(ctx, 5));
        ctx->rvalid = true;
    }
    ctx->have_F = true;
    TRY(ctl(ctx, OP_INIT_TRIAL, 0, -1.0)); // the first trial of this run
    return FCH_OK;
}

extern "C" fch_status fch_adaptive_begin(fch_ctx *ctx, fch_scheme scheme, double sigma, double t_final)
{
    return adaptive_begin(ctx, scheme, sigma, t_final, nullptr, nullptr);
}

// one adaptive trial: the scheme's trial step, F of the trial with the AM3
// predictor and norms, and the decision plus the set-up of the next trial
static fch_status enqueue_adaptive_trial(fch_ctx *ctx)
{
    TRY(enqueue_trial(ctx, ctx->ad_scheme, true));
    TRY(row(ctx, RM_F, FCH_FL_STORE_REAL, nullptr, nullptr, -1, 0.0, FCH_SRC_UNEW));
    TRY(col(ctx, CM_F_FINISH, FCH_SRC_UNEW, FCH_FL_AM3));
    TRY(ctl(ctx, OP_DECIDE_INIT, ctx->geom.col_blocks)); // decide, then set up the next trial
    return FCH_OK;
}

// capture one adaptive trial of the current scheme into ctx->trial_graph;
// returns false (and leaves eager launching in place) if capture is unavailable
static bool capture_trial(fch_ctx *ctx)
{
    const int sc = ctx->ad_scheme;
    if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    ctx->capturing = true;
    fch_status s = enqueue_adaptive_trial(ctx);
    ctx->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (s != FCH_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return false;
    }
    e = cudaGraphInstantiate(&ctx->trial_graph[sc], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ctx->trial_graph[sc] = nullptr;
        cudaGetLastError();
        return false;
    }
    return true;
}

extern "C" fch_status fch_adaptive_enqueue(fch_ctx *ctx, int n)
{
    if (!ctx || n < 0) return FCH_EINVAL;
    if (!ctx->ad_open || ctx->failed) return FCH_ESTATE;
    const int sc = ctx->ad_scheme;
    for (int i = 0; i < n; i++) {
        // the first trial runs eagerly (it also sets the kernels' attributes);
        // later ones replay the captured graph unless per-pass timing is on
        const bool graph_ok = !ctx->timing && ctx->trial_warm[sc] && !ctx->trial_nograph[sc];
        if (graph_ok && !ctx->trial_graph[sc] && !capture_trial(ctx)) ctx->trial_nograph[sc] = true;
        if (graph_ok && ctx->trial_graph[sc]) {
            ctx->hc_fresh = false;
            CKC(ctx, cudaGraphLaunch(ctx->trial_graph[sc], ctx->stream));
            continue;
        }
        fch_status s = enqueue_adaptive_trial(ctx);
        if (s != FCH_OK) {
            ctx->failed = true;
            return s;
        }
        ctx->trial_warm[sc] = true;
    }
    return FCH_OK;
}

// pulled: the host mirror already holds the device's control block (no launch since);
// done (may be NULL) receives whether the run had reached t_final
static fch_status adaptive_end(fch_ctx *ctx, fch_stats *stats, bool pulled, bool *done = nullptr)
{
    if (!ctx) return FCH_EINVAL;
    if (!pulled) TRY(pull_ctrl(ctx));
    if (done) *done = ctx->hc.done != 0;
    fch_status result = FCH_OK;
    if (ctx->hc.status) {
        ctx->failed = true;
        result = (fch_status)ctx->hc.status;
    }
    // leave the control block ready for further calls
    fch_ctrl &c = ctx->hc;
    c.done = 0;
    c.adaptive = 0;
    c.itol = ctx->p.psd_itol;
    c.kmax = ctx->p.k_max;
    // a copy from pageable host memory has staged hc when it returns: hc stays the
    // device's block without reading it back
    TRY(push_ctrl(ctx));
    ctx->ad_open = false;
    if (stats) fill_stats(ctx, stats);
    return result;
}

extern "C" fch_status fch_adaptive_end(fch_ctx *ctx, fch_stats *stats)
{
    return adaptive_end(ctx, stats, false);
}

// The host reads the control block once per batch of trials: the first batch is
// enqueued right after the run's set-up (trials enqueued after the run has ended,
// or failed, return at once on the device), and the last read serves the end.
extern "C" fch_status fch_run_adaptive(fch_ctx *ctx, fch_scheme scheme, double sigma, double t_final,
                                       long long max_attempts, fch_stats *stats)
{
    long long att0 = 0;
    bool started = false;
    TRY(adaptive_begin(ctx, scheme, sigma, t_final, &att0, &started));
    long long used = started ? 1 : 0; // the backward-Euler start is an attempt
    bool out_of_attempts = false, pulled = false;
    for (;;) {
        if (pulled) {
            const fch_status s = pull_ctrl(ctx);
            if (s != FCH_OK) return s;
            const fch_ctrl &c = ctx->hc;
            if (c.status || c.done) break;
            used = c.n_attempts - att0;
        }
        if (max_attempts > 0 && used >= max_attempts) {
            out_of_attempts = true;
            break;
        }
        long long nb = ctx->p.sync_every;
        if (max_attempts > 0 && nb > max_attempts - used) nb = max_attempts - used;
        const fch_status s = fch_adaptive_enqueue(ctx, (int)nb);
        if (s != FCH_OK) {
            ctx->ad_open = false;
            return s;
        }
        pulled = true; // from here on every pass of the loop begins with a read
    }
    // the loop ends right after a read of the block unless the start alone used up
    // the attempts (then the start was enqueued after adaptive_begin's read)
    bool done = false;
    const fch_status e = adaptive_end(ctx, stats, pulled, &done);
    if (e != FCH_OK) return e;
    return out_of_attempts && !done ? FCH_ETIMEOUT : FCH_OK;
}

// ---------------------------------------------------------------------------
// ensembles: independent instances advanced together by one CUDA graph whose
// branches (one per member, each on its own stream) hold `rounds` adaptive trials
// of that member; branches of different members run concurrently, so small grids
// fill the GPU together. Members are ordinary contexts: their control blocks keep
// every per-trial value on the device, and a finished member's passes return at once.

struct fch_ensemble {
    int m;
    cudaStream_t stream; // the stream graphs launch on
    bool own_stream;
    fch_ctx **ctx;
    cudaStream_t *mstream; // member streams (owned)
    cudaEvent_t fork, *join;
    fch_ctrl **dctrls;     // the members' control blocks (device array)
    int *dflags, *hflags;  // per member: done | status << 1 (device, pinned host)
    cudaGraphExec_t graph;
    int *graph_schemes;    // per member: the scheme the graph holds (host)
    int graph_rounds;
};

__global__ void fch_ensemble_flags_kernel(fch_ctrl *const *c, int m, int *out)
{
    for (int i = threadIdx.x; i < m; i += blockDim.x) out[i] = c[i]->done | (c[i]->status << 1);
}

extern "C" fch_status fch_ensemble_destroy(fch_ensemble *e)
{
    if (!e) return FCH_OK;
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->graph) cudaGraphExecDestroy(e->graph);
    for (int i = 0; i < e->m; i++) {
        if (e->ctx && e->ctx[i]) fch_destroy(e->ctx[i]);
        if (e->mstream && e->mstream[i]) cudaStreamDestroy(e->mstream[i]);
        if (e->join && e->join[i]) cudaEventDestroy(e->join[i]);
    }
    if (e->fork) cudaEventDestroy(e->fork);
    if (e->dctrls) cudaFree(e->dctrls);
    if (e->dflags) cudaFree(e->dflags);
    if (e->hflags) cudaFreeHost(e->hflags);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    free(e->ctx);
    free(e->mstream);
    free(e->join);
    free(e->graph_schemes);
    free(e);
    return FCH_OK;
}

extern "C" fch_status fch_ensemble_create(int m, const fch_grid *grids, const fch_params *params, void *stream,
                                          fch_ensemble **out)
{
    if (!out || !grids || !params || m < 1 || m > FCH_ENSEMBLE_MAX) {
        fch_set_thread_error("fch_ensemble_create: invalid argument");
        return FCH_EINVAL;
    }
    *out = nullptr;
    fch_ensemble *e = (fch_ensemble *)calloc(1, sizeof(fch_ensemble));
    if (!e) return FCH_ENOMEM;
    e->m = m;
    e->ctx = (fch_ctx **)calloc(m, sizeof(fch_ctx *));
    e->mstream = (cudaStream_t *)calloc(m, sizeof(cudaStream_t));
    e->join = (cudaEvent_t *)calloc(m, sizeof(cudaEvent_t));
    e->graph_schemes = (int *)calloc(m, sizeof(int));
    if (!e->ctx || !e->mstream || !e->join || !e->graph_schemes) {
        fch_ensemble_destroy(e);
        return FCH_ENOMEM;
    }
    cudaError_t ce = cudaSuccess;
    if (stream) {
        e->stream = (cudaStream_t)stream;
    } else {
        ce = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
        e->own_stream = true;
    }
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming);
    for (int i = 0; i < m && ce == cudaSuccess; i++) {
        ce = cudaStreamCreateWithFlags(&e->mstream[i], cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e->join[i], cudaEventDisableTiming);
    }
    if (ce == cudaSuccess) ce = cudaMalloc((void **)&e->dctrls, m * sizeof(fch_ctrl *));
    if (ce == cudaSuccess) ce = cudaMalloc((void **)&e->dflags, m * sizeof(int));
    if (ce == cudaSuccess) ce = cudaMallocHost((void **)&e->hflags, m * sizeof(int));
    if (ce != cudaSuccess) {
        snprintf(g_plan_err, sizeof(g_plan_err), "fch_ensemble_create: %s", cudaGetErrorString(ce));
        fch_ensemble_destroy(e);
        return ce == cudaErrorMemoryAllocation ? FCH_ENOMEM : FCH_ECUDA;
    }
    fch_ctrl **hc = (fch_ctrl **)malloc(m * sizeof(fch_ctrl *));
    if (!hc) {
        fch_ensemble_destroy(e);
        return FCH_ENOMEM;
    }
    for (int i = 0; i < m; i++) {
        const fch_status s = fch_create(&grids[i], &params[i], e->mstream[i], &e->ctx[i]);
        if (s != FCH_OK) {
            snprintf(g_plan_err, sizeof(g_plan_err), "fch_ensemble_create: member %d: %s", i,
                     fch_status_string(s));
            free(hc);
            fch_ensemble_destroy(e);
            return s;
        }
        hc[i] = e->ctx[i]->dctrl;
    }
    ce = cudaMemcpy(e->dctrls, hc, m * sizeof(fch_ctrl *), cudaMemcpyHostToDevice);
    free(hc);
    if (ce != cudaSuccess) {
        fch_ensemble_destroy(e);
        return FCH_ECUDA;
    }
    *out = e;
    return FCH_OK;
}

extern "C" fch_status fch_ensemble_member(fch_ensemble *e, int i, fch_ctx **ctx)
{
    if (!e || !ctx || i < 0 || i >= e->m) return FCH_EINVAL;
    *ctx = e->ctx[i];
    return FCH_OK;
}

// capture the ensemble graph: fork from e->stream to every member stream, `rounds`
// trials per member (each member's trial is that of its own scheme), join back, then
// gather the members' flags to pinned memory
static fch_status ensemble_capture(fch_ensemble *e, const fch_scheme *schemes, int rounds)
{
    bool same = e->graph && e->graph_rounds == rounds;
    for (int i = 0; i < e->m && same; i++) same = e->graph_schemes[i] == (int)schemes[i];
    if (same) return FCH_OK;
    if (e->graph) {
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
    cudaError_t ce = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeRelaxed);
    if (ce != cudaSuccess) return FCH_ECUDA;
    fch_status s = FCH_OK;
    if (cudaEventRecord(e->fork, e->stream) != cudaSuccess) s = FCH_ECUDA;
    for (int i = 0; i < e->m && s == FCH_OK; i++) {
        fch_ctx *c = e->ctx[i];
        if (cudaStreamWaitEvent(c->stream, e->fork, 0) != cudaSuccess) s = FCH_ECUDA;
        c->capturing = true;
        for (int r = 0; r < rounds && s == FCH_OK; r++) s = enqueue_adaptive_trial(c);
        c->capturing = false;
        if (s == FCH_OK && cudaEventRecord(e->join[i], c->stream) != cudaSuccess) s = FCH_ECUDA;
        if (s == FCH_OK && cudaStreamWaitEvent(e->stream, e->join[i], 0) != cudaSuccess) s = FCH_ECUDA;
    }
    if (s == FCH_OK) {
        fch_ensemble_flags_kernel<<<1, 256, 0, e->stream>>>(e->dctrls, e->m, e->dflags);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(e->hflags, e->dflags, e->m * sizeof(int), cudaMemcpyDeviceToHost, e->stream) !=
                cudaSuccess)
            s = FCH_ECUDA;
    }
    cudaGraph_t g = nullptr;
    ce = cudaStreamEndCapture(e->stream, &g);
    if (s == FCH_OK && (ce != cudaSuccess || !g)) s = FCH_ECUDA;
    if (s == FCH_OK && cudaGraphInstantiate(&e->graph, g, 0) != cudaSuccess) {
        e->graph = nullptr;
        s = FCH_ECUDA;
    }
    if (g) cudaGraphDestroy(g);
    if (s != FCH_OK) {
        cudaGetLastError();
        return s;
    }
    for (int i = 0; i < e->m; i++) e->graph_schemes[i] = (int)schemes[i];
    e->graph_rounds = rounds;
    return FCH_OK;
}

extern "C" fch_status fch_ensemble_run_adaptive_each(fch_ensemble *e, const fch_scheme *schemes,
                                                     const double *sigmas, double t_final, int rounds,
                                                     long long max_launches, fch_stats *stats)
{
    if (!e || !schemes || !sigmas || rounds < 1 || rounds > 1024 || max_launches < 0) return FCH_EINVAL;
    for (int i = 0; i < e->m; i++) {
        if (!(sigmas[i] > 0) || schemes[i] < FCH_IMEX || schemes[i] > FCH_ETD) return FCH_EINVAL;
        if (e->ctx[i]->timing) return FCH_ESTATE;
    }
    // every member begins (host checks, backward-Euler start) and runs one trial
    // on its own stream; the first trial also sets the kernels' attributes
    for (int i = 0; i < e->m; i++) {
        TRY(fch_adaptive_begin(e->ctx[i], schemes[i], sigmas[i], t_final));
        TRY(fch_adaptive_enqueue(e->ctx[i], 1));
        if (cudaEventRecord(e->join[i], e->ctx[i]->stream) != cudaSuccess ||
            cudaStreamWaitEvent(e->stream, e->join[i], 0) != cudaSuccess)
            return FCH_ECUDA;
    }
    fch_status result = ensemble_capture(e, schemes, rounds);
    if (result != FCH_OK) {
        for (int i = 0; i < e->m; i++) fch_adaptive_end(e->ctx[i], nullptr);
        return result;
    }
    for (int i = 0; i < e->m; i++) e->ctx[i]->hc_fresh = false; // the graph writes their blocks
    for (long long l = 0;; l++) {
        if (max_launches > 0 && l >= max_launches) {
            result = FCH_ETIMEOUT;
            break;
        }
        if (cudaGraphLaunch(e->graph, e->stream) != cudaSuccess || cudaStreamSynchronize(e->stream) != cudaSuccess) {
            result = FCH_ECUDA;
            break;
        }
        bool all_done = true;
        for (int i = 0; i < e->m; i++) {
            all_done = all_done && (e->hflags[i] & 1);
            if ((e->hflags[i] >> 1) && result == FCH_OK) result = (fch_status)(e->hflags[i] >> 1);
        }
        if (all_done || result != FCH_OK) break;
    }
    // the members' own streams follow the graph's work before their next calls
    if (cudaEventRecord(e->fork, e->stream) != cudaSuccess) return FCH_ECUDA;
    for (int i = 0; i < e->m; i++) {
        if (cudaStreamWaitEvent(e->ctx[i]->stream, e->fork, 0) != cudaSuccess) return FCH_ECUDA;
        const fch_status s = fch_adaptive_end(e->ctx[i], stats ? &stats[i] : nullptr);
        if (s != FCH_OK && result == FCH_OK) result = s;
    }
    return result;
}

extern "C" fch_status fch_ensemble_run_adaptive(fch_ensemble *e, fch_scheme scheme, double sigma, double t_final,
                                                int rounds, long long max_launches, fch_stats *stats)
{
    if (!e) return FCH_EINVAL;
    std::vector<fch_scheme> schemes(e->m, scheme);
    std::vector<double> sigmas(e->m, sigma);
    return fch_ensemble_run_adaptive_each(e, schemes.data(), sigmas.data(), t_final, rounds, max_launches, stats);
}

extern "C" fch_status fch_pass_timing(fch_ctx *ctx, int on)
{
    if (!ctx) return FCH_EINVAL;
    if (on && !ctx->timing) {
        for (int i = 0; i < 2 * 2048; i++)
            CKC(ctx, cudaEventCreate(&ctx->ev[i]));
        ctx->nev = 0;
        memset(ctx->t_ms, 0, sizeof(ctx->t_ms));
        memset(ctx->t_n, 0, sizeof(ctx->t_n));
        ctx->timing = true;
    } else if (!on && ctx->timing) {
        timing_flush(ctx);
        for (int i = 0; i < 2 * 2048; i++) cudaEventDestroy(ctx->ev[i]);
        ctx->timing = false;
    }
    return FCH_OK;
}

extern "C" fch_status fch_pass_times(fch_ctx *ctx, double *ms, long long *launches, int n)
{
    if (!ctx || !ms || !launches || n < FCH_NPASS) return FCH_EINVAL;
    timing_flush(ctx);
    for (int i = 0; i < FCH_NPASS; i++) {
        ms[i] = ctx->t_ms[i];
        launches[i] = ctx->t_n[i];
        ctx->t_ms[i] = 0;
        ctx->t_n[i] = 0;
    }
    return FCH_OK;
}

extern "C" fch_status fch_get_stats(fch_ctx *ctx, fch_stats *st)
{
    if (!ctx || !st) return FCH_EINVAL;
    TRY(pull_ctrl(ctx));
    fill_stats(ctx, st);
    return FCH_OK;
}

extern "C" fch_status fch_energy(fch_ctx *ctx, double *E)
{
    if (!ctx || !E) return FCH_EINVAL;
    if (!ctx->have_state) return FCH_ESTATE;
    TRY(col(ctx, CM_START, FCH_SRC_UN, FCH_FL_NOSKIP));
    TRY(rowt(ctx, RM_ENERGY, FCH_FL_NOSKIP, OP_ENERGY));
    TRY(fch_synchronize(ctx));
    *E = ctx->hc.energy;
    return FCH_OK;
}

extern "C" fch_status fch_mass(fch_ctx *ctx, double *m)
{
    if (!ctx || !m) return FCH_EINVAL;
    if (!ctx->have_state) return FCH_ESTATE;
    TRY(fch_synchronize(ctx));
    double re;
    const void *u0 = ctx->U[ctx->hc.iu_n];
    if (ctx->prec == FCH_MIXED) {
        float v[2];
        CKC(ctx, cudaMemcpy(v, u0, sizeof(v), cudaMemcpyDeviceToHost));
        re = v[0];
    } else if (ctx->prec == FCH_FP32X2) {
        float v[4]; // (re.hi, re.lo, im.hi, im.lo)
        CKC(ctx, cudaMemcpy(v, u0, sizeof(v), cudaMemcpyDeviceToHost));
        re = (double)v[0] + (double)v[1];
    } else {
        double v[2];
        CKC(ctx, cudaMemcpy(v, u0, sizeof(v), cudaMemcpyDeviceToHost));
        re = v[0];
    }
    // m = 1/2 int (u + 1) = 1/2 (h^2 sum u + L^2), sum u = the k = 0 coefficient
    const double L = ctx->grid.L;
    *m = 0.5 * (ctx->kp.h2 * re + L * L);
    return FCH_OK;
}

extern "C" fch_status fch_rhs_device(fch_ctx *ctx, const void *u_dev, void *F_dev, int dtype)
{
    if (!ctx || !u_dev || !F_dev || (dtype != 0 && dtype != 1)) return FCH_EINVAL;
    const int io = (dtype == 0 ? FCH_FL_F64IO : 0) | FCH_FL_NOSKIP;
    TRY(row(ctx, RM_R2C_LOAD, io, u_dev));
    TRY(col(ctx, CM_FWD_STORE, 0, FCH_FL_NOSKIP, nullptr, nullptr, ctx->Pb, nullptr));
    TRY(col(ctx, CM_START, FCH_SRC_IN0, FCH_FL_NOSKIP, ctx->Pb));
    TRY(row(ctx, RM_F, FCH_FL_NOSKIP));
    TRY(col(ctx, CM_F_FINISH, FCH_SRC_IN0, FCH_FL_NOSKIP, ctx->Pb, nullptr, ctx->Qb));
    TRY(col(ctx, CM_INV_LOAD, 0, FCH_FL_NOSKIP, ctx->Qb));
    TRY(row(ctx, RM_C2R_STORE, io, nullptr, F_dev));
    return FCH_OK;
}

extern "C" fch_status fch_get_sav_r(fch_ctx *ctx, double *r_n, double *r_nm1)
{
    if (!ctx || !r_n || !r_nm1) return FCH_EINVAL;
    TRY(fch_synchronize(ctx));
    *r_n = ctx->hc.r_n;
    *r_nm1 = ctx->hc.r_m;
    return FCH_OK;
}

// ---------------------------------------------------------------------------
// standalone transforms
// ---------------------------------------------------------------------------
// autotuner of the pass tiles

static std::mutex g_tune_mutex;
static fch_tile g_tune[3][12];
static bool g_tune_ok[3][12];

// the tiles fch_autotune chose for (n, prec) in this process, if it ran
static bool tuned_tiles(int n, int prec, int *row, int *col)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    const int l = ilog2(n);
    if (prec < 0 || prec > 2 || l < 0 || l >= 12 || !g_tune_ok[prec][l]) return false;
    *row = g_tune[prec][l].tile_row;
    *col = g_tune[prec][l].tile_col;
    return true;
}

// Mean time (us) of `reps` launches of one pass after two untimed ones.
static int plan_chunk(int n, int prec);

template <typename F> static cudaError_t time_pass(F launch, cudaStream_t s, int reps, double *us)
{
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    for (int i = 0; i < 2 && e == cudaSuccess; i++) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    for (int i = 0; i < reps && e == cudaSuccess; i++) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    *us = 1e3 * ms / reps;
    return e;
}

extern "C" fch_status fch_autotune(int n, int prec, void *stream, fch_tile *out)
{
    if (!out || !pow2_in_range(n) || prec < 0 || prec > 2) {
        fch_set_thread_error("fch_autotune: invalid argument");
        return FCH_EINVAL;
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        if (g_tune_ok[prec][ilog2(n)]) {
            *out = g_tune[prec][ilog2(n)];
            return FCH_OK;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool single = prec == FCH_MIXED;
    const size_t csz = single ? 8 : 16, rsz = single ? 4 : 8;
    // the passes are timed as a standalone transform plan launches them: as many
    // field pairs per launch as a plan's work array holds (FCH_FP32X2, which has no
    // plans, one pair)
    const int np = prec == FCH_FP32X2 ? 1 : plan_chunk(n, prec);
    const size_t rb = (size_t)n * n * rsz, cb = (size_t)(n / 2 + 1) * n * csz;
    void *x = nullptr, *Z = nullptr, *X = nullptr, *tw = nullptr, *tw2 = nullptr;
    cudaError_t e = cudaMalloc(&x, 2 * np * rb);
    if (e == cudaSuccess) e = cudaMalloc(&Z, (size_t)np * n * n * csz);
    if (e == cudaSuccess) e = cudaMalloc(&X, 2 * np * cb);
    if (e == cudaSuccess) e = cudaMalloc(&tw, (size_t)n * csz);
    if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, 2 * np * rb, s);
    fch_ctx dummy;
    if (e == cudaSuccess && upload_twiddles(&dummy, n, prec, tw, s) != FCH_OK) e = cudaErrorUnknown;
    if (e == cudaSuccess && single && n == 1024) e = upload_tw2(&tw2, s);
    fch_kparams kp;
    memset(&kp, 0, sizeof(kp));
    kp.N = n;
    kp.logN = ilog2(n);
    kp.inv_n2 = 1.0 / ((double)n * n);
    kp.Z = Z;
    kp.tw = tw;
    kp.tw2 = tw2;
    kp.tail_op = -1;
    kp.flags = FCH_FL_NOSKIP | (single ? 0 : FCH_FL_F64IO);
    kp.in0 = x;
    kp.in1 = (const char *)x + rb;
    kp.out0 = X;
    kp.out1 = (char *)X + cb;
    kp.npairs = np;
    kp.pdl = prec == FCH_FP32X2 ? 0 : 1; // as plans launch
    auto launch = [&](bool is_col, const fch_kparams &kk) {
        fch_kparams k = kk; // pair j reads fields 2j, 2j+1 and writes their spectra
        k.pstride_in = is_col ? 0 : 2 * (long long)rb;
        k.pstride_out = is_col ? 2 * (long long)cb : 0;
        if (is_col)
            return prec == FCH_MIXED    ? fch_launch_col_f32(CM_FWD_STORE, k, s)
                   : prec == FCH_FP32X2 ? fch_launch_col_dfl(CM_FWD_STORE, k, s)
                                        : fch_launch_col_f64(CM_FWD_STORE, k, s);
        return prec == FCH_MIXED    ? fch_launch_row_f32(RM_R2C_LOAD, k, s)
               : prec == FCH_FP32X2 ? fch_launch_row_dfl(RM_R2C_LOAD, k, s)
                                    : fch_launch_row_f64(RM_R2C_LOAD, k, s);
    };
    // candidates: the default tiles (timed first), the shared-memory kernels where the
    // default is the warp-level path, and the generic kernel at 1..16 rows (column
    // pairs) a block; another tile replaces the default only if 3 % faster
    fch_tile best;
    memset(&best, 0, sizeof(best));
    const int reps = n >= 1024 ? 10 : 20;
    for (int is_col = 0; is_col < 2 && e == cudaSuccess; is_col++) {
        double best_us = 1e30, def_us = 0;
        int best_t = 0;
        const int cands[] = {0, -1, -2, 1, 2, 4, 8, 16};
        for (int c : cands) {
            if (c < 0 && n != 1024) continue;
            if (!fch_tile_valid(n, single, is_col ? 0 : c, is_col ? c : 0)) continue;
            fch_kparams k = kp;
            k.tile_row = is_col ? 0 : c;
            k.tile_col = is_col ? c : 0;
            k.P = fch_geometry_tiled(n, single, 0, k.tile_col).P;
            double us = 0;
            e = time_pass([&] { return launch(is_col != 0, k); }, s, reps, &us);
            if (e != cudaSuccess) break;
            best.candidates++;
            if (c == 0) {
                def_us = us;
                best_us = us;
            } else if (us < best_us && us < 0.97 * def_us) { // the default unless 3 % faster
                best_us = us;
                best_t = c;
            }
        }
        if (is_col) {
            best.tile_col = best_t;
            best.col_us = best_us;
            best.col_default_us = def_us;
        } else {
            best.tile_row = best_t;
            best.row_us = best_us;
            best.row_default_us = def_us;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (void *b : {x, Z, X, tw, tw2})
        if (b) cudaFree(b);
    if (e != cudaSuccess) {
        snprintf(g_plan_err, sizeof(g_plan_err), "fch_autotune: %s", cudaGetErrorString(e));
        return FCH_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune[prec][ilog2(n)] = best;
    g_tune_ok[prec][ilog2(n)] = true;
    *out = best;
    return FCH_OK;
}

static fch_tile g_tune_step[3][12];
static bool g_tune_step_ok[3][12];

// Mean time (us) of one adaptive IMEX trial (sigma_tol 1e-5, the library's default
// parameters at q = 0) of an n x n context with the given tiles, on stream s: the
// start and four trials untimed (the second one captures the trial graph), then
// `reps` trials between two events. The state is a circular bilayer of radius 2.
static fch_status time_trials(int n, int prec, int tr, int tc, cudaStream_t s, int reps, double *us)
{
    fch_params p;
    fch_params_default(&p, 0.0);
    p.prec = prec;
    p.tile_row = tr;
    p.tile_col = tc;
    const double L = 4.0 * M_PI, h = L / n;
    const fch_grid g = {n, L, -0.5 * L};
    fch_ctx *c = nullptr;
    TRY(fch_create(&g, &p, s, &c));
    std::vector<double> u0((size_t)n * n);
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            const double x = g.x0 + i * h, y = g.x0 + j * h, r = sqrt(x * x + y * y) - 2.0;
            u0[(size_t)j * n + i] = -1.0 + 1.5 * exp(-r * r / (2.0 * p.eps * p.eps));
        }
    cudaEvent_t a = nullptr, b = nullptr;
    fch_status st = fch_set_state(c, u0.data(), u0.size());
    if (st == FCH_OK) st = fch_adaptive_begin(c, FCH_IMEX, 1e-5, 1e30);
    if (st == FCH_OK) st = fch_adaptive_enqueue(c, 4);
    // the context's stream (its own one when s is NULL)
    if (st == FCH_OK && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess ||
                         cudaEventRecord(a, c->stream) != cudaSuccess))
        st = FCH_ECUDA;
    if (st == FCH_OK) st = fch_adaptive_enqueue(c, reps);
    float ms = 0.f;
    if (st == FCH_OK && (cudaEventRecord(b, c->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
        st = FCH_ECUDA;
    if (st == FCH_OK) st = fch_adaptive_end(c, nullptr);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st != FCH_OK) snprintf(g_plan_err, sizeof(g_plan_err), "fch_autotune_step: %s", fch_last_cuda_error(c));
    fch_destroy(c);
    *us = 1e3 * ms / reps;
    return st;
}

extern "C" fch_status fch_autotune_step(int n, int prec, void *stream, fch_tile *out)
{
    if (!out || !pow2_in_range(n) || prec < 0 || prec > 2) {
        fch_set_thread_error("fch_autotune_step: invalid argument");
        return FCH_EINVAL;
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        if (g_tune_step_ok[prec][ilog2(n)]) {
            *out = g_tune_step[prec][ilog2(n)];
            return FCH_OK;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool single = prec == FCH_MIXED;
    const int reps = n >= 2048 ? 8 : n >= 1024 ? 16 : 32;
    // the row tiles with the default columns, then the column tiles with the chosen
    // rows; another tile replaces the default only if 3 % faster
    fch_tile best;
    memset(&best, 0, sizeof(best));
    // (columns also at four points a thread: -3, -4, -6 for 1, 2, 4 pairs a block; rows
    // at four points a thread are tested as fixed-step tiles only, so not candidates)
    const int cands[] = {0, -1, -2, 1, 2, 4, 8, 16, -3, -4, -6};
    for (int is_col = 0; is_col < 2; is_col++) {
        double best_us = 1e30, def_us = 0;
        int best_t = 0;
        for (int c : cands) {
            if ((c == -1 || c == -2) && n != 1024) continue;
            if (c <= -3 && !is_col) continue;
            const int tr = is_col ? best.tile_row : c, tc = is_col ? c : 0;
            if (!fch_tile_valid(n, single, tr, tc)) continue;
            double us = 0;
            if (is_col && c == 0) {
                us = best.row_us; // the rows' winner with the default columns
            } else {
                const fch_status st = time_trials(n, prec, tr, tc, s, reps, &us);
                if (st != FCH_OK) return st;
                best.candidates++;
            }
            if (c == 0) {
                def_us = us;
                best_us = us;
            } else if (us < best_us && us < 0.97 * def_us) {
                best_us = us;
                best_t = c;
            }
        }
        if (is_col) {
            best.tile_col = best_t;
            best.col_us = best_us;
            best.col_default_us = def_us;
        } else {
            best.tile_row = best_t;
            best.row_us = best_us;
            best.row_default_us = def_us;
        }
    }
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_step[prec][ilog2(n)] = best;
    g_tune_step_ok[prec][ilog2(n)] = true;
    *out = best;
    return FCH_OK;
}

extern "C" fch_status fch_autotune_reset(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    memset(g_tune_ok, 0, sizeof(g_tune_ok));
    memset(g_tune_step_ok, 0, sizeof(g_tune_step_ok));
    return FCH_OK;
}

struct fch_fft_plan {
    int N, prec;
    int chunk; // field pairs transformed by one launch (the work array holds that many)
    cudaStream_t stream;
    fch_geom geom;
    fch_kparams kp;
    void *Z, *tw, *tw2;
    int *err; // device word: set by a pass whose bounded wait on a bulk copy ran out
};

// Field pairs per launch of a standalone transform: as many as a 64 MiB work array
// holds (at most 64), so a batch runs as a few launches of many blocks rather than
// one launch pair per two fields, and the work array stays in L2 between the passes.
static int plan_chunk(int n, int prec)
{
    const size_t per = (size_t)n * n * (prec ? 8 : 16);
    size_t c = ((size_t)64 << 20) / per;
    if (c < 1) c = 1;
    if (c > 64) c = 64;
    return (int)c;
}

extern "C" fch_status fch_fft_plan_create(int n, int prec, void *stream, fch_fft_plan **out)
{
    if (!out || !pow2_in_range(n) || (prec != 0 && prec != 1)) return FCH_EINVAL;
    fch_fft_plan *pl = (fch_fft_plan *)calloc(1, sizeof(fch_fft_plan));
    if (!pl) return FCH_ENOMEM;
    pl->N = n;
    pl->prec = prec;
    pl->stream = (cudaStream_t)stream;
    int trow = 0, tcol = 0;
    tuned_tiles(n, prec, &trow, &tcol);
    pl->geom = fch_geometry_tiled(n, prec, trow, tcol);
    pl->chunk = plan_chunk(n, prec);
    const size_t csz = prec ? 8 : 16;
    cudaError_t e = cudaMalloc(&pl->Z, (size_t)pl->chunk * n * n * csz);
    if (e == cudaSuccess) e = cudaMalloc(&pl->tw, (size_t)n * csz);
    if (e == cudaSuccess) e = cudaMalloc(&pl->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->err, 0, sizeof(int), pl->stream);
    if (e != cudaSuccess) {
        fch_fft_plan_destroy(pl);
        return e == cudaErrorMemoryAllocation ? FCH_ENOMEM : FCH_ECUDA;
    }
    fch_ctx dummy;
    if (upload_twiddles(&dummy, n, prec, pl->tw, pl->stream) != FCH_OK) {
        fch_fft_plan_destroy(pl);
        return FCH_ECUDA;
    }
    memset(&pl->kp, 0, sizeof(pl->kp));
    pl->kp.N = n;
    pl->kp.logN = ilog2(n);
    pl->kp.P = pl->geom.P;
    pl->kp.tile_row = trow;
    pl->kp.tile_col = tcol;
    pl->kp.pdl = 1;
    pl->kp.inv_n2 = 1.0 / ((double)n * n);
    pl->kp.tail_op = -1;
    pl->kp.cf.inv_n2 = (float)pl->kp.inv_n2;
    pl->kp.cd.inv_n2 = pl->kp.inv_n2;
    pl->kp.Z = pl->Z;
    pl->kp.tw = pl->tw;
    pl->kp.err = pl->err;
    if (prec && n == 1024) {
        if (upload_tw2(&pl->tw2, pl->stream) != cudaSuccess) {
            fch_fft_plan_destroy(pl);
            return FCH_ECUDA;
        }
        pl->kp.tw2 = pl->tw2;
    }
    *out = pl;
    return FCH_OK;
}

extern "C" fch_status fch_fft_plan_destroy(fch_fft_plan *pl)
{
    if (!pl) return FCH_OK;
    if (pl->Z) cudaFree(pl->Z);
    if (pl->tw) cudaFree(pl->tw);
    if (pl->tw2) cudaFree(pl->tw2);
    if (pl->err) cudaFree(pl->err);
    free(pl);
    return FCH_OK;
}

extern "C" fch_status fch_fft_plan_status(fch_fft_plan *pl)
{
    if (!pl) return FCH_EINVAL;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, pl->err, sizeof(int), cudaMemcpyDeviceToHost, pl->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pl->stream);
    if (e != cudaSuccess) {
        snprintf(g_plan_err, sizeof(g_plan_err), "plan status: %s", cudaGetErrorString(e));
        return FCH_ECUDA;
    }
    if (h) {
        snprintf(g_plan_err, sizeof(g_plan_err), "a column pass's wait on a bulk copy ran out of time");
        if (cudaMemsetAsync(pl->err, 0, sizeof(int), pl->stream) == cudaSuccess)
            cudaStreamSynchronize(pl->stream);
        return FCH_ECUDA;
    }
    return FCH_OK;
}

static cudaError_t plan_pass(fch_fft_plan *pl, bool is_col, int mode, const void *in0, const void *in1,
                             void *out0, void *out1, int npairs, long long pstride_in, long long pstride_out)
{
    fch_kparams kp = pl->kp;
    kp.flags = FCH_FL_NOSKIP | (pl->prec ? 0 : FCH_FL_F64IO);
    kp.in0 = in0;
    kp.in1 = in1;
    kp.out0 = out0;
    kp.out1 = out1;
    kp.npairs = npairs;
    kp.pstride_in = pstride_in;
    kp.pstride_out = pstride_out;
    cudaError_t e;
    if (is_col)
        e = pl->prec ? fch_launch_col_f32(mode, kp, pl->stream) : fch_launch_col_f64(mode, kp, pl->stream);
    else
        e = pl->prec ? fch_launch_row_f32(mode, kp, pl->stream) : fch_launch_row_f64(mode, kp, pl->stream);
    if (e != cudaSuccess)
        snprintf(g_plan_err, sizeof(g_plan_err), "%s pass %d: %s", is_col ? "column" : "row", mode,
                 cudaGetErrorString(e));
    return e;
}

// Fields 2j and 2j+1 form pair j (one complex transform); pairs go chunk at a time,
// each chunk as one row and one column launch with a grid row per pair; an odd last
// field is a pair of its own with no second field.
extern "C" fch_status fch_fft_r2c(fch_fft_plan *pl, const void *x, void *X, int batch)
{
    if (!pl || !x || !X || batch < 0) return FCH_EINVAL;
    const long long N = pl->N, rb = N * N * (pl->prec ? 4 : 8), cb = (N / 2 + 1) * N * (pl->prec ? 8 : 16);
    const int full = batch / 2;
    for (int j = 0; j < full; j += pl->chunk) {
        const int np = full - j < pl->chunk ? full - j : pl->chunk;
        const char *x0 = (const char *)x + 2 * j * rb;
        char *X0 = (char *)X + 2 * j * cb;
        if (plan_pass(pl, false, RM_R2C_LOAD, x0, x0 + rb, nullptr, nullptr, np, 2 * rb, 0) != cudaSuccess)
            return FCH_ECUDA;
        if (plan_pass(pl, true, CM_FWD_STORE, nullptr, nullptr, X0, X0 + cb, np, 0, 2 * cb) != cudaSuccess)
            return FCH_ECUDA;
    }
    if (batch & 1) {
        const char *x0 = (const char *)x + (batch - 1) * rb;
        char *X0 = (char *)X + (batch - 1) * cb;
        if (plan_pass(pl, false, RM_R2C_LOAD, x0, nullptr, nullptr, nullptr, 1, 0, 0) != cudaSuccess)
            return FCH_ECUDA;
        if (plan_pass(pl, true, CM_FWD_STORE, nullptr, nullptr, X0, nullptr, 1, 0, 0) != cudaSuccess)
            return FCH_ECUDA;
    }
    return FCH_OK;
}

extern "C" fch_status fch_fft_c2r(fch_fft_plan *pl, const void *X, void *x, int batch)
{
    if (!pl || !x || !X || batch < 0) return FCH_EINVAL;
    const long long N = pl->N, rb = N * N * (pl->prec ? 4 : 8), cb = (N / 2 + 1) * N * (pl->prec ? 8 : 16);
    const int full = batch / 2;
    for (int j = 0; j < full; j += pl->chunk) {
        const int np = full - j < pl->chunk ? full - j : pl->chunk;
        const char *X0 = (const char *)X + 2 * j * cb;
        char *x0 = (char *)x + 2 * j * rb;
        if (plan_pass(pl, true, CM_INV_LOAD, X0, X0 + cb, nullptr, nullptr, np, 2 * cb, 0) != cudaSuccess)
            return FCH_ECUDA;
        if (plan_pass(pl, false, RM_C2R_STORE, nullptr, nullptr, x0, x0 + rb, np, 0, 2 * rb) != cudaSuccess)
            return FCH_ECUDA;
    }
    if (batch & 1) {
        const char *X0 = (const char *)X + (batch - 1) * cb;
        char *x0 = (char *)x + (batch - 1) * rb;
        if (plan_pass(pl, true, CM_INV_LOAD, X0, nullptr, nullptr, nullptr, 1, 0, 0) != cudaSuccess)
            return FCH_ECUDA;
        if (plan_pass(pl, false, RM_C2R_STORE, nullptr, nullptr, x0, nullptr, 1, 0, 0) != cudaSuccess)
            return FCH_ECUDA;
    }
    return FCH_OK;
}

// host-side geometry of tiles row / col and whether they launch (CPU tests);
// returns 1 valid, 0 invalid, -1 bad arguments
extern "C" int fch_debug_tile(int n, int prec, int row, int col, int *out)
{
    if (!pow2_in_range(n) || !out || prec < 0 || prec > 2) return -1;
    const fch_geom g = fch_geometry_tiled(n, prec, row, col);
    out[0] = g.col_blocks;
    out[1] = g.col_threads;
    out[2] = g.col_smem;
    out[3] = g.row_blocks;
    out[4] = g.row_threads;
    out[5] = g.row_smem;
    out[6] = g.rpb;
    out[7] = g.P;
    return fch_tile_valid(n, prec, row, col) ? 1 : 0;
}

// the per-stage twiddle table of the shared-memory transforms for radix-2^lp stages
// (lp 3: eight points a thread, 2: four), n complex entries as 2n doubles (CPU tests)
extern "C" int fch_debug_twiddles(int n, int lp, double *out)
{
    if (!pow2_in_range(n) || (lp != 2 && lp != 3) || !out) return 1;
    make_twiddles(n, out, lp);
    return 0;
}

// which trials and fixed steps of a context replay a captured graph (tests):
// out[s] for scheme s: 1 captured, -1 capture failed (eager launches), 0 not yet;
// out[4 + s]: 1 if a fixed step of scheme s is captured
extern "C" int fch_debug_graphs(const fch_ctx *ctx, int *out)
{
    if (!ctx || !out) return 1;
    for (int s = 0; s < 4; s++) {
        out[s] = ctx->trial_graph[s] ? 1 : ctx->trial_nograph[s] ? -1 : 0;
        out[4 + s] = ctx->fixed_graph[s] ? 1 : 0;
    }
    return 0;
}

// host-side geometry query (used by the CPU tests of the launch configuration)
extern "C" int fch_debug_geometry(int n, int prec, int *out)
{
    if (!pow2_in_range(n) || !out) return 1;
    const fch_geom g = fch_geometry(n, prec);
    out[0] = g.col_blocks;
    out[1] = g.col_threads;
    out[2] = g.col_smem;
    out[3] = g.row_blocks;
    out[4] = g.row_threads;
    out[5] = g.row_smem;
    out[6] = g.rpb;
    out[7] = g.P;
    out[8] = (int)sizeof(fch_ctrl);
    return 0;
}
