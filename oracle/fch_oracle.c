/*
 * fch_oracle.c -- plain, slow FP64 CPU oracle for the Fourier pseudo-spectral
 * steppers of the functionalized Cahn-Hilliard (FCH) gradient flow
 * (Christlieb, Promislow, Tan, Wang, Wetton, Wise, arXiv 2006.04784).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this library. It shares no code,
 * header, table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Design rules followed here:
 *   - every quantity is a double; spectra are FULL N x N complex arrays
 *     (no half-spectrum packing, no fused passes, no reordering);
 *   - the FFT is an iterative radix-2 transform written out below, applied to
 *     rows and then to columns; forward unnormalised, inverse scaled by 1/N^2;
 *   - differential operators are applied as symbols on those spectra
 *     (Laplacian = -|k|^2, k = 2*pi*m/L, m in [-N/2, N/2-1]);
 *   - each routine restates one passage of the paper, cited in its comment.
 *
 * Readings of points the paper leaves open (each is also listed in the design notes):
 *   R1 first step: backward Euler, the k_{n-1} -> infinity limit of the
 *      variable-step BDF2 (a = 1/k, b = -1/k, c = 0, u* = u^n).      (Sec. 3.2)
 *   R2 accepted step advances time by the accepted trial size; the A_dp
 *      proposal becomes the next trial size.                          (Sec. 3.2)
 *   R3 e = 0 in A_dp is replaced by 1e-16.                            (Sec. 3.2)
 *   R4 the trial step is clipped so the run ends exactly at t_final.
 *   R5 a trial of size <= k_min is accepted even if e > sigma_tol.    (Sec. 3.2)
 *   R6 discrete L2 norm ||f||^2 = h^2 sum f^2.                        (Sec. 3.2, 3.3)
 *   R7 PSD: residual and direction act on the k != 0 modes only.      (Sec. 3.3)
 *   R8 PSD lambda: linear interpolation in k between the columns of the
 *      search-size table, clamped at both ends.                       (Table SearchSize)
 *   R9 ETD phi_2 by its Taylor series for |z| < 1e-2.                 (Sec. 3.6)
 *   R10 SAV solved by the p/q split of the linear system.             (Sec. 3.5)
 *   R11 the |grad u|^2 term of the energy is -(u, Lap u).             (eq. Functional)
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* parameters                                                                 */
/* ------------------------------------------------------------------------- */
typedef struct {
    double eps, q, gamma, b_minus, b_plus, eta1, eta2; /* model, eqs. (e:Wq-def), (Functional) */
    double beta1, beta2, zeta, D0;                     /* SAV, eqs. (4.1)-(4.8) */
    double kappa0, kappa2;                             /* ETD, eq. (ETD-L) */
    double rho_s, k_min, k_max;                        /* controller, Sec. 3.2 */
    int zero_stab_cap;                                 /* A_dp <= (1+sqrt 2) k, Sec. 3.2 */
    int well;            /* 0: W_q of eq. (e:Wq-def); 1: quadratic test well alpha/2 (u-b_-)^2 */
    double psd_nu;       /* i_tol = nu * sigma_tol in adaptive runs, Sec. 3.3 */
    double psd_itol;     /* i_tol for fixed-step PSD */
    double psd_lambda;   /* > 0: fixed search step; <= 0: Table SearchSize */
    int psd_max_iter;
} orc_params;

/* ------------------------------------------------------------------------- */
/* FFT: iterative radix-2, decimation in time, in place                       */
/* ------------------------------------------------------------------------- */
/* sign = -1 forward (e^{-i...}), +1 inverse (unscaled). n is a power of two. */
void orc_fft1d(cplx *a, int n, int stride, int sign)
{
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            cplx t = a[(long)i * stride];
            a[(long)i * stride] = a[(long)j * stride];
            a[(long)j * stride] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        for (int i = 0; i < n; i += len) {
            for (int j = 0; j < len / 2; j++) {
                double ang = sign * 2.0 * M_PI * (double)j / (double)len;
                cplx w = cos(ang) + I * sin(ang);
                cplx x = a[(long)(i + j) * stride];
                cplx y = w * a[(long)(i + j + len / 2) * stride];
                a[(long)(i + j) * stride] = x + y;
                a[(long)(i + j + len / 2) * stride] = x - y;
            }
        }
    }
}

/* 2D transform of an N x N row-major array: every row, then every column.
 * Forward is unnormalised; the inverse is scaled by 1/N^2. */
void orc_fft2(cplx *a, int N, int sign)
{
    for (int r = 0; r < N; r++) orc_fft1d(a + (long)r * N, N, 1, sign);
    for (int c = 0; c < N; c++) orc_fft1d(a + c, N, N, sign);
    if (sign > 0) {
        double s = 1.0 / ((double)N * (double)N);
        for (long i = 0; i < (long)N * N; i++) a[i] *= s;
    }
}

/* Brute-force 2D DFT (test pin for orc_fft2). out may not alias in. */
void orc_dft2(const cplx *in, cplx *out, int N, int sign)
{
    for (int ky = 0; ky < N; ky++)
        for (int kx = 0; kx < N; kx++) {
            cplx s = 0;
            for (int y = 0; y < N; y++)
                for (int x = 0; x < N; x++) {
                    double ang = sign * 2.0 * M_PI *
                                 ((double)((long)kx * x % N) + (double)((long)ky * y % N)) / N;
                    s += in[(long)y * N + x] * (cos(ang) + I * sin(ang));
                }
            out[(long)ky * N + kx] = s;
        }
}

/* ------------------------------------------------------------------------- */
/* the regularised tilted double well, eq. (e:Wq-def), Sec. 2.1               */
/* ------------------------------------------------------------------------- */
/* W_q(u) = A(u) B(u),
 *   A = (u-b_-)^2/2 + q eps (1 - sech((u-b_-)/eps)),
 *   B = (u-b_+)^2/2 + gamma/3 (u - (3 b_+ - b_-)/2).
 * Derivatives by the product rule. With well = 1 the oracle instead uses the
 * quadratic test well alpha/2 (u-b_-)^2 with alpha = W_q''(b_-) (a test device,
 * not part of the paper's model). */
void orc_well(const orc_params *p, double u, double *W, double *W1, double *W2)
{
    double v = u - p->b_minus;
    if (p->well == 1) {
        double alpha = (1.0 + p->q / p->eps) *
                       (0.5 * (p->b_minus - p->b_plus) * (p->b_minus - p->b_plus) +
                        p->gamma / 3.0 * (p->b_minus - 0.5 * (3.0 * p->b_plus - p->b_minus)));
        *W = 0.5 * alpha * v * v;
        *W1 = alpha * v;
        *W2 = alpha;
        return;
    }
    double x = v / p->eps;
    double sech = fabs(x) > 700.0 ? 0.0 : 1.0 / cosh(x);
    double th = tanh(x);
    double A = 0.5 * v * v + p->q * p->eps * (1.0 - sech);
    double A1 = v + p->q * sech * th;
    double A2 = 1.0 + (p->q / p->eps) * sech * (2.0 * sech * sech - 1.0);
    double w = u - p->b_plus;
    double B = 0.5 * w * w + p->gamma / 3.0 * (u - 0.5 * (3.0 * p->b_plus - p->b_minus));
    double B1 = w + p->gamma / 3.0;
    double B2 = 1.0;
    *W = A * B;
    *W1 = A1 * B + A * B1;
    *W2 = A2 * B + 2.0 * A1 * B1 + A * B2;
}

/* alpha_m = W_q''(b_-), Sec. 3.3 / Table t:Benchmark */
double orc_alpha_m(const orc_params *p)
{
    double W, W1, W2;
    orc_well(p, p->b_minus, &W, &W1, &W2);
    return W2;
}

/* ------------------------------------------------------------------------- */
/* grid, symbols and spectral helpers                                         */
/* ------------------------------------------------------------------------- */
typedef struct {
    int N;
    double L;
    double *k2; /* |k|^2 on the full N x N grid, row index ky, column index kx */
} grid_t;

static double wavenumber(int N, double L, int j)
{
    int m = j < N / 2 ? j : j - N; /* m in [-N/2, N/2-1] */
    return 2.0 * M_PI * (double)m / L;
}

static void grid_init(grid_t *g, int N, double L)
{
    g->N = N;
    g->L = L;
    g->k2 = malloc(sizeof(double) * N * N);
    for (int ky = 0; ky < N; ky++)
        for (int kx = 0; kx < N; kx++) {
            double a = wavenumber(N, L, kx), b = wavenumber(N, L, ky);
            g->k2[(long)ky * N + kx] = a * a + b * b;
        }
}

static long npts(const grid_t *g) { return (long)g->N * g->N; }
static double h2(const grid_t *g) { return (g->L / g->N) * (g->L / g->N); }

static void to_spec(const grid_t *g, const double *f, cplx *fh)
{
    for (long i = 0; i < npts(g); i++) fh[i] = f[i];
    orc_fft2(fh, g->N, -1);
}

static void to_real(const grid_t *g, const cplx *fh, double *f, cplx *work)
{
    memcpy(work, fh, sizeof(cplx) * npts(g));
    orc_fft2(work, g->N, +1);
    for (long i = 0; i < npts(g); i++) f[i] = creal(work[i]);
}

/* real-space Laplacian through the symbol -|k|^2 */
static void lap_real(const grid_t *g, const double *f, double *out, cplx *w1, cplx *w2)
{
    to_spec(g, f, w1);
    for (long i = 0; i < npts(g); i++) w1[i] *= -g->k2[i];
    to_real(g, w1, out, w2);
}

static double inner(const grid_t *g, const double *f, const double *q)
{
    double s = 0;
    for (long i = 0; i < npts(g); i++) s += f[i] * q[i];
    return h2(g) * s;
}

/* ------------------------------------------------------------------------- */
/* energy, mass, chemical potential                                           */
/* ------------------------------------------------------------------------- */
/* E(u) = int 1/2 (eps^2 Lap u - W')^2 - (eps^2 eta1/2 |grad u|^2 + eta2 W), eq. (Functional) */
double orc_energy(const orc_params *p, int N, double L, const double *u)
{
    grid_t g;
    grid_init(&g, N, L);
    long n = npts(&g);
    double *lu = malloc(sizeof(double) * n);
    cplx *w1 = malloc(sizeof(cplx) * n), *w2 = malloc(sizeof(cplx) * n);
    lap_real(&g, u, lu, w1, w2);
    double s = 0;
    for (long i = 0; i < n; i++) {
        double W, W1, W2;
        orc_well(p, u[i], &W, &W1, &W2);
        double w = p->eps * p->eps * lu[i] - W1;
        s += 0.5 * w * w - p->eta2 * W;
    }
    double E = h2(&g) * s;
    /* int |grad u|^2 = -(u, Lap u) */
    double grad2 = -inner(&g, u, lu);
    E -= 0.5 * p->eps * p->eps * p->eta1 * grad2;
    free(lu); free(w1); free(w2); free(g.k2);
    return E;
}

/* m = 1/2 int (u + 1) dx, Sec. 2.3 */
double orc_mass(int N, double L, const double *u)
{
    double s = 0;
    for (long i = 0; i < (long)N * N; i++) s += u[i] + 1.0;
    return 0.5 * (L / N) * (L / N) * s;
}

/* mu = dE/du = (eps^2 Lap - W'')(eps^2 Lap u - W') + eps^2 eta1 Lap u - eta2 W', eq. (FCH) */
static void mu_real(const grid_t *g, const orc_params *p, const double *u, double *mu,
                    double *lu, double *w, double *lw, cplx *c1, cplx *c2)
{
    long n = npts(g);
    double e2 = p->eps * p->eps;
    lap_real(g, u, lu, c1, c2);
    for (long i = 0; i < n; i++) {
        double W, W1, W2;
        orc_well(p, u[i], &W, &W1, &W2);
        w[i] = e2 * lu[i] - W1;
    }
    lap_real(g, w, lw, c1, c2);
    for (long i = 0; i < n; i++) {
        double W, W1, W2;
        orc_well(p, u[i], &W, &W1, &W2);
        mu[i] = e2 * lw[i] - W2 * w[i] + e2 * p->eta1 * lu[i] - p->eta2 * W1;
    }
}

/* public: mu(u) and F(u) = Lap mu (eq. sFCH) on a real grid function */
void orc_mu(const orc_params *p, int N, double L, const double *u, double *mu)
{
    grid_t g;
    grid_init(&g, N, L);
    long n = npts(&g);
    double *lu = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n),
           *lw = malloc(sizeof(double) * n);
    cplx *c1 = malloc(sizeof(cplx) * n), *c2 = malloc(sizeof(cplx) * n);
    mu_real(&g, p, u, mu, lu, w, lw, c1, c2);
    free(lu); free(w); free(lw); free(c1); free(c2); free(g.k2);
}

void orc_rhs(const orc_params *p, int N, double L, const double *u, double *F)
{
    grid_t g;
    grid_init(&g, N, L);
    long n = npts(&g);
    double *mu = malloc(sizeof(double) * n);
    double *lu = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n),
           *lw = malloc(sizeof(double) * n);
    cplx *c1 = malloc(sizeof(cplx) * n), *c2 = malloc(sizeof(cplx) * n);
    mu_real(&g, p, u, mu, lu, w, lw, c1, c2);
    lap_real(&g, mu, F, c1, c2);
    free(mu); free(lu); free(w); free(lw); free(c1); free(c2); free(g.k2);
}

/* N_IMEX(u) = eps^2 (alpha_m - W'') Lap u + eps^2 Lap(alpha_m u - W') + W'' W'
 *             - alpha_m^2 u + eps^2 eta1 Lap u - eta2 W',            Sec. 3.4 */
static void n_imex_real(const grid_t *g, const orc_params *p, double am, const double *u,
                        double *out, double *lu, double *t1, double *t2, cplx *c1, cplx *c2)
{
    long n = npts(g);
    double e2 = p->eps * p->eps;
    lap_real(g, u, lu, c1, c2);
    for (long i = 0; i < n; i++) {
        double W, W1, W2;
        orc_well(p, u[i], &W, &W1, &W2);
        t1[i] = am * u[i] - W1;
    }
    lap_real(g, t1, t2, c1, c2);
    for (long i = 0; i < n; i++) {
        double W, W1, W2;
        orc_well(p, u[i], &W, &W1, &W2);
        out[i] = e2 * (am - W2) * lu[i] + e2 * t2[i] + W2 * W1 - am * am * u[i] +
                 e2 * p->eta1 * lu[i] - p->eta2 * W1;
    }
}

void orc_n_imex(const orc_params *p, int N, double L, const double *u, double *out)
{
    grid_t g;
    grid_init(&g, N, L);
    long n = npts(&g);
    double *lu = malloc(sizeof(double) * n), *t1 = malloc(sizeof(double) * n),
           *t2 = malloc(sizeof(double) * n);
    cplx *c1 = malloc(sizeof(cplx) * n), *c2 = malloc(sizeof(cplx) * n);
    n_imex_real(&g, p, orc_alpha_m(p), u, out, lu, t1, t2, c1, c2);
    free(lu); free(t1); free(t2); free(c1); free(c2); free(g.k2);
}

/* SAV pieces, Sec. 3.5:
 * G(u) = -eps^2 Lap u (W' + zeta u) + W'^2/2 - eta2 W               eq. (e:G-def)
 * V[u] = dE1/du = -eps^2 Lap(W' + zeta u) - eps^2 (W'' + zeta) Lap u + W' W'' - eta2 W'
 * E1(u) = int G(u)                                                     */
static double e1_and_v(const grid_t *g, const orc_params *p, const double *u, double *V,
                       double *lu, double *t1, double *t2, cplx *c1, cplx *c2)
{
    long n = npts(g);
    double e2 = p->eps * p->eps, s = 0;
    lap_real(g, u, lu, c1, c2);
    for (long i = 0; i < n; i++) {
        double W, W1, W2;
        orc_well(p, u[i], &W, &W1, &W2);
        s += -e2 * lu[i] * (W1 + p->zeta * u[i]) + 0.5 * W1 * W1 - p->eta2 * W;
        t1[i] = W1 + p->zeta * u[i];
    }
    if (V) {
        lap_real(g, t1, t2, c1, c2);
        for (long i = 0; i < n; i++) {
            double W, W1, W2;
            orc_well(p, u[i], &W, &W1, &W2);
            V[i] = -e2 * t2[i] - e2 * (W2 + p->zeta) * lu[i] + W1 * W2 - p->eta2 * W1;
        }
    }
    return h2(g) * s;
}

double orc_sav_e1(const orc_params *p, int N, double L, const double *u, double *V)
{
    grid_t g;
    grid_init(&g, N, L);
    long n = npts(&g);
    double *lu = malloc(sizeof(double) * n), *t1 = malloc(sizeof(double) * n),
           *t2 = malloc(sizeof(double) * n);
    cplx *c1 = malloc(sizeof(cplx) * n), *c2 = malloc(sizeof(cplx) * n);
    double E1 = e1_and_v(&g, p, u, V, lu, t1, t2, c1, c2);
    free(lu); free(t1); free(t2); free(c1); free(c2); free(g.k2);
    return E1;
}

/* ------------------------------------------------------------------------- */
/* BDF2 / AM3 coefficients, Sec. 3.1                                          */
/* ------------------------------------------------------------------------- */
/* eq. (BDF2Coef); kn <= 0 selects backward Euler (reading R1) */
void orc_bdf2_coef(double k1, double kn, double *a, double *b, double *c)
{
    if (kn <= 0) {
        *a = 1.0 / k1;
        *b = -1.0 / k1;
        *c = 0.0;
        return;
    }
    *a = 1.0 / k1 + 1.0 / (k1 + kn);
    *b = -1.0 / k1 - 1.0 / kn;
    *c = 1.0 / kn - 1.0 / (k1 + kn);
}

/* eq. (AM3-general): weights of F(u^{n+1}), F(u^n), F(u^{n-1}) */
void orc_am3_coef(double k1, double kn, double *w1, double *w2, double *w3)
{
    double g = k1 / kn;
    *w1 = k1 / 6.0 * (3.0 + 2.0 * g) / (1.0 + g);
    *w2 = k1 / 6.0 * (3.0 + g);
    *w3 = -k1 / 6.0 * g * g / (1.0 + g);
}

/* ------------------------------------------------------------------------- */
/* stepper state                                                              */
/* ------------------------------------------------------------------------- */
enum { ORC_IMEX = 0, ORC_SAV = 1, ORC_PSD = 2, ORC_ETD = 3 };

typedef struct {
    grid_t g;
    orc_params p;
    double am;           /* alpha_m */
    double *u, *um;      /* u^n, u^{n-1} (real space) */
    double *Fn, *Fm;     /* F(u^n), F(u^{n-1}) (real space) */
    double r, rm;        /* SAV r^n, r^{n-1} */
    double t, kn;        /* time, last accepted step size (0: no history) */
    int have_F;
    long n_steps, n_rejects, n_psd_iter, n_attempts;
    int last_psd_iter;
    double last_e;
    /* adaptive runs, Sec. 3.2: the next trial size (Step 0 / Step 4), the size and
     * the decision of the last trial, and the open run's scheme, sigma_tol, t_final */
    double ktrial, last_k;
    int last_accepted;
    int ad_scheme;
    double ad_sigma, ad_tfinal;
    const double *ustar_given; /* a caller's u* for the next step (orc_step_from), else NULL */
    /* work */
    double *w[10];
    cplx *c1, *c2, *c3, *c4;
} orc_ctx;

orc_ctx *orc_create(int N, double L, const orc_params *p)
{
    orc_ctx *s = calloc(1, sizeof(orc_ctx));
    grid_init(&s->g, N, L);
    s->p = *p;
    s->am = orc_alpha_m(p);
    long n = npts(&s->g);
    s->u = calloc(n, sizeof(double));
    s->um = calloc(n, sizeof(double));
    s->Fn = calloc(n, sizeof(double));
    s->Fm = calloc(n, sizeof(double));
    for (int i = 0; i < 10; i++) s->w[i] = calloc(n, sizeof(double));
    s->c1 = calloc(n, sizeof(cplx));
    s->c2 = calloc(n, sizeof(cplx));
    s->c3 = calloc(n, sizeof(cplx));
    s->c4 = calloc(n, sizeof(cplx));
    return s;
}

void orc_destroy(orc_ctx *s)
{
    if (!s) return;
    free(s->u); free(s->um); free(s->Fn); free(s->Fm);
    for (int i = 0; i < 10; i++) free(s->w[i]);
    free(s->c1); free(s->c2); free(s->c3); free(s->c4); free(s->g.k2);
    free(s);
}

static double sav_r_of(orc_ctx *s, const double *u)
{
    return sqrt(e1_and_v(&s->g, &s->p, u, NULL, s->w[7], s->w[8], s->w[9], s->c1, s->c2) +
                s->p.D0);
}

/* sets u^0; clears the history so the next step is a backward-Euler start */
void orc_set_state(orc_ctx *s, const double *u0)
{
    long n = npts(&s->g);
    memcpy(s->u, u0, sizeof(double) * n);
    memset(s->um, 0, sizeof(double) * n);
    s->kn = 0;
    s->ktrial = 0;
    s->t = 0;
    s->have_F = 0;
    s->r = sav_r_of(s, s->u);
    s->rm = 0;
    s->n_steps = s->n_rejects = s->n_psd_iter = s->n_attempts = 0;
}

/* sets (u^n, u^{n-1}, k_n) so the next step is a full variable-step BDF2 step.
 * The SAV variables take their consistent values r = sqrt(E1(u) + D0). */
void orc_set_history(orc_ctx *s, const double *un, const double *unm1, double kn)
{
    long n = npts(&s->g);
    memcpy(s->u, un, sizeof(double) * n);
    memcpy(s->um, unm1, sizeof(double) * n);
    s->kn = kn;
    s->ktrial = kn; /* Step 0: the first trial repeats k_n */
    s->have_F = 0;
    s->r = sav_r_of(s, s->u);
    s->rm = sav_r_of(s, s->um);
}

void orc_get_state(const orc_ctx *s, double *u) { memcpy(u, s->u, sizeof(double) * npts(&s->g)); }
void orc_get_prev(const orc_ctx *s, double *u) { memcpy(u, s->um, sizeof(double) * npts(&s->g)); }
double orc_get_time(const orc_ctx *s) { return s->t; }
double orc_get_r(const orc_ctx *s, int which) { return which ? s->rm : s->r; }
double orc_get_kn(const orc_ctx *s) { return s->kn; }
void orc_get_counts(const orc_ctx *s, long *out)
{
    out[0] = s->n_steps;
    out[1] = s->n_rejects;
    out[2] = s->n_psd_iter;
    out[3] = s->n_attempts;
    out[4] = s->last_psd_iter;
}
double orc_get_last_e(const orc_ctx *s) { return s->last_e; }
/* size of the last trial step, its decision (1 accepted), and the next trial size */
double orc_get_last_k(const orc_ctx *s) { return s->last_k; }
int orc_get_last_accepted(const orc_ctx *s) { return s->last_accepted; }
double orc_get_next_k(const orc_ctx *s) { return s->ktrial; }

/* u* = u^n + (k_{n+1}/k_n)(u^n - u^{n-1}), eq. (Richardson); u* = u^n at the start.
 * A u* given by orc_step_from replaces the extrapolation: eqs. (IMEX-eq) and
 * (4.7)-(4.8) take u* as an input like u^n and u^{n-1}. */
static void extrapolate(const orc_ctx *s, double k1, double *ustar)
{
    long n = npts(&s->g);
    if (s->ustar_given) {
        memcpy(ustar, s->ustar_given, sizeof(double) * n);
        return;
    }
    if (s->kn <= 0) {
        memcpy(ustar, s->u, sizeof(double) * n);
        return;
    }
    double gam = k1 / s->kn;
    for (long i = 0; i < n; i++) ustar[i] = s->u[i] + gam * (s->u[i] - s->um[i]);
}

/* symbol of L_IMEX = eps^4 Lap^2 - 2 alpha_m eps^2 Lap + alpha_m^2, eq. (e:IMEX-op) */
static double sym_limex(const orc_ctx *s, double k2)
{
    double e2 = s->p.eps * s->p.eps;
    return e2 * e2 * k2 * k2 + 2.0 * s->am * e2 * k2 + s->am * s->am;
}

/* BDF2-IMEX, eq. (IMEX-eq): (a - Lap L_IMEX) u^{n+1} = -b u^n - c u^{n-1} + Lap N_IMEX(u*) */
static void step_imex(orc_ctx *s, double k1, double *out)
{
    long n = npts(&s->g);
    double a, b, c;
    orc_bdf2_coef(k1, s->kn, &a, &b, &c);
    double *ustar = s->w[0], *nn = s->w[1];
    extrapolate(s, k1, ustar);
    n_imex_real(&s->g, &s->p, s->am, ustar, nn, s->w[2], s->w[3], s->w[4], s->c1, s->c2);
    cplx *uh = s->c3, *umh = s->c4, *nh = s->c1;
    to_spec(&s->g, s->u, uh);
    to_spec(&s->g, s->um, umh);
    to_spec(&s->g, nn, nh);
    for (long i = 0; i < n; i++) {
        double k2 = s->g.k2[i];
        nh[i] = (-b * uh[i] - c * umh[i] - k2 * nh[i]) / (a + k2 * sym_limex(s, k2));
    }
    to_real(&s->g, nh, out, s->c2);
}

/* BDF2-SAV, eqs. (4.7)-(4.8), solved by the p/q split (reading R10):
 *   (a - Lap L0) p = -b u^n - c u^{n-1} + Lap L1 u*,
 *   (a - Lap L0) q = Lap X,   X = V[u*] / sqrt(E1(u*) + D0),
 *   r^{n+1} = [-b r^n - c r^{n-1} + (X, a p + b u^n + c u^{n-1})/2] / (a (1 - (X, q)/2)),
 *   u^{n+1} = p + r^{n+1} q.                                               */
static void step_sav(orc_ctx *s, double k1, double *out, double *r_out)
{
    long n = npts(&s->g);
    double a, b, c;
    orc_bdf2_coef(k1, s->kn, &a, &b, &c);
    double e2 = s->p.eps * s->p.eps, am = s->am;
    double *ustar = s->w[0], *X = s->w[1], *pr = s->w[5], *qr = s->w[6];
    extrapolate(s, k1, ustar);
    double E1 = e1_and_v(&s->g, &s->p, ustar, X, s->w[2], s->w[3], s->w[4], s->c1, s->c2);
    double sq = sqrt(E1 + s->p.D0);
    for (long i = 0; i < n; i++) X[i] /= sq;
    cplx *ph = s->c1, *qh = s->c2, *uh = s->c3, *umh = s->c4;
    to_spec(&s->g, ustar, ph);
    to_spec(&s->g, X, qh);
    to_spec(&s->g, s->u, uh);
    to_spec(&s->g, s->um, umh);
    for (long i = 0; i < n; i++) {
        double k2 = s->g.k2[i];
        double l0 = e2 * e2 * k2 * k2 + s->p.beta1 * am * e2 * k2 + s->p.beta2 * am * am;
        double l1 = -e2 * (s->p.eta1 + 2.0 * s->p.zeta) * k2 - s->p.beta1 * am * e2 * k2 -
                    s->p.beta2 * am * am;
        double den = a + k2 * l0;
        ph[i] = (-b * uh[i] - c * umh[i] - k2 * l1 * ph[i]) / den;
        qh[i] = (-k2 * qh[i]) / den;
    }
    cplx *tmp = s->c3;
    to_real(&s->g, ph, pr, tmp);
    to_real(&s->g, qh, qr, tmp);
    double *rhs = s->w[2];
    for (long i = 0; i < n; i++) rhs[i] = a * pr[i] + b * s->u[i] + c * s->um[i];
    double xr = inner(&s->g, X, rhs), xq = inner(&s->g, X, qr);
    double rn1 = (-b * s->r - c * s->rm + 0.5 * xr) / (a * (1.0 - 0.5 * xq));
    for (long i = 0; i < n; i++) out[i] = pr[i] + rn1 * qr[i];
    *r_out = rn1;
}

/* Table SearchSize: optimal PSD search step lambda(k) for q = 0, 0.2, 0.5 (reading R8) */
static const double lam_k[10] = {1e-6, 1e-5, 5e-5, 1e-4, 5e-4, 1e-3, 5e-3, 1e-2, 2e-2, 3e-2};
static const double lam_tab[3][10] = {
    {1, 1.07, 1.11, 1.14, 1.24, 1.34, 1.60, 1.738, 1.804, 1.855},
    {1, 1.04, 1.15, 1.28, 1.50, 1.70, 1.87, 1.92, 1.95, 1.97},
    {1, 1.20, 1.32, 1.45, 1.72, 1.83, 1.965, 1.97, 1.985, 1.99},
};

double orc_psd_lambda(const orc_params *p, double k)
{
    if (p->psd_lambda > 0) return p->psd_lambda;
    int row = fabs(p->q) < 1e-12 ? 0 : (fabs(p->q - 0.2) < 1e-12 ? 1 : 2);
    if (k <= lam_k[0]) return lam_tab[row][0];
    if (k >= lam_k[9]) return lam_tab[row][9];
    for (int j = 0; j < 9; j++)
        if (k <= lam_k[j + 1]) {
            double th = (k - lam_k[j]) / (lam_k[j + 1] - lam_k[j]);
            return lam_tab[row][j] + th * (lam_tab[row][j + 1] - lam_tab[row][j]);
        }
    return lam_tab[row][9];
}

/* BDF2-PSD, Sec. 3.3:
 *   R(v) = Pi0 mu(v) - Lap^{-1}(a v) - Lap^{-1}(b u^n + c u^{n-1}),     eq. (residual)
 *   d = -L_PSD^{-1} R,  L_PSD = L_IMEX - a Lap^{-1},
 *   v_0 = u*,  v_{s+1} = v_s + lambda d_s,                              eq. (recurrence)
 *   stop when ||d_s|| / ||v_{s+1}|| < i_tol.  Returns 0, or -1 when max_iter is reached. */
static int step_psd(orc_ctx *s, double k1, double itol, double *out, int *iters)
{
    long n = npts(&s->g);
    double a, b, c;
    orc_bdf2_coef(k1, s->kn, &a, &b, &c);
    double lam = orc_psd_lambda(&s->p, k1);
    double *v = s->w[0], *mu = s->w[1], *d = s->w[5];
    extrapolate(s, k1, v);
    cplx *uh = s->c3, *umh = s->c4;
    to_spec(&s->g, s->u, uh);
    to_spec(&s->g, s->um, umh);
    for (int it = 1; it <= s->p.psd_max_iter; it++) {
        mu_real(&s->g, &s->p, v, mu, s->w[2], s->w[3], s->w[4], s->c1, s->c2);
        cplx *muh = s->c1, *vh = s->c2;
        to_spec(&s->g, mu, muh);
        to_spec(&s->g, v, vh);
        for (long i = 0; i < n; i++) {
            double k2 = s->g.k2[i];
            if (k2 == 0.0) {
                muh[i] = 0; /* Pi0 and Lap^{-1} act on the zero-mass part only */
                continue;
            }
            cplx R = muh[i] + (a * vh[i] + b * uh[i] + c * umh[i]) / k2;
            muh[i] = -R / (sym_limex(s, k2) + a / k2);
        }
        to_real(&s->g, muh, d, s->c2);
        for (long i = 0; i < n; i++) v[i] += lam * d[i];
        double nd = sqrt(inner(&s->g, d, d)), nv = sqrt(inner(&s->g, v, v));
        if (nd / nv < itol) {
            *iters = it;
            memcpy(out, v, sizeof(double) * n);
            return 0;
        }
    }
    *iters = s->p.psd_max_iter;
    memcpy(out, v, sizeof(double) * n);
    return -1;
}

/* ETD phi functions (reading R9): phi1 = (e^z - 1)/z, phi2 = (e^z - 1 - z)/z^2 */
void orc_phi(double z, double *e, double *p1, double *p2)
{
    *e = exp(z);
    if (fabs(z) < 1e-2) {
        /* Taylor series: phi1 = sum z^j/(j+1)!, phi2 = sum z^j/(j+2)! */
        double t1 = 1, t2 = 0.5, s1 = 0, s2 = 0;
        for (int j = 0; j < 12; j++) {
            s1 += t1;
            s2 += t2;
            t1 *= z / (j + 2);
            t2 *= z / (j + 3);
        }
        *p1 = s1;
        *p2 = s2;
    } else {
        *p1 = expm1(z) / z;
        *p2 = (expm1(z) - z) / (z * z);
    }
}

/* ETDRK2, eqs. (ETDRK2), (ETD-L):
 *   L = Lap L_IMEX - kappa0 I + kappa2 eps^2 Lap,  N(u) = Lap N_IMEX(u) + kappa0 u - kappa2 eps^2 Lap u,
 *   ut = e^{Lk} u^n + k phi1(Lk) N(u^n),  u^{n+1} = ut + k phi2(Lk) (N(ut) - N(u^n)). */
static void etd_nhat(orc_ctx *s, const double *u, cplx *out)
{
    long n = npts(&s->g);
    double e2 = s->p.eps * s->p.eps;
    double *nn = s->w[1];
    n_imex_real(&s->g, &s->p, s->am, u, nn, s->w[2], s->w[3], s->w[4], s->c1, s->c2);
    cplx *uh = s->c1;
    to_spec(&s->g, u, uh);
    to_spec(&s->g, nn, out);
    for (long i = 0; i < n; i++) {
        double k2 = s->g.k2[i];
        out[i] = -k2 * out[i] + s->p.kappa0 * uh[i] + s->p.kappa2 * e2 * k2 * uh[i];
    }
}

static void step_etd(orc_ctx *s, double k1, double *out)
{
    long n = npts(&s->g);
    double e2 = s->p.eps * s->p.eps;
    cplx *n0 = s->c3, *uh = s->c4;
    etd_nhat(s, s->u, n0);
    to_spec(&s->g, s->u, uh);
    for (long i = 0; i < n; i++) {
        double k2 = s->g.k2[i];
        double ell = -k2 * sym_limex(s, k2) - s->p.kappa0 - s->p.kappa2 * e2 * k2;
        double ez, p1, p2;
        orc_phi(ell * k1, &ez, &p1, &p2);
        uh[i] = ez * uh[i] + k1 * p1 * n0[i];
    }
    double *ut = s->w[0];
    to_real(&s->g, uh, ut, s->c1);
    cplx *n1 = s->c2;
    /* etd_nhat uses c1 as scratch and writes into its out argument */
    {
        double *nn = s->w[1];
        n_imex_real(&s->g, &s->p, s->am, ut, nn, s->w[2], s->w[3], s->w[4], s->c1, s->c2);
        to_spec(&s->g, nn, n1);
        cplx *uth = s->c1;
        to_spec(&s->g, ut, uth);
        for (long i = 0; i < n; i++) {
            double k2 = s->g.k2[i];
            n1[i] = -k2 * n1[i] + s->p.kappa0 * uth[i] + s->p.kappa2 * e2 * k2 * uth[i];
        }
    }
    to_spec(&s->g, ut, uh);
    for (long i = 0; i < n; i++) {
        double k2 = s->g.k2[i];
        double ell = -k2 * sym_limex(s, k2) - s->p.kappa0 - s->p.kappa2 * e2 * k2;
        double ez, p1, p2;
        orc_phi(ell * k1, &ez, &p1, &p2);
        uh[i] = uh[i] + k1 * p2 * (n1[i] - n0[i]);
    }
    to_real(&s->g, uh, out, s->c1);
}

/* one trial step of size k1 from the current history into out. Returns 0, or -1
 * when the PSD iteration did not converge. */
static int trial(orc_ctx *s, int scheme, double k1, double itol, double *out, double *r_out)
{
    int it = 0;
    *r_out = s->r;
    switch (scheme) {
    case ORC_IMEX: step_imex(s, k1, out); return 0;
    case ORC_SAV: step_sav(s, k1, out, r_out); return 0;
    case ORC_PSD: {
        int rc = step_psd(s, k1, itol, out, &it);
        s->last_psd_iter = it;
        s->n_psd_iter += it;
        return rc;
    }
    case ORC_ETD: step_etd(s, k1, out); return 0;
    }
    return -2;
}

static void accept(orc_ctx *s, const double *unew, double rnew, double k1)
{
    long n = npts(&s->g);
    memcpy(s->um, s->u, sizeof(double) * n);
    memcpy(s->u, unew, sizeof(double) * n);
    s->rm = s->r;
    s->r = rnew;
    s->kn = k1;
    s->ktrial = k1; /* Step 0: the next step's first trial repeats k_n */
    s->t += k1;
    s->n_steps++;
}

int orc_step(orc_ctx *s, int scheme, double dt);

/* one fixed IMEX or SAV step whose extrapolation u* is the given field (real
 * space, N x N) instead of eq. (Richardson); otherwise as orc_step */
int orc_step_from(orc_ctx *s, int scheme, double dt, const double *ustar)
{
    if (scheme != ORC_IMEX && scheme != ORC_SAV) return -2;
    s->ustar_given = ustar;
    int rc = orc_step(s, scheme, dt);
    s->ustar_given = NULL;
    return rc;
}

/* fixed step of size dt (first step after orc_set_state is backward Euler) */
int orc_step(orc_ctx *s, int scheme, double dt)
{
    double *out = s->w[9]; /* w[7..9] are free during a trial */
    double rnew;
    int rc = trial(s, scheme, dt, s->p.psd_itol, out, &rnew);
    if (rc) return rc;
    accept(s, out, rnew, dt);
    s->have_F = 0;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* adaptive time stepping, Sec. 3.2                                           */
/* ------------------------------------------------------------------------- */
static double a_dp(const orc_params *p, double sigma, double e, double k)
{
    double ee = e > 1e-16 ? e : 1e-16; /* reading R3 */
    double kn = p->rho_s * cbrt(sigma / ee) * k;
    if (p->zero_stab_cap && kn > (1.0 + sqrt(2.0)) * k) kn = (1.0 + sqrt(2.0)) * k;
    return kn;
}

static double clampk(const orc_params *p, double k)
{
    double kk = k < p->k_max ? k : p->k_max;
    return kk > p->k_min ? kk : p->k_min;
}

/* Set-up of an adaptive run, Sec. 3.2: the first step k_1 = k_min by the
 * backward-Euler start when there is no history (reading R1), and the F history
 * F(u^n), F(u^{n-1}) the predictor needs. The run continues from the current trial
 * size (Step 0 after a fixed step or a new history; the last proposal of Step 4
 * when a run is resumed). Returns 0, or -1 when the PSD iteration failed. */
int orc_adaptive_begin(orc_ctx *s, int scheme, double sigma, double t_final)
{
    long n = npts(&s->g);
    double itol = s->p.psd_nu * sigma;
    double *ut = s->w[9];
    double rnew;
    s->ad_scheme = scheme;
    s->ad_sigma = sigma;
    s->ad_tfinal = t_final;
    if (s->kn <= 0) {
        double k1 = s->p.k_min;
        orc_rhs(&s->p, s->g.N, s->g.L, s->u, s->Fn);
        int rc = trial(s, scheme, k1, itol, ut, &rnew);
        s->n_attempts++;
        if (rc) return rc;
        memcpy(s->Fm, s->Fn, sizeof(double) * n);
        accept(s, ut, rnew, k1);
        orc_rhs(&s->p, s->g.N, s->g.L, s->u, s->Fn);
        s->have_F = 1;
    } else if (!s->have_F) {
        orc_rhs(&s->p, s->g.N, s->g.L, s->u, s->Fn);
        orc_rhs(&s->p, s->g.N, s->g.L, s->um, s->Fm);
        s->have_F = 1;
    }
    return 0;
}

/* One pass through Steps 1-4 of the adaptive algorithm of Sec. 3.2 for the run
 * opened by orc_adaptive_begin: the trial of size k~ (clipped to t_final, reading
 * R4), the AM3 predictor of eq. (Predictor), e = ||ut - u_p|| / ||u_p|| (reading R6),
 * and the decision: accept when e <= sigma_tol or k~ <= k_min (reading R5); either
 * way the next trial size is max(k_min, min(A_dp(e, k~), k_max)) (reading R2).
 * Returns 0 after a trial, 2 when t_final is reached (no trial), -1 when the PSD
 * iteration did not converge. */
int orc_adaptive_trial(orc_ctx *s)
{
    long n = npts(&s->g);
    const double sigma = s->ad_sigma, t_final = s->ad_tfinal;
    double itol = s->p.psd_nu * sigma;
    double *ut = s->w[9], *up = s->w[8], *Ft = s->w[7];
    double rnew;
    if (!(t_final - s->t > 1e-12 * (t_final > 1 ? t_final : 1))) return 2;
    double k1 = s->ktrial;
    if (k1 > t_final - s->t) k1 = t_final - s->t; /* reading R4 */
    s->last_k = k1;
    int rc = trial(s, s->ad_scheme, k1, itol, ut, &rnew); /* Step 1 */
    s->n_attempts++;
    if (rc) return rc;
    /* Step 2: AM3 predictor */
    orc_rhs(&s->p, s->g.N, s->g.L, ut, Ft);
    double w1, w2, w3;
    orc_am3_coef(k1, s->kn, &w1, &w2, &w3);
    for (long i = 0; i < n; i++) up[i] = s->u[i] + w1 * Ft[i] + w2 * s->Fn[i] + w3 * s->Fm[i];
    /* Step 3: relative error (reading R6) */
    double num = 0, den = 0;
    for (long i = 0; i < n; i++) {
        num += (ut[i] - up[i]) * (ut[i] - up[i]);
        den += up[i] * up[i];
    }
    double e = sqrt(num) / sqrt(den);
    s->last_e = e;
    double knew = clampk(&s->p, a_dp(&s->p, sigma, e, k1));
    /* Step 4 */
    if (e <= sigma || k1 <= s->p.k_min) {
        accept(s, ut, rnew, k1);
        memcpy(s->Fm, s->Fn, sizeof(double) * n);
        memcpy(s->Fn, Ft, sizeof(double) * n);
        s->last_accepted = 1;
    } else {
        s->n_rejects++;
        s->last_accepted = 0;
    }
    s->ktrial = knew;
    return 0;
}

/* One trial of the open adaptive run (as orc_adaptive_trial) whose extrapolation is
 * the given field (real space, N x N) instead of eq. (Richardson): the explicit part
 * of IMEX and SAV (eqs. (IMEX-eq), (4.7)-(4.8)), or the first PSD iterate v_0
 * (Sec. 3.3). Returns as orc_adaptive_trial, or -2 for ETD. */
int orc_adaptive_trial_from(orc_ctx *s, const double *ustar)
{
    if (s->ad_scheme == ORC_ETD) return -2;
    s->ustar_given = ustar;
    int rc = orc_adaptive_trial(s);
    s->ustar_given = NULL;
    return rc;
}

/* The adaptive algorithm of Sec. 3.2, Steps 0-4 (orc_adaptive_begin, then
 * orc_adaptive_trial until t_final or max_attempts trial steps).
 * Returns 0, -1 (PSD did not converge), or 1 (attempt budget used up). */
int orc_run_adaptive(orc_ctx *s, int scheme, double sigma, double t_final, long max_attempts)
{
    int rc = orc_adaptive_begin(s, scheme, sigma, t_final);
    if (rc) return rc;
    for (long attempts = 0;; attempts++) {
        if (!(t_final - s->t > 1e-12 * (t_final > 1 ? t_final : 1))) return 0;
        if (attempts >= max_attempts) return 1;
        rc = orc_adaptive_trial(s);
        if (rc == 2) return 0;
        if (rc) return rc;
    }
}
