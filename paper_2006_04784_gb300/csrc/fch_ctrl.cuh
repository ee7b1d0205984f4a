// fch_ctrl.cuh -- the device-side control logic of the adaptive steppers:
// FP64 reductions of per-block partial sums, the step-size controller of
// Sec. 3.2, the SAV scalar update and the PSD stopping test. Run either by the
// single-block control kernel or by the last block of the pass that produced
// the partial sums.
#pragma once
#include <math.h>
#include <stddef.h>
#include "fch_internal.h"
#include "../../include/fch.h"

// Programmatic dependent launch: the passes and the control kernel are launched
// with programmatic stream serialization, so a launch may begin while its
// predecessor in the stream drains. Every kernel first waits for the predecessor to
// complete (its writes visible), before it reads anything, then allows its own
// successor to begin launching; the successor's blocks wait in turn. Launched
// without the attribute, both instructions return at once.
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Double-precision reciprocal and sixth root from single-precision seeds and
// Newton steps (two steps take a 1e-7 seed to full double precision). This
// GPU's double pipe is slow and the controller runs on one thread, so the
// short dependent chains matter.
__device__ inline double rcp_nr(double a)
{
    double r = (double)(1.0f / (float)a);
    r = r * (2.0 - a * r);
    r = r * (2.0 - a * r);
    return r;
}

// x^(1/6) for x in [1e-30, 1e30]: z = x^(-1/6) by Newton on z^-6 = x, then x z^5
__device__ inline double root6_nr(double x)
{
    double z = (double)powf((float)x, -1.0f / 6.0f);
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const double z2 = z * z, z6 = z2 * z2 * z2;
        z = z * (7.0 - x * z6) * (1.0 / 6.0);
    }
    const double z2 = z * z;
    return x * z2 * z2 * z;
}

// one control operation; returns false when the run stopped (done or failure)
__device__ inline bool ctrl_op(fch_ctrl *c, const fch_kparams &kp, int op, double S0, double S1,
                               double arg0)
{
    switch (op) {
    case OP_INIT_TRIAL: {
        double k1;
        if (arg0 > 0) {
            k1 = arg0; // fixed step
        } else {
            const double rem = c->t_final - c->t;
            if (rem <= 1e-12 * fmax(1.0, fabs(c->t_final))) {
                c->done = 1;
                return false;
            }
            k1 = fmin(c->ktrial, rem); // the run ends exactly at t_final
        }
        c->k1 = k1;
        if (c->kn <= 0) { // backward-Euler start: k_{n-1} -> infinity in eq. (BDF2Coef)
            const double r1 = rcp_nr(k1);
            c->a = r1;
            c->b = -r1;
            c->c = 0.0;
            c->gam = 0.0;
        } else {
            // eq. (BDF2Coef) and the eq. (Predictor) weights from three independent
            // reciprocals (1/(1+gam) = k_n/(k_{n+1}+k_n)), so their latencies overlap
            const double kn = c->kn;
            const double r1 = rcp_nr(k1), rn = rcp_nr(kn), rs = rcp_nr(k1 + kn);
            c->a = r1 + rs;
            c->b = -r1 - rn;
            c->c = rn - rs;
            const double g = k1 * rn;
            c->gam = g;
            const double k6 = k1 * (1.0 / 6.0), ig = kn * rs; // 1/(1+g)
            c->w1 = k6 * (3.0 + 2.0 * g) * ig;
            c->w2 = k6 * (3.0 + g);
            c->w3 = -k6 * g * g * ig;
        }
        // PSD search step: Table SearchSize row, linear in k, clamped (slopes precomputed)
        if (c->lam_k[0] < 0 || k1 <= c->lam_k[0]) {
            c->lam = c->lam_tab[0];
        } else if (k1 >= c->lam_k[9]) {
            c->lam = c->lam_tab[9];
        } else {
            int j = 0;
            while (j < 8 && k1 > c->lam_k[j + 1]) j++;
            c->lam = c->lam_tab[j] + (k1 - c->lam_k[j]) * c->lam_slope[j];
        }
        c->psd_conv = 0;
        c->psd_iter = 0;
        break;
    }
    case OP_SAV_E1: {
        const double e1 = kp.h2 * S0;
        const double v = e1 + kp.D0;
        if (!isfinite(v) || v <= 0) {
            c->status = FCH_ENONFINITE;
            c->done = 1;
            return false;
        }
        c->e1 = e1;
        c->inv_sqrt_e1 = 1.0 / sqrt(v);
        if (arg0 == 1.0) c->r_n = sqrt(v);
        if (arg0 == 2.0) c->r_m = sqrt(v);
        break;
    }
    case OP_SAV_R: {
        // eq. (4.8) with u^{n+1} = p + r q:
        // r (a - a (X, q)/2) = -b r^n - c r^{n-1} + (X, a p + b u^n + c u^{n-1})/2
        const double sc = kp.h2 * kp.inv_n2; // Parseval on the unnormalised half spectra
        const double xr = sc * S0, xq = sc * S1;
        const double r = (-c->b * c->r_n - c->c * c->r_m + 0.5 * xr) / (c->a * (1.0 - 0.5 * xq));
        if (!isfinite(r)) {
            c->status = FCH_ENONFINITE;
            c->done = 1;
            return false;
        }
        c->r_new = r;
        break;
    }
    case OP_PSD_CHECK: {
        const double ratio = sqrt(S0) / sqrt(S1); // ||d|| / ||v_{s+1}||, h cancels
        c->psd_iter++;
        c->n_psd_iter++;
        c->psd_ratio = ratio;
        if (!isfinite(ratio)) {
            c->status = FCH_ENONFINITE;
            c->done = 1;
        } else if (S0 < c->itol * c->itol * S1) {
            c->psd_conv = 1;
            c->last_psd_iter = c->psd_iter;
        } else if (c->psd_iter >= c->psd_max_iter) {
            c->status = FCH_ENOCONV;
            c->done = 1;
            c->last_psd_iter = c->psd_iter;
        }
        break;
    }
    case OP_DECIDE: {
        // Steps 3-4 of the adaptive algorithm, Sec. 3.2, with e^2 = S0/S1:
        // accept iff S0 <= sigma^2 S1 (or k <= k_min);
        // A_dp = rho_s k (sigma/e)^(1/3) = rho_s k (sigma^2 S1 / S0)^(1/6), e >= 1e-16
        c->n_attempts++;
        if (!isfinite(S0) || !isfinite(S1) || !(S1 > 0)) {
            c->status = FCH_ENONFINITE;
            c->done = 1;
            return false;
        }
        c->lte_num = S0;
        c->lte_den = S1;
        const double k1 = c->k1;
        const double x = fmin(c->sigma2 * S1 * rcp_nr(fmax(S0, 1e-32 * S1)), 1e30);
        double kn = c->rho_s * k1 * root6_nr(x);
        if (c->cap) kn = fmin(kn, 2.414213562373095 * k1); // (1 + sqrt 2) k
        kn = fmax(c->kmin, fmin(kn, c->kmax));
        if (S0 <= c->sigma2 * S1 || k1 <= c->kmin) {
            const int un = c->iu_n, um = c->iu_m, fn = c->if_n, fm = c->if_m;
            c->iu_m = un;
            c->iu_n = c->iu_new;
            c->iu_new = um;
            c->if_m = fn;
            c->if_n = c->if_new;
            c->if_new = fm;
            c->r_m = c->r_n;
            c->r_n = c->r_new;
            c->kn = k1;
            c->t += k1;
            c->n_steps++;
            c->accepted_last = 1;
        } else {
            c->n_rejects++;
            c->accepted_last = 0;
        }
        c->ktrial = kn;
        break;
    }
    case OP_ACCEPT: {
        const int un = c->iu_n, um = c->iu_m;
        c->iu_m = un;
        c->iu_n = c->iu_new;
        c->iu_new = um;
        if (arg0 == 1.0) { // also rotate the F history (adaptive start)
            const int fn = c->if_n, fm = c->if_m;
            c->if_m = fn;
            c->if_n = c->if_new;
            c->if_new = fm;
        }
        c->r_m = c->r_n;
        c->r_n = c->r_new;
        c->kn = c->k1;
        c->ktrial = c->k1;
        c->t += c->k1;
        c->n_steps++;
        c->n_attempts++;
        break;
    }
    case OP_ENERGY: {
        c->energy = kp.h2 * S0;
        break;
    }
    }
    return !c->done;
}

// Float, double and double-float mirrors of the per-trial coefficients read by
// the passes, lane i of the calling warp converting coefficient i: conversions run
// on the double pipe, where one warp instruction costs the same for eleven lanes as
// for one, so the eleven conversions cost one instruction sequence instead of eleven.
static_assert(offsetof(fch_ctrl, lam) == offsetof(fch_ctrl, a) + 7 * sizeof(double),
              "a, b, c, gam, w1, w2, w3, lam are consecutive doubles");
static_assert(sizeof(fch_coef<float>) == 11 * sizeof(float) && sizeof(fch_coef<double>) == 11 * sizeof(double) &&
                  sizeof(fch_coef<fch::df>) == 11 * sizeof(fch::df),
              "fch_coef is eleven coefficients in declaration order");
__device__ inline void sync_coef_lanes(fch_ctrl *c, int lane)
{
    if (lane < 11) {
        const double v = lane < 8 ? (&c->a)[lane] : lane == 8 ? c->k1 : lane == 9 ? c->r_new : c->inv_sqrt_e1;
        ((float *)&c->cof)[lane] = (float)v;
        ((double *)&c->cod)[lane] = v;
        ((fch::df *)&c->codf)[lane] = fch::df(v);
    }
}


// The whole control step by one block (any multiple of 32 threads up to 1024):
// the control block is staged through shared memory with coalesced copies, the
// first na partials of slots 0 and 1 are summed in a fixed order (per-thread
// strided sums, warp shuffles, then thread 0 over the warp sums), thread 0 runs
// the operation, and the block writes the control block back.
__device__ inline void ctrl_block(const fch_kparams &kp, int op, int na, double arg0)
{
    __shared__ double sh[2][32];
    __shared__ fch_ctrl cs;
    const int nw = (int)(sizeof(fch_ctrl) / 8);
    const int nthr = blockDim.x;
    for (int i = threadIdx.x; i < nw; i += nthr) ((long long *)&cs)[i] = ((const long long *)kp.ctrl)[i];
    // the partial sums load while the control block arrives (discarded if it says done)
    double s0 = 0, s1 = 0;
    for (int i = threadIdx.x; i < na; i += nthr) {
        s0 += kp.part[i];
        s1 += kp.part[FCH_MAXBLK + i];
    }
    __syncthreads();
    if (cs.done && !(kp.flags & FCH_FL_NOSKIP)) return;
    if (op == OP_PSD_CHECK && cs.psd_conv) return;
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s0;
        sh[1][threadIdx.x >> 5] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S0 = 0, S1 = 0;
        for (int w = 0; w < (nthr >> 5); w++) {
            S0 += sh[0][w];
            S1 += sh[1][w];
        }
        // the combined operations: the decision (adaptive) or the acceptance of a fixed
        // step, then the set-up of the next trial (adaptive: arg0 -1; fixed: arg0 = dt)
        bool again = false;
        double next_arg = -1.0;
        if (op == OP_DECIDE_INIT) {
            op = OP_DECIDE;
            again = true;
        } else if (op == OP_ACCEPT_INIT) {
            op = OP_ACCEPT;
            next_arg = arg0;
            arg0 = 0.0;
            again = true;
        }
        for (;;) {
            if (!ctrl_op(&cs, kp, op, S0, S1, arg0)) break;
            if (!again) break;
            again = false;
            op = OP_INIT_TRIAL;
            arg0 = next_arg;
        }
    }
    if (threadIdx.x < 32) {
        __syncwarp();
        sync_coef_lanes(&cs, threadIdx.x);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nw; i += nthr) ((long long *)kp.ctrl)[i] = ((const long long *)&cs)[i];
}

// Called by every block of a pass after its partial sums are written: the last
// block to arrive (atomic ticket after a fence) runs the control operation
// kp.tail_op over the partials of all gridDim.x blocks, then resets the ticket.
__device__ inline void pass_tail(const fch_kparams &kp)
{
    __shared__ unsigned int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(kp.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    ctrl_block(kp, kp.tail_op, gridDim.x, kp.tail_arg);
    if (threadIdx.x == 0) *kp.ticket = 0;
}
