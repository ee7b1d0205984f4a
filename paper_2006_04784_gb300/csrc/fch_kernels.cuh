// fch_kernels.cuh -- the passes of the pseudo-spectral FCH steppers on sm_103a.
//
// A 2D transform of two real fields a, b is one complex N x N transform of
// z = a + i b, done as two passes over HBM/L2:
//   row pass:    one block owns rpb rows; each row is transformed along x in
//                shared memory (mixed radix-8/4/2 Stockham, E = 8 elements per
//                thread per stage);
//   column pass: one block owns P column pairs (kx, N-kx); they are transformed
//                along y in shared memory, and the Hermitian split
//                A(k) = (Z(k) + conj Z(-k))/2, B(k) = (Z(k) - conj Z(-k))/(2i)
//                turns the pair into the half spectra of a and b.
// The work array Z between the passes is stored in "pair layout": row y holds
// N/2 pairs (kx, N-kx) for kx = 1..N/2-1 and (0, N/2) for pair 0, so a column
// block reads contiguous 2P-element segments of every row.
// Each pass fuses a stage of the method into its middle: the column pass the
// diagonal Fourier-space operations of Secs. 3.3-3.6 (and the AM3 predictor of
// Sec. 3.2), the row pass the pointwise chemical-potential pieces of eq. (FCH).
// Half spectra of the state live kx-major: S[kx*N + ky].
#pragma once
#include <math.h>
#include "fch_internal.h"

namespace fch {

template <typename T> struct CT;
template <> struct CT<double> { typedef double2 t; };
template <> struct CT<float> { typedef float2 t; };

template <typename C> __device__ __forceinline__ C mk(decltype(C().x) x, decltype(C().x) y)
{
    C r;
    r.x = x;
    r.y = y;
    return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s)
{
    return mk<C>(a.x * s, a.y * s);
}
// a * (DIR i): DIR = -1 forward (-i), +1 inverse (+i)
template <int DIR, typename C> __device__ __forceinline__ C rot(C a)
{
    return DIR < 0 ? mk<C>(a.y, -a.x) : mk<C>(-a.y, a.x);
}

template <int DIR, typename C> __device__ __forceinline__ void bfly2(C &a, C &b)
{
    C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int DIR, typename C> __device__ __forceinline__ void bfly4(C &x0, C &x1, C &x2, C &x3)
{
    C a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = rot<DIR>(csub(x1, x3));
    x0 = cadd(a, c);
    x1 = cadd(b, d);
    x2 = csub(a, c);
    x3 = csub(b, d);
}

template <int DIR, typename C> __device__ __forceinline__ void bfly8(C *v)
{
    typedef decltype(C().x) R;
    // even / odd 4-point transforms, then the W_8^k combination
    bfly4<DIR>(v[0], v[2], v[4], v[6]);
    bfly4<DIR>(v[1], v[3], v[5], v[7]);
    const R s = (R)0.70710678118654752440;
    C o1 = cmul(v[3], mk<C>(s, DIR * s));
    C o2 = rot<DIR>(v[5]);
    C o3 = cmul(v[7], mk<C>(-s, DIR * s));
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

// In-place Stockham transform of one length-N sequence held in shared memory at
// s[n*stride + off], by tps = N/8 threads (t = 0..tps-1), 8 elements per
// thread per stage. tw[m] = exp(-2 pi i m/N). Starts and ends with a barrier of
// the whole block (all sequences of a block run in lockstep).
template <int DIR, typename C>
__device__ void fft_smem(C *s, int N, int logN, int stride, int off, const C *tw, int t)
{
    const int tps = N >> 3;
    int Ns = 1, lNs = 0, rem = logN;
    __syncthreads();
    while (rem > 0) {
        const int lR = rem >= 3 ? 3 : rem;
        const int R = 1 << lR;
        const int nb = N >> lR;
        C v[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int b = i >> lR, r = i & (R - 1);
            const int j = t + b * tps;
            v[i] = s[(j + r * nb) * stride + off];
        }
        const int nbt = 8 >> lR; // butterflies per thread
#pragma unroll
        for (int b = 0; b < 8; b++) {
            if (b >= nbt) break;
            const int j = t + b * tps;
            const int jj = j & (Ns - 1);
            // twiddle index r * jj * N / (Ns R)
            const int step = (jj << (logN - lNs - lR));
            C *w = v + b * R;
#pragma unroll
            for (int r = 1; r < 8; r++) {
                if (r >= R) break;
                C tv = tw[(r * step) & (N - 1)];
                if (DIR > 0) tv = cconj(tv);
                w[r] = cmul(w[r], tv);
            }
            if (R == 8)
                bfly8<DIR>(w);
            else if (R == 4)
                bfly4<DIR>(w[0], w[1], w[2], w[3]);
            else
                bfly2<DIR>(w[0], w[1]);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int b = i >> lR, r = i & (R - 1);
            const int j = t + b * tps;
            const int jj = j & (Ns - 1);
            const int idxD = ((j >> lNs) << (lNs + lR)) + jj;
            s[(idxD + r * Ns) * stride + off] = v[i];
        }
        __syncthreads();
        Ns <<= lR;
        lNs += lR;
        rem -= lR;
    }
}

// natural kx of slot q of a pair-layout row
__device__ __forceinline__ int pair_kx(int q, int N)
{
    const int p = q >> 1, s = q & 1;
    if (p == 0) return s ? (N >> 1) : 0;
    return s ? N - p : p;
}

// ---------------------------------------------------------------------------
// the regularised well W_q, eq. (e:Wq-def), with an overflow-free sech/tanh
template <typename T>
__device__ __forceinline__ void well(const fch_kparams &kp, T u, T &W, T &W1, T &W2)
{
    const T bm = (T)kp.bm, bp = (T)kp.bp, eps = (T)kp.eps, q = (T)kp.q, g3 = (T)(kp.gamma / 3.0);
    const T v = u - bm;
    T A = (T)0.5 * v * v, A1 = v, A2 = (T)1;
    if (kp.q != 0.0) {
        const T x = v / eps;
        const T e = exp(-fabs(x));           // e^{-|x|} in (0, 1]
        const T den = (T)1 + e * e;
        const T sech = (T)2 * e / den;
        const T th = copysign(((T)1 - e * e) / den, x);
        A += q * eps * ((T)1 - sech);
        A1 += q * sech * th;
        A2 += (q / eps) * sech * ((T)2 * sech * sech - (T)1);
    }
    const T w = u - bp;
    const T B = (T)0.5 * w * w + g3 * (u - (T)0.5 * ((T)3 * bp - bm));
    const T B1 = w + g3;
    W = A * B;
    W1 = A1 * B + A * B1;
    W2 = A2 * B + (T)2 * A1 * B1 + A;
}

// ---------------------------------------------------------------------------
// block reduction of up to FCH_NRED doubles into part[slot][blockIdx.x]
template <int NR, typename T>
__device__ void block_partials(const T *red, double *part, double *scratch)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int r = 0; r < NR; r++) {
        double v = (double)red[r];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) scratch[r * 32 + wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < NR) {
        double s = 0;
        for (int w = 0; w < nw; w++) s += scratch[threadIdx.x * 32 + w];
        part[threadIdx.x * FCH_MAXBLK + blockIdx.x] = s;
    }
}

__device__ __forceinline__ bool pass_skipped(const fch_kparams &kp)
{
    if (kp.flags & FCH_FL_NOSKIP) return false;
    const fch_ctrl *c = kp.ctrl;
    if (c->done) return true;
    if ((kp.flags & FCH_FL_PSDSKIP) && c->psd_conv) return true;
    return false;
}

// ---------------------------------------------------------------------------
// ETD phi functions: phi1 = (e^z - 1)/z, phi2 = (e^z - 1 - z)/z^2, in double
__device__ __forceinline__ void etd_phi(double z, double &ez, double &p1, double &p2)
{
    ez = exp(z);
    if (fabs(z) < 1e-2) {
        // Horner forms of sum z^j/(j+1)! and sum z^j/(j+2)!, j < 9
        const double f1[9] = {1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040,
                              1.0 / 40320, 1.0 / 362880};
        const double f2[9] = {1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040,
                              1.0 / 40320, 1.0 / 362880, 1.0 / 3628800};
        double a = f1[8], b = f2[8];
        for (int j = 7; j >= 0; j--) {
            a = a * z + f1[j];
            b = b * z + f2[j];
        }
        p1 = a;
        p2 = b;
    } else {
        const double em = expm1(z);
        p1 = em / z;
        p2 = (em - z) / (z * z);
    }
}

// ---------------------------------------------------------------------------
// column pass: [forward columns + Hermitian split] -> spectral stage ->
//              [Hermitian pack + inverse columns]
template <typename T, int MODE> struct ColTraits {
    static const bool FWD = MODE != CM_INV_LOAD && MODE != CM_START && MODE != CM_SAV_COMBINE;
    static const bool INV_ALWAYS = MODE == CM_INV_LOAD || MODE == CM_START || MODE == CM_PSD_ITER ||
                                   MODE == CM_ETD_STAGE1;
    static const bool INV_OPT = MODE == CM_IMEX_SOLVE || MODE == CM_SAV_COMBINE ||
                                MODE == CM_ETD_STAGE2;
};

template <typename T, int MODE>
__device__ __forceinline__ void spec_elem(const fch_kparams &kp, const fch_ctrl *cs, int kx, int ky,
                                          typename CT<T>::t A, typename CT<T>::t B,
                                          typename CT<T>::t &Co, typename CT<T>::t &Do, T *red)
{
    typedef typename CT<T>::t C;
    const int N = kp.N;
    const long idx = (long)kx * N + ky;
    const int my = ky < (N >> 1) ? ky : ky - N;
    const T k2 = (T)(kp.kf * kp.kf) * (T)(kx * kx + my * my);
    const T e2 = (T)kp.eps2, am = (T)kp.am;
    const T sk = (e2 * k2 + am) * (e2 * k2 + am); // symbol of L_IMEX, eq. (e:IMEX-op)
    const T wgt = (kx == 0 || kx == (N >> 1)) ? (T)1 : (T)2;
    const T in2 = (T)kp.inv_n2;
    C v = mk<C>(0, 0);
    bool pack = false;

    if (MODE == CM_FWD_STORE) {
        ((C *)kp.out0)[idx] = A;
        if (kp.out1) ((C *)kp.out1)[idx] = B;
        return;
    }
    if (MODE == CM_INV_LOAD) {
        Co = cscale(((const C *)kp.in0)[idx], in2);
        Do = kp.in1 ? cscale(((const C *)kp.in1)[idx], in2) : mk<C>(0, 0);
        return;
    }
    const C *Un = (const C *)kp.U[cs->iu_n];
    const C *Um = (const C *)kp.U[cs->iu_m];
    C *Unew = (C *)kp.U[cs->iu_new];
    if (MODE == CM_START) {
        switch (kp.src) {
        case FCH_SRC_UN: v = Un[idx]; break;
        case FCH_SRC_UNEW: v = Unew[idx]; break;
        case FCH_SRC_V:
            v = ((const C *)kp.Vb)[idx];
            if (kp.flags & FCH_FL_COPYV) Unew[idx] = v;
            break;
        case FCH_SRC_IN0: v = ((const C *)kp.in0)[idx]; break;
        case 4: { // u* = u^n + gam (u^n - u^{n-1}), eq. (Richardson); gam = 0 at the start
            const T g = (T)cs->gam;
            const C un = Un[idx];
            v = g != (T)0 ? cadd(un, cscale(csub(un, Um[idx]), g)) : un;
            if (kp.flags & 128) ((C *)kp.Vb)[idx] = v; // PSD: v_0 = u*, eq. (recurrence)
            break;
        }
        case 5: v = Um[idx]; break;
        }
        pack = true;
    } else if (MODE == CM_IMEX_SOLVE) {
        // eq. (IMEX-eq): (a + |k|^2 s) u^{n+1} = -b u^n - c u^{n-1} - |k|^2 N_IMEX(u*)^
        const C Nh = csub(A, cscale(B, e2 * k2));
        const T a = (T)cs->a, b = (T)cs->b, c = (T)cs->c;
        const C rhs = csub(cscale(Un[idx], -b), cadd(cscale(Um[idx], c), cscale(Nh, k2)));
        v = cscale(rhs, (T)1 / (a + k2 * sk));
        Unew[idx] = v;
        pack = kp.flags & FCH_FL_PACK_F;
    } else if (MODE == CM_F_FINISH) {
        // mu^ = eps^4 |k|^4 u^ + eps^2 |k|^2 W'^ + (rest)^ ; F^ = -|k|^2 mu^ (eq. sFCH)
        const C *src;
        C *dst;
        switch (kp.src) {
        case FCH_SRC_UN: src = Un; dst = (C *)kp.F[cs->if_n]; break;
        case 5: src = Um; dst = (C *)kp.F[cs->if_m]; break;
        case FCH_SRC_UNEW: src = Unew; dst = (C *)kp.F[cs->if_new]; break;
        default: src = (const C *)kp.in0; dst = (C *)kp.out0; break;
        }
        const C u = src[idx];
        const C mu = cadd(cadd(cscale(u, e2 * e2 * k2 * k2), cscale(A, e2 * k2)), B);
        const C F = cscale(mu, -k2);
        dst[idx] = F;
        if (kp.flags & FCH_FL_AM3) {
            // eq. (Predictor): u_p = u^n + w1 F(u~) + w2 F(u^n) + w3 F(u^{n-1})
            const C Fn = ((const C *)kp.F[cs->if_n])[idx];
            const C Fm = ((const C *)kp.F[cs->if_m])[idx];
            const T w1 = (T)cs->w1, w2 = (T)cs->w2, w3 = (T)cs->w3;
            const C un = Un[idx];
            const C up = cadd(cadd(un, cscale(F, w1)), cadd(cscale(Fn, w2), cscale(Fm, w3)));
            const C df = csub(u, up);
            red[0] += wgt * (df.x * df.x + df.y * df.y);
            red[1] += wgt * (up.x * up.x + up.y * up.y);
        }
        return;
    } else if (MODE == CM_SAV_PQ) {
        // eqs. (4.7)-(4.8): (a + |k|^2 l0) p = -b u^n - c u^{n-1} - |k|^2 l1 u*,
        //                   (a + |k|^2 l0) q = -|k|^2 X,  X = V[u*]/sqrt(E1(u*) + D0)
        const T isq = (T)cs->inv_sqrt_e1;
        const C X = cscale(cadd(cscale(A, e2 * k2), B), isq);
        const T g = (T)cs->gam;
        const C un = Un[idx], um = Um[idx];
        const C us = g != (T)0 ? cadd(un, cscale(csub(un, um), g)) : un;
        const T b1 = (T)kp.beta1, b2 = (T)kp.beta2;
        const T l0 = e2 * e2 * k2 * k2 + b1 * am * e2 * k2 + b2 * am * am;
        const T l1 = -e2 * (T)(kp.eta1 + 2.0 * kp.zeta) * k2 - b1 * am * e2 * k2 - b2 * am * am;
        const T a = (T)cs->a, b = (T)cs->b, c = (T)cs->c;
        const T iden = (T)1 / (a + k2 * l0);
        const C p = cscale(csub(cscale(un, -b), cadd(cscale(um, c), cscale(us, k2 * l1))), iden);
        const C q = cscale(X, -k2 * iden);
        ((C *)kp.Pb)[idx] = p;
        ((C *)kp.Qb)[idx] = q;
        const C rr = cadd(cscale(p, a), cadd(cscale(un, b), cscale(um, c)));
        red[0] += wgt * (X.x * rr.x + X.y * rr.y);
        red[1] += wgt * (X.x * q.x + X.y * q.y);
        return;
    } else if (MODE == CM_SAV_COMBINE) {
        const T r = (T)cs->r_new;
        v = cadd(((const C *)kp.Pb)[idx], cscale(((const C *)kp.Qb)[idx], r));
        Unew[idx] = v;
        pack = kp.flags & FCH_FL_PACK_F;
    } else if (MODE == CM_PSD_ITER) {
        // R = mu(v) + (a v + b u^n + c u^{n-1}) / |k|^2,  d = -R / (s + a/|k|^2)  (k != 0),
        // v <- v + lambda d, eqs. (residual), (recurrence)
        C *Vb = (C *)kp.Vb;
        const C vv = Vb[idx];
        C d = mk<C>(0, 0);
        if (k2 > (T)0) {
            const C mu = cadd(cadd(cscale(vv, e2 * e2 * k2 * k2), cscale(A, e2 * k2)), B);
            const T a = (T)cs->a, b = (T)cs->b, c = (T)cs->c;
            const T ik2 = (T)1 / k2;
            const C R = cadd(mu, cscale(cadd(cscale(vv, a), cadd(cscale(Un[idx], b), cscale(Um[idx], c))), ik2));
            d = cscale(R, (T)-1 / (sk + a * ik2));
        }
        v = cadd(vv, cscale(d, (T)cs->lam));
        Vb[idx] = v;
        red[0] += wgt * (d.x * d.x + d.y * d.y);
        red[1] += wgt * (v.x * v.x + v.y * v.y);
        pack = true;
    } else if (MODE == CM_ETD_STAGE1 || MODE == CM_ETD_STAGE2) {
        // eqs. (ETDRK2), (ETD-L): l = -|k|^2 s - kappa0 - kappa2 eps^2 |k|^2, z = l k
        const T k0 = (T)kp.kappa0, kk2 = (T)kp.kappa2;
        const C Nim = csub(A, cscale(B, e2 * k2));
        const double ell = -(double)k2 * (double)sk - kp.kappa0 - kp.kappa2 * kp.eps2 * (double)k2;
        double ez, p1, p2;
        etd_phi(ell * cs->k1, ez, p1, p2);
        const T k1 = (T)cs->k1;
        C *Nb = (C *)kp.Nb;
        if (MODE == CM_ETD_STAGE1) {
            const C un = Un[idx];
            const C N0 = cadd(cscale(Nim, -k2), cscale(un, k0 + kk2 * e2 * k2));
            Nb[idx] = N0;
            v = cadd(cscale(un, (T)ez), cscale(N0, k1 * (T)p1));
            Unew[idx] = v;
            pack = true;
        } else {
            const C ut = Unew[idx];
            const C N1 = cadd(cscale(Nim, -k2), cscale(ut, k0 + kk2 * e2 * k2));
            v = cadd(ut, cscale(csub(N1, Nb[idx]), k1 * (T)p2));
            Unew[idx] = v;
            pack = kp.flags & FCH_FL_PACK_F;
        }
    }
    if (pack) {
        Co = cscale(v, in2);
        Do = cscale(v, -k2 * in2);
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(1024) col_pass(const fch_kparams kp)
{
    typedef typename CT<T>::t C;
    typedef ColTraits<T, MODE> TR;
    if (pass_skipped(kp)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red_scratch[FCH_NRED * 32];
    const int N = kp.N, P = kp.P, nc = 2 * P;
    C *tw = (C *)smem_raw;
    C *tile = tw + N;
    const int c = threadIdx.x % nc, t = threadIdx.x / nc;
    const int p0 = blockIdx.x * P;
    const fch_ctrl *cs = kp.ctrl;
    const bool inv = TR::INV_ALWAYS || (TR::INV_OPT && (kp.flags & FCH_FL_PACK_F));
    const bool has_red = MODE == CM_SAV_PQ || MODE == CM_PSD_ITER ||
                         (MODE == CM_F_FINISH && (kp.flags & FCH_FL_AM3));
    C *Z = (C *)kp.Z;

    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = ((const C *)kp.tw)[i];
    if (TR::FWD) {
        for (int i = threadIdx.x; i < N * nc; i += blockDim.x) {
            const int n = i / nc, cc = i - n * nc;
            tile[i] = Z[(long)n * N + 2 * p0 + cc];
        }
        fft_smem<-1>(tile, N, kp.logN, nc, c, tw, t);
    } else {
        __syncthreads();
    }

    T red[FCH_NRED] = {0, 0, 0, 0};
    // spectral stage: work item (pair p, ky); pair 0 covers columns 0 and N/2
    for (int i = threadIdx.x; i < P * N; i += blockDim.x) {
        const int pp = i / N, ky = i - pp * N;
        const int p = p0 + pp;
        const int s0 = 2 * pp, s1 = 2 * pp + 1;
        const int mky = (N - ky) & (N - 1);
        if (p > 0) {
            C A = mk<C>(0, 0), B = mk<C>(0, 0);
            if (TR::FWD) {
                const C z0 = tile[ky * nc + s0], z1 = cconj(tile[mky * nc + s1]);
                A = cscale(cadd(z0, z1), (T)0.5);
                const C dm = csub(z0, z1);
                B = mk<C>((T)0.5 * dm.y, (T)-0.5 * dm.x);
            }
            C Co = mk<C>(0, 0), Do = mk<C>(0, 0);
            spec_elem<T, MODE>(kp, cs, p, ky, A, B, Co, Do, red);
            if (inv) {
                tile[ky * nc + s0] = mk<C>(Co.x - Do.y, Co.y + Do.x);
                tile[mky * nc + s1] = mk<C>(Co.x + Do.y, Do.x - Co.y);
            }
        } else {
            if (ky > (N >> 1)) continue;
            // columns kx = 0 (slot s0) and kx = N/2 (slot s1), rows ky and -ky
            const int nrow = (ky == 0 || ky == (N >> 1)) ? 1 : 2;
            C za[2], zb[2];
            za[0] = tile[ky * nc + s0];
            za[1] = tile[mky * nc + s0];
            zb[0] = tile[ky * nc + s1];
            zb[1] = tile[mky * nc + s1];
            C outa[2], outb[2];
#pragma unroll
            for (int side = 0; side < 2; side++) {
                const C *zz = side ? zb : za;
                C *oo = side ? outb : outa;
                const int kx = side ? (N >> 1) : 0;
                for (int rr = 0; rr < nrow; rr++) {
                    const int kyy = rr ? mky : ky;
                    C A = mk<C>(0, 0), B = mk<C>(0, 0);
                    if (TR::FWD) {
                        const C z0 = zz[rr], z1 = cconj(zz[rr ^ 1]);
                        A = cscale(cadd(z0, z1), (T)0.5);
                        const C dm = csub(z0, z1);
                        B = mk<C>((T)0.5 * dm.y, (T)-0.5 * dm.x);
                    }
                    C Co = mk<C>(0, 0), Do = mk<C>(0, 0);
                    spec_elem<T, MODE>(kp, cs, kx, kyy, A, B, Co, Do, red);
                    oo[rr] = mk<C>(Co.x - Do.y, Co.y + Do.x);
                }
            }
            if (inv) {
                tile[ky * nc + s0] = outa[0];
                tile[ky * nc + s1] = outb[0];
                if (nrow == 2) {
                    tile[mky * nc + s0] = outa[1];
                    tile[mky * nc + s1] = outb[1];
                }
            }
        }
    }
    if (has_red) block_partials<2>(red, kp.part, red_scratch);
    if (inv) {
        fft_smem<+1>(tile, N, kp.logN, nc, c, tw, t);
        for (int i = threadIdx.x; i < N * nc; i += blockDim.x) {
            const int n = i / nc, cc = i - n * nc;
            Z[(long)n * N + 2 * p0 + cc] = tile[i];
        }
    }
}

// ---------------------------------------------------------------------------
// row pass: [inverse rows] -> pointwise stage -> [forward rows]
template <typename T, int MODE>
__global__ void __launch_bounds__(256) row_pass(const fch_kparams kp)
{
    typedef typename CT<T>::t C;
    if (pass_skipped(kp)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red_scratch[FCH_NRED * 32];
    const int N = kp.N, tps = N >> 3;
    if (kp.nfft && blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(kp.nfft, (MODE == RM_R2C_LOAD || MODE == RM_C2R_STORE || MODE == RM_ENERGY) ? 2ull : 4ull);
    C *tw = (C *)smem_raw;
    C *rows = tw + N;
    const int rpb = blockDim.x / tps;
    const int rr = threadIdx.x / tps, t = threadIdx.x - rr * tps;
    const int y0 = blockIdx.x * rpb;
    C *Z = (C *)kp.Z;
    const bool f64io = kp.flags & FCH_FL_F64IO;

    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = ((const C *)kp.tw)[i];
    if (MODE == RM_R2C_LOAD) {
        for (int i = threadIdx.x; i < rpb * N; i += blockDim.x) {
            const long g = (long)y0 * N + i;
            T a, b = 0;
            if (f64io) {
                a = (T)((const double *)kp.in0)[g];
                if (kp.in1) b = (T)((const double *)kp.in1)[g];
            } else {
                a = (T)((const float *)kp.in0)[g];
                if (kp.in1) b = (T)((const float *)kp.in1)[g];
            }
            rows[i] = mk<C>(a, b);
        }
    } else {
        for (int i = threadIdx.x; i < rpb * N; i += blockDim.x) {
            const int r = i / N, q = i - r * N;
            rows[r * N + pair_kx(q, N)] = Z[(long)(y0 + r) * N + q];
        }
        fft_smem<+1>(rows + rr * N, N, kp.logN, 1, 0, tw, t);
    }

    T red[FCH_NRED] = {0, 0, 0, 0};
    C *s = rows + rr * N;
    const int y = y0 + rr;
    if (MODE != RM_R2C_LOAD) {
        const T e2 = (T)kp.eps2, am = (T)kp.am, eta1 = (T)kp.eta1, eta2 = (T)kp.eta2,
                zeta = (T)kp.zeta;
        for (int x = t; x < N; x += tps) {
            const C z = s[x];
            const T u = z.x, lu = z.y; // u and Lap u
            if (MODE == RM_C2R_STORE) {
                const long g = (long)y * N + x;
                if (f64io) {
                    if (kp.out0) ((double *)kp.out0)[g] = (double)u;
                    if (kp.out1) ((double *)kp.out1)[g] = (double)lu;
                } else {
                    if (kp.out0) ((float *)kp.out0)[g] = (float)u;
                    if (kp.out1) ((float *)kp.out1)[g] = (float)lu;
                }
                continue;
            }
            T W, W1, W2;
            well<T>(kp, u, W, W1, W2);
            C o = mk<C>(0, 0);
            if (MODE == RM_NIMEX) {
                // N_IMEX = [eps^2 (am - W'' + eta1) Lap u + W''W' - am^2 u - eta2 W'] + eps^2 Lap (am u - W')
                o.x = e2 * (am - W2 + eta1) * lu + W2 * W1 - am * am * u - eta2 * W1;
                o.y = am * u - W1;
            } else if (MODE == RM_F || MODE == RM_ENERGY) {
                // mu = eps^2 Lap w - W'' w + eps^2 eta1 Lap u - eta2 W', w = eps^2 Lap u - W'
                const T w = e2 * lu - W1;
                o.x = W1;
                o.y = -W2 * w - eta2 * W1 + e2 * eta1 * lu;
                if (MODE == RM_ENERGY || (kp.flags & FCH_FL_ENERGY))
                    red[0] += (T)0.5 * w * w - eta2 * W + (T)0.5 * e2 * eta1 * u * lu;
            } else if (MODE == RM_SAV) {
                // V = -eps^2 Lap (W' + zeta u) + [-eps^2 (W'' + zeta) Lap u + W' W'' - eta2 W']
                o.x = W1 + zeta * u;
                o.y = -e2 * (W2 + zeta) * lu + W1 * W2 - eta2 * W1;
                red[0] += -e2 * lu * (W1 + zeta * u) + (T)0.5 * W1 * W1 - eta2 * W;
            }
            s[x] = o;
        }
    }
    const bool has_red = MODE == RM_SAV || MODE == RM_ENERGY || (MODE == RM_F && (kp.flags & FCH_FL_ENERGY));
    if (has_red) block_partials<1>(red, kp.part, red_scratch);
    if (MODE == RM_C2R_STORE || MODE == RM_ENERGY) return;

    fft_smem<-1>(rows + rr * N, N, kp.logN, 1, 0, tw, t);
    for (int i = threadIdx.x; i < rpb * N; i += blockDim.x) {
        const int r = i / N, q = i - r * N;
        Z[(long)(y0 + r) * N + q] = rows[r * N + pair_kx(q, N)];
    }
}

} // namespace fch
