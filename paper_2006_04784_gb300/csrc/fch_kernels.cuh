// fch_kernels.cuh -- the passes of the pseudo-spectral FCH steppers on sm_103a.
//
// A 2D transform of two real fields a, b is one complex N x N transform of
// z = a + i b, done as two passes over HBM/L2:
//   row pass:    one block owns rpb rows; each row is transformed along x in
//                shared memory (Stockham, radix-8 stages then one radix-4 or
//                radix-2 stage, 8 elements per thread per stage);
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
//
// Single-precision passes do no double-precision arithmetic per element: the
// double pipe of this GPU runs at a small fraction of the float rate, so every
// constant arrives precomputed in the pass precision (fch_consts, fch_coef).
#pragma once
#include <cooperative_groups.h>
#include <math.h>
#include "fch_ctrl.cuh"
#include "fch_df.cuh"
#include "fch_internal.h"

namespace fch {

template <typename T> struct CT;
template <> struct CT<double> { typedef double2 t; };
template <> struct CT<float> { typedef float2 t; };

template <> struct CT<df> { typedef df2 t; };

template <typename T> __device__ __forceinline__ const fch_consts<T> &consts(const fch_kparams &kp);
template <> __device__ __forceinline__ const fch_consts<float> &consts<float>(const fch_kparams &kp) { return kp.cf; }
template <> __device__ __forceinline__ const fch_consts<double> &consts<double>(const fch_kparams &kp) { return kp.cd; }
template <> __device__ __forceinline__ const fch_consts<df> &consts<df>(const fch_kparams &kp) { return kp.cdf; }

template <typename T> __device__ __forceinline__ fch_coef<T> load_coef(const fch_ctrl *c);
template <> __device__ __forceinline__ fch_coef<float> load_coef<float>(const fch_ctrl *c) { return c->cof; }
template <> __device__ __forceinline__ fch_coef<double> load_coef<double>(const fch_ctrl *c) { return c->cod; }
template <> __device__ __forceinline__ fch_coef<df> load_coef<df>(const fch_ctrl *c) { return c->codf; }

// type of the warp-level sums of per-thread partials (double-float partials are
// summed as doubles)
template <typename T> struct RedType { typedef T t; };
template <> struct RedType<df> { typedef double t; };

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
// a s for an exact power of two s
template <typename C, typename S> __device__ __forceinline__ C cscale_p2(C a, S s)
{
    return mk<C>(mul_p2(a.x, s), mul_p2(a.y, s));
}
// Butterfly arithmetic: the plain complex operations for float and double; for
// double-float the unrenormalised sums and twiddle product of fch_df.cuh, with
// bnorm() renormalising where the last transform stage stores its results.
template <typename R> __device__ __forceinline__ R radd(R a, R b) { return a + b; }
template <typename R> __device__ __forceinline__ R rsub(R a, R b) { return a - b; }
template <> __device__ __forceinline__ df radd(df a, df b) { return add_lazy(a, b); }
template <> __device__ __forceinline__ df rsub(df a, df b) { return sub_lazy(a, b); }

template <typename R> __device__ __forceinline__ R rmul(R a, R b) { return a * b; }
template <> __device__ __forceinline__ df rmul(df a, df b) { return mul_lazy(a, b); }

template <typename C> __device__ __forceinline__ C badd(C a, C b) { return mk<C>(radd(a.x, b.x), radd(a.y, b.y)); }
template <typename C> __device__ __forceinline__ C bsub(C a, C b) { return mk<C>(rsub(a.x, b.x), rsub(a.y, b.y)); }
template <typename C> __device__ __forceinline__ C btw(C a, C w) { return cmul(a, w); }
template <> __device__ __forceinline__ df2 btw(df2 a, df2 w) { return cmul_lazy(a, w); }
template <typename C> __device__ __forceinline__ C bnorm(C a) { return a; }
template <> __device__ __forceinline__ df2 bnorm(df2 a) { return mk<df2>(renorm(a.x), renorm(a.y)); }
// The pointwise and spectral stages use the same unrenormalised arithmetic for
// double-float (radd, rsub, rmul; lscale below) and renormalise exactly (lnorm) what
// they store; for float and double these are the plain operations.
template <typename C, typename S> __device__ __forceinline__ C lscale(C a, S s)
{
    return mk<C>(rmul(a.x, s), rmul(a.y, s));
}
template <typename C> __device__ __forceinline__ C lnorm(C a) { return a; }
template <> __device__ __forceinline__ df2 lnorm(df2 a) { return mk<df2>(renorm_exact(a.x), renorm_exact(a.y)); }

// a * (DIR i): DIR = -1 forward (-i), +1 inverse (+i)
template <int DIR, typename C> __device__ __forceinline__ C rot(C a)
{
    return DIR < 0 ? mk<C>(a.y, -a.x) : mk<C>(-a.y, a.x);
}

template <int DIR, typename C> __device__ __forceinline__ void bfly2(C &a, C &b)
{
    C t = a;
    a = badd(t, b);
    b = bsub(t, b);
}

template <int DIR, typename C> __device__ __forceinline__ void bfly4(C &x0, C &x1, C &x2, C &x3)
{
    C a = badd(x0, x2), b = bsub(x0, x2), c = badd(x1, x3), d = rot<DIR>(bsub(x1, x3));
    x0 = badd(a, c);
    x1 = badd(b, d);
    x2 = bsub(a, c);
    x3 = bsub(b, d);
}

template <int DIR, typename C> __device__ __forceinline__ void bfly8(C *v)
{
    typedef decltype(C().x) R;
    // even / odd 4-point transforms, then the W_8^k combination
    bfly4<DIR>(v[0], v[2], v[4], v[6]);
    bfly4<DIR>(v[1], v[3], v[5], v[7]);
    const R s = (R)0.70710678118654752440;
    // x W8 and x W8^3 with W8 = s (1 + DIR i): two adds and two scalings each
    const C a = v[3], b = v[7];
    C o1, o3;
    if (DIR < 0) {
        o1 = mk<C>(rmul(radd(a.x, a.y), s), rmul(rsub(a.y, a.x), s));
        o3 = mk<C>(rmul(rsub(b.y, b.x), s), -rmul(radd(b.x, b.y), s));
    } else {
        o1 = mk<C>(rmul(rsub(a.x, a.y), s), rmul(radd(a.x, a.y), s));
        o3 = mk<C>(-rmul(radd(b.x, b.y), s), rmul(rsub(b.x, b.y), s));
    }
    C o2 = rot<DIR>(v[5]);
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = badd(e0, o0);
    v[4] = bsub(e0, o0);
    v[1] = badd(e1, o1);
    v[5] = bsub(e1, o1);
    v[2] = badd(e2, o2);
    v[6] = bsub(e2, o2);
    v[3] = badd(e3, o3);
    v[7] = bsub(e3, o3);
}

// Shared-memory skew: element n of a sequence is stored at n + n/8, which spreads
// the stride-R stores of the first Stockham stages over the banks.
__device__ __forceinline__ int skew(int n) { return n + (n >> 3); }
__host__ __device__ inline int skewed_len(int n) { return n + (n >> 3); }

// One Stockham stage of radix R = 2^LR on a length-N sequence at
// s[skew(n)*stride + off]; thread t of tps = N/PPT owns PPT/R butterflies (PPT points a
// thread: 8 with radix-8 stages, 4 with radix-4 stages).
template <int DIR, int LR, bool TWG, int PPT, typename C>
__device__ __forceinline__ void fft_stage(C *s, int N, int logN, int stride, int off, const C *tw,
                                          int t, int Ns, int lNs)
{
    constexpr int R = 1 << LR;
    constexpr int NB = PPT / R;
    static_assert(NB >= 1 && (PPT == 8 || PPT == 4), "a stage's radix divides the points a thread");
    const int tps = N / PPT, nb = N >> LR;
    // double-float values stay unrenormalised between stages (the sums and twiddle
    // products take such operands); the last stage renormalises what it stores
    const bool last = (Ns << LR) == N;
    C v[PPT];
#pragma unroll
    for (int b = 0; b < NB; b++) {
        const int j = t + b * tps;
#pragma unroll
        for (int r = 0; r < R; r++) v[b * R + r] = s[skew(j + r * nb) * stride + off];
    }
#pragma unroll
    for (int b = 0; b < NB; b++) {
        const int j = t + b * tps;
        if (Ns > 1) {
            // twiddle exp(DIR 2 pi i r (j mod Ns) / (Ns R)) from the per-stage table
            // (every stage before the last has radix PPT, so this stage starts at
            // Ns - PPT; entry [r-1][j mod Ns]: consecutive lanes read consecutive entries)
            const C *tws = tw + (Ns - PPT) + (j & (Ns - 1));
#pragma unroll
            for (int r = 1; r < R; r++) {
                C tv = TWG ? ldg(tws + (r - 1) * Ns) : tws[(r - 1) * Ns];
                if (DIR > 0) tv = cconj(tv);
                v[b * R + r] = btw(v[b * R + r], tv);
            }
        }
        if (LR == 3)
            bfly8<DIR>(v + b * R);
        else if (LR == 2)
            bfly4<DIR>(v[b * R], v[b * R + 1], v[b * R + 2], v[b * R + 3]);
        else
            bfly2<DIR>(v[b * R], v[b * R + 1]);
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; b++) {
        const int j = t + b * tps;
        const int idxD = ((j >> lNs) << (lNs + LR)) + (j & (Ns - 1));
#pragma unroll
        for (int r = 0; r < R; r++)
            s[skew(idxD + r * Ns) * stride + off] = last ? bnorm(v[b * R + r]) : v[b * R + r];
    }
    __syncthreads();
}

// In-place transform of one sequence (all sequences of a block in lockstep);
// starts and ends with a barrier of the whole block. PPT points a thread (t < N/PPT):
// radix-8 stages (PPT 8) or radix-4 stages (PPT 4), then one stage of the remaining
// radix. tw holds the forward twiddles of every stage with Ns > 1 (stage with Ns:
// entries Ns - PPT + (r-1) Ns + j, value exp(-2 pi i r j / (Ns R)), r = 1..R-1,
// j < Ns; a table per PPT), in shared memory, or in global memory read through the
// read-only cache when TWG.
template <int DIR, bool TWG = false, int PPT = 8, typename C>
__device__ void fft_smem(C *s, int N, int logN, int stride, int off, const C *tw, int t)
{
    constexpr int LP = PPT == 8 ? 3 : 2;
    int Ns = 1, lNs = 0, rem = logN;
    __syncthreads();
    while (rem >= LP) {
        fft_stage<DIR, LP, TWG, PPT>(s, N, logN, stride, off, tw, t, Ns, lNs);
        Ns <<= LP;
        lNs += LP;
        rem -= LP;
    }
    if constexpr (LP == 3) {
        if (rem == 2) fft_stage<DIR, 2, TWG, PPT>(s, N, logN, stride, off, tw, t, Ns, lNs);
    }
    if (rem == 1) fft_stage<DIR, 1, TWG, PPT>(s, N, logN, stride, off, tw, t, Ns, lNs);
}

// natural kx of slot q of a pair-layout row
__device__ __forceinline__ int pair_kx(int q, int N)
{
    const int p = q >> 1, s = q & 1;
    if (p == 0) return s ? (N >> 1) : 0;
    return s ? N - p : p;
}

// ---------------------------------------------------------------------------
// c[0] + c[1] u + ... + c[M-1] u^(M-1) by Horner's rule
template <typename T, int M> __device__ __forceinline__ T horner(const T *c, T u)
{
    T p = c[M - 1];
#pragma unroll
    for (int i = M - 2; i >= 0; i--) p = radd(rmul(p, u), c[i]);
    return p;
}

// the regularised well W_q, eq. (e:Wq-def), with an overflow-free sech/tanh
// (W itself only where need_w: the energy density and the SAV functional use it)
template <typename T>
__device__ __forceinline__ void well(const fch_consts<T> &k, T u, T &W, T &W1, T &W2, bool need_w)
{
    if (k.q == (T)0) {
        // a quartic: W, W' and W'' by Horner's rule from the host's expansion
        W = need_w ? horner<T, 5>(k.wp, u) : (T)0;
        W1 = horner<T, 4>(k.w1p, u);
        W2 = horner<T, 3>(k.w2p, u);
        return;
    }
    const T v = rsub(u, k.bm);
    T A = mul_p2(rmul(v, v), (T)0.5), A1 = v, A2 = (T)1;
    if (k.q != (T)0) {
        const T x = v / k.eps;
        const T e = exp(-fabs(x)); // e^{-|x|} in (0, 1]
        const T id = recip((T)1 + e * e);
        const T sech = mul_p2(e * id, (T)2);
        const T th = copysign(((T)1 - e * e) * id, x);
        A += k.qeps * ((T)1 - sech);
        A1 += k.q * sech * th;
        A2 += k.qoe * sech * (mul_p2(sech * sech, (T)2) - (T)1);
    }
    const T w = rsub(u, k.bp);
    const T B = radd(mul_p2(rmul(w, w), (T)0.5), rmul(k.g3, rsub(u, k.c3)));
    const T B1 = radd(w, k.g3);
    W = rmul(A, B);
    W1 = radd(rmul(A1, B), rmul(A, B1));
    W2 = radd(radd(k.q != (T)0 ? rmul(A2, B) : B, mul_p2(rmul(A1, B1), (T)2)), A);
}

// ---------------------------------------------------------------------------
// block reduction of NR per-thread partials into part[slot][blockIdx.x]:
// warp sums in the pass precision, the per-block sum of warp sums in double.
template <int NR, typename T>
__device__ void block_partials(const T *red, double *part, double *scratch)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    typedef typename RedType<T>::t R;
#pragma unroll
    for (int r = 0; r < NR; r++) {
        R v = (R)red[r];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) scratch[r * 32 + wid] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < NR) {
        double s = 0;
        for (int w = 0; w < nw; w++) s += scratch[threadIdx.x * 32 + w];
        part[threadIdx.x * FCH_MAXBLK + blockIdx.x] = s;
    }
}

// Double-float partials: the warp and block sums in double-float arithmetic on the
// FP32 pipe (the double pipe runs a warp instruction in many cycles, and a block
// sum in double would cost dozens of them per block), one conversion per slot.
template <int NR>
__device__ void block_partials(const df *red, double *part, double *scratch)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    float2 *sc = (float2 *)scratch;
#pragma unroll
    for (int r = 0; r < NR; r++) {
        df v = red[r];
        for (int o = 16; o > 0; o >>= 1)
            v = v + df(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
        if (lane == 0) sc[r * 32 + wid] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    if (threadIdx.x < NR) {
        df s(0.f, 0.f);
        for (int w = 0; w < nw; w++) {
            const float2 e = sc[threadIdx.x * 32 + w];
            s = s + df(e.x, e.y);
        }
        part[threadIdx.x * FCH_MAXBLK + blockIdx.x] = (double)s;
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
// ETD phi functions in precision T: phi1 = (e^z - 1)/z, phi2 = (e^z - 1 - z)/z^2.
// Below a threshold (1e-2 in double, 0.1 in float, where the direct forms lose
// digits to cancellation) the Taylor series sum_j z^j/(j+1)!, sum_j z^j/(j+2)!
// in Horner form, j < 10; the direct forms above.
template <typename T> __device__ __forceinline__ void etd_phi(T z, T &ez, T &p1, T &p2)
{
    ez = exp(z);
    const T thr = sizeof(T) == 8 ? (T)1e-2 : (T)0.1;
    if (fabs(z) < thr) {
        // inverse factorials 1/1! .. 1/11!
        const T f[11] = {(T)1.0, (T)(1.0 / 2), (T)(1.0 / 6), (T)(1.0 / 24), (T)(1.0 / 120),
                         (T)(1.0 / 720), (T)(1.0 / 5040), (T)(1.0 / 40320), (T)(1.0 / 362880),
                         (T)(1.0 / 3628800), (T)(1.0 / 39916800)};
        T a = f[9], b = f[10];
#pragma unroll
        for (int j = 8; j >= 0; j--) {
            a = a * z + f[j];
            b = b * z + f[j + 1];
        }
        p1 = a;
        p2 = b;
    } else {
        const T em = expm1(z);
        p1 = em / z;
        p2 = (em - z) / (z * z);
    }
}

// ---------------------------------------------------------------------------
// column pass: [forward columns + Hermitian split] -> spectral stage ->
//              [Hermitian pack + inverse columns]
template <int MODE> struct ColTraits {
    static const bool FWD = MODE != CM_INV_LOAD && MODE != CM_START && MODE != CM_SAV_COMBINE;
    static const bool INV_ALWAYS = MODE == CM_INV_LOAD || MODE == CM_START || MODE == CM_PSD_ITER ||
                                   MODE == CM_ETD_STAGE1;
    static const bool INV_OPT = MODE == CM_IMEX_SOLVE || MODE == CM_SAV_COMBINE ||
                                MODE == CM_ETD_STAGE2;
};

// buffers a column pass works on, resolved once per block from the control block
template <typename C> struct ColBufs {
    const C *Un, *Um, *src, *Fn, *Fm;
    C *Unew, *dst;
    const C *i0, *i1; // standalone transforms: this pair's half spectra in / out
    C *o0, *o1;
};

// Standalone transforms of several field pairs in one launch: pair blockIdx.y
// reads and writes its own fields (pstride_in / pstride_out bytes after the
// previous pair's) and its own N x N slice of the work array. Other launches have
// one pair (blockIdx.y = 0).
__device__ __forceinline__ const void *pair_in(const void *p, const fch_kparams &kp)
{
    return p ? (const void *)((const char *)p + blockIdx.y * kp.pstride_in) : nullptr;
}
__device__ __forceinline__ void *pair_out(void *p, const fch_kparams &kp)
{
    return p ? (void *)((char *)p + blockIdx.y * kp.pstride_out) : nullptr;
}
template <typename C> __device__ __forceinline__ C *pair_Z(const fch_kparams &kp, int N)
{
    return (C *)kp.Z + (size_t)blockIdx.y * N * N;
}

template <typename T, int MODE>
__device__ __forceinline__ void spec_elem(const fch_kparams &kp, const fch_consts<T> &K,
                                          const fch_coef<T> &co, const ColBufs<typename CT<T>::t> &bf,
                                          int kx, int ky, typename CT<T>::t A, typename CT<T>::t B,
                                          typename CT<T>::t &Co, typename CT<T>::t &Do, T *red)
{
    typedef typename CT<T>::t C;
    const int N = kp.N;
    const long idx = (long)kx * N + ky;
    const int my = ky < (N >> 1) ? ky : ky - N;
    const T k2 = rmul(K.kf2, (T)(kx * kx + my * my));
    const T sq = radd(rmul(K.e2, k2), K.am);
    const T sk = rmul(sq, sq); // symbol of L_IMEX, eq. (e:IMEX-op)
    const T wgt = (kx == 0 || kx == (N >> 1)) ? (T)1 : (T)2;
    C v = mk<C>(0, 0);
    bool pack = false;

    if (MODE == CM_FWD_STORE) {
        bf.o0[idx] = lnorm(A);
        if (bf.o1) bf.o1[idx] = lnorm(B);
        return;
    }
    if (MODE == CM_INV_LOAD) {
        Co = cscale_p2(bf.i0[idx], K.inv_n2);
        Do = bf.i1 ? cscale_p2(bf.i1[idx], K.inv_n2) : mk<C>(0, 0);
        return;
    }
    if (MODE == CM_START) {
        if (kp.src == 4) { // u* = u^n + gam (u^n - u^{n-1}), eq. (Richardson); gam = 0 at the start
            const C un = ldg(bf.Un + idx);
            v = co.gam != (T)0 ? cadd(un, cscale(csub(un, ldg(bf.Um + idx)), co.gam)) : un;
            if (kp.flags & 128) ((C *)kp.Vb)[idx] = v; // PSD: v_0 = u*, eq. (recurrence)
        } else {
            v = bf.src[idx];
            if (kp.flags & FCH_FL_COPYV) bf.Unew[idx] = v;
        }
        pack = true;
    } else if (MODE == CM_IMEX_SOLVE) {
        // eq. (IMEX-eq): (a + |k|^2 s) u^{n+1} = -b u^n - c u^{n-1} - |k|^2 N_IMEX(u*)^
        if ((kx | ky) == 0) {
            // the mean mode (k = 0) carries the mass: renormalised arithmetic and a
            // division there, where a bias of the one-Newton-step reciprocal (or the
            // coarser rounding of unrenormalised low words) would repeat every step
            const C rhs = csub(cscale(ldg(bf.Un + idx), -co.b), cscale(ldg(bf.Um + idx), co.c));
            v = mk<C>(rhs.x / co.a, rhs.y / co.a);
        } else {
            const C Nh = bsub(A, lscale(B, rmul(K.e2, k2)));
            const C rhs =
                bsub(lscale(ldg(bf.Un + idx), -co.b), badd(lscale(ldg(bf.Um + idx), co.c), lscale(Nh, k2)));
            v = lscale(rhs, recip(radd(co.a, rmul(k2, sk))));
        }
        bf.Unew[idx] = lnorm(v);
        pack = kp.flags & FCH_FL_PACK_F;
    } else if (MODE == CM_F_FINISH) {
        // mu^ = eps^4 |k|^4 u^ + eps^2 |k|^2 W'^ + (rest)^ ; F^ = -|k|^2 mu^ (eq. sFCH)
        const C u = ldg(bf.src + idx);
        const C mu = badd(badd(lscale(u, rmul(rmul(K.e4, k2), k2)), lscale(A, rmul(K.e2, k2))), B);
        const C F = lscale(mu, -k2);
        bf.dst[idx] = lnorm(F);
        if (kp.flags & FCH_FL_AM3) {
            // eq. (Predictor): u_p = u^n + w1 F(u~) + w2 F(u^n) + w3 F(u^{n-1})
            const C up = badd(badd(ldg(bf.Un + idx), lscale(F, co.w1)),
                              badd(lscale(ldg(bf.Fn + idx), co.w2), lscale(ldg(bf.Fm + idx), co.w3)));
            // the difference cancels the high words where the error is small: it is
            // renormalised before it is squared (a product drops lo x lo, which then
            // carries the whole value)
            const C df = lnorm(bsub(u, up));
            // lazy sums of squares (the weight 1 or 2 scales exactly); |u_p|^2 is a sum of
            // large terms, where a dropped lo x lo is far below the sum's own rounding
            red[0] = radd(red[0], mul_p2(radd(rmul(df.x, df.x), rmul(df.y, df.y)), wgt));
            red[1] = radd(red[1], mul_p2(radd(rmul(up.x, up.x), rmul(up.y, up.y)), wgt));
        }
        return;
    } else if (MODE == CM_SAV_PQ) {
        // eqs. (4.7)-(4.8): (a + |k|^2 l0) p = -b u^n - c u^{n-1} - |k|^2 l1 u*,
        //                   (a + |k|^2 l0) q = -|k|^2 X,  X = V[u*]/sqrt(E1(u*) + D0)
        const C X = lscale(badd(lscale(A, rmul(K.e2, k2)), B), co.isq);
        const C un = ldg(bf.Un + idx), um = ldg(bf.Um + idx);
        const C us = (kp.flags & FCH_FL_USTAR_V) ? ((const C *)kp.Vb)[idx]
                     : co.gam != (T)0           ? badd(un, lscale(bsub(un, um), co.gam))
                                                : un;
        const T l0 = radd(radd(rmul(rmul(K.e4, k2), k2), rmul(K.b1am_e2, k2)), K.b2am2);
        const T l1 = rsub(rsub(rmul(-K.l1c, k2), rmul(K.b1am_e2, k2)), K.b2am2);
        const T den = radd(co.a, rmul(k2, l0));
        const T iden = recip(den);
        C p;
        if ((kx | ky) == 0) { // the mean mode: as in the IMEX solve
            const C pr = csub(cscale(un, -co.b), cscale(um, co.c));
            p = mk<C>(pr.x / co.a, pr.y / co.a);
        } else {
            p = lnorm(lscale(bsub(lscale(un, -co.b), badd(lscale(um, co.c), lscale(us, rmul(k2, l1)))), iden));
        }
        const C q = lnorm(lscale(X, rmul(-k2, iden)));
        ((C *)kp.Pb)[idx] = p;
        ((C *)kp.Qb)[idx] = q;
        // a p + b u^n + c u^{n-1} cancels (a + b + c = 0): renormalised before its product
        const C rr = lnorm(badd(lscale(p, co.a), badd(lscale(un, co.b), lscale(um, co.c))));
        red[0] = radd(red[0], mul_p2(radd(rmul(X.x, rr.x), rmul(X.y, rr.y)), wgt));
        red[1] = radd(red[1], mul_p2(radd(rmul(X.x, q.x), rmul(X.y, q.y)), wgt));
        return;
    } else if (MODE == CM_SAV_COMBINE) {
        v = badd(((const C *)kp.Pb)[idx], lscale(((const C *)kp.Qb)[idx], co.r_new));
        bf.Unew[idx] = lnorm(v);
        pack = kp.flags & FCH_FL_PACK_F;
    } else if (MODE == CM_PSD_ITER) {
        // R = mu(v) + (a v + b u^n + c u^{n-1}) / |k|^2,  d = -R / (s + a/|k|^2)  (k != 0),
        // v <- v + lambda d, eqs. (residual), (recurrence)
        C *Vb = (C *)kp.Vb;
        const C vv = Vb[idx];
        C d = mk<C>(0, 0);
        if (k2 > (T)0) {
            const C mu = badd(badd(lscale(vv, rmul(rmul(K.e4, k2), k2)), lscale(A, rmul(K.e2, k2))), B);
            const T ik2 = recip(k2);
            const C R = badd(mu, lscale(badd(lscale(vv, co.a), badd(lscale(bf.Un[idx], co.b),
                                                                    lscale(bf.Um[idx], co.c))), ik2));
            // the residual shrinks as the iteration converges: d is renormalised before
            // its square enters the stopping test
            d = lnorm(lscale(R, -recip(radd(sk, rmul(co.a, ik2)))));
        }
        v = lnorm(badd(vv, lscale(d, co.lam)));
        Vb[idx] = v;
        red[0] = radd(red[0], mul_p2(radd(rmul(d.x, d.x), rmul(d.y, d.y)), wgt));
        red[1] = radd(red[1], mul_p2(radd(rmul(v.x, v.x), rmul(v.y, v.y)), wgt));
        pack = true;
    } else if (MODE == CM_ETD_STAGE1 || MODE == CM_ETD_STAGE2) {
        // eqs. (ETDRK2), (ETD-L): l = -|k|^2 s - kappa0 - kappa2 eps^2 |k|^2, z = l k
        const C Nim = bsub(A, lscale(B, rmul(K.e2, k2)));
        const T ell = rsub(rsub(rmul(-k2, sk), K.kappa0), rmul(K.k2e2, k2));
        T ez, p1, p2;
        etd_phi<T>(rmul(ell, co.k1), ez, p1, p2);
        C *Nb = (C *)kp.Nb;
        const T lin = radd(K.kappa0, rmul(K.k2e2, k2));
        if (MODE == CM_ETD_STAGE1) {
            const C un = bf.Un[idx];
            const C N0 = lnorm(badd(lscale(Nim, -k2), lscale(un, lin)));
            Nb[idx] = N0;
            v = badd(lscale(un, ez), lscale(N0, rmul(co.k1, p1)));
            bf.Unew[idx] = lnorm(v);
            pack = true;
        } else {
            const C ut = bf.Unew[idx];
            const C N1 = badd(lscale(Nim, -k2), lscale(ut, lin));
            v = badd(ut, lscale(bsub(N1, Nb[idx]), rmul(co.k1, p2)));
            bf.Unew[idx] = lnorm(v);
            pack = kp.flags & FCH_FL_PACK_F;
        }
    }
    if (pack) {
        Co = cscale_p2(v, K.inv_n2);
        Do = lscale(v, -mul_p2(k2, K.inv_n2));
    }
}

// column pairs per block at a compile-time size, the same rule as fch_geometry:
// max(pmin, 1024 / N), pmin = 2 for 8-byte elements and 1 for 16-byte ones
template <typename T, int LOGN> constexpr int spec_pairs()
{
    return (1024 >> LOGN) > (sizeof(T) == 4 ? 2 : 1) ? (1024 >> LOGN) : (sizeof(T) == 4 ? 2 : 1);
}

// Resident blocks per SM a compile-time pass is built for: four blocks of 256
// threads (at most 64 registers a thread) at N <= 1024, so that the 512 blocks of a
// 1024^2 pass run in one wave on the 152 SMs (with three per SM, 56 blocks would be
// left for a second wave); other sizes keep the compiler's choice.
template <int THREADS, int LOGN> constexpr int pass_min_blocks()
{
    return (LOGN > 0 && LOGN <= 10 && THREADS == 256) ? 4 : 1;
}
// The standalone transforms' column passes of 512 threads (single precision, N = 1024,
// two column pairs a block) are built for three resident blocks an SM (at most 42
// registers a thread): their launches carry many field pairs, so occupancy, not the
// wave count, is what they need.
template <int THREADS, int LOGN, int MODE> constexpr int col_min_blocks()
{
    return (THREADS == 512 && LOGN == 10 && (MODE == CM_FWD_STORE || MODE == CM_INV_LOAD))
               ? 3
               : pass_min_blocks<THREADS, LOGN>();
}

// Pair 0 of a column tile of an N-point transform (columns kx = 0 in slot s0 and
// kx = N/2 in slot s1 of a tile whose row n sits at skew(n) * nc), work item ky in [0, N/2]: rows ky and -ky of
// both columns (one row where they coincide). Each of the two columns is the
// transform of a real pair of its own, so the Hermitian split pairs row ky with row
// -ky of the same column.
template <typename T, int MODE>
__device__ __forceinline__ void pair0_item(const fch_kparams &kp, const fch_consts<T> &K, const fch_coef<T> &co,
                                           const ColBufs<typename CT<T>::t> &bf, typename CT<T>::t *tile, int N,
                                           int nc, int s0, int s1, int ky, bool inv, T *red)
{
    typedef typename CT<T>::t C;
    typedef ColTraits<MODE> TR;
    const int mky = (N - ky) & (N - 1);
    const int rk = skew(ky) * nc, rm = skew(mky) * nc;
    const int nrow = (ky == 0 || ky == (N >> 1)) ? 1 : 2;
    C za[2], zb[2];
    za[0] = tile[rk + s0];
    za[1] = tile[rm + s0];
    zb[0] = tile[rk + s1];
    zb[1] = tile[rm + s1];
    C outa[2], outb[2];
#pragma unroll
    for (int side = 0; side < 2; side++) {
        const int kx = side ? (N >> 1) : 0;
#pragma unroll
        for (int rr = 0; rr < 2; rr++) {
            if (rr >= nrow) break;
            const int kyy = rr ? mky : ky;
            const C zr = side ? zb[rr] : za[rr];
            const C zo = side ? zb[rr ^ 1] : za[rr ^ 1];
            C A = mk<C>(0, 0), B = mk<C>(0, 0);
            if (TR::FWD) {
                const C z1 = cconj(zo);
                A = cscale_p2(badd(zr, z1), (T)0.5);
                const C dm = bsub(zr, z1);
                B = mk<C>(mul_p2(dm.y, (T)0.5), mul_p2(dm.x, (T)-0.5));
            }
            C Co = mk<C>(0, 0), Do = mk<C>(0, 0);
            spec_elem<T, MODE>(kp, K, co, bf, kx, kyy, A, B, Co, Do, red);
            const C o = mk<C>(rsub(Co.x, Do.y), radd(Co.y, Do.x));
            if (side)
                outb[rr] = o;
            else
                outa[rr] = o;
        }
    }
    if (inv) {
        tile[rk + s0] = outa[0];
        tile[rk + s1] = outb[0];
        if (nrow == 2) {
            tile[rm + s0] = outa[1];
            tile[rm + s1] = outb[1];
        }
    }
}

// LOGN > 0: the grid size is a compile-time constant (N = 2^LOGN >= 512), so the
// index arithmetic of the transforms folds into immediates; LOGN = 0 reads N and P
// from the parameters. PPT: points of a column a thread transforms (8: radix-8
// stages, nc N / 8 threads; 4, generic kernel only: radix-4 stages, twice the threads
// and half the dependent work a thread, for small grids whose passes are too few
// warps to fill the GPU; twiddles from kp.tw4).
template <typename T, int MODE, int LOGN, int PPT = 8>
__global__ void __launch_bounds__(LOGN ? ((spec_pairs<T, LOGN>() << LOGN) >> 2) : 1024,
                                  col_min_blocks<LOGN ? ((spec_pairs<T, LOGN>() << LOGN) >> 2) : 1024, LOGN, MODE>())
col_pass(const fch_kparams kp)
{
    static_assert(PPT == 8 || (PPT == 4 && LOGN == 0), "four points a thread in the generic kernel only");
    typedef typename CT<T>::t C;
    typedef ColTraits<MODE> TR;
    pdl_begin();
    if (pass_skipped(kp)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red_scratch[FCH_NRED * 32];
    const int N = LOGN ? (1 << LOGN) : kp.N, P = LOGN ? spec_pairs<T, LOGN>() : kp.P, nc = 2 * P;
    const int logN = LOGN ? LOGN : kp.logN;
    const int nthr = LOGN ? (P << LOGN) / 4 : (int)blockDim.x;
    C *tw = (C *)smem_raw;
    C *tile = tw + N;
    const int c = threadIdx.x % nc, t = threadIdx.x / nc;
    const int p0 = blockIdx.x * P;
    const fch_consts<T> &K = consts<T>(kp);
    const bool inv = TR::INV_ALWAYS || (TR::INV_OPT && (kp.flags & FCH_FL_PACK_F));
    const bool has_red = MODE == CM_SAV_PQ || MODE == CM_PSD_ITER ||
                         (MODE == CM_F_FINISH && (kp.flags & FCH_FL_AM3));
    C *Z = pair_Z<C>(kp, N);

    // per-block constants from the control block
    fch_coef<T> co;
    ColBufs<C> bf;
    bf.i0 = (const C *)pair_in(kp.in0, kp);
    bf.i1 = (const C *)pair_in(kp.in1, kp);
    bf.o0 = (C *)pair_out(kp.out0, kp);
    bf.o1 = (C *)pair_out(kp.out1, kp);
    if (kp.ctrl) {
        const fch_ctrl *cs = kp.ctrl;
        co = load_coef<T>(cs);
        bf.Un = (const C *)kp.U[cs->iu_n];
        bf.Um = (const C *)kp.U[cs->iu_m];
        bf.Unew = (C *)kp.U[cs->iu_new];
        bf.Fn = (const C *)kp.F[cs->if_n];
        bf.Fm = (const C *)kp.F[cs->if_m];
        switch (kp.src) {
        case FCH_SRC_UN: bf.src = bf.Un; bf.dst = (C *)kp.F[cs->if_n]; break;
        case 5: bf.src = bf.Um; bf.dst = (C *)kp.F[cs->if_m]; break;
        case FCH_SRC_UNEW: bf.src = bf.Unew; bf.dst = (C *)kp.F[cs->if_new]; break;
        case FCH_SRC_V: bf.src = (const C *)kp.Vb; bf.dst = nullptr; break;
        default: bf.src = (const C *)kp.in0; bf.dst = (C *)kp.out0; break;
        }
    } else {
        bf.Un = bf.Um = bf.src = bf.Fn = bf.Fm = nullptr;
        bf.Unew = bf.dst = nullptr;
        co = fch_coef<T>();
    }

    const C *twsrc = (const C *)(PPT == 8 ? kp.tw : kp.tw4);
    for (int i = threadIdx.x; i < N; i += nthr) tw[i] = ldg(twsrc + i);
    if (TR::FWD) {
        // blockDim = nc N / PPT: exactly PPT elements of the tile per thread
        C ld[PPT];
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int i = threadIdx.x + k * nthr;
            const int n = i / nc, cc = i - n * nc;
            ld[k] = Z[(long)n * N + 2 * p0 + cc];
        }
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int i = threadIdx.x + k * nthr;
            const int n = i / nc, cc = i - n * nc;
            tile[skew(n) * nc + cc] = ld[k];
        }
        fft_smem<-1, false, PPT>(tile, N, logN, nc, c, tw, t);
    } else {
        __syncthreads();
    }

    T red[FCH_NRED] = {0, 0, 0, 0};
    // spectral stage: work item (pair p, ky); pair 0 covers columns 0 and N/2
    // blockDim = 2 P N / PPT: exactly PPT / 2 work items per thread
#pragma unroll 1
    for (int it = 0; it < PPT / 2; it++) {
        const int i = threadIdx.x + it * nthr;
        const int pp = i / N, ky = i - pp * N;
        const int p = p0 + pp;
        const int s0 = 2 * pp, s1 = 2 * pp + 1;
        const int mky = (N - ky) & (N - 1);
        const int rk = skew(ky) * nc, rm = skew(mky) * nc;
        if (p > 0) {
            C A = mk<C>(0, 0), B = mk<C>(0, 0);
            if (TR::FWD) {
                const C z0 = tile[rk + s0], z1 = cconj(tile[rm + s1]);
                A = cscale_p2(badd(z0, z1), (T)0.5);
                const C dm = bsub(z0, z1);
                B = mk<C>(mul_p2(dm.y, (T)0.5), mul_p2(dm.x, (T)-0.5));
            }
            C Co = mk<C>(0, 0), Do = mk<C>(0, 0);
            spec_elem<T, MODE>(kp, K, co, bf, p, ky, A, B, Co, Do, red);
            if (inv) {
                tile[rk + s0] = mk<C>(rsub(Co.x, Do.y), radd(Co.y, Do.x));
                tile[rm + s1] = mk<C>(radd(Co.x, Do.y), rsub(Do.x, Co.y));
            }
        } else {
            if (ky > (N >> 1)) continue;
            pair0_item<T, MODE>(kp, K, co, bf, tile, N, nc, s0, s1, ky, inv, red);
        }
    }
    if (has_red) {
        block_partials<2>(red, kp.part, red_scratch);
        if (kp.tail_op >= 0) pass_tail(kp);
    }
    if (inv) {
        fft_smem<+1, false, PPT>(tile, N, logN, nc, c, tw, t);
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int i = threadIdx.x + k * nthr;
            const int n = i / nc, cc = i - n * nc;
            Z[(long)n * N + 2 * p0 + cc] = tile[skew(n) * nc + cc];
        }
    }
}

// ---------------------------------------------------------------------------
// Column pass for 16-byte elements at N = 1024 as clusters of two blocks: block
// rank r of cluster p owns column slot r of pair p (r = 0: kx, r = 1: N - kx; pair
// 0: kx = 0 and N/2), 128 threads, one column in shared memory, twiddles read from
// global memory. The spectral stage couples the pair's columns (the Hermitian split
// reads Z(kx, ky) and Z(N - kx, -ky)); each block takes half of the pair's work
// items and reaches the partner's column through distributed shared memory, with a
// cluster barrier before (forward transforms done) and after (before the inverse
// transforms, and before any block may exit while its partner still reads it).
// 1024 blocks of 128 threads fit seven to an SM: one wave over the 152 SMs at six or
// seven blocks each, where 512 blocks of a pair each leave a fifth of the SM time idle.
template <typename T, int MODE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(128, 7) col_pass_cl(const fch_kparams kp)
{
    typedef typename CT<T>::t C;
    typedef ColTraits<MODE> TR;
    namespace cg = cooperative_groups;
    pdl_begin();
    if (pass_skipped(kp)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red_scratch[FCH_NRED * 32];
    constexpr int N = 1024, LOGN = 10, NT = 128;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank(), p = blockIdx.x >> 1;
    C *tile = (C *)smem_raw;                      // own column, skewed
    C *peer = cluster.map_shared_rank(tile, rank ^ 1); // the partner's column
    const C *tw = (const C *)kp.tw;
    const fch_consts<T> &K = consts<T>(kp);
    const bool inv = TR::INV_ALWAYS || (TR::INV_OPT && (kp.flags & FCH_FL_PACK_F));
    const bool has_red = MODE == CM_SAV_PQ || MODE == CM_PSD_ITER ||
                         (MODE == CM_F_FINISH && (kp.flags & FCH_FL_AM3));
    C *Z = pair_Z<C>(kp, N);
    const int col = 2 * p + rank; // pair-layout slot of this block's column

    fch_coef<T> co;
    ColBufs<C> bf;
    bf.i0 = (const C *)pair_in(kp.in0, kp);
    bf.i1 = (const C *)pair_in(kp.in1, kp);
    bf.o0 = (C *)pair_out(kp.out0, kp);
    bf.o1 = (C *)pair_out(kp.out1, kp);
    if (kp.ctrl) {
        const fch_ctrl *cs = kp.ctrl;
        co = load_coef<T>(cs);
        bf.Un = (const C *)kp.U[cs->iu_n];
        bf.Um = (const C *)kp.U[cs->iu_m];
        bf.Unew = (C *)kp.U[cs->iu_new];
        bf.Fn = (const C *)kp.F[cs->if_n];
        bf.Fm = (const C *)kp.F[cs->if_m];
        switch (kp.src) {
        case FCH_SRC_UN: bf.src = bf.Un; bf.dst = (C *)kp.F[cs->if_n]; break;
        case 5: bf.src = bf.Um; bf.dst = (C *)kp.F[cs->if_m]; break;
        case FCH_SRC_UNEW: bf.src = bf.Unew; bf.dst = (C *)kp.F[cs->if_new]; break;
        case FCH_SRC_V: bf.src = (const C *)kp.Vb; bf.dst = nullptr; break;
        default: bf.src = (const C *)kp.in0; bf.dst = (C *)kp.out0; break;
        }
    } else {
        bf.Un = bf.Um = bf.src = bf.Fn = bf.Fm = nullptr;
        bf.Unew = bf.dst = nullptr;
        co = fch_coef<T>();
    }

    if (TR::FWD) {
        C ld[8];
#pragma unroll
        for (int k = 0; k < 8; k++) ld[k] = Z[(long)(threadIdx.x + k * NT) * N + col];
#pragma unroll
        for (int k = 0; k < 8; k++) tile[skew(threadIdx.x + k * NT)] = ld[k];
        fft_smem<-1, true>(tile, N, LOGN, 1, 0, tw, (int)threadIdx.x);
    }
    cluster.sync(); // both columns transformed (or, without a forward part, nothing read yet)

    // slot 0 / slot 1 of the pair at skewed row r: own tile or the partner's
    auto s0 = [&](int r) -> C & { return rank == 0 ? tile[skew(r)] : peer[skew(r)]; };
    auto s1 = [&](int r) -> C & { return rank == 1 ? tile[skew(r)] : peer[skew(r)]; };
    T red[FCH_NRED] = {0, 0, 0, 0};
    if (p > 0) {
        // items ky in [rank N/2, (rank + 1) N/2): rows ky of slot 0 and -ky of slot 1
#pragma unroll 1
        for (int it = 0; it < 4; it++) {
            const int ky = rank * (N / 2) + threadIdx.x + it * NT;
            const int mky = (N - ky) & (N - 1);
            C A = mk<C>(0, 0), B = mk<C>(0, 0);
            if (TR::FWD) {
                const C z0 = s0(ky), z1 = cconj(s1(mky));
                A = cscale_p2(badd(z0, z1), (T)0.5);
                const C dm = bsub(z0, z1);
                B = mk<C>(mul_p2(dm.y, (T)0.5), mul_p2(dm.x, (T)-0.5));
            }
            C Co = mk<C>(0, 0), Do = mk<C>(0, 0);
            spec_elem<T, MODE>(kp, K, co, bf, p, ky, A, B, Co, Do, red);
            if (inv) {
                s0(ky) = mk<C>(rsub(Co.x, Do.y), radd(Co.y, Do.x));
                s1(mky) = mk<C>(radd(Co.x, Do.y), rsub(Do.x, Co.y));
            }
        }
    } else {
        // pair 0: columns kx = 0 (slot 0) and kx = N/2 (slot 1), items ky in [0, N/2]
        // (rows ky and -ky of both), even ky to rank 0 and odd ky to rank 1
#pragma unroll 1
        for (int ky = rank + 2 * (int)threadIdx.x; ky <= (N >> 1); ky += 2 * NT) {
            const int mky = (N - ky) & (N - 1);
            const int nrow = (ky == 0 || ky == (N >> 1)) ? 1 : 2;
            C za[2], zb[2];
            za[0] = s0(ky);
            za[1] = s0(mky);
            zb[0] = s1(ky);
            zb[1] = s1(mky);
            C outa[2], outb[2];
#pragma unroll
            for (int side = 0; side < 2; side++) {
                const int kx = side ? (N >> 1) : 0;
#pragma unroll
                for (int rr = 0; rr < 2; rr++) {
                    if (rr >= nrow) break;
                    const int kyy = rr ? mky : ky;
                    const C zr = side ? zb[rr] : za[rr];
                    const C zo = side ? zb[rr ^ 1] : za[rr ^ 1];
                    C A = mk<C>(0, 0), B = mk<C>(0, 0);
                    if (TR::FWD) {
                        const C z1 = cconj(zo);
                        A = cscale_p2(badd(zr, z1), (T)0.5);
                        const C dm = bsub(zr, z1);
                        B = mk<C>(mul_p2(dm.y, (T)0.5), mul_p2(dm.x, (T)-0.5));
                    }
                    C Co = mk<C>(0, 0), Do = mk<C>(0, 0);
                    spec_elem<T, MODE>(kp, K, co, bf, kx, kyy, A, B, Co, Do, red);
                    const C o = mk<C>(rsub(Co.x, Do.y), radd(Co.y, Do.x));
                    if (side)
                        outb[rr] = o;
                    else
                        outa[rr] = o;
                }
            }
            if (inv) {
                s0(ky) = outa[0];
                s1(ky) = outb[0];
                if (nrow == 2) {
                    s0(mky) = outa[1];
                    s1(mky) = outb[1];
                }
            }
        }
    }
    if (has_red) {
        block_partials<2>(red, kp.part, red_scratch);
        if (kp.tail_op >= 0) pass_tail(kp);
    }
    cluster.sync(); // every write into the partner's column is done and visible
    if (inv) {
        fft_smem<+1, true>(tile, N, LOGN, 1, 0, tw, (int)threadIdx.x);
#pragma unroll
        for (int k = 0; k < 8; k++) Z[(long)(threadIdx.x + k * NT) * N + col] = tile[skew(threadIdx.x + k * NT)];
    }
}

// ---------------------------------------------------------------------------
// row pass: [inverse rows] -> pointwise stage -> [forward rows]
// Threads a compile-time row pass is built for: one row of 128 threads at N = 1024
// (seven blocks an SM with at most 73 registers a thread: the 1024 rows run in one
// wave on the 152 SMs, six or seven to an SM), N/8 at N = 2048, else 256.
template <int LOGN> constexpr int row_threads()
{
    return LOGN == 10 ? 128 : (LOGN >= 11 ? (1 << LOGN) / 8 : 256);
}
template <int LOGN> constexpr int row_min_blocks()
{
    return LOGN == 10 ? 7 : pass_min_blocks<256, LOGN>();
}

// PPT: points of a row a thread transforms (8: radix-8 stages; 4, generic kernel only:
// radix-4 stages and twice the threads, twiddles from kp.tw4), as in col_pass.
template <typename T, int MODE, int LOGN, int PPT = 8>
__global__ void __launch_bounds__(LOGN ? row_threads<LOGN>() : 256, LOGN ? row_min_blocks<LOGN>() : 1)
row_pass(const fch_kparams kp)
{
    static_assert(PPT == 8 || (PPT == 4 && LOGN == 0), "four points a thread in the generic kernel only");
    typedef typename CT<T>::t C;
    pdl_begin();
    if (pass_skipped(kp)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red_scratch[FCH_NRED * 32];
    const int N = LOGN ? (1 << LOGN) : kp.N, tps = N / PPT, SL = skewed_len(N);
    const int logN = LOGN ? LOGN : kp.logN;
    const int nthr = LOGN ? row_threads<LOGN>() : (int)blockDim.x;
    if (kp.nfft && blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(kp.nfft, (MODE == RM_R2C_LOAD || MODE == RM_C2R_STORE || MODE == RM_ENERGY) ? 2ull : 4ull);
    // twiddles stay in global memory (read-only cache): the shared memory holds
    // only the rows, so more blocks fit an SM
    const C *tw = (const C *)(PPT == 8 ? kp.tw : kp.tw4);
    C *rows = (C *)smem_raw;
    const int rpb = nthr / tps;
    const int rr = threadIdx.x / tps, t = threadIdx.x - rr * tps;
    const int y0 = blockIdx.x * rpb;
    C *Z = pair_Z<C>(kp, N);
    const bool f64io = kp.flags & FCH_FL_F64IO;
    const fch_consts<T> &K = consts<T>(kp);

    const bool direct = MODE == RM_NIMEX_DIRECT || MODE == RM_SAV_DIRECT;
    if (direct) {
        // (u*, Lap u*) = (u^n, Lap u^n) + gam [(u^n, Lap u^n) - (u^{n-1}, Lap u^{n-1})]
        // pointwise from the stored real-space slots (eq. Richardson): no inverse transform
        const fch_ctrl *cs = kp.ctrl;
        const C *Rn = (const C *)kp.Rs[cs->iu_n];
        const C *Rm = (const C *)kp.Rs[cs->iu_m];
        const T g = load_coef<T>(cs).gam;
        const bool plain = (kp.flags & FCH_FL_GAMMA0) || g == (T)0;
        for (int i = threadIdx.x; i < rpb * N; i += nthr) {
            const int r = i / N, x = i - r * N;
            const long gi = (long)(y0 + r) * N + x;
            const C zn = ldg(Rn + gi);
            rows[r * SL + skew(x)] = plain ? zn : badd(zn, lscale(bsub(zn, ldg(Rm + gi)), g));
        }
        __syncthreads();
    } else if (MODE == RM_R2C_LOAD) {
        const void *in0 = pair_in(kp.in0, kp), *in1 = pair_in(kp.in1, kp);
        for (int i = threadIdx.x; i < rpb * N; i += nthr) {
            const int r = i / N, x = i - r * N;
            const long g = (long)y0 * N + i;
            T a, b = 0;
            if (f64io) {
                a = (T)((const double *)in0)[g];
                if (in1) b = (T)((const double *)in1)[g];
            } else {
                a = (T)((const float *)in0)[g];
                if (in1) b = (T)((const float *)in1)[g];
            }
            rows[r * SL + skew(x)] = mk<C>(a, b);
        }
    } else {
        // blockDim = rpb N / PPT: each thread moves PPT / 2 pairs (kx, N-kx) of its rows
        C ld[PPT];
#pragma unroll
        for (int k = 0; k < PPT / 2; k++) {
            const int i = threadIdx.x + k * nthr;
            const int r = i / (N >> 1), pp = i - r * (N >> 1);
            const C *src = Z + (long)(y0 + r) * N + 2 * pp;
            ld[2 * k] = src[0];
            ld[2 * k + 1] = src[1];
        }
#pragma unroll
        for (int k = 0; k < PPT / 2; k++) {
            const int i = threadIdx.x + k * nthr;
            const int r = i / (N >> 1), pp = i - r * (N >> 1);
            rows[r * SL + skew(pp)] = ld[2 * k];
            rows[r * SL + skew(pp ? N - pp : (N >> 1))] = ld[2 * k + 1];
        }
        fft_smem<+1, true, PPT>(rows + rr * SL, N, logN, 1, 0, tw, t);
    }

    T red[FCH_NRED] = {0, 0, 0, 0};
    C *s = rows + rr * SL;
    const int y = y0 + rr;
    // F row pass of an adaptive trial: keep (u, Lap u) of this state in real space
    C *store = nullptr;
    if (MODE == RM_F && (kp.flags & FCH_FL_STORE_REAL)) {
        const fch_ctrl *cs = kp.ctrl;
        const int slot = kp.src == FCH_SRC_UNEW ? cs->iu_new : (kp.src == 5 ? cs->iu_m : cs->iu_n);
        store = (C *)kp.Rs[slot] + (long)y * N;
    }
    if (MODE != RM_R2C_LOAD) {
#pragma unroll 1
        for (int x = t; x < N; x += tps) {
            const C z = s[skew(x)];
            if (MODE == RM_F && store) store[x] = z;
            const T u = z.x, lu = z.y; // u and Lap u
            if (MODE == RM_C2R_STORE) {
                const long g = (long)y * N + x;
                void *out0 = pair_out(kp.out0, kp), *out1 = pair_out(kp.out1, kp);
                if (f64io) {
                    if (out0) ((double *)out0)[g] = (double)u;
                    if (out1) ((double *)out1)[g] = (double)lu;
                } else {
                    if (out0) ((float *)out0)[g] = (float)u;
                    if (out1) ((float *)out1)[g] = (float)lu;
                }
                continue;
            }
            T W, W1, W2;
            well<T>(K, u, W, W1, W2,
                    MODE == RM_SAV || MODE == RM_SAV_DIRECT || MODE == RM_ENERGY ||
                        (MODE == RM_F && (kp.flags & FCH_FL_ENERGY)));
            C o = mk<C>(0, 0);
            if (MODE == RM_NIMEX || MODE == RM_NIMEX_DIRECT) {
                // N_IMEX = [eps^2 (am - W'' + eta1) Lap u + W''W' - am^2 u - eta2 W'] + eps^2 Lap (am u - W')
                o.x = rsub(rsub(radd(rmul(rmul(K.e2, radd(rsub(K.am, W2), K.eta1)), lu), rmul(W2, W1)),
                                rmul(K.am2, u)),
                           rmul(K.eta2, W1));
                o.y = rsub(rmul(K.am, u), W1);
            } else if (MODE == RM_F || MODE == RM_ENERGY) {
                // mu = eps^2 Lap w - W'' w + eps^2 eta1 Lap u - eta2 W', w = eps^2 Lap u - W'
                const T w = rsub(rmul(K.e2, lu), W1);
                o.x = W1;
                o.y = radd(rsub(rmul(-W2, w), rmul(K.eta2, W1)), rmul(rmul(K.e2, K.eta1), lu));
                if (MODE == RM_ENERGY || (kp.flags & FCH_FL_ENERGY))
                    red[0] += (T)0.5 * w * w - K.eta2 * W + (T)0.5 * K.e2 * K.eta1 * u * lu;
            } else if (MODE == RM_SAV || MODE == RM_SAV_DIRECT) {
                // V = -eps^2 Lap (W' + zeta u) + [-eps^2 (W'' + zeta) Lap u + W' W'' - eta2 W']
                o.x = radd(W1, rmul(K.zeta, u));
                o.y = rsub(radd(rmul(rmul(-K.e2, radd(W2, K.zeta)), lu), rmul(W1, W2)), rmul(K.eta2, W1));
                red[0] += -K.e2 * lu * (W1 + K.zeta * u) + (T)0.5 * W1 * W1 - K.eta2 * W;
            }
            s[skew(x)] = o;
        }
    }
    const bool has_red = MODE == RM_SAV || MODE == RM_SAV_DIRECT || MODE == RM_ENERGY ||
                         (MODE == RM_F && (kp.flags & FCH_FL_ENERGY));
    if (has_red) {
        block_partials<1>(red, kp.part, red_scratch);
        if (kp.tail_op >= 0) pass_tail(kp);
    }
    if (MODE == RM_C2R_STORE || MODE == RM_ENERGY) return;

    fft_smem<-1, true, PPT>(rows + rr * SL, N, logN, 1, 0, tw, t);
#pragma unroll
    for (int k = 0; k < PPT / 2; k++) {
        const int i = threadIdx.x + k * nthr;
        const int r = i / (N >> 1), pp = i - r * (N >> 1);
        C *dst = Z + (long)(y0 + r) * N + 2 * pp;
        dst[0] = rows[r * SL + skew(pp)];
        dst[1] = rows[r * SL + skew(pp ? N - pp : (N >> 1))];
    }
}

} // namespace fch
