// fch_warpfft.cuh -- single-precision passes for N = 1024 built on a warp-level
// transform: one warp owns one length-1024 sequence, 32 elements per lane.
//
// With n = n1 + 32 n2 and k = k2 + 32 k1,
//   X[k2 + 32 k1] = sum_{n1} W32^{n1 k1} W1024^{n1 k2} sum_{n2} W32^{n2 k2} x[n1 + 32 n2],
// so lane n1 transforms its 32 elements x[n1 + 32 n2] in registers, multiplies by
// W1024^{n1 k2}, the warp transposes through a padded 32 x 33 shared buffer, and
// lane k2 transforms again, ending with X[k2 + 32 k1] in register k1. The output
// layout of an inverse transform (lane = x mod 32, register = x / 32) is the input
// layout of a forward one, so the pointwise stage of a row pass runs on registers
// between the two transforms. Only __syncwarp is needed inside a transform.
#pragma once
#include "fch_kernels.cuh"

namespace fch {

// cos(pi j / 16), j = 0..16
__device__ __forceinline__ float cos16f(int j)
{
    switch (j) {
    case 0: return 1.0f;
    case 1: return 0.9807852804032304f;
    case 2: return 0.9238795325112867f;
    case 3: return 0.8314696123025452f;
    case 4: return 0.7071067811865476f;
    case 5: return 0.5555702330196023f;
    case 6: return 0.38268343236508984f;
    case 7: return 0.19509032201612833f;
    case 8: return 0.0f;
    default: return -cos16f(16 - j);
    }
}

// x * W_M^k with W_M = exp(DIR 2 pi i / M), M | 32, k < M/2 (compile-time after unrolling)
template <int M, int DIR> __device__ __forceinline__ float2 twm(int k, float2 x)
{
    const int j = (32 / M) * k; // angle = pi j / 16
    if (j == 0) return x;
    if (j == 8) return rot<DIR>(x);
    const float c = cos16f(j), s = j <= 8 ? cos16f(8 - j) : cos16f(j - 8);
    return cmul(x, mk<float2>(c, DIR * s));
}

// In-register radix-2 transform of length M, natural order in and out.
template <int M, int DIR> struct RegFFT {
    __device__ __forceinline__ static void run(float2 *v)
    {
        float2 e[M / 2], o[M / 2];
#pragma unroll
        for (int i = 0; i < M / 2; i++) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        RegFFT<M / 2, DIR>::run(e);
        RegFFT<M / 2, DIR>::run(o);
#pragma unroll
        for (int k = 0; k < M / 2; k++) {
            const float2 t = twm<M, DIR>(k, o[k]);
            v[k] = cadd(e[k], t);
            v[k + M / 2] = csub(e[k], t);
        }
    }
};
template <int DIR> struct RegFFT<1, DIR> {
    __device__ __forceinline__ static void run(float2 *) {}
};

// Length-1024 transform by one warp. In: v[n2] = x[lane + 32 n2]. Out: v[k1] =
// X[lane + 32 k1]. buf: this warp's 32 x 33 shared buffer. tw2[k2 * 32 + n1] =
// exp(-2 pi i n1 k2 / 1024) (read through the read-only cache).
template <int DIR>
__device__ __forceinline__ void warp_fft1024(float2 *v, float2 *buf, const float2 *__restrict__ tw2, int lane)
{
    RegFFT<32, DIR>::run(v);
#pragma unroll
    for (int k2 = 1; k2 < 32; k2++) {
        float2 w = __ldg(tw2 + k2 * 32 + lane);
        if (DIR > 0) w = cconj(w);
        v[k2] = cmul(v[k2], w);
    }
    __syncwarp();
#pragma unroll
    for (int k2 = 0; k2 < 32; k2++) buf[k2 * 33 + lane] = v[k2];
    __syncwarp();
#pragma unroll
    for (int n1 = 0; n1 < 32; n1++) v[n1] = buf[lane * 33 + n1];
    RegFFT<32, DIR>::run(v);
}

// pointwise stage of a row pass on (u, Lap u); returns the pair to transform forward
template <int MODE>
__device__ __forceinline__ float2 pointwise(const fch_kparams &kp, const fch_consts<float> &K, float u,
                                            float lu, float *red)
{
    float W, W1, W2;
    well<float>(K, u, W, W1, W2,
                MODE == RM_SAV || MODE == RM_SAV_DIRECT || MODE == RM_ENERGY ||
                    (MODE == RM_F && (kp.flags & FCH_FL_ENERGY)));
    float2 o = mk<float2>(0.f, 0.f);
    if (MODE == RM_NIMEX || MODE == RM_NIMEX_DIRECT) {
        o.x = K.e2 * (K.am - W2 + K.eta1) * lu + W2 * W1 - K.am2 * u - K.eta2 * W1;
        o.y = K.am * u - W1;
    } else if (MODE == RM_F || MODE == RM_ENERGY) {
        const float w = K.e2 * lu - W1;
        o.x = W1;
        o.y = -W2 * w - K.eta2 * W1 + K.e2 * K.eta1 * lu;
        if (MODE == RM_ENERGY || (kp.flags & FCH_FL_ENERGY))
            red[0] += 0.5f * w * w - K.eta2 * W + 0.5f * K.e2 * K.eta1 * u * lu;
    } else if (MODE == RM_SAV || MODE == RM_SAV_DIRECT) {
        o.x = W1 + K.zeta * u;
        o.y = -K.e2 * (W2 + K.zeta) * lu + W1 * W2 - K.eta2 * W1;
        red[0] += -K.e2 * lu * (W1 + K.zeta * u) + 0.5f * W1 * W1 - K.eta2 * W;
    }
    return o;
}

// row pass, N = 1024, single precision: one warp (= one block) per row
template <int MODE>
// (the standalone transforms' row passes, launched over many field pairs, are built
// for sixteen resident warps an SM: at most 128 registers a thread)
__global__ void __launch_bounds__(32, (MODE == RM_R2C_LOAD || MODE == RM_C2R_STORE) ? 16 : 1)
row_pass_w(const fch_kparams kp)
{
    typedef float2 C;
    pdl_begin();
    if (pass_skipped(kp)) return;
    constexpr int N = 1024;
    __shared__ __align__(16) C buf[33 * 32];
    __shared__ double red_scratch[FCH_NRED * 32];
    const int lane = threadIdx.x, y = blockIdx.x;
    if (kp.nfft && blockIdx.x == 0 && lane == 0)
        atomicAdd(kp.nfft, (MODE == RM_R2C_LOAD || MODE == RM_C2R_STORE || MODE == RM_ENERGY) ? 2ull : 4ull);
    const C *tw2 = (const C *)kp.tw2;
    const bool f64io = kp.flags & FCH_FL_F64IO;
    C *row = pair_Z<C>(kp, N) + (long)y * N;
    C v[32];
    if (MODE == RM_NIMEX_DIRECT || MODE == RM_SAV_DIRECT) {
        // (u*, Lap u*) pointwise from the stored real-space slots (eq. Richardson)
        const fch_ctrl *cs = kp.ctrl;
        const C *Rn = (const C *)kp.Rs[cs->iu_n] + (long)y * N;
        const C *Rm = (const C *)kp.Rs[cs->iu_m] + (long)y * N;
        const float g = cs->cof.gam;
        const bool plain = (kp.flags & FCH_FL_GAMMA0) || g == 0.f;
#pragma unroll
        for (int n2 = 0; n2 < 32; n2++) {
            const C zn = __ldg(Rn + lane + 32 * n2);
            v[n2] = plain ? zn : cadd(zn, cscale(csub(zn, __ldg(Rm + lane + 32 * n2)), g));
        }
    } else if (MODE == RM_R2C_LOAD && !f64io && kp.in1) {
        // two float fields (the common case, without a branch per element)
        const float *a = (const float *)pair_in(kp.in0, kp) + (long)y * N + lane;
        const float *b = (const float *)pair_in(kp.in1, kp) + (long)y * N + lane;
#pragma unroll
        for (int n2 = 0; n2 < 32; n2++) v[n2] = mk<C>(__ldcs(a + 32 * n2), __ldcs(b + 32 * n2));
    } else if (MODE == RM_R2C_LOAD) {
        const void *in0 = pair_in(kp.in0, kp), *in1 = pair_in(kp.in1, kp);
#pragma unroll
        for (int n2 = 0; n2 < 32; n2++) {
            const long g = (long)y * N + lane + 32 * n2;
            float a, b = 0.f;
            if (f64io) {
                a = (float)((const double *)in0)[g];
                if (in1) b = (float)((const double *)in1)[g];
            } else {
                a = ((const float *)in0)[g];
                if (in1) b = ((const float *)in1)[g];
            }
            v[n2] = mk<C>(a, b);
        }
    } else {
        // pairs (kx, N-kx) of the pair-layout row into natural order, 16 per lane
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const int p = lane + 32 * j;
            const float4 z = __ldcg((const float4 *)(row + 2 * p));
            buf[p] = mk<C>(z.x, z.y);
            buf[p ? N - p : N / 2] = mk<C>(z.z, z.w);
        }
        __syncwarp();
#pragma unroll
        for (int n2 = 0; n2 < 32; n2++) v[n2] = buf[lane + 32 * n2];
        warp_fft1024<+1>(v, buf, tw2, lane);
    }

    float red[FCH_NRED] = {0.f, 0.f, 0.f, 0.f};
    C *store = nullptr;
    if (MODE == RM_F && (kp.flags & FCH_FL_STORE_REAL)) {
        const fch_ctrl *cs = kp.ctrl;
        const int slot = kp.src == FCH_SRC_UNEW ? cs->iu_new : (kp.src == 5 ? cs->iu_m : cs->iu_n);
        store = (C *)kp.Rs[slot] + (long)y * N;
    }
    if (MODE == RM_C2R_STORE && !f64io && kp.out0 && kp.out1) {
        // two float fields (the common case, without a branch per element)
        float *o0 = (float *)pair_out(kp.out0, kp) + (long)y * N + lane;
        float *o1 = (float *)pair_out(kp.out1, kp) + (long)y * N + lane;
#pragma unroll
        for (int k1 = 0; k1 < 32; k1++) {
            __stcs(o0 + 32 * k1, v[k1].x);
            __stcs(o1 + 32 * k1, v[k1].y);
        }
        return;
    }
    if (MODE == RM_F && store) {
#pragma unroll
        for (int k1 = 0; k1 < 32; k1++) store[lane + 32 * k1] = v[k1];
    }
    if (MODE != RM_R2C_LOAD) {
        const fch_consts<float> &K = kp.cf;
#pragma unroll
        for (int k1 = 0; k1 < 32; k1++) {
            const int x = lane + 32 * k1;
            const float u = v[k1].x, lu = v[k1].y;
            if (MODE == RM_C2R_STORE) {
                const long g = (long)y * N + x;
                void *out0 = pair_out(kp.out0, kp), *out1 = pair_out(kp.out1, kp);
                if (f64io) {
                    if (out0) ((double *)out0)[g] = (double)u;
                    if (out1) ((double *)out1)[g] = (double)lu;
                } else {
                    if (out0) ((float *)out0)[g] = u;
                    if (out1) ((float *)out1)[g] = lu;
                }
                continue;
            }
            v[k1] = pointwise<MODE>(kp, K, u, lu, red);
        }
    }
    const bool has_red = MODE == RM_SAV || MODE == RM_SAV_DIRECT || MODE == RM_ENERGY ||
                         (MODE == RM_F && (kp.flags & FCH_FL_ENERGY));
    if (has_red) {
        block_partials<1>(red, kp.part, red_scratch);
        if (kp.tail_op >= 0) pass_tail(kp);
    }
    if (MODE == RM_C2R_STORE || MODE == RM_ENERGY) return;

    warp_fft1024<-1>(v, buf, tw2, lane);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < 32; k1++) buf[lane + 32 * k1] = v[k1];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 16; j++) {
        const int p = lane + 32 * j;
        const C z0 = buf[p], z1 = buf[p ? N - p : N / 2];
        __stcg((float4 *)(row + 2 * p), make_float4(z0.x, z0.y, z1.x, z1.y));
    }
}

// column pass, N = 1024, single precision: P = 2 column pairs (4 columns) per
// block, one warp per column; the tile rows are padded to 5 elements so a warp
// reading one column of consecutive rows hits distinct banks.
template <int MODE>
__global__ void __launch_bounds__(128) col_pass_w(const fch_kparams kp)
{
    typedef float2 C;
    typedef ColTraits<MODE> TR;
    pdl_begin();
    if (pass_skipped(kp)) return;
    constexpr int N = 1024, P = 2, RS = 5, NT = 128; // 2P = 4 columns, rows padded to 5
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red_scratch[FCH_NRED * 32];
    C *tile = (C *)smem_raw;           // N x RS
    C *bufs = tile + N * RS;           // 4 x (32 x 33)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C *buf = bufs + warp * 33 * 32;
    const int p0 = blockIdx.x * P;
    const fch_consts<float> &K = kp.cf;
    const C *tw2 = (const C *)kp.tw2;
    const bool inv = TR::INV_ALWAYS || (TR::INV_OPT && (kp.flags & FCH_FL_PACK_F));
    const bool has_red = MODE == CM_SAV_PQ || MODE == CM_PSD_ITER ||
                         (MODE == CM_F_FINISH && (kp.flags & FCH_FL_AM3));
    C *Z = pair_Z<C>(kp, N);

    fch_coef<float> co = fch_coef<float>();
    ColBufs<C> bf = ColBufs<C>();
    bf.i0 = (const C *)pair_in(kp.in0, kp);
    bf.i1 = (const C *)pair_in(kp.in1, kp);
    bf.o0 = (C *)pair_out(kp.out0, kp);
    bf.o1 = (C *)pair_out(kp.out1, kp);
    if (kp.ctrl) {
        const fch_ctrl *cs = kp.ctrl;
        co = load_coef<float>(cs);
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
    }

    if (TR::FWD) {
        // 4096 tile elements, 32 per thread, in 4 batches of 8 loads in flight
#pragma unroll
        for (int b = 0; b < 4; b++) {
            C ld[8];
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int i = threadIdx.x + (b * 8 + k) * NT;
                ld[k] = __ldcg(Z + (long)(i >> 2) * N + 2 * p0 + (i & 3));
            }
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int i = threadIdx.x + (b * 8 + k) * NT;
                tile[(i >> 2) * RS + (i & 3)] = ld[k];
            }
        }
        __syncthreads();
        C v[32];
#pragma unroll
        for (int n2 = 0; n2 < 32; n2++) v[n2] = tile[(lane + 32 * n2) * RS + warp];
        warp_fft1024<-1>(v, buf, tw2, lane);
#pragma unroll
        for (int k1 = 0; k1 < 32; k1++) tile[(lane + 32 * k1) * RS + warp] = v[k1];
    }
    __syncthreads();

    float red[FCH_NRED] = {0.f, 0.f, 0.f, 0.f};
    for (int i = threadIdx.x; i < P * N; i += NT) {
        const int pp = i / N, ky = i - pp * N;
        const int p = p0 + pp;
        const int s0 = 2 * pp, s1 = 2 * pp + 1;
        const int mky = (N - ky) & (N - 1);
        const int rk = ky * RS, rm = mky * RS;
        if (p > 0) {
            C A = mk<C>(0.f, 0.f), B = mk<C>(0.f, 0.f);
            if (TR::FWD) {
                const C z0 = tile[rk + s0], z1 = cconj(tile[rm + s1]);
                A = cscale(cadd(z0, z1), 0.5f);
                const C dm = csub(z0, z1);
                B = mk<C>(0.5f * dm.y, -0.5f * dm.x);
            }
            C Co = mk<C>(0.f, 0.f), Do = mk<C>(0.f, 0.f);
            spec_elem<float, MODE>(kp, K, co, bf, p, ky, A, B, Co, Do, red);
            if (inv) {
                tile[rk + s0] = mk<C>(Co.x - Do.y, Co.y + Do.x);
                tile[rm + s1] = mk<C>(Co.x + Do.y, Do.x - Co.y);
            }
        } else {
            if (ky > (N >> 1)) continue;
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
                    C A = mk<C>(0.f, 0.f), B = mk<C>(0.f, 0.f);
                    if (TR::FWD) {
                        const C z1 = cconj(zo);
                        A = cscale(cadd(zr, z1), 0.5f);
                        const C dm = csub(zr, z1);
                        B = mk<C>(0.5f * dm.y, -0.5f * dm.x);
                    }
                    C Co = mk<C>(0.f, 0.f), Do = mk<C>(0.f, 0.f);
                    spec_elem<float, MODE>(kp, K, co, bf, kx, kyy, A, B, Co, Do, red);
                    const C o = mk<C>(Co.x - Do.y, Co.y + Do.x);
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
    }
    if (has_red) {
        block_partials<2>(red, kp.part, red_scratch);
        if (kp.tail_op >= 0) pass_tail(kp);
    }
    if (inv) {
        __syncthreads();
        C v[32];
#pragma unroll
        for (int n2 = 0; n2 < 32; n2++) v[n2] = tile[(lane + 32 * n2) * RS + warp];
        warp_fft1024<+1>(v, buf, tw2, lane);
#pragma unroll
        for (int k1 = 0; k1 < 32; k1++) tile[(lane + 32 * k1) * RS + warp] = v[k1];
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; k++) {
            const int i = threadIdx.x + k * NT;
            __stcg(Z + (long)(i >> 2) * N + 2 * p0 + (i & 3), tile[(i >> 2) * RS + (i & 3)]);
        }
    }
}

} // namespace fch
