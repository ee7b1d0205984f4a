// fch_fno.cu -- a Fourier neural operator (FNO) that predicts the initial iterate
// of the PSD iteration (Sec. 3.3 leaves v_0 free): forward pass, backward pass,
// mean-square loss and Adam, all in FP32 on this library's own kernels and its
// own batched real 2D transforms (no cuFFT, no cuBLAS).
//
// Network (restating Li et al.'s Fourier neural operator): two input channels per
// point, a = (u^n, (u* - u^n)/s), u* the extrapolation of eq. (Richardson), s the
// RMS of u* - u^n; output y = predicted (u^{n+1} - u*)/s.
//   h_0 = P a + bP;  h_{l+1} = act_l(W_l h_l + b_l + S_l(h_l));  y = Q2 GELU(Q1 h_L + bQ1) + bQ2
//   S(h)[o] = C2R(H(sum_i R[m][o][i] R2C(h[i])(m)))  over the retained modes m,
// act = GELU (x Phi(x), with erf) except after the last layer (identity). Retained
// modes: kx in [0, M), ky in {0..M-1} and {N-M+1..N-1}, weight index
// kx (2M-1) + kyi with ky = kyi (kyi < M) or -(kyi - M + 1). H replaces the kx = 0
// column of the retained modes by its Hermitian part (Y(ky) + conj Y(-ky))/2, the
// part a real inverse transform reads. The backward pass uses the adjoints: of C2R
// on retained modes w(kx)/N^2 R2C (w = 1 at kx = 0, else 2), of R2C
// N^2 C2R(v(kx) .), v = 1 at kx = 0, else 1/2, both through H at kx = 0.
//
// Layouts: fields [b][c][y][x] (channel fields contiguous, n x n each); spectra as
// the library's transforms write them, kx-major [field][kx][ky]; parameters one
// flat float vector in the order P, bP, {W_l, b_l, R_l} for each layer, Q1, bQ1,
// Q2, bQ2, with R_l as [K][W_out][W_in] complex (re, im interleaved).
// Weight gradients are summed over points in a fixed order (per-block partials,
// then one pass over the blocks), so a backward pass is deterministic.
#include <cuda.h> // CUtensorMap and its enums (the encoder is fetched at run time)
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../../include/fch.h"
#include "fch_internal.h"
#include "fch_tc.cuh"
#include "fch_tmap.h"

namespace {

constexpr int kMaxW2 = 128;  // hidden channels of the projection

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// Two floats in one 64-bit register, for the packed FP32 instructions of this GPU
// (add / mul / fma .rn.f32x2: both lanes in one instruction).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 x2(float a, float b)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 x2_split(f32x2 v)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return make_float2(a, b);
}
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// GELU of two values at once for the tensor-core inference kernels. erf comes from the
// rational approximation of Abramowitz and Stegun, Handbook of Mathematical Functions,
// eq. 7.1.28: for u >= 0, 1 - erf(u) = p(u)^-16 with p(u) = 1 + a1 u + ... + a6 u^6,
// |error| <= 3e-7. With h = x/2 and a = |h| (u = a sqrt 2),
//   GELU(x) = x/2 (1 + erf(x / sqrt 2)) = (a + h) - a p(u)^-16,
// which for x < 0 is -a p^-16 itself (no cancellation); a is capped in the last term. One reciprocal per value (with
// a Newton step), the rest packed: about twelve instructions a value against the
// library erff's branches. In float, p^-16 carries ~2e-6 relative rounding: GELU
// within 0.5 |x| 3e-6. Its outputs feed bfloat16 operands (relative rounding 2^-9) or
// FP32 sums with bfloat16 weights.
__device__ __forceinline__ f32x2 gelu_as2(f32x2 x)
{
    const f32x2 h = x2_mul(x, x2(0.5f, 0.5f));
    const f32x2 a = h & 0x7FFFFFFF7FFFFFFFull; // |h|
    // the tail term takes |h| capped at 5.65 (u = |h| sqrt 2 at most 8, where 1 - erf is
    // 1e-29 and p stays finite for the Newton step)
    const float2 as = x2_split(a);
    const f32x2 acn = x2(-fminf(as.x, 5.65f), -fminf(as.y, 5.65f));
    const f32x2 u = x2_mul(acn, x2(-1.41421356237309505f, -1.41421356237309505f));
    f32x2 p = x2_fma(x2(0.0000430638f, 0.0000430638f), u, x2(0.0002765672f, 0.0002765672f));
    p = x2_fma(p, u, x2(0.0001520143f, 0.0001520143f));
    p = x2_fma(p, u, x2(0.0092705272f, 0.0092705272f));
    p = x2_fma(p, u, x2(0.0422820123f, 0.0422820123f));
    p = x2_fma(p, u, x2(0.0705230784f, 0.0705230784f));
    p = x2_fma(p, u, x2(1.0f, 1.0f)); // in [1, 22]
    const float2 ps = x2_split(p);
    f32x2 r = x2(rcp_approx(ps.x), rcp_approx(ps.y));
    r = x2_fma(r, x2_fma(p ^ 0x8000000080000000ull, r, x2(1.0f, 1.0f)), r); // Newton: r (2 - p r)
    r = x2_mul(r, r);
    r = x2_mul(r, r);
    r = x2_mul(r, r);
    r = x2_mul(r, r); // p^-16
    return x2_fma(acn, r, x2_add(a, h));
}

// ky of retained-mode row kyi
__device__ __forceinline__ int mode_ky(int kyi, int M, int n) { return kyi < M ? kyi : n - (kyi - M + 1); }

// a weight as float: the forward pass reads FP32 weights, or (inference with
// fch_fno_set_bf16) their bfloat16 copy; sums stay in FP32 either way
__device__ __forceinline__ float wld(const float *p, long i) { return p[i]; }
__device__ __forceinline__ float wld(const __nv_bfloat16 *p, long i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float2 wld2(const float *p, long i) { return make_float2(p[2 * i], p[2 * i + 1]); }
__device__ __forceinline__ float2 wld2(const __nv_bfloat16 *p, long i)
{
    return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(p)[i]);
}

__global__ void fno_to_bf16(const float *__restrict__ w, __nv_bfloat16 *__restrict__ out, long cnt)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt) out[t] = __float2bfloat16_rn(w[t]);
}

// h0[b][c][p] = sum_i P[c][i] a[b][i][p] + bP[c] (the weights staged in shared memory)
template <typename WT>
__global__ void fno_lift(const float *__restrict__ a, const WT *__restrict__ P, const WT *__restrict__ bP,
                         float *__restrict__ h, int B, int n2, int W, int cin)
{
    __shared__ float ps[32 * 4], bs[32];
    for (int i = threadIdx.x; i < W * cin; i += blockDim.x) ps[i] = wld(P, i);
    for (int i = threadIdx.x; i < W; i += blockDim.x) bs[i] = wld(bP, i);
    __syncthreads();
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)B * n2) return;
    const int b = (int)(t / n2), p = (int)(t - (long)b * n2);
    float in[4];
    for (int i = 0; i < cin; i++) in[i] = a[((long)b * cin + i) * n2 + p];
    for (int c = 0; c < W; c++) {
        float acc = bs[c];
        for (int i = 0; i < cin; i++) acc += ps[c * cin + i] * in[i];
        h[((long)b * W + c) * n2 + p] = acc;
    }
}

// the same with the channel counts fixed at compile time (the tensor-core forward
// pass): loops unrolled, each output channel one multiply-add chain and one store at a
// running pointer
template <typename WT, int W, int CIN>
__global__ void __launch_bounds__(256) fno_lift_t(const float *__restrict__ a, const WT *__restrict__ P,
                                                  const WT *__restrict__ bP, float *__restrict__ h, long pts, int n2)
{
    __shared__ float ps[W * CIN], bs[W];
    for (int i = threadIdx.x; i < W * CIN; i += blockDim.x) ps[i] = wld(P, i);
    for (int i = threadIdx.x; i < W; i += blockDim.x) bs[i] = wld(bP, i);
    __syncthreads();
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pts) return;
    const long b = t / n2, p = t - b * n2;
    float in[CIN];
#pragma unroll
    for (int i = 0; i < CIN; i++) in[i] = __ldcs(a + (b * CIN + i) * n2 + p);
    float *hp = h + b * W * n2 + p;
#pragma unroll
    for (int c = 0; c < W; c++) {
        float acc = bs[c];
#pragma unroll
        for (int i = 0; i < CIN; i++) acc = fmaf(ps[c * CIN + i], in[i], acc);
        *hp = acc;
        hp += n2;
    }
}

// z[b][c][p] = sum_j Wl[c][j] h[b][j][p] + bl[c] + s[b][c][p];  out = act(z)
// (W, the channel count, is a compile-time constant so the per-point channel
// vectors stay in registers)
template <int W, typename WT = float>
__global__ void fno_pointwise(const float *__restrict__ h, const float *__restrict__ s,
                              const WT *__restrict__ Wl, const WT *__restrict__ bl, float *__restrict__ z,
                              float *__restrict__ out, int B, int n2, int act)
{
    __shared__ float ws[W * W];
    __shared__ float bs[W];
    for (int i = threadIdx.x; i < W * W; i += blockDim.x) ws[i] = wld(Wl, i);
    for (int i = threadIdx.x; i < W; i += blockDim.x) bs[i] = wld(bl, i);
    __syncthreads();
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)B * n2) return;
    const int b = (int)(t / n2), p = (int)(t - (long)b * n2);
    float in[W];
#pragma unroll
    for (int j = 0; j < W; j++) in[j] = h[((long)b * W + j) * n2 + p];
    for (int c = 0; c < W; c++) {
        const long o = ((long)b * W + c) * n2 + p;
        float acc = bs[c] + s[o];
#pragma unroll
        for (int j = 0; j < W; j++) acc += ws[c * W + j] * in[j];
        z[o] = acc;
        out[o] = act ? gelu(acc) : acc;
    }
}

// y[b][p] = bQ2 + sum_d Q2[d] GELU(bQ1[d] + sum_c Q1[d][c] h[b][c][p])
template <int W, typename WT = float>
__global__ void fno_project(const float *__restrict__ h, const WT *__restrict__ Q1, const WT *__restrict__ bQ1,
                            const WT *__restrict__ Q2, const WT *__restrict__ bQ2, float *__restrict__ y,
                            int B, int n2, int W2)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)B * n2) return;
    const int b = (int)(t / n2), p = (int)(t - (long)b * n2);
    float in[W];
#pragma unroll
    for (int c = 0; c < W; c++) in[c] = h[((long)b * W + c) * n2 + p];
    float acc = wld(bQ2, 0);
    for (int d = 0; d < W2; d++) {
        float zq = wld(bQ1, d);
#pragma unroll
        for (int c = 0; c < W; c++) zq += wld(Q1, d * W + c) * in[c];
        acc += wld(Q2, d) * gelu(zq);
    }
    y[(long)b * n2 + p] = acc;
}

// Backward of the projection and the loss mean((y - target)^2): per point dy, the
// hidden activations q, their gradients dzq and dh = Q1^T dzq; also (y - target)^2
// per point for the loss.
template <int W>
__global__ void fno_project_bwd(const float *__restrict__ h, const float *__restrict__ Q1,
                                const float *__restrict__ bQ1, const float *__restrict__ Q2,
                                const float *__restrict__ y, const float *__restrict__ target, float *__restrict__ dy,
                                float *__restrict__ q, float *__restrict__ dzq, float *__restrict__ dh,
                                float *__restrict__ sq, int B, int n2, int W2, float scale)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)B * n2) return;
    const int b = (int)(t / n2), p = (int)(t - (long)b * n2);
    float in[W], g[W];
#pragma unroll
    for (int c = 0; c < W; c++) {
        in[c] = h[((long)b * W + c) * n2 + p];
        g[c] = 0.f;
    }
    const float r = y[t] - target[t];
    const float d = scale * r;
    dy[t] = d;
    sq[t] = r * r;
    for (int k = 0; k < W2; k++) {
        float zq = bQ1[k];
#pragma unroll
        for (int c = 0; c < W; c++) zq += Q1[k * W + c] * in[c];
        const long o = ((long)b * W2 + k) * n2 + p;
        q[o] = gelu(zq);
        const float dz = d * Q2[k] * gelu_grad(zq);
        dzq[o] = dz;
#pragma unroll
        for (int c = 0; c < W; c++) g[c] += Q1[k * W + c] * dz;
    }
#pragma unroll
    for (int c = 0; c < W; c++) dh[((long)b * W + c) * n2 + p] = g[c];
}

// Backward of a Fourier layer's pointwise part: dz = dout act'(z); dh = Wl^T dz.
template <int W>
__global__ void fno_pointwise_bwd(const float *__restrict__ dout, const float *__restrict__ z,
                                  const float *__restrict__ Wl, float *__restrict__ dz, float *__restrict__ dh,
                                  int B, int n2, int act)
{
    __shared__ float ws[W * W];
    for (int i = threadIdx.x; i < W * W; i += blockDim.x) ws[i] = Wl[i];
    __syncthreads();
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)B * n2) return;
    const int b = (int)(t / n2), p = (int)(t - (long)b * n2);
    float g[W], acc[W];
#pragma unroll
    for (int c = 0; c < W; c++) {
        const long o = ((long)b * W + c) * n2 + p;
        g[c] = act ? dout[o] * gelu_grad(z[o]) : dout[o];
        dz[o] = g[c];
        acc[c] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < W; c++)
#pragma unroll
        for (int j = 0; j < W; j++) acc[j] += ws[c * W + j] * g[c];
#pragma unroll
    for (int j = 0; j < W; j++) dh[((long)b * W + j) * n2 + p] = acc[j];
}

// Y[b W + o](m) = sum_i R[m][o][i] X[b W + i](m) on the retained modes, written
// through H at kx = 0 (work item: one mode, or at kx = 0 the pair ky, -ky).
// X and Y are spectra [field][kx][ky]; S = (n/2 + 1) n complex per field.
template <typename WT>
__global__ void fno_mix(const float2 *__restrict__ X, const WT *__restrict__ R, float2 *__restrict__ Y,
                        int B, int W, int M, int n)
{
    const int items = M + (M - 1) * (2 * M - 1);
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)B * W * items) return;
    const int it = (int)(t % items), o = (int)((t / items) % W), b = (int)(t / ((long)items * W));
    const long S = (long)(n / 2 + 1) * n;
    const int K2 = 2 * M - 1;
    auto mixed = [&](int kx, int kyi) {
        const int ky = mode_ky(kyi, M, n);
        const long r = ((long)(kx * K2 + kyi) * W + o) * W; // complex index of R[m][o][0]
        float re = 0.f, im = 0.f;
        for (int i = 0; i < W; i++) {
            const float2 x = X[((long)b * W + i) * S + (long)kx * n + ky];
            const float2 w = wld2(R, r + i);
            re += w.x * x.x - w.y * x.y;
            im += w.x * x.y + w.y * x.x;
        }
        return make_float2(re, im);
    };
    float2 *Yf = Y + ((long)b * W + o) * S;
    if (it < M) { // kx = 0: ky = it and -it
        const int ky = it;
        const float2 yp = mixed(0, ky);
        if (ky == 0) {
            Yf[0] = make_float2(yp.x, 0.f);
        } else {
            const float2 ym = mixed(0, ky + M - 1);
            const float2 hh = make_float2(0.5f * (yp.x + ym.x), 0.5f * (yp.y - ym.y));
            Yf[ky] = hh;
            Yf[n - ky] = make_float2(hh.x, -hh.y);
        }
    } else {
        const int j = it - M, kx = 1 + j / K2, kyi = j % K2;
        Yf[(long)kx * n + mode_ky(kyi, M, n)] = mixed(kx, kyi);
    }
}

// ---------------------------------------------------------------------------
// Inference with the spectral convolutions as truncated DFTs over the retained
// modes (fch_fno_set_bf16(f, 2)): for a layer input h[b][i][y][x],
//   X[b][i][y][kx] = sum_x h (cos - i sin)(2 pi kx x / n),  kx < M     (rows)
//   Y[b][i][kyi][kx] = sum_y X e^{-2 pi i ky y / n}                     (columns)
//   Z[b][o][kyi][kx] = sum_i R[m][o][i] Y[b][i][kyi][kx], m = kx (2M-1) + kyi
//   V[b][o][y][kx] = sum_kyi Z e^{+2 pi i ky y / n}
//   S[b][o][y][x] = (1/n^2) sum_kx w(kx) Re(V e^{+2 pi i kx x / n}),  w(0) = 1, else 2
// which is the C2R of the retained spectrum through H (the real part of the kx = 0
// sum is what H keeps), without the full 2D transforms of every channel. The row
// DFT, a GEMM with K = n, runs on the tensor cores (tcgen05, BF16 operands, FP32
// sums); the other stages are small and run as plain kernels in FP32.

constexpr int kTcRows = 128, kTcLBO = 144, kTcSBO = 8 * kTcLBO, kTcNB = 32;
constexpr uint64_t kTcBound = 1000000000ull; // ns an mbarrier wait lasts before a kernel gives up

// Bt[j][x] (bf16): cos(2 pi j x / n) for j < 16, -sin(2 pi (j - 16) x / n) for j >= 16;
// tw[kx][x] (float2): (cos, sin)(2 pi kx x / n), kx < 16
__global__ void fno_dft_tables(__nv_bfloat16 *__restrict__ Bt, float2 *__restrict__ tw, int n)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 16L * n) return;
    const int kx = (int)(t / n), x = (int)(t - (long)kx * n);
    double sn, cs;
    sincospi(2.0 * (double)((kx * (long)x) % n) / (double)n, &sn, &cs);
    Bt[(long)kx * n + x] = __double2bfloat16(cs);
    Bt[(long)(16 + kx) * n + x] = __double2bfloat16(-sn);
    tw[(long)kx * n + x] = make_float2((float)cs, (float)sn);
}

// X[r][kx] = (D[r][kx], D[r][16 + kx]) with D = bf16(h) Bt^T over K = n: one CTA of 128
// threads per 128 rows, K in chunks of 32. A chunk of the FP32 rows arrives as one 2D
// tile of a tensor map over h (the TMA engine: 128 rows x 32 floats, two chunks ahead,
// completion counted in bytes on the stage's `full` mbarrier; rows beyond R read as
// zero); the threads round it to bfloat16 into the core-matrix layout of the stage's A
// tile (see fch_tc.cuh) and copy the table's chunk; thread 0 issues two K = 16 MMAs
// into a 128 x 32 FP32 accumulator in tensor memory and commits them to the stage's
// `mma` mbarrier, which guards the stage's tiles. A wait that runs out of time (1 s) sets
// *err; the CTA then stops, waits (bounded) for the loads and MMAs it issued, frees its
// tensor memory and returns.
constexpr int kDftKc = 32;                                  // K of a chunk (two K = 16 MMAs)
// 160 bytes between K cores: a half warp's 8-byte stores (two rows x four cores x two
// halves, one 128-byte wavefront) then fall on 16 distinct bank pairs, and a quarter
// warp's 16-byte stores of the table (two rows x four cores) on 8 distinct bank quads
constexpr int kDftLBO = 160;
constexpr int kDftSBO = (kDftKc / 8) * kDftLBO;             // 8-row groups of four K cores
constexpr int kRawBytes = kTcRows * kDftKc * 4;             // one tile of FP32 rows (16 KB)
constexpr int kAtBytes = (kTcRows / 8) * kDftSBO, kBtBytes = (kTcNB / 8) * kDftSBO;
// the stages, then the mbarriers and the tensor-memory address, and 1 KB of slack to
// align the tiles to 1024 bytes
constexpr int kRowdftSmem = 2 * kRawBytes + 2 * kAtBytes + 2 * kBtBytes + 64 + 1024;

__global__ void __launch_bounds__(128) fno_rowdft_tc(const __grid_constant__ CUtensorMap tmap,
                                                     const __nv_bfloat16 *__restrict__ Bt, float2 *__restrict__ X,
                                                     int R, int n, int *err)
{
    extern __shared__ unsigned char dsm_raw[];
    // the TMA destination wants an aligned tile: the window's start rounded up to 1024 B
    unsigned char *dsm = dsm_raw + ((1024u - (fch::tc::smem_u32(dsm_raw) & 1023u)) & 1023u);
    unsigned char *raw = dsm, *sA = dsm + 2 * kRawBytes, *sB = sA + 2 * kAtBytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + 2 * kBtBytes), *mmab = full + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mmab + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long row0 = (long)blockIdx.x * kTcRows;
    const int nch = n / kDftKc;
    if (warp == 0) {
        fch::tc::tmem_alloc(tslot, 32);
        fch::tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < 2; i++) {
            fch::tc::mbar_init(&full[i], 1);
            fch::tc::mbar_init(&mmab[i], 1);
        }
        fch::tc::mbar_init_fence();
    }
    fch::tc::fence_before_sync();
    __syncthreads();
    fch::tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    auto fetch = [&](int c) { // thread 0
        fch::tc::mbar_expect_tx(&full[c & 1], kRawBytes);
        fch::tc::tma_load_2d(raw + (c & 1) * kRawBytes, &tmap, c * kDftKc, (int)row0, &full[c & 1]);
    };
    if (tid == 0)
        for (int c = 0; c < 2 && c < nch; c++) fetch(c);
    constexpr uint32_t idesc = fch::tc::idesc_bf16_f32(kTcRows, kTcNB);
    bool ok = true;
    int fetched = nch < 2 ? nch : 2, issued = 0;
    for (int c = 0; c < nch; c++) {
        const int st = c & 1;
        ok = fch::tc::mbar_wait(&full[st], (uint32_t)((c >> 1) & 1), kTcBound);
        if (ok && c >= 2) ok = fch::tc::mbar_wait(&mmab[st], (uint32_t)(((c >> 1) - 1) & 1), kTcBound);
        if (!__syncthreads_and(ok)) break;
        // raw -> A: 16 bytes (4 floats) a thread and step, a warp reading four whole rows
        const unsigned char *rs = raw + st * kRawBytes;
        unsigned char *a = sA + st * kAtBytes;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int idx = tid + 128 * i, r = idx >> 3, q = idx & 7, kc = q >> 1, half = q & 1;
            const float4 f4 = *reinterpret_cast<const float4 *>(rs + r * (kDftKc * 4) + q * 16);
            __nv_bfloat162 b0 = __floats2bfloat162_rn(f4.x, f4.y), b1 = __floats2bfloat162_rn(f4.z, f4.w);
            const uint2 v = make_uint2(*reinterpret_cast<uint32_t *>(&b0), *reinterpret_cast<uint32_t *>(&b1));
            *reinterpret_cast<uint2 *>(a + (r >> 3) * kDftSBO + kc * kDftLBO + (r & 7) * 16 + half * 8) = v;
        }
        unsigned char *bb = sB + st * kBtBytes;
        {
            const int r = tid >> 2, kc = tid & 3; // 32 table rows x 4 K cores
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(Bt + (long)r * n + (long)c * kDftKc + kc * 8));
            *reinterpret_cast<uint4 *>(bb + (r >> 3) * kDftSBO + kc * kDftLBO + (r & 7) * 16) = v;
        }
        // the tiles go to the tensor core and the raw stage back to the copy engine
        fch::tc::fence_async_smem();
        fch::tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            if (c + 2 < nch) {
                fetch(c + 2);
                fetched = c + 3;
            }
            fch::tc::fence_after_sync();
            const uint32_t sa = fch::tc::smem_u32(a), sb = fch::tc::smem_u32(bb);
#pragma unroll
            for (int k = 0; k < kDftKc / 16; k++)
                fch::tc::mma_bf16(tmem, fch::tc::smem_desc(sa + 2 * k * kDftLBO, kDftLBO, kDftSBO),
                                  fch::tc::smem_desc(sb + 2 * k * kDftLBO, kDftLBO, kDftSBO), idesc,
                                  (c | k) != 0);
            fch::tc::mma_commit(&mmab[st]);
        }
        issued = c + 1;
    }
    // the last commit covers every MMA issued; tiles fetched beyond what was consumed (an
    // early stop) are waited for before the CTA's shared memory goes away
    bool done = true;
    if (issued > 0)
        done = fch::tc::mbar_wait(&mmab[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1), kTcBound);
    if (tid == 0)
        for (int c = issued; c < fetched; c++)
            fch::tc::mbar_wait(&full[c & 1], (uint32_t)((c >> 1) & 1), kTcBound);
    ok = __syncthreads_and(ok && done && issued == nch);
    fch::tc::fence_after_sync();
    if (ok) {
        float v[32];
        fch::tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
        const long r = row0 + warp * 32 + lane;
        if (r < R) {
            float4 *dst = reinterpret_cast<float4 *>(X + r * 16);
#pragma unroll
            for (int k = 0; k < 8; k++)
                dst[k] = make_float4(v[2 * k], v[16 + 2 * k], v[2 * k + 1], v[16 + 2 * k + 1]);
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    fch::tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) fch::tc::tmem_dealloc(tmem, 32);
}

// launch of fno_rowdft_tc over R rows of n floats at h (n a multiple of 32), with its
// tensor map and dynamic shared memory (the limit raised once)
cudaError_t launch_rowdft_tc(const float *h, const __nv_bfloat16 *Bt, float2 *X, long R, int n, int *err,
                             cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(fno_rowdft_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowdftSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap m;
    // R rows of n floats, tiles of 128 rows x 32 floats, zero past the last row
    const cudaError_t e = fch_tmap_f32_2d(&m, h, (uint64_t)n, (uint64_t)R, (uint64_t)n * 4, kDftKc, kTcRows);
    if (e != cudaSuccess) return e;
    fno_rowdft_tc<<<(unsigned)((R + kTcRows - 1) / kTcRows), 128, kRowdftSmem, s>>>(m, Bt, X, (int)R, n, err);
    return cudaGetLastError();
}

// Y[f][kyi][kx] = sum_y X[f][y][kx] e^{-2 pi i ky y / n}: one block per (field f, kx).
// The column X[f][.][kx] and the twiddle table (cos, sin)(2 pi j / n) go to shared
// memory; eight threads share each retained ky (thread j of the eight sums the y = j
// mod 8), then three shuffle levels add the eight partial sums in a fixed order.
// n a multiple of 128; dynamic shared memory: 2 n float2.
template <int MM>
__global__ void __launch_bounds__(256) fno_coldft(const float2 *__restrict__ X, const float2 *__restrict__ tw1,
                                                  float2 *__restrict__ Y, int n)
{
    constexpr int K2 = 2 * MM - 1;
    static_assert(K2 <= 32, "eight threads a retained ky in 256 threads");
    extern __shared__ float2 cd_sm[];
    float2 *col = cd_sm, *tw = cd_sm + n;
    const int f = blockIdx.x, kx = blockIdx.y, tid = threadIdx.x;
    for (int y = tid; y < n; y += 256) {
        col[y] = X[((long)f * n + y) * 16 + kx];
        tw[y] = tw1[y];
    }
    __syncthreads();
    const int k = tid >> 3, j = tid & 7; // k = K2 (the last eight threads) computes nothing kept
    const int ky = k < MM ? k : n - (k - MM + 1);
    // the twiddle of y + 8 is the twiddle of y times (cos, sin)(2 pi 8 ky / n): a table
    // read starts each run of 16 such steps (the reads of a warp would meet bank
    // conflicts at stride ky in the table; the products stay within ~16 roundings)
    const float2 step = tw[(8 * ky) & (n - 1)];
    float2 acc = make_float2(0.f, 0.f);
    for (int y0 = j; y0 < n; y0 += 128) {
        float2 w = tw[(ky * y0) & (n - 1)];
#pragma unroll
        for (int r = 0; r < 16; r++) {
            const float2 v = col[y0 + 8 * r];
            acc.x = fmaf(v.x, w.x, fmaf(v.y, w.y, acc.x));
            acc.y = fmaf(v.y, w.x, fmaf(-v.x, w.y, acc.y));
            w = make_float2(fmaf(w.x, step.x, -w.y * step.y), fmaf(w.x, step.y, w.y * step.x));
        }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (j == 0 && k < K2) Y[((long)f * K2 + k) * MM + kx] = acc;
}

// Z[b][o][kyi][kx] = sum_i R[m][o][i] Y[b][i][kyi][kx], m = kx (2M-1) + kyi
template <typename WT>
__global__ void fno_mix_modes(const float2 *__restrict__ Y, const WT *__restrict__ R, float2 *__restrict__ Z,
                              int B, int W, int M)
{
    const int K2 = 2 * M - 1, K = M * K2;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)B * W * K) return;
    const int q = (int)(t % K), o = (int)((t / K) % W), b = (int)(t / ((long)K * W));
    const int kyi = q / M, kx = q - kyi * M, m = kx * K2 + kyi;
    float re = 0.f, im = 0.f;
    for (int i = 0; i < W; i++) {
        const float2 x = Y[(((long)b * W + i) * K2 + kyi) * M + kx];
        const float2 w = wld2(R, ((long)m * W + o) * W + i);
        re += w.x * x.x - w.y * x.y;
        im += w.x * x.y + w.y * x.x;
    }
    Z[(((long)b * W + o) * K2 + kyi) * M + kx] = make_float2(re, im);
}

// V[f][y][kx] = sum_kyi Z[f][kyi][kx] e^{+2 pi i ky y / n}: one block per (field f, 64
// rows y); Z[f] and the twiddle table (cos, sin)(2 pi j / n) in shared memory, thread
// (y, kx) four outputs. Dynamic shared memory: n float2.
template <int MM>
__global__ void __launch_bounds__(256) fno_icoldft(const float2 *__restrict__ Z, const float2 *__restrict__ tw1,
                                                   float2 *__restrict__ V, long nf, int n)
{
    constexpr int K2 = 2 * MM - 1, YB = 64;
    __shared__ float2 zs[K2 * MM];
    extern __shared__ float2 ic_tw[];
    const int nyb = n / YB;
    const long f = blockIdx.x / nyb;
    const int y0 = (int)(blockIdx.x % nyb) * YB, tid = threadIdx.x;
    for (int i = tid; i < K2 * MM; i += 256) zs[i] = Z[f * K2 * MM + i];
    for (int i = tid; i < n; i += 256) ic_tw[i] = tw1[i];
    __syncthreads();
    for (int i = tid; i < YB * MM; i += 256) {
        const int y = y0 + i / MM, kx = i % MM;
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int k = 0; k < K2; k++) {
            const int ky = k < MM ? k : n - (k - MM + 1);
            const float2 z = zs[k * MM + kx], w = ic_tw[(ky * y) & (n - 1)];
            re = fmaf(z.x, w.x, fmaf(-z.y, w.y, re));
            im = fmaf(z.x, w.y, fmaf(z.y, w.x, im));
        }
        V[(f * n + y) * 16 + kx] = make_float2(re, im);
    }
}

// 8 floats rounded to bfloat16 (nearest even), packed as one 16-byte core row
__device__ __forceinline__ uint4 pack8_bf16(const float *f)
{
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        __nv_bfloat162 b = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t *>(&b);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}
// row r, K-core kc of a core-layout tile (see fch_tc.cuh)
__device__ __forceinline__ void core_store(unsigned char *tile, int r, int kc, uint4 v)
{
    *reinterpret_cast<uint4 *>(tile + (r >> 3) * kTcSBO + kc * kTcLBO + (r & 7) * 16) = v;
}

// set up (tensor memory, mbarrier) and tear down of the one-tile tensor-core kernels
struct TcTile {
    uint32_t tmem;
};

// The pointwise layer on the tensor cores: for the 128 points x of one row segment
// (thread t, TMEM lane t), z[o] = sum_j W[o][j] h[j] + b[o] + S[o] with S the inverse
// x DFT of V, as one MMA chain with K = W + 32:
//   A[t][:] = (bf16 h[b][j][y][x], j < W | bf16 cos(2 pi kx x/n), kx < 16 | bf16 sin(...))
//   B[o][:] = (W[o][j] | bf16(w(kx)/n^2 Re V[o][y][kx]) | bf16(-w(kx)/n^2 Im V[o][y][kx]))
// D = A B^T (128 x W, FP32 in tensor memory); out = act(D + b).
template <int W>
__global__ void __launch_bounds__(128) fno_pw_tc(const float *__restrict__ h, const float2 *__restrict__ V,
                                                 const float2 *__restrict__ tw, const __nv_bfloat16 *__restrict__ Wl,
                                                 const __nv_bfloat16 *__restrict__ bl, float *__restrict__ out,
                                                 int n, int act, int *err)
{
    constexpr int K = W + 32, NKC = K / 8;
    __shared__ __align__(128) unsigned char sA[16 * kTcSBO];
    __shared__ __align__(128) unsigned char sB[(W / 8) * kTcSBO];
    __shared__ float bs[W];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int segs = n >> 7, seg = blockIdx.x % segs, y = blockIdx.x / segs, b = blockIdx.y;
    const int x = seg * 128 + tid;
    const long n2 = (long)n * n, p = (long)y * n + x;
    if (warp == 0) {
        fch::tc::tmem_alloc(&tslot, 32);
        fch::tc::tmem_relinquish();
    }
    if (tid == 0) {
        fch::tc::mbar_init(&bar, 1);
        fch::tc::mbar_init_fence();
    }
    float f[8];
    const float *hp = h + (long)b * W * n2 + p;
#pragma unroll
    for (int kc = 0; kc < W / 8; kc++) {
#pragma unroll
        for (int e = 0; e < 8; e++) {
            f[e] = *hp;
            hp += n2;
        }
        core_store(sA, tid, kc, pack8_bf16(f));
    }
#pragma unroll
    for (int part = 0; part < 2; part++)
#pragma unroll
        for (int kc = 0; kc < 2; kc++) {
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const float2 t = tw[(long)(kc * 8 + e) * n + x];
                f[e] = part ? t.y : t.x;
            }
            core_store(sA, tid, W / 8 + 2 * part + kc, pack8_bf16(f));
        }
    const float sc = 1.0f / ((float)n * (float)n);
    for (int i = tid; i < W * NKC; i += 128) {
        const int o = i / NKC, kc = i - o * NKC;
        uint4 v;
        if (kc < W / 8) {
            v = *reinterpret_cast<const uint4 *>(Wl + o * W + kc * 8); // already bf16
        } else {
            const int part = (kc - W / 8) >> 1, k0 = ((kc - W / 8) & 1) * 8;
            const float2 *Vr = V + (((long)b * W + o) * n + y) * 16;
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const int k = k0 + e;
                const float wk = (k == 0 ? 1.f : 2.f) * sc;
                const float2 vv = Vr[k];
                f[e] = part ? -wk * vv.y : wk * vv.x;
            }
            v = pack8_bf16(f);
        }
        core_store(sB, o, kc, v);
    }
    for (int i = tid; i < W; i += 128) bs[i] = __bfloat162float(bl[i]);
    fch::tc::fence_async_smem();
    fch::tc::fence_before_sync();
    __syncthreads();
    fch::tc::fence_after_sync();
    const uint32_t tmem = tslot;
    if (tid == 0) {
        constexpr uint32_t idesc = fch::tc::idesc_bf16_f32(128, W);
        const uint32_t sa = fch::tc::smem_u32(sA), sb = fch::tc::smem_u32(sB);
#pragma unroll
        for (int k = 0; k < K / 16; k++)
            fch::tc::mma_bf16(tmem, fch::tc::smem_desc(sa + 2 * k * kTcLBO, kTcLBO, kTcSBO),
                              fch::tc::smem_desc(sb + 2 * k * kTcLBO, kTcLBO, kTcSBO), idesc, k != 0);
        fch::tc::mma_commit(&bar);
    }
    const bool ok = __syncthreads_and(fch::tc::mbar_wait(&bar, 0, kTcBound));
    fch::tc::fence_after_sync();
    if (ok) {
        float v[32];
        fch::tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
        float *op = out + (long)b * W * n2 + p;
        if (act) {
#pragma unroll
            for (int o = 0; o < W; o += 2) {
                const float2 g2 = x2_split(gelu_as2(x2_add(x2(v[o], v[o + 1]), x2(bs[o], bs[o + 1]))));
                op[0] = g2.x;
                op[n2] = g2.y;
                op += 2 * n2;
            }
        } else {
#pragma unroll
            for (int o = 0; o < W; o++) {
                *op = v[o] + bs[o];
                op += n2;
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    fch::tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) fch::tc::tmem_dealloc(tmem, 32);
}

// The projection on the tensor cores: for 128 points (thread t, TMEM lane t),
// zq = Q1 bf16(h) + bQ1 as D = A B^T with A[t][:] = bf16 h[b][c][p] (K = W) and
// B = Q1 (W2 x W), then y = bQ2 + sum_d Q2[d] GELU(zq[d]) in the epilogue.
template <int W>
__global__ void __launch_bounds__(128) fno_proj_tc(const float *__restrict__ h, const __nv_bfloat16 *__restrict__ Q1,
                                                   const __nv_bfloat16 *__restrict__ bQ1,
                                                   const __nv_bfloat16 *__restrict__ Q2,
                                                   const __nv_bfloat16 *__restrict__ bQ2, float *__restrict__ y,
                                                   long pts, int n2, int W2, int *err)
{
    __shared__ __align__(128) unsigned char sA[16 * kTcSBO];
    __shared__ __align__(128) unsigned char sB[(kMaxW2 / 8) * kTcSBO];
    __shared__ __align__(16) float bq[kMaxW2], q2[kMaxW2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long g = (long)blockIdx.x * 128 + tid;
    const bool live = g < pts;
    const long b = live ? g / n2 : 0, p = live ? g - b * n2 : 0;
    const uint32_t ncols = W2 <= 32 ? 32 : (W2 <= 64 ? 64 : 128);
    if (warp == 0) {
        fch::tc::tmem_alloc(&tslot, ncols);
        fch::tc::tmem_relinquish();
    }
    if (tid == 0) {
        fch::tc::mbar_init(&bar, 1);
        fch::tc::mbar_init_fence();
    }
    float f[8];
    const float *hp = h + b * W * n2 + p;
#pragma unroll
    for (int kc = 0; kc < W / 8; kc++) {
#pragma unroll
        for (int e = 0; e < 8; e++) {
            f[e] = live ? __ldcs(hp) : 0.f;
            hp += n2;
        }
        core_store(sA, tid, kc, pack8_bf16(f));
    }
    for (int i = tid; i < W2 * (W / 8); i += 128) {
        const int d = i / (W / 8), kc = i - d * (W / 8);
        core_store(sB, d, kc, *reinterpret_cast<const uint4 *>(Q1 + d * W + kc * 8));
    }
    for (int i = tid; i < W2; i += 128) {
        bq[i] = __bfloat162float(bQ1[i]);
        q2[i] = __bfloat162float(Q2[i]);
    }
    fch::tc::fence_async_smem();
    fch::tc::fence_before_sync();
    __syncthreads();
    fch::tc::fence_after_sync();
    const uint32_t tmem = tslot;
    if (tid == 0) {
        const uint32_t idesc = fch::tc::idesc_bf16_f32(128, W2);
        const uint32_t sa = fch::tc::smem_u32(sA), sb = fch::tc::smem_u32(sB);
#pragma unroll
        for (int k = 0; k < W / 16; k++)
            fch::tc::mma_bf16(tmem, fch::tc::smem_desc(sa + 2 * k * kTcLBO, kTcLBO, kTcSBO),
                              fch::tc::smem_desc(sb + 2 * k * kTcLBO, kTcLBO, kTcSBO), idesc, k != 0);
        fch::tc::mma_commit(&bar);
    }
    const bool ok = __syncthreads_and(fch::tc::mbar_wait(&bar, 0, kTcBound));
    fch::tc::fence_after_sync();
    if (ok) {
        // W2 is a multiple of 16: sixteen accumulator columns at a time, the biases and
        // the second layer's weights four at a time from shared memory
        f32x2 acc = x2(__bfloat162float(bQ2[0]), 0.f); // two partial sums, added at the end
        for (int c0 = 0; c0 < W2; c0 += 16) {
            float v[16];
            fch::tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int d = 0; d < 16; d += 4) {
                const float4 b4 = *reinterpret_cast<const float4 *>(bq + c0 + d);
                const float4 q4 = *reinterpret_cast<const float4 *>(q2 + c0 + d);
                acc = x2_fma(x2(q4.x, q4.y), gelu_as2(x2_add(x2(v[d], v[d + 1]), x2(b4.x, b4.y))), acc);
                acc = x2_fma(x2(q4.z, q4.w), gelu_as2(x2_add(x2(v[d + 2], v[d + 3]), x2(b4.z, b4.w))), acc);
            }
        }
        const float2 a2 = x2_split(acc);
        if (live) y[g] = a2.x + a2.y;
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    fch::tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) fch::tc::tmem_dealloc(tmem, ncols);
}

// dY[b][o][m] (compact, K modes a field) = H(w(kx)/n^2 Fd(m)), Fd = R2C of the
// spectral branch's output gradient
__global__ void fno_dY(const float2 *__restrict__ Fd, float2 *__restrict__ dY, int B, int W, int M, int n)
{
    const int K2 = 2 * M - 1, K = M * K2;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)B * W * K) return;
    const int m = (int)(t % K);
    const long f = t / K;
    const long S = (long)(n / 2 + 1) * n;
    const int kx = m / K2, kyi = m % K2, ky = mode_ky(kyi, M, n);
    const float inv = 1.0f / ((float)n * (float)n);
    const float2 *F = Fd + f * S;
    float2 v;
    if (kx == 0) {
        const float2 a = F[ky], c = F[(n - ky) % n]; // w = 1 at kx = 0
        v = make_float2(0.5f * (a.x + c.x) * inv, 0.5f * (a.y - c.y) * inv);
    } else {
        const float2 a = F[(long)kx * n + ky];
        v = make_float2(2.f * a.x * inv, 2.f * a.y * inv);
    }
    dY[t] = v;
}

// dR[m][o][i] = sum_b dY[b][o][m] conj(X[b][i](m))
__global__ void fno_dR(const float2 *__restrict__ dY, const float2 *__restrict__ X, float2 *__restrict__ dR,
                       int B, int W, int M, int n)
{
    const int K2 = 2 * M - 1, K = M * K2;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)K * W * W) return;
    const int i = (int)(t % W), o = (int)((t / W) % W), m = (int)(t / ((long)W * W));
    const long S = (long)(n / 2 + 1) * n;
    const int kx = m / K2, ky = mode_ky(m % K2, M, n);
    float re = 0.f, im = 0.f;
    for (int b = 0; b < B; b++) {
        const float2 d = dY[((long)b * W + o) * K + m];
        const float2 x = X[((long)b * W + i) * S + (long)kx * n + ky];
        re += d.x * x.x + d.y * x.y;
        im += d.y * x.x - d.x * x.y;
    }
    dR[t] = make_float2(re, im);
}

// Z[b W + i](m) = n^2 v(kx) sum_o conj(R[m][o][i]) dY[b][o][m], through H at kx = 0,
// so that C2R(Z) is the gradient of the layer input through the spectral branch
__global__ void fno_dX(const float2 *__restrict__ dY, const float2 *__restrict__ R, float2 *__restrict__ Z,
                       int B, int W, int M, int n)
{
    const int K2 = 2 * M - 1, K = M * K2;
    const int items = M + (M - 1) * K2;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)B * W * items) return;
    const int it = (int)(t % items), i = (int)((t / items) % W), b = (int)(t / ((long)items * W));
    const long S = (long)(n / 2 + 1) * n;
    const float n2 = (float)n * (float)n;
    auto back = [&](int m) {
        float re = 0.f, im = 0.f;
        for (int o = 0; o < W; o++) {
            const float2 d = dY[((long)b * W + o) * K + m];
            const float2 w = R[((long)m * W + o) * W + i];
            re += w.x * d.x + w.y * d.y;
            im += w.x * d.y - w.y * d.x;
        }
        return make_float2(re, im);
    };
    float2 *Zf = Z + ((long)b * W + i) * S;
    if (it < M) { // kx = 0, v = 1
        const int ky = it;
        const float2 dp = back(ky);
        if (ky == 0) {
            Zf[0] = make_float2(n2 * dp.x, 0.f);
        } else {
            const float2 dm = back(ky + M - 1);
            const float2 hh = make_float2(0.5f * n2 * (dp.x + dm.x), 0.5f * n2 * (dp.y - dm.y));
            Zf[ky] = hh;
            Zf[n - ky] = make_float2(hh.x, -hh.y);
        }
    } else { // v = 1/2
        const int j = it - M, kx = 1 + j / K2, kyi = j % K2;
        const float2 d = back(kx * K2 + kyi);
        Zf[(long)kx * n + mode_ky(kyi, M, n)] = make_float2(0.5f * n2 * d.x, 0.5f * n2 * d.y);
    }
}

__global__ void fno_add(float *__restrict__ a, const float *__restrict__ b, long cnt)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt) a[t] += b[t];
}

// Weight-gradient partials: G[a][c] = sum over points of A(a, pt) Bm(c, pt), with
// A(a, (b, p)) = A[(b CA + a) n2 + p] (Bm alike; Bm null: 1). Block k sums points
// [k chunk, (k+1) chunk) in order into part[k][a nb + c].
__global__ void fno_wgrad_part(const float *__restrict__ A, int CA, int na, const float *__restrict__ Bm, int CB,
                               int nb, int n2, long npts, int chunk, float *__restrict__ part)
{
    extern __shared__ float sm[];
    float *sa = sm, *sb = sm + (long)na * 32;
    const int nout = na * nb;
    const long p0 = (long)blockIdx.x * chunk;
    float acc[8];
    for (int k = 0; k < 8; k++) acc[k] = 0.f;
    for (long q0 = p0; q0 < p0 + chunk && q0 < npts; q0 += 32) {
        const int cnt = (int)min((long)32, min(p0 + chunk, npts) - q0);
        __syncthreads();
        for (int e = threadIdx.x; e < na * 32; e += blockDim.x) {
            const int a = e / 32, k = e % 32;
            float v = 0.f;
            if (k < cnt) {
                const long pt = q0 + k, b = pt / n2, p = pt - b * n2;
                v = A[(b * CA + a) * n2 + p];
            }
            sa[e] = v;
        }
        for (int e = threadIdx.x; e < nb * 32; e += blockDim.x) {
            const int c = e / 32, k = e % 32;
            float v = 0.f;
            if (k < cnt) {
                const long pt = q0 + k, b = pt / n2, p = pt - b * n2;
                v = Bm ? Bm[(b * CB + c) * n2 + p] : 1.f;
            }
            sb[e] = v;
        }
        __syncthreads();
        for (int k = 0; k < 8; k++) {
            const int o = threadIdx.x + k * blockDim.x;
            if (o >= nout) break;
            const int a = o / nb, c = o % nb;
            float s = 0.f;
            for (int j = 0; j < cnt; j++) s += sa[a * 32 + j] * sb[c * 32 + j];
            acc[k] += s;
        }
    }
    for (int k = 0; k < 8; k++) {
        const int o = threadIdx.x + k * blockDim.x;
        if (o < nout) part[(long)blockIdx.x * nout + o] = acc[k];
    }
}

__global__ void fno_wgrad_sum(const float *__restrict__ part, int nblk, int nout, float *__restrict__ out)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nout) return;
    float s = 0.f;
    for (int k = 0; k < nblk; k++) s += part[(long)k * nout + o];
    out[o] = s;
}

// Adam (Kingma & Ba), bias-corrected, on the flat parameter vector
__global__ void fno_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                         float *__restrict__ v, long cnt, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const float gg = g[t];
    const float mm = b1 * m[t] + (1.f - b1) * gg;
    const float vv = b2 * v[t] + (1.f - b2) * gg * gg;
    m[t] = mm;
    v[t] = vv;
    w[t] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

} // namespace

struct fch_fno {
    int W, L, M, W2, cin, K;
    cudaStream_t stream;
    size_t np;
    float *params, *grads, *am, *av;
    long long adam_t;
    // per (B, n) buffers
    int B, n;
    fch_fft_plan *plan;
    float *h;     // (L + 1) x [B][W][n^2]
    float *z;     // L x [B][W][n^2]
    float2 *X;    // L x [B W][(n/2+1) n]
    float2 *Ysp;  // [B W][(n/2+1) n], zero outside the retained modes
    float2 *Fd;   // [B W][(n/2+1) n]
    float2 *dY;   // [B][W][K]
    float *s;     // [B][W][n^2]
    float *dh, *dz, *tmp; // [B][W][n^2]
    float *q, *dzq;       // [B][W2][n^2]
    float *y, *dy, *sq;   // [B][n^2]
    float *part;          // weight-gradient partials
    const float *a;       // the last forward pass's input
    bool have_fwd;
    __nv_bfloat16 *pbf;   // bfloat16 copy of params (fch_fno_set_bf16), else null
    bool fwd_bf16;        // the last forward pass read the bfloat16 copy
    // truncated-DFT spectral convolutions (fch_fno_set_bf16(f, 2)): tables for tc_n,
    // work arrays for (tc_B, tc_n), the device error flag of the tensor-core kernel
    bool tc;
    int tc_B, tc_n;
    __nv_bfloat16 *tc_Bt; // [32][n]
    float2 *tc_tw;        // [16][n]
    float2 *tc_X, *tc_V;  // [B W n][16]
    float2 *tc_Y, *tc_Z;  // [B W][2M-1][M]
    int *tc_err;
    double *hsum;
    char err[256];
};

namespace {

size_t offset_of(const fch_fno *f, int what, int l)
{
    // what: 0 P, 1 bP, 2 W_l, 3 b_l, 4 R_l, 5 Q1, 6 bQ1, 7 Q2, 8 bQ2
    const size_t W = f->W, lay = W * W + W + (size_t)f->K * W * W * 2;
    const size_t base = W * f->cin + W;
    switch (what) {
    case 0: return 0;
    case 1: return W * f->cin;
    case 2: return base + l * lay;
    case 3: return base + l * lay + W * W;
    case 4: return base + l * lay + W * W + W;
    case 5: return base + f->L * lay;
    case 6: return base + f->L * lay + (size_t)f->W2 * W;
    case 7: return base + f->L * lay + (size_t)f->W2 * W + f->W2;
    default: return base + f->L * lay + (size_t)f->W2 * W + 2 * f->W2;
    }
}

void free_buffers(fch_fno *f)
{
    void *bufs[] = {f->h, f->z, f->X, f->Ysp, f->Fd, f->dY, f->s, f->dh, f->dz, f->tmp,
                    f->q, f->dzq, f->y, f->dy, f->sq, f->part};
    for (void *b : bufs)
        if (b) cudaFree(b);
    f->h = f->z = f->s = f->dh = f->dz = f->tmp = f->q = f->dzq = f->y = f->dy = f->sq = f->part = nullptr;
    f->X = f->Ysp = f->Fd = f->dY = nullptr;
    if (f->plan) fch_fft_plan_destroy(f->plan);
    f->plan = nullptr;
    f->B = f->n = 0;
}

fch_status ensure_buffers(fch_fno *f, int B, int n)
{
    if (f->B == B && f->n == n) return FCH_OK;
    free_buffers(f);
    const size_t n2 = (size_t)n * n, fld = (size_t)B * f->W * n2, S = (size_t)(n / 2 + 1) * n;
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    al((void **)&f->h, (f->L + 1) * fld * 4);
    al((void **)&f->z, f->L * fld * 4);
    al((void **)&f->X, (size_t)f->L * B * f->W * S * 8);
    al((void **)&f->Ysp, (size_t)B * f->W * S * 8);
    al((void **)&f->Fd, (size_t)B * f->W * S * 8);
    al((void **)&f->dY, (size_t)B * f->W * f->K * 8);
    al((void **)&f->s, fld * 4);
    al((void **)&f->dh, fld * 4);
    al((void **)&f->dz, fld * 4);
    al((void **)&f->tmp, fld * 4);
    al((void **)&f->q, (size_t)B * f->W2 * n2 * 4);
    al((void **)&f->dzq, (size_t)B * f->W2 * n2 * 4);
    al((void **)&f->y, (size_t)B * n2 * 4);
    al((void **)&f->dy, (size_t)B * n2 * 4);
    al((void **)&f->sq, (size_t)B * n2 * 4);
    al((void **)&f->part, (size_t)1024 * 2048 * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->Ysp, 0, (size_t)B * f->W * S * 8, f->stream);
    if (e != cudaSuccess) {
        snprintf(f->err, sizeof(f->err), "fch_fno: %s", cudaGetErrorString(e));
        free_buffers(f);
        return e == cudaErrorMemoryAllocation ? FCH_ENOMEM : FCH_ECUDA;
    }
    fch_status s = fch_fft_plan_create(n, 1, f->stream, &f->plan);
    if (s != FCH_OK) {
        free_buffers(f);
        return s;
    }
    f->B = B;
    f->n = n;
    return FCH_OK;
}

inline unsigned grid(long cnt, int bs) { return (unsigned)((cnt + bs - 1) / bs); }

// launch kernel<W> for the channel count W (8, 16 or 32)
#define WDISPATCH(Wv, kern, g, b, st, ...)                                                          \
    do {                                                                                           \
        if ((Wv) == 8)                                                                             \
            kern<8><<<(g), (b), 0, (st)>>>(__VA_ARGS__);                                           \
        else if ((Wv) == 16)                                                                       \
            kern<16><<<(g), (b), 0, (st)>>>(__VA_ARGS__);                                          \
        else                                                                                       \
            kern<32><<<(g), (b), 0, (st)>>>(__VA_ARGS__);                                          \
    } while (0)

// the same for a kernel templated on the channel count and the weight type
#define WDISPATCH_T(Wv, kern, WT, g, b, st, ...)                                                   \
    do {                                                                                           \
        if ((Wv) == 8)                                                                             \
            kern<8, WT><<<(g), (b), 0, (st)>>>(__VA_ARGS__);                                       \
        else if ((Wv) == 16)                                                                       \
            kern<16, WT><<<(g), (b), 0, (st)>>>(__VA_ARGS__);                                      \
        else                                                                                       \
            kern<32, WT><<<(g), (b), 0, (st)>>>(__VA_ARGS__);                                      \
    } while (0)

// weight gradient G[na][nb] = sum_points A Bm^T into out (device)
cudaError_t wgrad(fch_fno *f, const float *A, int CA, int na, const float *Bm, int CB, int nb, float *out)
{
    const long npts = (long)f->B * f->n * f->n;
    int nblk = 1024;
    const int chunk = (int)((npts + nblk - 1) / nblk);
    nblk = (int)((npts + chunk - 1) / chunk);
    const int nthr = 256;
    const size_t smem = (size_t)(na + nb) * 32 * 4;
    fno_wgrad_part<<<nblk, nthr, smem, f->stream>>>(A, CA, na, Bm, CB, nb, f->n * f->n, npts, chunk, f->part);
    fno_wgrad_sum<<<grid(na * nb, 256), 256, 0, f->stream>>>(f->part, nblk, na * nb, out);
    return cudaGetLastError();
}

} // namespace

cudaStream_t fch_fno_stream_of(const fch_fno *f) { return f->stream; }

extern "C" fch_status fch_fno_create(int width, int layers, int modes, int proj, void *stream, fch_fno **out)
{
    if (!out || (width != 8 && width != 16 && width != 32) || layers < 1 || layers > 16 || modes < 1 ||
        proj < 1 || proj > kMaxW2 || proj * width > 8 * 256) {
        fch_set_thread_error("fch_fno_create: invalid argument");
        return FCH_EINVAL;
    }
    fch_fno *f = (fch_fno *)calloc(1, sizeof(fch_fno));
    if (!f) return FCH_ENOMEM;
    f->W = width;
    f->L = layers;
    f->M = modes;
    f->W2 = proj;
    f->cin = 2;
    f->K = modes * (2 * modes - 1);
    f->stream = (cudaStream_t)stream;
    f->np = offset_of(f, 8, 0) + 1;
    cudaError_t e = cudaMalloc((void **)&f->params, f->np * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&f->grads, f->np * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&f->am, f->np * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&f->av, f->np * 4);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&f->hsum, sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(f->params, 0, f->np * 4, f->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->grads, 0, f->np * 4, f->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->am, 0, f->np * 4, f->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->av, 0, f->np * 4, f->stream);
    if (e != cudaSuccess) {
        fch_set_thread_error(cudaGetErrorString(e));
        fch_fno_destroy(f);
        return FCH_ECUDA;
    }
    *out = f;
    return FCH_OK;
}

extern "C" fch_status fch_fno_destroy(fch_fno *f)
{
    if (!f) return FCH_OK;
    if (f->stream) cudaStreamSynchronize(f->stream);
    free_buffers(f);
    for (void *b : {(void *)f->params, (void *)f->grads, (void *)f->am, (void *)f->av, (void *)f->pbf,
                    (void *)f->tc_Bt, (void *)f->tc_tw, (void *)f->tc_X, (void *)f->tc_V, (void *)f->tc_Y,
                    (void *)f->tc_Z, (void *)f->tc_err})
        if (b) cudaFree(b);
    if (f->hsum) cudaFreeHost(f->hsum);
    free(f);
    return FCH_OK;
}

extern "C" fch_status fch_fno_num_params(const fch_fno *f, size_t *count)
{
    if (!f || !count) return FCH_EINVAL;
    *count = f->np;
    return FCH_OK;
}

static fch_status refresh_bf16(fch_fno *f);

static fch_status copy_vec(fch_fno *f, float *dev, const float *src_host, float *dst_host, size_t cnt)
{
    if (!f || cnt != f->np) return FCH_EINVAL;
    cudaError_t e = src_host ? cudaMemcpyAsync(dev, src_host, cnt * 4, cudaMemcpyHostToDevice, f->stream)
                             : cudaMemcpyAsync(dst_host, dev, cnt * 4, cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    return e == cudaSuccess ? FCH_OK : FCH_ECUDA;
}

extern "C" fch_status fch_fno_set_params(fch_fno *f, const float *host, size_t cnt)
{
    if (!host) return FCH_EINVAL;
    fch_status s = copy_vec(f, f ? f->params : nullptr, host, nullptr, cnt);
    if (s == FCH_OK) {
        cudaMemsetAsync(f->am, 0, f->np * 4, f->stream);
        cudaMemsetAsync(f->av, 0, f->np * 4, f->stream);
        f->adam_t = 0;
        s = refresh_bf16(f);
    }
    return s;
}

extern "C" fch_status fch_fno_get_params(fch_fno *f, float *host, size_t cnt)
{
    if (!host) return FCH_EINVAL;
    return copy_vec(f, f ? f->params : nullptr, nullptr, host, cnt);
}

extern "C" fch_status fch_fno_get_grads(fch_fno *f, float *host, size_t cnt)
{
    if (!host) return FCH_EINVAL;
    return copy_vec(f, f ? f->grads : nullptr, nullptr, host, cnt);
}

// the forward pass with weights P of type WT (FP32 parameters or their bfloat16 copy)
template <typename WT>
static fch_status forward_impl(fch_fno *f, int batch, int n, const float *a, float *y, const WT *P)
{
    fch_status st = ensure_buffers(f, batch, n);
    if (st != FCH_OK) return st;
    const int W = f->W, n2 = n * n;
    const long pts = (long)batch * n2;
    const size_t fld = (size_t)batch * W * n2, S = (size_t)(n / 2 + 1) * n;
    cudaStream_t s = f->stream;
    fno_lift<WT><<<grid(pts, 256), 256, 0, s>>>(a, P + offset_of(f, 0, 0), P + offset_of(f, 1, 0), f->h, batch, n2,
                                                W, f->cin);
    for (int l = 0; l < f->L; l++) {
        float *hin = f->h + l * fld, *hout = f->h + (l + 1) * fld;
        float2 *X = f->X + (size_t)l * batch * W * S;
        if ((st = fch_fft_r2c(f->plan, hin, X, batch * W)) != FCH_OK) return st;
        const int items = f->M + (f->M - 1) * (2 * f->M - 1);
        fno_mix<WT><<<grid((long)batch * W * items, 256), 256, 0, s>>>(X, P + offset_of(f, 4, l), f->Ysp, batch, W,
                                                                      f->M, n);
        if ((st = fch_fft_c2r(f->plan, f->Ysp, f->s, batch * W)) != FCH_OK) return st;
        WDISPATCH_T(W, fno_pointwise, WT, grid(pts, 128), 128, s, hin, f->s, P + offset_of(f, 2, l),
                    P + offset_of(f, 3, l), f->z + l * fld, hout, batch, n2, l < f->L - 1);
    }
    WDISPATCH_T(W, fno_project, WT, grid(pts, 128), 128, s, f->h + f->L * fld, P + offset_of(f, 5, 0),
                P + offset_of(f, 6, 0), P + offset_of(f, 7, 0), P + offset_of(f, 8, 0), y, batch, n2, f->W2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(f->err, sizeof(f->err), "fch_fno_forward: %s", cudaGetErrorString(e));
        fch_set_thread_error(f->err);
        return FCH_ECUDA;
    }
    f->a = a;
    f->have_fwd = true;
    // keep y for the backward pass (the caller owns its array)
    e = cudaMemcpyAsync(f->y, y, (size_t)pts * 4, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? FCH_OK : FCH_ECUDA;
}

// tables and work arrays of the truncated-DFT forward pass for (B, n)
static fch_status ensure_tc(fch_fno *f, int B, int n)
{
    if (f->tc_B == B && f->tc_n == n) return FCH_OK;
    for (void *b : {(void *)f->tc_Bt, (void *)f->tc_tw, (void *)f->tc_X, (void *)f->tc_V, (void *)f->tc_Y,
                    (void *)f->tc_Z})
        if (b) cudaFree(b);
    f->tc_Bt = nullptr;
    f->tc_tw = f->tc_X = f->tc_V = f->tc_Y = f->tc_Z = nullptr;
    f->tc_B = f->tc_n = 0;
    const size_t rows = (size_t)B * f->W * n, modes = (size_t)B * f->W * f->K;
    cudaError_t e = cudaMalloc((void **)&f->tc_Bt, (size_t)32 * n * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc((void **)&f->tc_tw, (size_t)16 * n * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&f->tc_X, rows * 16 * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&f->tc_V, rows * 16 * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&f->tc_Y, modes * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&f->tc_Z, modes * sizeof(float2));
    if (e == cudaSuccess && !f->tc_err) e = cudaMalloc((void **)&f->tc_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(f->tc_err, 0, sizeof(int), f->stream);
    if (e == cudaSuccess) {
        fno_dft_tables<<<grid(16L * n, 256), 256, 0, f->stream>>>(f->tc_Bt, f->tc_tw, n);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        snprintf(f->err, sizeof(f->err), "fch_fno (truncated DFT): %s", cudaGetErrorString(e));
        fch_set_thread_error(f->err);
        return e == cudaErrorMemoryAllocation ? FCH_ENOMEM : FCH_ECUDA;
    }
    f->tc_B = B;
    f->tc_n = n;
    return FCH_OK;
}

// the forward pass with the spectral convolutions as truncated DFTs, the row DFT on
// the tensor cores (BF16 operands, FP32 sums); BF16 weights elsewhere, FP32 sums
static fch_status forward_tc(fch_fno *f, int batch, int n, const float *a, float *y)
{
    typedef __nv_bfloat16 WT;
    const WT *P = f->pbf;
    fch_status st = ensure_buffers(f, batch, n);
    if (st == FCH_OK) st = ensure_tc(f, batch, n);
    if (st != FCH_OK) return st;
    const int W = f->W, M = f->M, n2 = n * n;
    const long pts = (long)batch * n2, R = (long)batch * W * n;
    const size_t fld = (size_t)batch * W * n2;
    cudaStream_t s = f->stream;
    {
        const WT *P0 = P + offset_of(f, 0, 0), *P1 = P + offset_of(f, 1, 0);
        const unsigned gl = grid(pts, 256);
        switch (f->cin * 64 + W) {
        case 1 * 64 + 16: fno_lift_t<WT, 16, 1><<<gl, 256, 0, s>>>(a, P0, P1, f->h, pts, n2); break;
        case 2 * 64 + 16: fno_lift_t<WT, 16, 2><<<gl, 256, 0, s>>>(a, P0, P1, f->h, pts, n2); break;
        case 1 * 64 + 32: fno_lift_t<WT, 32, 1><<<gl, 256, 0, s>>>(a, P0, P1, f->h, pts, n2); break;
        case 2 * 64 + 32: fno_lift_t<WT, 32, 2><<<gl, 256, 0, s>>>(a, P0, P1, f->h, pts, n2); break;
        default: fno_lift<WT><<<gl, 256, 0, s>>>(a, P0, P1, f->h, batch, n2, W, f->cin);
        }
    }
    for (int l = 0; l < f->L; l++) {
        float *hin = f->h + l * fld, *hout = f->h + (l + 1) * fld;
        launch_rowdft_tc(hin, f->tc_Bt, f->tc_X, R, n, f->tc_err, s);
        fno_coldft<16><<<dim3(batch * W, M), 256, 2 * n * sizeof(float2), s>>>(f->tc_X, f->tc_tw + n, f->tc_Y, n);
        fno_mix_modes<WT><<<grid((long)batch * W * f->K, 256), 256, 0, s>>>(f->tc_Y, P + offset_of(f, 4, l),
                                                                           f->tc_Z, batch, W, M);
        fno_icoldft<16><<<(unsigned)((long)batch * W * (n / 64)), 256, n * sizeof(float2), s>>>(
            f->tc_Z, f->tc_tw + n, f->tc_V, (long)batch * W, n);
        // the channel mixing and the inverse x DFT: one MMA chain per 128 points
        const dim3 g((unsigned)(n / 128 * n), (unsigned)batch);
        const int act = l < f->L - 1;
        if (W == 16)
            fno_pw_tc<16><<<g, 128, 0, s>>>(hin, f->tc_V, f->tc_tw, P + offset_of(f, 2, l), P + offset_of(f, 3, l),
                                           hout, n, act, f->tc_err);
        else
            fno_pw_tc<32><<<g, 128, 0, s>>>(hin, f->tc_V, f->tc_tw, P + offset_of(f, 2, l), P + offset_of(f, 3, l),
                                           hout, n, act, f->tc_err);
    }
    const unsigned gp = (unsigned)((pts + 127) / 128);
    if (W == 16)
        fno_proj_tc<16><<<gp, 128, 0, s>>>(f->h + f->L * fld, P + offset_of(f, 5, 0), P + offset_of(f, 6, 0),
                                           P + offset_of(f, 7, 0), P + offset_of(f, 8, 0), y, pts, n2, f->W2,
                                           f->tc_err);
    else
        fno_proj_tc<32><<<gp, 128, 0, s>>>(f->h + f->L * fld, P + offset_of(f, 5, 0), P + offset_of(f, 6, 0),
                                           P + offset_of(f, 7, 0), P + offset_of(f, 8, 0), y, pts, n2, f->W2,
                                           f->tc_err);
    cudaError_t e = cudaGetLastError();
    int herr = 0;
    // the tensor-core kernel's bounded waits report through a device flag
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, f->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess || herr) {
        snprintf(f->err, sizeof(f->err), "fch_fno_forward (tensor cores): %s",
                 e != cudaSuccess ? cudaGetErrorString(e) : "an mbarrier wait ran out");
        fch_set_thread_error(f->err);
        return FCH_ECUDA;
    }
    f->a = a;
    f->have_fwd = true;
    return FCH_OK;
}

// refresh the bfloat16 copy of the parameters (round to nearest even)
static fch_status refresh_bf16(fch_fno *f)
{
    if (!f->pbf) return FCH_OK;
    fno_to_bf16<<<grid((long)f->np, 256), 256, 0, f->stream>>>(f->params, f->pbf, (long)f->np);
    return cudaGetLastError() == cudaSuccess ? FCH_OK : FCH_ECUDA;
}

extern "C" fch_status fch_fno_set_bf16(fch_fno *f, int on)
{
    if (!f || on < 0 || on > 2) return FCH_EINVAL;
    if (on && !f->pbf) {
        if (cudaMalloc((void **)&f->pbf, f->np * sizeof(__nv_bfloat16)) != cudaSuccess) {
            f->pbf = nullptr;
            return FCH_ENOMEM;
        }
        f->tc = on == 2;
        return refresh_bf16(f);
    }
    f->tc = on == 2;
    if (!on && f->pbf) {
        cudaStreamSynchronize(f->stream);
        cudaFree(f->pbf);
        f->pbf = nullptr;
    }
    return FCH_OK;
}

extern "C" fch_status fch_fno_forward(fch_fno *f, int batch, int n, const float *a, float *y)
{
    if (!f || !a || !y || batch < 1 || n < 2 * f->M || n < 16 || n > 2048 || (n & (n - 1))) {
        fch_set_thread_error("fch_fno_forward: invalid argument");
        return FCH_EINVAL;
    }
    f->fwd_bf16 = f->pbf != nullptr;
    if (f->tc && f->pbf) {
        if (f->M != 16 || n % 128 != 0 || (f->W != 16 && f->W != 32) || f->W2 % 16 != 0) {
            fch_set_thread_error("fch_fno_forward: the tensor-core pass needs modes = 16, width 16 or 32, "
                                 "proj a multiple of 16 and n a multiple of 128");
            return FCH_EINVAL;
        }
        return forward_tc(f, batch, n, a, y);
    }
    return f->pbf ? forward_impl(f, batch, n, a, y, (const __nv_bfloat16 *)f->pbf)
                  : forward_impl(f, batch, n, a, y, (const float *)f->params);
}

extern "C" fch_status fch_fno_backward(fch_fno *f, const float *target, double *loss)
{
    if (!f || !target) return FCH_EINVAL;
    if (!f->have_fwd || f->fwd_bf16) return FCH_ESTATE; // training runs on the FP32 weights
    const int B = f->B, n = f->n, W = f->W, W2 = f->W2, n2 = n * n;
    const long pts = (long)B * n2;
    const size_t fld = (size_t)B * W * n2, S = (size_t)(n / 2 + 1) * n;
    cudaStream_t s = f->stream;
    const float *P = f->params;
    float *G = f->grads;
    cudaError_t e = cudaSuccess;
    // projection and the loss (y kept by the forward pass)
    WDISPATCH(W, fno_project_bwd, grid(pts, 128), 128, s, f->h + f->L * fld, P + offset_of(f, 5, 0),
              P + offset_of(f, 6, 0), P + offset_of(f, 7, 0), f->y, target, f->dy, f->q, f->dzq, f->dh, f->sq, B,
              n2, W2, 2.0f / (float)pts);
    if (e == cudaSuccess) e = wgrad(f, f->dy, 1, 1, nullptr, 1, 1, G + offset_of(f, 8, 0));         // bQ2
    if (e == cudaSuccess) e = wgrad(f, f->q, W2, W2, f->dy, 1, 1, G + offset_of(f, 7, 0));          // Q2
    if (e == cudaSuccess) e = wgrad(f, f->dzq, W2, W2, nullptr, 1, 1, G + offset_of(f, 6, 0));      // bQ1
    if (e == cudaSuccess) e = wgrad(f, f->dzq, W2, W2, f->h + f->L * fld, W, W, G + offset_of(f, 5, 0)); // Q1
    for (int l = f->L - 1; l >= 0 && e == cudaSuccess; l--) {
        float *hin = f->h + l * fld;
        const float2 *R = (const float2 *)(P + offset_of(f, 4, l));
        // dz = dh act'(z); dh_l = W^T dz (into tmp)
        WDISPATCH(W, fno_pointwise_bwd, grid(pts, 128), 128, s, f->dh, f->z + l * fld, P + offset_of(f, 2, l),
                  f->dz, f->tmp, B, n2, l < f->L - 1);
        e = wgrad(f, f->dz, W, W, nullptr, 1, 1, G + offset_of(f, 3, l)); // b_l
        if (e == cudaSuccess) e = wgrad(f, f->dz, W, W, hin, W, W, G + offset_of(f, 2, l)); // W_l
        if (e != cudaSuccess) break;
        // spectral branch
        if (fch_fft_r2c(f->plan, f->dz, f->Fd, B * W) != FCH_OK) return FCH_ECUDA;
        const int K = f->K;
        fno_dY<<<grid((long)B * W * K, 256), 256, 0, s>>>(f->Fd, f->dY, B, W, f->M, n);
        fno_dR<<<grid((long)K * W * W, 256), 256, 0, s>>>(f->dY, f->X + (size_t)l * B * W * S,
                                                          (float2 *)(G + offset_of(f, 4, l)), B, W, f->M, n);
        const int items = f->M + (f->M - 1) * (2 * f->M - 1);
        fno_dX<<<grid((long)B * W * items, 256), 256, 0, s>>>(f->dY, R, f->Ysp, B, W, f->M, n);
        if (fch_fft_c2r(f->plan, f->Ysp, f->dh, B * W) != FCH_OK) return FCH_ECUDA;
        fno_add<<<grid((long)fld, 256), 256, 0, s>>>(f->dh, f->tmp, (long)fld);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = wgrad(f, f->dh, W, W, nullptr, 1, 1, G + offset_of(f, 1, 0));     // bP
    if (e == cudaSuccess) e = wgrad(f, f->dh, W, W, f->a, f->cin, f->cin, G + offset_of(f, 0, 0)); // P
    // loss = mean of the squared residuals (host sum of a device copy, in double)
    if (e == cudaSuccess && loss) {
        float *hb = (float *)malloc((size_t)pts * 4);
        if (!hb) return FCH_ENOMEM;
        e = cudaMemcpyAsync(hb, f->sq, (size_t)pts * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        double acc = 0;
        for (long i = 0; i < pts; i++) acc += hb[i];
        free(hb);
        *loss = acc / (double)pts;
    }
    if (e != cudaSuccess) {
        snprintf(f->err, sizeof(f->err), "fch_fno_backward: %s", cudaGetErrorString(e));
        fch_set_thread_error(f->err);
        return FCH_ECUDA;
    }
    return FCH_OK;
}

extern "C" fch_status fch_fno_adam(fch_fno *f, float lr, float beta1, float beta2, float eps)
{
    if (!f || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0)) return FCH_EINVAL;
    f->adam_t++;
    const float c1 = 1.f - powf(beta1, (float)f->adam_t), c2 = 1.f - powf(beta2, (float)f->adam_t);
    fno_adam<<<grid((long)f->np, 256), 256, 0, f->stream>>>(f->params, f->grads, f->am, f->av, (long)f->np, lr, beta1,
                                                            beta2, eps, c1, c2);
    if (cudaGetLastError() != cudaSuccess) return FCH_ECUDA;
    return refresh_bf16(f);
}

__global__ void fno_gelu_eval(const float *__restrict__ x, float *__restrict__ y, long cnt, int as)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (!as) {
        if (t < cnt) y[t] = gelu(x[t]);
        return;
    }
    // the inference GELU works on pairs: elements 2t and 2t + 1 (the last alone twice)
    const long i = 2 * t;
    if (i >= cnt) return;
    const bool pair = i + 1 < cnt;
    const float2 g = x2_split(gelu_as2(x2(x[i], pair ? x[i + 1] : x[i])));
    y[i] = g.x;
    if (pair) y[i + 1] = g.y;
}

// test hook (not part of the C ABI of fch.h): the GELU of the inference kernels
// (as = 1) or of the training path (as = 0) on cnt device floats; 0 or a status
extern "C" int fch_debug_fno_gelu(const float *x, float *y, long cnt, int as, void *stream)
{
    if (!x || !y || cnt < 1) return FCH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    fno_gelu_eval<<<grid(cnt, 256), 256, 0, s>>>(x, y, cnt, as);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        fch_set_thread_error(cudaGetErrorString(e));
        return FCH_ECUDA;
    }
    return FCH_OK;
}

// test hook (not part of the C ABI of fch.h): the tensor-core row DFT alone,
// X[r][kx] for kx < 16 of R rows of n floats (device arrays); returns 0 or a status
extern "C" int fch_debug_rowdft_tc(const float *h, float *X, int R, int n, void *stream)
{
    if (!h || !X || R < 1 || n < 64 || n % 64 != 0 || n > 2048) return FCH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    __nv_bfloat16 *Bt = nullptr;
    float2 *tw = nullptr;
    int *err = nullptr, herr = 0;
    cudaError_t e = cudaMalloc((void **)&Bt, (size_t)32 * n * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc((void **)&tw, (size_t)16 * n * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        fno_dft_tables<<<grid(16L * n, 256), 256, 0, s>>>(Bt, tw, n);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_rowdft_tc(h, Bt, (float2 *)X, R, n, err, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (void *b : {(void *)Bt, (void *)tw, (void *)err})
        if (b) cudaFree(b);
    if (e != cudaSuccess) {
        fch_set_thread_error(cudaGetErrorString(e));
        return FCH_ECUDA;
    }
    return herr ? FCH_ECUDA : FCH_OK;
}
