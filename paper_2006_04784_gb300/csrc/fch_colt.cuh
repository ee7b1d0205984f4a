// fch_colt.cuh -- column passes of the standalone single-precision transforms at
// N = 1024 with their input staged by the TMA engine.
//
// A tile is P = 2 column pairs: four columns, 32 bytes of every row of the
// pair-layout work array Z. 512 threads transform its four columns in shared memory
// as col_pass does (radix-8, 8, 8, 2 Stockham stages over the skewed tile; thread
// (c, t) = (tid mod 4, tid / 4) works on column c). Blocks are persistent: block b
// takes tiles b, b + B, b + 2B, ... of all the launch's field pairs (tile g: pair
// g / 256, column pairs 2 (g mod 256) and the next), and the next tile's input lands
// in a 32 KB stage while the current tile is transformed:
//  - forward (R2C): four 2D tensor-map boxes of Z (256 rows x 8 floats each,
//    cp.async.bulk.tensor) fill the stage densely, row n at 32 n bytes. The first
//    radix-8 stage reads it there (rows t + 128 r of column c: a warp reads 256
//    contiguous bytes) and writes the skewed tile, after which the stage is free;
//  - inverse (C2R): the rows kx of the two half spectra (8 KB each, cp.async.bulk)
//    of the tile's two column pairs; the first radix-8 stage forms its inputs from
//    them there (the spectral stage folded into it) and writes the skewed tile. The
//    tile of pair 0 (kx = 0 and N/2 need four rows) reads its spectra from global
//    memory and takes the separate spectral stage.
// The forward spectral stage gives each thread rows ky and -ky of the tile, read as
// whole 32-byte rows, and the four work items that touch only them.
// Copies complete in bytes on the block's mbarrier; a wait that runs out of time (1 s)
// sets *kp.err, and the block stops after waiting (bounded) for the copy it started.
#pragma once
#include <cuda.h>
#include "fch_kernels.cuh"
#include "fch_tc.cuh"

namespace fch {

constexpr int kColtThreads = 512;
constexpr int kColtStageBytes = 4 * 1024 * 8;           // the next tile's input
constexpr int kColtTileBytes = 4 * 1152 * 8;            // four skewed columns (skewed_len(1024) = 1152)
constexpr int kColtTwBytes = 1024 * 8;                  // the per-stage twiddles, loaded once a block
constexpr int kColtSmem = kColtStageBytes + kColtTileBytes + kColtTwBytes + 16 + 128; // + mbarrier, + slack
constexpr uint64_t kColtWaitNs = 1000000000ull;

// a 32-byte row of four complex values of the tile, as two 16-byte accesses
__device__ __forceinline__ void load_row4(const float2 *row, float2 *v)
{
    const float4 a = *(const float4 *)row, b = *(const float4 *)(row + 2);
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y);
    v[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void store_row4(float2 *row, const float2 *v)
{
    *(float4 *)row = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    *(float4 *)(row + 2) = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
}

// the Hermitian split of one work item: z0 = Z(kx, ky), z1 = Z(N - kx, -ky) give
// A = (z0 + conj z1) / 2 and B = (z0 - conj z1) / (2i) at o0[idx], o1[idx]
__device__ __forceinline__ void split_store(float2 z0, float2 z1, float2 *o0, float2 *o1, long idx)
{
    const float2 c1 = cconj(z1);
    o0[idx] = cscale(cadd(z0, c1), 0.5f);
    if (o1) {
        const float2 dm = csub(z0, c1);
        o1[idx] = mk<float2>(0.5f * dm.y, -0.5f * dm.x);
    }
}

template <int MODE>
__global__ void __launch_bounds__(kColtThreads, 2) col_pass_t(const fch_kparams kp,
                                                              const __grid_constant__ CUtensorMap zmap)
{
    static_assert(MODE == CM_FWD_STORE || MODE == CM_INV_LOAD, "the standalone transform modes");
    typedef float2 C;
    constexpr bool FWD = MODE == CM_FWD_STORE;
    constexpr int N = 1024, LOGN = 10, NC = 4, NT = kColtThreads;
    pdl_begin();
    extern __shared__ unsigned char smem_raw[];
    // the TMA destination wants 128-byte alignment
    unsigned char *base = smem_raw + ((128u - (fch::tc::smem_u32(smem_raw) & 127u)) & 127u);
    C *stage = (C *)base;
    C *tile = (C *)(base + kColtStageBytes);
    C *tws = (C *)(base + kColtStageBytes + kColtTileBytes);
    uint64_t *bar = (uint64_t *)(base + kColtStageBytes + kColtTileBytes + kColtTwBytes);
    const int c = threadIdx.x % NC, t = threadIdx.x / NC;
    const long npairs = kp.npairs > 1 ? kp.npairs : 1;
    const long ntiles = npairs * (N / 4);
    for (int i = threadIdx.x; i < N; i += NT) tws[i] = ldg((const C *)kp.tw + i);
    const C *tw = tws;
    const fch_consts<float> &K = kp.cf;
    const fch_coef<float> co = fch_coef<float>();
    const float inv_n2 = K.inv_n2;
    const bool two = kp.in1 != nullptr; // inverse: a second half spectrum

    // a tile's input reaches the stage unless it is an inverse tile of pair 0
    auto staged = [&](long g) { return FWD || (g & 255) != 0; };
    auto fetch = [&](long g) { // thread 0
        const long pr = g >> 8;
        const int p0 = 2 * (int)(g & 255);
        if (FWD) {
            fch::tc::mbar_expect_tx(bar, kColtStageBytes);
#pragma unroll
            for (int q = 0; q < 4; q++)
                fch::tc::tma_load_2d(stage + q * 256 * NC, &zmap, 4 * p0, (int)(pr * N + 256 * q), bar);
        } else if (p0 != 0) {
            const char *i0 = (const char *)kp.in0 + pr * kp.pstride_in;
            const char *i1 = two ? (const char *)kp.in1 + pr * kp.pstride_in : nullptr;
            fch::tc::mbar_expect_tx(bar, (two ? 4 : 2) * N * 8);
#pragma unroll
            for (int pp = 0; pp < 2; pp++) {
                fch::tc::bulk_g2s(stage + 2 * pp * N, i0 + (long)(p0 + pp) * N * 8, N * 8, bar);
                if (two) fch::tc::bulk_g2s(stage + (2 * pp + 1) * N, i1 + (long)(p0 + pp) * N * 8, N * 8, bar);
            }
        }
    };

    long g = blockIdx.x;
    if (threadIdx.x == 0) {
        fch::tc::mbar_init(bar, 1);
        fch::tc::mbar_init_fence();
        if (g < ntiles) fetch(g);
    }
    __syncthreads();
    uint32_t phase = 0;
    bool ok = true;
    for (; g < ntiles; g += gridDim.x) {
        const long pr = g >> 8;
        const int p0 = 2 * (int)(g & 255);
        const bool st = staged(g);
        if (st) {
            ok = __syncthreads_and(fch::tc::mbar_wait(bar, phase, kColtWaitNs));
            if (!ok) break;
            phase ^= 1u;
        }
        ColBufs<C> bf = ColBufs<C>();
        bf.i0 = kp.in0 ? (const C *)((const char *)kp.in0 + pr * kp.pstride_in) : nullptr;
        bf.i1 = two ? (const C *)((const char *)kp.in1 + pr * kp.pstride_in) : nullptr;
        bf.o0 = kp.out0 ? (C *)((char *)kp.out0 + pr * kp.pstride_out) : nullptr;
        bf.o1 = kp.out1 ? (C *)((char *)kp.out1 + pr * kp.pstride_out) : nullptr;
        float red[FCH_NRED] = {0.f, 0.f, 0.f, 0.f};
        if (FWD) {
            // first radix-8 stage (no twiddles) from the stage into the skewed tile
            C v[8];
#pragma unroll
            for (int r = 0; r < 8; r++) v[r] = stage[(t + 128 * r) * NC + c];
            bfly8<-1>(v);
#pragma unroll
            for (int r = 0; r < 8; r++) tile[skew(8 * t + r) * NC + c] = v[r];
            __syncthreads(); // stage consumed, tile written
            if (threadIdx.x == 0) {
                fch::tc::fence_async_smem(); // the stage's reads come before the next copy's writes
                if (g + gridDim.x < ntiles) fetch(g + gridDim.x);
            }
            fft_stage<-1, 3, false, 8>(tile, N, LOGN, NC, c, tw, t, 8, 3);
            fft_stage<-1, 3, false, 8>(tile, N, LOGN, NC, c, tw, t, 64, 6);
            fft_stage<-1, 1, false, 8>(tile, N, LOGN, NC, c, tw, t, 512, 9);
            // spectral stage: the Hermitian split into the two half spectra. A thread
            // owns rows ky and -ky (both 32-byte rows of the tile, read whole) and all
            // four work items (pair p0 + pp, row ky or -ky) that touch only them.
            if (p0 > 0) {
                for (int ky = threadIdx.x; ky <= (N >> 1); ky += NT) {
                    const int mky = (N - ky) & (N - 1);
                    C rk[4], rm[4];
                    load_row4(tile + skew(ky) * NC, rk);
                    load_row4(tile + skew(mky) * NC, rm);
#pragma unroll
                    for (int pp = 0; pp < 2; pp++) {
                        const long base = (long)(p0 + pp) * N;
                        // item (pp, ky): slot 0 at row ky, slot 1 at row -ky; item (pp, -ky): the other way
                        split_store(rk[2 * pp], rm[2 * pp + 1], bf.o0, bf.o1, base + ky);
                        if (mky != ky) split_store(rm[2 * pp], rk[2 * pp + 1], bf.o0, bf.o1, base + mky);
                    }
                }
            } else {
                // pair 0 (columns 0 and N/2) and pair 1, item by item
#pragma unroll 1
                for (int it = 0; it < 4; it++) {
                    const int i = threadIdx.x + it * NT;
                    const int pp = i / N, ky = i - pp * N;
                    const int s0 = 2 * pp, s1 = 2 * pp + 1;
                    if (pp > 0) {
                        const int mky = (N - ky) & (N - 1);
                        split_store(tile[skew(ky) * NC + s0], tile[skew(mky) * NC + s1], bf.o0, bf.o1,
                                    (long)pp * N + ky);
                    } else if (ky <= (N >> 1)) {
                        pair0_item<float, MODE>(kp, K, co, bf, tile, N, NC, s0, s1, ky, false, red);
                    }
                }
            }
        } else {
            if (p0 > 0) {
                // the spectral stage fused into the first radix-8 stage: thread (c, t)
                // forms rows t + 128 r of column c straight from the staged spectra. With
                // (C, D) the two half spectra over N^2, slot 0 (column kx) of a pair holds
                // C + i D at (kx, ky) and slot 1 (column N - kx) conj(C) + i conj(D) taken
                // at (kx, -ky).
                const int pp = c >> 1;
                const bool odd = c & 1;
                const C *a = stage + 2 * pp * N, *b = stage + (2 * pp + 1) * N;
                C v[8];
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    const int ky = t + 128 * r, kk = odd ? (N - ky) & (N - 1) : ky;
                    const C Co = cscale(a[kk], inv_n2);
                    const C Do = two ? cscale(b[kk], inv_n2) : mk<C>(0.f, 0.f);
                    v[r] = odd ? mk<C>(Co.x + Do.y, Do.x - Co.y) : mk<C>(Co.x - Do.y, Co.y + Do.x);
                }
                bfly8<+1>(v);
#pragma unroll
                for (int r = 0; r < 8; r++) tile[skew(8 * t + r) * NC + c] = v[r];
                __syncthreads(); // stage consumed, tile written
                if (threadIdx.x == 0) {
                    fch::tc::fence_async_smem(); // the stage's reads come before the next copy's writes
                    if (g + gridDim.x < ntiles) fetch(g + gridDim.x);
                }
                fft_stage<+1, 3, false, 8>(tile, N, LOGN, NC, c, tw, t, 8, 3);
                fft_stage<+1, 3, false, 8>(tile, N, LOGN, NC, c, tw, t, 64, 6);
                fft_stage<+1, 1, false, 8>(tile, N, LOGN, NC, c, tw, t, 512, 9);
            } else {
                // pair 0 (columns 0 and N/2) and pair 1, item by item from global memory
#pragma unroll 1
                for (int it = 0; it < 4; it++) {
                    const int i = threadIdx.x + it * NT;
                    const int pp = i / N, ky = i - pp * N;
                    const int s0 = 2 * pp, s1 = 2 * pp + 1;
                    if (pp > 0) {
                        const int mky = (N - ky) & (N - 1);
                        const C Co = cscale(bf.i0[(long)pp * N + ky], inv_n2);
                        const C Do = two ? cscale(bf.i1[(long)pp * N + ky], inv_n2) : mk<C>(0.f, 0.f);
                        tile[skew(ky) * NC + s0] = mk<C>(Co.x - Do.y, Co.y + Do.x);
                        tile[skew(mky) * NC + s1] = mk<C>(Co.x + Do.y, Do.x - Co.y);
                    } else if (ky <= (N >> 1)) {
                        pair0_item<float, MODE>(kp, K, co, bf, tile, N, NC, s0, s1, ky, true, red);
                    }
                }
                __syncthreads();
                if (threadIdx.x == 0) { // the stage is idle here
                    fch::tc::fence_async_smem();
                    if (g + gridDim.x < ntiles) fetch(g + gridDim.x);
                }
                fft_smem<+1, false>(tile, N, LOGN, NC, c, tw, t);
            }
            // the four columns back to Z: half a 32-byte row per thread and store
            C *Z = (C *)kp.Z + pr * N * N;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int i = threadIdx.x + k * NT;
                const int n = i >> 1, h = i & 1;
                __stcg((float4 *)(Z + (long)n * N + 2 * p0 + 2 * h), *(const float4 *)(tile + skew(n) * NC + 2 * h));
            }
        }
        __syncthreads(); // the tile is read before the next tile's first writes
    }
    if (!ok && threadIdx.x == 0) {
        // the copy this block waits for may still land: let it, then report
        fch::tc::mbar_wait(bar, phase, kColtWaitNs);
        if (kp.err) atomicExch(kp.err, 1);
    }
}

} // namespace fch
