// fch_peak.cu -- measured peak rates of this GPU's FP32 and FP64 fused
// multiply-add pipes. The paper has no counterpart: these are the denominators of
// the arithmetic roofline of the passes (the FP32 pipe carries the double-float
// passes, the FP64 pipe the double-precision ones), measured on the device the
// library runs on instead of taken from unit counts.
//
// Every thread runs eight independent FMA chains (enough independent work to hide
// the pipe's latency at eight resident blocks of 256 threads per SM); the grid is
// eight blocks per SM. The chains' sum is stored only when it equals a value it
// never reaches, so the compiler keeps every FMA and no memory traffic is timed.
#include <cuda_runtime.h>
#include <string.h>

#include "../../include/fch.h"
#include "fch_internal.h"

namespace {

template <typename T> __global__ void __launch_bounds__(256) fma_chains(T a, T b, int iters, T *sink)
{
    T x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < 16; r++) {
#pragma unroll
            for (int j = 0; j < 8; j++) x[j] = fma(x[j], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) s += x[j];
    if (s == (T)-1234.5) *sink = s;
}

template <typename T> cudaError_t time_chains(int sms, int iters, cudaStream_t st, T *sink, double *rate)
{
    const int blocks = 8 * sms, threads = 256;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    const T a = (T)0.999, b = (T)1e-4; // x converges to b / (1 - a); never -1234.5
    double best = 0.0;
    for (int rep = 0; rep < 6 && e == cudaSuccess; rep++) {
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3(blocks);
        cfg.blockDim = dim3(threads);
        cfg.stream = st;
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, fma_chains<T>, a, b, iters, sink);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        // one FMA = two floating-point operations; rep 0 is a warm-up
        const double flops = 2.0 * 8.0 * 16.0 * (double)iters * blocks * threads;
        if (e == cudaSuccess && rep > 0 && ms > 0.f && flops / (ms * 1e-3) > best) best = flops / (ms * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *rate = best;
    return e;
}

} // namespace

extern "C" fch_status fch_alu_peak(int prec, void *stream, double *flops_per_s, int *sm_count)
{
    if ((prec != FCH_FP64 && prec != FCH_MIXED) || !flops_per_s) {
        fch_set_thread_error("fch_alu_peak: prec must be FCH_FP64 or FCH_MIXED, flops_per_s not NULL");
        return FCH_EINVAL;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        fch_set_thread_error(cudaGetErrorString(e));
        return FCH_ECUDA;
    }
    void *sink = nullptr;
    e = cudaMalloc(&sink, sizeof(double));
    if (e != cudaSuccess) {
        fch_set_thread_error(cudaGetErrorString(e));
        return FCH_ENOMEM;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double rate = 0.0;
    if (prec == FCH_MIXED)
        e = time_chains<float>(sms, 2048, st, (float *)sink, &rate); // ~2 ms a launch at the FP32 rate
    else
        e = time_chains<double>(sms, 64, st, (double *)sink, &rate); // ~2 ms a launch at ~1 TFLOP/s
    cudaError_t ef = cudaFree(sink);
    if (e == cudaSuccess) e = ef;
    if (e != cudaSuccess) {
        fch_set_thread_error(cudaGetErrorString(e));
        return FCH_ECUDA;
    }
    *flops_per_s = rate;
    if (sm_count) *sm_count = sms;
    return FCH_OK;
}
