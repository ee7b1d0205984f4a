// fch_noalloc.cu -- a standalone R2C transform that allocates no device memory.
//
// Some callers must not allocate device memory once they are running: another
// component may own the device's whole memory budget, cudaMalloc/cudaFree may
// synchronize the device and stall unrelated work, or the caller's rules forbid
// dynamic allocation after start-up. fch_fft_r2c_noalloc serves them: it is the
// transform of fch_fft_r2c with its work array and twiddle table taken from a
// fixed-size array in this file instead of a plan. The caller still passes the
// input and output arrays.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (FCH_NOALLOC_BYTES) until the process exits. In host code its
// name is only a host-side stand-in, never a device address: the device address
// is looked up once per device with cudaGetSymbolAddress (with that device
// current) and cached. The cached address belongs to the device's context of that
// moment; after cudaDeviceReset the entry point must not be called again in the
// process. All calls share the array and it keeps the last call's
// contents; nothing in it needs clearing, because every call rewrites the twiddle
// table and writes each work element before reading it. Calls whose GPU work
// overlaps (other streams, other host threads) race on the array.
#include <mutex>
#include <stdio.h>
#include <string.h>

#include "../../include/fch.h"
#include "fch_internal.h"

// work array N x N complex + twiddle table N complex, at most N = 512 in double
#define FCH_NOALLOC_BYTES ((size_t)FCH_NOALLOC_MAX_N * FCH_NOALLOC_MAX_N * 16 + (size_t)FCH_NOALLOC_MAX_N * 16)

static __device__ __align__(256) unsigned char g_noalloc_scratch[FCH_NOALLOC_BYTES];

namespace {

std::mutex g_setup_mutex;
void *g_scratch_addr[64];   // device address of g_noalloc_scratch per device ordinal
bool g_scratch_ready[64];

// Per-stage Stockham twiddles in the layout the passes read (stage with sub-length
// Ns and radix R: entry Ns - 8 + (r-1) Ns + j = exp(-2 pi i r j / (Ns R)),
// r = 1..R-1, j < Ns), written on the device so no host copy is needed.
template <typename T> __global__ void noalloc_twiddles(T *tw, int N, int logN)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    tw[2 * m] = (T)0;
    tw[2 * m + 1] = (T)0;
    int Ns = 1, rem = logN;
    while (rem > 0) {
        const int lr = rem >= 3 ? 3 : rem, R = 1 << lr;
        if (Ns > 1 && m >= Ns - 8 && m < Ns - 8 + (R - 1) * Ns) {
            const int r = (m - (Ns - 8)) / Ns + 1, j = (m - (Ns - 8)) % Ns;
            double s, c;
            sincospi(-2.0 * (double)(r * j) / (double)(Ns * R), &s, &c);
            tw[2 * m] = (T)c;
            tw[2 * m + 1] = (T)s;
        }
        Ns <<= lr;
        rem -= lr;
    }
}

// the device address of the scratch array on the current device (looked up once)
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ready[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
        g_scratch_ready[dev] = true;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

} // namespace

extern "C" fch_status fch_fft_r2c_noalloc(int n, int prec, const void *x, void *X, int batch, void *stream)
{
    if (n > FCH_NOALLOC_MAX_N) {
        char msg[160];
        snprintf(msg, sizeof(msg),
                 "fch_fft_r2c_noalloc: n = %d exceeds the static work array (n <= %d)", n,
                 FCH_NOALLOC_MAX_N);
        fch_set_thread_error(msg);
        return FCH_EINVAL;
    }
    if (n < FCH_MIN_N || (n & (n - 1)) || (prec != 0 && prec != 1) || !x || !X || batch < 0) {
        fch_set_thread_error("fch_fft_r2c_noalloc: invalid argument");
        return FCH_EINVAL;
    }
    void *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        fch_set_thread_error(cudaGetErrorString(e));
        return FCH_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t csz = prec ? 8 : 16;
    int logN = 0;
    while ((1 << logN) < n) logN++;
    void *Z = scratch;
    void *tw = (unsigned char *)scratch + (size_t)n * n * csz;
    // launched through cudaLaunchKernelEx so that the status is this launch's own,
    // not an error left pending by earlier, unrelated work on this thread
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((n + 127) / 128);
    cfg.blockDim = dim3(128);
    cfg.stream = s;
    if (prec)
        e = cudaLaunchKernelEx(&cfg, noalloc_twiddles<float>, (float *)tw, n, logN);
    else
        e = cudaLaunchKernelEx(&cfg, noalloc_twiddles<double>, (double *)tw, n, logN);

    fch_kparams kp;
    memset(&kp, 0, sizeof(kp));
    kp.N = n;
    kp.logN = logN;
    kp.P = fch_geometry(n, prec).P;
    kp.pdl = 0; // n <= 512: passes of several waves, where programmatic launch measured slower
    kp.inv_n2 = 1.0 / ((double)n * n);
    kp.cf.inv_n2 = (float)kp.inv_n2;
    kp.cd.inv_n2 = kp.inv_n2;
    kp.Z = Z;
    kp.tw = tw;
    kp.tail_op = -1;
    kp.flags = FCH_FL_NOSKIP | (prec ? 0 : FCH_FL_F64IO);
    const size_t rb = (size_t)n * n * (prec ? 4 : 8), cb = (size_t)(n / 2 + 1) * n * csz;
    for (int b = 0; b < batch && e == cudaSuccess; b += 2) {
        kp.in0 = (const char *)x + b * rb;
        kp.in1 = b + 1 < batch ? (const char *)kp.in0 + rb : nullptr;
        kp.out0 = (char *)X + b * cb;
        kp.out1 = b + 1 < batch ? (char *)kp.out0 + cb : nullptr;
        e = prec ? fch_launch_row_f32(RM_R2C_LOAD, kp, s) : fch_launch_row_f64(RM_R2C_LOAD, kp, s);
        if (e == cudaSuccess)
            e = prec ? fch_launch_col_f32(CM_FWD_STORE, kp, s) : fch_launch_col_f64(CM_FWD_STORE, kp, s);
    }
    if (e != cudaSuccess) {
        fch_set_thread_error(cudaGetErrorString(e));
        return FCH_ECUDA;
    }
    return FCH_OK;
}
