// fch_launch.cuh -- host launchers of the column and row passes for one precision.
// Included once per precision by fch_f64.cu / fch_f32.cu with FCH_T and FCH_SUFFIX set.
#include "fch_kernels.cuh"
#include "fch_warpfft.cuh"
#include "fch_colt.cuh"
#include "fch_tmap.h"

namespace {

typedef void (*pass_fn)(const fch_kparams);

// launch a pass with programmatic stream serialization (fch_pdl_config)
inline cudaError_t launch_pass(pass_fn f, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const fch_kparams &kp)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    fch_pdl_config(cfg, at, grid, block, smem, s, kp.pdl != 0);
    return cudaLaunchKernelEx(&cfg, f, kp);
}

// grid y: the field pairs of a batched standalone transform (one otherwise)
inline unsigned pair_grid(const fch_kparams &kp) { return kp.npairs > 1 ? (unsigned)kp.npairs : 1u; }

// Raise the kernel's dynamic shared-memory limit, at its first launch to what the
// default tiles of the largest grid (FCH_MAX_N) need, later only for larger tuned
// tiles (those launch first while a context or the tuner is set up, before any
// stream capture).
inline cudaError_t set_smem(pass_fn f, int bytes, int floor_bytes, int &cur)
{
    const int want = bytes > floor_bytes ? bytes : floor_bytes;
    if (want <= cur) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
    if (e == cudaSuccess) cur = want;
    return e;
}

// compile-time grid sizes: 512, 1024, 2048 (with FCH_ONLY_1024: 1024 only, which
// keeps the double-float translation units small); others use the generic kernel
template <typename T, int M> pass_fn col_fn(int logN)
{
    switch (logN) {
#ifndef FCH_ONLY_1024
    case 9: return fch::col_pass<T, M, 9>;
    case 11: return fch::col_pass<T, M, 11>;
#endif
    case 10: return fch::col_pass<T, M, 10>;
    }
    return fch::col_pass<T, M, 0>;
}

// the slot of the kernel launched for a grid of 2^logN at the default tiles: logN
// where a compile-time kernel is built in this translation unit, else 0 (the
// generic kernel), so that one kernel has one shared-memory limit record
inline int kernel_slot(int logN)
{
#ifndef FCH_ONLY_1024
    if (logN == 9 || logN == 11) return logN;
#endif
    return logN == 10 ? 10 : 0;
}

template <typename T, int M> pass_fn row_fn(int logN)
{
    switch (logN) {
#ifndef FCH_ONLY_1024
    case 9: return fch::row_pass<T, M, 9>;
    case 11: return fch::row_pass<T, M, 11>;
#endif
    case 10: return fch::row_pass<T, M, 10>;
    }
    return fch::row_pass<T, M, 0>;
}

// single precision at N = 1024: the warp-transform passes (one warp per sequence)
template <typename T> constexpr bool warp_path() { return sizeof(T) == 4; }

template <int M> cudaError_t launch_col_w(const fch_kparams &kp, cudaStream_t s)
{
    static int attr = 0;
    const int smem = (1024 * 5 + 4 * 33 * 32) * 8;
    pass_fn f = fch::col_pass_w<M>;
    cudaError_t e = set_smem(f, smem, 0, attr);
    if (e != cudaSuccess) return e;
    return launch_pass(f, dim3(256, pair_grid(kp)), dim3(128), smem, s, kp);
}

template <int M> cudaError_t launch_row_w(const fch_kparams &kp, cudaStream_t s)
{
    return launch_pass(fch::row_pass_w<M>, dim3(1024, pair_grid(kp)), dim3(32), 0, s, kp);
}

// Tiles (fch_kparams::tile_col, tile_row): 0 takes the two-block-cluster column pass
// for double and double-float at N = 1024, the warp-level row pass for single
// precision at N = 1024, else the compile-time kernel of the grid size where one is
// built, else the generic kernel; -1 the same without the clusters and the warp-level
// rows; -2 (columns, single precision at N = 1024) the warp-level column pass; > 0 the
// generic kernel with that many column pairs (rows) per block. The generic column
// kernel reads P from kp.P, which the caller sets.
// N = 1024, double and double-float: the column pass as clusters of two blocks
template <typename T, int M> cudaError_t launch_col_cl(const fch_kparams &kp, cudaStream_t s)
{
    static int attr = 0;
    const int smem = fch::skewed_len(1024) * (int)sizeof(typename fch::CT<T>::t);
    pass_fn f = fch::col_pass_cl<T, M>;
    cudaError_t e = set_smem(f, smem, 0, attr);
    if (e != cudaSuccess) return e;
    return launch_pass(f, dim3(1024, pair_grid(kp)), dim3(128), smem, s, kp);
}

// N = 1024, single precision, the column passes of standalone transform plans (which
// carry an error word): the persistent TMA-staged kernel, as many blocks as are
// resident at once; the inverse needs 16-byte aligned half spectra (bulk copies)
template <int M> bool col_t_applies(const fch_kparams &kp)
{
    if (M != CM_FWD_STORE && M != CM_INV_LOAD) return false;
    if (!kp.err || kp.npairs < 1 || kp.N != 1024 || kp.tile_col != 0 || (kp.flags & FCH_FL_F64IO)) return false;
    if (M == CM_INV_LOAD)
        return kp.in0 && !(((uintptr_t)kp.in0 | (uintptr_t)kp.in1 | (uintptr_t)kp.pstride_in) & 15);
    return true;
}

template <int M> cudaError_t launch_col_t(const fch_kparams &kp, cudaStream_t s)
{
    if constexpr (M == CM_FWD_STORE || M == CM_INV_LOAD) {
        static int resident = 0;
        if (!resident) {
            int dev = 0, sms = 0, per = 0;
            cudaError_t e = cudaFuncSetAttribute(fch::col_pass_t<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 fch::kColtSmem);
            if (e == cudaSuccess) e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fch::col_pass_t<M>, fch::kColtThreads,
                                                                  fch::kColtSmem);
            if (e != cudaSuccess) return e;
            if (per < 1) return cudaErrorInvalidConfiguration;
            resident = sms * per;
        }
        const long np = pair_grid(kp), tiles = np * 256;
        // Z of the launch's pairs: np * N rows of 2N floats, boxes of 256 rows x 8 floats
        CUtensorMap m;
        cudaError_t e = fch_tmap_f32_2d(&m, kp.Z, 2048, (uint64_t)np * 1024, 8192, 8, 256);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        fch_pdl_config(cfg, at, dim3((unsigned)(tiles < resident ? tiles : resident)), dim3(fch::kColtThreads),
                       fch::kColtSmem, s, kp.pdl != 0);
        return cudaLaunchKernelEx(&cfg, fch::col_pass_t<M>, kp, m);
    }
    return cudaErrorInvalidValue;
}

template <typename T, int M> cudaError_t launch_col(const fch_kparams &kp, cudaStream_t s)
{
    if constexpr (sizeof(T) == 4) {
        if (col_t_applies<M>(kp)) return launch_col_t<M>(kp, s);
    }
    if (warp_path<T>() && kp.N == 1024 && kp.tw2 && kp.tile_col == -2) return launch_col_w<M>(kp, s);
    if constexpr (sizeof(T) == 8) {
        if (kp.N == 1024 && kp.tile_col == 0) return launch_col_cl<T, M>(kp, s);
    }
    if (kp.tile_col <= -3) {
        // the generic kernel at four points a thread: needs the radix-4 twiddle table
        // (contexts carry one, standalone plans do not)
        if (!kp.tw4) return cudaErrorInvalidValue;
        static int attr4 = 0;
        const fch_geom g = fch_geometry_tiled(kp.N, sizeof(T) == 4, 0, kp.tile_col);
        pass_fn f = fch::col_pass<T, M, 0, 4>;
        cudaError_t e = set_smem(f, g.col_smem, 0, attr4);
        if (e != cudaSuccess) return e;
        return launch_pass(f, dim3(g.col_blocks, pair_grid(kp)), dim3(g.col_threads), g.col_smem, s, kp);
    }
    static int attr[12] = {};
    // the warp-level tile without its table (a context made with fft_path = 1) is -1
    const int tc = kp.tile_col == -2 ? -1 : kp.tile_col;
    const fch_geom g = fch_geometry_tiled(kp.N, sizeof(T) == 4, 0, tc);
    const int li = tc <= 0 ? kernel_slot(kp.logN) : 0;
    pass_fn f = col_fn<T, M>(li);
    cudaError_t e = set_smem(f, g.col_smem, fch_geometry(FCH_MAX_N, sizeof(T) == 4).col_smem, attr[li]);
    if (e != cudaSuccess) return e;
    return launch_pass(f, dim3(g.col_blocks, pair_grid(kp)), dim3(g.col_threads), g.col_smem, s, kp);
}

template <typename T, int M> cudaError_t launch_row(const fch_kparams &kp, cudaStream_t s)
{
    if (warp_path<T>() && kp.N == 1024 && kp.tw2 && kp.tile_row == 0) return launch_row_w<M>(kp, s);
    if (kp.tile_row <= -3) {
        // the generic kernel at four points a thread (radix-4 twiddle table: contexts only)
        if (!kp.tw4) return cudaErrorInvalidValue;
        static int attr4 = 0;
        const fch_geom g = fch_geometry_tiled(kp.N, sizeof(T) == 4, kp.tile_row, 0);
        pass_fn f = fch::row_pass<T, M, 0, 4>;
        cudaError_t e = set_smem(f, g.row_smem, 0, attr4);
        if (e != cudaSuccess) return e;
        return launch_pass(f, dim3(g.row_blocks, pair_grid(kp)), dim3(g.row_threads), g.row_smem, s, kp);
    }
    static int attr[12] = {};
    const fch_geom g = fch_geometry_tiled(kp.N, sizeof(T) == 4, kp.tile_row, 0);
    const int li = kp.tile_row <= 0 ? kernel_slot(kp.logN) : 0;
    pass_fn f = row_fn<T, M>(li);
    cudaError_t e = set_smem(f, g.row_smem, fch_geometry(FCH_MAX_N, sizeof(T) == 4).row_smem, attr[li]);
    if (e != cudaSuccess) return e;
    return launch_pass(f, dim3(g.row_blocks, pair_grid(kp)), dim3(g.row_threads), g.row_smem, s, kp);
}

} // namespace

#define FCH_CAT2(a, b) a##b
#define FCH_CAT(a, b) FCH_CAT2(a, b)

#ifndef FCH_NO_COL
cudaError_t FCH_CAT(fch_launch_col_, FCH_SUFFIX)(int mode, const fch_kparams &kp, cudaStream_t s)
{
    switch (mode) {
    case CM_FWD_STORE: return launch_col<FCH_T, CM_FWD_STORE>(kp, s);
    case CM_INV_LOAD: return launch_col<FCH_T, CM_INV_LOAD>(kp, s);
    case CM_START: return launch_col<FCH_T, CM_START>(kp, s);
    case CM_IMEX_SOLVE: return launch_col<FCH_T, CM_IMEX_SOLVE>(kp, s);
    case CM_F_FINISH: return launch_col<FCH_T, CM_F_FINISH>(kp, s);
    case CM_SAV_PQ: return launch_col<FCH_T, CM_SAV_PQ>(kp, s);
    case CM_SAV_COMBINE: return launch_col<FCH_T, CM_SAV_COMBINE>(kp, s);
    case CM_PSD_ITER: return launch_col<FCH_T, CM_PSD_ITER>(kp, s);
    case CM_ETD_STAGE1: return launch_col<FCH_T, CM_ETD_STAGE1>(kp, s);
    case CM_ETD_STAGE2: return launch_col<FCH_T, CM_ETD_STAGE2>(kp, s);
    }
    return cudaErrorInvalidValue;
}

#endif

#ifndef FCH_NO_ROW
cudaError_t FCH_CAT(fch_launch_row_, FCH_SUFFIX)(int mode, const fch_kparams &kp, cudaStream_t s)
{
    switch (mode) {
    case RM_R2C_LOAD: return launch_row<FCH_T, RM_R2C_LOAD>(kp, s);
    case RM_C2R_STORE: return launch_row<FCH_T, RM_C2R_STORE>(kp, s);
    case RM_NIMEX: return launch_row<FCH_T, RM_NIMEX>(kp, s);
    case RM_F: return launch_row<FCH_T, RM_F>(kp, s);
    case RM_SAV: return launch_row<FCH_T, RM_SAV>(kp, s);
    case RM_ENERGY: return launch_row<FCH_T, RM_ENERGY>(kp, s);
    case RM_NIMEX_DIRECT: return launch_row<FCH_T, RM_NIMEX_DIRECT>(kp, s);
    case RM_SAV_DIRECT: return launch_row<FCH_T, RM_SAV_DIRECT>(kp, s);
    }
    return cudaErrorInvalidValue;
}
#endif
