// fch_tmap.h -- tensor maps (the descriptors of the TMA engine's tiled copies) of
// row-major FP32 matrices, encoded by the driver's cuTensorMapEncodeTiled, which the
// runtime looks up once.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

// A map of `outer` rows of `inner` floats, `row_bytes` apart (a multiple of 16; the
// base 16-byte aligned), copied in boxes of box_outer rows x box_inner floats
// (box_inner x 4 a multiple of 16; both at most 256); elements outside the matrix
// read as zero; no swizzle, L2 promotion by 128 bytes.
cudaError_t fch_tmap_f32_2d(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                            uint32_t box_inner, uint32_t box_outer);
