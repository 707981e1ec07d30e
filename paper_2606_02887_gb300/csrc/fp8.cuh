// FP8 (E4M3 + power-of-two 128 x 128 tile scale) storage of A and its CUDA-core product
// (defined in fp8.cu).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime.h>

#include "tune.cuh"

namespace snmf {

// Leading dimension (bytes) of the code matrix and the number of 128-wide tiles per side.
int64_t fp8_ld(int64_t n);
int fp8_ntiles(int64_t n);
// A (n x n, dtype 0 f64 / 1 f32, lda) -> scales (fp8_ntiles^2, row-major) and codes A8
// (n x fp8_ld(n), zero beyond column n).
void launch_fp8_encode(int src_dtype, const void* A, int64_t n, int64_t lda, void* A8, float* scales,
                       cudaStream_t s);
// FP64 partial (sum of squares, sum) of the decoded A~ per block into part[2*block]; returns blocks.
int launch_fp8_sums(const void* A8, int64_t n, const float* scales, double* part, cudaStream_t s);
// Y = A~ X (X, Y: n x cols FP32, leading dimension ld); split-K slices go to ws (n x ld
// each).  Returns the number of splits (1 = result in Y).
int launch_ax_fp8(const void* A8, const float* scales, int64_t n, const float* X, int cols, int64_t ld, float* Y,
                  float* ws, size_t ws_elems, const int* run, cudaStream_t s, const ProdTune* tune = nullptr);

}  // namespace snmf
