// Tensor-core (tcgen05) A*X product for BF16 A (defined in ax_tc.cu).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime.h>

namespace snmf {

struct TcPlan {
  int BN, tiles_n, tiles_m, stages, splits, k_iters, tmem_cols;
  size_t smem;
};

// Leading dimension (elements) of the BF16 copy of A and of the transposed X parts.
int64_t tc_ld(int64_t n);
// diagnostics of the last launch_ax_tc failure: CUresult of the encoder, or 10000 + cudaError_t
int tc_last_status();
int tc_plan(int64_t n, int N, TcPlan* plan);
// FP64 partial sums of squares / sums of a BF16 array into part[2*block]; returns blocks.
int launch_sums_bf16(const void* A16, int64_t elems, double* part, cudaStream_t s);
// A (n x n, dtype 0 f64 / 1 f32, lda) -> A16 (n x tc_ld(n) BF16, zero-padded columns)
void launch_to_bf16(int src_dtype, const void* A, int64_t n, int64_t lda, void* A16, cudaStream_t s);
// Y = A16 (Xh + Xl) with X (n x N FP32, ld ldx) split into BF16 parts in xh, xl (each
// N x tc_ld(n) BF16).  Split-K slices go to ws (n x ldx each).  err: device error code
// (nonzero after a timed-out wait), budget: clock64 cycles per wait.  Returns the number
// of splits (1 = Y written directly), or -1 when the tensor maps cannot be encoded.
int launch_ax_tc(const void* A16, int64_t n, const float* X, int N, int64_t ldx, void* xh, void* xl,
                 float* Y, float* ws, size_t ws_elems, int* err, long long budget, cudaStream_t s);

}  // namespace snmf
