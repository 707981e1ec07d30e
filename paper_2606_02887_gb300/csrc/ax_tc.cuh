// Tensor-core (tcgen05) A*X product for BF16 A (defined in ax_tc.cu).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "tune.cuh"

namespace snmf {

struct TcPlan {
  int BN, tiles_n, tiles_m, stages, splits, k_iters, tmem_cols;
  size_t smem;
};

// Epilogue fused into the tensor-core product (fused = 1): the last K slice of each output
// tile to finish sums the slices in slice order and writes Y = A X (+ c X2), with the
// per-restart partials <P1, A X> -> part[slot][j][q0], <P2, A X> -> [q0 + 1] over 64-row
// slots (P1 / P2 may be NULL; with either set, r must be a multiple of 16 dividing the tile
// width).  counters: one zeroed unsigned per output tile, left zeroed.
struct TcEpilogue {
  int fused = 0;
  float* Y = nullptr;
  unsigned* counters = nullptr;
  float c = 0.f;
  const float* X2 = nullptr;
  const float* P1 = nullptr;
  const float* P2 = nullptr;
  double* part = nullptr;
  int q0 = 0;
  int r = 1;
  int b = 1;
};

// FP32 tensor map of a row-major matrix (rows x cols, row pitch ld elements) for tiles of
// 128 rows x 32 columns with the 128-byte swizzle; false when it cannot be encoded (base not
// 16-byte aligned, pitch not a multiple of 16 bytes, no encoder).
bool make_map_f32_tile(CUtensorMap* m, const void* base, int64_t cols, int64_t rows, int64_t ld);
// Leading dimension (elements) of the BF16 copy of A and of the transposed X parts.
int64_t tc_ld(int64_t n);
// diagnostics of the last launch_ax_tc failure: CUresult of the encoder, or 10000 + cudaError_t
int tc_last_status();
// Built-in plan, or the autotuned (per_sm, stages, splits) when `tune` sets them; returns
// -1 when a tuned ring does not fit in shared memory.
int tc_plan(int64_t n, int N, TcPlan* plan, const ProdTune* tune = nullptr, int xparts = 2, int a8 = 0);
// FP64 partial sums of squares / sums of a BF16 array into part[2*block]; returns blocks.
int launch_sums_bf16(const void* A16, int64_t elems, double* part, cudaStream_t s);
// The same sums over the whole symmetric matrix held as its upper tiles (the tiles above the
// diagonal count twice); returns blocks.
int launch_sums_bf16_sym(const void* A16s, int64_t n, double* part, cudaStream_t s);
// A (n x n, dtype 0 f64 / 1 f32, lda; only the tiles on and above the diagonal are read)
// -> its upper tiles in BF16 (sym_tiles(n) x 128 x 128)
void launch_to_bf16_sym(int src_dtype, const void* A, int64_t n, int64_t lda, void* A16s, cudaStream_t s);
// A (n x n, dtype 0 f64 / 1 f32, lda) -> A16 (n x tc_ld(n) BF16, zero-padded columns)
void launch_to_bf16(int src_dtype, const void* A, int64_t n, int64_t lda, void* A16, cudaStream_t s);
// Y = A16 (Xh + Xl) with X (n x N FP32, ld ldx) split into BF16 parts in xh, xl (each
// N x tc_ld(n) BF16).  Split-K slices go to ws (n x ldx each).  err: device error code
// (nonzero after a timed-out wait), budget: clock64 cycles per wait.  Returns the number
// of splits (1 = Y written directly), or -1 when the tensor maps cannot be encoded.
int launch_ax_tc(const void* A16, int64_t n, const float* X, int N, int64_t ldx, void* xh, void* xl,
                 float* Y, float* ws, size_t ws_elems, int* err, long long budget, cudaStream_t s,
                 const ProdTune* tune = nullptr, int xparts = 2, int sym = 0);
// The same product with the epilogue fused (see TcEpilogue) and X seen as xparts BF16 parts
// (2: hi + lo, 1: X rounded to BF16, one MMA pass).  The slices of a split K go to ws.  Returns
// 0 when the product and epilogue are complete in Y, or < 0 as launch_ax_tc.  xl may be NULL
// when xparts == 1.  run: a solve's device run flag (NULL: always); when it reads 0 the launch
// does nothing.  sym = 1: A16 holds the upper tiles of A (sym_tile) instead of n x tc_ld(n).
int launch_ax_tc_fused(const void* A16, int64_t n, const float* X, int N, int64_t ldx, void* xh, void* xl,
                       int xparts, float* ws, size_t ws_elems, int* err, long long budget, const TcEpilogue& epi,
                       const int* run, cudaStream_t s, const ProdTune* tune = nullptr, int sym = 0);
// The same product with A stored as E4M3 codes (n x fp8_ld(n) bytes) and a power-of-two scale
// per 128 x 128 tile (scales[fp8_ntiles(n)^2], row-major): the kernel decodes each code tile to
// BF16 in shared memory (exactly) and runs the BF16 MMAs and epilogue.  Returns as
// launch_ax_tc / launch_ax_tc_fused (< 0: the tensor map could not be encoded).
int launch_ax_tc8(const void* A8, const float* scales, int64_t n, const float* X, int N, int64_t ldx, void* xh,
                  void* xl, float* Y, float* ws, size_t ws_elems, int* err, long long budget, cudaStream_t s,
                  const ProdTune* tune = nullptr, int xparts = 2);
int launch_ax_tc8_fused(const void* A8, const float* scales, int64_t n, const float* X, int N, int64_t ldx,
                        void* xh, void* xl, int xparts, float* ws, size_t ws_elems, int* err, long long budget,
                        const TcEpilogue& epi, const int* run, cudaStream_t s, const ProdTune* tune = nullptr);

// ---- grouped product of the uneven batch (one CTA per 128-row tile of a problem) ----
// A_all: BF16, rows of all problems packed, pitch lda; X parts: BF16 hi / lo, row xrow_p + c
// holds column c of X_p (K-major, pitch lda, zero beyond n_p and beyond r_p).
struct TcItem {
  int64_t arow;   // first A_all row of the tile (problem's first row + m0)
  int64_t xoff;   // element offset of the problem's n_p x r_p factor blocks (ld r_p)
  int m0;         // first row of the tile within the problem
  int n;          // n_p
  int r;          // r_p
  int bn;         // MMA N: r_p rounded up to a multiple of 16 (<= 64)
  int xrow;       // first row of the problem's columns in the X parts
  int kt;         // K tiles of 64 columns
  int prob;       // problem index (active flag)
  int slot;       // partial slot of the item
  float lam;      // lambda_p (epilogue Y += lambda_p X)
  int pad;
};

// Xh/Xl rows xrow_p .. xrow_p + r_p, columns m0 .. m0 + 128 of every live item's problem.
// nitems: grid size; *cnt (device): the items actually present (CTAs beyond it return).
void launch_bsplit_x(const TcItem* items, int nitems, const int* cnt, const float* X, void* xh, void* xl,
                     int64_t lda, const void* ctl, size_t ctl_stride, size_t active_off, const int* run,
                     cudaStream_t s);
// Y_p rows of every live item = A_p (Xh + Xl) (+ lambda_p X_p), and, when part != NULL, the
// item's partial <P1, A_p X_p> in part[slot * nq].  Returns 0, or < 0 when the tensor maps
// cannot be encoded or the launch fails (tc_last_status has the code).
int launch_bgemm_tc(const void* A16, int64_t lda, int64_t rows_total, const void* xh, const void* xl,
                    int64_t xt_rows, const TcItem* items, int nitems, const int* cnt, const float* X, float* Y,
                    int add_lam,
                    const float* P1, double* part, int nq, const void* ctl, size_t ctl_stride,
                    size_t active_off, const int* run, int* err, long long budget, cudaStream_t s);

}  // namespace snmf
