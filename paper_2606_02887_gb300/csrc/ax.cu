// A*X products of SNMPBB: the only O(n^2 r) (dense) / O(nnz r) (sparse) step of an
// iteration (Sec. 4.1 complexity list; the V H^T product of Eqs. (2.1)-(2.2)).
//
//   k_gemm_dense : CUDA-core tiled GEMM for FP64 / FP32 A (64x64 CTA tile, 4x4 register
//                  micro-tile, smem staged, register prefetch).  Split-K writes each split
//                  to its own workspace slice; the finish pass sums the slices in a fixed
//                  order, so results are deterministic.
//   k_spmm_csr   : one warp per row, lanes across the factor columns (coalesced rows of X).
//   k_ax_finish  : fused epilogue: sum of split slices, Y += c X2, and per-restart FP64
//                  partials of <P1, A X> and <P2, A X> (e.g. tr(W^T A W)).
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace snmf {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;

__device__ __forceinline__ float ld_a(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ld_a(const float* p) { return *p; }
__device__ __forceinline__ double ld_a(const double* p) { return *p; }

// TA: stored type of A (T, or BF16 read into FP32 registers: the FP32-accumulated product
// of the stored BF16 operator, used where the tensor-core accumulation is not accurate
// enough, i.e. the closed-form objective of the final evaluation)
// SYM: A holds the upper 128 x 128 tiles of the symmetric matrix (sym_tile, lda = tiles a side);
// entry (r, k) below the diagonal tiles is entry (k, r) of the stored mirror tile.
template <typename T, typename TA = T, bool SYM = false>
__global__ void __launch_bounds__(256)
k_gemm_dense(const TA* __restrict__ A, int64_t lda, const T* __restrict__ X, int64_t ld,
             T* __restrict__ Y, int64_t n, int cols, int64_t kchunk, const int* run) {
  if (run && *run == 0) return;
  __shared__ T As[2][BK][BM + 4];
  __shared__ T Xs[2][BK][BN + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t row0 = (int64_t)blockIdx.y * BM;
  const int col0 = blockIdx.x * BN;
  const int64_t k_begin = (int64_t)blockIdx.z * kchunk;
  const int64_t k_end = min(n, k_begin + kchunk);
  T* Yout = Y + (int64_t)blockIdx.z * n * ld;

  // loader mapping: A tile BM x BK (row-major A: consecutive k contiguous)
  // each thread loads 4 elements: rows la_r + 16*m, column la_c
  const int la_c = threadIdx.x & 15;      // k offset
  const int la_r = threadIdx.x >> 4;      // 0..15
  // X tile BK x BN: thread loads 4 elements: row lx_r, cols lx_c + 16*m
  const int lx_c = threadIdx.x & 15;
  const int lx_r = threadIdx.x >> 4;

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  T ra[4], rx[4];
  auto load_regs = [&](int64_t k0) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      int64_t r = row0 + la_r + 16 * m;
      int64_t k = k0 + la_c;
      const TA* pa;
      if constexpr (SYM) {
        const int64_t ta = r >> 7, tb = k >> 7;
        pa = ta <= tb ? A + (sym_tile(ta, tb, lda) << 14) + ((r & 127) << 7) + (k & 127)
                      : A + (sym_tile(tb, ta, lda) << 14) + ((k & 127) << 7) + (r & 127);
      } else {
        pa = A + r * lda + k;
      }
      ra[m] = (r < n && k < k_end) ? (T)ld_a(pa) : T(0);
      int c = col0 + lx_c + 16 * m;
      int64_t kr = k0 + lx_r;
      rx[m] = (kr < k_end && c < cols) ? X[kr * ld + c] : T(0);
    }
  };
  auto store_smem = [&](int buf) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      As[buf][la_c][la_r + 16 * m] = ra[m];
      Xs[buf][lx_r][lx_c + 16 * m] = rx[m];
    }
  };

  int buf = 0;
  if (k_begin < k_end) {
    load_regs(k_begin);
    store_smem(0);
  }
  __syncthreads();
  for (int64_t k0 = k_begin; k0 < k_end; k0 += BK) {
    const bool more = (k0 + BK) < k_end;
    if (more) load_regs(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], x[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) x[j] = Xs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], x[j], acc[i][j]);
    }
    if (more) store_smem(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t r = row0 + ty + 16 * i;
    if (r >= n) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int c = col0 + tx + 16 * j;
      if (c < cols) Yout[r * ld + c] = acc[i][j];
    }
  }
}

// CSR SpMM: warp per row, lane owns columns lane + 32 m (m < CPL) of a column window.
template <typename TV, typename T, int CPL>
__global__ void __launch_bounds__(256)
k_spmm_csr(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
           const TV* __restrict__ vals, const T* __restrict__ X, int64_t ld,
           T* __restrict__ Y, int64_t n, int cols, const int* run) {
  if (run && *run == 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int c0 = blockIdx.y * (32 * CPL);
  if (row >= n) return;
  T acc[CPL];
#pragma unroll
  for (int m = 0; m < CPL; ++m) acc[m] = T(0);
  const int beg = rowptr[row], end = rowptr[row + 1];
  for (int e = beg; e < end; ++e) {
    const int64_t col = colidx[e];
    const T v = (T)vals[e];
    const T* xr = X + col * ld;
#pragma unroll
    for (int m = 0; m < CPL; ++m) {
      int c = c0 + lane + 32 * m;
      if (c < cols) acc[m] = fma(v, xr[c], acc[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < CPL; ++m) {
    int c = c0 + lane + 32 * m;
    if (c < cols) Y[row * ld + c] = acc[m];
  }
}

// Epilogue over a row tile x one restart.  splits > 1: Y = sum_s ws[s] (fixed order).
template <typename T>
__global__ void __launch_bounds__(256)
k_ax_finish(int64_t n, int r, int64_t ld, T* __restrict__ Y, const T* __restrict__ ws,
            int splits, double c, const T* __restrict__ X2, const T* __restrict__ P1,
            const T* __restrict__ P2, double* __restrict__ part, int q0, int b,
            const int* run, int dots_after) {
  __shared__ T sh[32];
  const int j = blockIdx.y;
  const int64_t i0 = (int64_t)blockIdx.x * kRowTile;
  T d1 = T(0), d2 = T(0);  // per-CTA partials in the working type (FP64 across CTAs)
  if (!(run && *run == 0)) {
    const int tile = kRowTile * r;
    for (int e = threadIdx.x; e < tile; e += blockDim.x) {
      const int64_t i = i0 + e / r;
      if (i >= n) break;
      const int64_t idx = i * ld + (int64_t)j * r + (e % r);
      T y;
      if (splits > 1) {
        y = ws[idx];
        for (int s = 1; s < splits; ++s) y += ws[(int64_t)s * n * ld + idx];
      } else {
        y = Y[idx];
      }
      if (!dots_after) {
        if (P1) d1 += P1[idx] * y;
        if (P2) d2 += P2[idx] * y;
      }
      if (X2) y = y + (T)c * X2[idx];
      if (dots_after) {
        if (P1) d1 += P1[idx] * y;
        if (P2) d2 += P2[idx] * y;
      }
      Y[idx] = y;
    }
  }
  d1 = block_sum_t(d1, sh);
  d2 = block_sum_t(d2, sh);
  if (threadIdx.x == 0) {
    double* p = part + ((int64_t)blockIdx.x * b + j) * kNQ;
    p[q0] = (double)d1;
    p[q0 + 1] = (double)d2;
  }
}

inline int cdiv64(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Structure check of a device-resident CSR matrix before its first product: rowptr[0] = 0,
// rowptr[n] = nnz, rowptr non-decreasing (bit 0 of *bad) and every column index in [0, n)
// (bit 1).  Grid-stride; only reads inside rowptr[0..n] and colidx[0..nnz).
__global__ void k_csr_check(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int64_t n,
                            int64_t nnz, int* __restrict__ bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int flag = 0;
  if (t0 == 0 && (rowptr[0] != 0 || (int64_t)rowptr[n] != nnz)) flag |= 1;
  for (int64_t i = t0; i < n; i += stride)
    if (rowptr[i + 1] < rowptr[i]) flag |= 1;
  for (int64_t e = t0; e < nnz; e += stride) {
    const int32_t c = colidx[e];
    if (c < 0 || (int64_t)c >= n) flag |= 2;
  }
  if (flag) atomicOr(bad, flag);
}

}  // namespace

void launch_csr_check(const int32_t* rowptr, const int32_t* colidx, int64_t n, int64_t nnz, int* bad,
                      cudaStream_t s) {
  const int64_t work = n > nnz ? n : nnz;
  int blocks = cdiv64(work > 0 ? work : 1, 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_csr_check<<<blocks, 256, 0, s>>>(rowptr, colidx, n, nnz, bad);
}

int launch_ax(const AxArgs& a, int tdtype, int64_t n, int cols, int64_t ld, const void* X,
              void* Y, void* ws, size_t ws_elems, const int* run, cudaStream_t s, const ProdTune* tune) {
  if (a.kind == AX_DENSE) {
    const int gx = cdiv64(cols, BN), gy = cdiv64(n, BM);
    // split-K: aim for >= 2 CTAs per SM (152 SMs) with chunks of >= 256
    int splits = 1;
    const int target = 2 * 152;
    while (gx * gy * splits < target && n / (splits * 2) >= 256) splits *= 2;
    if (tune && tune->splits > 0) splits = tune->splits;  // autotuned
    if ((size_t)splits * (size_t)n * (size_t)ld > ws_elems) splits = 1;
    int64_t kchunk = (n + splits - 1) / splits;
    kchunk = (kchunk + BK - 1) / BK * BK;
    dim3 grid(gx, gy, splits);
    void* out = splits > 1 ? ws : Y;
    if (a.a_dtype == 2 && a.sym)
      k_gemm_dense<float, __nv_bfloat16, true><<<grid, 256, 0, s>>>((const __nv_bfloat16*)a.A, a.lda,
                                                                    (const float*)X, ld, (float*)out, n, cols,
                                                                    kchunk, run);
    else if (a.a_dtype == 2)
      k_gemm_dense<float, __nv_bfloat16><<<grid, 256, 0, s>>>((const __nv_bfloat16*)a.A, a.lda, (const float*)X,
                                                              ld, (float*)out, n, cols, kchunk, run);
    else if (tdtype == 0)
      k_gemm_dense<double><<<grid, 256, 0, s>>>((const double*)a.A, a.lda, (const double*)X, ld,
                                                (double*)out, n, cols, kchunk, run);
    else
      k_gemm_dense<float><<<grid, 256, 0, s>>>((const float*)a.A, a.lda, (const float*)X, ld,
                                               (float*)out, n, cols, kchunk, run);
    return splits;
  }
  // CSR
  const int cpl = cols > 128 ? 8 : (cols > 64 ? 4 : (cols > 32 ? 2 : 1));
  dim3 grid(cdiv64(n, 8), cdiv64(cols, 32 * cpl));
#define SPMM_CASE(TV, T, C)                                                              \
  k_spmm_csr<TV, T, C><<<grid, 256, 0, s>>>(a.rowptr, a.colidx, (const TV*)a.vals,       \
                                            (const T*)X, ld, (T*)Y, n, cols, run)
#define SPMM_CPL(TV, T)                \
  switch (cpl) {                       \
    case 1: SPMM_CASE(TV, T, 1); break; \
    case 2: SPMM_CASE(TV, T, 2); break; \
    case 4: SPMM_CASE(TV, T, 4); break; \
    default: SPMM_CASE(TV, T, 8); break; \
  }
  if (tdtype == 0) {
    if (a.v_dtype == 0) { SPMM_CPL(double, double) } else { SPMM_CPL(float, double) }
  } else {
    if (a.v_dtype == 0) { SPMM_CPL(double, float) } else { SPMM_CPL(float, float) }
  }
#undef SPMM_CPL
#undef SPMM_CASE
  return 1;
}

int launch_ax_finish_impl(int tdtype, const Dims& d, void* Y, const void* ws, int splits,
                          double c, const void* X2, const void* P1, const void* P2,
                          double* part, int q0, const int* run, cudaStream_t s, int dots_after) {
  dim3 grid(cdiv64(d.n, kRowTile), d.b);
  if (tdtype == 0)
    k_ax_finish<double><<<grid, 256, 0, s>>>(d.n, d.r, d.ld, (double*)Y, (const double*)ws, splits,
                                             c, (const double*)X2, (const double*)P1,
                                             (const double*)P2, part, q0, d.b, run, dots_after);
  else
    k_ax_finish<float><<<grid, 256, 0, s>>>(d.n, d.r, d.ld, (float*)Y, (const float*)ws, splits, c,
                                            (const float*)X2, (const float*)P1, (const float*)P2,
                                            part, q0, d.b, run, dots_after);
  return grid.x;
}

// ---------------------------------------------------------------------------------------
// The paper's normalized graph Laplacian L = I - D^-1/2 A D^-1/2, d_i = sum_j a_ij (Sec. 2.2):
// the scaling s_i = d_i^-1/2 (0 for rows of zero degree) and the operator -D^-1/2 A D^-1/2
// in the factor type, applied as L X = X + (-D^-1/2 A D^-1/2) X.
// ---------------------------------------------------------------------------------------
namespace {

template <typename TA>
__global__ void k_degree_scale(int kind, const TA* __restrict__ A, int64_t lda, const int32_t* __restrict__ rowptr,
                               int64_t n, double* __restrict__ s) {
  // one warp per row, FP64 sum in a fixed order (lane stride, then a fixed butterfly)
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= n) return;
  double acc = 0.0;
  if (kind == AX_DENSE) {
    for (int64_t k = lane; k < n; k += 32) acc += (double)ld_a(A + i * lda + k);
  } else {
    for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) acc += (double)A[e];
  }
  acc = warp_sum(acc);
  if (lane == 0) s[i] = acc > 0.0 ? 1.0 / sqrt(acc) : 0.0;
}

template <typename TA, typename T>
__global__ void k_scaled_neg_csr(const TA* __restrict__ vals, const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ colidx, int64_t n, const double* __restrict__ s,
                                 T* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= n) return;
  for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32)
    out[e] = (T)(-(s[i] * (double)vals[e] * s[colidx[e]]));
}

template <typename TA, typename T>
__global__ void k_scaled_neg_dense(const TA* __restrict__ A, int64_t lda, int64_t n, const double* __restrict__ s,
                                   T* __restrict__ out) {
  const int64_t total = n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, k = e % n;
    out[e] = (T)(-(s[i] * (double)ld_a(A + i * lda + k) * s[k]));
  }
}

}  // namespace

void launch_normalized_adjacency(const AxArgs& a, int tdtype, int64_t n, double* s, void* out, cudaStream_t st) {
  const int rb = cdiv64(n, 8);
  if (a.kind == AX_DENSE) {
    const int blocks = (int)std::min<int64_t>(cdiv64(n * n, 256), 152 * 32);
    if (a.a_dtype == 0) {
      k_degree_scale<double><<<rb, 256, 0, st>>>(AX_DENSE, (const double*)a.A, a.lda, nullptr, n, s);
      if (tdtype == 0) k_scaled_neg_dense<double, double><<<blocks, 256, 0, st>>>((const double*)a.A, a.lda, n, s, (double*)out);
      else k_scaled_neg_dense<double, float><<<blocks, 256, 0, st>>>((const double*)a.A, a.lda, n, s, (float*)out);
    } else {
      k_degree_scale<float><<<rb, 256, 0, st>>>(AX_DENSE, (const float*)a.A, a.lda, nullptr, n, s);
      if (tdtype == 0) k_scaled_neg_dense<float, double><<<blocks, 256, 0, st>>>((const float*)a.A, a.lda, n, s, (double*)out);
      else k_scaled_neg_dense<float, float><<<blocks, 256, 0, st>>>((const float*)a.A, a.lda, n, s, (float*)out);
    }
    return;
  }
  if (a.v_dtype == 0) {
    k_degree_scale<double><<<rb, 256, 0, st>>>(AX_CSR, (const double*)a.vals, 0, a.rowptr, n, s);
    if (tdtype == 0) k_scaled_neg_csr<double, double><<<rb, 256, 0, st>>>((const double*)a.vals, a.rowptr, a.colidx, n, s, (double*)out);
    else k_scaled_neg_csr<double, float><<<rb, 256, 0, st>>>((const double*)a.vals, a.rowptr, a.colidx, n, s, (float*)out);
  } else {
    k_degree_scale<float><<<rb, 256, 0, st>>>(AX_CSR, (const float*)a.vals, 0, a.rowptr, n, s);
    if (tdtype == 0) k_scaled_neg_csr<float, double><<<rb, 256, 0, st>>>((const float*)a.vals, a.rowptr, a.colidx, n, s, (double*)out);
    else k_scaled_neg_csr<float, float><<<rb, 256, 0, st>>>((const float*)a.vals, a.rowptr, a.colidx, n, s, (float*)out);
  }
}

}  // namespace snmf
