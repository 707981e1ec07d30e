// FP8 storage of A for the A*X products: A~ = E4M3(A / s_t) * s_t with a power-of-two
// scale s_t per 128 x 128 tile (the smallest 2^k with max|A_t| / 2^k <= 448), and the
// CUDA-core product Y = A~ X that dequantizes the codes while staging them (the final
// evaluation's product, with X in FP32; the iteration's products run on the tensor cores,
// k_gemm_tc<true> in ax_tc.cu).
//
//   k_fp8_scales : one CTA per tile: max|A_t| (fixed-shape block reduction), s_t exactly
//                  from frexp (no rounding in the exponent choice)
//   k_fp8_encode : codes q = E4M3(A / s_t), round to nearest even, saturating at +-448
//   k_fp8_sums   : ||A~||^2 and sum(A~) of the stored values (FP64 partial per CTA)
//   k_gemm_fp8   : 64 x 64 CTA tile over a K chunk (split-K into workspace slices like
//                  the FP32 product): 4 codes per thread per stage, decoded to FP32 and
//                  scaled in registers, then the same shared-memory FFMA tile as FP32
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "fp8.cuh"

namespace snmf {

namespace {

constexpr int kTile = 128;
constexpr int BM = 64, BN = 64, BK = 16;

template <typename TS>
__global__ void __launch_bounds__(256)
k_fp8_scales(const TS* __restrict__ A, int64_t n, int64_t lda, float* __restrict__ scales, int nt) {
  __shared__ double sh[32];
  const int ti = blockIdx.y, tj = blockIdx.x;
  double m = 0.0;
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    const int64_t i = (int64_t)ti * kTile + e / kTile, k = (int64_t)tj * kTile + e % kTile;
    if (i < n && k < n) m = fmax(m, fabs((double)A[i * lda + k]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, sh[w]);
    float s = 1.0f;
    if (mx > 0.0) {
      // mx / 448 = f 2^e, f in [0.5, 1): the smallest k with mx / 2^k <= 448 is e - 1 when
      // f == 0.5 (an exact power of two), else e
      int e;
      const double f = frexp(mx / 448.0, &e);
      const int k = (f == 0.5) ? e - 1 : e;
      s = (float)ldexp(1.0, k);
    }
    scales[ti * nt + tj] = s;
  }
}

template <typename TS>
__global__ void __launch_bounds__(256)
k_fp8_encode(const TS* __restrict__ A, int64_t n, int64_t lda, const float* __restrict__ scales, int nt,
             __nv_fp8_storage_t* __restrict__ A8, int64_t lda8) {
  const int64_t total = n * lda8;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / lda8, k = e % lda8;
    __nv_fp8_storage_t q = 0;
    if (k < n) {
      const double s = scales[(i / kTile) * nt + (k / kTile)];
      q = __nv_cvt_double_to_fp8((double)A[i * lda + k] / s, __NV_SATFINITE, __NV_E4M3);
    }
    A8[e] = q;
  }
}

__device__ __forceinline__ float fp8_value(__nv_fp8_storage_t q) {
  const __half_raw h = __nv_cvt_fp8_to_halfraw(q, __NV_E4M3);
  return __half2float(__half(h));
}

__global__ void __launch_bounds__(256)
k_fp8_sums(const __nv_fp8_storage_t* __restrict__ A8, int64_t n, int64_t lda8, const float* __restrict__ scales,
           int nt, double* __restrict__ part) {
  __shared__ double sh2[32], sh1[32];
  double s2 = 0.0, s1 = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * lda8; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / lda8, k = e % lda8;
    if (k >= n) continue;
    const double v = (double)fp8_value(A8[e]) * (double)scales[(i / kTile) * nt + (k / kTile)];
    s2 += v * v;
    s1 += v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sh2[wid] = s2; sh1[wid] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sh2[w]; b += sh1[w]; }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// Y (or split slice z of ws) = A~[rows, K chunk z] X[K chunk z, cols]
__global__ void __launch_bounds__(256)
k_gemm_fp8(const __nv_fp8_storage_t* __restrict__ A8, int64_t lda8, const float* __restrict__ scales, int nt,
           const float* __restrict__ X, int64_t ld, float* __restrict__ Y, int64_t n, int cols, int64_t kchunk,
           const int* run) {
  if (run && *run == 0) return;
  __shared__ float As[2][BK][BM + 4];
  __shared__ float Xs[2][BK][BN + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t row0 = (int64_t)blockIdx.y * BM;
  const int col0 = blockIdx.x * BN;
  const int64_t k_begin = (int64_t)blockIdx.z * kchunk;
  const int64_t k_end = min(n, k_begin + kchunk);
  float* Yout = Y + (int64_t)blockIdx.z * n * ld;
  const float* srow = scales + (row0 / kTile) * nt;  // the CTA's 64 rows lie in one scale row
  // A loader: row la_r, 4 consecutive codes at k offset la_k (4-byte aligned: lda8 and the
  // chunk start are multiples of 16)
  const int la_r = threadIdx.x >> 2, la_k = (threadIdx.x & 3) * 4;
  const int lx_c = threadIdx.x & 15, lx_r = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  uint32_t ra;
  float rx[4];
  auto load_regs = [&](int64_t k0) {
    const int64_t r = row0 + la_r;
    ra = r < n ? *reinterpret_cast<const uint32_t*>(A8 + r * lda8 + k0 + la_k) : 0u;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int c = col0 + lx_c + 16 * m;
      const int64_t kr = k0 + lx_r;
      rx[m] = (kr < k_end && c < cols) ? X[kr * ld + c] : 0.f;
    }
  };
  auto store_smem = [&](int buf, int64_t k0) {
    const float s = srow[k0 / kTile];  // the 16-code chunk lies in one scale column
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const __nv_fp8_storage_t q = (__nv_fp8_storage_t)((ra >> (8 * u)) & 0xFFu);
      const bool in = k0 + la_k + u < k_end;  // codes of the next split are not this CTA's
      As[buf][la_k + u][la_r] = in ? fp8_value(q) * s : 0.f;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) Xs[buf][lx_r][lx_c + 16 * m] = rx[m];
  };
  int buf = 0;
  if (k_begin < k_end) {
    load_regs(k_begin);
    store_smem(0, k_begin);
  }
  __syncthreads();
  for (int64_t k0 = k_begin; k0 < k_end; k0 += BK) {
    const bool more = (k0 + BK) < k_end;
    if (more) load_regs(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], x[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = Xs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], x[j], acc[i][j]);
    }
    if (more) store_smem(buf ^ 1, k0 + BK);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t r = row0 + ty + 16 * i;
    if (r >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx + 16 * j;
      if (c < cols) Yout[r * ld + c] = acc[i][j];
    }
  }
}

inline int cdiv64(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace

int64_t fp8_ld(int64_t n) { return (n + 15) / 16 * 16; }
int fp8_ntiles(int64_t n) { return cdiv64(n, kTile); }

void launch_fp8_encode(int src_dtype, const void* A, int64_t n, int64_t lda, void* A8, float* scales,
                       cudaStream_t s) {
  const int nt = fp8_ntiles(n);
  const int64_t lda8 = fp8_ld(n);
  dim3 g(nt, nt);
  const int64_t tot = n * lda8;
  const int blocks = (int)((tot + 255) / 256 < 152 * 16 ? (tot + 255) / 256 : 152 * 16);
  if (src_dtype == 0) {
    k_fp8_scales<double><<<g, 256, 0, s>>>((const double*)A, n, lda, scales, nt);
    k_fp8_encode<double><<<blocks, 256, 0, s>>>((const double*)A, n, lda, scales, nt, (__nv_fp8_storage_t*)A8, lda8);
  } else {
    k_fp8_scales<float><<<g, 256, 0, s>>>((const float*)A, n, lda, scales, nt);
    k_fp8_encode<float><<<blocks, 256, 0, s>>>((const float*)A, n, lda, scales, nt, (__nv_fp8_storage_t*)A8, lda8);
  }
}

int launch_fp8_sums(const void* A8, int64_t n, const float* scales, double* part, cudaStream_t s) {
  const int64_t lda8 = fp8_ld(n);
  const int blocks = (int)((n * lda8 + 255) / 256 < 1024 ? (n * lda8 + 255) / 256 : 1024);
  k_fp8_sums<<<blocks, 256, 0, s>>>((const __nv_fp8_storage_t*)A8, n, lda8, scales, fp8_ntiles(n), part);
  return blocks;
}

int launch_ax_fp8(const void* A8, const float* scales, int64_t n, const float* X, int cols, int64_t ld, float* Y,
                  float* ws, size_t ws_elems, const int* run, cudaStream_t s, const ProdTune* tune) {
  const int gx = cdiv64(cols, BN), gy = cdiv64(n, BM);
  int splits = 1;
  while (gx * gy * splits < 2 * 152 && n / (splits * 2) >= 256) splits *= 2;
  if (tune && tune->splits > 0) splits = tune->splits;  // autotuned
  if ((size_t)splits * (size_t)n * (size_t)ld > ws_elems) splits = 1;
  int64_t kchunk = (n + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  dim3 grid(gx, gy, splits);
  k_gemm_fp8<<<grid, 256, 0, s>>>((const __nv_fp8_storage_t*)A8, fp8_ld(n), scales, fp8_ntiles(n), X, ld,
                                  splits > 1 ? ws : Y, n, cols, kchunk, run);
  return splits;
}

}  // namespace snmf
