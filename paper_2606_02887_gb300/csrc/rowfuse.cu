// Row kernels of an Algorithm-1 step for FP32 penalty blocks with r in {16, 32, 64}: the
// D step and the relaxed update, with the two row products X G on register tiles.
//
// Data flow per step (restart j, block variable X, fixed Gram G = H H^T + lambda I, fixed
// B = A H^T + lambda H^T; Eqs. (2.1)-(2.2)):
//   D step : reads X, g = grad f(X), B;  Z = Proj[X - g / rho]        (Alg. 1 line 2)
//            g(Z) = Z G - B;  D = Proj[Z - alpha g(Z)] - Z            (Alg. 1 line 3)
//            writes g(Z) only; partials <g(Z), D>, ||D||^2, f(Z) - f(X), <D G, D>; the last
//            CTA of each restart runs the closed-form line search   (Alg. 1 line 4)
//   update : reads X, g, g(Z), B;  Z and D recomputed with the same instructions (the same
//            values bit for bit, so neither is stored);  X' = Proj[Z + phi beta D]
//            g(X') = X' G - B;  writes X', g(X') over X, g;  partials ||P grad||^2,
//            f(X') - const, <S,S>, <S,Y>, <Y,Y>, f(X') - f(Z), zero entries; the last CTA
//            of each restart computes the next BB step                (Alg. 1 line 3)
// So a step moves 4 + 6 arrays of n x r per restart instead of 6 + 8 when Z and D are
// stored.  Partial layout and control steps are those of the general row kernel.
//
// CTA: restart blockIdx.y, rows [BM blockIdx.x, BM (blockIdx.x + 1)), all R columns;
// 256 threads as TY row groups x TX = R / 4 column groups; thread (tx, ty) owns rows
// ty MR .. ty MR + MR - 1 and columns 4 tx .. 4 tx + 3 (float4 global accesses).  The row
// product Y = T G keeps T transposed in shared memory (Ts[k][row]), so a thread reads its
// MR rows of column k as MR / 4 16-byte broadcasts and its four G entries as one.
#include <math.h>

#include "common.cuh"
#include "rowops.cuh"
#include "rowops_dev.cuh"

namespace snmf {

namespace {

template <int R, int MR>
struct FuseCfg {
  static constexpr int TX = R / 4;       // column groups of four
  static constexpr int TY = 256 / TX;    // row groups
  static constexpr int BM = TY * MR;     // rows per CTA
  static constexpr int TS = BM + 4;      // row stride of the transposed tile (floats)
  static constexpr size_t smem = ((size_t)R * TS + (size_t)R * R) * sizeof(float);
};

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// Z = Proj[X - g / rho] and D = Proj[Z - alpha g(Z)] - Z, written with explicit FMAs so the D
// step and the update compute the same bits.
__device__ __forceinline__ float zstep1(float x, float g, float inv_rho) {
  const float t = __fmaf_rn(-g, inv_rho, x);
  return t > 0.f ? t : 0.f;
}
__device__ __forceinline__ float dir1(float z, float gz, float alpha) {
  const float t = __fmaf_rn(-alpha, gz, z);
  return (t > 0.f ? t : 0.f) - z;
}
__device__ __forceinline__ float upd1(float z, float d, float pb) {
  const float t = __fmaf_rn(pb, d, z);
  return t > 0.f ? t : 0.f;
}

__device__ __forceinline__ float comp(const float4& v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}

// Store the thread's MR x 4 values v[p][q] into Ts[4 tx + q][ty MR + p] (16-byte stores).
template <int R, int MR>
__device__ __forceinline__ void store_transposed(float* Ts, const float (&v)[MR][4], int tx, int ty) {
  using C = FuseCfg<R, MR>;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float* dst = Ts + (4 * tx + q) * C::TS + ty * MR;
    if (MR % 4 == 0) {
#pragma unroll
      for (int p = 0; p < MR; p += 4) st4(dst + p, make_float4(v[p][q], v[p + 1][q], v[p + 2][q], v[p + 3][q]));
    } else {
#pragma unroll
      for (int p = 0; p < MR; p += 2)
        *reinterpret_cast<float2*>(dst + p) = make_float2(v[p][q], v[p + 1][q]);
    }
  }
}

// acc[p][q] = sum_k Ts[k][ty MR + p] G[k][4 tx + q]
template <int R, int MR>
__device__ __forceinline__ void row_product(const float* Ts, const float* Gs, int tx, int ty, float (&acc)[MR][4]) {
  using C = FuseCfg<R, MR>;
#pragma unroll
  for (int p = 0; p < MR; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
  const float* ta = Ts + ty * MR;
  const float* gb = Gs + 4 * tx;
#pragma unroll 4
  for (int k = 0; k < R; ++k) {
    float a[MR];
    if (MR % 4 == 0) {
#pragma unroll
      for (int p = 0; p < MR; p += 4) {
        const float4 t = ld4(ta + k * C::TS + p);
        a[p] = t.x; a[p + 1] = t.y; a[p + 2] = t.z; a[p + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int p = 0; p < MR; p += 2) {
        const float2 t = *reinterpret_cast<const float2*>(ta + k * C::TS + p);
        a[p] = t.x; a[p + 1] = t.y;
      }
    }
    const float4 b = ld4(gb + k * R);
#pragma unroll
    for (int p = 0; p < MR; ++p) {
      acc[p][0] = fmaf(a[p], b.x, acc[p][0]);
      acc[p][1] = fmaf(a[p], b.y, acc[p][1]);
      acc[p][2] = fmaf(a[p], b.z, acc[p][2]);
      acc[p][3] = fmaf(a[p], b.w, acc[p][3]);
    }
  }
}

// Fixed-order CTA reduction of the 8 partial values, slot write, and the control step of
// the last CTA of restart j (arrival counter, as in the general row kernel).
__device__ __forceinline__ void finish_partials(const RowArgs& a, const float (&dq)[8], int j, int slot,
                                                unsigned per, float (*shq)[8], unsigned* ticket, int nc) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const float v = warp_sum(dq[m]);
    if (lane == 0) shq[m][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) v += shq[threadIdx.x][w];
    a.part[((int64_t)slot * a.b + j) * kNQ + threadIdx.x] = (double)v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *ticket = atomicAdd(&a.counters[j], 1u);
  __syncthreads();
  if (*ticket == per - 1) {
    if (threadIdx.x == 0) a.counters[j] = 0u;
    if (threadIdx.x < 32)
      fused_control(a.ctl_mode, const_cast<Ctl&>(a.ctl[j]), a.part, (int)per, a.b, a.r, j, a.P, a.G64fix, nullptr,
                    nc);
  }
}

template <int R>
__device__ __forceinline__ void load_gram(const RowArgs& a, int j, float* Gs) {
  const float4* G = reinterpret_cast<const float4*>((const float*)a.G + (int64_t)j * R * R);
  for (int e = threadIdx.x; e < R * R / 4; e += 256) reinterpret_cast<float4*>(Gs)[e] = G[e];
}

// ---------------------------------------------------------------------------------------
// D step: q0 <g(Z), D>, q1 ||D||^2, q2 f(Z) - f(X) (trapezoid, exact for the quadratic
// block), q4 <D G, D>; q3 zero.  NC = 2 (learned step with fallback): D is the proposal's
// direction (step cand_alpha[0]) and q5 <g(Z), D_1>, q6 ||D_1||^2, q7 <D_1 G, D_1> belong to
// the plain BB direction D_1 (step cand_alpha[1]); the line search picks one (Ctl::dsel) and
// the update recomputes that one.  NC = 1: q5-q7 zero, step Ctl::alpha.
// ---------------------------------------------------------------------------------------
template <int R, int MR, int NC>
__global__ void __launch_bounds__(256, MR >= 8 ? 2 : 3) k_rowfuse_dstep(RowArgs a) {
  using C = FuseCfg<R, MR>;
  extern __shared__ __align__(16) float fsm[];
  float* Ts = fsm;
  float* Gs = fsm + R * C::TS;
  __shared__ float shq[8][8];
  __shared__ unsigned ticket;
  const int j = blockIdx.y;
  const Ctl& cj = a.ctl[j];
  const bool live = cj.active && !(a.run && *a.run == 0);
  float dq[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) dq[m] = 0.f;
  if (live) {
    const int tx = threadIdx.x % C::TX, ty = threadIdx.x / C::TX;
    const int64_t row0 = (int64_t)blockIdx.x * C::BM + ty * MR;
    const int64_t col = (int64_t)j * R + 4 * tx;
    const float* X = (const float*)a.X;
    const float* g = (const float*)a.g_in;
    const float* B = (const float*)a.B;
    float* gZo = (float*)a.gZout;
    const float inv_rho = (float)(1.0 / cj.rho);
    const float alpha = (float)(NC == 1 ? cj.alpha : cj.cand_alpha[0]);
    const float alpha1 = (float)(NC == 1 ? cj.alpha : cj.cand_alpha[1]);
    load_gram<R>(a, j, Gs);
    float v[MR][4];
    {  // Z tile (transposed) for the row product
      float4 x4[MR], g4[MR];
#pragma unroll
      for (int p = 0; p < MR; ++p) {
        const int64_t i = row0 + p;
        x4[p] = g4[p] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < a.n) {
          x4[p] = ld4(X + i * a.ld + col);
          g4[p] = ld4(g + i * a.ld + col);
        }
      }
#pragma unroll
      for (int p = 0; p < MR; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) v[p][q] = zstep1(comp(x4[p], q), comp(g4[p], q), inv_rho);
    }
    store_transposed<R, MR>(Ts, v, tx, ty);
    __syncthreads();
    float acc[MR][4];
    row_product<R, MR>(Ts, Gs, tx, ty, acc);
    // epilogue: g(Z), D, the partial inner products; D kept in acc for <D G, D> (NC = 2:
    // g(Z) kept in v for the second direction)
#pragma unroll
    for (int p = 0; p < MR; ++p) {
      const int64_t i = row0 + p;
      if (i < a.n) {
        const int64_t off = i * a.ld + col;
        const float4 x4 = ld4(X + off), g4 = ld4(g + off), b4 = ld4(B + off);
        float gz[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float x = comp(x4, q), gx = comp(g4, q);
          const float z = zstep1(x, gx, inv_rho);
          gz[q] = acc[p][q] - comp(b4, q);
          const float d = dir1(z, gz[q], alpha);
          dq[0] += gz[q] * d;
          dq[1] += d * d;
          dq[2] += 0.5f * (z - x) * (gz[q] + gx);
          if (NC == 2) {
            const float d1 = dir1(z, gz[q], alpha1);
            dq[5] += gz[q] * d1;
            dq[6] += d1 * d1;
            v[p][q] = d1;
          }
          acc[p][q] = d;
        }
        st4(gZo + off, make_float4(gz[0], gz[1], gz[2], gz[3]));
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = v[p][q] = 0.f;
      }
    }
    __syncthreads();  // every thread is done reading the Z tile
    store_transposed<R, MR>(Ts, acc, tx, ty);
    __syncthreads();
    float dg[MR][4];
    row_product<R, MR>(Ts, Gs, tx, ty, dg);
    float qq = 0.f;
#pragma unroll
    for (int p = 0; p < MR; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) qq = fmaf(dg[p][q], acc[p][q], qq);
    dq[4] = qq;
    if (NC == 2) {  // <D_1 G, D_1> of the plain BB direction
      __syncthreads();
      store_transposed<R, MR>(Ts, v, tx, ty);
      __syncthreads();
      row_product<R, MR>(Ts, Gs, tx, ty, dg);
      float q1 = 0.f;
#pragma unroll
      for (int p = 0; p < MR; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) q1 = fmaf(dg[p][q], v[p][q], q1);
      dq[7] = q1;
    }
  }
  finish_partials(a, dq, j, blockIdx.x, gridDim.x, shq, &ticket, NC);
}

// ---------------------------------------------------------------------------------------
// Update: q0 ||P grad f(X')||^2, q1 1/2 <g' - B, X'>, q2 <S,S>, q3 <S,Y>, q4 <Y,Y>,
// q5 f(X') - f(Z) (trapezoid), q6 zero entries of X'; q7 zero.
// ---------------------------------------------------------------------------------------
template <int R, int MR, int NC>
__global__ void __launch_bounds__(256, MR >= 8 ? 2 : 3) k_rowfuse_update(RowArgs a) {
  using C = FuseCfg<R, MR>;
  extern __shared__ __align__(16) float fsm[];
  float* Ts = fsm;
  float* Gs = fsm + R * C::TS;
  __shared__ float shq[8][8];
  __shared__ unsigned ticket;
  const int j = blockIdx.y;
  const Ctl& cj = a.ctl[j];
  const bool live = cj.active && !(a.run && *a.run == 0);
  float dq[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) dq[m] = 0.f;
  if (live) {
    const int tx = threadIdx.x % C::TX, ty = threadIdx.x / C::TX;
    const int64_t row0 = (int64_t)blockIdx.x * C::BM + ty * MR;
    const int64_t col = (int64_t)j * R + 4 * tx;
    float* X = (float*)a.Xout;        // in place: X_k in, X_{k+1} out
    float* g = (float*)a.gout;        // in place: g(X_k) in, g(X_{k+1}) out
    const float* gZ = (const float*)a.gZold;
    const float* B = (const float*)a.B;
    const float inv_rho = (float)(1.0 / cj.rho);
    // the step of the direction the line search kept: NC = 2 selects the proposal or the
    // plain BB direction (dsel); the same float as the D step used
    const float alpha = (float)(NC == 1 ? cj.alpha : cj.cand_alpha[cj.dsel ? 1 : 0]);
    const float pb = (float)cj.phibeta;
    load_gram<R>(a, j, Gs);
    float v[MR][4];
    {  // X' tile (transposed) for the row product
      float4 x4[MR], g4[MR], z4[MR];
#pragma unroll
      for (int p = 0; p < MR; ++p) {
        const int64_t i = row0 + p;
        x4[p] = g4[p] = z4[p] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < a.n) {
          x4[p] = ld4(X + i * a.ld + col);
          g4[p] = ld4(g + i * a.ld + col);
          z4[p] = ld4(gZ + i * a.ld + col);
        }
      }
#pragma unroll
      for (int p = 0; p < MR; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float z = zstep1(comp(x4[p], q), comp(g4[p], q), inv_rho);
          v[p][q] = upd1(z, dir1(z, comp(z4[p], q), alpha), pb);
        }
    }
    store_transposed<R, MR>(Ts, v, tx, ty);
    __syncthreads();
    float acc[MR][4];
    row_product<R, MR>(Ts, Gs, tx, ty, acc);
#pragma unroll
    for (int p = 0; p < MR; ++p) {
      const int64_t i = row0 + p;
      if (i >= a.n) continue;
      const int64_t off = i * a.ld + col;
      const float4 x4 = ld4(X + off), g4 = ld4(g + off), gz4 = ld4(gZ + off), b4 = ld4(B + off);
      float xo[4], go[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float x = comp(x4, q), gx = comp(g4, q), gz = comp(gz4, q), bb = comp(b4, q);
        const float z = zstep1(x, gx, inv_rho);
        const float xn = upd1(z, dir1(z, gz, alpha), pb);
        const float gn = acc[p][q] - bb;
        const float pgv = xn > 0.f ? gn : (gn < 0.f ? gn : 0.f);
        dq[0] += pgv * pgv;
        dq[1] += 0.5f * (gn - bb) * xn;
        const float sv = xn - x, yv = gn - gx;
        dq[2] += sv * sv;
        dq[3] += sv * yv;
        dq[4] += yv * yv;
        dq[5] += 0.5f * (xn - z) * (gn + gz);
        if (xn == 0.f) dq[6] += 1.f;
        xo[q] = xn;
        go[q] = gn;
      }
      st4(X + off, make_float4(xo[0], xo[1], xo[2], xo[3]));
      st4(g + off, make_float4(go[0], go[1], go[2], go[3]));
    }
  }
  finish_partials(a, dq, j, blockIdx.x, gridDim.x, shq, &ticket, NC);
}

template <int R, int MR, int NC>
void launch_pair(int which, const RowArgs& a, cudaStream_t s) {
  using C = FuseCfg<R, MR>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rowfuse_dstep<R, MR, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    cudaFuncSetAttribute(k_rowfuse_update<R, MR, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    attr = true;
  }
  dim3 grid((unsigned)((a.n + C::BM - 1) / C::BM), (unsigned)a.b);
  if (which == 0) k_rowfuse_dstep<R, MR, NC><<<grid, 256, C::smem, s>>>(a);
  else k_rowfuse_update<R, MR, NC><<<grid, 256, C::smem, s>>>(a);
}

template <int NC>
void dispatch_nc(int which, const RowArgs& a, int bm, cudaStream_t s) {
  switch (a.r) {
    case 64:
      if (bm == 64) launch_pair<64, 4, NC>(which, a, s); else launch_pair<64, 8, NC>(which, a, s);
      break;
    case 32:
      if (bm == 64) launch_pair<32, 2, NC>(which, a, s); else launch_pair<32, 4, NC>(which, a, s);
      break;
    default:
      if (bm == 256) launch_pair<16, 4, NC>(which, a, s); else launch_pair<16, 2, NC>(which, a, s);
      break;
  }
}

void dispatch(int which, const RowArgs& a, int bm, int nc, cudaStream_t s) {
  if (nc == 2) dispatch_nc<2>(which, a, bm, s);
  else dispatch_nc<1>(which, a, bm, s);
}

}  // namespace

bool rowfuse_supported(int tdtype, int r) { return tdtype == 1 && (r == 16 || r == 32 || r == 64); }

int rowfuse_bm(int r, int bm_req) {
  if (r == 16) return bm_req == 256 ? 256 : 128;
  return bm_req == 64 ? 64 : 128;
}

void launch_rowfuse_dstep(const RowArgs& a, int bm, int nc, cudaStream_t s) {
  dispatch(0, a, rowfuse_bm(a.r, bm), nc, s);
}

void launch_rowfuse_update(const RowArgs& a, int bm, int nc, cudaStream_t s) {
  dispatch(1, a, rowfuse_bm(a.r, bm), nc, s);
}

}  // namespace snmf
