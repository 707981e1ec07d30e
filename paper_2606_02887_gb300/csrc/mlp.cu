// Learned step controller: training of the 5 -> 64 (ReLU) -> 1 MLP on the GPU.
//
// Loss (mean over samples): (2 tanh(o) - t)^2 with o = W2 relu(W1 phi + b1) + b2 and t the
// log2 of the best candidate multiplier recorded by the solver's record mode.  Forward and
// backward in FP32: one thread per sample, per-CTA partial gradients reduced in a fixed
// order, then an Adam step on FP32 master weights (k_mlp_step).  Parameter layout:
// W1[64][5], b1[64], W2[64], b2 (449 floats).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "../../include/snmf.h"
#include "common.cuh"
#include "mlp_dev.cuh"

namespace snmf {
namespace {

constexpr int NP = kMlpParams;

// One warp per feature vector: the solver's inference routine on BF16 weights.
__global__ void __launch_bounds__(256)
k_mlp_eval(const __nv_bfloat16* __restrict__ w, const float* __restrict__ feat, int count, float* __restrict__ mult) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= count) return;
  float phi[kMlpIn];
#pragma unroll
  for (int u = 0; u < kMlpIn; ++u) phi[u] = feat[(int64_t)i * kMlpIn + u];
  const float m = mlp_multiplier(w, phi);
  if ((threadIdx.x & 31) == 0) mult[i] = m;
}

// per-CTA partial gradient (NP floats) and loss at pgrad[blockIdx.x][NP + 1]
__global__ void __launch_bounds__(256)
k_mlp_grad(const float* __restrict__ feat, const float* __restrict__ targ, int count,
           const float* __restrict__ w, float* __restrict__ pgrad) {
  __shared__ float wsh[NP];
  __shared__ float red[8][32];
  for (int e = threadIdx.x; e < NP; e += blockDim.x) wsh[e] = w[e];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < count;
  float phi[kMlpIn];
#pragma unroll
  for (int u = 0; u < kMlpIn; ++u) phi[u] = valid ? feat[(int64_t)i * kMlpIn + u] : 0.f;
  const float* W1 = wsh;
  const float* b1 = wsh + kMlpIn * kMlpHidden;
  const float* W2 = b1 + kMlpHidden;
  const float b2 = wsh[NP - 1];
  float h[kMlpHidden];
  float o = b2;
#pragma unroll
  for (int k = 0; k < kMlpHidden; ++k) {
    float z = b1[k];
#pragma unroll
    for (int u = 0; u < kMlpIn; ++u) z = fmaf(W1[k * kMlpIn + u], phi[u], z);
    h[k] = fmaxf(z, 0.f);
    o = fmaf(W2[k], h[k], o);
  }
  const float th = tanhf(o);
  const float err = 2.f * th - (valid ? targ[i] : 0.f);
  const float inv_n = 1.f / (float)count;
  const float loss = valid ? err * err * inv_n : 0.f;
  const float dlo = valid ? 2.f * err * 2.f * (1.f - th * th) * inv_n : 0.f;  // dL/do
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  auto emit = [&](float v, int p) {
    v = warp_sum(v);
    if (lane == 0) red[wid][p & 31] = v;
  };
  float* out = pgrad + (int64_t)blockIdx.x * (NP + 1);
  // process the NP + 1 outputs in groups of 32 (fixed-order reductions)
  for (int g0 = 0; g0 < NP + 1; g0 += 32) {
    for (int p = g0; p < g0 + 32 && p < NP + 1; ++p) {
      float v;
      if (p < kMlpIn * kMlpHidden) {
        const int k = p / kMlpIn, u = p % kMlpIn;
        v = (h[k] > 0.f) ? dlo * W2[k] * phi[u] : 0.f;
      } else if (p < kMlpIn * kMlpHidden + kMlpHidden) {
        const int k = p - kMlpIn * kMlpHidden;
        v = (h[k] > 0.f) ? dlo * W2[k] : 0.f;
      } else if (p < NP - 1) {
        const int k = p - kMlpIn * kMlpHidden - kMlpHidden;
        v = dlo * h[k];
      } else if (p == NP - 1) {
        v = dlo;
      } else {
        v = loss;
      }
      emit(v, p);
    }
    __syncthreads();
    if (threadIdx.x < 32 && g0 + threadIdx.x < NP + 1) {
      float t = 0.f;
      for (int u = 0; u < 8; ++u) t += red[u][threadIdx.x];
      out[g0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// sum the CTA partials in order; Adam step (lr, 0.9, 0.999, 1e-8) on w with moments m, v
__global__ void k_mlp_step(const float* __restrict__ pgrad, int nblocks, float* __restrict__ w,
                           float* __restrict__ m, float* __restrict__ v, float* __restrict__ grad_out,
                           float* __restrict__ loss_out, int step, float lr, int apply) {
  for (int p = threadIdx.x; p < NP + 1; p += blockDim.x) {
    float g = 0.f;
    for (int b = 0; b < nblocks; ++b) g += pgrad[(int64_t)b * (NP + 1) + p];
    if (p == NP) { *loss_out = g; continue; }
    if (grad_out) grad_out[p] = g;
    if (!apply) continue;
    const float b1 = 0.9f, b2 = 0.999f;
    m[p] = b1 * m[p] + (1.f - b1) * g;
    v[p] = b2 * v[p] + (1.f - b2) * g * g;
    const float mh = m[p] / (1.f - powf(b1, (float)step));
    const float vh = v[p] / (1.f - powf(b2, (float)step));
    w[p] -= lr * mh / (sqrtf(vh) + 1e-8f);
  }
}

}  // namespace
}  // namespace snmf

using namespace snmf;

extern "C" snmf_status snmf_mlp_train(const float* feats, const float* targets, int count, float* weights,
                                      int steps, double lr, double* loss_out, float* grad0) {
  if (!feats || !targets || !weights || count < 1 || steps < 0 || !(lr > 0.0)) return SNMF_ERR_ARG;
  const int nb = (count + 255) / 256;
  float *df = nullptr, *dt = nullptr, *dw = nullptr, *dm = nullptr, *dv = nullptr, *pg = nullptr, *dg = nullptr,
        *dl = nullptr;
  auto cleanup = [&] {
    cudaFree(df); cudaFree(dt); cudaFree(dw); cudaFree(dm); cudaFree(dv); cudaFree(pg); cudaFree(dg); cudaFree(dl);
  };
  snmf_status st = SNMF_OK;
#define MCK(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) { st = e_ == cudaErrorMemoryAllocation ? SNMF_ERR_OOM : SNMF_ERR_CUDA; cleanup(); return st; } \
  } while (0)
  MCK(cudaMalloc(&df, (size_t)count * kMlpIn * sizeof(float)));
  MCK(cudaMalloc(&dt, (size_t)count * sizeof(float)));
  MCK(cudaMalloc(&dw, NP * sizeof(float)));
  MCK(cudaMalloc(&dm, NP * sizeof(float)));
  MCK(cudaMalloc(&dv, NP * sizeof(float)));
  MCK(cudaMalloc(&dg, NP * sizeof(float)));
  MCK(cudaMalloc(&dl, sizeof(float)));
  MCK(cudaMalloc(&pg, (size_t)nb * (NP + 1) * sizeof(float)));
  MCK(cudaMemcpy(df, feats, (size_t)count * kMlpIn * sizeof(float), cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(dt, targets, (size_t)count * sizeof(float), cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(dw, weights, NP * sizeof(float), cudaMemcpyHostToDevice));
  MCK(cudaMemset(dm, 0, NP * sizeof(float)));
  MCK(cudaMemset(dv, 0, NP * sizeof(float)));
  // gradient at the initial weights (for checking), then `steps` Adam steps
  k_mlp_grad<<<nb, 256>>>(df, dt, count, dw, pg);
  k_mlp_step<<<1, 512>>>(pg, nb, dw, dm, dv, dg, dl, 1, (float)lr, 0);
  if (grad0) MCK(cudaMemcpy(grad0, dg, NP * sizeof(float), cudaMemcpyDeviceToHost));
  for (int s = 1; s <= steps; ++s) {
    k_mlp_grad<<<nb, 256>>>(df, dt, count, dw, pg);
    k_mlp_step<<<1, 512>>>(pg, nb, dw, dm, dv, nullptr, dl, s, (float)lr, 1);
  }
  k_mlp_grad<<<nb, 256>>>(df, dt, count, dw, pg);
  k_mlp_step<<<1, 512>>>(pg, nb, dw, dm, dv, nullptr, dl, 1, (float)lr, 0);
  float lossf = 0.f;
  MCK(cudaMemcpy(&lossf, dl, sizeof(float), cudaMemcpyDeviceToHost));
  MCK(cudaMemcpy(weights, dw, NP * sizeof(float), cudaMemcpyDeviceToHost));
  MCK(cudaGetLastError());
  if (loss_out) *loss_out = lossf;
  cleanup();
  return SNMF_OK;
#undef MCK
}

extern "C" snmf_status snmf_mlp_eval(const float* weights, const float* feats, int count, float* mult) {
  if (!weights || !feats || !mult || count < 1) return SNMF_ERR_ARG;
  std::vector<__nv_bfloat16> wb(NP);
  for (int i = 0; i < NP; ++i) wb[i] = __float2bfloat16_rn(weights[i]);  // as snmf_create rounds them
  __nv_bfloat16* dw = nullptr;
  float *df = nullptr, *dm = nullptr;
  auto cleanup = [&] { cudaFree(dw); cudaFree(df); cudaFree(dm); };
  snmf_status st = SNMF_OK;
#define ECK(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) { st = e_ == cudaErrorMemoryAllocation ? SNMF_ERR_OOM : SNMF_ERR_CUDA; cleanup(); return st; } \
  } while (0)
  ECK(cudaMalloc(&dw, NP * sizeof(__nv_bfloat16)));
  ECK(cudaMalloc(&df, (size_t)count * kMlpIn * sizeof(float)));
  ECK(cudaMalloc(&dm, (size_t)count * sizeof(float)));
  ECK(cudaMemcpy(dw, wb.data(), NP * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
  ECK(cudaMemcpy(df, feats, (size_t)count * kMlpIn * sizeof(float), cudaMemcpyHostToDevice));
  k_mlp_eval<<<(count + 7) / 8, 256>>>(dw, df, count, dm);
  ECK(cudaGetLastError());
  ECK(cudaMemcpy(mult, dm, (size_t)count * sizeof(float), cudaMemcpyDeviceToHost));
#undef ECK
  cleanup();
  return st;
}
