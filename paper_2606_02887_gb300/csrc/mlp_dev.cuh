// Inference of the learned step controller's MLP on the device, shared by the solver's
// control step (rowops_dev.cuh) and the evaluation entry point snmf_mlp_eval (mlp.cu).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace snmf {

// o = W2 relu(W1 phi + b1) + b2 with BF16 weights (layout W1[64][5], b1[64], W2[64], b2) and
// FP32 accumulation, by one warp (lane l owns hidden units l and l + 32; the two partial
// sums of W2 h are combined by a fixed butterfly); returns the multiplier 2^(2 tanh o) in
// every lane.
__device__ __forceinline__ float mlp_multiplier(const __nv_bfloat16* w, const float* phi) {
  const int lane = threadIdx.x & 31;
  float part = 0.f;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int hdn = lane + 32 * u;
    float z = __bfloat162float(w[kMlpIn * kMlpHidden + hdn]);
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) z = fmaf(__bfloat162float(w[hdn * kMlpIn + i]), phi[i], z);
    z = fmaxf(z, 0.f);
    part = fmaf(__bfloat162float(w[kMlpIn * kMlpHidden + kMlpHidden + hdn]), z, part);
  }
  const float o = warp_sum(part) + __bfloat162float(w[kMlpParams - 1]);
  return exp2f(2.f * tanhf(o));
}

}  // namespace snmf
