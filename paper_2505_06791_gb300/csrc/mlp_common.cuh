// Pieces of the warm-start network shared by its training kernels and its fused inference
// kernel: the activation and the layer widths.
#pragma once
#include <cuda_runtime.h>

namespace cprrtc {

// gelu(z) = z Phi(z), Phi the standard normal CDF (exact form, through erf).
__device__ __forceinline__ float mlp_gelu(float z) {
  return 0.5f * z * (1.f + erff(z * 0.70710678118654752f));
}

// d gelu / dz = Phi(z) + z phi(z)
__device__ __forceinline__ float mlp_gelu_grad(float z) {
  const float cdf = 0.5f * (1.f + erff(z * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * __expf(-0.5f * z * z);
  return cdf + z * pdf;
}

constexpr float kMlpInvPi = 0.318309886183790671538f;  // inputs are q / pi

}  // namespace cprrtc
