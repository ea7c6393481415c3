// Pieces of the warm-start network shared by its training kernels and its fused inference
// kernel: the activation and the input scaling.
#pragma once
#include <cuda_runtime.h>

namespace cprrtc {

// Abramowitz and Stegun, Handbook of Mathematical Functions, formula 7.1.28:
//   erf(x) = 1 - (1 + a1 x + a2 x^2 + ... + a6 x^6)^-16 + e(x),  |e(x)| <= 3e-7, x >= 0.
// Returns P = (1 + a1 x + ... + a6 x^6)^16 for x = |z| / sqrt 2, so that the normal tail is
// 1 - Phi(|z|) = (1 - erf(x)) / 2 = 0.5 / P (P = inf, tail 0, for large |z|).
__device__ __forceinline__ float mlp_tail_denominator(float z) {
  const float x = fabsf(z) * 0.70710678118654752f;
  float p = fmaf(x, 0.0000430638f, 0.0002765672f);
  p = fmaf(x, p, 0.0001520143f);
  p = fmaf(x, p, 0.0092705272f);
  p = fmaf(x, p, 0.0422820123f);
  p = fmaf(x, p, 0.0705230784f);
  p = fmaf(x, p, 1.0f);
  p = p * p;  // ^2
  p = p * p;  // ^4
  p = p * p;  // ^8
  return p * p;  // ^16
}

// Standard normal CDF Phi(z) = (1 + erf(z / sqrt 2)) / 2 (erf(-x) = -erf(x)). The error
// of the formula is far below the BF16 rounding of the activations it feeds.
__device__ __forceinline__ float mlp_phi(float z) {
  const float tail = __fdividef(0.5f, mlp_tail_denominator(z));
  return z >= 0.f ? 1.f - tail : tail;
}

// gelu(z) = z Phi(z) = max(z, 0) - |z| (1 - Phi(|z|))
__device__ __forceinline__ float mlp_gelu(float z) {
  return fmaxf(z, 0.f) - __fdividef(0.5f * fabsf(z), mlp_tail_denominator(z));
}

// d gelu / dz = Phi(z) + z phi(z)
__device__ __forceinline__ float mlp_gelu_grad(float z) {
  return fmaf(z * 0.39894228040143268f, __expf(-0.5f * z * z), mlp_phi(z));
}

constexpr float kMlpInvPi = 0.318309886183790671538f;  // inputs are q / pi

}  // namespace cprrtc
