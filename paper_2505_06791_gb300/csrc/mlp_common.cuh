// Pieces of the warm-start network shared by its training kernels and its fused inference
// kernel: the activation and the input scaling.
#pragma once
#include <cuda_runtime.h>

namespace cprrtc {

// Abramowitz and Stegun, Handbook of Mathematical Functions, formula 7.1.28:
//   erf(x) = 1 - (1 + a1 x + a2 x^2 + ... + a6 x^6)^-16 + e(x),  |e(x)| <= 3e-7, x >= 0.
// With x = |z| / sqrt 2 folded into the coefficients (b_k = a_k 2^(-k/2)), the normal tail is
// 1 - Phi(|z|) = (1 - erf(x)) / 2 = 0.5 / P with P = (1 + b1 |z| + ... + b6 |z|^6)^16
// (P = inf, tail 0, for large |z|).
constexpr float kPhiB1 = 4.9867346967e-02f, kPhiB2 = 2.1141006150e-02f, kPhiB3 = 3.2776263241e-03f,
                kPhiB4 = 3.8003575000e-05f, kPhiB5 = 4.8890635643e-05f, kPhiB6 = 5.3829750000e-06f;

__device__ __forceinline__ float mlp_tail_denominator(float z) {
  const float x = fabsf(z);
  float p = fmaf(x, kPhiB6, kPhiB5);
  p = fmaf(x, p, kPhiB4);
  p = fmaf(x, p, kPhiB3);
  p = fmaf(x, p, kPhiB2);
  p = fmaf(x, p, kPhiB1);
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

// Two GELUs at once: the polynomial and its powers in packed FP32x2 arithmetic (one
// instruction per pair, the same roundings as mlp_gelu), the division per element.
__device__ __forceinline__ unsigned long long f32x2_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ unsigned long long f32x2_fma(unsigned long long a, unsigned long long b,
                                                        unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long f32x2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ void mlp_gelu2(float z0, float z1, float& g0, float& g1) {
  const float x0 = fabsf(z0), x1 = fabsf(z1);
  const unsigned long long x = f32x2_pack(x0, x1);
  unsigned long long p = f32x2_fma(x, f32x2_pack(kPhiB6, kPhiB6), f32x2_pack(kPhiB5, kPhiB5));
  p = f32x2_fma(x, p, f32x2_pack(kPhiB4, kPhiB4));
  p = f32x2_fma(x, p, f32x2_pack(kPhiB3, kPhiB3));
  p = f32x2_fma(x, p, f32x2_pack(kPhiB2, kPhiB2));
  p = f32x2_fma(x, p, f32x2_pack(kPhiB1, kPhiB1));
  p = f32x2_fma(x, p, f32x2_pack(1.0f, 1.0f));
  p = f32x2_mul(p, p);
  p = f32x2_mul(p, p);
  p = f32x2_mul(p, p);
  p = f32x2_mul(p, p);
  float p0, p1;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(p0), "=f"(p1) : "l"(p));
  g0 = fmaxf(z0, 0.f) - __fdividef(0.5f * x0, p0);
  g1 = fmaxf(z1, 0.f) - __fdividef(0.5f * x1, p1);
}

// d gelu / dz = Phi(z) + z phi(z)
__device__ __forceinline__ float mlp_gelu_grad(float z) {
  return fmaf(z * 0.39894228040143268f, __expf(-0.5f * z * z), mlp_phi(z));
}

constexpr float kMlpInvPi = 0.318309886183790671538f;  // inputs are q / pi

}  // namespace cprrtc
