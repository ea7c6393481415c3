// Sphere-vs-primitive collision predicates in FP32 (Sec. IV). Each returns true when the
// robot sphere (centre c, radius r) penetrates the obstacle; touching counts as free.
#pragma once
#include "device_types.cuh"

namespace cprrtc {

// Obstacle sphere o = {x, y, z, rho}: |c - o|^2 < (r + rho)^2.
__device__ __forceinline__ bool hit_sphere(float cx, float cy, float cz, float r, float4 o) {
  const float dx = cx - o.x, dy = cy - o.y, dz = cz - o.z;
  const float rr = r + o.w;
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rr * rr;
}

// Oriented box b0 = {c, hx}, b1 = {col0, hy}, b2 = {col1, hz}, b3 = {col2, -}: the point in
// box coordinates is l_k = col_k . (c - centre); squared distance to the solid box is
// sum_k max(|l_k| - h_k, 0)^2 (0 inside), compared with r^2.
__device__ __forceinline__ bool hit_box(float cx, float cy, float cz, float r, float4 b0,
                                        float4 b1, float4 b2, float4 b3) {
  const float dx = cx - b0.x, dy = cy - b0.y, dz = cz - b0.z;
  const float l0 = fmaf(b1.x, dx, fmaf(b1.y, dy, b1.z * dz));
  const float l1 = fmaf(b2.x, dx, fmaf(b2.y, dy, b2.z * dz));
  const float l2 = fmaf(b3.x, dx, fmaf(b3.y, dy, b3.z * dz));
  const float e0 = fmaxf(fabsf(l0) - b0.w, 0.f);
  const float e1 = fmaxf(fabsf(l1) - b1.w, 0.f);
  const float e2 = fmaxf(fabsf(l2) - b2.w, 0.f);
  return fmaf(e0, e0, fmaf(e1, e1, e2 * e2)) < r * r;
}

// Capsule k0 = {p0, rc}, k1 = {u = p1 - p0, 1/|u|^2}: closest point p0 + t u with
// t = clamp((c - p0).u / |u|^2, 0, 1); compared with (r + rc)^2.
__device__ __forceinline__ bool hit_capsule(float cx, float cy, float cz, float r, float4 k0,
                                            float4 k1) {
  const float wx = cx - k0.x, wy = cy - k0.y, wz = cz - k0.z;
  float t = fmaf(wx, k1.x, fmaf(wy, k1.y, wz * k1.z)) * k1.w;
  t = fminf(fmaxf(t, 0.f), 1.f);
  const float dx = fmaf(-t, k1.x, wx), dy = fmaf(-t, k1.y, wy), dz = fmaf(-t, k1.z, wz);
  const float rr = r + k0.w;
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rr * rr;
}

}  // namespace cprrtc
