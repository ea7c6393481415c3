// One configuration through the warm-start network by one warp, for the planner's learned
// form: the correction f(q) of the end of an extend motion. The weights stay in global memory
// (L2-resident, BF16) in the transposed layout, so the 32 lanes read one input's 256 outputs
// as 32 consecutive 16-byte pieces; lane l owns outputs 8l..8l+7 of the hidden layers, and the
// activations pass between layers through 256 floats of the warp's shared scratch. Products
// accumulate in FP32; GELU is the training kernels' (mlp_common.cuh).
#pragma once
#include <cuda_bf16.h>

#include "launch.h"
#include "mlp_common.cuh"

namespace cprrtc {

__device__ __forceinline__ void bf16x8_to_float(const uint4 v, float (&f)[8]) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 t = __bfloat1622float2(h[i]);
    f[2 * i] = t.x;
    f[2 * i + 1] = t.y;
  }
}

// out[0..dof) = f(q) (shared memory, written by lanes < dof); q: dof floats (shared memory,
// identical for every lane); act: 256 floats of the warp's shared scratch.
__device__ __forceinline__ void net_correction_warp(const MlpView& net, const float* q, int dof,
                                                    float* act, float* out) {
  const int lane = threadIdx.x & 31;
  const int j0 = 8 * lane;  // this lane's hidden outputs
  float h[8];
  // layer 0: x = q / pi, inputs k < dof of the padded 16
  {
    const float* b = net.b[0] + j0;
#pragma unroll
    for (int m = 0; m < 8; ++m) h[m] = b[m];
    const uint4* w = reinterpret_cast<const uint4*>(net.wt[0]);  // [16][256]
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) {
      if (k < dof) {
        const float x = q[k] * kMlpInvPi;
        float wk[8];
        bf16x8_to_float(w[k * 32 + lane], wk);
#pragma unroll
        for (int m = 0; m < 8; ++m) h[m] = fmaf(wk[m], x, h[m]);
      }
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) h[m] = mlp_gelu(h[m]);
  }
  // layers 1 and 2: 256 -> 256
#pragma unroll 1
  for (int l = 1; l <= 2; ++l) {
    __syncwarp();
    *reinterpret_cast<float4*>(act + j0) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(act + j0 + 4) = make_float4(h[4], h[5], h[6], h[7]);
    __syncwarp();
    const float* b = net.b[l] + j0;
#pragma unroll
    for (int m = 0; m < 8; ++m) h[m] = b[m];
    const uint4* w = reinterpret_cast<const uint4*>(net.wt[l]);  // [256][256]
#pragma unroll 4
    for (int k = 0; k < 256; ++k) {
      const float x = act[k];
      float wk[8];
      bf16x8_to_float(w[k * 32 + lane], wk);
#pragma unroll
      for (int m = 0; m < 8; ++m) h[m] = fmaf(wk[m], x, h[m]);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) h[m] = mlp_gelu(h[m]);
  }
  // layer 3: 256 -> dof; lane l sums its 8 inputs for every output, then the warp adds up
  const uint4* w3 = reinterpret_cast<const uint4*>(net.w3);  // [16][256]
  float y = 0.f;
#pragma unroll
  for (int o = 0; o < kMaxDof; ++o) {
    float s = 0.f;
    if (o < dof) {
      float wk[8];
      bf16x8_to_float(w3[o * 32 + lane], wk);
#pragma unroll
      for (int m = 0; m < 8; ++m) s = fmaf(wk[m], h[m], s);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(kFull, s, d);
    if (lane == o) y = s;
  }
  __syncwarp();
  if (lane < dof) out[lane] = y + net.b[3][lane];
  __syncwarp();
}

}  // namespace cprrtc
