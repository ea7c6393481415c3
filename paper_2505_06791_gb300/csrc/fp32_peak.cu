// FP32 FMA throughput of this GPU, measured: the denominator of the FP32-ALU rooflines of the
// validation and planning kernels (the nominal figure is SMs x 128 lanes x 2 FLOP x clock).
// Every thread runs 16 independent FMA chains a = a * b + c (b, c kernel arguments, so
// nothing folds; the chains converge to c / (1 - b) and stay normal), either as scalar FMAs
// or as packed FP32x2 FMAs, which issue two lanes' worth per instruction.
#include <cuda_runtime.h>

#include "launch.h"
#include "mlp_common.cuh"

namespace cprrtc {
namespace {

constexpr int kPeakChains = 16;

template <bool PACKED>
__global__ void fp32_peak_kernel(float* sink, int iters, float b, float c) {
  float s = 0.f;
  if (PACKED) {
    unsigned long long a[kPeakChains / 2];
#pragma unroll
    for (int k = 0; k < kPeakChains / 2; ++k)
      a[k] = f32x2_pack(1e-3f * (float)(threadIdx.x + 2 * k), 1e-3f * (float)(threadIdx.x + 2 * k + 1));
    const unsigned long long bb = f32x2_pack(b, b), cc = f32x2_pack(c, c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kPeakChains / 2; ++k) a[k] = f32x2_fma(a[k], bb, cc);
    }
#pragma unroll
    for (int k = 0; k < kPeakChains / 2; ++k)
      s += __uint_as_float((unsigned)a[k]) + __uint_as_float((unsigned)(a[k] >> 32));
  } else {
    float a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) a[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) a[k] = fmaf(a[k], b, c);
    }
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += a[k];
  }
  if (s == -1.f) sink[0] = s;  // never true; keeps the chains live
}

}  // namespace

cudaError_t measure_fp32_peak(const DeviceInfo& dev, cudaStream_t stream, double* tflops) {
  constexpr int kThreads = 256, kBlocksPerSm = 8, kIters = 8192, kReps = 3;
  const int grid = dev.sm_count * kBlocksPerSm;
  const double flop = 2.0 * kPeakChains * (double)kIters * kThreads * grid;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0.0;
  for (int packed = 0; packed < 2 && e == cudaSuccess; ++packed) {
    for (int rep = 0; rep <= kReps && e == cudaSuccess; ++rep) {  // rep 0 warms up
      e = cudaEventRecord(e0, stream);
      if (e == cudaSuccess) {
        if (packed)
          fp32_peak_kernel<true><<<grid, kThreads, 0, stream>>>(sink, kIters, 0.999f, 1e-3f);
        else
          fp32_peak_kernel<false><<<grid, kThreads, 0, stream>>>(sink, kIters, 0.999f, 1e-3f);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && rep > 0 && ms > 0.f) {
        const double t = flop / (ms * 1e-3) / 1e12;
        if (t > best) best = t;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e == cudaSuccess) *tflops = best;
  return e;
}

}  // namespace cprrtc
