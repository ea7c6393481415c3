// Batched constrained motion validation (Sec. III, Alg. 1, Sec. IV) and single-
// configuration projection kernels, with their host launchers.
#include "launch.h"
#include "motion.cuh"

namespace cprrtc {

// Robot spheres, their frames and each warp's frame cache live in shared memory; the
// obstacle stream is staged there too when it fits (coalesced float4 copies), else read
// from global memory through L1 (every lane reads the same obstacle: one broadcast).
template <int WPL>
__global__ void __launch_bounds__(kValidateWarps * 32)
    validate_kernel(RobotDev rb, SceneDev sc, ConsDev cs, ValidateArgs a) {
  extern __shared__ float4 smem[];
  const int n4 = sc.n_float4();
  float4* s_obs = smem;
  float4* s_sph = smem + (a.stage_obs ? n4 : 0);
  int* s_sfr = reinterpret_cast<int*>(s_sph + rb.n_spheres);
  float* s_fr = reinterpret_cast<float*>(s_sfr + ((rb.n_spheres + 3) & ~3));
  if (a.stage_obs)
    for (int i = threadIdx.x; i < n4; i += blockDim.x) s_obs[i] = sc.obs[i];
  for (int i = threadIdx.x; i < rb.n_spheres; i += blockDim.x) {
    s_sph[i] = rb.spheres[i];
    s_sfr[i] = rb.sphere_frame[i];
  }
  __syncthreads();
  const float4* obs = a.stage_obs ? s_obs : sc.obs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int dof = rb.dof, W = a.W;
  float* fr = s_fr + warp * W * frame_stride(dof);

  for (int m = blockIdx.x * kValidateWarps + warp; m < a.n; m += gridDim.x * kValidateWarps) {
    float q0[kMaxDof], q1[kMaxDof];
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) {
      if (k < dof) {
        q0[k] = a.q_start[(size_t)m * dof + k];
        q1[k] = a.q_end[(size_t)m * dof + k];
      }
    }
    float q[WPL][kMaxDof];
#pragma unroll
    for (int s = 0; s < WPL; ++s) interp(q0, q1, min(lane + 32 * s, W - 1), W, dof, q[s]);
    const float tau = step_threshold(cs, q0, q1, W, dof);
    const ProjResult pr = project_warp<WPL>(rb, cs, q, W, tau, fr);
    __syncwarp();
    int st = pr.status, ff = pr.first_fail;
    if (st == kValid) {
      ff = collide_warp(rb, sc, obs, s_sph, s_sfr, W, a.cc_skip_first, fr);
      if (ff >= 0) st = kCollision;
    }
    if (a.out_q) {
#pragma unroll
      for (int s = 0; s < WPL; ++s) {
        const int i = lane + 32 * s;
        if (i < W) {
          float* o = a.out_q + ((size_t)m * W + i) * dof;
#pragma unroll
          for (int k = 0; k < kMaxDof; ++k)
            if (k < dof) o[k] = q[s][k];
        }
      }
    }
    if (lane == 0) {
      a.status[m] = (uint8_t)st;
      if (a.first_fail) a.first_fail[m] = ff;
      if (a.iters) a.iters[m] = (uint8_t)pr.iters;
      if (a.resid) a.resid[m] = pr.resid;
    }
    __syncwarp();
  }
}

// One thread per configuration: damped steps until ||E_task||_inf < tol_task.
__global__ void project_configs_kernel(RobotDev rb, ConsDev cs, const float* __restrict__ q_in,
                                       int n, int max_iters, float* q_out, uint8_t* ok,
                                       float* resid) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  const int dof = rb.dof;
  float q[kMaxDof];
#pragma unroll
  for (int k = 0; k < kMaxDof; ++k) q[k] = k < dof ? q_in[(size_t)m * dof + k] : 0.f;
  TaskEval t;
  int success = 0;
  float err = 0.f;
  for (int it = 0; it <= max_iters; ++it) {
    chain<true>(rb, cs, q, nullptr, t);
    err = task_err_inf(t);
    if (err < cs.tol_task) {
      success = 1;
      break;
    }
    if (it == max_iters) break;
    float g[kMaxDof];
    damped_step(rb, cs, t, g);
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k)
      if (k < dof) q[k] = fminf(fmaxf(fmaf(-cs.alpha, g[k], q[k]), rb.j[k].lo), rb.j[k].hi);
  }
#pragma unroll
  for (int k = 0; k < kMaxDof; ++k)
    if (k < dof) q_out[(size_t)m * dof + k] = q[k];
  if (ok) ok[m] = (uint8_t)success;
  if (resid) resid[m] = err;
}

size_t validate_smem_bytes(const RobotDev& rb, const SceneDev& sc, int W, bool stage_obs) {
  size_t b = 0;
  if (stage_obs) b += (size_t)sc.n_float4() * sizeof(float4);
  b += (size_t)rb.n_spheres * sizeof(float4);
  b += (size_t)((rb.n_spheres + 3) & ~3) * sizeof(int);
  b += (size_t)kValidateWarps * W * frame_stride(rb.dof) * sizeof(float);
  return b;
}

cudaError_t launch_validate(const RobotDev& rb, const SceneDev& sc, const ConsDev& cs,
                            ValidateArgs a, const DeviceInfo& dev, cudaStream_t stream) {
  if (a.n <= 0) return cudaSuccess;
  size_t smem = validate_smem_bytes(rb, sc, a.W, true);
  a.stage_obs = smem <= dev.smem_optin ? 1 : 0;
  if (!a.stage_obs) smem = validate_smem_bytes(rb, sc, a.W, false);
  if (smem > dev.smem_optin) return cudaErrorInvalidConfiguration;
  const void* fn = a.W <= 32 ? (const void*)validate_kernel<1> : (const void*)validate_kernel<2>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kValidateWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long need = (a.n + kValidateWarps - 1) / kValidateWarps;
  const long long cap = (long long)per_sm * dev.sm_count;
  const int grid = (int)(need < cap ? need : cap);
  if (a.W <= 32)
    validate_kernel<1><<<grid, kValidateWarps * 32, smem, stream>>>(rb, sc, cs, a);
  else
    validate_kernel<2><<<grid, kValidateWarps * 32, smem, stream>>>(rb, sc, cs, a);
  return cudaGetLastError();
}

cudaError_t launch_project_configs(const RobotDev& rb, const ConsDev& cs, const float* q_in,
                                   int n, int max_iters, float* q_out, uint8_t* ok,
                                   float* resid, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int block = 128;
  project_configs_kernel<<<(n + block - 1) / block, block, 0, stream>>>(rb, cs, q_in, n, max_iters,
                                                                       q_out, ok, resid);
  return cudaGetLastError();
}

}  // namespace cprrtc
