// Batched constrained motion validation (Sec. III, Alg. 1, Sec. IV) and single-
// configuration projection kernels, with their host launchers.
#include "launch.h"
#include "motion.cuh"

namespace cprrtc {

// Robot tables and each warp's collision scratch live in shared memory; the obstacle
// stream is staged there too when it fits (coalesced float4 copies), else read from
// global memory through L1. The first colliding waypoint is exact (no early exit).
template <int CT, int WPL, bool SEQ>
__device__ __forceinline__ void validate_body(const RobotDev& rb, const SceneDev& sc, const ConsDev& cs,
                                              const ValidateArgs& a) {
  extern __shared__ __align__(16) char smem[];
  const int n4 = sc.n_float4();
  const SmemLayout L(a.stage_obs ? n4 : 0, rb.n_spheres, a.W, kValidateWarps, 0);
  float4* s_obs = reinterpret_cast<float4*>(smem + L.obs);
  if (a.stage_obs)
    for (int i = threadIdx.x; i < n4; i += blockDim.x) s_obs[i] = sc.obs[i];
  stage_robot(rb, smem, L);
  __syncthreads();
  const float4* obs = a.stage_obs ? s_obs : sc.obs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int dof = rb.dof, W = a.W;
  const CcShared S = cc_shared(smem, L, warp);
  WorkCount work{};

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
    const float tau = step_threshold(cs, q0, q1, W, dof);
    // pass 0 (warm start only): interpolation + learned correction, refine_iters
    // iterations. The correction of waypoint i is f(xi_i) - (1 - i/(W-1)) f(xi_0): waypoint 0
    // lies on the manifold, so f(xi_0) is the network's local error, removed where the
    // segment joins its fixed start; pass 1: Alg. 1 from the interpolation. The plain pass runs when the warm
    // one did not project the whole segment. The warm start is tried only when its largest
    // task residual over waypoints 1..W-1 is below the interpolation's.
    ProjResult pr;
    int spent = 0, warm_ok = 0, first_pass = 1;
    if (a.warm && !(a.warm_error && *a.warm_error)) {
      float e_warm = 0.f, e_plain = 0.f;
#pragma unroll
      for (int s = 0; s < WPL; ++s) {
        const int i = lane + 32 * s;
        if (i >= 1 && i < W) {
          float qp[kMaxDof], qw[kMaxDof];
          interp(q0, q1, i, W, dof, qp);
          const float* y = a.warm + ((size_t)m * W + i) * 16;
          const float* y0 = a.warm + (size_t)m * W * 16;
          const float taper = 1.f - (float)i / (float)(W - 1);
#pragma unroll
          for (int k = 0; k < kMaxDof; ++k)
            qw[k] = k < dof ? fminf(fmaxf(qp[k] + fmaf(-taper, y0[k], y[k]), rb.j[k].lo), rb.j[k].hi)
                            : 0.f;
          ChainState ch;
          TaskEval<CT> te;
          chain(rb, qp, nullptr, ch);
          te.eval(rb, cs, ch);
          e_plain = fmaxf(e_plain, te.err_inf());
          chain(rb, qw, nullptr, ch);
          te.eval(rb, cs, ch);
          e_warm = fmaxf(e_warm, te.err_inf());
          work.updates += 2u;
        }
      }
      first_pass = warp_max(e_warm) < warp_max(e_plain) ? 0 : 1;
    }
    for (int pass = first_pass; pass < 2; ++pass) {
#pragma unroll
      for (int s = 0; s < WPL; ++s) {
        const int i = min(lane + 32 * s, W - 1);
        interp(q0, q1, i, W, dof, q[s]);
        if (pass == 0 && i > 0) {
          const float* y = a.warm + ((size_t)m * W + i) * 16;
          const float* y0 = a.warm + (size_t)m * W * 16;
          const float taper = 1.f - (float)i / (float)(W - 1);
#pragma unroll
          for (int k = 0; k < kMaxDof; ++k)
            if (k < dof)
              q[s][k] = fminf(fmaxf(q[s][k] + fmaf(-taper, y0[k], y[k]), rb.j[k].lo), rb.j[k].hi);
        }
      }
      if constexpr (SEQ)
        pr = project_sequential<CT, WPL>(rb, cs, cs.max_iters, q0, q1, q, W, tau);
      else
        pr = project_warp<CT, WPL>(rb, cs, pass == 0 ? a.refine_iters : cs.max_iters, q, W, tau, S.wq);
      work.updates += (unsigned)pr.updates;
      if (pass == 0 && pr.status == kValid) {
        warm_ok = 1;
        break;
      }
      if (pass == 0) spent = pr.iters;
    }
    pr.iters += spent;
    int st = pr.status, ff = pr.first_fail;
    if (st == kValid && !a.skip_cc) {
      ff = collide_motion<WPL>(rb, sc, obs, S, q, W, a.cc_skip_first, false, work, !a.no_early_exit,
                               !SEQ && CT != kConsNone);
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
      if (a.iters) a.iters[m] = (uint8_t)min(pr.iters, 255);
      if (a.resid) a.resid[m] = pr.resid;
      if (a.warm_used) a.warm_used[m] = (uint8_t)warm_ok;
    }
    __syncwarp();
  }
  work.flush(a.work_counters);
}

// Most instantiations get the compiler's register choice (a cap of 128 spills them). The
// roll-pitch kernel with one waypoint per lane (the batched validation of configuration 1)
// fits 128 registers without spilling, so it is held to four 4-warp CTAs per SM instead of
// the three its 150 registers allow: more warps to hide its dependent-instruction latency.
template <int CT, int WPL, bool SEQ = false>
__global__ void validate_kernel(RobotDev rb, SceneDev sc, ConsDev cs, ValidateArgs a) {
  validate_body<CT, WPL, SEQ>(rb, sc, cs, a);
}

template <int CT>
__global__ void __launch_bounds__(kValidateWarps * 32, 4) validate_kernel_4(RobotDev rb, SceneDev sc,
                                                                             ConsDev cs, ValidateArgs a) {
  validate_body<CT, 1, false>(rb, sc, cs, a);
}

// One thread per configuration: damped steps until ||E_task||_inf < tol_task.
template <int CT>
__global__ void project_configs_kernel(RobotDev rb, ConsDev cs, const float* __restrict__ q_in,
                                       int n, int max_iters, float* q_out, uint8_t* ok,
                                       float* resid) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  const int dof = rb.dof;
  float q[kMaxDof];
#pragma unroll
  for (int k = 0; k < kMaxDof; ++k) q[k] = k < dof ? q_in[(size_t)m * dof + k] : 0.f;
  ChainState s;
  int success = 0;
  float err = 0.f;
  for (int it = 0; it <= max_iters; ++it) {
    chain(rb, q, nullptr, s);
    TaskEval<CT> te;
    te.eval(rb, cs, s);
    err = te.err_inf();
    if (err < cs.tol_task) {
      success = 1;
      break;
    }
    if (it == max_iters) break;
    te.solve(rb, cs, s);
    float g[kMaxDof];  // every step from the same configuration before any joint moves
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) g[k] = k < dof ? te.step(rb, s, k) : 0.f;
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

static const void* validate_fn(int ct, int W, bool sequential) {
  const bool two = W > 32;
  if (sequential) {  // the naive baseline's projection: roll-pitch and z-plane
    if (ct == kConsRollPitch)
      return two ? (const void*)validate_kernel<kConsRollPitch, 2, true>
                 : (const void*)validate_kernel<kConsRollPitch, 1, true>;
    if (ct == kConsZPlane)
      return two ? (const void*)validate_kernel<kConsZPlane, 2, true>
                 : (const void*)validate_kernel<kConsZPlane, 1, true>;
    return nullptr;
  }
  switch (ct) {
    case kConsRollPitch:
      return two ? (const void*)validate_kernel<kConsRollPitch, 2> : (const void*)validate_kernel_4<kConsRollPitch>;
    case kConsZPlane:
      return two ? (const void*)validate_kernel<kConsZPlane, 2> : (const void*)validate_kernel<kConsZPlane, 1>;
    case kConsLine:
      return two ? (const void*)validate_kernel<kConsLine, 2> : (const void*)validate_kernel<kConsLine, 1>;
    case kConsOrientPlane:
      return two ? (const void*)validate_kernel<kConsOrientPlane, 2>
                 : (const void*)validate_kernel<kConsOrientPlane, 1>;
    case kConsOrientLine:
      return two ? (const void*)validate_kernel<kConsOrientLine, 2>
                 : (const void*)validate_kernel<kConsOrientLine, 1>;
    default:
      return two ? (const void*)validate_kernel<kConsNone, 2> : (const void*)validate_kernel<kConsNone, 1>;
  }
}

size_t validate_smem_bytes(const RobotDev& rb, const SceneDev& sc, int W, bool stage_obs) {
  return SmemLayout(stage_obs ? sc.n_float4() : 0, rb.n_spheres, W, kValidateWarps, 0).total;
}

cudaError_t launch_validate(const RobotDev& rb, const SceneDev& sc, const ConsDev& cs,
                            ValidateArgs a, const DeviceInfo& dev, cudaStream_t stream) {
  if (a.n <= 0) return cudaSuccess;
  size_t smem = validate_smem_bytes(rb, sc, a.W, true);
  a.stage_obs = smem <= dev.smem_optin ? 1 : 0;
  if (!a.stage_obs) smem = validate_smem_bytes(rb, sc, a.W, false);
  if (smem > dev.smem_optin) return cudaErrorInvalidConfiguration;
  const void* fn = validate_fn(cs.type, a.W, a.sequential != 0 && cs.type != kConsNone);
  if (!fn) return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kValidateWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long need = (a.n + kValidateWarps - 1) / kValidateWarps;
  const long long cap = (long long)per_sm * dev.sm_count;
  const int grid = (int)(need < cap ? need : cap);
  void* args[] = {const_cast<RobotDev*>(&rb), const_cast<SceneDev*>(&sc),
                  const_cast<ConsDev*>(&cs), &a};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(kValidateWarps * 32), args, smem, stream);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_project_configs(const RobotDev& rb, const ConsDev& cs, const float* q_in,
                                   int n, int max_iters, float* q_out, uint8_t* ok,
                                   float* resid, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int block = 128;
  const int grid = (n + block - 1) / block;
  switch (cs.type) {
    case kConsZPlane:
      project_configs_kernel<kConsZPlane><<<grid, block, 0, stream>>>(rb, cs, q_in, n, max_iters, q_out, ok, resid);
      break;
    case kConsLine:
      project_configs_kernel<kConsLine><<<grid, block, 0, stream>>>(rb, cs, q_in, n, max_iters, q_out, ok, resid);
      break;
    case kConsOrientPlane:
      project_configs_kernel<kConsOrientPlane><<<grid, block, 0, stream>>>(rb, cs, q_in, n, max_iters, q_out, ok,
                                                                         resid);
      break;
    case kConsOrientLine:
      project_configs_kernel<kConsOrientLine><<<grid, block, 0, stream>>>(rb, cs, q_in, n, max_iters, q_out, ok,
                                                                        resid);
      break;
    default:
      project_configs_kernel<kConsRollPitch><<<grid, block, 0, stream>>>(rb, cs, q_in, n, max_iters, q_out, ok,
                                                                       resid);
  }
  return cudaGetLastError();
}

}  // namespace cprrtc
