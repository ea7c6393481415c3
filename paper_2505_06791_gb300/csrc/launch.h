// Host-side launcher declarations shared between the C-ABI layer and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "device_types.cuh"

namespace cprrtc {

constexpr int kValidateWarps = 4;  // warps (motions in flight) per CTA

struct DeviceInfo {
  int sm_count;
  size_t smem_optin;  // max dynamic shared memory per block
};

struct ValidateArgs {
  const float* q_start;
  const float* q_end;
  int n;
  int W;
  int cc_skip_first;
  float* out_q;
  uint8_t* status;
  int32_t* first_fail;
  uint8_t* iters;
  float* resid;
  int stage_obs;  // set by the launcher
};

size_t validate_smem_bytes(const RobotDev& rb, const SceneDev& sc, int W, bool stage_obs);
cudaError_t launch_validate(const RobotDev& rb, const SceneDev& sc, const ConsDev& cs,
                            ValidateArgs a, const DeviceInfo& dev, cudaStream_t stream);
cudaError_t launch_project_configs(const RobotDev& rb, const ConsDev& cs, const float* q_in,
                                   int n, int max_iters, float* q_out, uint8_t* ok,
                                   float* resid, cudaStream_t stream);

}  // namespace cprrtc
