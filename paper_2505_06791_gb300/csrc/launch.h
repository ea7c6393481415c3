// Host-side launcher declarations shared between the C-ABI layer and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "device_types.cuh"

namespace cprrtc {

constexpr int kValidateWarps = 4;  // warps (motions in flight) per CTA
constexpr int kWorkCounters = 6;   // updates, chains, transforms, sphere / box / capsule tests

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
  unsigned long long* work_counters;  // [6] executed-work totals (may be null)
  int stage_obs;  // set by the launcher
};

constexpr int kMaxWorkers = 16;  // warps per planning problem

struct PlanArgs {
  const float* start;
  const float* goal;
  int n;
  float range;
  int W, max_rounds, workers, max_nodes, max_connect, max_path;
  uint32_t seed;
  const float4* scene_obs;  // scene batch: obstacle stream
  const int4* scenes;       // [n] {float4 offset, n_sph, n_box, n_cap}; null: shared scene
  int max_scene_f4;         // largest scene, float4 slots
  float* nodes;             // [n][2][max_nodes][8]
  int* parent;              // [n][2][max_nodes]
  float* edges;             // [n][2][max_nodes][W][dof]
  float* pend;              // [n][workers][8] node a warp produced this round
  float* pend_edges;        // [n][workers][2][W][dof] its motion, and the closing hop
  int32_t* path_len;
  float* path;
  float* path_edges;
  int32_t* rounds;
  long long* waypoints;
  float* plan_ms;
  long long* work;          // [n][2] Alg. 1 waypoint updates, collision-checked waypoints
  unsigned long long* work_counters;  // [6] executed-work totals (may be null)
  int stage_obs;            // set by the launcher
};

// Persistent batch of uneven planning problems (one launch).
// Robot and constraint tables of a batch, passed by value (kernel parameter space).
constexpr int kBatchMaxRobots = 8;
constexpr int kBatchMaxCons = 8;
struct BatchTables {
  RobotDev robots[kBatchMaxRobots];
  ConsDev cons[kBatchMaxCons];
};

struct BatchArgs {
  PlanArgs a;                // shared parameters, scene batch, outputs ([n][8] configurations)
  const int4* problems;      // [n] {robot, constraint, scene, W}
  const int* order;          // [n_class] this class's problems in dequeue order
  int n_class;
  unsigned* counter;         // this class's dequeue counter (zeroed by the launcher)
  int max_S, max_W;          // largest robot sphere count and W of this class
  int out_max_W;             // largest W of the whole batch (path_edges row stride)
  float* nodes;              // per CTA slot: [2][max_nodes][8]
  int* parent;               // per CTA slot: [2][max_nodes]
  float* edges;              // per CTA slot: [2][max_nodes][max_W * 8]
  float* pend;               // per CTA slot: [workers][8]
  float* pend_edges;         // per CTA slot: [workers][2][max_W * 8]
};

// Problem classes: 2 * constraint type + (W > 32).
constexpr int kBatchClasses = 6;
size_t plan_batch_smem_bytes(int max_scene_f4, int max_S, int max_W, int workers, bool stage);
int plan_batch_occupancy(int cls, int workers, size_t smem);
cudaError_t launch_plan_batch(int cls, BatchArgs b, const BatchTables& T, int grid, size_t smem,
                              cudaStream_t stream);

size_t plan_smem_bytes(const RobotDev& rb, int max_scene_f4, int W, int workers, bool stage);
cudaError_t launch_plan(const RobotDev& rb, const SceneDev& sc, const ConsDev& cs, PlanArgs a,
                        const DeviceInfo& dev, cudaStream_t stream);
cudaError_t launch_philox(uint32_t k0, uint32_t k1, const uint32_t* ctr, int n, uint32_t* out,
                          cudaStream_t stream);

size_t validate_smem_bytes(const RobotDev& rb, const SceneDev& sc, int W, bool stage_obs);
cudaError_t launch_validate(const RobotDev& rb, const SceneDev& sc, const ConsDev& cs,
                            ValidateArgs a, const DeviceInfo& dev, cudaStream_t stream);
cudaError_t launch_project_configs(const RobotDev& rb, const ConsDev& cs, const float* q_in,
                                   int n, int max_iters, float* q_out, uint8_t* ok,
                                   float* resid, cudaStream_t stream);

}  // namespace cprrtc
