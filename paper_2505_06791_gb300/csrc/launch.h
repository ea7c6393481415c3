// Host-side launcher declarations shared between the C-ABI layer and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "device_types.cuh"

namespace cprrtc {

// Frame pairs whose spheres are tested against each other (self-collision): bit b of rows[a]
// for a < b; `on` = 0 when none.
struct SelfMask {
  unsigned short rows[kMaxDof + 1];
  int on;
};

constexpr int kValidateWarps = 4;  // warps (motions in flight) per CTA
// updates, chains, transforms, sphere / box / capsule tests, warm-started motions tried and
// accepted (the planner's learned form)
constexpr int kWorkCounters = 8;

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
  // learned warm start: corrections [n*W][16] (row m*W+i, dof used) added to waypoints
  // i >= 1 before refine_iters Alg. 1 iterations; plain Alg. 1 from the interpolation when
  // that does not project. Null: plain Alg. 1 only.
  const float* warm;
  int refine_iters;
  uint8_t* warm_used;  // [n] 1 when the warm-started segment was accepted (may be null)
  const int* warm_error;  // nonzero: the corrections are not valid; plain Alg. 1 only
  int skip_cc;            // 1: projection only (collision checking is done elsewhere)
  int no_early_exit;      // 1: collision checking evaluates every waypoint and candidate
  int sequential;         // 1: the naive baseline's sequential projection instead of Alg. 1
  int stage_obs;  // set by the launcher
};

constexpr int kMaxWorkers = 16;  // warps per planning problem

// The warm-start network as the planner's kernels read it: BF16 transposes [in][out] of
// layers 0..2 (input widths 16, 256, 256; outputs 256), layer 3 as [16][256], FP32 biases.
struct MlpView {
  const void* wt[3];
  const void* w3;
  const float* b[4];
  int dof;
};

struct PlanArgs {
  const float* start;
  const float* goal;
  int n;
  float range;
  int W, max_rounds, workers, max_nodes, max_connect, max_path;
  uint32_t seed;
  unsigned long long budget_ns;  // per-problem device-time budget (0: none)
  int sequential;                // 1: the naive baseline's sequential projection
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
  long long* span;          // [n][2] global-timer ns at each problem's start and end (may be null)
  long long* work;          // [n][2] Alg. 1 waypoint updates, collision-checked waypoints
  unsigned long long* work_counters;  // executed-work totals (may be null)
  int stage_obs;            // set by the launcher
  // learned warm start of extend motions (warm_refine > 0): the network and the Alg. 1
  // iterations the corrected segment gets before plain Alg. 1 takes over
  MlpView net;
  int warm_refine;
  // self-collision of the robot: bit b of self_rows[a] (a < b) pairs frames a and b
  unsigned short self_rows[kMaxDof + 1];
  int self_on;
  // Time-sliced schedule (queue set): persistent CTAs take problems from the queue; a
  // problem runs first_slice rounds, then slice rounds at a time, going back to the queue's
  // tail between slices while other problems wait. Null queue: one CTA per problem.
  struct PlanQueue* queue;
  struct PlanState* state;  // [n] each problem between slices
  int first_slice, slice;
  int* status;                 // set to 1 when a wait of the queue timed out (may be null)
  unsigned long long wait_ns;  // limit of the queue's bounded wait (0: 1 s)
};

// A problem between two slices: its next round, tree sizes, each worker's chain and the work
// counted so far.
struct PlanState {
  int r_next;
  int cnt[2];
  int pad;
  long long t_first;    // global timer at the start of its first slice
  long long active_ns;  // device time of its slices so far
  int mode[kMaxWorkers], ta[kMaxWorkers], last[kMaxWorkers], target[kMaxWorkers],
      steps[kMaxWorkers];
  unsigned wp[kMaxWorkers], proj[kMaxWorkers], cc[kMaxWorkers];
  float cur[kMaxWorkers][8], qt[kMaxWorkers][8];
};

// Queue of the time-sliced schedule (a bounded ring of n slots). Ticket t < n is problem t's
// first slice; ticket t >= n takes the problem pushed as number u = t - n, in slot s = u % n
// of lap L = u / n: its pusher waits for seq[s] = 2 L (the slot's previous occupant taken),
// stores ring[s] and sets 2 L + 1; the taker waits for 2 L + 1, reads ring[s] and sets
// 2 L + 2. Both waits are short (a ticket is taken only while a problem waits for it, so the
// other side is a running CTA a few instructions away) and bounded. The whole queue (header,
// seq [n] 64-bit, ring [n] int) is zeroed before each launch; head and tail are 64-bit, as a
// launch may hand problems over more than 2^32 times.
struct PlanQueue {
  unsigned long long head, tail;
  // device time and rounds of every slice that ended with rounds left: the launch's mean
  // round time, against which a problem's own decides whether it goes back to the queue
  unsigned long long sum_ns, sum_rounds;
};
inline size_t plan_queue_bytes(int n) {
  return sizeof(PlanQueue) + (sizeof(long long) + sizeof(int)) * (size_t)n;
}

// Persistent batch of uneven planning problems (one launch).
// Robot and constraint tables of a batch, passed by value (kernel parameter space).
constexpr int kBatchMaxRobots = 8;
constexpr int kBatchMaxCons = 8;
struct BatchTables {
  RobotDev robots[kBatchMaxRobots];
  ConsDev cons[kBatchMaxCons];
  SelfMask self[kBatchMaxRobots];  // each robot's self-collision frame pairs
  // the learned form's network of each (robot, constraint) pair (dof 0: none)
  MlpView nets[kBatchMaxRobots][kBatchMaxCons];
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

// Problem classes: 2 * constraint type + (W > 32). K = warps per worker: 1, or 2 in the
// plain form (a warp pair per motion, split by waypoints in the classes of 33..64 waypoints,
// by obstacles in the others).
constexpr int kBatchClasses = 6;
size_t plan_batch_smem_bytes(int max_scene_f4, int max_S, int max_W, int workers, bool stage, int K = 1);
int plan_batch_occupancy(int cls, int workers, size_t smem, bool warm = false, int K = 1);
cudaError_t launch_plan_batch(int cls, BatchArgs b, const BatchTables& T, int grid, size_t smem,
                              int K, cudaStream_t stream);

size_t plan_smem_bytes(const RobotDev& rb, int max_scene_f4, int W, int workers, bool stage);
// Most workers (warps per CTA) the planner kernel for this constraint type and W can launch
// with (its registers per thread bound the CTA size); 0 if the query fails.
int plan_max_workers(int cons_type, int W, bool sequential = false, bool warm = false);
cudaError_t launch_plan(const RobotDev& rb, const SceneDev& sc, const ConsDev& cs, PlanArgs a,
                        const DeviceInfo& dev, cudaStream_t stream);
cudaError_t launch_philox(uint32_t k0, uint32_t k1, const uint32_t* ctr, int n, uint32_t* out,
                          cudaStream_t stream);
// Self-collision after validation (self_collide.cu): motions that are valid or collide
// later get the first waypoint where spheres of two paired frames overlap.
struct SelfArgs {
  const float* q;        // [n][W][dof] the returned waypoints
  int n, W, i0;          // waypoints i0..W-1 are checked
  uint8_t* status;       // [n] updated in place
  int* first_fail;       // [n] updated in place
  unsigned short rows[kMaxDof + 1];  // bit b of rows[a] (a < b): test frames a and b
};
size_t self_collide_smem_bytes();
cudaError_t launch_self_collide(const RobotDev& rb, const SelfArgs& a, cudaStream_t stream);

// FP32 FMA throughput (TFLOP/s) measured with FMA chains on every SM (fp32_peak.cu).
cudaError_t measure_fp32_peak(const DeviceInfo& dev, cudaStream_t stream, double* tflops);

// ---- learned warm start (mlp.cu) ----
constexpr int kMlpLayers = 4;
constexpr int kMlpHidden = 256;
constexpr int kMlpIO = 16;  // input / output width (dof used, zero padding)
struct MlpDev;
size_t mlp_param_count();
size_t mlp_compact_count(int dof);
cudaError_t mlp_create(MlpDev** out, int dof);
void mlp_destroy(MlpDev* d);
int mlp_dof(const MlpDev* d);
void mlp_set_fp32(MlpDev* d, bool on);  // FP32 checking mode (no BF16 rounding)
MlpView mlp_view(MlpDev* d);             // the BF16 network for the planner's kernels
void mlp_set_wait_ns(MlpDev* d, unsigned long long ns);  // bounded-wait limit of inference
bool mlp_fp32(const MlpDev* d);
int mlp_step(const MlpDev* d);
cudaError_t mlp_set_params(MlpDev* d, const float* host, cudaStream_t s);
cudaError_t mlp_get_params(MlpDev* d, float* host, cudaStream_t s);
// full optimiser state in the compact layout (checkpoints)
cudaError_t mlp_get_state(MlpDev* d, float* params, float* m, float* v, int* step, cudaStream_t s);
cudaError_t mlp_set_state(MlpDev* d, const float* params, const float* m, const float* v, int step,
                          cudaStream_t s);
cudaError_t mlp_init(MlpDev* d, uint64_t seed, cudaStream_t s);
cudaError_t mlp_infer(MlpDev* d, const float* q, int ldq, int rows, float* Y, cudaStream_t s);
cudaError_t mlp_infer_motions(MlpDev* d, const float* q0, const float* q1, int n, int W, float* Y,
                              cudaStream_t s);
cudaError_t mlp_grad(MlpDev* d, const float* q, const float* t, int rows, float* grads_host,
                     float* loss_host, cudaStream_t s);
cudaError_t mlp_train_step(MlpDev* d, const float* q, const float* t, int rows, float lr,
                           float* loss_dev, cudaStream_t s);
cudaError_t mlp_train(MlpDev* d, const float* q, const float* t, int n, int batch, int epochs,
                      float lr, uint64_t seed, float* loss_host, cudaStream_t s);
// Collision checking in GEMM form (gemm_cc.cu): motions with status kValid get their
// waypoints (q, [n][W][dof]) checked against the sphere obstacles; colliding motions get
// status kCollision and their first colliding waypoint.
struct GemmCcArgs {
  const float* q;
  int n, W;
  uint8_t* status;
  int32_t* first_fail;
  const uint8_t* bimage;  // packed B' (32 KB chunks)
  int n_tiles;            // N tiles of 256 obstacles
  const float4* obs;      // obstacle spheres {x, y, z, rho}, the image's row order
  int n_obs;
  float4 origin;          // {o, guard / 2}
  float bound;            // E: pairs with s >= E cannot collide
  unsigned long long* counters;  // [1] exact rechecks (may be null)
  int* error;
  int* next;  // motion counter for the CTAs' dynamic scheduling, zeroed before the launch
  unsigned long long wait_ns;  // limit of every bounded wait (0: the default, 1 s)
};
size_t gemm_cc_smem_bytes();
cudaError_t launch_gemm_cc(int tf32, const RobotDev& rb, const GemmCcArgs& a, int sm_count, cudaStream_t s);

// Fused tensor-core inference (mlp_fused.cu). Rows are configurations q [rows][ldq] when q
// is set, else waypoints of motions (row m * W + i of the interpolation q0[m] -> q1[m]).
struct FusedMlpArgs {
  const float* q;
  int ldq;
  const float* q0;
  const float* q1;
  int W;
  int dof;
  int rows;
  const uint8_t* wpack;  // packed weight image (launch_mlp_pack)
  const float* bias;     // [3][256] + [16] FP32
  float* out;            // [rows][16] corrections
  int* error;            // set to 1 when a wait timed out
  unsigned long long wait_ns;  // limit of every bounded wait (0: the default, 1 s)
};
size_t mlp_fused_image_bytes();
int mlp_fused_bias_floats();
size_t mlp_fused_smem_bytes();
// w0..w3: BF16 weights, padded [out][in] per layer ([256][16], [256][256] x 2, [16][256])
cudaError_t launch_mlp_pack(const void* w0, const void* w1, const void* w2, const void* w3,
                            uint8_t* image, cudaStream_t s);
cudaError_t launch_mlp_fused(const FusedMlpArgs& a, int sm_count, cudaStream_t s);
const char* mlp_fused_diag();  // why the last fused launch was refused, if it was
const int* mlp_error_flag(const MlpDev* d);
cudaError_t launch_residual_target(const float* q, const float* t, int rows, int dof, float* T,
                                   cudaStream_t s);
cudaError_t launch_accumulate(float* dst, const float* src, cudaStream_t s);

size_t validate_smem_bytes(const RobotDev& rb, const SceneDev& sc, int W, bool stage_obs);
cudaError_t launch_validate(const RobotDev& rb, const SceneDev& sc, const ConsDev& cs,
                            ValidateArgs a, const DeviceInfo& dev, cudaStream_t stream);
cudaError_t launch_project_configs(const RobotDev& rb, const ConsDev& cs, const float* q_in,
                                   int n, int max_iters, float* q_out, uint8_t* ok,
                                   float* resid, cudaStream_t stream);

}  // namespace cprrtc
