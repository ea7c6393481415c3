/*
 * cprrtc.h — C ABI of the GB300 (sm_103a) constrained-motion library.
 *
 * The library implements the data-parallel hot path of cpRRTC (Hu, Wang, Christensen,
 * "cpRRTC: GPU-Parallel RRT-Connect for Constrained Motion Planning"): for each candidate
 * motion, straight-line interpolation (Sec. III), parallel projection of the waypoints onto
 * a task-constraint manifold (Sec. III-A, Algorithm 1), forward kinematics of the robot's
 * collision spheres and sphere-vs-obstacle collision checks with early termination
 * (Sec. IV), and RRT-Connect tree extension with greedy connect (Sec. III, Sec. II).
 *
 * Conventions shared by every call:
 *  - Return value: CPRRTC_OK (0) or a negative CPRRTC_E_* code. On error nothing is written
 *    to outputs except where stated, and cprrtc_last_error(ctx) describes the failure.
 *    Per-motion and per-problem outcomes are reported in status arrays, never as errors.
 *  - Arrays are C-contiguous. Configurations are FP32, [n][dof]. Robot and scene
 *    parameters are passed as doubles and stored on the device as FP32.
 *  - Array pointers may be host or device memory (detected per pointer). If every array of
 *    a call is device memory the call is asynchronous on the context's stream; otherwise
 *    the library copies through its own device buffers and returns after the results are in
 *    host memory. Device memory must belong to the context's GPU (managed memory is
 *    accepted as it is); an array in another GPU's memory is E_INVALID_ARG.
 *  - The caller owns every buffer it passes. set_* calls copy their arguments into
 *    library-owned device memory, replacing the previous copy.
 *  - One context per host thread; contexts are independent.
 */
#ifndef CPRRTC_H
#define CPRRTC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CPRRTC_MAX_DOF 8
#define CPRRTC_MAX_W 64
#define CPRRTC_MAX_SPHERES 256

/* ---- error codes ---- */
#define CPRRTC_OK 0
#define CPRRTC_E_INVALID_ARG (-1)
#define CPRRTC_E_NOT_CONFIGURED (-2)
#define CPRRTC_E_CUDA (-3)
#define CPRRTC_E_OOM (-4)
#define CPRRTC_E_CAPACITY (-5)
#define CPRRTC_E_TIMEOUT (-6)
#define CPRRTC_E_UNSUPPORTED (-7)

/* ---- enums ---- */
#define CPRRTC_JOINT_REVOLUTE 0
#define CPRRTC_JOINT_PRISMATIC 1

#define CPRRTC_CONSTRAINT_NONE 0       /* no projection; collision checks only */
#define CPRRTC_CONSTRAINT_ROLL_PITCH 1 /* end-effector roll and pitch held at 0 */
#define CPRRTC_CONSTRAINT_Z_PLANE 2    /* end-effector point on the plane z = target */
/* The paper's other constraint variants (Sec. V-B: a line, and a fixed orientation added to
 * a plane or a line); the fixed orientation is roll = pitch = 0 and yaw = `yaw`. Validation,
 * projection and plan only (not the uneven batch). */
#define CPRRTC_CONSTRAINT_LINE 3         /* end-effector point on {y = line_y, z = target} */
#define CPRRTC_CONSTRAINT_ORIENT_PLANE 4 /* fixed orientation and the plane z = target */
#define CPRRTC_CONSTRAINT_ORIENT_LINE 5  /* fixed orientation and the line of LINE */

#define CPRRTC_MOTION_VALID 0
#define CPRRTC_MOTION_PROJ_FAIL 1 /* Alg. 1 returned None (not projected in max_iters) */
#define CPRRTC_MOTION_COLLISION 2

/* ---- robot and scene ---- */

/* One joint in standard Denavit-Hartenberg form (Sec. III: FK per waypoint):
 * revolute  T = Rz(theta0 + q) Tz(d) Tx(a) Rx(alpha);
 * prismatic T = Rz(theta0) Tz(d + q) Tx(a) Rx(alpha). Limits [lo, hi] clamp projection. */
typedef struct {
  int type;
  double d, a, alpha, theta0, lo, hi;
} cprrtc_joint;

/* A collision sphere rigidly attached to a frame: frame 0 is the base (world), frame k the
 * frame after joint k; centre (x, y, z) in that frame, radius r > 0. */
typedef struct {
  int frame;
  double x, y, z, r;
} cprrtc_sphere;

typedef struct {
  double x, y, z, r;
} cprrtc_obs_sphere;

/* Oriented box: centre c, half-extents h, rotation R (row-major) with world = c + R local. */
typedef struct {
  double c[3];
  double h[3];
  double R[9];
} cprrtc_obs_box;

/* Capsule: segment p0-p1 swept by a ball of radius r. */
typedef struct {
  double p0[3];
  double p1[3];
  double r;
} cprrtc_obs_capsule;

/* Task constraint and the parameters of Algorithm 1 (Sec. III-A). A waypoint is valid when
 * ||E_task||_inf < tol_task and max_k E_sm,k < tol_sm, with
 * E_sm,k = max(0, |xi_k[i] - xi_k[i-1]| - tau) and
 * tau = max(c_sm * ||q_end - q_start||_inf / (W - 1), tau_floor).
 * Update: xi_new[i] = clamp(xi[i] - alpha (J^+ E_task + (xi[i] - xi[i-1]) * E_sm)), with
 * the damped pseudoinverse J^+ = J^T (J J^T + lambda^2 I)^-1. Task errors (m rows):
 * ROLL_PITCH [roll, pitch] (ZYX Euler angles of the end-effector rotation); Z_PLANE
 * [p_z - target]; LINE [p_y - line_y, p_z - target]; ORIENT_PLANE [roll, pitch,
 * yaw - yaw (wrapped to (-pi, pi]), p_z - target]; ORIENT_LINE [roll, pitch, yaw - yaw,
 * p_y - line_y, p_z - target]; p is the end-effector point. */
typedef struct {
  int type;         /* CPRRTC_CONSTRAINT_* */
  double target;    /* plane height (Z_PLANE, ORIENT_PLANE) or line height (LINE, ORIENT_LINE) */
  double tol_task;  /* default 1e-4 */
  double c_sm;      /* default 2 */
  double tau_floor; /* default 1e-3 */
  double tol_sm;    /* default 1e-4 */
  double alpha;     /* default 1 */
  double lambda;    /* default 1e-3 */
  int max_iters;    /* 1..255, default 20 */
  double line_y;    /* LINE, ORIENT_LINE: y of the line */
  double yaw;       /* ORIENT_PLANE, ORIENT_LINE: end-effector yaw, rad */
} cprrtc_constraint;

typedef struct cprrtc_ctx cprrtc_ctx;

/* ---- lifecycle ---- */

/* Creates a context on CUDA device `device`. `stream` is a cudaStream_t (NULL: the legacy
 * default stream). *out receives the context; it is NULL on failure.
 * Errors: E_INVALID_ARG (out NULL, bad device), E_CUDA, E_OOM. */
int cprrtc_create(cprrtc_ctx** out, int device, void* stream);

/* Waits for the context's stream (the whole device when it runs on the legacy default
 * stream), then frees the context and every device buffer it owns. Accepts NULL. Always
 * returns CPRRTC_OK. */
int cprrtc_destroy(cprrtc_ctx* ctx);

/* Replaces the stream later calls run on (a cudaStream_t; NULL: the legacy default stream).
 * Work already queued stays on the previous stream; order the two streams yourself if a
 * later call reads its results. Errors: E_INVALID_ARG (null context). */
int cprrtc_set_stream(cprrtc_ctx* ctx, void* stream);

/* Message for the last error on this context ("" if none). Owned by the context. */
const char* cprrtc_last_error(const cprrtc_ctx* ctx);

/* Robot kinematic table and collision spheres (Sec. III: every waypoint of a motion is
 * placed by the arm's kinematic chain and its spheres tested against the obstacles).
 * 1 <= dof <= 8, 1 <= n_spheres <= 256,
 * sphere frames in [0, dof], ee = end-effector point in frame dof (host pointers).
 * Errors: E_INVALID_ARG, E_UNSUPPORTED (sizes beyond the maxima), E_CUDA, E_OOM. */
int cprrtc_set_robot(cprrtc_ctx* ctx, const cprrtc_joint* joints, int dof,
                     const cprrtc_sphere* spheres, int n_spheres, const double ee[3]);

/* Obstacle set (Sec. IV; cuboid obstacles in Sec. V). Host pointers; a pointer may be NULL
 * when its count is 0. Counts >= 0; the total may be 0. Errors: E_INVALID_ARG, E_CUDA,
 * E_OOM. */
int cprrtc_set_obstacles(cprrtc_ctx* ctx, const cprrtc_obs_sphere* spheres, int n_spheres,
                         const cprrtc_obs_box* boxes, int n_boxes,
                         const cprrtc_obs_capsule* capsules, int n_capsules);

/* Task constraint and Algorithm 1 parameters (Sec. III-A). Errors: E_INVALID_ARG. */
int cprrtc_set_constraint(cprrtc_ctx* ctx, const cprrtc_constraint* c);

/* ---- motion validation (Sec. III, Alg. 1, Sec. IV) ---- */

/* Validates n motions q_start[m] -> q_end[m], each as W >= 2 interpolated waypoints
 * (W <= 64): interpolation, Alg. 1 projection (unless the constraint is NONE), then FK and
 * CC of every waypoint of the projected segment, waypoint 0 included.
 * Outputs (any may be NULL except status):
 *   out_q      [n][W][dof] projected segment (for PROJ_FAIL: the segment after the last
 *              iteration);
 *   status     [n] CPRRTC_MOTION_*;
 *   first_fail [n] first unaccepted waypoint (PROJ_FAIL), first colliding waypoint
 *              (COLLISION) or -1 (VALID);
 *   iters      [n] iteration at which Alg. 1 accepted the segment (0 for NONE;
 *              max_iters on PROJ_FAIL);
 *   resid      [n] max over waypoints 1..W-1 of the last evaluated ||E_task||_inf.
 * Requires set_robot. Errors: E_NOT_CONFIGURED, E_INVALID_ARG, E_UNSUPPORTED, E_CUDA,
 * E_OOM. n = 0 is a no-op. */
int cprrtc_validate(cprrtc_ctx* ctx, const float* q_start, const float* q_end, int n, int W,
                    float* out_q, uint8_t* status, int32_t* first_fail, uint8_t* iters,
                    float* resid);

/* Projects n single configurations onto the constraint manifold by repeated damped steps
 * q <- clamp(q - alpha J^+ E_task) until ||E_task||_inf < tol_task, at most max_iters
 * steps (the per-waypoint update of Alg. 1 without the smoothing term; the projection
 * operator of CBiRRT-style planners, Sec. II). q_out [n][dof]; ok [n] 1/0; resid [n]
 * (may be NULL). Requires set_robot and a constraint other than NONE. */
int cprrtc_project_configs(cprrtc_ctx* ctx, const float* q_in, int n, int max_iters,
                           float* q_out, uint8_t* ok, float* resid);

/* ---- collision checking in GEMM form ---- */

#define CPRRTC_CC_EXACT 0     /* per-pair FP32 tests with culling (default) */
#define CPRRTC_CC_GEMM_TF32 1 /* dense distance contraction on the tensor cores, TF32 */
#define CPRRTC_CC_GEMM_BF16 2 /* the same in BF16 */

/* Selects how cprrtc_validate checks collisions (Sec. IV's check, computed differently; the
 * paper has no GEMM form). In the GEMM modes the squared distances of all robot-sphere x
 * obstacle pairs of a waypoint, less the squared contact distance inflated by `guard_m`
 * (metres, in [0, 0.1]; 0.005 is a 5 mm band), are one dense contraction of hi/lo-split
 * operands with FP32 accumulation; the library bounds its error (cprrtc_cc_stats), and every
 * pair it cannot clear is rechecked with the exact FP32 test. The outputs (status,
 * first_fail, waypoints) are identical to CPRRTC_CC_EXACT's. GEMM modes take sphere
 * obstacles only and at most 128 robot spheres (else cprrtc_validate returns
 * E_UNSUPPORTED); they apply to cprrtc_validate (not to the planner or the warm-start call).
 * Requires set_robot for the GEMM modes. Errors: E_INVALID_ARG, E_NOT_CONFIGURED, E_CUDA,
 * E_OOM. */
int cprrtc_set_cc_mode(cprrtc_ctx* ctx, int mode, double guard_m);

/* The GEMM-form check's error bound E (m^2; 0 in EXACT mode) and its counters since the
 * last reset: counters[0] = pairs rechecked exactly, counters[1] = unused (0). Synchronises
 * the context's stream; reset = 1 zeroes the counters. */
int cprrtc_cc_stats(cprrtc_ctx* ctx, double* bound_m2, int64_t* counters, int reset);

/* ---- learned projection warm start ---- */

/* A multilayer perceptron that predicts, for a configuration q, the correction
 * proj(q) - q that the projection (cprrtc_project_configs) would apply, so that Alg. 1 can
 * start closer to the manifold. The paper has no learned component: this is an addition,
 * and the plain Alg. 1 stays both the fallback and the judge of every warm-started segment
 * (cprrtc_validate_ws).
 * Network (one per context, for the dof of the robot set when it is created):
 *   x = q / pi; h1 = gelu(W1 x + b1); h2 = gelu(W2 h1 + b2); h3 = gelu(W3 h2 + b3);
 *   correction = W4 h3 + b4, widths dof -> 256 -> 256 -> 256 -> dof,
 *   gelu(z) = z Phi(z) with Phi the standard normal CDF (the erf form; on the GPU erf is
 *   evaluated with Abramowitz and Stegun 7.1.28, |error| <= 3e-7, below BF16 resolution).
 * Weights and activations are BF16 and products accumulate in FP32 on the tensor cores;
 * biases, the FP32 master weights and the Adam state stay FP32.
 * Parameter layout (compact, FP32, cprrtc_mlp_param_count(dof) entries): for l = 1..4,
 * W_l [out_l][in_l] row-major then b_l [out_l]. */
int64_t cprrtc_mlp_param_count(int dof);

/* Creates (or re-creates) the network for the current robot, He-normal weights (the last
 * layer scaled by 0.1) and zero biases from `seed`; resets the optimiser.
 * Requires set_robot. Errors: E_NOT_CONFIGURED, E_CUDA, E_OOM. */
int cprrtc_mlp_init(cprrtc_ctx* ctx, uint64_t seed);

/* Limit of every bounded wait in the tensor-core kernels (the GEMM-form collision check, the
 * warm-start network's fused inference and its training GEMMs), in seconds: 0 restores the
 * default of 1 s; otherwise 1e-6 .. 10. A wait that reaches it makes the kernel give up: it
 * raises its abort flag, lets its copies and MMAs in flight complete, frees its tensor
 * memory and exits, and the call reports it: cprrtc_validate with a GEMM mode and
 * cprrtc_mlp_infer return E_TIMEOUT when they are synchronous (some array in host memory;
 * their outputs are then not valid), cprrtc_mlp_grad and cprrtc_mlp_train return
 * E_TIMEOUT, and cprrtc_validate_ws falls back to plain Alg. 1 for every motion. The
 * next call starts afresh. The paper has no counterpart: this is a failure-detection
 * setting, and a very short limit lets a test make the waits run out on an ordinary input.
 * Errors: E_INVALID_ARG. */
int cprrtc_set_wait_limit(cprrtc_ctx* ctx, double seconds);

/* Arithmetic of the network's calls (cprrtc_mlp_grad, cprrtc_mlp_train, cprrtc_mlp_infer,
 * cprrtc_validate_ws): CPRRTC_MLP_BF16 (the default; BF16 weights and activations, FP32
 * accumulation, tensor-core inference) or CPRRTC_MLP_FP32, a checking mode with the FP32
 * master weights and FP32 activations on FP32 FMA kernels (no BF16 rounding anywhere; the
 * inference is the unfused forward pass). The checking mode separates the layers'
 * arithmetic from BF16 rounding when the kernels are compared with an FP64 evaluation; it
 * is not a production path. The setting persists across cprrtc_mlp_init.
 * Errors: E_INVALID_ARG (unknown precision). */
#define CPRRTC_MLP_BF16 0
#define CPRRTC_MLP_FP32 1
int cprrtc_mlp_set_precision(cprrtc_ctx* ctx, int precision);

/* Sets / reads the parameters (host arrays of `count` = cprrtc_mlp_param_count(dof)
 * floats). Setting resets the Adam state. Errors: E_NOT_CONFIGURED (no network),
 * E_INVALID_ARG (count mismatch, null), E_CUDA. */
int cprrtc_mlp_set_params(cprrtc_ctx* ctx, const float* params, int64_t count);
int cprrtc_mlp_get_params(cprrtc_ctx* ctx, float* params, int64_t count);

/* Checkpoints of the network: parameters, Adam moments and step count in a versioned
 * binary file (little-endian): magic "CPRMLP01", uint32 version (1), dof, hidden (256),
 * layers (4), int32 step, uint32 0, uint64 count, then count floats each of parameters,
 * first and second moments (compact layout), then the CRC-32 (IEEE) of all preceding
 * bytes. Load requires set_robot with the file's dof (creating the network if needed) and
 * rejects a wrong magic, version, shape, size or checksum. Synchronous. Errors:
 * E_NOT_CONFIGURED, E_INVALID_ARG (I/O or format), E_CUDA, E_OOM. */
int cprrtc_mlp_save(cprrtc_ctx* ctx, const char* path);
int cprrtc_mlp_load(cprrtc_ctx* ctx, const char* path);

/* Loss L = (1 / rows) sum_r 0.5 |f(q_r) - (t_r - q_r)|^2 over rows pairs (q [rows][dof],
 * t [rows][dof]: q's projection) and its gradient with respect to every parameter
 * (grads: host array of cprrtc_mlp_param_count(dof) floats, compact layout; loss: host,
 * 1 float; either may be NULL). Does not change the parameters. Synchronous. The GEMMs run
 * on the tensor cores (BF16, FP32 accumulation; FP32 FMAs in the checking mode), every wait
 * bounded by cprrtc_set_wait_limit's limit.
 * Errors: E_NOT_CONFIGURED, E_INVALID_ARG, E_CUDA, E_OOM, E_TIMEOUT (a wait ran out; the
 * outputs are then not valid). */
int cprrtc_mlp_grad(cprrtc_ctx* ctx, const float* q, const float* t, int rows, float* grads,
                    float* loss);

/* Trains on n pairs (q, t) as above: `epochs` passes of minibatch Adam (beta1 0.9, beta2
 * 0.999, eps 1e-8, learning rate lr) over floor(n / batch) batches in an order drawn per
 * epoch from `seed`. loss_per_epoch [epochs] (host, may be NULL) receives each epoch's mean
 * batch loss. Synchronous. Errors: E_NOT_CONFIGURED, E_INVALID_ARG (n < batch, batch < 1,
 * epochs < 0, lr not finite), E_CUDA, E_OOM, E_TIMEOUT (a wait of the tensor-core GEMMs ran
 * out; the parameters are then not valid). */
int cprrtc_mlp_train(cprrtc_ctx* ctx, const float* q, const float* t, int n, int batch,
                     int epochs, float lr, uint64_t seed, float* loss_per_epoch);

/* q_out [rows][dof] = q + correction(q) for rows configurations (no clamping).
 * Errors: E_NOT_CONFIGURED, E_INVALID_ARG, E_CUDA, E_OOM. */
int cprrtc_mlp_infer(cprrtc_ctx* ctx, const float* q, int rows, float* q_out);

/* cprrtc_validate with the learned warm start: waypoint i = 1..W-1 of each motion's
 * interpolation xi gets the correction f(xi_i) - (1 - i / (W - 1)) f(xi_0), clamped to the
 * joint limits (xi_0 = q_start is taken to lie on the manifold, so f(xi_0) is the network's
 * local error and is removed where the segment leaves its fixed start). If the largest
 * ||E_task||_inf over those waypoints is then below that of the plain interpolation, Alg. 1
 * runs from the corrected segment for at most refine_iters (1..20) iterations with the
 * same thresholds. If the corrected start is not closer, or its run does not accept the
 * whole segment, Alg. 1 runs from the plain interpolation with max_iters iterations,
 * exactly as in cprrtc_validate. Collision checking then proceeds on the accepted segment.
 * iters [n] counts the iterations of both runs; warm_used [n] (may be NULL) is 1 when the
 * warm-started segment was the one accepted. Other arguments
 * and outputs as cprrtc_validate. Requires set_robot, a constraint other than NONE and a
 * network for the robot's dof. Errors: as cprrtc_validate. */
int cprrtc_validate_ws(cprrtc_ctx* ctx, const float* q_start, const float* q_end, int n, int W,
                       int refine_iters, float* out_q, uint8_t* status, int32_t* first_fail,
                       uint8_t* iters, float* resid, uint8_t* warm_used);

/* ---- planning (Sec. III: RRT-Connect tree extension with constrained motions) ---- */

/* Per-problem obstacle sets for cprrtc_plan with use_scene_batch = 1: problem p uses
 * scene p. Scene s owns spheres [sphere_offsets[s], sphere_offsets[s+1]) of `spheres`, and
 * likewise boxes and capsules; each offsets array has n_scenes + 1 non-decreasing entries
 * starting at 0 (host pointers). Errors: E_INVALID_ARG, E_CUDA, E_OOM. */
int cprrtc_set_scene_batch(cprrtc_ctx* ctx, int n_scenes, const cprrtc_obs_sphere* spheres,
                           const int32_t* sphere_offsets, const cprrtc_obs_box* boxes,
                           const int32_t* box_offsets, const cprrtc_obs_capsule* capsules,
                           const int32_t* capsule_offsets);

/* RRT-Connect parameters. Each round, `workers` extensions run in parallel against the
 * trees as they stood at the round's start; worker w extends tree (round + w) mod 2 toward
 * a Philox4x32-10 sample (counter {problem, round, w, draw}, key {seed, 0}), then greedily
 * extends the same tree toward the nearest node of the other tree while each projected
 * motion is valid and ends strictly closer (Sec. III). The trees connect when the closing
 * hop (within 10 * tau_floor in inf-norm) is valid without projection. New nodes are
 * appended in worker order; the lowest worker that connects wins. Deterministic for a
 * seed. */
typedef struct {
  double range;        /* steering step, L2 in joint space; default 0.3 */
  int W;               /* waypoints per motion, 2..64; default 32 */
  int max_rounds;      /* rounds per problem (>= 1); default 200 */
  int workers;         /* extensions per round = warps per problem, 1..16 (fewer for
                          W > 32, where the kernel's registers bound the CTA size: more is
                          E_UNSUPPORTED); default 8 */
  int max_nodes;       /* capacity of each tree (>= 2); default 2048 */
  int max_connect;     /* greedy connect steps per extension (>= 0); default 32 */
  int max_path;        /* capacity of the path outputs, in nodes (>= 2); default 512 */
  uint32_t seed;
  int use_scene_batch; /* 1: problem p uses scene p of cprrtc_set_scene_batch; 0: the
                          cprrtc_set_obstacles scene for every problem */
  double time_budget_ms; /* device time per problem (>= 0; 0: none): a problem whose budget
                            is spent stops at the end of its round with path_len 0 unless
                            it connected; results then depend on timing */
} cprrtc_plan_params;

/* Plans n problems start[p] -> goal[p] ([n][dof], on the constraint manifold and
 * collision-free for a meaningful result). Outputs (path_len required, the rest may be
 * NULL):
 *   path_len   [n] nodes in the path (0: not solved in max_rounds; -needed if the path
 *              did not fit in max_path);
 *   path       [n][max_path][dof] nodes from start to goal;
 *   path_edges [n][max_path-1][W][dof] the validated (projected) motion between path
 *              nodes j and j+1, waypoint 0 at node j (rows of path and path_edges
 *              beyond path_len are not written);
 *   rounds     [n] rounds run; waypoints [n] waypoints validated (W per motion checked);
 *   plan_ms    [n] device time the problem was planned, ms (the sum of its slices under
 *              the time-sliced schedule, see cprrtc_set_plan_slicing);
 *   work       [n][2] work evaluated: Alg. 1 waypoint updates (iterations x (W-1) summed
 *              over motions) and waypoints collision-checked (early exit included).
 * The library keeps the trees in its own device memory (about
 * n * 2 * max_nodes * (W * dof + 9) * 4 bytes). Requires set_robot, and set_obstacles or
 * set_scene_batch (n_scenes = n). Errors: E_NOT_CONFIGURED, E_INVALID_ARG, E_UNSUPPORTED,
 * E_CUDA, E_OOM, and E_TIMEOUT (some array in host memory, time-sliced schedule) if a wait
 * of the schedule's queue ran out (outputs then not valid). */
int cprrtc_plan(cprrtc_ctx* ctx, const float* start, const float* goal, int n,
                const cprrtc_plan_params* params, int32_t* path_len, float* path,
                float* path_edges, int32_t* rounds, int64_t* waypoints, float* plan_ms,
                int64_t* work);

/* The planner's learned form (not in the paper; the warm start of cprrtc_validate_ws inside
 * RRT-Connect): with refine_iters in 1..20, cprrtc_plan and cprrtc_plan_static warm-start every
 * extend motion (the first motion of a chain, toward a sample). The network's correction
 * f(q1) of the motion's end q1 moves waypoint i by (i / (W-1)) f(q1), clamped to the joint
 * limits: cprrtc_validate_ws's correction f(xi_i) - (1 - i/(W-1)) f(xi_0) with f taken linear
 * along the motion, where the start term cancels (one network evaluation per motion instead
 * of W). The corrected segment is tried only if its largest ||E_task||_inf over waypoints
 * 1..W-1 is below the interpolation's, for refine_iters Alg. 1 iterations; if they do not
 * accept the whole segment, plain Alg. 1 runs from the interpolation with max_iters, so Alg. 1
 * stays the judge of every motion. Connect steps and closing hops are planned as without it.
 * The network is the context's (cprrtc_mlp_init / cprrtc_mlp_load for the robot's dof, BF16
 * weights); each warp evaluates its motion's row itself. Constraints ROLL_PITCH and Z_PLANE
 * with the parallel projection; planning otherwise returns E_UNSUPPORTED, and without a
 * network for the robot E_NOT_CONFIGURED. 0 turns it off (the default).
 * Errors: E_INVALID_ARG (refine_iters outside 0..20). */
int cprrtc_set_plan_warm_start(cprrtc_ctx* ctx, int refine_iters);

/* Schedule of cprrtc_plan's problems on the GPU (not in the paper, which plans one problem per
 * run; the search and every output but plan_ms's timing are the same for every setting).
 * With first_slice > 0 (the default: first_slice 100, slice 50) the planner runs as many
 * persistent CTAs as fit the GPU at once; a CTA takes a problem from a queue and runs its
 * first first_slice rounds, later ones slice rounds at a time. Between slices an unsolved
 * problem goes back to the queue's tail while other problems wait for a CTA, unless its
 * rounds have taken more than 1.1 times the launch's mean round time so far, and stays with
 * its CTA otherwise (its state between slices, about 1.6 KB, lives in the library's device
 * memory beside the trees). Problems that solve within their first slice plan in one stretch;
 * the long ones share the GPU round-robin, the slowest keeping their CTAs, so a large batch
 * no longer ends with the long problems that happened to start last. first_slice = 0: one CTA per problem, each planned
 * in one stretch (cprrtc_plan_static always plans so). The queue's one wait (for another
 * CTA's store of a handed-over problem, a few instructions) gives up after 1 s.
 * Errors: E_INVALID_ARG (first_slice < 0, or slice < 1 with first_slice > 0). */
int cprrtc_set_plan_slicing(cprrtc_ctx* ctx, int first_slice, int slice);

/* ---- batches of uneven planning problems ---- */

/* An addition for serving: the paper plans one problem per run. Every problem of a batch
 * is planned as cprrtc_plan plans it (Sec. III), with its own robot, constraint, scene
 * and W; only the launch (persistent kernels, a CUDA graph, tuned shapes) differs. */

/* One robot of a robot table (arguments of cprrtc_set_robot). */
typedef struct {
  const cprrtc_joint* joints;
  int dof;
  const cprrtc_sphere* spheres;
  int n_spheres;
  double ee[3];
} cprrtc_robot_desc;

#define CPRRTC_BATCH_MAX_ROBOTS 8
#define CPRRTC_BATCH_MAX_CONSTRAINTS 8
/* Problem classes of a batch: 2 * constraint type + (W > 32). */
#define CPRRTC_BATCH_CLASSES 6

/* Robot table for cprrtc_plan_batch (1 <= n <= CPRRTC_BATCH_MAX_ROBOTS; host pointers).
 * Errors: as cprrtc_set_robot, E_UNSUPPORTED for n beyond the maximum. */
int cprrtc_set_robot_table(cprrtc_ctx* ctx, const cprrtc_robot_desc* robots, int n);
/* The uneven batch's learned form (not in the paper): a copy of the context's current network
 * (cprrtc_mlp_init / cprrtc_mlp_train / cprrtc_mlp_load, trained for the table robot's dof
 * and that constraint) for the problems of table robot `robot` and table constraint
 * `constraint` (ROLL_PITCH or Z_PLANE). With cprrtc_set_plan_warm_start on, cprrtc_plan_batch,
 * cprrtc_autotune_batch and cprrtc_batch_capture warm-start the extend motions of those
 * problems as cprrtc_plan does; problems of a pair without a network plan as without it.
 * Adopting again for a pair replaces its copy; cprrtc_set_robot_table and
 * cprrtc_set_constraint_table drop every copy. Errors: E_INVALID_ARG (no such robot or
 * constraint), E_UNSUPPORTED (another constraint type), E_NOT_CONFIGURED (no network, or one
 * of another dof), E_CUDA, E_OOM. */
int cprrtc_batch_adopt_network(cprrtc_ctx* ctx, int robot, int constraint);
/* Self-collision frame pairs of robot `robot` of the table, as cprrtc_set_self_collision's
 * frame_pairs for that robot's dof (n = (dof+1)^2; 0 or NULL: none): the uneven batch checks
 * every motion of that robot's problems against them. cprrtc_set_robot_table clears every
 * robot's pairs. Errors: E_INVALID_ARG (no such robot, wrong n). */
int cprrtc_set_table_self_collision(cprrtc_ctx* ctx, int robot, const uint8_t* frame_pairs, int n);

/* Constraint table for cprrtc_plan_batch (1 <= n <= CPRRTC_BATCH_MAX_CONSTRAINTS; host
 * array). Every entry is checked as cprrtc_set_constraint checks it; the context's own
 * constraint is left as it was. Errors: E_INVALID_ARG (empty table, bad field),
 * E_UNSUPPORTED (n beyond the maximum, a type other than NONE, ROLL_PITCH or Z_PLANE). */
int cprrtc_set_constraint_table(cprrtc_ctx* ctx, const cprrtc_constraint* constraints, int n);

/* One problem of a batch: indices into the robot table, the constraint table and the scene
 * batch (cprrtc_set_scene_batch), and its waypoints per motion (2..64). */
typedef struct {
  int robot;
  int constraint;
  int scene;
  int W;
} cprrtc_problem;

/* Launch shape of each problem class (class = 2 * constraint type + (W > 32)): CTAs per SM
 * of its one-warp part (0: as many as fit), whether the class stages its obstacles into
 * shared memory (else they are read through L1), warps per motion, and pair_problems.
 * Warps per motion is 1, or 2 for the whole class on warp pairs (each worker's motion held
 * by two warps; plain form only, at most 8 workers; any other value means 1). With 1,
 * pair_problems (0 or more) of the class's problems, its heaviest by the batch's cost
 * estimate, are planned on warp pairs all the same, and the rest with one warp per motion:
 * the heaviest problems end the batch, and pairs shorten them. A pair splits a motion of
 * 33..64 waypoints by waypoints (one per lane: Alg. 1 runs in step on both warps, each
 * checks its own waypoints for collisions) and a motion of up to 32 waypoints by obstacles
 * (both warps run Alg. 1 on the whole motion, each checks half of the obstacle chunks).
 * None of them changes any result: a problem's search depends only on its own inputs and
 * the plan parameters. Only the executed-work counts differ with warp pairs
 * (cprrtc_work_counters, the `work` output): a pair's halves stop their collision walks
 * when either finds a collision, so their collision work depends on timing. */
typedef struct {
  int ctas_per_sm[CPRRTC_BATCH_CLASSES];
  int stage_obstacles[CPRRTC_BATCH_CLASSES];
  int warps_per_motion[CPRRTC_BATCH_CLASSES];
  int pair_problems[CPRRTC_BATCH_CLASSES];
} cprrtc_tuning;

/* Plans n problems of mixed robots, constraints, scenes and W in one go: every problem class
 * runs one persistent kernel (grid of SMs x CTAs per SM) that takes problems from an atomic
 * queue, longest expected first; the classes run concurrently. Each problem is planned
 * exactly as cprrtc_plan would plan it with its own robot, constraint, scene and W (problem
 * index p in the Philox counter). problems: host array. start, goal: [n][8] (first dof
 * entries used). params: range, max_rounds, workers, max_nodes, max_connect, max_path and
 * seed are used; W and use_scene_batch are ignored. tuning: NULL uses the last
 * cprrtc_autotune_batch result (as many CTAs as fit, staging when it fits, one warp per
 * motion, if none). Outputs as cprrtc_plan with configurations padded to 8 floats: path
 * [n][max_path][8], path_edges [n][max_path-1][Wmax][8] (Wmax = largest W of the batch; NULL
 * allowed). Errors: E_NOT_CONFIGURED (tables or scene batch missing), E_INVALID_ARG (bad
 * index, W, parameter), E_CUDA, E_OOM. */
int cprrtc_plan_batch(cprrtc_ctx* ctx, const cprrtc_problem* problems, int n, const float* start,
                      const float* goal, const cprrtc_plan_params* params,
                      const cprrtc_tuning* tuning, int32_t* path_len, float* path,
                      float* path_edges, int32_t* rounds, int64_t* waypoints, float* plan_ms,
                      int64_t* work);

/* Autotuner: for every class present in the batch, times short runs (trial_rounds rounds)
 * of each launch shape (obstacles staged or read through L1; 1 up to the fitting number of
 * CTAs per SM; one warp per motion with none, 4 or 16 of the class's heaviest problems on warp
 * pairs, or warp pairs for the whole class; no pairs in the learned form) and keeps
 * the shape with the most waypoints validated per second. The result is written to *out (may be NULL) and becomes the default of later
 * batch calls on this context. start, goal: device or host, as cprrtc_plan_batch. The trial
 * outputs go to library buffers; returns after the trials. Errors: as cprrtc_plan_batch,
 * and E_INVALID_ARG for trial_rounds < 1. */
int cprrtc_autotune_batch(cprrtc_ctx* ctx, const cprrtc_problem* problems, int n,
                          const float* start, const float* goal, const cprrtc_plan_params* params,
                          int trial_rounds, cprrtc_tuning* out);

/* Records one cprrtc_plan_batch into a CUDA graph held by the context (replacing any
 * previous one); cprrtc_batch_replay launches it on the context's stream. Every array must
 * be device memory; a replay reads the current contents of start and goal and overwrites
 * the outputs. The problems, tables and scene batch are the ones at capture time.
 * Capture errors: as cprrtc_plan_batch, and E_INVALID_ARG for a host array. Replay errors:
 * E_NOT_CONFIGURED (nothing captured), E_CUDA. */
int cprrtc_batch_capture(cprrtc_ctx* ctx, const cprrtc_problem* problems, int n,
                         const float* start, const float* goal, const cprrtc_plan_params* params,
                         const cprrtc_tuning* tuning, int32_t* path_len, float* path,
                         float* path_edges, int32_t* rounds, int64_t* waypoints, float* plan_ms,
                         int64_t* work);
int cprrtc_batch_replay(cprrtc_ctx* ctx);

/* When each problem of the last batch run on this context (cprrtc_plan_batch, a
 * cprrtc_batch_replay, or the autotuner's last trial) started and ended, in nanoseconds of
 * the GPU's global timer (the %globaltimer register read by the problem's CTA as it takes the
 * problem and as it writes its results): span[2p] and span[2p + 1], a host array of 2n
 * entries, n being that batch's problem count. Problems that did not run in it (an autotuner
 * trial runs one class) read 0 and 0. A measurement aid: the spans show how many problems
 * are in flight over the run, and so whether the run ends with the SMs idle behind its
 * slowest problems. Synchronises the context's stream. Errors: E_NOT_CONFIGURED (no batch has
 * run), E_INVALID_ARG (n other than that count, span NULL or not host memory), E_CUDA. */
int cprrtc_batch_spans(cprrtc_ctx* ctx, int64_t* span, int n);

/* ---- planning without allocation ---- */

/* Size of the library's fixed device scratch for cprrtc_plan_static: 16 MiB, held by every
 * GPU that loads the library until the process exits. */
#define CPRRTC_STATIC_SCRATCH_BYTES (16u << 20)

/* cprrtc_plan for callers that must not allocate device memory while they run: a control
 * loop that cannot absorb the latency and implicit device synchronisation of cudaMalloc,
 * or a process whose device memory is all held by another allocator (a framework's caching
 * pool). The paper has no counterpart; results are those of cprrtc_plan on the same
 * arguments.
 *  - It allocates nothing: the trees live in a file-scope device array of
 *    CPRRTC_STATIC_SCRATCH_BYTES instead of library-allocated memory. Inputs and outputs
 *    are the caller's and must all be device memory of the context's GPU (host pointers,
 *    or another GPU's memory: E_INVALID_ARG).
 *  - Sizes beyond the array (n * 2 * max_nodes * (W * dof + 9) * 4 bytes plus
 *    n * workers * (2 * W * dof + 8) * 4 bytes, each part rounded up to 256 bytes) are
 *    rejected with E_CAPACITY before anything is launched; the sizes are checked factor by
 *    factor, so no product can wrap around and pass.
 *  - The first call on a device looks up the array's device address (once per device and
 *    CUDA context); make that first call before any stream capture. A device reset
 *    (cudaDeviceReset, or a reset of the primary context) makes a new context, and the
 *    next call after it looks the address up again.
 *  - Every call on a device shares the one array, whose contents persist between calls;
 *    calls that overlap on the GPU (other streams, other host threads) race on it. The
 *    planner initialises every tree it reads, so a call never depends on an earlier
 *    call's contents.
 *  - Its work is added to cprrtc_work_counters like cprrtc_plan's. Kernel timing
 *    (cprrtc_set_timing) does not cover this call.
 * Errors: as cprrtc_plan, plus E_CAPACITY. */
int cprrtc_plan_static(cprrtc_ctx* ctx, const float* start, const float* goal, int n,
                       const cprrtc_plan_params* params, int32_t* path_len, float* path,
                       float* path_edges, int32_t* rounds, int64_t* waypoints,
                       float* plan_ms, int64_t* work);

/* ---- counter-based random numbers ---- */

/* Philox4x32-10 (Salmon et al., SC'11) of n counters [n][4] under key {key0, key1}, on the
 * device: out [n][4]. The generator the planner samples with (the paper samples with a
 * Halton sequence, Sec. V; a counter-based generator keeps every problem's samples
 * independent of the launch). n = 0 does nothing. Errors: E_INVALID_ARG (n < 0, null
 * array), E_CUDA, E_OOM. */
int cprrtc_philox(cprrtc_ctx* ctx, uint32_t key0, uint32_t key1, const uint32_t* counters,
                  int n, uint32_t* out);

/* ---- timing ---- */

/* Measurement helpers with no counterpart in the paper. When enabled, the library records
 * CUDA events around each launch of its kernels on the context's stream.
 * cprrtc_kernel_time returns the summed device time (ms) and the launch count of the
 * kernel named `name` ("validate", "project", "plan", "mlp_infer", "gemm_cc",
 * "self_collide") since the last reset, waiting for the recorded events (a name never
 * launched gives 0 and 0); cprrtc_reset_timing waits for them too and drops the sums.
 * Errors: E_INVALID_ARG (null argument), E_CUDA (kernel_time). */
int cprrtc_set_timing(cprrtc_ctx* ctx, int enabled);

/* Work the validate and plan kernels of this context evaluated since creation or the last
 * reset, for throughput accounting (out has 8 entries): out[0] Alg. 1 waypoint updates (per
 * iteration, the waypoints after prog; with a warm start also the two task-error evaluations
 * per waypoint that decide whether to use it), out[1] DH chains evaluated by collision
 * checking (per checked waypoint and pass), out[2] points moved to world coordinates (frame
 * bounding spheres and robot spheres), out[3..5] ball-vs-primitive tests against spheres,
 * boxes and capsules (swept bounds, frame bounds and robot spheres together), out[6] extend
 * motions of the planner's learned form that evaluated the network, out[7] those whose
 * warm-started segment was accepted. Synchronises the context's stream; reset = 1 zeroes
 * them. */
int cprrtc_work_counters(cprrtc_ctx* ctx, int64_t* out, int reset);
int cprrtc_kernel_time(cprrtc_ctx* ctx, const char* name, double* ms, long long* launches);
int cprrtc_reset_timing(cprrtc_ctx* ctx);

/* Self-collision, an addition for realistic arms (the paper's robots' own links are implied
 * obstacles, Sec. V): frame_pairs [(dof+1)][(dof+1)] (host, row-major; entry (a, b) or
 * (b, a) nonzero, a != b: the robot spheres of frames a and b are tested against each other,
 * touching counts as free; pairs on one frame are never tested). After cprrtc_validate's
 * collision check, motions that are valid or collide later get the first waypoint where
 * such a pair overlaps (status COLLISION, first_fail that waypoint). cprrtc_plan and
 * cprrtc_plan_static check every motion they validate in the same way (waypoints 1..W-1,
 * after its obstacles): a motion whose robot meets itself is not valid, so no returned path
 * self-collides. n = (dof+1)^2, or 0 (or frame_pairs NULL) to switch it off; set_robot
 * switches it off. cprrtc_validate_ws does not test it; the uneven batch takes each table
 * robot's pairs from cprrtc_set_table_self_collision. Errors: E_INVALID_ARG,
 * E_NOT_CONFIGURED. */
int cprrtc_set_self_collision(cprrtc_ctx* ctx, const uint8_t* frame_pairs, int n);

/* The projection the validation and the planner use: CPRRTC_PROJECTION_PARALLEL (Alg. 1,
 * the default) or CPRRTC_PROJECTION_SEQUENTIAL, the paper's naive baseline (cpRRTC-Naive,
 * Sec. V, CBiRRT-style): waypoints 1..W-1 one after another, each by damped steps from its
 * interpolated point moved by the previous waypoint's correction until ||E_task||_inf <
 * tol_task (at most max_iters steps), failing at the first waypoint that does not converge
 * or ends farther than tau + tol_sm from its predecessor; iters reports the total steps
 * (capped at 255). It takes ROLL_PITCH or Z_PLANE, and W <= 32 for planning (else
 * E_UNSUPPORTED); cprrtc_validate_ws and the uneven batch always use
 * Alg. 1. Errors: E_INVALID_ARG. */
#define CPRRTC_PROJECTION_PARALLEL 0
#define CPRRTC_PROJECTION_SEQUENTIAL 1
int cprrtc_set_projection(cprrtc_ctx* ctx, int mode);

/* Ablation of the paper's early termination (Sec. IV: a collision found by one thread ends
 * the motion's checks): with enabled = 0, cprrtc_validate and cprrtc_validate_ws check
 * every waypoint against every candidate obstacle, with the same outputs; the default is 1.
 * The planner always stops early. Errors: E_INVALID_ARG. */
int cprrtc_set_early_exit(cprrtc_ctx* ctx, int enabled);

/* Measurement helper with no counterpart in the paper: the FP32 FMA throughput of the
 * context's GPU (TFLOP/s, the best of scalar and packed FP32x2 FMA chains on every SM, CUDA
 * events on the context's stream), the denominator of the FP32 rooflines. Runs for a few
 * milliseconds and synchronises the stream; *tflops is a host pointer.
 * Errors: E_INVALID_ARG, E_CUDA, E_OOM. */
int cprrtc_measure_fp32_peak(cprrtc_ctx* ctx, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* CPRRTC_H */
