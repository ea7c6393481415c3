/*
 * FP64 CPU oracle for cpRRTC constrained motion validation and planning.
 *
 * TEST INFRASTRUCTURE ONLY. This library exists to check the CUDA path: only the test
 * suite, the smoke check and the benchmark's CPU legs (its cpu_baseline figure and its
 * reference arm) load it. It shares no code, header or table with the CUDA library, and
 * the CUDA library never calls it.
 *
 * It follows the paper (Hu, Wang, Christensen, "cpRRTC: GPU-Parallel RRT-Connect for
 * Constrained Motion Planning") step by step, in double precision, one motion at a time:
 *   - Sec. III: straight-line interpolation of a motion segment between q_near and q_steer,
 *     projection, then, per waypoint, the sphere positions from the kinematic chain (FK)
 *     and the sphere-obstacle tests (CC).
 *   - Sec. III-A, Algorithm 1 (ParallelProject): Jacobi-style projection of all waypoints
 *     at once, a task term J^+ E_task and a smoothing term J_sm E_sm, a shared prefix
 *     `prog` of accepted waypoints, success when the whole segment is accepted.
 *   - Sec. IV: CC reports the motion invalid at its first colliding waypoint.
 *   - Sec. III / Sec. II: RRT-Connect with greedy connect toward the other tree.
 *   - Sec. V: the baseline's sequential (CBiRRT-style) projection, and the other task
 *     constraints of Sec. V-B (a line; a fixed orientation with a plane or a line).
 *   - Optional self-collision: robot sphere pairs on frames the caller names.
 *
 * Array conventions (all row-major, double):
 *   joints   [dof][7]  {type (0 revolute, 1 prismatic), d, a, alpha, theta0, lo, hi}
 *   ee       [3]       end-effector point in the last joint frame
 *   spheres  [S][5]    {frame, x, y, z, r}, frame 0 = base, frame k = after joint k
 *   obs sph  [n][4]    {x, y, z, r}
 *   obs box  [n][15]   {cx, cy, cz, hx, hy, hz, R (3x3 row-major)}, world = c + R local
 *   obs cap  [n][7]    {p0 (3), p1 (3), r}
 */
#ifndef CPRRTC_ORACLE_H
#define CPRRTC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_DOF 8
#define ORC_MAX_W 64

enum { ORC_NONE = 0, ORC_ROLL_PITCH = 1, ORC_Z_PLANE = 2, ORC_LINE = 3, ORC_ORIENT_PLANE = 4,
       ORC_ORIENT_LINE = 5 };
enum { ORC_VALID = 0, ORC_PROJ_FAIL = 1, ORC_COLLISION = 2 };

typedef struct {
  int dof;
  const double* joints;   /* [dof][7] */
  const double* ee;       /* [3] */
  int n_spheres;
  const double* spheres;  /* [n_spheres][5] */
  /* self-collision: [(dof+1)][(dof+1)], nonzero at (a, b), a != b, when spheres of frames a
   * and b are tested against each other; NULL: no self-collision test */
  const unsigned char* self_pairs;
} orc_robot;

typedef struct {
  int n_sph;
  const double* sph;      /* [n_sph][4] */
  int n_box;
  const double* box;      /* [n_box][15] */
  int n_cap;
  const double* cap;      /* [n_cap][7] */
} orc_scene;

typedef struct {
  int type;               /* ORC_NONE .. ORC_ORIENT_LINE */
  double target;          /* plane height (Z_PLANE, ORIENT_PLANE) or line height (LINE, ORIENT_LINE) */
  double tol_task;        /* tau_task of Alg. 1 (on ||E_task||_inf) */
  double c_sm;            /* step threshold tau = max(c_sm ||q1-q0||_inf/(W-1), tau_floor) */
  double tau_floor;
  double tol_sm;          /* tau_sm of Alg. 1 (on max_k E_sm,k) */
  double alpha;           /* step size alpha of Alg. 1 */
  double lambda;          /* damping of the pseudoinverse J^+ */
  int max_iters;          /* max_iters of Alg. 1 */
  double line_y;          /* y of the line {y = line_y, z = target} (LINE, ORIENT_LINE) */
  double yaw;             /* end-effector yaw of the fixed orientation (ORIENT_*) */
} orc_constraint;

/* ---- kinematics ---------------------------------------------------------------------- */
/* frames[(dof+2)][16]: 4x4 transforms of frame 0 (identity) .. frame dof, then the EE. */
void orc_fk(const orc_robot* rb, const double* q, double* frames);
/* J[6][dof]: geometric Jacobian of the EE point, rows vx vy vz wx wy wz. */
void orc_jacobian(const orc_robot* rb, const double* q, double* J);
/* World centres of all robot spheres: out[S][3]. */
void orc_sphere_centres(const orc_robot* rb, const double* q, double* out);
/* Task error e[m] and task Jacobian Jt[m][dof]; returns m (0 for ORC_NONE). */
int orc_task(const orc_robot* rb, const orc_constraint* c, const double* q, double* e,
             double* Jt);
/* Damped pseudoinverse step g = J^T (J J^T + lambda^2 I)^-1 e, J is [m][dof]. */
void orc_damped_step(const double* J, const double* e, int m, int dof, double lambda,
                     double* g);

/* ---- Algorithm 1 ----------------------------------------------------------------------- */
/* Projects xi_init[W][dof] (waypoint 0 fixed). xi_out[W][dof] is the segment after the last
 * iteration. Returns 1 on success. iters = iteration at which the segment was accepted
 * (max_iters on failure); first_fail = first unaccepted waypoint (-1 on success);
 * resid = max over waypoints 1..W-1 of the last evaluated ||E_task||_inf;
 * margin = smallest distance of any acceptance decision taken from its threshold.
 * prog_trace[max_iters] (optional) records prog after each iteration. */
int orc_project_motion(const orc_robot* rb, const orc_constraint* c, const double* xi_init,
                       int W, double tau, double* xi_out, int* iters, int* first_fail,
                       double* resid, double* margin, int* prog_trace);

/* Single-configuration projection: repeated damped steps q <- clamp(q - alpha J^+ e) until
 * ||e||_inf < tol_task (tested before each step). Returns 1 on success. */
int orc_project_config(const orc_robot* rb, const orc_constraint* c, const double* q_in,
                       int max_iters, double* q_out, int* iters, double* resid);

/* Sequential ("naive", CBiRRT-style) motion projection, Sec. II / Fig. 1 upper: waypoint i
 * starts from its interpolated value shifted by the correction found for waypoint i-1 and
 * is projected alone; each step must stay within tau of its predecessor. */
int orc_project_motion_sequential(const orc_robot* rb, const orc_constraint* c,
                                  const double* xi_init, int W, double tau, double* xi_out,
                                  int* first_fail, int* total_iters);

/* ---- collision ------------------------------------------------------------------------- */
/* Signed clearance between a ball (centre p, radius r) and each primitive. < 0: collision. */
double orc_clear_sphere(const double* p, double r, const double* o);
double orc_clear_box(const double* p, double r, const double* b);
double orc_clear_capsule(const double* p, double r, const double* cp);
/* Min clearance of configuration q over all sphere x obstacle pairs. */
double orc_config_clearance(const orc_robot* rb, const orc_scene* sc, const double* q);

/* ---- motion validation (Sec. III + Alg. 1 + Sec. IV) ----------------------------------- */
/* q_start, q_end: [n][dof] FP32 inputs, promoted. out_q [n][W][dof]; status ORC_*;
 * first_fail (-1 if valid); iters; resid; proj_margin (Alg. 1 decisions, +inf if none);
 * cc_margin (smallest |clearance| of any pair that decides the CC verdict).
 * Any of the per-motion output pointers may be NULL. cc_skip_first: 1 skips waypoint 0. */
int orc_validate(const orc_robot* rb, const orc_scene* sc, const orc_constraint* c,
                 const float* q_start, const float* q_end, int n, int W, int cc_skip_first,
                 int n_threads, double* out_q, int* status, int* first_fail, int* iters,
                 double* resid, double* proj_margin, double* cc_margin);

/* Re-validation of a given segment xi[W][dof]: largest task error (waypoints 1..W-1),
 * largest step excess over tau, smallest clearance (all waypoints). */
void orc_check_segment(const orc_robot* rb, const orc_scene* sc, const orc_constraint* c,
                       const double* xi, int W, double tau, double* max_task,
                       double* max_step_excess, double* min_clearance);

/* Batch of orc_project_config calls over n_threads threads: q_in, q_out [n][dof] (FP32 in,
 * FP64 out), ok [n], resid [n] (either may be NULL). */
void orc_project_configs(const orc_robot* rb, const orc_constraint* c, const float* q_in, int n,
                         int max_iters, int n_threads, double* q_out, int* ok, double* resid);

/* ---- learned warm start network (no counterpart in the paper) --------------------------
 * f(q) = W4 g(W3 g(W2 g(W1 (q / pi) + b1) + b2) + b3) + b4, g(z) = z Phi(z) (exact GELU,
 * Phi the standard normal CDF), widths dof -> H -> H -> H -> dof. Parameters in the
 * compact layout: for l = 1..4, W_l [out_l][in_l] row-major then b_l [out_l]. */
long orc_mlp_param_count(int dof, int H);
/* corr [rows][dof] = f(q) for q [rows][dof]. */
void orc_mlp_forward(int dof, int H, const double* params, const double* q, int rows,
                     double* corr);
/* Loss (1/rows) sum_r 0.5 |f(q_r) - (t_r - q_r)|^2; grads (compact layout, may be NULL)
 * receives its gradient by reverse-mode differentiation written out layer by layer. */
double orc_mlp_loss_grad(int dof, int H, const double* params, const double* q,
                         const double* t, int rows, int n_threads, double* grads);

/* ---- counter-based RNG ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- RRT-Connect planner ------------------------------------------------------------------ */
typedef struct {
  double range;           /* steering step (L2, rad) */
  int W;                  /* waypoints per motion */
  int max_rounds;         /* rounds (extensions per worker) */
  int n_workers;          /* extensions attempted per round */
  int max_nodes;          /* per tree */
  int max_connect;        /* greedy connect steps per extension */
  uint32_t seed;
  uint32_t first_problem; /* problem p of a call draws with Philox problem index first_problem + p */
  int sequential;         /* 1: motions projected by orc_project_motion_sequential (the naive
                             baseline, R27) instead of Alg. 1 */
} orc_plan_params;

/* Plans each problem; path_len[p] = nodes in the path (0 on failure), path[p][max_path][dof],
 * rounds[p] = rounds used, waypoints[p] = waypoints validated. Returns number solved. */
int orc_plan(const orc_robot* rb, const orc_scene* sc, const orc_constraint* c,
             const float* start, const float* goal, int n_problems,
             const orc_plan_params* pp, int max_path, int n_threads, int* path_len,
             double* path, int* rounds, long long* waypoints);

#ifdef __cplusplus
}
#endif
#endif
