/*
 * FP64 CPU oracle for cpRRTC (Hu, Wang, Christensen): constrained motion validation and
 * RRT-Connect planning. TEST INFRASTRUCTURE ONLY; see cprrtc_oracle.h.
 *
 * Written for readability, not speed: plain 4x4 matrix products, one motion at a time,
 * every step in the order the paper states it. Readings of passages the paper leaves open
 * are marked "Reading:".
 */
#include "cprrtc_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ========================================================================================
 * Kinematics: standard Denavit-Hartenberg chain.
 * ======================================================================================== */

static void mat4_identity(double T[16]) {
  memset(T, 0, 16 * sizeof(double));
  T[0] = T[5] = T[10] = T[15] = 1.0;
}

static void mat4_mul(const double A[16], const double B[16], double C[16]) {
  double R[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += A[4 * i + k] * B[4 * k + j];
      R[4 * i + j] = s;
    }
  memcpy(C, R, sizeof(R));
}

/* T = Rz(theta) * Tz(d) * Tx(a) * Rx(alpha), built as the product of the four factors. */
static void dh_link(const double* jt, double q, double T[16]) {
  int prismatic = (int)jt[0] == 1;
  double theta = jt[4] + (prismatic ? 0.0 : q);
  double d = jt[1] + (prismatic ? q : 0.0);
  double a = jt[2], alpha = jt[3];
  double Rz[16], Tz[16], Tx[16], Rx[16], M[16];
  mat4_identity(Rz);
  Rz[0] = cos(theta); Rz[1] = -sin(theta);
  Rz[4] = sin(theta); Rz[5] = cos(theta);
  mat4_identity(Tz);
  Tz[11] = d;
  mat4_identity(Tx);
  Tx[3] = a;
  mat4_identity(Rx);
  Rx[5] = cos(alpha); Rx[6] = -sin(alpha);
  Rx[9] = sin(alpha); Rx[10] = cos(alpha);
  mat4_mul(Rz, Tz, M);
  mat4_mul(M, Tx, M);
  mat4_mul(M, Rx, T);
}

void orc_fk(const orc_robot* rb, const double* q, double* frames) {
  int n = rb->dof;
  mat4_identity(frames);
  for (int k = 0; k < n; ++k) {
    double Tk[16];
    dh_link(rb->joints + 7 * k, q[k], Tk);
    mat4_mul(frames + 16 * k, Tk, frames + 16 * (k + 1));
  }
  double Te[16];
  mat4_identity(Te);
  Te[3] = rb->ee[0]; Te[7] = rb->ee[1]; Te[11] = rb->ee[2];
  mat4_mul(frames + 16 * n, Te, frames + 16 * (n + 1));
}

/* Geometric Jacobian of the EE point. Column k belongs to joint k+1, whose axis is z of
 * frame k through the origin of frame k. */
void orc_jacobian(const orc_robot* rb, const double* q, double* J) {
  int n = rb->dof;
  double F[(ORC_MAX_DOF + 2) * 16];
  orc_fk(rb, q, F);
  const double* Fe = F + 16 * (n + 1);
  double pe[3] = {Fe[3], Fe[7], Fe[11]};
  for (int k = 0; k < n; ++k) {
    const double* Fk = F + 16 * k;
    double z[3] = {Fk[2], Fk[6], Fk[10]};
    double p[3] = {Fk[3], Fk[7], Fk[11]};
    double r[3] = {pe[0] - p[0], pe[1] - p[1], pe[2] - p[2]};
    if ((int)rb->joints[7 * k] == 1) { /* prismatic: linear velocity along the axis */
      J[0 * n + k] = z[0]; J[1 * n + k] = z[1]; J[2 * n + k] = z[2];
      J[3 * n + k] = 0.0;  J[4 * n + k] = 0.0;  J[5 * n + k] = 0.0;
    } else {                           /* revolute: v = z x (pe - p), w = z */
      J[0 * n + k] = z[1] * r[2] - z[2] * r[1];
      J[1 * n + k] = z[2] * r[0] - z[0] * r[2];
      J[2 * n + k] = z[0] * r[1] - z[1] * r[0];
      J[3 * n + k] = z[0]; J[4 * n + k] = z[1]; J[5 * n + k] = z[2];
    }
  }
}

void orc_sphere_centres(const orc_robot* rb, const double* q, double* out) {
  double F[(ORC_MAX_DOF + 2) * 16];
  orc_fk(rb, q, F);
  for (int s = 0; s < rb->n_spheres; ++s) {
    const double* sp = rb->spheres + 5 * s;
    const double* T = F + 16 * (int)sp[0];
    for (int r = 0; r < 3; ++r)
      out[3 * s + r] = T[4 * r + 0] * sp[1] + T[4 * r + 1] * sp[2] + T[4 * r + 2] * sp[3] +
                       T[4 * r + 3];
  }
}

/* ========================================================================================
 * Task constraints: GetTaskError / GetTaskJacobian of Alg. 1.
 *
 * Reading: the paper names the two functions without defining them. Its constraints hold
 * end-effector axes fixed (orientation, plane, line; Sec. V-B). Two are implemented:
 *  - ORC_ROLL_PITCH: with ZYX Euler angles (yaw psi, pitch theta, roll phi) of the EE
 *    rotation R, e = [phi, theta]; the manifold is {R = Rz(psi)}.
 *    J_task = E(psi, theta) J_w, where E maps world angular velocity to Euler rates:
 *    phi_dot = (c_psi w_x + s_psi w_y) / c_theta,  theta_dot = -s_psi w_x + c_psi w_y.
 *  - ORC_Z_PLANE: e = p_z - target, J_task = row z of J_v.
 * The paper's other variants (Sec. V-B: a line; a fixed orientation with a plane or a line):
 *  - ORC_LINE: the EE point on the line {y = line_y, z = target}: e = [p_y - line_y,
 *    p_z - target], J_task = rows y and z of J_v.
 *  - ORC_ORIENT_PLANE / ORC_ORIENT_LINE: the orientation fixed at roll = pitch = 0 and
 *    yaw = c->yaw, with the plane or the line: e = [phi, theta, psi - yaw (wrapped into
 *    (-pi, pi]), position rows]. The yaw rate of ZYX Euler angles is
 *    psi_dot = w_z + tan(theta) (c_psi w_x + s_psi w_y), from w = psi_dot z +
 *    theta_dot Rz(psi) y + phi_dot Rz(psi) Ry(theta) x.
 * ======================================================================================== */

int orc_task(const orc_robot* rb, const orc_constraint* c, const double* q, double* e,
             double* Jt) {
  int n = rb->dof;
  if (c->type == ORC_NONE) return 0;
  double F[(ORC_MAX_DOF + 2) * 16];
  double J[6 * ORC_MAX_DOF];
  orc_fk(rb, q, F);
  orc_jacobian(rb, q, J);
  const double* Fe = F + 16 * (n + 1);
  if (c->type == ORC_Z_PLANE) {
    e[0] = Fe[11] - c->target;
    for (int k = 0; k < n; ++k) Jt[k] = J[2 * n + k];
    return 1;
  }
  if (c->type == ORC_LINE) {
    e[0] = Fe[7] - c->line_y;
    e[1] = Fe[11] - c->target;
    for (int k = 0; k < n; ++k) {
      Jt[0 * n + k] = J[1 * n + k];
      Jt[1 * n + k] = J[2 * n + k];
    }
    return 2;
  }
  /* ORC_ROLL_PITCH and the fixed orientations */
  double R11 = Fe[0], R21 = Fe[4], R31 = Fe[8], R32 = Fe[9], R33 = Fe[10];
  double roll = atan2(R32, R33);
  double pitch = atan2(-R31, sqrt(R32 * R32 + R33 * R33));
  double yaw = atan2(R21, R11);
  e[0] = roll;
  e[1] = pitch;
  double cy = cos(yaw), sy = sin(yaw), cp = cos(pitch), tp = tan(pitch);
  for (int k = 0; k < n; ++k) {
    double wx = J[3 * n + k], wy = J[4 * n + k];
    Jt[0 * n + k] = (cy * wx + sy * wy) / cp;
    Jt[1 * n + k] = -sy * wx + cy * wy;
  }
  if (c->type == ORC_ROLL_PITCH) return 2;
  double dyaw = yaw - c->yaw;
  const double pi = 3.14159265358979323846;
  while (dyaw > pi) dyaw -= 2.0 * pi;
  while (dyaw <= -pi) dyaw += 2.0 * pi;
  e[2] = dyaw;
  for (int k = 0; k < n; ++k)
    Jt[2 * n + k] = J[5 * n + k] + tp * (cy * J[3 * n + k] + sy * J[4 * n + k]);
  if (c->type == ORC_ORIENT_PLANE) {
    e[3] = Fe[11] - c->target;
    for (int k = 0; k < n; ++k) Jt[3 * n + k] = J[2 * n + k];
    return 4;
  }
  /* ORC_ORIENT_LINE */
  e[3] = Fe[7] - c->line_y;
  e[4] = Fe[11] - c->target;
  for (int k = 0; k < n; ++k) {
    Jt[3 * n + k] = J[1 * n + k];
    Jt[4 * n + k] = J[2 * n + k];
  }
  return 5;
}

/* Solves A x = b (m x m, m <= 6) by Gaussian elimination with partial pivoting. */
static void solve_small(double* A, double* b, int m) {
  for (int col = 0; col < m; ++col) {
    int piv = col;
    for (int r = col + 1; r < m; ++r)
      if (fabs(A[r * m + col]) > fabs(A[piv * m + col])) piv = r;
    if (piv != col) {
      for (int k = 0; k < m; ++k) {
        double t = A[col * m + k]; A[col * m + k] = A[piv * m + k]; A[piv * m + k] = t;
      }
      double t = b[col]; b[col] = b[piv]; b[piv] = t;
    }
    for (int r = col + 1; r < m; ++r) {
      double f = A[r * m + col] / A[col * m + col];
      for (int k = col; k < m; ++k) A[r * m + k] -= f * A[col * m + k];
      b[r] -= f * b[col];
    }
  }
  for (int r = m - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < m; ++k) s -= A[r * m + k] * b[k];
    b[r] = s / A[r * m + r];
  }
}

/* Reading: J^+ of Alg. 1 is the damped pseudoinverse J^T (J J^T + lambda^2 I)^-1. */
void orc_damped_step(const double* J, const double* e, int m, int dof, double lambda,
                     double* g) {
  double A[36], y[6];
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int k = 0; k < dof; ++k) s += J[i * dof + k] * J[j * dof + k];
      A[i * m + j] = s + (i == j ? lambda * lambda : 0.0);
    }
    y[i] = e[i];
  }
  solve_small(A, y, m);
  for (int k = 0; k < dof; ++k) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += J[i * dof + k] * y[i];
    g[k] = s;
  }
}

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

static double norm_inf(const double* v, int n) {
  double m = 0.0;
  for (int i = 0; i < n; ++i) m = fmax(m, fabs(v[i]));
  return m;
}

/* ========================================================================================
 * Algorithm 1, ParallelProject (Sec. III-A).
 *
 * Readings (the listing is terse):
 *  - prog is the index of the last accepted waypoint; q0 (index 0) is accepted from the
 *    start, so prog starts at 0 and waypoints prog+1 .. W-1 are worked on.
 *  - Acceptance advances prog over the contiguous run of valid waypoints after it, stopping
 *    at the first invalid one, so that accepted waypoints are never left with a moving
 *    predecessor ("left unchanged in subsequent iterations", Sec. III-A).
 *  - Success when prog = W-1; the segment returned is the one just validated. Otherwise
 *    xi <- xi_new for the waypoints after prog only.
 *  - E_sm,k = max(0, |xi_k[i] - xi_k[i-1]| - tau) per joint (a hinge: waypoints closer than
 *    tau are not pushed apart), grad_sm,k = (xi_k[i] - xi_k[i-1]) * E_sm,k.
 *  - valid[i] = ||E_task||_inf < tau_task and max_k E_sm,k < tau_sm, both at the current xi.
 *  - xi_new[i] is clamped to the joint limits.
 * ======================================================================================== */
int orc_project_motion(const orc_robot* rb, const orc_constraint* c, const double* xi_init,
                       int W, double tau, double* xi_out, int* iters, int* first_fail,
                       double* resid, double* margin, int* prog_trace) {
  const int n = rb->dof;
  double* xi = xi_out;                       /* shared memory xi = xi_init */
  double xi_new[ORC_MAX_W * ORC_MAX_DOF];
  int valid[ORC_MAX_W];                      /* shared memory valid */
  double last_err[ORC_MAX_W];
  int prog = 0;                              /* shared memory prog */
  double mg = INFINITY;
  memcpy(xi, xi_init, sizeof(double) * W * n);
  memset(last_err, 0, sizeof(last_err));

  for (int it = 1; it <= c->max_iters; ++it) {
    /* Stage 1: every waypoint after prog computes its update and its validity. */
    for (int i = prog + 1; i < W; ++i) {
      double e[6], Jt[6 * ORC_MAX_DOF], g_task[ORC_MAX_DOF];
      int m = orc_task(rb, c, xi + i * n, e, Jt);
      orc_damped_step(Jt, e, m, n, c->lambda, g_task);
      double e_sm_max = 0.0;
      for (int k = 0; k < n; ++k) {
        double dk = xi[i * n + k] - xi[(i - 1) * n + k];
        double e_sm = fmax(0.0, fabs(dk) - tau);
        double g_sm = dk * e_sm;
        const double* jt = rb->joints + 7 * k;
        xi_new[i * n + k] = clampd(xi[i * n + k] - c->alpha * (g_task[k] + g_sm), jt[5], jt[6]);
        e_sm_max = fmax(e_sm_max, e_sm);
      }
      double e_task = norm_inf(e, m);
      valid[i] = (e_sm_max < c->tol_sm) && (e_task < c->tol_task);
      last_err[i] = e_task;
      mg = fmin(mg, fabs(e_task - c->tol_task));
      mg = fmin(mg, fabs(e_sm_max - c->tol_sm));
    }
    /* Stage 2: advance prog over the contiguous valid run; accept or commit xi_new. */
    int j = prog + 1;
    while (j < W && valid[j]) {
      prog = j;
      ++j;
    }
    if (prog_trace) prog_trace[it - 1] = prog;
    if (prog == W - 1) {
      *iters = it;
      *first_fail = -1;
      *resid = norm_inf(last_err + 1, W - 1);
      *margin = mg;
      return 1;
    }
    for (int i = prog + 1; i < W; ++i)
      for (int k = 0; k < n; ++k) xi[i * n + k] = xi_new[i * n + k];
  }
  *iters = c->max_iters;
  *first_fail = prog + 1;
  *resid = norm_inf(last_err + 1, W - 1);
  *margin = mg;
  return 0;
}

int orc_project_config(const orc_robot* rb, const orc_constraint* c, const double* q_in,
                       int max_iters, double* q_out, int* iters, double* resid) {
  const int n = rb->dof;
  memcpy(q_out, q_in, sizeof(double) * n);
  double e[6], Jt[6 * ORC_MAX_DOF], g[ORC_MAX_DOF];
  for (int it = 0; it <= max_iters; ++it) {
    int m = orc_task(rb, c, q_out, e, Jt);
    double err = norm_inf(e, m);
    if (err < c->tol_task) {
      *iters = it;
      *resid = err;
      return 1;
    }
    if (it == max_iters) {
      *iters = it;
      *resid = err;
      return 0;
    }
    orc_damped_step(Jt, e, m, n, c->lambda, g);
    for (int k = 0; k < n; ++k) {
      const double* jt = rb->joints + 7 * k;
      q_out[k] = clampd(q_out[k] - c->alpha * g[k], jt[5], jt[6]);
    }
  }
  return 0;
}

int orc_project_motion_sequential(const orc_robot* rb, const orc_constraint* c,
                                  const double* xi_init, int W, double tau, double* xi_out,
                                  int* first_fail, int* total_iters) {
  const int n = rb->dof;
  memcpy(xi_out, xi_init, sizeof(double) * n);
  int total = 0;
  for (int i = 1; i < W; ++i) {
    /* start from the interpolated point carried along by the previous correction */
    double start[ORC_MAX_DOF];
    for (int k = 0; k < n; ++k) {
      const double* jt = rb->joints + 7 * k;
      start[k] = clampd(xi_init[i * n + k] + (xi_out[(i - 1) * n + k] - xi_init[(i - 1) * n + k]),
                        jt[5], jt[6]);
    }
    int it = 0;
    double res = 0.0;
    int ok = orc_project_config(rb, c, start, c->max_iters, xi_out + i * n, &it, &res);
    total += it;
    double step = 0.0;
    for (int k = 0; k < n; ++k)
      step = fmax(step, fabs(xi_out[i * n + k] - xi_out[(i - 1) * n + k]) - tau);
    if (!ok || step >= c->tol_sm) {
      *first_fail = i;
      *total_iters = total;
      return 0;
    }
  }
  *first_fail = -1;
  *total_iters = total;
  return 1;
}

/* ========================================================================================
 * Collision checking: signed clearance of a ball against each primitive.
 * ======================================================================================== */

double orc_clear_sphere(const double* p, double r, const double* o) {
  double dx = p[0] - o[0], dy = p[1] - o[1], dz = p[2] - o[2];
  return sqrt(dx * dx + dy * dy + dz * dz) - (r + o[3]);
}

/* Box {c, h, R}: the point in box coordinates is R^T (p - c). Outside: distance to the
 * closest point of the solid box; inside: minus the distance to the nearest face. */
double orc_clear_box(const double* p, double r, const double* b) {
  const double* R = b + 6;
  double d[3] = {p[0] - b[0], p[1] - b[1], p[2] - b[2]};
  double l[3];
  for (int i = 0; i < 3; ++i) l[i] = R[0 + i] * d[0] + R[3 + i] * d[1] + R[6 + i] * d[2];
  double out2 = 0.0, inside_gap = INFINITY;
  int inside = 1;
  for (int i = 0; i < 3; ++i) {
    double h = b[3 + i];
    double ex = fabs(l[i]) - h;
    if (ex > 0.0) {
      out2 += ex * ex;
      inside = 0;
    }
    inside_gap = fmin(inside_gap, h - fabs(l[i]));
  }
  if (inside) return -inside_gap - r;
  return sqrt(out2) - r;
}

/* Capsule {p0, p1, rc}: distance to the segment minus both radii. */
double orc_clear_capsule(const double* p, double r, const double* cp) {
  double u[3] = {cp[3] - cp[0], cp[4] - cp[1], cp[5] - cp[2]};
  double w[3] = {p[0] - cp[0], p[1] - cp[1], p[2] - cp[2]};
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double t = uu > 0.0 ? (w[0] * u[0] + w[1] * u[1] + w[2] * u[2]) / uu : 0.0;
  t = clampd(t, 0.0, 1.0);
  double dx = w[0] - t * u[0], dy = w[1] - t * u[1], dz = w[2] - t * u[2];
  return sqrt(dx * dx + dy * dy + dz * dz) - (r + cp[6]);
}

/* Min clearance of one configuration over every sphere x obstacle pair, and, when the robot
 * names frame pairs for self-collision, over every pair of its spheres on such frames
 * (distance of the centres minus both radii). */
static double config_clearance(const orc_robot* rb, const orc_scene* sc, const double* q,
                               double* centres) {
  orc_sphere_centres(rb, q, centres);
  double best = INFINITY;
  for (int s = 0; s < rb->n_spheres; ++s) {
    const double* p = centres + 3 * s;
    double r = rb->spheres[5 * s + 4];
    for (int o = 0; o < sc->n_sph; ++o) best = fmin(best, orc_clear_sphere(p, r, sc->sph + 4 * o));
    for (int o = 0; o < sc->n_box; ++o) best = fmin(best, orc_clear_box(p, r, sc->box + 15 * o));
    for (int o = 0; o < sc->n_cap; ++o) best = fmin(best, orc_clear_capsule(p, r, sc->cap + 7 * o));
  }
  if (rb->self_pairs) {
    const int nf = rb->dof + 1;
    for (int s = 0; s < rb->n_spheres; ++s) {
      const int fs = (int)rb->spheres[5 * s];
      for (int t = s + 1; t < rb->n_spheres; ++t) {
        const int ft = (int)rb->spheres[5 * t];
        if (fs == ft || !rb->self_pairs[fs * nf + ft]) continue;
        const double* a = centres + 3 * s;
        const double* b = centres + 3 * t;
        double d[3] = {a[0] - b[0], a[1] - b[1], a[2] - b[2]};
        best = fmin(best, sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) -
                              (rb->spheres[5 * s + 4] + rb->spheres[5 * t + 4]));
      }
    }
  }
  return best;
}

double orc_config_clearance(const orc_robot* rb, const orc_scene* sc, const double* q) {
  double* centres = (double*)malloc(sizeof(double) * 3 * (rb->n_spheres + 1));
  double v = config_clearance(rb, sc, q, centres);
  free(centres);
  return v;
}

/* ========================================================================================
 * Motion validation (Sec. III): interpolate, project (Alg. 1), then FK + CC per waypoint.
 * Sec. IV: the motion is invalid at its first colliding waypoint; the verdict and that
 * index do not depend on when other waypoints stop.
 * ======================================================================================== */

static double step_threshold(const orc_constraint* c, const double* q0, const double* q1,
                             int n, int W) {
  /* Reading: tau ("a predefined threshold", Sec. III-A) scales with the nominal spacing. */
  double span = 0.0;
  for (int k = 0; k < n; ++k) span = fmax(span, fabs(q1[k] - q0[k]));
  return fmax(c->c_sm * span / (double)(W - 1), c->tau_floor);
}

typedef struct {
  int status, first_fail, iters;
  double resid, proj_margin, cc_margin;
} motion_result;

static motion_result validate_one(const orc_robot* rb, const orc_scene* sc,
                                  const orc_constraint* c, const double* q0, const double* q1,
                                  int W, int cc_skip_first, double* xi, double* centres,
                                  int sequential) {
  const int n = rb->dof;
  motion_result res = {ORC_VALID, -1, 0, 0.0, INFINITY, INFINITY};
  double xi_init[ORC_MAX_W * ORC_MAX_DOF];
  for (int i = 0; i < W; ++i) {
    double t = (double)i / (double)(W - 1);
    for (int k = 0; k < n; ++k) xi_init[i * n + k] = q0[k] + t * (q1[k] - q0[k]);
  }
  if (c->type == ORC_NONE) {
    memcpy(xi, xi_init, sizeof(double) * W * n);
  } else {
    double tau = step_threshold(c, q0, q1, n, W);
    int ok = sequential
                 ? orc_project_motion_sequential(rb, c, xi_init, W, tau, xi, &res.first_fail, &res.iters)
                 : orc_project_motion(rb, c, xi_init, W, tau, xi, &res.iters, &res.first_fail,
                                      &res.resid, &res.proj_margin, NULL);
    if (!ok) {
      res.status = ORC_PROJ_FAIL;
      return res;
    }
  }
  /* FK + CC, waypoints in order; the first colliding waypoint decides. */
  double mg = INFINITY;
  for (int i = cc_skip_first ? 1 : 0; i < W; ++i) {
    double cl = config_clearance(rb, sc, xi + i * n, centres);
    if (cl < 0.0) {
      res.status = ORC_COLLISION;
      res.first_fail = i;
      mg = fmin(mg, -cl);
      break;
    }
    mg = fmin(mg, cl);
  }
  res.cc_margin = mg;
  return res;
}

typedef struct {
  const orc_robot* rb;
  const orc_scene* sc;
  const orc_constraint* c;
  const float *q_start, *q_end;
  int W, cc_skip_first, lo, hi;
  double* out_q;
  int *status, *first_fail, *iters;
  double *resid, *proj_margin, *cc_margin;
} validate_job;

static void* validate_worker(void* arg) {
  validate_job* jb = (validate_job*)arg;
  const int n = jb->rb->dof, W = jb->W;
  double xi[ORC_MAX_W * ORC_MAX_DOF];
  double* centres = (double*)malloc(sizeof(double) * 3 * (jb->rb->n_spheres + 1));
  for (int m = jb->lo; m < jb->hi; ++m) {
    double q0[ORC_MAX_DOF], q1[ORC_MAX_DOF];
    for (int k = 0; k < n; ++k) {
      q0[k] = (double)jb->q_start[m * n + k];
      q1[k] = (double)jb->q_end[m * n + k];
    }
    motion_result r = validate_one(jb->rb, jb->sc, jb->c, q0, q1, W, jb->cc_skip_first, xi,
                                   centres, 0);
    if (jb->out_q) memcpy(jb->out_q + (size_t)m * W * n, xi, sizeof(double) * W * n);
    if (jb->status) jb->status[m] = r.status;
    if (jb->first_fail) jb->first_fail[m] = r.first_fail;
    if (jb->iters) jb->iters[m] = r.iters;
    if (jb->resid) jb->resid[m] = r.resid;
    if (jb->proj_margin) jb->proj_margin[m] = r.proj_margin;
    if (jb->cc_margin) jb->cc_margin[m] = r.cc_margin;
  }
  free(centres);
  return NULL;
}

int orc_validate(const orc_robot* rb, const orc_scene* sc, const orc_constraint* c,
                 const float* q_start, const float* q_end, int n, int W, int cc_skip_first,
                 int n_threads, double* out_q, int* status, int* first_fail, int* iters,
                 double* resid, double* proj_margin, double* cc_margin) {
  if (rb->dof < 1 || rb->dof > ORC_MAX_DOF || W < 2 || W > ORC_MAX_W || n < 0) return -1;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n) n_threads = n > 0 ? n : 1;
  pthread_t th[256];
  validate_job jobs[256];
  if (n_threads > 256) n_threads = 256;
  for (int t = 0; t < n_threads; ++t) {
    validate_job jb = {rb, sc, c, q_start, q_end, W, cc_skip_first,
                       (int)((long long)n * t / n_threads),
                       (int)((long long)n * (t + 1) / n_threads),
                       out_q, status, first_fail, iters, resid, proj_margin, cc_margin};
    jobs[t] = jb;
  }
  if (n_threads == 1) {
    validate_worker(&jobs[0]);
    return 0;
  }
  for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, validate_worker, &jobs[t]);
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  return 0;
}

/* ========================================================================================
 * Batch single-configuration projection (orc_project_config over threads).
 * ======================================================================================== */

typedef struct {
  const orc_robot* rb;
  const orc_constraint* c;
  const float* q_in;
  int lo, hi, max_iters;
  double* q_out;
  int* ok;
  double* resid;
} proj_job;

static void* project_worker(void* arg) {
  proj_job* j = (proj_job*)arg;
  const int n = j->rb->dof;
  for (int m = j->lo; m < j->hi; ++m) {
    double q[ORC_MAX_DOF];
    for (int k = 0; k < n; ++k) q[k] = (double)j->q_in[(size_t)m * n + k];
    int it = 0;
    double res = 0.0;
    int ok = orc_project_config(j->rb, j->c, q, j->max_iters, j->q_out + (size_t)m * n, &it, &res);
    if (j->ok) j->ok[m] = ok;
    if (j->resid) j->resid[m] = res;
  }
  return NULL;
}

void orc_project_configs(const orc_robot* rb, const orc_constraint* c, const float* q_in, int n,
                         int max_iters, int n_threads, double* q_out, int* ok, double* resid) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  proj_job jobs[256];
  for (int t = 0; t < n_threads; ++t) {
    jobs[t] = (proj_job){rb, c, q_in, (int)((long)n * t / n_threads),
                         (int)((long)n * (t + 1) / n_threads), max_iters, q_out, ok, resid};
    pthread_create(&th[t], NULL, project_worker, &jobs[t]);
  }
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
}

/* ========================================================================================
 * Learned warm start network: a plain FP64 multilayer perceptron, forward pass and
 * reverse-mode gradient of the mean squared correction error, one row at a time.
 * ======================================================================================== */

static void mlp_dims(int dof, int H, int l, int* out, int* in) {
  *in = l == 0 ? dof : H;
  *out = l == 3 ? dof : H;
}

long orc_mlp_param_count(int dof, int H) {
  long n = 0;
  for (int l = 0; l < 4; ++l) {
    int o, i;
    mlp_dims(dof, H, l, &o, &i);
    n += (long)o * i + o;
  }
  return n;
}

static long mlp_layer_off(int dof, int H, int l) {
  long off = 0;
  for (int k = 0; k < l; ++k) {
    int o, i;
    mlp_dims(dof, H, k, &o, &i);
    off += (long)o * i + o;
  }
  return off;
}

static const double kPi = 3.14159265358979323846;

static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }
/* d/dz of z Phi(z): Phi(z) + z phi(z) */
static double gelu_d(double z) {
  return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * exp(-0.5 * z * z) / sqrt(2.0 * kPi);
}

/* One row: a[l] = input of layer l (l = 0..3, stride H), z[l] = pre-activation of hidden
 * layer l (l = 0..2, stride H), y = output. */
static void mlp_row(int dof, int H, const double* params, const double* q, double* a, double* z,
                    double* y) {
  for (int k = 0; k < dof; ++k) a[k] = q[k] / kPi;
  for (int l = 0; l < 4; ++l) {
    int o, in;
    mlp_dims(dof, H, l, &o, &in);
    const double* Wl = params + mlp_layer_off(dof, H, l);
    const double* bl = Wl + (long)o * in;
    const double* x = a + (long)l * H;
    for (int r = 0; r < o; ++r) {
      double s = bl[r];
      for (int c = 0; c < in; ++c) s += Wl[(long)r * in + c] * x[c];
      if (l < 3) {
        z[(long)l * H + r] = s;
        a[(long)(l + 1) * H + r] = gelu(s);
      } else {
        y[r] = s;
      }
    }
  }
}

void orc_mlp_forward(int dof, int H, const double* params, const double* q, int rows,
                     double* corr) {
  double* a = (double*)malloc(sizeof(double) * 4 * (size_t)H);
  double* z = (double*)malloc(sizeof(double) * 3 * (size_t)H);
  for (int r = 0; r < rows; ++r)
    mlp_row(dof, H, params, q + (size_t)r * dof, a, z, corr + (size_t)r * dof);
  free(a);
  free(z);
}

typedef struct {
  int dof, H, lo, hi, rows;
  const double *params, *q, *t;
  double* grads; /* this thread's accumulator (compact layout) or NULL */
  double loss;
} mlp_job;

static void* mlp_worker(void* arg) {
  mlp_job* j = (mlp_job*)arg;
  const int dof = j->dof, H = j->H;
  const int wide = H > dof ? H : dof;
  double* a = (double*)malloc(sizeof(double) * 4 * (size_t)H);
  double* z = (double*)malloc(sizeof(double) * 3 * (size_t)H);
  double* d = (double*)malloc(sizeof(double) * (size_t)wide);  /* dL/d(output of layer l) */
  double* dn = (double*)malloc(sizeof(double) * (size_t)wide);
  double y[ORC_MAX_DOF];
  j->loss = 0.0;
  for (int r = j->lo; r < j->hi; ++r) {
    const double* q = j->q + (size_t)r * dof;
    const double* t = j->t + (size_t)r * dof;
    mlp_row(dof, H, j->params, q, a, z, y);
    /* error of the predicted correction; dL/dy = error / rows */
    for (int k = 0; k < dof; ++k) {
      const double res = y[k] - (t[k] - q[k]);
      j->loss += 0.5 * res * res / j->rows;
      d[k] = res / j->rows;
    }
    if (!j->grads) continue;
    for (int l = 3; l >= 0; --l) {
      int o, in;
      mlp_dims(dof, H, l, &o, &in);
      const long off = mlp_layer_off(dof, H, l);
      const double* Wl = j->params + off;
      double* gW = j->grads + off;
      double* gb = gW + (long)o * in;
      const double* x = a + (long)l * H;
      for (int rr = 0; rr < o; ++rr) {
        gb[rr] += d[rr];
        for (int c = 0; c < in; ++c) gW[(long)rr * in + c] += d[rr] * x[c];
      }
      if (l == 0) break;
      /* back through W_l, then through the GELU of hidden layer l-1 */
      for (int c = 0; c < in; ++c) {
        double s = 0.0;
        for (int rr = 0; rr < o; ++rr) s += Wl[(long)rr * in + c] * d[rr];
        dn[c] = s * gelu_d(z[(long)(l - 1) * H + c]);
      }
      memcpy(d, dn, sizeof(double) * (size_t)in);
    }
  }
  free(a);
  free(z);
  free(d);
  free(dn);
  return NULL;
}

double orc_mlp_loss_grad(int dof, int H, const double* params, const double* q,
                         const double* t, int rows, int n_threads, double* grads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 64) n_threads = 64;
  if (n_threads > rows) n_threads = rows > 0 ? rows : 1;
  const long np = orc_mlp_param_count(dof, H);
  pthread_t th[64];
  mlp_job jobs[64];
  for (int k = 0; k < n_threads; ++k) {
    jobs[k] = (mlp_job){dof, H, (int)((long)rows * k / n_threads),
                        (int)((long)rows * (k + 1) / n_threads), rows, params, q, t,
                        grads ? (double*)calloc((size_t)np, sizeof(double)) : NULL, 0.0};
    pthread_create(&th[k], NULL, mlp_worker, &jobs[k]);
  }
  double loss = 0.0;
  if (grads) memset(grads, 0, sizeof(double) * (size_t)np);
  for (int k = 0; k < n_threads; ++k) {
    pthread_join(th[k], NULL);
    loss += jobs[k].loss;
    if (grads) {
      for (long i = 0; i < np; ++i) grads[i] += jobs[k].grads[i];
      free(jobs[k].grads);
    }
  }
  return loss;
}

/* ========================================================================================
 * Philox4x32-10, from the definition in Salmon et al., "Parallel random numbers: as easy
 * as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplications with the key added by
 * XOR and bumped by two Weyl constants between rounds.
 * ======================================================================================== */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * x0;
    uint64_t p1 = (uint64_t)M1 * x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ========================================================================================
 * RRT-Connect (Sec. II, Sec. III): extend one tree toward a random sample, then greedily
 * extend the same tree from the new node toward its nearest node in the other tree.
 *
 * Round structure (reading; the paper runs many extensions at once, one per thread block):
 * n_workers workers each validate one motion per round, against the trees as they stood
 * when the round began. Each worker carries a chain across rounds:
 *   - EXTEND: tree a = (round + w) mod 2; a sample from Philox4x32-10 with counter
 *     {problem, round, w, draw} and key {seed, 0} (each 32-bit output x gives
 *     u = (x >> 8) * 2^-24, q_k = lo_k + u_k (hi_k - lo_k)); q_near = nearest node (L2, lowest
 *     index on ties); q_steer = q_near moved toward the sample by at most `range` (L2); the
 *     motion q_near -> q_steer is validated with waypoint 0 skipped. A valid end q_end (the
 *     end is free under projection) becomes a node with parent q_near, and the chain's
 *     target becomes the nearest node of the other tree.
 *   - CONNECT: steer from the chain's last node toward the target; the projected end becomes
 *     a node only if the motion is valid and the end is strictly closer (L2) to the target.
 *   - HOP: once the last node is within 10 * tau_floor (inf-norm) of the target, the closing
 *     motion must be valid as it stands (Alg. 1 with one iteration, then CC); then the trees
 *     are connected.
 *   After a new node the chain continues with HOP if in reach, else CONNECT (at most
 *   max_connect CONNECT motions per chain); a rejected motion returns the worker to EXTEND.
 * The nodes of a round are appended in worker order (dropped beyond max_nodes, which ends
 * that chain), and the lowest worker that connected ends the problem.
 * ======================================================================================== */

typedef struct {
  double* nodes;   /* [max_nodes][dof] */
  int* parent;
  int count;
} orc_tree;

static void sample_config(const orc_robot* rb, uint32_t problem, uint32_t round,
                          uint32_t worker, uint32_t seed, double* q) {
  uint32_t key[2] = {seed, 0u};
  uint32_t u32[8];
  for (uint32_t draw = 0; draw < 2; ++draw) {
    uint32_t ctr[4] = {problem, round, worker, draw};
    orc_philox4x32_10(ctr, key, u32 + 4 * draw);
  }
  for (int k = 0; k < rb->dof; ++k) {
    double u = (double)(u32[k] >> 8) * (1.0 / 16777216.0);
    const double* jt = rb->joints + 7 * k;
    q[k] = jt[5] + u * (jt[6] - jt[5]);
  }
}

static int nearest(const orc_tree* t, int count, const double* q, int n) {
  int best = 0;
  double bd = INFINITY;
  for (int i = 0; i < count; ++i) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
      double d = t->nodes[i * n + k] - q[k];
      s += d * d;
    }
    if (s < bd) {
      bd = s;
      best = i;
    }
  }
  return best;
}

static double dist2(const double* a, const double* b, int n) {
  double s = 0.0;
  for (int k = 0; k < n; ++k) s += (a[k] - b[k]) * (a[k] - b[k]);
  return sqrt(s);
}

static void steer(const double* from, const double* to, double range, int n, double* out) {
  double d = dist2(from, to, n);
  double f = d > range ? range / d : 1.0;
  for (int k = 0; k < n; ++k) out[k] = from[k] + f * (to[k] - from[k]);
}

typedef struct {
  const orc_robot* rb;
  const orc_scene* sc;
  const orc_constraint* c;
  const orc_plan_params* pp;
} plan_env;

/* Validates q0 -> q1 (waypoint 0 skipped); on success copies the motion's end to q_end. */
static int motion_ok(const plan_env* env, const orc_constraint* c, const double* q0,
                     const double* q1, double* q_end, double* xi, double* centres,
                     long long* wp) {
  int n = env->rb->dof, W = env->pp->W;
  motion_result r = validate_one(env->rb, env->sc, c, q0, q1, W, 1, xi, centres, env->pp->sequential);
  *wp += W;
  if (r.status != ORC_VALID) return 0;
  memcpy(q_end, xi + (W - 1) * n, sizeof(double) * n);
  return 1;
}

typedef struct {
  int mode;          /* 0 EXTEND, 1 CONNECT, 2 HOP */
  int tree, last, target, steps;
  double cur[ORC_MAX_DOF], qt[ORC_MAX_DOF];
  /* this round */
  int add, conn;
  double qe[ORC_MAX_DOF];
} worker_state;

static int plan_one(const plan_env* env, const double* start, const double* goal,
                    uint32_t problem, int max_path, double* path, int* rounds_used,
                    long long* waypoints) {
  const int n = env->rb->dof;
  const orc_plan_params* pp = env->pp;
  const int cap = pp->max_nodes;
  orc_tree T[2];
  for (int t = 0; t < 2; ++t) {
    T[t].nodes = (double*)malloc(sizeof(double) * cap * n);
    T[t].parent = (int*)malloc(sizeof(int) * cap);
    T[t].count = 1;
    T[t].parent[0] = -1;
  }
  memcpy(T[0].nodes, start, sizeof(double) * n);
  memcpy(T[1].nodes, goal, sizeof(double) * n);
  worker_state* ws = (worker_state*)calloc(pp->n_workers, sizeof(worker_state));
  double xi[ORC_MAX_W * ORC_MAX_DOF];
  double* centres = (double*)malloc(sizeof(double) * 3 * (env->rb->n_spheres + 1));
  orc_constraint hop = *env->c;
  hop.max_iters = 1;
  const double connect_radius = 10.0 * env->c->tau_floor;
  long long wp = 0;
  int path_len = 0;

  for (int r = 0; r < pp->max_rounds; ++r) {
    const int count0[2] = {T[0].count, T[1].count};
    int win = -1;
    for (int w = 0; w < pp->n_workers; ++w) {
      worker_state* s = &ws[w];
      double q1[ORC_MAX_DOF];
      s->add = 0;
      s->conn = 0;
      if (s->mode == 0) {
        double q_rand[ORC_MAX_DOF];
        s->tree = (r + w) & 1;
        sample_config(env->rb, problem, (uint32_t)r, (uint32_t)w, pp->seed, q_rand);
        s->last = nearest(&T[s->tree], count0[s->tree], q_rand, n);
        memcpy(s->cur, T[s->tree].nodes + s->last * n, sizeof(double) * n);
        steer(s->cur, q_rand, pp->range, n, q1);
      } else if (s->mode == 1) {
        steer(s->cur, s->qt, pp->range, n, q1);
      } else {
        memcpy(q1, s->qt, sizeof(double) * n);
      }
      double q_end[ORC_MAX_DOF];
      if (!motion_ok(env, s->mode == 2 ? &hop : env->c, s->cur, q1, q_end, xi, centres, &wp))
        continue;
      if (s->mode == 2) {
        s->conn = 1;
        if (win < 0) win = w;
        continue;
      }
      int accept = 1;
      if (s->mode == 0) {
        const orc_tree* tb = &T[s->tree ^ 1];
        s->target = nearest(tb, count0[s->tree ^ 1], q_end, n);
        memcpy(s->qt, tb->nodes + s->target * n, sizeof(double) * n);
      } else {
        accept = dist2(q_end, s->qt, n) < dist2(s->cur, s->qt, n);
      }
      if (accept) {
        s->add = 1;
        memcpy(s->qe, q_end, sizeof(double) * n);
      }
    }
    *rounds_used = r + 1;
    if (win >= 0) {
      /* root_a .. last, target .. root_b; reversed when tree a is the goal tree */
      const worker_state* s = &ws[win];
      const int a = s->tree, b = a ^ 1;
      int len_a = 0, len_b = 0;
      for (int v = s->last; v >= 0; v = T[a].parent[v]) ++len_a;
      for (int v = s->target; v >= 0; v = T[b].parent[v]) ++len_b;
      const int total = len_a + len_b;
      if (total > max_path) {
        path_len = -total;
        break;
      }
      double* seq = (double*)malloc(sizeof(double) * total * n);
      int pos = len_a - 1;
      for (int v = s->last; v >= 0; v = T[a].parent[v], --pos)
        memcpy(seq + pos * n, T[a].nodes + v * n, sizeof(double) * n);
      pos = len_a;
      for (int v = s->target; v >= 0; v = T[b].parent[v], ++pos)
        memcpy(seq + pos * n, T[b].nodes + v * n, sizeof(double) * n);
      for (int j = 0; j < total; ++j) {
        const int src = (a == 0) ? j : total - 1 - j;
        memcpy(path + j * n, seq + src * n, sizeof(double) * n);
      }
      free(seq);
      path_len = total;
      break;
    }
    /* append this round's nodes in worker order; advance each chain */
    for (int w = 0; w < pp->n_workers; ++w) {
      worker_state* s = &ws[w];
      int stored = -1;
      if (s->add) {
        orc_tree* t = &T[s->tree];
        if (t->count < cap) {
          stored = t->count;
          memcpy(t->nodes + stored * n, s->qe, sizeof(double) * n);
          t->parent[stored] = s->last;
          t->count++;
        }
      }
      if (stored >= 0) {
        s->last = stored;
        memcpy(s->cur, s->qe, sizeof(double) * n);
        double gap = 0.0;
        for (int k = 0; k < n; ++k) gap = fmax(gap, fabs(s->cur[k] - s->qt[k]));
        if (gap <= connect_radius) {
          s->mode = 2;
        } else if (s->steps < pp->max_connect) {
          s->mode = 1;
          s->steps++;
        } else {
          s->mode = 0;
          s->steps = 0;
        }
      } else {
        s->mode = 0;
        s->steps = 0;
      }
    }
  }
  *waypoints = wp;
  for (int t = 0; t < 2; ++t) {
    free(T[t].nodes);
    free(T[t].parent);
  }
  free(ws);
  free(centres);
  return path_len;
}

typedef struct {
  const plan_env* env;
  const float *start, *goal;
  int lo, hi, max_path;
  int* path_len;
  double* path;
  int* rounds;
  long long* waypoints;
} plan_job;

static void* plan_worker(void* arg) {
  plan_job* jb = (plan_job*)arg;
  int n = jb->env->rb->dof;
  for (int p = jb->lo; p < jb->hi; ++p) {
    double s[ORC_MAX_DOF], g[ORC_MAX_DOF];
    for (int k = 0; k < n; ++k) {
      s[k] = (double)jb->start[p * n + k];
      g[k] = (double)jb->goal[p * n + k];
    }
    int rounds = 0;
    long long wp = 0;
    jb->path_len[p] = plan_one(jb->env, s, g, jb->env->pp->first_problem + (uint32_t)p, jb->max_path,
                               jb->path + (size_t)p * jb->max_path * n, &rounds, &wp);
    if (jb->rounds) jb->rounds[p] = rounds;
    if (jb->waypoints) jb->waypoints[p] = wp;
  }
  return NULL;
}

int orc_plan(const orc_robot* rb, const orc_scene* sc, const orc_constraint* c,
             const float* start, const float* goal, int n_problems,
             const orc_plan_params* pp, int max_path, int n_threads, int* path_len,
             double* path, int* rounds, long long* waypoints) {
  if (rb->dof < 1 || rb->dof > ORC_MAX_DOF || pp->W < 2 || pp->W > ORC_MAX_W) return -1;
  plan_env env = {rb, sc, c, pp};
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n_problems) n_threads = n_problems > 0 ? n_problems : 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  plan_job jobs[256];
  for (int t = 0; t < n_threads; ++t) {
    plan_job jb = {&env, start, goal,
                   (int)((long long)n_problems * t / n_threads),
                   (int)((long long)n_problems * (t + 1) / n_threads),
                   max_path, path_len, path, rounds, waypoints};
    jobs[t] = jb;
  }
  if (n_threads == 1) {
    plan_worker(&jobs[0]);
  } else {
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, plan_worker, &jobs[t]);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  }
  int solved = 0;
  for (int p = 0; p < n_problems; ++p) solved += path_len[p] > 0;
  return solved;
}

/* ========================================================================================
 * Checks of a given waypoint sequence (used to re-validate planner output): the largest
 * ||E_task||_inf over waypoints 1..W-1, the largest per-joint step excess
 * max_k |xi_k[i] - xi_k[i-1]| - tau, and the smallest clearance over waypoints.
 * ======================================================================================== */
void orc_check_segment(const orc_robot* rb, const orc_scene* sc, const orc_constraint* c,
                       const double* xi, int W, double tau, double* max_task,
                       double* max_step_excess, double* min_clearance) {
  const int n = rb->dof;
  double* centres = (double*)malloc(sizeof(double) * 3 * (rb->n_spheres + 1));
  double mt = 0.0, ms = -INFINITY, mc = INFINITY;
  for (int i = 0; i < W; ++i) {
    if (i > 0) {
      double e[6], Jt[6 * ORC_MAX_DOF];
      int m = orc_task(rb, c, xi + i * n, e, Jt);
      mt = fmax(mt, norm_inf(e, m));
      for (int k = 0; k < n; ++k) ms = fmax(ms, fabs(xi[i * n + k] - xi[(i - 1) * n + k]) - tau);
    }
    mc = fmin(mc, config_clearance(rb, sc, xi + i * n, centres));
  }
  free(centres);
  *max_task = mt;
  *max_step_excess = ms;
  *min_clearance = mc;
}
