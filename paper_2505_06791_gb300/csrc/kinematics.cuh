// Per-thread forward kinematics, task error and task Jacobian (GetTaskError /
// GetTaskJacobian of Alg. 1, Sec. III-A), and the damped pseudoinverse step, in FP32.
//
// The DH chain is advanced with the column form of T_k = Rz(theta) Tz(d) Tx(a) Rx(alpha):
// with the previous frame's axes x, y, z and origin p,
//   u = x cos(theta) + y sin(theta),  v = y cos(theta) - x sin(theta),
//   p' = p + a u + d z,  x' = u,  y' = v cos(alpha) + z sin(alpha),  z' = z cos(alpha) - v sin(alpha)
// (48 FLOP and one sincos per joint).
//
// The constraint type is a template parameter: per-joint quantities the task Jacobian does
// not read are dead code and take no registers. The Jacobian is not stored: its entries
// are linear in the stored joint axes and are recomputed where the damped step needs them.
#pragma once
#include "device_types.cuh"

namespace cprrtc {

// Floats stored per frame: axes x, y, z then origin p (columns of the 3x4 transform).
constexpr int kFrameFloats = 12;

// 1/pi in FP32: joint angles are reduced exactly by sincospif(angle / pi).
constexpr float kInvPi = 0.318309886183790671538f;

// What one chain evaluation leaves for the task error and Jacobian.
struct ChainState {
  float x0, x1, x2, y0, y1, y2, z0, z1, z2, p0, p1, p2;  // last frame (dof)
  float zx[kMaxDof], zy[kMaxDof];  // x, y of the axis of joint k (z of frame k)
  // z-plane Jacobian term of joint k: (z_k x p_k)_z for revolute joints (so that
  // J_k = zx_k pe_y - zy_k pe_x - zm_k), -z_k,z for prismatic ones (zx = zy = 0 there)
  float zm[kMaxDof];
  // the same axes in full and m_k = z_k x p_k, for the line and fixed-orientation tasks
  // (J_v,k = z_k x p_e - m_k and J_w,k = z_k for revolute joints; z_k and 0 for prismatic)
  float gz0[kMaxDof], gz1[kMaxDof], gz2[kMaxDof], gm0[kMaxDof], gm1[kMaxDof], gm2[kMaxDof];
};

// Runs the DH chain for configuration q. If `fr` is non-null, frames 1..dof are written to
// fr[(k-1)*12 ..] as {x, y, z, p}; if `wq` is non-null, each joint's {sin, cos} (revolute)
// or {q, 0} (prismatic) to wq[k] (the collision check's per-waypoint cache).
__device__ __forceinline__ void chain(const RobotDev& rb, const float* q, float* fr,
                                      ChainState& s, float2* wq = nullptr) {
  float x0 = 1.f, x1 = 0.f, x2 = 0.f;
  float y0 = 0.f, y1 = 1.f, y2 = 0.f;
  float z0 = 0.f, z1 = 0.f, z2 = 1.f;
  float p0 = 0.f, p1 = 0.f, p2 = 0.f;
#pragma unroll
  for (int k = 0; k < kMaxDof; ++k) {
    if (k < rb.dof) {
      const JointDev& J = rb.j[k];
      if (J.prismatic) {
        s.zx[k] = 0.f; s.zy[k] = 0.f; s.zm[k] = -z2;
      } else {
        s.zx[k] = z0; s.zy[k] = z1; s.zm[k] = fmaf(z0, p1, -z1 * p0);
      }
      s.gz0[k] = z0; s.gz1[k] = z1; s.gz2[k] = z2;
      s.gm0[k] = fmaf(z1, p2, -z2 * p1);
      s.gm1[k] = fmaf(z2, p0, -z0 * p2);
      s.gm2[k] = fmaf(z0, p1, -z1 * p0);
      float ct, st, d = J.d;
      if (J.prismatic) {
        ct = J.ct0;
        st = J.st0;
        d += q[k];
        if (wq) wq[k] = make_float2(q[k], 0.f);
      } else {
        sincospif((J.theta0 + q[k]) * kInvPi, &st, &ct);
        if (wq) wq[k] = make_float2(st, ct);
      }
      const float u0 = fmaf(x0, ct, y0 * st), u1 = fmaf(x1, ct, y1 * st), u2 = fmaf(x2, ct, y2 * st);
      const float v0 = fmaf(y0, ct, -x0 * st), v1 = fmaf(y1, ct, -x1 * st), v2 = fmaf(y2, ct, -x2 * st);
      p0 = fmaf(J.a, u0, fmaf(d, z0, p0));
      p1 = fmaf(J.a, u1, fmaf(d, z1, p1));
      p2 = fmaf(J.a, u2, fmaf(d, z2, p2));
      x0 = u0; x1 = u1; x2 = u2;
      y0 = fmaf(v0, J.ca, z0 * J.sa); y1 = fmaf(v1, J.ca, z1 * J.sa); y2 = fmaf(v2, J.ca, z2 * J.sa);
      const float nz0 = fmaf(z0, J.ca, -v0 * J.sa), nz1 = fmaf(z1, J.ca, -v1 * J.sa),
                  nz2 = fmaf(z2, J.ca, -v2 * J.sa);
      z0 = nz0; z1 = nz1; z2 = nz2;
      if (fr) {
        float* f = fr + k * kFrameFloats;
        f[0] = x0; f[1] = x1; f[2] = x2;
        f[3] = y0; f[4] = y1; f[5] = y2;
        f[6] = z0; f[7] = z1; f[8] = z2;
        f[9] = p0; f[10] = p1; f[11] = p2;
      }
    }
  }
  s.x0 = x0; s.x1 = x1; s.x2 = x2; s.y0 = y0; s.y1 = y1; s.y2 = y2;
  s.z0 = z0; s.z1 = z1; s.z2 = z2; s.p0 = p0; s.p1 = p1; s.p2 = p2;
}

// Task error, the scalars its Jacobian needs, and the damped step of one configuration.
template <int CT>
struct Task {
  float e0, e1;
  // roll/pitch: J0_k = (x0 zx_k + x1 zy_k) * c0,  J1_k = (x0 zy_k - x1 zx_k) * c1
  // z-plane:    J0_k = zx_k pe1 - zy_k pe0 - zm_k  (= (z_k x (p_e - p_k))_z, or z_k,z)
  float c0, c1, pe0, pe1;
};

template <int CT>
__device__ __forceinline__ Task<CT> task_error(const RobotDev& rb, const ConsDev& c,
                                               const ChainState& s) {
  Task<CT> t{};
  if (CT == kConsRollPitch) {
    // ZYX Euler angles of R = [x y z]: R11 = x0, R21 = x1, R31 = x2, R32 = y2, R33 = z2.
    t.e0 = atan2f(s.y2, s.z2);                                   // roll
    t.e1 = atan2f(-s.x2, sqrtf(fmaf(s.y2, s.y2, s.z2 * s.z2)));  // pitch
    // Euler-rate map rows: (cos(yaw), sin(yaw)) / cos(pitch) = (R11, R21) / c2 and
    // (-sin(yaw), cos(yaw)) = (-R21, R11) / c, with c2 = R11^2 + R21^2 = cos(pitch)^2.
    const float c2 = fmaf(s.x0, s.x0, s.x1 * s.x1);
    t.c0 = 1.0f / c2;
    t.c1 = rsqrtf(c2);
  } else if (CT == kConsZPlane) {
    t.pe0 = fmaf(s.x0, rb.ee[0], fmaf(s.y0, rb.ee[1], fmaf(s.z0, rb.ee[2], s.p0)));
    t.pe1 = fmaf(s.x1, rb.ee[0], fmaf(s.y1, rb.ee[1], fmaf(s.z1, rb.ee[2], s.p1)));
    const float pe2 = fmaf(s.x2, rb.ee[0], fmaf(s.y2, rb.ee[1], fmaf(s.z2, rb.ee[2], s.p2)));
    t.e0 = pe2 - c.target;
    t.e1 = 0.f;
  } else {
    t.e0 = t.e1 = 0.f;
  }
  return t;
}

template <int CT>
__device__ __forceinline__ void jac_entry(const RobotDev& rb, const ChainState& s,
                                          const Task<CT>& t, int k, float& j0, float& j1) {
  if (CT == kConsRollPitch) {
    const bool rev = !rb.j[k].prismatic;
    j0 = rev ? fmaf(s.x0, s.zx[k], s.x1 * s.zy[k]) * t.c0 : 0.f;
    j1 = rev ? fmaf(s.x0, s.zy[k], -s.x1 * s.zx[k]) * t.c1 : 0.f;
  } else if (CT == kConsZPlane) {
    j0 = fmaf(s.zx[k], t.pe1, fmaf(-s.zy[k], t.pe0, -s.zm[k]));
    j1 = 0.f;
  } else {
    j0 = j1 = 0.f;
  }
}

// Solves (J J^T + lambda^2 I) y = e for m <= 2 (Cramer's rule); the step is g_k = J_k . y.
template <int CT>
__device__ __forceinline__ void damped_solve(const RobotDev& rb, const ConsDev& c,
                                             const ChainState& s, const Task<CT>& t,
                                             float& y0, float& y1) {
  float a = c.lam2, b = 0.f, d = c.lam2;
#pragma unroll
  for (int k = 0; k < kMaxDof; ++k) {
    if (k < rb.dof) {
      float j0, j1;
      jac_entry<CT>(rb, s, t, k, j0, j1);
      a = fmaf(j0, j0, a);
      b = fmaf(j0, j1, b);
      d = fmaf(j1, j1, d);
    }
  }
  if (CT == kConsRollPitch) {
    const float inv_det = 1.0f / fmaf(a, d, -b * b);
    y0 = fmaf(d, t.e0, -b * t.e1) * inv_det;
    y1 = fmaf(a, t.e1, -b * t.e0) * inv_det;
  } else if (CT == kConsZPlane) {
    y0 = t.e0 / a;
    y1 = 0.f;
  } else {
    y0 = y1 = 0.f;
  }
}

template <int CT>
__device__ __forceinline__ float task_err_inf(const Task<CT>& t) {
  return CT == kConsRollPitch ? fmaxf(fabsf(t.e0), fabsf(t.e1))
                              : (CT == kConsZPlane ? fabsf(t.e0) : 0.f);
}

// ---- the line and fixed-orientation tasks (m = 2, 4, 5 rows) ------------------------------
//
// Rows, with p_e the end-effector point and R = [x y z] its rotation:
//   LINE          [p_y - line_y, p_z - target]
//   ORIENT_PLANE  [roll, pitch, yaw - yaw0, p_z - target]
//   ORIENT_LINE   [roll, pitch, yaw - yaw0, p_y - line_y, p_z - target]
// with ZYX Euler angles (yaw - yaw0 wrapped into (-pi, pi]). Jacobian rows from the
// geometric columns (v, w) of joint k: position rows are v_y, v_z; with c2 = R11^2 + R21^2
// (= cos^2 pitch) the Euler-rate rows are roll (R11 w_x + R21 w_y) / c2, pitch
// (R11 w_y - R21 w_x) / sqrt(c2) and yaw w_z - R31 (R11 w_x + R21 w_y) / c2.
template <int CT>
__host__ __device__ constexpr int task_rows() {
  return CT == kConsLine ? 2 : CT == kConsOrientPlane ? 4 : CT == kConsOrientLine ? 5 : 1;
}

template <int CT>
struct TaskN {
  float e[task_rows<CT>()];
  float pe0, pe1, pe2;   // end-effector point
  float r11, r21, r31;   // rotation entries of the Euler-rate rows
  float inv_c2, inv_c;   // 1 / cos^2 pitch, 1 / cos pitch
};

template <int CT>
__device__ __forceinline__ TaskN<CT> task_error_n(const RobotDev& rb, const ConsDev& c,
                                                  const ChainState& s) {
  TaskN<CT> t{};
  t.pe0 = fmaf(s.x0, rb.ee[0], fmaf(s.y0, rb.ee[1], fmaf(s.z0, rb.ee[2], s.p0)));
  t.pe1 = fmaf(s.x1, rb.ee[0], fmaf(s.y1, rb.ee[1], fmaf(s.z1, rb.ee[2], s.p1)));
  t.pe2 = fmaf(s.x2, rb.ee[0], fmaf(s.y2, rb.ee[1], fmaf(s.z2, rb.ee[2], s.p2)));
  if (CT == kConsLine) {
    t.e[0] = t.pe1 - c.target_y;
    t.e[1] = t.pe2 - c.target;
  } else {
    t.r11 = s.x0;
    t.r21 = s.x1;
    t.r31 = s.x2;
    t.e[0] = atan2f(s.y2, s.z2);
    t.e[1] = atan2f(-s.x2, sqrtf(fmaf(s.y2, s.y2, s.z2 * s.z2)));
    float dy = atan2f(s.x1, s.x0) - c.yaw;
    const float two_pi = 6.28318530717958647692f;
    while (dy > 3.14159265358979323846f) dy -= two_pi;
    while (dy <= -3.14159265358979323846f) dy += two_pi;
    t.e[2] = dy;
    const float c2 = fmaf(s.x0, s.x0, s.x1 * s.x1);
    t.inv_c2 = 1.0f / c2;
    t.inv_c = rsqrtf(c2);
    if (CT == kConsOrientPlane) {
      t.e[3] = t.pe2 - c.target;
    } else {
      t.e[3] = t.pe1 - c.target_y;
      t.e[4] = t.pe2 - c.target;
    }
  }
  return t;
}

// Column k of the task Jacobian.
template <int CT>
__device__ __forceinline__ void jac_column_n(const RobotDev& rb, const ChainState& s,
                                             const TaskN<CT>& t, int k,
                                             float (&j)[task_rows<CT>()]) {
  const bool rev = !rb.j[k].prismatic;
  const float z0 = s.gz0[k], z1 = s.gz1[k], z2 = s.gz2[k];
  // v = z x p_e - m (revolute) or z (prismatic)
  const float vy = rev ? fmaf(z2, t.pe0, -z0 * t.pe2) - s.gm1[k] : z1;
  const float vz = rev ? fmaf(z0, t.pe1, -z1 * t.pe0) - s.gm2[k] : z2;
  if (CT == kConsLine) {
    j[0] = vy;
    j[1] = vz;
  } else {
    const float wx = rev ? z0 : 0.f, wy = rev ? z1 : 0.f, wz = rev ? z2 : 0.f;
    const float a = fmaf(t.r11, wx, t.r21 * wy);
    j[0] = a * t.inv_c2;
    j[1] = fmaf(t.r11, wy, -t.r21 * wx) * t.inv_c;
    j[2] = fmaf(-t.r31 * a, t.inv_c2, wz);
    if (CT == kConsOrientPlane) {
      j[3] = vz;
    } else {
      j[3] = vy;
      j[4] = vz;
    }
  }
}

// Solves (J J^T + lambda^2 I) y = e (m x m, symmetric positive definite) by Cholesky.
template <int CT>
__device__ __forceinline__ void damped_solve_n(const RobotDev& rb, const ConsDev& c,
                                               const ChainState& s, const TaskN<CT>& t,
                                               float (&y)[task_rows<CT>()]) {
  constexpr int M = task_rows<CT>();
  float A[M][M];
#pragma unroll
  for (int r = 0; r < M; ++r)
#pragma unroll
    for (int q = 0; q < M; ++q) A[r][q] = r == q ? c.lam2 : 0.f;
#pragma unroll
  for (int k = 0; k < kMaxDof; ++k) {
    if (k < rb.dof) {
      float j[M];
      jac_column_n<CT>(rb, s, t, k, j);
#pragma unroll
      for (int r = 0; r < M; ++r)
#pragma unroll
        for (int q = 0; q <= r; ++q) A[r][q] = fmaf(j[r], j[q], A[r][q]);
    }
  }
  // A = L L^T, L in the lower triangle of A
#pragma unroll
  for (int q = 0; q < M; ++q) {
    float d = A[q][q];
#pragma unroll
    for (int p = 0; p < q; ++p) d = fmaf(-A[q][p], A[q][p], d);
    const float lqq = sqrtf(d), inv = 1.0f / lqq;
    A[q][q] = lqq;
#pragma unroll
    for (int r = q + 1; r < M; ++r) {
      float v = A[r][q];
#pragma unroll
      for (int p = 0; p < q; ++p) v = fmaf(-A[r][p], A[q][p], v);
      A[r][q] = v * inv;
    }
  }
  // L z = e, then L^T y = z
#pragma unroll
  for (int r = 0; r < M; ++r) {
    float v = t.e[r];
#pragma unroll
    for (int p = 0; p < r; ++p) v = fmaf(-A[r][p], y[p], v);
    y[r] = v / A[r][r];
  }
#pragma unroll
  for (int r = M - 1; r >= 0; --r) {
    float v = y[r];
#pragma unroll
    for (int p = r + 1; p < M; ++p) v = fmaf(-A[p][r], y[p], v);
    y[r] = v / A[r][r];
  }
}

// One configuration's task evaluation for Alg. 1, whatever the constraint type: the error,
// its infinity norm, and per joint the component g_k of J^+ e. The roll-pitch and z-plane
// forms keep their closed-form arithmetic.
template <int CT, bool GENERIC = (CT >= kConsLine)>
struct TaskEval;

template <int CT>
struct TaskEval<CT, false> {
  Task<CT> t;
  float y0, y1;
  __device__ __forceinline__ void eval(const RobotDev& rb, const ConsDev& c, const ChainState& s) {
    t = task_error<CT>(rb, c, s);
  }
  __device__ __forceinline__ float err_inf() const { return task_err_inf<CT>(t); }
  __device__ __forceinline__ void solve(const RobotDev& rb, const ConsDev& c, const ChainState& s) {
    damped_solve<CT>(rb, c, s, t, y0, y1);
  }
  __device__ __forceinline__ float step(const RobotDev& rb, const ChainState& s, int k) const {
    float j0, j1;
    jac_entry<CT>(rb, s, t, k, j0, j1);
    return fmaf(j0, y0, j1 * y1);
  }
};

template <int CT>
struct TaskEval<CT, true> {
  TaskN<CT> t;
  float y[task_rows<CT>()];
  __device__ __forceinline__ void eval(const RobotDev& rb, const ConsDev& c, const ChainState& s) {
    t = task_error_n<CT>(rb, c, s);
  }
  __device__ __forceinline__ float err_inf() const {
    float m = 0.f;
#pragma unroll
    for (int r = 0; r < task_rows<CT>(); ++r) m = fmaxf(m, fabsf(t.e[r]));
    return m;
  }
  __device__ __forceinline__ void solve(const RobotDev& rb, const ConsDev& c, const ChainState& s) {
    damped_solve_n<CT>(rb, c, s, t, y);
  }
  __device__ __forceinline__ float step(const RobotDev& rb, const ChainState& s, int k) const {
    float j[task_rows<CT>()];
    jac_column_n<CT>(rb, s, t, k, j);
    float g = 0.f;
#pragma unroll
    for (int r = 0; r < task_rows<CT>(); ++r) g = fmaf(j[r], y[r], g);
    return g;
  }
};

}  // namespace cprrtc
