// Per-thread forward kinematics, task error and task Jacobian (GetTaskError /
// GetTaskJacobian of Alg. 1, Sec. III-A), and the damped pseudoinverse step, in FP32.
//
// The DH chain is advanced with the column form of T_k = Rz(theta) Tz(d) Tx(a) Rx(alpha):
// with the previous frame's axes x, y, z and origin p,
//   u = x cos(theta) + y sin(theta),  v = y cos(theta) - x sin(theta),
//   p' = p + a u + d z,  x' = u,  y' = v cos(alpha) + z sin(alpha),  z' = z cos(alpha) - v sin(alpha)
// (about 24 FMA-class operations and one sincos per joint).
#pragma once
#include "device_types.cuh"

namespace cprrtc {

// Floats stored per frame: axes x, y, z then origin p (columns of the 3x4 transform).
constexpr int kFrameFloats = 12;

struct TaskEval {
  int m;              // task rows (0, 1 or 2)
  float e0, e1;       // task error
  float J0[kMaxDof];  // task Jacobian rows
  float J1[kMaxDof];
};

// Runs the DH chain for configuration q. If `fr` is non-null, frames 1..dof are written to
// fr[(k-1)*12 .. ] as {x, y, z, p}. If `task`, fills t with the task error and Jacobian of
// constraint c.
template <bool task>
__device__ __forceinline__ void chain(const RobotDev& rb, const ConsDev& c, const float* q,
                                      float* fr, TaskEval& t) {
  float x0 = 1.f, x1 = 0.f, x2 = 0.f;
  float y0 = 0.f, y1 = 1.f, y2 = 0.f;
  float z0 = 0.f, z1 = 0.f, z2 = 1.f;
  float p0 = 0.f, p1 = 0.f, p2 = 0.f;
  float zx[kMaxDof], zy[kMaxDof], zz[kMaxDof], px[kMaxDof], py[kMaxDof];
#pragma unroll
  for (int k = 0; k < kMaxDof; ++k) {
    if (k < rb.dof) {
      zx[k] = z0; zy[k] = z1; zz[k] = z2; px[k] = p0; py[k] = p1;
      const JointDev& J = rb.j[k];
      float ct, st, d = J.d;
      if (J.prismatic) {
        ct = J.ct0;
        st = J.st0;
        d += q[k];
      } else {
        sincosf(J.theta0 + q[k], &st, &ct);
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
  if (!task) return;
  if (c.type == kConsRollPitch) {
    // ZYX Euler angles of R = [x y z]: R11 = x0, R21 = x1, R31 = x2, R32 = y2, R33 = z2.
    t.m = 2;
    t.e0 = atan2f(y2, z2);                                  // roll
    t.e1 = atan2f(-x2, sqrtf(fmaf(y2, y2, z2 * z2)));       // pitch
    // Euler-rate map: cos(yaw)/cos(pitch) = R11 / c2, sin(yaw)/cos(pitch) = R21 / c2 with
    // c2 = R11^2 + R21^2 = cos(pitch)^2; second row uses cos(yaw), sin(yaw) = R11, R21 / c.
    const float c2 = fmaf(x0, x0, x1 * x1);
    const float inv_c2 = 1.0f / c2;
    const float inv_c = rsqrtf(c2);
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) {
      if (k < rb.dof) {
        const bool rev = !rb.j[k].prismatic;
        t.J0[k] = rev ? fmaf(x0, zx[k], x1 * zy[k]) * inv_c2 : 0.f;
        t.J1[k] = rev ? fmaf(x0, zy[k], -x1 * zx[k]) * inv_c : 0.f;
      }
    }
  } else if (c.type == kConsZPlane) {
    t.m = 1;
    const float e0 = fmaf(x0, rb.ee[0], fmaf(y0, rb.ee[1], fmaf(z0, rb.ee[2], p0)));
    const float e1 = fmaf(x1, rb.ee[0], fmaf(y1, rb.ee[1], fmaf(z1, rb.ee[2], p1)));
    const float e2 = fmaf(x2, rb.ee[0], fmaf(y2, rb.ee[1], fmaf(z2, rb.ee[2], p2)));
    t.e0 = e2 - c.target;
    t.e1 = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) {
      if (k < rb.dof) {
        // z component of z_k x (p_e - p_k) (revolute) or z_k (prismatic)
        t.J0[k] = rb.j[k].prismatic ? zz[k] : fmaf(zx[k], e1 - py[k], -zy[k] * (e0 - px[k]));
        t.J1[k] = 0.f;
      }
    }
  } else {
    t.m = 0;
    t.e0 = t.e1 = 0.f;
  }
}

// g = J^T (J J^T + lambda^2 I)^-1 e for m <= 2 (Cramer's rule on the 2x2 system).
__device__ __forceinline__ void damped_step(const RobotDev& rb, const ConsDev& c,
                                            const TaskEval& t, float* g) {
  if (t.m == 2) {
    float a = c.lam2, b = 0.f, d = c.lam2;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k)
      if (k < rb.dof) {
        a = fmaf(t.J0[k], t.J0[k], a);
        b = fmaf(t.J0[k], t.J1[k], b);
        d = fmaf(t.J1[k], t.J1[k], d);
      }
    const float inv_det = 1.0f / fmaf(a, d, -b * b);
    const float y0 = fmaf(d, t.e0, -b * t.e1) * inv_det;
    const float y1 = fmaf(a, t.e1, -b * t.e0) * inv_det;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k)
      if (k < rb.dof) g[k] = fmaf(t.J0[k], y0, t.J1[k] * y1);
  } else if (t.m == 1) {
    float a = c.lam2;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k)
      if (k < rb.dof) a = fmaf(t.J0[k], t.J0[k], a);
    const float y0 = t.e0 / a;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k)
      if (k < rb.dof) g[k] = t.J0[k] * y0;
  } else {
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) g[k] = 0.f;
  }
}

__device__ __forceinline__ float task_err_inf(const TaskEval& t) {
  return t.m == 2 ? fmaxf(fabsf(t.e0), fabsf(t.e1)) : (t.m == 1 ? fabsf(t.e0) : 0.f);
}

}  // namespace cprrtc
