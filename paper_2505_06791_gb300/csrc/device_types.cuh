// Device-side parameter blocks shared by the kernels of the constrained-motion library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cprrtc {

constexpr int kMaxDof = 8;
constexpr int kMaxW = 64;
constexpr int kMaxSpheres = 256;
constexpr unsigned kFull = 0xffffffffu;

enum : int { kConsNone = 0, kConsRollPitch = 1, kConsZPlane = 2 };
enum : int { kValid = 0, kProjFail = 1, kCollision = 2 };

// One DH joint, FP32, with the trigonometry of the fixed angles precomputed on the host.
struct JointDev {
  float ca, sa;    // cos(alpha), sin(alpha)
  float a, d;
  float theta0;
  float ct0, st0;  // cos(theta0), sin(theta0): prismatic joints only
  float lo, hi;
  int prismatic;
};

// Robot passed by value in the kernel parameter space (constant bank).
struct RobotDev {
  int dof;
  int n_spheres;
  JointDev j[kMaxDof];
  float ee[3];
  // bounding sphere of each frame's robot spheres {centre in that frame, radius + 1e-5 m};
  // radius -1 for a frame without spheres
  float4 bound[kMaxDof + 1];
  int n_per_frame[kMaxDof + 1];  // robot spheres on each frame
  int bound_count;               // frames with spheres
  const float4* spheres;     // [n_spheres] {x, y, z, r} in the sphere's frame, sorted by frame
  const int* sphere_frame;   // [n_spheres] frame index, 0 = base
};

// Obstacles as one float4 stream, component arrays per primitive so that lanes reading
// consecutive obstacles read consecutive float4s: spheres [n_sph] {x,y,z,rho}; boxes
// 4 arrays of [n_box]: {cx,cy,cz,hx} {col0, hy} {col1, hz} {col2, 0} where col_k is column
// k of R (box axis k); capsules 2 arrays of [n_cap]: {p0, rc} {u = p1 - p0, 1/|u|^2}.
// After the obstacle arrays, every chunk of 32 consecutive obstacles (in the order spheres,
// boxes, capsules) has an axis-aligned box containing all of them: 2 float4 {min, -} {max, -}.
constexpr int kChunk = 32;
struct SceneDev {
  const float4* obs;
  int n_sph, n_box, n_cap;
  __host__ __device__ int n_obs() const { return n_sph + n_box + n_cap; }
  __host__ __device__ int n_chunks() const { return (n_obs() + kChunk - 1) / kChunk; }
  __host__ __device__ int chunk_off() const { return n_sph + 4 * n_box + 2 * n_cap; }
  __host__ __device__ int n_float4() const { return chunk_off() + 2 * n_chunks(); }
};

// Task constraint and Algorithm 1 parameters in FP32.
struct ConsDev {
  int type;
  float target;
  float tol_task;
  float c_sm;
  float tau_floor;
  float tol_sm;
  float alpha;
  float lam2;   // lambda^2
  int max_iters;
};

}  // namespace cprrtc
