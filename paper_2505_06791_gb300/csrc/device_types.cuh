// Device-side parameter blocks shared by the kernels of the constrained-motion library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cprrtc {

constexpr int kMaxDof = 8;
constexpr int kMaxW = 64;
constexpr int kMaxSpheres = 256;
constexpr unsigned kFull = 0xffffffffu;

// Task constraints (Sec. V-B): the end effector's roll and pitch, a plane, a line, and the
// fixed orientation (roll, pitch, yaw) with a plane or a line.
enum : int {
  kConsNone = 0,
  kConsRollPitch = 1,
  kConsZPlane = 2,
  kConsLine = 3,
  kConsOrientPlane = 4,
  kConsOrientLine = 5
};
constexpr int kNumCons = 6;
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
// 4 arrays of [n_box]: {cx,cy,cz,hx} {col0, hy} {col1, hz} {col2, rb} where col_k is column
// k of R (box axis k) and rb the radius of a ball about the centre that contains the box;
// capsules 2 arrays of [n_cap]: {p0, rc} {u = p1 - p0, 1/|u|^2}.
// After the obstacle arrays come chunk boxes: the obstacles of each kind, in stream order,
// are cut into chunks of kChunk (a kind's last chunk may be shorter; no chunk mixes kinds),
// sphere chunks first, then box and capsule chunks; each chunk has an axis-aligned box
// containing its obstacles: 2 float4 {min, -} {max, -}.
constexpr int kChunk = 8;
struct SceneDev {
  const float4* obs;
  int n_sph, n_box, n_cap;
  __host__ __device__ int n_obs() const { return n_sph + n_box + n_cap; }
  __host__ __device__ int chunks_sph() const { return (n_sph + kChunk - 1) / kChunk; }
  __host__ __device__ int chunks_box() const { return (n_box + kChunk - 1) / kChunk; }
  __host__ __device__ int n_chunks() const {
    return chunks_sph() + chunks_box() + (n_cap + kChunk - 1) / kChunk;
  }
  // kind of chunk c: 0 spheres, 1 boxes, 2 capsules
  __host__ __device__ int chunk_kind(int c) const {
    return c < chunks_sph() ? 0 : c < chunks_sph() + chunks_box() ? 1 : 2;
  }
  // obstacles [chunk_first(c), chunk_end(c)) of chunk c
  __host__ __device__ int chunk_first(int c) const {
    const int k = chunk_kind(c);
    return k == 0 ? c * kChunk
                  : k == 1 ? n_sph + (c - chunks_sph()) * kChunk
                           : n_sph + n_box + (c - chunks_sph() - chunks_box()) * kChunk;
  }
  __host__ __device__ int chunk_end(int c) const {
    const int k = chunk_kind(c);
    const int end = k == 0 ? n_sph : k == 1 ? n_sph + n_box : n_obs();
    const int f = chunk_first(c) + kChunk;
    return f < end ? f : end;
  }
  __host__ __device__ int chunk_off() const { return n_sph + 4 * n_box + 2 * n_cap; }
  __host__ __device__ int n_float4() const { return chunk_off() + 2 * n_chunks(); }
};

// Task constraint and Algorithm 1 parameters in FP32.
struct ConsDev {
  int type;
  float target;    // plane or line height z
  float target_y;  // line: y of the line {y = target_y, z = target} (parallel to x)
  float yaw;       // fixed orientation: yaw of the end effector
  float tol_task;
  float c_sm;
  float tau_floor;
  float tol_sm;
  float alpha;
  float lam2;   // lambda^2
  int max_iters;
};

}  // namespace cprrtc
