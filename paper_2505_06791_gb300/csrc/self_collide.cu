// Self-collision of the robot (spheres of two frames that the caller pairs, tested against
// each other), run after validation on the returned waypoints: the arm's own links are
// obstacles too once the motion folds it. One warp per motion, lanes over its waypoints;
// per waypoint the DH chain (the same `chain` as the projection) gives every frame, each
// named frame pair is screened by the frames' bounding spheres and then tested sphere by
// sphere (touching counts as free, as for obstacles). The motion's first self-colliding
// waypoint is merged with the obstacle verdict: the smaller index wins.
#include <cuda_runtime.h>

#include "device_types.cuh"
#include "kinematics.cuh"
#include "launch.h"

namespace cprrtc {
namespace {

constexpr int kSelfWarps = 4;

struct FrameRef {
  const float* f;  // x, y, z, p (12 floats); nullptr: the base frame (identity)
  __device__ __forceinline__ void world(float lx, float ly, float lz, float& cx, float& cy,
                                        float& cz) const {
    if (!f) {
      cx = lx;
      cy = ly;
      cz = lz;
      return;
    }
    cx = fmaf(f[0], lx, fmaf(f[3], ly, fmaf(f[6], lz, f[9])));
    cy = fmaf(f[1], lx, fmaf(f[4], ly, fmaf(f[7], lz, f[10])));
    cz = fmaf(f[2], lx, fmaf(f[5], ly, fmaf(f[8], lz, f[11])));
  }
};

__global__ void __launch_bounds__(kSelfWarps * 32)
self_collide_kernel(RobotDev rb, SelfArgs a) {
  extern __shared__ float s_frames[];  // per lane: frames 1..dof, 12 floats each
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = blockIdx.x * kSelfWarps + warp;
  if (m >= a.n) return;  // warp-uniform
  const int st = a.status[m];
  if (st != kValid && st != kCollision) return;  // nothing was checked
  const int W = a.W, dof = rb.dof;
  const int end = st == kCollision ? a.first_fail[m] : W;  // only earlier waypoints matter
  float* fr = s_frames + (size_t)(warp * 32 + lane) * kMaxDof * kFrameFloats;
  int off[kMaxDof + 2];  // first sphere of each frame (spheres are sorted by frame)
  off[0] = 0;
#pragma unroll
  for (int f = 0; f <= kMaxDof; ++f) off[f + 1] = off[f] + (f <= dof ? rb.n_per_frame[f] : 0);
  int mine = 0x7fffffff;  // this lane's first self-colliding waypoint
  for (int i = a.i0 + lane; i < end; i += 32) {
    float q[kMaxDof];
    const float* src = a.q + ((size_t)m * W + i) * dof;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) q[k] = k < dof ? src[k] : 0.f;
    ChainState cs;
    chain(rb, q, fr, cs);
    bool hit = false;
    for (int fa = 0; fa <= dof && !hit; ++fa) {
      const float4 ba = rb.bound[fa];
      if (ba.w < 0.f || !a.rows[fa]) continue;
      const FrameRef A{fa ? fr + (fa - 1) * kFrameFloats : nullptr};
      float ax, ay, az;
      A.world(ba.x, ba.y, ba.z, ax, ay, az);
      for (int fb = fa + 1; fb <= dof && !hit; ++fb) {
        const float4 bb = rb.bound[fb];
        if (bb.w < 0.f || !((a.rows[fa] >> fb) & 1u)) continue;
        const FrameRef B{fr + (fb - 1) * kFrameFloats};
        float bx, by, bz;
        B.world(bb.x, bb.y, bb.z, bx, by, bz);
        const float dx = ax - bx, dy = ay - by, dz = az - bz, rr = ba.w + bb.w;
        if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= rr * rr) continue;  // bounds apart
        for (int sa = off[fa]; sa < off[fa + 1] && !hit; ++sa) {
          const float4 la = rb.spheres[sa];
          float cx, cy, cz;
          A.world(la.x, la.y, la.z, cx, cy, cz);
          for (int sb = off[fb]; sb < off[fb + 1]; ++sb) {
            const float4 lb = rb.spheres[sb];
            float ex, ey, ez;
            B.world(lb.x, lb.y, lb.z, ex, ey, ez);
            const float ux = cx - ex, uy = cy - ey, uz = cz - ez, r = la.w + lb.w;
            if (fmaf(ux, ux, fmaf(uy, uy, uz * uz)) < r * r) {
              hit = true;
              break;
            }
          }
        }
      }
    }
    if (hit) {
      mine = i;  // waypoints rise along the lane's loop
      break;
    }
  }
  const int first = __reduce_min_sync(kFull, mine);
  if (lane == 0 && first < end) {
    a.status[m] = (uint8_t)kCollision;
    a.first_fail[m] = first;
  }
}

}  // namespace

size_t self_collide_smem_bytes() { return (size_t)kSelfWarps * 32 * kMaxDof * kFrameFloats * sizeof(float); }

cudaError_t launch_self_collide(const RobotDev& rb, const SelfArgs& a, cudaStream_t stream) {
  if (a.n <= 0) return cudaSuccess;
  const int smem = (int)self_collide_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(self_collide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int grid = (a.n + kSelfWarps - 1) / kSelfWarps;
  self_collide_kernel<<<grid, kSelfWarps * 32, smem, stream>>>(rb, a);
  return cudaGetLastError();
}

}  // namespace cprrtc
