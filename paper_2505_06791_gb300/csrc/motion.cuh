// One motion per warp: interpolation (Sec. III), Algorithm 1 ParallelProject (Sec. III-A)
// and FK + collision checking with early termination (Sec. IV).
//
// Mapping. Lane l holds waypoints l + 32 s for s < WPL (WPL = 1 for W <= 32, 2 for
// W <= 64). Alg. 1's shared `valid[]` becomes a warp ballot, `prog` a warp-uniform
// register advanced with find-first-set on the complement of the ballot, and the
// `__syncthreads()` pair disappears: a warp executes the acceptance step in lockstep.
// Every lane evaluates its waypoints in every iteration (a frozen waypoint reproduces the
// same values), so the loop has no divergence; only waypoints after `prog` commit.
//
// Collision checking walks the waypoints in order with the lanes spread over the robot's
// spheres. The first waypoint with any penetrating pair ends the walk: the warp-wide vote
// plays the role of the paper's shared collision flag, checked every few primitives, and
// the index it reports is the smallest colliding waypoint whatever the lane timing.
#pragma once
#include "collide.cuh"
#include "kinematics.cuh"

namespace cprrtc {

// Floats per waypoint in the per-warp frame cache: 12 per frame 1..dof, plus one pad so
// that consecutive waypoints fall in different shared-memory banks.
__host__ __device__ inline int frame_stride(int dof) { return kFrameFloats * dof + 1; }

// Interpolated waypoint i of q0 -> q1 (W waypoints): q0 + (i / (W-1)) (q1 - q0).
__device__ __forceinline__ void interp(const float* q0, const float* q1, int i, int W, int dof,
                                       float* q) {
  const float t = (float)i / (float)(W - 1);
#pragma unroll
  for (int k = 0; k < kMaxDof; ++k)
    if (k < dof) q[k] = fmaf(t, q1[k] - q0[k], q0[k]);
}

// tau = max(c_sm ||q1 - q0||_inf / (W-1), tau_floor).
__device__ __forceinline__ float step_threshold(const ConsDev& c, const float* q0,
                                                const float* q1, int W, int dof) {
  float span = 0.f;
#pragma unroll
  for (int k = 0; k < kMaxDof; ++k)
    if (k < dof) span = fmaxf(span, fabsf(q1[k] - q0[k]));
  return fmaxf(c.c_sm * span / (float)(W - 1), c.tau_floor);
}

struct ProjResult {
  int status;      // kValid (projected / no constraint) or kProjFail
  int iters;
  int first_fail;  // first unaccepted waypoint on failure
  float resid;     // max over waypoints 1..W-1 of the last evaluated ||E_task||_inf
};

// Alg. 1 on the warp's motion, constraint type CT, at most max_iters iterations.
// q[WPL][kMaxDof] holds this lane's waypoints (the interpolated segment on entry, the
// segment after the last iteration on exit). Frames of every waypoint's evaluation are
// written to fr (stride frame_stride(dof)); on success they describe the returned segment.
// With CT = kConsNone only the frames are computed.
template <int CT, int WPL>
__device__ __forceinline__ ProjResult project_warp(const RobotDev& rb, const ConsDev& c,
                                                   int max_iters, float (&q)[WPL][kMaxDof],
                                                   int W, float tau, float* fr) {
  const int lane = threadIdx.x & 31;
  const int dof = rb.dof;
  const int fs = frame_stride(dof);
  ProjResult res{kValid, 0, -1, 0.f};
  ChainState cs;
  if (CT == kConsNone) {
#pragma unroll
    for (int s = 0; s < WPL; ++s) {
      const int i = lane + 32 * s;
      if (i < W) chain(rb, q[s], fr + i * fs, cs);
    }
    return res;
  }
  // waypoints [0, W) as a 64-bit mask
  const unsigned long long in_range = (W >= 64) ? ~0ull : ((1ull << W) - 1ull);
  float last_err[WPL];
#pragma unroll
  for (int s = 0; s < WPL; ++s) last_err[s] = 0.f;
  int prog = 0;
  for (int it = 1; it <= max_iters; ++it) {
    float qn[WPL][kMaxDof];
    unsigned long long valid_mask = 0ull;
#pragma unroll
    for (int s = 0; s < WPL; ++s) {
      const int i = lane + 32 * s;
      // every lane evaluates (lanes past W on a clamped copy) so that the shuffles below
      // run converged; only in-range lanes write frames
      chain(rb, q[s], i < W ? fr + i * fs : nullptr, cs);
      const Task<CT> t = task_error<CT>(rb, c, cs);
      float y0, y1;
      damped_solve<CT>(rb, c, cs, t, y0, y1);
      float esm_max = 0.f;
#pragma unroll
      for (int k = 0; k < kMaxDof; ++k) {
        if (k < dof) {
          // predecessor waypoint i-1 (lane 0 of slot s > 0 takes lane 31 of slot s-1)
          float prev = __shfl_up_sync(kFull, q[s][k], 1);
          if (s > 0) {
            const float wrap = __shfl_sync(kFull, q[s > 0 ? s - 1 : 0][k], 31);
            if (lane == 0) prev = wrap;
          }
          float j0, j1;
          jac_entry<CT>(rb, cs, t, k, j0, j1);
          const float g = fmaf(j0, y0, j1 * y1);
          const float dk = q[s][k] - prev;
          const float esm = fmaxf(0.f, fabsf(dk) - tau);
          const float v = fmaf(-c.alpha, fmaf(dk, esm, g), q[s][k]);
          qn[s][k] = fminf(fmaxf(v, rb.j[k].lo), rb.j[k].hi);
          esm_max = fmaxf(esm_max, esm);
        }
      }
      const float et = task_err_inf<CT>(t);
      const bool valid = (i >= W) || ((esm_max < c.tol_sm) && (et < c.tol_task));
      if (i > prog && i < W) last_err[s] = et;
      valid_mask |= (unsigned long long)__ballot_sync(kFull, valid) << (32 * s);
    }
    // acceptance: advance prog over the contiguous valid run after it
    const unsigned long long after = in_range & ~((2ull << prog) - 1ull);  // (prog, W)
    const unsigned long long invalid = after & ~valid_mask;
    if (invalid == 0ull) {
      prog = W - 1;
      res.iters = it;
      break;
    }
    prog = __ffsll((long long)invalid) - 2;
#pragma unroll
    for (int s = 0; s < WPL; ++s) {
      const int i = lane + 32 * s;
      if (i > prog && i < W) {
#pragma unroll
        for (int k = 0; k < kMaxDof; ++k)
          if (k < dof) q[s][k] = qn[s][k];
      }
    }
  }
  float m = 0.f;
#pragma unroll
  for (int s = 0; s < WPL; ++s)
    if (lane + 32 * s >= 1) m = fmaxf(m, last_err[s]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
  res.resid = m;
  if (prog != W - 1) {
    res.status = kProjFail;
    res.iters = max_iters;
    res.first_fail = prog + 1;
  }
  return res;
}

// World centre of robot sphere `s` at the waypoint whose frames start at `fw`.
__device__ __forceinline__ void sphere_world(const float4 loc, int frame, const float* fw,
                                             float& cx, float& cy, float& cz) {
  if (frame == 0) {
    cx = loc.x; cy = loc.y; cz = loc.z;
    return;
  }
  const float* f = fw + (frame - 1) * kFrameFloats;
  cx = fmaf(f[0], loc.x, fmaf(f[3], loc.y, fmaf(f[6], loc.z, f[9])));
  cy = fmaf(f[1], loc.x, fmaf(f[4], loc.y, fmaf(f[7], loc.z, f[10])));
  cz = fmaf(f[2], loc.x, fmaf(f[5], loc.y, fmaf(f[8], loc.z, f[11])));
}

// Primitives tested between two votes on the warp's collision flag.
constexpr int kVoteEvery = 8;

// FK + CC of waypoints [i0, W) in order; returns the first colliding waypoint or -1.
// sph/sfr: robot spheres (shared memory), obs: obstacle stream (shared or global).
__device__ __forceinline__ int collide_warp(const RobotDev& rb, const SceneDev& sc,
                                            const float4* __restrict__ obs,
                                            const float4* sph, const int* sfr, int W, int i0,
                                            const float* fr) {
  const int lane = threadIdx.x & 31;
  const int fs = frame_stride(rb.dof);
  const int S = rb.n_spheres;
  const float4* box = obs + sc.n_sph;
  const float4* cap = box + 4 * sc.n_box;
  for (int i = i0; i < W; ++i) {
    const float* fw = fr + i * fs;
    bool hit = false;
    for (int s = lane; s - lane < S; s += 32) {
      const bool act = s < S;
      float cx = 0.f, cy = 0.f, cz = 0.f, r = 0.f;
      if (act) {
        const float4 loc = sph[s];
        sphere_world(loc, sfr[s], fw, cx, cy, cz);
        r = loc.w;
      }
      for (int o0 = 0; o0 < sc.n_sph; o0 += kVoteEvery) {
        const int o1 = min(o0 + kVoteEvery, sc.n_sph);
#pragma unroll 4
        for (int o = o0; o < o1; ++o) hit |= act && hit_sphere(cx, cy, cz, r, obs[o]);
        if (__any_sync(kFull, hit)) break;
      }
      if (__any_sync(kFull, hit)) break;
      for (int o0 = 0; o0 < sc.n_box; o0 += kVoteEvery) {
        const int o1 = min(o0 + kVoteEvery, sc.n_box);
#pragma unroll 2
        for (int o = o0; o < o1; ++o)
          hit |= act && hit_box(cx, cy, cz, r, box[4 * o], box[4 * o + 1], box[4 * o + 2],
                                box[4 * o + 3]);
        if (__any_sync(kFull, hit)) break;
      }
      if (__any_sync(kFull, hit)) break;
      for (int o0 = 0; o0 < sc.n_cap; o0 += kVoteEvery) {
        const int o1 = min(o0 + kVoteEvery, sc.n_cap);
#pragma unroll 2
        for (int o = o0; o < o1; ++o)
          hit |= act && hit_capsule(cx, cy, cz, r, cap[2 * o], cap[2 * o + 1]);
        if (__any_sync(kFull, hit)) break;
      }
      if (__any_sync(kFull, hit)) break;
    }
    if (__any_sync(kFull, hit)) return i;
  }
  return -1;
}

}  // namespace cprrtc
