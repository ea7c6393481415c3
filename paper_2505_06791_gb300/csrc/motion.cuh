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
// Collision checking walks the waypoints in order (see collide_warp). The first waypoint
// with any penetrating pair ends the walk: the warp-wide vote plays the role of the paper's
// shared collision flag, and the index it reports is the smallest colliding waypoint
// whatever the lane timing.
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

// World position of a point given in the frame whose 12 floats {x, y, z, p} start at f
// (frame 0, the base, is the identity: f == nullptr).
__device__ __forceinline__ void to_world(const float* f, float lx, float ly, float lz,
                                         float& cx, float& cy, float& cz) {
  if (!f) {
    cx = lx; cy = ly; cz = lz;
    return;
  }
  cx = fmaf(f[0], lx, fmaf(f[3], ly, fmaf(f[6], lz, f[9])));
  cy = fmaf(f[1], lx, fmaf(f[4], ly, fmaf(f[7], lz, f[10])));
  cz = fmaf(f[2], lx, fmaf(f[5], ly, fmaf(f[8], lz, f[11])));
}

// Per-warp shared-memory scratch of the collision walk.
struct CcScratch {
  const float4* bnd;  // [dof + 1] frame bounding spheres, local coordinates (shared by the CTA)
  float4* wsph;       // [S] world centre + radius of each robot sphere at the current waypoint
  float4* wbnd;       // [dof + 1] world centre + padded radius of each frame's bounding sphere
};

// Shared-memory layout of the motion kernels, in bytes from the dynamic shared base:
//   obstacles (staged only when they fit) | robot spheres | frame bounds | sphere frames |
//   per warp: world spheres, world bounds, frame cache | extra (kernel-specific, 16-aligned)
struct SmemLayout {
  size_t obs, sph, bnd, sfr, warp0, warp_bytes, wsph, wbnd, frames, extra, total;
  __host__ __device__ SmemLayout(int stage_f4, int S, int dof, int W, int warps,
                                 size_t extra_bytes) {
    auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
    obs = 0;
    sph = al(obs + (size_t)stage_f4 * 16);
    bnd = al(sph + (size_t)S * 16);
    sfr = al(bnd + (size_t)(kMaxDof + 1) * 16);
    warp0 = al(sfr + (size_t)S * 4);
    wsph = 0;
    wbnd = al(wsph + (size_t)S * 16);
    frames = al(wbnd + (size_t)(kMaxDof + 1) * 16);
    warp_bytes = al(frames + (size_t)W * (kFrameFloats * dof + 1) * 4);
    extra = al(warp0 + (size_t)warps * warp_bytes);
    total = extra + extra_bytes;
  }
};

// Stages robot spheres, their frames and the frame bounds into shared memory.
__device__ __forceinline__ void stage_robot(const RobotDev& rb, char* base, const SmemLayout& L) {
  float4* sph = reinterpret_cast<float4*>(base + L.sph);
  float4* bnd = reinterpret_cast<float4*>(base + L.bnd);
  int* sfr = reinterpret_cast<int*>(base + L.sfr);
  for (int i = threadIdx.x; i < rb.n_spheres; i += blockDim.x) {
    sph[i] = rb.spheres[i];
    sfr[i] = rb.sphere_frame[i];
  }
#pragma unroll
  for (int f = 0; f <= kMaxDof; ++f)
    if (threadIdx.x == f) bnd[f] = rb.bound[f];
}

// Tests obstacle o (index into the sphere / box / capsule ranges) against ball (c, r).
__device__ __forceinline__ bool hit_obstacle(const SceneDev& sc, const float4* __restrict__ obs,
                                             int o, float cx, float cy, float cz, float r) {
  if (o < sc.n_sph) return hit_sphere(cx, cy, cz, r, obs[o]);
  o -= sc.n_sph;
  if (o < sc.n_box) {
    const float4* b = obs + sc.n_sph + 4 * o;
    return hit_box(cx, cy, cz, r, b[0], b[1], b[2], b[3]);
  }
  o -= sc.n_box;
  const float4* k = obs + sc.n_sph + 4 * sc.n_box + 2 * o;
  return hit_capsule(cx, cy, cz, r, k[0], k[1]);
}

// FK + CC of waypoints [i0, W) in order; returns the first colliding waypoint or -1.
//
// Two levels per waypoint, exact: each lane takes one obstacle of a 32-obstacle chunk and
// tests it against the bounding sphere of every frame's robot spheres (radius padded by
// 1e-5 m, far above the FP32 error of either test, so a miss there proves every sphere of
// that frame misses). Only the (obstacle, frame) pairs that survive are tested sphere by
// sphere, lanes over the robot's spheres. The warp-wide vote after each such obstacle
// plays the role of the paper's shared collision flag (Sec. IV).
__device__ __forceinline__ int collide_warp(const RobotDev& rb, const SceneDev& sc,
                                            const float4* __restrict__ obs,
                                            const float4* sph, const int* sfr, int W, int i0,
                                            const float* fr, CcScratch cc) {
  const int lane = threadIdx.x & 31;
  const int dof = rb.dof;
  const int fs = frame_stride(dof);
  const int S = rb.n_spheres;
  const int n_obs = sc.n_sph + sc.n_box + sc.n_cap;
  for (int i = i0; i < W; ++i) {
    const float* fw = fr + i * fs;
    if (lane <= dof) {
      const float4 b = cc.bnd[lane];
      float x, y, z;
      to_world(lane == 0 ? nullptr : fw + (lane - 1) * kFrameFloats, b.x, b.y, b.z, x, y, z);
      cc.wbnd[lane] = make_float4(x, y, z, b.w);
    }
    for (int s = lane; s < S; s += 32) {
      const float4 l = sph[s];
      const int f = sfr[s];
      float x, y, z;
      to_world(f == 0 ? nullptr : fw + (f - 1) * kFrameFloats, l.x, l.y, l.z, x, y, z);
      cc.wsph[s] = make_float4(x, y, z, l.w);
    }
    __syncwarp();
    bool hit = false;
    for (int base = 0; base < n_obs && !hit; base += 32) {
      const int o = base + lane;
      unsigned mask = 0u;
      if (o < n_obs) {
        for (int f = 0; f <= dof; ++f) {
          const float4 b = cc.wbnd[f];
          if (b.w >= 0.f && hit_obstacle(sc, obs, o, b.x, b.y, b.z, b.w)) mask |= 1u << f;
        }
      }
      unsigned cand = __ballot_sync(kFull, mask != 0u);
      while (cand) {
        const int src = __ffs(cand) - 1;
        cand &= cand - 1;
        const int oo = base + src;
        const unsigned m = __shfl_sync(kFull, mask, src);
        bool h = false;
        for (int s = lane; s < S; s += 32) {
          if ((m >> sfr[s]) & 1u) {
            const float4 c = cc.wsph[s];
            h |= hit_obstacle(sc, obs, oo, c.x, c.y, c.z, c.w);
          }
        }
        if (__any_sync(kFull, h)) {
          hit = true;
          break;
        }
      }
    }
    __syncwarp();
    if (hit) return i;
  }
  return -1;
}

}  // namespace cprrtc
