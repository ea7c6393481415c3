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
#include "launch.h"

namespace cprrtc {

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
  int updates;     // waypoint updates Alg. 1 needed: sum over iterations of (W - 1 - prog)
};

// Work a warp evaluated, for roofline accounting (warp-uniform counts). 32-bit per warp:
// one warp's launch stays far below 2^32 of each (the totals are summed in 64 bits).
struct WorkCount {
  unsigned updates;     // Alg. 1 waypoint updates
  unsigned chains;      // DH chains evaluated for collision checking
  unsigned transforms;  // points moved to world coordinates (frame bounds, robot spheres)
  unsigned p_sph, p_box, p_cap;  // ball-vs-primitive tests by primitive
  unsigned warm_tried, warm_used; // planner's learned form: extend motions warm-started, accepted
  __device__ __forceinline__ void add_type(const SceneDev& sc, int o, unsigned n) {
    if (o < sc.n_sph)
      p_sph += n;
    else if (o < sc.n_sph + sc.n_box)
      p_box += n;
    else
      p_cap += n;
  }
  // swept-bound tests of obstacles [lo, hi) against nb frame bounds
  __device__ __forceinline__ void add_tests(const SceneDev& sc, int lo, int hi, int nb) {
    const int c_s = max(0, min(hi, sc.n_sph) - lo);
    const int c_b = max(0, min(hi, sc.n_sph + sc.n_box) - max(lo, sc.n_sph));
    p_sph += (unsigned)(nb * c_s);
    p_box += (unsigned)(nb * c_b);
    p_cap += (unsigned)(nb * (hi - lo - c_s - c_b));
  }
  __device__ __forceinline__ void count_test(const SceneDev& sc, int o, int n) { add_type(sc, o, n); }
  __device__ __forceinline__ void count_fine(const SceneDev& sc, int o, int n) {
    add_type(sc, o, n);
    transforms += n;
  }
  __device__ void flush(unsigned long long* dst) const {
    if (!dst || (threadIdx.x & 31) != 0) return;
    atomicAdd(dst + 0, (unsigned long long)updates);
    atomicAdd(dst + 1, (unsigned long long)chains);
    atomicAdd(dst + 2, (unsigned long long)transforms);
    atomicAdd(dst + 3, (unsigned long long)p_sph);
    atomicAdd(dst + 4, (unsigned long long)p_box);
    atomicAdd(dst + 5, (unsigned long long)p_cap);
    if (warm_tried) atomicAdd(dst + 6, (unsigned long long)warm_tried);
    if (warm_used) atomicAdd(dst + 7, (unsigned long long)warm_used);
  }
};

// Alg. 1 on the warp's motion, constraint type CT, at most max_iters iterations.
// q[WPL][kMaxDof] holds this lane's waypoints (the interpolated segment on entry, the
// segment after the last iteration on exit). With CT = kConsNone nothing is done.
// With `wq` (the warp's collision-check cache [W][9]), every evaluation also stores each
// waypoint's joint {sin, cos}: after a success the cache holds those of the returned segment,
// which the last iteration evaluated.
template <int CT, int WPL>
__device__ __forceinline__ ProjResult project_warp(const RobotDev& rb, const ConsDev& c,
                                                   int max_iters, float (&q)[WPL][kMaxDof],
                                                   int W, float tau, float2* wq = nullptr) {
  const int lane = threadIdx.x & 31;
  const int dof = rb.dof;
  ProjResult res{kValid, 0, -1, 0.f, 0};
  ChainState cs;
  if (CT == kConsNone) return res;
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
      // run converged
      chain(rb, q[s], nullptr, cs, (wq && i < W) ? wq + i * 9 : nullptr);
      TaskEval<CT> te;
      te.eval(rb, c, cs);
      te.solve(rb, c, cs);
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
          const float g = te.step(rb, cs, k);
          const float dk = q[s][k] - prev;
          const float esm = fmaxf(0.f, fabsf(dk) - tau);
          const float v = fmaf(-c.alpha, fmaf(dk, esm, g), q[s][k]);
          qn[s][k] = fminf(fmaxf(v, rb.j[k].lo), rb.j[k].hi);
          esm_max = fmaxf(esm_max, esm);
        }
      }
      const float et = te.err_inf();
      const bool valid = (i >= W) || ((esm_max < c.tol_sm) && (et < c.tol_task));
      if (i > prog && i < W) last_err[s] = et;
      valid_mask |= (unsigned long long)__ballot_sync(kFull, valid) << (32 * s);
    }
    res.updates += W - 1 - prog;
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

// ---- one motion on two warps (33 <= W <= 64) ----------------------------------------------
//
// Warp h of the pair holds waypoints 32 h + lane, one per lane. The two warps run Alg. 1 in
// step: each iteration they publish their `valid` ballots (and warp 0 its candidate update of
// waypoint 31, the predecessor of warp 1's first waypoint) to this exchange area, meet at a
// named barrier of 64 threads and both advance `prog` over the same 64-bit mask. Slots are
// double-buffered by iteration parity, so one barrier per iteration suffices: a slot is
// written again two iterations later, after the reader has passed the barrier in between.
// The collision check then splits the same way (each warp its own waypoints); `hit` holds
// the generation of the last motion in which either warp found a collision.
struct SplitX {
  unsigned ballot[2][2];     // [parity][warp]
  float qn31[2][kMaxDof];    // [parity] warp 0's candidate update of waypoint 31
  float p31[kMaxDof];        // waypoint 31 as it stands (kept by warp 1's lane 0 alone)
  float qend[kMaxDof];       // the projected motion's last waypoint (held by warp 1)
  float resid[2];            // [warp] largest last-evaluated ||E_task||_inf over its waypoints
  int hit;                   // generation of the last motion found colliding
  int pad;
};

__device__ __forceinline__ void pair_barrier(int id) {
  asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

// Alg. 1 on the motion q0 -> q1 held by a warp pair, this warp being half h (0 or 1): q[0]
// is this lane's waypoint min(32 h + lane, W - 1) on entry, as project_warp<CT, 1> would
// hold it; results (status, iterations, prog, updates, resid) are those of the one-warp
// form with WPL = 2 on the same motion, identical in both warps. Every call made by one warp
// of the pair must be made by the other (the barriers pair them up).
template <int CT>
__device__ __forceinline__ ProjResult project_pair(const RobotDev& rb, const ConsDev& c,
                                                   int max_iters, float (&q)[1][kMaxDof], int W,
                                                   float tau, float2* wq, int h, SplitX* x,
                                                   int bar, const float* q0, const float* q1) {
  const int lane = threadIdx.x & 31;
  const int dof = rb.dof;
  const int i = 32 * h + lane;
  ProjResult res{kValid, 0, -1, 0.f, 0};
  ChainState cs;
  if (CT == kConsNone) return res;
  const unsigned long long in_range = (W >= 64) ? ~0ull : ((1ull << W) - 1ull);
  if (h == 1 && lane == 0) interp(q0, q1, 31, W, dof, x->p31);
  float last_err = 0.f;
  int prog = 0;
  for (int it = 1; it <= max_iters; ++it) {
    const int par = it & 1;
    float qn[kMaxDof];
    chain(rb, q[0], nullptr, cs, (wq && i < W) ? wq + i * 9 : nullptr);
    TaskEval<CT> te;
    te.eval(rb, c, cs);
    te.solve(rb, c, cs);
    float esm_max = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) {
      if (k < dof) {
        float prev = __shfl_up_sync(kFull, q[0][k], 1);
        if (h == 1 && lane == 0) prev = x->p31[k];
        const float g = te.step(rb, cs, k);
        const float dk = q[0][k] - prev;
        const float esm = fmaxf(0.f, fabsf(dk) - tau);
        const float v = fmaf(-c.alpha, fmaf(dk, esm, g), q[0][k]);
        qn[k] = fminf(fmaxf(v, rb.j[k].lo), rb.j[k].hi);
        esm_max = fmaxf(esm_max, esm);
      }
    }
    const float et = te.err_inf();
    const bool valid = (i >= W) || ((esm_max < c.tol_sm) && (et < c.tol_task));
    if (i > prog && i < W) last_err = et;
    const unsigned b = __ballot_sync(kFull, valid);
    if (lane == 0) x->ballot[par][h] = b;
    if (h == 0 && lane == 31) {
#pragma unroll
      for (int k = 0; k < kMaxDof; ++k)
        if (k < dof) x->qn31[par][k] = qn[k];
    }
    pair_barrier(bar);
    const unsigned long long valid_mask =
        (unsigned long long)x->ballot[par][0] | ((unsigned long long)x->ballot[par][1] << 32);
    res.updates += W - 1 - prog;
    const unsigned long long after = in_range & ~((2ull << prog) - 1ull);  // (prog, W)
    const unsigned long long invalid = after & ~valid_mask;
    if (invalid == 0ull) {
      prog = W - 1;
      res.iters = it;
      break;
    }
    prog = __ffsll((long long)invalid) - 2;
    if (i > prog && i < W) {
#pragma unroll
      for (int k = 0; k < kMaxDof; ++k)
        if (k < dof) q[0][k] = qn[k];
    }
    if (h == 1 && lane == 0 && prog < 31) {
#pragma unroll
      for (int k = 0; k < kMaxDof; ++k)
        if (k < dof) x->p31[k] = x->qn31[par][k];
    }
  }
  float m = i >= 1 ? last_err : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
  if (lane == 0) x->resid[h] = m;
  pair_barrier(bar);
  res.resid = fmaxf(x->resid[0], x->resid[1]);
  if (prog != W - 1) {
    res.status = kProjFail;
    res.iters = max_iters;
    res.first_fail = prog + 1;
  }
  return res;
}

// The sequential projection of the naive baseline (cpRRTC-Naive, Sec. V; CBiRRT-style):
// waypoints 1..W-1 one after another, each by damped steps from its interpolated point moved
// by the previous waypoint's correction, until ||E_task||_inf < tol_task (at most max_iters
// steps). It fails at the first waypoint that does not converge or ends farther than
// tau + tol_sm (in some joint) from its predecessor. Every lane takes the same steps (the
// other waypoints wait, as in the baseline); lane i % 32 keeps waypoint i. iters is the
// total number of steps.
template <int CT, int WPL>
__device__ __forceinline__ ProjResult project_sequential(const RobotDev& rb, const ConsDev& c,
                                                         int max_iters, const float* q0,
                                                         const float* q1,
                                                         float (&q)[WPL][kMaxDof], int W,
                                                         float tau) {
  const int lane = threadIdx.x & 31;
  const int dof = rb.dof;
  ProjResult res{kValid, 0, -1, 0.f, 0};
  if (CT == kConsNone) return res;
  float prev_p[kMaxDof], prev_i[kMaxDof];  // previous waypoint: projected, interpolated
#pragma unroll
  for (int k = 0; k < kMaxDof; ++k) prev_p[k] = prev_i[k] = k < dof ? q0[k] : 0.f;
  float resid = 0.f;
  for (int i = 1; i < W; ++i) {
    float qi[kMaxDof], x[kMaxDof];
    interp(q0, q1, i, W, dof, qi);
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k)
      x[k] = k < dof ? fminf(fmaxf(qi[k] + (prev_p[k] - prev_i[k]), rb.j[k].lo), rb.j[k].hi) : 0.f;
    ChainState cs;
    bool ok = false;
    float err = 0.f;
    int it = 0;
    for (;; ++it) {
      chain(rb, x, nullptr, cs);
      TaskEval<CT> te;
      te.eval(rb, c, cs);
      err = te.err_inf();
      if (err < c.tol_task) {
        ok = true;
        break;
      }
      if (it == max_iters) break;
      te.solve(rb, c, cs);
      float g[kMaxDof];
#pragma unroll
      for (int k = 0; k < kMaxDof; ++k) g[k] = k < dof ? te.step(rb, cs, k) : 0.f;
#pragma unroll
      for (int k = 0; k < kMaxDof; ++k)
        if (k < dof) x[k] = fminf(fmaxf(fmaf(-c.alpha, g[k], x[k]), rb.j[k].lo), rb.j[k].hi);
    }
    res.iters += it;
    res.updates += it;
    float step = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k)
      if (k < dof) step = fmaxf(step, fabsf(x[k] - prev_p[k]) - tau);
#pragma unroll
    for (int s = 0; s < WPL; ++s)
      if (i == lane + 32 * s) {
#pragma unroll
        for (int k = 0; k < kMaxDof; ++k) q[s][k] = x[k];
      }
    resid = fmaxf(resid, err);
    if (!ok || step >= c.tol_sm) {
      res.status = kProjFail;
      res.first_fail = i;
      break;
    }
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) {
      prev_p[k] = x[k];
      prev_i[k] = qi[k];
    }
  }
  res.resid = resid;
  return res;
}

// Shared-memory layout of the motion kernels, in bytes from the dynamic shared base:
//   obstacles (staged only when they fit) | robot spheres (sorted by frame) | frame bounds |
//   spheres per frame | first sphere of each frame | joints |
//   per warp: waypoints [W][9] floats, swept bounds [dof + 1], candidate list |
//   extra (kernel-specific, 16-aligned)
constexpr int kCandMax = 512;  // candidate obstacles listed per pass of the collision check

struct SmemLayout {
  size_t obs, sph, bnd, nsf, foff, jnt, warp0, warp_bytes, wq, sbnd, cand, extra, total;
  __host__ __device__ SmemLayout(int stage_f4, int S, int W, int warps, size_t extra_bytes) {
    auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
    obs = 0;
    sph = al(obs + (size_t)stage_f4 * 16);
    bnd = al(sph + (size_t)S * 16);
    nsf = al(bnd + (size_t)(kMaxDof + 1) * 16);
    foff = al(nsf + (size_t)(kMaxDof + 1) * 4);
    jnt = al(foff + (size_t)(kMaxDof + 2) * 4);
    warp0 = al(jnt + sizeof(JointDev) * kMaxDof);
    wq = 0;
    sbnd = al(wq + (size_t)W * 9 * 8);
    cand = al(sbnd + (size_t)(kMaxDof + 1) * 16);
    warp_bytes = al(cand + (size_t)kCandMax * 4);
    extra = al(warp0 + (size_t)warps * warp_bytes);
    total = extra + extra_bytes;
  }
};

// What the collision check reads from shared memory.
struct CcShared {
  const float4* sph;    // [S] robot spheres {x, y, z, r} in their frames, sorted by frame
  const float4* bnd;    // [dof + 1] frame bounding spheres (local centre, padded radius)
  const int* nsf;       // [dof + 1] spheres per frame
  const int* foff;      // [dof + 2] first sphere of each frame
  const JointDev* jnt;  // [dof]
  float2* wq;           // this warp: per waypoint and joint {sin, cos} of the joint angle
                        // (revolute) or {q, 0} (prismatic), [W][9]
  float4* sbnd;         // this warp: swept frame bounds [dof + 1]
  unsigned* cand;       // this warp: candidate list, obstacle | frame mask << 20
};

__device__ __forceinline__ CcShared cc_shared(char* base, const SmemLayout& L, int warp) {
  char* w = base + L.warp0 + (size_t)warp * L.warp_bytes;
  return CcShared{reinterpret_cast<const float4*>(base + L.sph),
                  reinterpret_cast<const float4*>(base + L.bnd),
                  reinterpret_cast<const int*>(base + L.nsf),
                  reinterpret_cast<const int*>(base + L.foff),
                  reinterpret_cast<const JointDev*>(base + L.jnt),
                  reinterpret_cast<float2*>(w + L.wq), reinterpret_cast<float4*>(w + L.sbnd),
                  reinterpret_cast<unsigned*>(w + L.cand)};
}

// Stages robot spheres, frame bounds, per-frame counts and offsets and the joint table.
__device__ __forceinline__ void stage_robot(const RobotDev& rb, char* base, const SmemLayout& L) {
  float4* sph = reinterpret_cast<float4*>(base + L.sph);
  float4* bnd = reinterpret_cast<float4*>(base + L.bnd);
  int* nsf = reinterpret_cast<int*>(base + L.nsf);
  int* foff = reinterpret_cast<int*>(base + L.foff);
  JointDev* jnt = reinterpret_cast<JointDev*>(base + L.jnt);
  for (int i = threadIdx.x; i < rb.n_spheres; i += blockDim.x) sph[i] = rb.spheres[i];
  if (threadIdx.x == 0) {  // small tables, constant indices into the parameter block
    int o = 0;
#pragma unroll
    for (int f = 0; f <= kMaxDof; ++f) {
      bnd[f] = rb.bound[f];
      nsf[f] = rb.n_per_frame[f];
      foff[f] = o;
      o += rb.n_per_frame[f];
    }
    foff[kMaxDof + 1] = o;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) jnt[k] = rb.j[k];
  }
}

// Tests obstacle o (index into the sphere / box / capsule ranges) against ball (c, r).
__device__ __forceinline__ bool hit_obstacle(const SceneDev& sc, const float4* __restrict__ obs,
                                             int o, float cx, float cy, float cz, float r) {
  if (o < sc.n_sph) return hit_sphere(cx, cy, cz, r, obs[o]);
  o -= sc.n_sph;
  if (o < sc.n_box) {
    const float4* b = obs + sc.n_sph + o;  // component j at b[j * n_box]
    return hit_box(cx, cy, cz, r, b[0], b[sc.n_box], b[2 * sc.n_box], b[3 * sc.n_box]);
  }
  o -= sc.n_box;
  const float4* k = obs + sc.n_sph + 4 * sc.n_box + o;  // component j at k[j * n_cap]
  return hit_capsule(cx, cy, cz, r, k[0], k[sc.n_cap]);
}

// One obstacle's rows, read once from shared memory for the repeated tests of the chain
// walk (kind: 0 sphere, 1 box, 2 capsule; the same predicates as `hit_obstacle`).
struct ObsView {
  int kind;
  float4 a, b, c, d;
};

__device__ __forceinline__ ObsView load_obstacle(const SceneDev& sc,
                                                 const float4* __restrict__ obs, int o) {
  ObsView v;
  v.b = v.c = v.d = make_float4(0.f, 0.f, 0.f, 0.f);
  if (o < sc.n_sph) {
    v.kind = 0;
    v.a = obs[o];
    return v;
  }
  o -= sc.n_sph;
  if (o < sc.n_box) {
    const float4* b = obs + sc.n_sph + o;
    v.kind = 1;
    v.a = b[0];
    v.b = b[sc.n_box];
    v.c = b[2 * sc.n_box];
    v.d = b[3 * sc.n_box];
    return v;
  }
  o -= sc.n_box;
  const float4* k = obs + sc.n_sph + 4 * sc.n_box + o;
  v.kind = 2;
  v.a = k[0];
  v.b = k[sc.n_cap];
  return v;
}

__device__ __forceinline__ bool hit_view(const ObsView& v, float cx, float cy, float cz,
                                         float r) {
  if (v.kind == 0) return hit_sphere(cx, cy, cz, r, v.a);
  if (v.kind == 1) return hit_box(cx, cy, cz, r, v.a, v.b, v.c, v.d);
  return hit_capsule(cx, cy, cz, r, v.a, v.b);
}

// One DH frame of a lane's waypoint: axes x, y, z and origin p (world).
struct Frame {
  float x0, x1, x2, y0, y1, y2, z0, z1, z2, p0, p1, p2;
  __device__ __forceinline__ void identity() {
    x0 = 1.f; x1 = 0.f; x2 = 0.f; y0 = 0.f; y1 = 1.f; y2 = 0.f;
    z0 = 0.f; z1 = 0.f; z2 = 1.f; p0 = 0.f; p1 = 0.f; p2 = 0.f;
  }
  // Advances by joint J at joint value q (same arithmetic as `chain`).
  __device__ __forceinline__ void advance(const JointDev& J, float q) {
    float ct, st, d = J.d;
    if (J.prismatic) {
      ct = J.ct0;
      st = J.st0;
      d += q;
    } else {
      sincospif((J.theta0 + q) * kInvPi, &st, &ct);
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
  }
  // The same step from a cached {sin, cos} (revolute) or {q, 0} (prismatic): the values are
  // those `advance` computes, so the frames are identical.
  __device__ __forceinline__ void advance_cached(const JointDev& J, float2 v) {
    float ct, st, d = J.d;
    if (J.prismatic) {
      ct = J.ct0;
      st = J.st0;
      d += v.x;
    } else {
      st = v.x;
      ct = v.y;
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
  }
  __device__ __forceinline__ void world(float lx, float ly, float lz, float& cx, float& cy,
                                        float& cz) const {
    cx = fmaf(x0, lx, fmaf(y0, ly, fmaf(z0, lz, p0)));
    cy = fmaf(x1, lx, fmaf(y1, ly, fmaf(z1, lz, p1)));
    cz = fmaf(x2, lx, fmaf(y2, ly, fmaf(z2, lz, p2)));
  }
};

// Spheres of frames fa < fb of one waypoint (joint terms wq[0..dof), the collision check's
// cache) against each other: true if two of them overlap (touching is free).
static __device__ __noinline__ bool self_pair_spheres(const JointDev* jnt, const float4* sph,
                                                      const int* foff, const float2* wq, int fa,
                                                      int fb) {
  Frame F, A;
  F.identity();
  A.identity();
#pragma unroll 1
  for (int f = 1; f <= fb; ++f) {
    F.advance_cached(jnt[f - 1], wq[f - 1]);
    if (f == fa) A = F;
  }
#pragma unroll 1
  for (int sa = foff[fa]; sa < foff[fa + 1]; ++sa) {
    const float4 la = sph[sa];
    float ax, ay, az;
    A.world(la.x, la.y, la.z, ax, ay, az);
#pragma unroll 1
    for (int sb = foff[fb]; sb < foff[fb + 1]; ++sb) {
      const float4 lb = sph[sb];
      float bx, by, bz;
      F.world(lb.x, lb.y, lb.z, bx, by, bz);
      const float dx = ax - bx, dy = ay - by, dz = az - bz, r = la.w + lb.w;
      if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < r * r) return true;
    }
  }
  return false;
}

// Self-collision of one waypoint: each paired frames' bounding spheres (padded) first, the
// spheres only where those overlap. The predicates of the self-collision kernel of
// cprrtc_validate (self_collide.cu). Out of line, with runtime loops and the frame centres
// in a small per-thread array, so that the callers' register allocation does not grow.
static __device__ __noinline__ bool self_hit_waypoint(int dof, const JointDev* jnt, const float4* bnd,
                                                      const float4* sph, const int* foff,
                                                      const float2* wq, SelfMask m) {
  float4 c[kMaxDof + 1];  // frame bounding spheres in world coordinates {centre, radius}
  Frame F;
  F.identity();
#pragma unroll 1
  for (int f = 0; f <= dof; ++f) {
    if (f > 0) F.advance_cached(jnt[f - 1], wq[f - 1]);
    const float4 b = bnd[f];
    float x, y, z;
    F.world(b.x, b.y, b.z, x, y, z);
    c[f] = make_float4(x, y, z, b.w);
  }
#pragma unroll 1
  for (int fa = 0; fa < dof; ++fa) {
    const unsigned rows = m.rows[fa];
    if (!rows || c[fa].w < 0.f) continue;
#pragma unroll 1
    for (int fb = fa + 1; fb <= dof; ++fb) {
      if (!((rows >> fb) & 1u) || c[fb].w < 0.f) continue;
      const float dx = c[fa].x - c[fb].x, dy = c[fa].y - c[fb].y, dz = c[fa].z - c[fb].z;
      const float rr = c[fa].w + c[fb].w;
      if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= rr * rr) continue;
      if (self_pair_spheres(jnt, sph, foff, wq, fa, fb)) return true;
    }
  }
  return false;
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Order-preserving map of non-NaN floats to signed integers (negative floats have their
// magnitude bits flipped), so that one integer warp reduction finds a float minimum or
// maximum.
__device__ __forceinline__ int float_key(float x) {
  const int i = __float_as_int(x);
  return i < 0 ? i ^ 0x7fffffff : i;
}
__device__ __forceinline__ float key_float(int k) {
  return __int_as_float(k < 0 ? k ^ 0x7fffffff : k);
}
__device__ __forceinline__ float warp_min_exact(float v) {
  return key_float(__reduce_min_sync(kFull, float_key(v)));
}
__device__ __forceinline__ float warp_max_exact(float v) {
  return key_float(__reduce_max_sync(kFull, float_key(v)));
}

// Frames (bits of fmask) whose swept bound sbnd[f] = {centre, radius} the ball test `hit`
// accepts; the tests are independent, unrolled over the frames.
template <class Hit>
__device__ __forceinline__ unsigned frames_touched(const float4* sbnd, unsigned fmask, Hit hit) {
  unsigned m = 0u;
#pragma unroll
  for (int f = 0; f <= kMaxDof; ++f)
    if ((fmask >> f) & 1u) {
      if (hit(sbnd[f])) m |= 1u << f;
    }
  return m;
}

// The same predicates as `hit_view` with the swept bounds as balls, one obstacle per lane;
// `box_tests` counts the exact box tests made after the containing-ball test.
__device__ __forceinline__ unsigned swept_mask(const ObsView& v, const float4* sbnd,
                                               unsigned fmask, int& box_tests) {
  if (v.kind == 0)
    return frames_touched(sbnd, fmask,
                          [&](float4 b) { return hit_sphere(b.x, b.y, b.z, b.w, v.a); });
  if (v.kind == 1) {
    // the ball containing the box first; the box test only for the frames that ball touches
    const float4 ball = make_float4(v.a.x, v.a.y, v.a.z, v.d.w);
    unsigned m = frames_touched(sbnd, fmask,
                                [&](float4 b) { return hit_sphere(b.x, b.y, b.z, b.w, ball); });
    unsigned out = 0u;
    while (m) {
      const int f = __ffs(m) - 1;
      m &= m - 1u;
      const float4 b = sbnd[f];
      if (hit_box(b.x, b.y, b.z, b.w, v.a, v.b, v.c, v.d)) out |= 1u << f;
      ++box_tests;
    }
    return out;
  }
  return frames_touched(sbnd, fmask,
                        [&](float4 b) { return hit_capsule(b.x, b.y, b.z, b.w, v.a, v.b); });
}

// FK + CC of waypoints [i0, W) of the warp's segment (lane l holds waypoints l + 32 s in
// q). Returns the smallest colliding waypoint, or -1. With `any_hit`, returns as soon as
// some waypoint is known to collide (the index is then a colliding waypoint, not
// necessarily the smallest): the paper's shared flag (Sec. IV), for callers that only need
// the verdict. With early = false (an ablation) nothing is skipped: every waypoint is
// tested against every candidate and the answer is the same.
//
// Exact culling in three levels (a miss at a level proves a miss of everything under it,
// every radius padded by at least 1e-5 m, far above the FP32 error of the tests):
//  1. per motion: each frame's bounding sphere is swept over the waypoints (a ball around
//     the box of its centres); each chunk of 32 obstacles is tested through its bounding
//     box, then each obstacle of a touched chunk against every swept bound, and the
//     obstacles that touch one are listed with the frames they touch;
//  2. per waypoint (lane), frame by frame along the chain: the frame's bounding sphere
//     against each listed obstacle of that frame;
//  3. the frame's robot spheres, for lanes whose bound touched the obstacle.
//
// A motion shared by a warp pair (see SplitX) is split either by waypoints (PAIR: lane l
// holds waypoint wbase + l and the walk covers this warp's waypoints) or by obstacles
// (NSPLIT = 2: both warps hold every waypoint, and warp kw lists and walks only the chunks
// c with c mod NSPLIT = kw, its swept bounds being the same as the other's). Either way
// any_hit is assumed, and the warp gives up as soon as x->hit shows that the other warp
// found a collision in this motion (generation gen): the pair's verdict is the flag, and the
// count returned covers this warp's part.
template <int WPL, bool PAIR = false, int NSPLIT = 1>
__device__ __forceinline__ int collide_motion(const RobotDev& rb, const SceneDev& sc,
                                              const float4* __restrict__ obs, const CcShared& S,
                                              const float (&q)[WPL][kMaxDof], int W, int i0,
                                              bool any_hit, WorkCount& work, bool early = true,
                                              bool wq_ready = false, int wbase = 0,
                                              const SplitX* x = nullptr, int gen = 0, int kw = 0) {
  constexpr bool kShared = PAIR || NSPLIT > 1;
  const int lane = threadIdx.x & 31;
  const int dof = rb.dof;
  const int n_obs = sc.n_sph + sc.n_box + sc.n_cap;
  // the other warp of a pair has found a collision in this motion (warp-uniform)
  auto other_hit = [&]() {
    if constexpr (kShared) {
      return __any_sync(kFull, *reinterpret_cast<const volatile int*>(&x->hit) == gen);
    } else {
      return false;
    }
  };
  // each waypoint's joint terms to shared memory once (the chains below walk frames in a
  // runtime loop, once for the swept bounds and once per pass), unless the projection's last
  // evaluation left them there (wq_ready)
#pragma unroll
  for (int s = 0; s < WPL && !wq_ready; ++s) {
    const int i = wbase + lane + 32 * s;
    if (i < W) {
#pragma unroll
      for (int k = 0; k < kMaxDof; ++k) {
        if (k < dof) {
          const JointDev& J = S.jnt[k];
          float2 v = make_float2(q[s][k], 0.f);
          if (!J.prismatic) sincospif((J.theta0 + q[s][k]) * kInvPi, &v.x, &v.y);
          S.wq[i * 9 + k] = v;
        }
      }
    }
  }
  __syncwarp();
  bool act[WPL];
  int n_act = 0;
#pragma unroll
  for (int s = 0; s < WPL; ++s) {
    const int i = wbase + lane + 32 * s;
    act[s] = i >= i0 && i < W;
  }
  n_act = max(0, min(W, wbase + 32 * WPL) - max(i0, wbase));
  if (n_act == 0 || n_obs == 0) return -1;

  // ---- level 1: swept frame bounds over the segment ----
  unsigned fmask = 0u;  // frames that carry spheres (warp-uniform)
  {
    Frame F[WPL];
#pragma unroll
    for (int s = 0; s < WPL; ++s) F[s].identity();
    for (int f = 0; f <= dof; ++f) {
      if (f > 0) {
        const JointDev J = S.jnt[f - 1];
#pragma unroll
        for (int s = 0; s < WPL; ++s) F[s].advance_cached(J, S.wq[min(wbase + lane + 32 * s, W - 1) * 9 + f - 1]);
      }
      const float4 b = S.bnd[f];
      if (b.w < 0.f) continue;  // no spheres on this frame (warp-uniform)
      fmask |= 1u << f;
      float lo0 = INFINITY, lo1 = INFINITY, lo2 = INFINITY;
      float hi0 = -INFINITY, hi1 = -INFINITY, hi2 = -INFINITY;
      float c[WPL][3];
#pragma unroll
      for (int s = 0; s < WPL; ++s) {
        F[s].world(b.x, b.y, b.z, c[s][0], c[s][1], c[s][2]);
        if (act[s]) {
          lo0 = fminf(lo0, c[s][0]); lo1 = fminf(lo1, c[s][1]); lo2 = fminf(lo2, c[s][2]);
          hi0 = fmaxf(hi0, c[s][0]); hi1 = fmaxf(hi1, c[s][1]); hi2 = fmaxf(hi2, c[s][2]);
        }
      }
      const float m0 = 0.5f * (warp_min_exact(lo0) + warp_max_exact(hi0));
      const float m1 = 0.5f * (warp_min_exact(lo1) + warp_max_exact(hi1));
      const float m2 = 0.5f * (warp_min_exact(lo2) + warp_max_exact(hi2));
      float r2 = 0.f;
#pragma unroll
      for (int s = 0; s < WPL; ++s) {
        if (act[s]) {
          const float d0 = c[s][0] - m0, d1 = c[s][1] - m1, d2 = c[s][2] - m2;
          r2 = fmaxf(r2, fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
        }
      }
      const float rad = sqrtf(warp_max_exact(r2)) * 1.000001f + b.w + 1e-5f;
      if (lane == 0) S.sbnd[f] = make_float4(m0, m1, m2, rad);
    }
    if (NSPLIT == 1 || kw == 0) {  // both warps of an obstacle split sweep the same bounds
      work.chains += n_act;
      work.transforms += (unsigned)(n_act * (dof + 1));
    }
    __syncwarp();
  }
  if (other_hit()) return -1;

  int best = 0x7fffffff;  // smallest colliding waypoint found so far
  const int n_chunks = sc.n_chunks();
  // this warp's chunks as slots: slot t is chunk t * NSPLIT + kw (every chunk when NSPLIT = 1)
  auto chunk_of = [&](int t) { return NSPLIT == 1 ? t : t * NSPLIT + kw; };
  auto slots_below = [&](int c) { return NSPLIT == 1 ? c : (c - kw + NSPLIT - 1) / NSPLIT; };
  const int n_slots = slots_below(n_chunks);
  int cb = 0;          // next group of 32 slots to screen
  unsigned near = 0u;  // slots of the current group (base cb - 32) still to list
  unsigned cfr = 0u;   // lane j: the frames whose swept bound slot cb - 32 + j's chunk box touches
  bool listed_all = false;
  while (!listed_all) {
    // ---- candidate list: obstacles touching a swept bound, with the frames they touch ----
    int n_cand = 0;
    while (n_cand + 32 <= kCandMax) {
      if (!near) {
        if (cb >= n_slots) {
          listed_all = true;
          break;
        }
        if (other_hit()) return -1;
        // lanes screen 32 chunks at once: chunk box against every swept frame bound
        const int ch = chunk_of(cb + lane);
        cfr = 0u;
        if (cb + lane < n_slots) {
          const float4* cbx = obs + sc.chunk_off() + 2 * ch;
          const float4 lo = cbx[0], hi = cbx[1];
          cfr = frames_touched(S.sbnd, fmask, [&](float4 b) {
                  const float e0 = fmaxf(fmaxf(lo.x - b.x, b.x - hi.x), 0.f);
                  const float e1 = fmaxf(fmaxf(lo.y - b.y, b.y - hi.y), 0.f);
                  const float e2 = fmaxf(fmaxf(lo.z - b.z, b.z - hi.z), 0.f);
                  const float rr = b.w + 1e-5f;
                  return fmaf(e0, e0, fmaf(e1, e1, e2 * e2)) < rr * rr;
                });
        }
        near = __ballot_sync(kFull, cfr != 0u);
        work.p_box += (unsigned)(rb.bound_count * min(32, n_slots - cb));
        cb += 32;
        continue;
      }
      // up to 32 / kChunk touched chunks of one kind, kChunk lanes each (one code path)
      const int base = cb - 32;  // slot of bit 0 of `near`
      const int kind = sc.chunk_kind(chunk_of(base + __ffs(near) - 1));
      const int cs = sc.chunks_sph(), cbx = sc.chunks_box();
      const int k_c1 = kind == 0 ? cs : kind == 1 ? cs + cbx : n_chunks;  // kind's chunk end
      const int k_o0 = kind == 0 ? 0 : kind == 1 ? sc.n_sph : sc.n_sph + sc.n_box;
      const int k_o1 = kind == 0 ? sc.n_sph : kind == 1 ? sc.n_sph + sc.n_box : n_obs;
      const int k_c0 = kind == 0 ? 0 : kind == 1 ? cs : cs + cbx;
      // bits of `near` for chunks of this kind (slot end relative to base, at most 32)
      const int rel_end = slots_below(k_c1) - base;
      const unsigned kmask = near & (rel_end >= 32 ? kFull : (1u << rel_end) - 1u);
      unsigned m = kmask;
      int my_c = -1;
#pragma unroll
      for (int t = 0; t < 32 / kChunk; ++t) {
        const int c = base + __ffs(m) - 1;
        if (m && t == lane / kChunk) my_c = c;
        m &= m - 1u;
      }
      near &= ~(kmask ^ m);  // the chunks taken
      // an obstacle can only touch the swept bounds its chunk's box touches
      const unsigned my_fr = __shfl_sync(kFull, cfr, my_c >= 0 ? my_c - base : 0);
      int o = -1;
      unsigned mask = 0u;
      if (my_c >= 0) o = k_o0 + (chunk_of(my_c) - k_c0) * kChunk + lane % kChunk;
      const bool valid = o >= 0 && o < k_o1;
      int box_tests = 0;
      if (valid) mask = swept_mask(load_obstacle(sc, obs, o), S.sbnd, my_fr, box_tests);
      {  // balls (spheres, and the balls containing boxes) or capsules against those bounds
        const unsigned tested = __reduce_add_sync(kFull, valid ? (unsigned)__popc(my_fr) : 0u);
        if (kind == 2)
          work.p_cap += tested;
        else
          work.p_sph += tested;
        if (kind == 1) work.p_box += __reduce_add_sync(kFull, (unsigned)box_tests);
      }
      const unsigned bal = __ballot_sync(kFull, mask != 0u);
      if (mask) S.cand[n_cand + __popc(bal & ((1u << lane) - 1u))] = (unsigned)o | (mask << 20);
      n_cand += __popc(bal);
    }
    __syncwarp();
    if (n_cand == 0) continue;
    // waypoints at or after the smallest colliding one found so far cannot change the answer
    bool any_act = false;
#pragma unroll
    for (int s = 0; s < WPL; ++s) {
      act[s] = act[s] && (!early || wbase + lane + 32 * s < best);
      any_act |= act[s];
    }
    if (!__any_sync(kFull, any_act)) break;
    // ---- levels 2 and 3: lanes walk their waypoints' chains frame by frame ----
    Frame F[WPL];
#pragma unroll
    for (int s = 0; s < WPL; ++s) F[s].identity();
    bool hit[WPL];
#pragma unroll
    for (int s = 0; s < WPL; ++s) hit[s] = false;
    for (int f = 0; f <= dof; ++f) {
      if (f > 0) {
        const JointDev J = S.jnt[f - 1];
#pragma unroll
        for (int s = 0; s < WPL; ++s) F[s].advance_cached(J, S.wq[min(wbase + lane + 32 * s, W - 1) * 9 + f - 1]);
      }
      const float4 b = S.bnd[f];
      if (b.w < 0.f) continue;
      float bc[WPL][3];
#pragma unroll
      for (int s = 0; s < WPL; ++s) F[s].world(b.x, b.y, b.z, bc[s][0], bc[s][1], bc[s][2]);
      const int s_lo = S.foff[f], s_hi = S.foff[f + 1];
      // candidates of this frame, 32 at a time: one ballot finds them, the entries travel
      // by shuffle, in increasing list order
      for (int g = 0; g < n_cand; g += 32) {
        const unsigned eg = g + lane < n_cand ? S.cand[g + lane] : 0u;
        unsigned fm = __ballot_sync(kFull, (eg >> (20 + f)) & 1u);
        while (fm) {
          const unsigned e = __shfl_sync(kFull, eg, __ffs(fm) - 1);
          fm &= fm - 1u;
          const int o = (int)(e & 0xFFFFFu);
          const ObsView ov = load_obstacle(sc, obs, o);
          bool near[WPL];
          bool any = false;
#pragma unroll
          for (int s = 0; s < WPL; ++s) {
            near[s] = act[s] && (!early || !hit[s]) && hit_view(ov, bc[s][0], bc[s][1], bc[s][2], b.w);
            any |= near[s];
          }
          work.count_test(sc, o, n_act);
          const unsigned nb = __ballot_sync(kFull, any);
          if (!nb) continue;
          for (int si = s_lo; si < s_hi; ++si) {
            const float4 l = S.sph[si];
#pragma unroll
            for (int s = 0; s < WPL; ++s) {
              if (near[s]) {
                float cx, cy, cz;
                F[s].world(l.x, l.y, l.z, cx, cy, cz);
                hit[s] |= hit_view(ov, cx, cy, cz, l.w);
              }
            }
          }
          int near_cnt = 0;
#pragma unroll
          for (int s = 0; s < WPL; ++s) near_cnt += __popc(__ballot_sync(kFull, near[s]));
          work.count_fine(sc, o, near_cnt * (s_hi - s_lo));
        }
      }
      if (any_hit) {
        bool h = false;
#pragma unroll
        for (int s = 0; s < WPL; ++s) h |= hit[s];
        if (__any_sync(kFull, h)) break;
        if (other_hit()) return -1;
      }
    }
    work.chains += n_act;
    work.transforms += (unsigned)(n_act * (dof + 1));
    // smallest colliding waypoint of this pass
#pragma unroll
    for (int s = 0; s < WPL; ++s) {
      const unsigned hb = __ballot_sync(kFull, hit[s]);
      if (hb) best = min(best, wbase + 32 * s + __ffs(hb) - 1);
    }
    if (early && best != 0x7fffffff && (any_hit || best == i0)) break;
  }
  return best == 0x7fffffff ? -1 : best;
}

}  // namespace cprrtc
