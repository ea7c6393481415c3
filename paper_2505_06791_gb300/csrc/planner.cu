// RRT-Connect with constrained motions (Sec. III, Sec. II): one CTA per planning problem,
// one warp per tree extension, one motion per warp per round.
//
// Each warp carries an extension chain across rounds: mode EXTEND picks tree
// a = (round + w) mod 2, draws a Philox sample (counter {problem, round, w, draw}, key
// {seed, 0}), steers from its nearest node by at most `range` and validates the motion
// (Alg. 1 + FK + CC, waypoint 0 skipped); a valid end becomes a node and the chain turns to
// the nearest node of the other tree (the target). Mode CONNECT steers toward the target
// and keeps the projected end only if it is strictly closer; within 10 * tau_floor
// (inf-norm) of the target, mode HOP checks the closing motion as it stands (one Alg. 1
// iteration + CC) and a valid hop connects the trees. Warps read the trees as they stood at
// the start of the round; the nodes of a round are appended in warp order after a barrier,
// and the lowest warp that connected returns the path. One motion per round keeps the
// barrier wait short; the search is deterministic for a seed.
//
// Trees live in global memory (nodes padded to 8 floats, parent indices, and each node's
// projected incoming motion, so that returned paths are dense). The problem's obstacles
// are staged into shared memory when they fit.
#include "launch.h"
#include "motion.cuh"
#include "philox.cuh"
#include "warm_net.cuh"

namespace cprrtc {

// One planning problem's inputs, scratch and outputs.
struct ProblemView {
  int p;                  // problem index: Philox counter and output slot
  const float* start;     // dof floats
  const float* goal;
  int W;
  float* nodes;           // [2][max_nodes][8]
  int* parent;            // [2][max_nodes]
  float* edges;           // [2][max_nodes][W * dof]
  float* pend;            // [workers][8]
  float* pend_edges;      // [workers][2][W * dof]
  float* path;            // [max_path][ostride]
  float* path_edges;      // [max_path - 1][estride] or null
  int ostride;            // floats per configuration in the path outputs
  int estride;            // floats per edge in path_edges (>= W * ostride)
};

struct PlanShared {
  ProblemView pv;              // the problem being planned (uniform over the CTA)
  int count0[2];               // tree sizes when the round began
  int padd[kMaxWorkers];       // 1 if the warp produced a node this round
  int ptree[kMaxWorkers];      // the warp's chain tree
  int pparent[kMaxWorkers];    // parent of the produced node (the chain's last node)
  int ptarget[kMaxWorkers];    // the chain's target in the other tree
  int pconn[kMaxWorkers];      // 1 if the warp connected the trees
  long long wp[kMaxWorkers];   // waypoints validated by each warp
  long long wproj[kMaxWorkers];
  long long wcc[kMaxWorkers];
  long long t_start;           // globaltimer at the start of the problem (of its slice)
  long long t_prior;           // device time of the problem's earlier slices
  int stop;                    // 1 once the problem's time budget is spent
  // each warp's configurations, identical across its lanes: kept here instead of in every
  // lane's registers: [0] current chain node, [1] target, [2] motion end, [3] scratch
  float cfg[kMaxWorkers][4][8];
};

__device__ __forceinline__ void load_cfg(const float* src, int dof, float* q) {
#pragma unroll
  for (int k = 0; k < kMaxDof; ++k) q[k] = k < dof ? src[k] : 0.f;
}

// Nearest of nodes[0, count) (stride 8 floats) to q in L2; lowest index on ties. The nodes
// are written during the launch (by this CTA, or by another one in an earlier slice), so the
// pointer is not marked read-only.
__device__ __forceinline__ int nearest_warp(const float* nodes, int count,
                                            const float* q, int dof) {
  const int lane = threadIdx.x & 31;
  float best = INFINITY;
  int bi = 0x7fffffff;
  for (int j = lane; j < count; j += 32) {
    const float4* n4 = reinterpret_cast<const float4*>(nodes + (size_t)j * 8);
    const float4 a = n4[0], b = n4[1];
    const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    float d = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k)
      if (k < dof) {
        const float t = v[k] - q[k];
        d = fmaf(t, t, d);
      }
    if (d < best) {
      best = d;
      bi = j;
    }
  }
  // smallest distance, then the smallest index holding it (distances are >= 0, so their
  // bit patterns order like the values)
  const int kb = __reduce_min_sync(kFull, __float_as_int(best));
  const int r = __reduce_min_sync(kFull, __float_as_int(best) == kb ? bi : 0x7fffffff);
  // no finite distance (configurations out of any sensible range, or NaN): node 0, so that
  // the index always lies in the tree
  return r < count ? r : 0;
}

// dst[0..7] = src[0..dof) padded with zeros (lanes 0..7), then the warp synchronises.
__device__ __forceinline__ void copy_cfg(float* dst, const float* src, int dof) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  if (lane < 8) dst[lane] = lane < dof ? src[lane] : 0.f;
  __syncwarp();
}

__device__ __forceinline__ float dist2(const float* a, const float* b, int dof) {
  float d = 0.f;
#pragma unroll
  for (int k = 0; k < kMaxDof; ++k)
    if (k < dof) {
      const float t = a[k] - b[k];
      d = fmaf(t, t, d);
    }
  return d;
}

// out = from + min(1, range / |to - from|) (to - from); from, to, out in shared memory.
__device__ __forceinline__ void steer(const float* from, const float* to, float range, int dof,
                                      float* out) {
  const int lane = threadIdx.x & 31;
  const float d = sqrtf(dist2(from, to, dof));
  const float f = d > range ? range / d : 1.f;
  __syncwarp();
  if (lane < 8) out[lane] = lane < dof ? fmaf(f, to[lane] - from[lane], from[lane]) : 0.f;
  __syncwarp();
}

// The warp's segment waypoint W-1 written to out (shared memory) by the lane holding it.
template <int WPL>
__device__ __forceinline__ void last_waypoint(const float (&q)[WPL][kMaxDof], int W, int dof,
                                              float* out) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  if (lane == ((W - 1) & 31)) {
    const bool hi = (W - 1) >= 32;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k)
      out[k] = k < dof ? ((WPL > 1 && hi) ? q[WPL > 1 ? 1 : 0][k] : q[0][k]) : 0.f;
  }
  __syncwarp();
}

// The lanes' waypoints wbase + lane + 32 s (< W) to dst[W][dof] (each warp of a pair writes
// its half).
template <int WPL>
__device__ __forceinline__ void store_edge(float* dst, const float (&q)[WPL][kMaxDof], int W,
                                           int dof, int wbase = 0) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < WPL; ++s) {
    const int i = wbase + lane + 32 * s;
    if (i < W) {
#pragma unroll
      for (int k = 0; k < kMaxDof; ++k)
        if (k < dof) dst[i * dof + k] = q[s][k];
    }
  }
}

__device__ __forceinline__ void store_cfg(float* dst, const float* q, int dof) {
  const int lane = threadIdx.x & 31;
  if (lane < 8) {
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k)
      if (k == lane) v = k < dof ? q[k] : 0.f;
    dst[lane] = v;
  }
}

// Copies `count` floats (lanes in parallel).
__device__ __forceinline__ void copy_warp(float* dst, const float* src, int count) {
  for (int i = threadIdx.x & 31; i < count; i += 32) dst[i] = src[i];
}

// Copies a W x dof edge (packed) to rows of `ostride` floats, reversing the waypoint order
// when `rev`; row entries past dof are zeroed.
__device__ __forceinline__ void copy_edge(float* dst, const float* src, int W, int dof,
                                          int ostride, bool rev) {
  for (int i = threadIdx.x & 31; i < W * ostride; i += 32) {
    const int w = i / ostride, k = i - w * ostride;
    dst[i] = k < dof ? src[(rev ? (W - 1 - w) : w) * dof + k] : 0.f;
  }
}

struct MotionWork {  // per warp (32-bit suffices for one launch)
  unsigned proj;  // waypoint updates Alg. 1 needed
  unsigned cc;    // waypoints collision-checked
};

// Interpolate q0 -> q1, project (at most max_iters iterations), FK + CC from waypoint 1
// stopping at the first collision found.
//
// Learned form (WARM, `net` set: extend motions): the network's correction f(q1) of the motion's
// end is spread along the segment, waypoint i moving by (i / (W-1)) f(q1) (clamped to the
// limits). This is the warm start of cprrtc_validate_ws, f(xi_i) - (1 - t_i) f(xi_0), with f
// taken linear along the short motion between f(xi_0) and f(q1): the start term cancels, so one
// network row per motion. The corrected segment is used only if its largest ||E_task||_inf over
// waypoints 1..W-1 is below the interpolation's, and only for warm_refine Alg. 1 iterations;
// otherwise, or if they do not accept the whole segment, plain Alg. 1 runs from the
// interpolation with max_iters, as without the network.
template <int CT, int WPL, bool SEQ = false, bool WARM = false>
__device__ __forceinline__ int validate_motion(const RobotDev& rb, const SceneDev& sc,
                                               const ConsDev& cs, int max_iters, MotionWork& work,
                                               WorkCount& wc, const float4* obs,
                                               const CcShared& S, const float* q0,
                                               const float* q1, int W,
                                               float (&q)[WPL][kMaxDof],
                                               const MlpView* net = nullptr, int warm_refine = 0,
                                               float* fcorr = nullptr, const SelfMask* self = nullptr) {
  const int lane = threadIdx.x & 31;
  const int dof = rb.dof;
  const float tau = step_threshold(cs, q0, q1, W, dof);
  ProjResult pr;
  int first_pass = 1;
  if constexpr (WARM && !SEQ && CT != kConsNone) {
    if (net) {
      net_correction_warp(*net, q1, dof, reinterpret_cast<float*>(S.cand), fcorr);
      float e_warm = 0.f, e_plain = 0.f;
#pragma unroll
      for (int s = 0; s < WPL; ++s) {
        const int i = lane + 32 * s;
        if (i >= 1 && i < W) {
          float qp[kMaxDof], qw[kMaxDof];
          interp(q0, q1, i, W, dof, qp);
          const float t = (float)i / (float)(W - 1);
#pragma unroll
          for (int k = 0; k < kMaxDof; ++k)
            qw[k] = k < dof ? fminf(fmaxf(fmaf(t, fcorr[k], qp[k]), rb.j[k].lo), rb.j[k].hi) : 0.f;
          ChainState ch;
          TaskEval<CT> te;
          chain(rb, qp, nullptr, ch);
          te.eval(rb, cs, ch);
          e_plain = fmaxf(e_plain, te.err_inf());
          chain(rb, qw, nullptr, ch);
          te.eval(rb, cs, ch);
          e_warm = fmaxf(e_warm, te.err_inf());
        }
      }
      const unsigned gate = 2u * (unsigned)(W - 1);
      work.proj += gate;
      wc.updates += gate;
      wc.warm_tried += 1u;
      first_pass = warp_max(e_warm) < warp_max(e_plain) ? 0 : 1;
    }
  }
  for (int pass = first_pass; pass < 2; ++pass) {
#pragma unroll
    for (int s = 0; s < WPL; ++s) {
      const int i = min(lane + 32 * s, W - 1);
      interp(q0, q1, i, W, dof, q[s]);
      if (WARM && pass == 0 && i > 0) {
        const float t = (float)i / (float)(W - 1);
#pragma unroll
        for (int k = 0; k < kMaxDof; ++k)
          if (k < dof) q[s][k] = fminf(fmaxf(fmaf(t, fcorr[k], q[s][k]), rb.j[k].lo), rb.j[k].hi);
      }
    }
    if constexpr (SEQ)
      pr = project_sequential<CT, WPL>(rb, cs, max_iters, q0, q1, q, W, tau);
    else
      pr = project_warp<CT, WPL>(rb, cs, pass == 0 ? warm_refine : max_iters, q, W, tau, S.wq);
    __syncwarp();
    work.proj += (unsigned)pr.updates;
    wc.updates += (unsigned)pr.updates;
    if (pass == 0 && pr.status == kValid) {
      wc.warm_used += 1u;
      break;
    }
  }
  if (pr.status != kValid) return kProjFail;
  int ff = collide_motion<WPL>(rb, sc, obs, S, q, W, 1, true, wc, true, !SEQ && CT != kConsNone);
  __syncwarp();
  work.cc += (unsigned)(ff >= 0 ? ff : W - 1);
  if (ff < 0 && self && self->on) {
    // the robot against itself on waypoints 1..W-1 (joint terms in the collision cache)
    bool h = false;
#pragma unroll
    for (int s = 0; s < WPL; ++s) {
      const int i = lane + 32 * s;
      if (i >= 1 && i < W && !h)
        h = self_hit_waypoint(rb.dof, S.jnt, S.bnd, S.sph, S.foff, S.wq + i * 9, *self);
    }
    wc.chains += (unsigned)(W - 1);
    if (__any_sync(kFull, h)) ff = 1;
  }
  return ff >= 0 ? kCollision : kValid;
}

// validate_motion for a motion of 33..64 waypoints held by a warp pair (see SplitX), this warp
// being half h: the same verdict as validate_motion<CT, 2> on the motion (Alg. 1 in step over
// the exchange area, each warp checking its own waypoints, the collision verdict through
// x->hit with generation gen), returned identically in both warps, and with a valid motion
// its last waypoint in x->qend. Work counts: Alg. 1 updates by half 0, collision work by each
// half for its part. No learned form, no sequential projection.
template <int CT>
__device__ __forceinline__ int validate_motion_pair(const RobotDev& rb, const SceneDev& sc,
                                                    const ConsDev& cs, int max_iters,
                                                    MotionWork& work, WorkCount& wc,
                                                    const float4* obs, const CcShared& S,
                                                    const float* q0, const float* q1, int W,
                                                    float (&q)[1][kMaxDof], const SelfMask* self,
                                                    int h, SplitX* x, int bar, int gen) {
  const int lane = threadIdx.x & 31;
  const int dof = rb.dof;
  const int i = 32 * h + lane;
  const float tau = step_threshold(cs, q0, q1, W, dof);
  interp(q0, q1, min(i, W - 1), W, dof, q[0]);
  const ProjResult pr = project_pair<CT>(rb, cs, max_iters, q, W, tau, S.wq, h, x, bar, q0, q1);
  __syncwarp();
  if (h == 0) {
    work.proj += (unsigned)pr.updates;
    wc.updates += (unsigned)pr.updates;
  }
  if (pr.status != kValid) return kProjFail;  // both halves, from the same exchange
  if (i == W - 1) {
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) x->qend[k] = k < dof ? q[0][k] : 0.f;
  }
  const int lo = max(1, 32 * h), hi = min(W, 32 * h + 32);  // this half's waypoints
  int ff = collide_motion<1, true>(rb, sc, obs, S, q, W, 1, true, wc, true, CT != kConsNone,
                                   32 * h, x, gen);
  __syncwarp();
  work.cc += (unsigned)(ff >= 0 ? ff - lo + 1 : hi - lo);
  bool hit = ff >= 0;
  if (!hit && self && self->on &&
      !__any_sync(kFull, *reinterpret_cast<volatile int*>(&x->hit) == gen)) {
    const bool hs = i >= 1 && i < W &&
                    self_hit_waypoint(rb.dof, S.jnt, S.bnd, S.sph, S.foff, S.wq + i * 9, *self);
    wc.chains += (unsigned)(hi - lo);
    hit = __any_sync(kFull, hs);
  }
  if (hit && lane == 0) x->hit = gen;
  pair_barrier(bar);
  return x->hit == gen ? kCollision : kValid;
}

// validate_motion for a motion of at most 32 waypoints held by a warp pair split by obstacles,
// this warp being half h: both warps run Alg. 1 on the whole motion (the same instructions on
// the same inputs, so the same segment), each checks the chunks c with c mod 2 = h, and the
// verdict goes through x->hit as in validate_motion_pair; it is that of
// validate_motion<CT, 1>. Self-collision is checked by half 0 alone. Work counts: Alg. 1
// updates and swept bounds by half 0, the listing and chain walks by each half for its part.
template <int CT>
__device__ __forceinline__ int validate_motion_osplit(const RobotDev& rb, const SceneDev& sc,
                                                      const ConsDev& cs, int max_iters,
                                                      MotionWork& work, WorkCount& wc,
                                                      const float4* obs, const CcShared& S,
                                                      const float* q0, const float* q1, int W,
                                                      float (&q)[1][kMaxDof], const SelfMask* self,
                                                      int h, SplitX* x, int bar, int gen) {
  const int lane = threadIdx.x & 31;
  const int dof = rb.dof;
  const float tau = step_threshold(cs, q0, q1, W, dof);
  interp(q0, q1, min(lane, W - 1), W, dof, q[0]);
  const ProjResult pr = project_warp<CT, 1>(rb, cs, max_iters, q, W, tau, S.wq);
  __syncwarp();
  if (h == 0) {
    work.proj += (unsigned)pr.updates;
    wc.updates += (unsigned)pr.updates;
  }
  if (pr.status != kValid) return kProjFail;  // both halves: the same projection
  int ff = collide_motion<1, false, 2>(rb, sc, obs, S, q, W, 1, true, wc, true, CT != kConsNone,
                                       0, x, gen, h);
  __syncwarp();
  work.cc += (unsigned)(ff >= 0 ? ff : W - 1);
  bool hit = ff >= 0;
  if (h == 0 && !hit && self && self->on &&
      !__any_sync(kFull, *reinterpret_cast<volatile int*>(&x->hit) == gen)) {
    const bool hs = lane >= 1 && lane < W &&
                    self_hit_waypoint(rb.dof, S.jnt, S.bnd, S.sph, S.foff, S.wq + lane * 9, *self);
    wc.chains += (unsigned)(W - 1);
    hit = __any_sync(kFull, hs);
  }
  if (hit && lane == 0) x->hit = gen;
  pair_barrier(bar);
  return x->hit == gen ? kCollision : kValid;
}

// How the warps of a worker share its motions: one warp (kSplitNone), or a pair split by
// waypoints (W = 33..64) or by obstacles (W <= 32).
enum : int { kSplitNone = 0, kSplitWaypoints = 1, kSplitObstacles = 2 };

// Register cap of the planner kernel (0: the compiler's choice). Fewer registers let more
// 8-warp CTAs share an SM at the price of some spills.
#ifndef CPRRTC_PLAN_MAXNREG
#define CPRRTC_PLAN_MAXNREG 0
#endif
#if CPRRTC_PLAN_MAXNREG > 0
#define CPRRTC_PLAN_REGS __maxnreg__(CPRRTC_PLAN_MAXNREG)
#else
#define CPRRTC_PLAN_REGS
#endif


// The planner for one problem, run by the whole CTA (one warp per worker, or with SPLIT a warp
// pair per worker, its motions split by waypoints or by obstacles, see SplitX; the pairs'
// exchange areas xs[worker]). Shared memory (robot tables, obstacles, per-warp scratch) is
// staged by the caller. Both warps of a pair follow the same chain (identical copies of its
// state, computed from identical inputs); the pair's half 0 writes the worker's shared flags,
// tree nodes and path, and a motion's edge is written by the warps holding its waypoints
// (each its half when split by waypoints, half 0 when split by obstacles).
//
// Slices (ps set, one warp per worker): the call runs rounds [r_begin, r_end) of the problem
// (r_begin > 0 resumes from the state in *ps). It returns false, with the problem's state saved
// back to *ps, if rounds remain after r_end; otherwise it writes the problem's outputs and
// returns true. The rounds are those of one uninterrupted call: the state holds everything a
// round reads besides the trees in global memory, and the Philox counter names the round.
template <int CT, int WPL, bool SEQ = false, bool WARM = false, int SPLIT = kSplitNone>
__device__ __forceinline__ bool plan_problem(const RobotDev& rb, const SceneDev& sc,
                                             const float4* obs, const ConsDev& cs,
                                             const PlanArgs& a, const ProblemView& P,
                                             const CcShared& S, PlanShared* sh,
                                             WorkCount& wc, const SelfMask& self,
                                             const MlpView* net = nullptr, SplitX* xs = nullptr,
                                             int r_begin = 0, int r_end = 0x7fffffff,
                                             bool sliced = false) {
  static_assert(SPLIT == kSplitNone || (WPL == 1 && !SEQ && !WARM), "warp pairs: plain Alg. 1, one waypoint per lane");
  constexpr int K = SPLIT == kSplitNone ? 1 : 2;
  const int p = P.p;
  PlanState* const ps = SPLIT == kSplitNone && sliced ? a.state + p : nullptr;
  const bool resume = ps && r_begin > 0;
  const int pw = threadIdx.x >> 5, lane = threadIdx.x & 31;  // physical warp
  const int warp = pw / K, h = pw % K;                        // worker, half of its pair
  const int NW = blockDim.x >> 5, B = NW / K, dof = rb.dof, W = P.W;
  if (threadIdx.x == 0) {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    sh->t_start = t;
    sh->t_prior = resume ? ps->active_ns : 0;
    sh->stop = 0;
  }
  if (K > 1 && threadIdx.x < B) xs[threadIdx.x].hit = 0;

  const size_t wd = (size_t)W * dof;
  const int MN = a.max_nodes;
  // tree t of this problem (computed, not tabulated: a table indexed by t lives in local memory)
  auto nodes = [&](int t) { return P.nodes + (size_t)t * MN * 8; };
  auto parent = [&](int t) { return P.parent + (size_t)t * MN; };
  auto edges = [&](int t) { return P.edges + (size_t)t * MN * wd; };
  // per-worker global scratch: the closing hop's motion is kept at wedge + wd
  float* wedge = P.pend_edges + (size_t)warp * 2 * wd;

  if (resume) {
    if (threadIdx.x == 0) {
      sh->count0[0] = ps->cnt[0];
      sh->count0[1] = ps->cnt[1];
    }
  } else if (pw == 0) {
    float q[kMaxDof];
    load_cfg(P.start, dof, q);
    store_cfg(nodes(0), q, dof);
    load_cfg(P.goal, dof, q);
    store_cfg(nodes(1), q, dof);
    if (lane == 0) {
      parent(0)[0] = -1;
      parent(1)[0] = -1;
      sh->count0[0] = 1;
      sh->count0[1] = 1;
    }
  }
  __syncthreads();
  // tree sizes when the round began: every warp keeps its own copy, advanced from the
  // round's shared flags (identically in every warp)
  int cnt0 = sh->count0[0], cnt1 = sh->count0[1];
  auto count_of = [&](int t) { return t ? cnt1 : cnt0; };
  const float connect_radius = 10.f * cs.tau_floor;
  unsigned wp = 0;
  MotionWork work{0u, 0u};
  int rounds_used = 0, win = -1;
  // chain state (warp-uniform): 0 extend, 1 connect, 2 closing hop
  int mode = 0, ta = 0, last = 0, target = -1, steps = 0;
  float* cur = sh->cfg[pw][0];
  float* qt = sh->cfg[pw][1];
  float* q1 = sh->cfg[pw][2];
  float* qe = sh->cfg[pw][3];
  if (resume) {  // the chain as the last slice left it
    mode = ps->mode[warp];
    ta = ps->ta[warp];
    last = ps->last[warp];
    target = ps->target[warp];
    steps = ps->steps[warp];
    wp = ps->wp[warp];
    work.proj = ps->proj[warp];
    work.cc = ps->cc[warp];
    rounds_used = r_begin;
    __syncwarp();
    if (lane < 8) {
      cur[lane] = ps->cur[warp][lane];
      qt[lane] = ps->qt[warp][lane];
    }
    __syncwarp();
  }
  const int r_stop = min(r_end, a.max_rounds);
  for (int r = resume ? r_begin : 0; r < r_stop; ++r) {
    if (mode == 0) {
      ta = (r + warp) & 1;
      const U32x4 u0 = philox4x32_10(U32x4{(uint32_t)p, (uint32_t)r, (uint32_t)warp, 0u}, a.seed, 0u);
      const U32x4 u1 = philox4x32_10(U32x4{(uint32_t)p, (uint32_t)r, (uint32_t)warp, 1u}, a.seed, 0u);
      const uint32_t w8[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
      float v = 0.f;
#pragma unroll
      for (int k = 0; k < kMaxDof; ++k)  // lane k takes word k (no dynamic register index)
        if (k == lane && k < dof) v = fmaf(u24(w8[k]), rb.j[k].hi - rb.j[k].lo, rb.j[k].lo);
      __syncwarp();
      if (lane < 8) qe[lane] = v;  // the sample, in the scratch slot
      __syncwarp();
      last = nearest_warp(nodes(ta), count_of(ta), qe, dof);
      copy_cfg(cur, nodes(ta) + (size_t)last * 8, dof);
      steer(cur, qe, a.range, dof, q1);
    } else if (mode == 1) {
      steer(cur, qt, a.range, dof, q1);
    } else {
      copy_cfg(q1, qt, dof);
    }
    float q[WPL][kMaxDof];
    // the closing hop is checked as it stands (one Alg. 1 iteration); the learned form
    // warm-starts extend motions only: connect steps and the closing hop head for a node on
    // the manifold
    int st;
    const int iters = mode == 2 ? 1 : cs.max_iters;
    if constexpr (SPLIT == kSplitNone) {
      st = validate_motion<CT, WPL, SEQ, WARM>(rb, sc, cs, iters, work, wc, obs, S, cur, q1, W, q,
                                               WARM && mode == 0 ? net : nullptr,
                                               a.warm_refine, qe, &self);
    } else if constexpr (SPLIT == kSplitWaypoints) {
      st = validate_motion_pair<CT>(rb, sc, cs, iters, work, wc, obs, S, cur, q1, W, q, &self, h,
                                    xs + warp, 1 + warp, r + 1);
    } else {
      st = validate_motion_osplit<CT>(rb, sc, cs, iters, work, wc, obs, S, cur, q1, W, q, &self, h,
                                      xs + warp, 1 + warp, r + 1);
    }
    // this warp's part of an edge: its waypoints (every waypoint, or none for half 1 of an
    // obstacle split)
    auto store_mine = [&](float* dst) {
      if (SPLIT != kSplitObstacles || h == 0)
        store_edge<WPL>(dst, q, W, dof, SPLIT == kSplitWaypoints ? 32 * h : 0);
    };
    wp += W;
    int add = 0, conn = 0;
    if (st == kValid) {
      if (mode == 2) {
        conn = 1;
        store_mine(wedge + wd);
      } else {
        if constexpr (SPLIT != kSplitWaypoints) {
          last_waypoint<WPL>(q, W, dof, qe);
        } else {
          __syncwarp();  // the pair barrier made x->qend visible
          if (lane < 8) qe[lane] = xs[warp].qend[lane];
          __syncwarp();
        }
        bool accept = true;
        if (mode == 0) {
          target = nearest_warp(nodes(ta ^ 1), count_of(ta ^ 1), qe, dof);
          copy_cfg(qt, nodes(ta ^ 1) + (size_t)target * 8, dof);
        } else {
          accept = dist2(qe, qt, dof) < dist2(cur, qt, dof);
        }
        // an accepted node stays in qe (shared) and its motion in q (registers) until its
        // index in the tree is known after the barrier
        add = accept ? 1 : 0;
      }
    }
    if (lane == 0 && h == 0) {
      sh->padd[warp] = add;
      sh->ptree[warp] = ta;
      sh->pparent[warp] = last;
      sh->ptarget[warp] = target;
      sh->pconn[warp] = conn;
    }
    __syncthreads();
    rounds_used = r + 1;
    win = -1;
    for (int w = 0; w < B; ++w)
      if (sh->pconn[w]) {
        win = w;
        break;
      }
    if (win >= 0) break;
    // append this round's nodes in warp order
    int dst = -1;
    if (add) {
      int off = 0;
      for (int w = 0; w < warp; ++w)
        if (sh->padd[w] && sh->ptree[w] == ta) ++off;
      dst = count_of(ta) + off;
      if (dst < a.max_nodes) {
        if (lane < 8 && h == 0) nodes(ta)[(size_t)dst * 8 + lane] = qe[lane];
        store_mine(edges(ta) + (size_t)dst * wd);
        if (lane == 0 && h == 0) parent(ta)[dst] = last;
      } else {
        dst = -1;
      }
    }
    {
      int n_add0 = 0, n_add1 = 0;
      for (int w = 0; w < B; ++w)
        if (sh->padd[w]) (sh->ptree[w] ? n_add1 : n_add0) += 1;
      cnt0 = min(cnt0 + n_add0, a.max_nodes);
      cnt1 = min(cnt1 + n_add1, a.max_nodes);
    }
    // optional time budget: decided by one thread, seen by all after the barrier (earlier
    // slices' device time included)
    if (a.budget_ns && threadIdx.x == 0) {
      long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if ((unsigned long long)(t - sh->t_start + (ps ? sh->t_prior : 0)) > a.budget_ns) sh->stop = 1;
    }
    // the appended nodes are visible to every warp's next nearest-neighbour scan, and the
    // flags may be overwritten
    __syncthreads();
    if (sh->stop) break;
    // next motion of the chain
    if (dst >= 0) {
      last = dst;
      copy_cfg(cur, qe, dof);
      float gap = 0.f;
#pragma unroll
      for (int k = 0; k < kMaxDof; ++k)
        if (k < dof) gap = fmaxf(gap, fabsf(cur[k] - qt[k]));
      if (gap <= connect_radius) {
        mode = 2;
      } else if (steps < a.max_connect) {
        mode = 1;
        ++steps;
      } else {
        mode = 0;
        steps = 0;
      }
    } else {
      mode = 0;
      steps = 0;
    }
  }
  if (SPLIT == kSplitNone && ps && win < 0 && !sh->stop && rounds_used < a.max_rounds) {
    // rounds remain: save the chain for the next slice (tree appends are in global memory)
    if (lane == 0) {
      ps->mode[warp] = mode;
      ps->ta[warp] = ta;
      ps->last[warp] = last;
      ps->target[warp] = target;
      ps->steps[warp] = steps;
      ps->wp[warp] = wp;
      ps->proj[warp] = work.proj;
      ps->cc[warp] = work.cc;
    }
    if (lane < 8) {
      ps->cur[warp][lane] = cur[lane];
      ps->qt[warp][lane] = qt[lane];
    }
    if (threadIdx.x == 0) {
      ps->r_next = rounds_used;
      ps->cnt[0] = cnt0;
      ps->cnt[1] = cnt1;
      long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (!resume) ps->t_first = sh->t_start;
      ps->active_ns = sh->t_prior + (t - sh->t_start);
    }
    __syncthreads();
    return false;
  }
  if (lane == 0) {  // per physical warp: a pair's half 1 adds its collision work only
    sh->wp[pw] = h == 0 ? wp : 0;
    sh->wproj[pw] = work.proj;
    sh->wcc[pw] = work.cc;
  }

  if (win >= 0 && warp == win && h == 0) {
    // path: root_a .. last, closing hop, target .. root_b; reversed when tree a is the
    // goal tree
    const int tb = ta ^ 1;
    int len_a = 0, len_b = 0;
    for (int v = last; v >= 0; v = parent(ta)[v]) ++len_a;
    for (int v = target; v >= 0; v = parent(tb)[v]) ++len_b;
    const int total = len_a + len_b;
    const bool flip = ta == 1;
    const int os = P.ostride;
    const size_t we = (size_t)P.estride;  // floats per output edge
    float* path = P.path;
    float* pe = P.path_edges;
    if (total <= a.max_path) {
      int pos = len_a - 1;
      for (int v = last; v >= 0; v = parent(ta)[v], --pos) {
        const int np = flip ? total - 1 - pos : pos;
        copy_warp(path + (size_t)np * os, nodes(ta) + (size_t)v * 8, os);
        if (pe && parent(ta)[v] >= 0) {  // edge pos-1 -> pos is v's incoming motion
          const int e = flip ? total - 1 - pos : pos - 1;
          copy_edge(pe + (size_t)e * we, edges(ta) + (size_t)v * wd, W, dof, os, flip);
        }
      }
      if (pe) {  // closing hop: last -> target
        const int e = flip ? total - 1 - len_a : len_a - 1;
        copy_edge(pe + (size_t)e * we, wedge + wd, W, dof, os, flip);
      }
      pos = len_a;
      for (int v = target; v >= 0; v = parent(tb)[v], ++pos) {
        const int np = flip ? total - 1 - pos : pos;
        copy_warp(path + (size_t)np * os, nodes(tb) + (size_t)v * 8, os);
        if (pe && parent(tb)[v] >= 0) {  // edge pos -> pos+1 is v's incoming motion reversed
          const int e = flip ? total - 2 - pos : pos;
          copy_edge(pe + (size_t)e * we, edges(tb) + (size_t)v * wd, W, dof, os, !flip);
        }
      }
    }
    if (lane == 0) a.path_len[p] = total <= a.max_path ? total : -total;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (win < 0) a.path_len[p] = 0;
    long long total_wp = 0, tp = 0, tc = 0;
    for (int w = 0; w < NW; ++w) {
      total_wp += sh->wp[w];
      tp += sh->wproj[w];
      tc += sh->wcc[w];
    }
    if (a.rounds) a.rounds[p] = rounds_used;
    if (a.waypoints) a.waypoints[p] = total_wp;
    if (a.work) {
      a.work[2 * p] = tp;
      a.work[2 * p + 1] = tc;
    }
    long long t_end;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
    // plan time: the device time of the problem's slices (one slice without a queue)
    const long long prior = ps ? sh->t_prior : 0;
    if (a.plan_ms) a.plan_ms[p] = (float)((double)(t_end - sh->t_start + prior) * 1e-6);
    if (a.span) {
      a.span[2 * p] = resume ? ps->t_first : sh->t_start;
      a.span[2 * p + 1] = t_end;
    }
  }
  return true;
}

// ---- the time-sliced schedule's queue (see PlanQueue) ---------------------------------------

__device__ __forceinline__ long long ld_acquire(const long long* p) {
  long long v;
  asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(long long* p, long long v) {
  asm volatile("st.release.gpu.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// Thread 0: waits until seq[slot] = want (bounded; false and status set on timeout).
__device__ bool queue_wait(const long long* seq, unsigned long long slot, long long want,
                           unsigned long long wait_ns, int* status) {
  const unsigned long long limit = wait_ns ? wait_ns : 1000000000ull;
  long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (ld_acquire(seq + slot) != want) {
    long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if ((unsigned long long)(t1 - t0) > limit) {
      if (status) atomicExch(status, 1);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

// Thread 0: the next problem, or -1 when no problem waits (the CTA then ends: every problem
// left is held by a running CTA, which keeps it). *fresh is set when the problem has not
// started. A ticket is taken only while a problem waits for it, so no pushed problem is ever
// left without a taker, and the ticket's retries are bounded too.
__device__ int queue_pop(PlanQueue* q, int n, unsigned long long wait_ns, int* status,
                         bool* fresh) {
  const unsigned long long un = (unsigned long long)n;
  unsigned long long t = 0;
  bool got = false;
  for (int tries = 0; tries < (1 << 22) && !got; ++tries) {
    const unsigned long long h = ld_volatile(&q->head);
    const unsigned long long tl = ld_volatile(&q->tail);
    if (h >= un && h - un >= tl) return -1;
    if (atomicCAS(&q->head, h, h + 1ull) == h) {
      t = h;
      got = true;
    }
  }
  if (!got) {
    if (status) atomicExch(status, 1);
    return -1;
  }
  *fresh = t < un;
  if (t < un) return (int)t;
  long long* seq = reinterpret_cast<long long*>(q + 1);
  const int* ring = reinterpret_cast<const int*>(seq + n);
  const unsigned long long u = t - un, slot = u % un, lap = u / un;
  if (!queue_wait(seq, slot, (long long)(2 * lap + 1), wait_ns, status)) return -1;
  const int p = ring[slot];
  st_release(seq + slot, (long long)(2 * lap + 2));  // the slot is free for the next lap
  return p;
}

// Thread 0, after a barrier that follows every write of the problem's slice: problem p to
// the queue's tail. False (status set) if the slot did not come free in time; the caller then
// keeps the problem.
__device__ bool queue_push(PlanQueue* q, int n, int p, unsigned long long wait_ns, int* status) {
  long long* seq = reinterpret_cast<long long*>(q + 1);
  int* ring = reinterpret_cast<int*>(seq + n);
  __threadfence();
  const unsigned long long un = (unsigned long long)n;
  const unsigned long long u = atomicAdd(&q->tail, 1ull), slot = u % un, lap = u / un;
  if (!queue_wait(seq, slot, (long long)(2 * lap), wait_ns, status)) return false;
  ring[slot] = p;
  st_release(seq + slot, (long long)(2 * lap + 1));
  return true;
}

// Thread 0: a problem waits in the queue (one not started, or one pushed and not taken).
__device__ __forceinline__ bool queue_waiting(PlanQueue* q, int n) {
  const unsigned long long un = (unsigned long long)n;
  const unsigned long long h = ld_volatile(&q->head);
  const unsigned long long tl = ld_volatile(&q->tail);
  return h < un || tl > h - un;
}

// Mean round time of a problem, relative to the launch's, above which it keeps its CTA.
constexpr double kKeepFactor = 1.1;

// Thread 0, after a slice of problem p (rounds r0 .. its next round; `prior`: its device time
// before the slice) that left rounds: p's next holder, -1 when p went back to the queue. A problem whose
// rounds take longer than the launch's mean by kKeepFactor keeps its CTA: the job ends with
// the problems of most remaining time, and round-robin would stretch those most. The others
// go back to the queue's tail while problems wait. Out of line, so that the planner's
// register allocation does not carry it.
__device__ __noinline__ int after_slice(const PlanArgs& a, int p, int r0, long long prior) {
  const PlanState& ps = a.state[p];
  const unsigned long long sum_ns = atomicAdd(&a.queue->sum_ns, (unsigned long long)(ps.active_ns - prior));
  const unsigned long long sum_r = atomicAdd(&a.queue->sum_rounds, (unsigned long long)(ps.r_next - r0));
  const bool slow = sum_r > 0 && (double)ps.active_ns * (double)sum_r >=
                                     kKeepFactor * (double)sum_ns * (double)ps.r_next;
  if (!slow && queue_waiting(a.queue, a.n) && queue_push(a.queue, a.n, p, a.wait_ns, a.status)) return -1;
  return p;
}

// One CTA per problem (no queue), or persistent CTAs on the time-sliced queue: a CTA takes a
// problem, runs its next slice, and either keeps it (nothing waits), hands it to the queue's
// tail (other problems wait), or takes the next one once it is done. Problems that end within
// their first slice plan in one stretch; the ones that run long share the SMs round-robin, so
// the job no longer ends with the long problems that happened to start last.
template <int CT, int WPL, bool SEQ, bool WARM>
__device__ __forceinline__ void plan_kernel_body(const RobotDev& rb, const SceneDev& shared_scene,
                                                 const ConsDev& cs, const PlanArgs& a) {
  const bool queued = a.queue != nullptr;
  if (!queued && (int)blockIdx.x >= a.n) return;
  __shared__ int s_p, s_r0, s_held, s_staged, s_restage;
  const int warp = threadIdx.x >> 5;
  const int B = a.workers, dof = rb.dof, W = a.W;
  extern __shared__ __align__(16) char smem[];
  const SmemLayout L(a.stage_obs ? a.max_scene_f4 : 0, rb.n_spheres, W, B, sizeof(PlanShared));
  float4* s_obs = reinterpret_cast<float4*>(smem + L.obs);
  stage_robot(rb, smem, L);
  const CcShared S = cc_shared(smem, L, warp);
  PlanShared* sh = reinterpret_cast<PlanShared*>(smem + L.extra);
  WorkCount wc{};
  const size_t wd = (size_t)W * dof;
  SelfMask self;
#pragma unroll
  for (int f = 0; f <= kMaxDof; ++f) self.rows[f] = a.self_on ? a.self_rows[f] : (unsigned short)0;
  self.on = a.self_on;
  // s_held: the problem this CTA keeps for its next slice (-1: none; -2: the CTA's one problem
  // without a queue is done); s_staged: the problem whose scene is in shared memory
  if (threadIdx.x == 0) {
    s_held = -1;
    s_staged = -1;
  }
  for (;;) {
    __syncthreads();  // shared memory is free for the next slice
    if (threadIdx.x == 0) {
      int p = -1, r0 = 0;
      const int held = s_held;
      if (!queued) {
        p = held == -1 ? (int)blockIdx.x : -1;
        s_held = -2;
      } else if (held >= 0) {
        p = held;
        r0 = a.state[p].r_next;
      } else {
        bool fresh = true;
        p = queue_pop(a.queue, a.n, a.wait_ns, a.status, &fresh);
        if (p >= 0 && !fresh) r0 = a.state[p].r_next;
      }
      s_p = p;
      s_r0 = r0;
      // decided here, before the barrier, so that no thread reads s_staged while it changes
      s_restage = p >= 0 && (s_staged < 0 || (a.scenes && s_staged != p));
      if (p >= 0) s_staged = p;
    }
    __syncthreads();
    const int p = s_p, r0 = s_r0;
    if (p < 0) break;
    SceneDev sc = shared_scene;
    if (a.scenes) {
      const int4 d = a.scenes[p];
      sc.obs = a.scene_obs + d.x;
      sc.n_sph = d.y;
      sc.n_box = d.z;
      sc.n_cap = d.w;
    }
    if (a.stage_obs && s_restage) {
      const int n4 = sc.n_float4();
      for (int i = threadIdx.x; i < n4; i += blockDim.x) s_obs[i] = sc.obs[i];
    }
    const float4* obs = a.stage_obs ? s_obs : sc.obs;
    const size_t tree0 = (size_t)p * 2 * a.max_nodes;  // first node slot of this problem
    if (threadIdx.x == 0) {
      ProblemView& P = sh->pv;
      P.p = p;
      P.start = a.start + (size_t)p * dof;
      P.goal = a.goal + (size_t)p * dof;
      P.W = W;
      P.nodes = a.nodes + tree0 * 8;
      P.parent = a.parent + tree0;
      P.edges = a.edges + tree0 * wd;
      P.pend = a.pend + (size_t)p * B * 8;
      P.pend_edges = a.pend_edges + (size_t)p * B * 2 * wd;
      P.path = a.path + (size_t)p * a.max_path * dof;
      P.path_edges = a.path_edges ? a.path_edges + (size_t)p * (a.max_path - 1) * wd : nullptr;
      P.ostride = dof;
      P.estride = (int)wd;
    }
    __syncthreads();
    int r1 = a.max_rounds;
    if (queued) {
      const int sl = r0 == 0 ? a.first_slice : a.slice;
      r1 = sl >= a.max_rounds - r0 ? a.max_rounds : r0 + sl;
    }
    const bool done = plan_problem<CT, WPL, SEQ, WARM>(rb, sc, obs, cs, a, sh->pv, S, sh, wc, self,
                                                       WARM ? &a.net : nullptr, nullptr, r0, r1,
                                                       queued);
    if (queued && threadIdx.x == 0) s_held = done ? -1 : after_slice(a, p, s_r0, sh->t_prior);
  }
  wc.flush(a.work_counters);
}

template <int CT, int WPL, bool SEQ = false>
__global__ void CPRRTC_PLAN_REGS plan_kernel(RobotDev rb, SceneDev shared_scene, ConsDev cs,
                                             PlanArgs a) {
  plan_kernel_body<CT, WPL, SEQ, false>(rb, shared_scene, cs, a);
}

// The learned form, held to two CTAs of 8 warps per SM (the network's evaluation otherwise
// takes registers that halve the warps an SM holds).
template <int CT, int WPL>
__global__ void __launch_bounds__(256, 2) plan_warm_kernel(RobotDev rb, SceneDev shared_scene,
                                                           ConsDev cs, PlanArgs a) {
  plan_kernel_body<CT, WPL, false, true>(rb, shared_scene, cs, a);
}

// ---- persistent batch of uneven problems --------------------------------------------------
//
// One persistent kernel per (constraint type, waypoints per lane) class, each specialised and
// register-allocated for its class; the host launches the classes concurrently. A class's
// grid of (SMs x CTAs per SM) CTAs dequeues its problems from an atomic counter in a given
// order (longest expected first). Each problem names its robot, constraint, scene and W; the
// CTA stages that robot and scene into shared memory and runs plan_problem. Trees live in a
// per-CTA scratch slot reused across problems.
// With WARM (the learned form), problems whose robot and constraint have a network in the
// table warm-start their extend motions with it; the others plan as without it.
// Bytes after the per-warp areas: the planner's shared state, and with warp pairs their
// exchange areas (one per worker).
__host__ __device__ constexpr size_t plan_extra_bytes(int K) {
  return ((sizeof(PlanShared) + 15) & ~size_t(15)) + (K > 1 ? sizeof(SplitX) * kMaxWorkers / 2 : 0);
}

template <int CT, int WPL, bool WARM, int SPLIT = kSplitNone>
__device__ __forceinline__ void plan_batch_body(const BatchArgs& b, const BatchTables& T) {
  constexpr int K = SPLIT == kSplitNone ? 1 : 2;
  extern __shared__ __align__(16) char smem[];
  __shared__ SceneDev s_sc;
  __shared__ int s_t, s_robot, s_cons;
  const PlanArgs& a = b.a;
  const int NW = blockDim.x >> 5, B = NW / K;  // warps, workers
  const int warp = threadIdx.x >> 5;
  const SmemLayout L(a.stage_obs ? a.max_scene_f4 : 0, b.max_S, b.max_W, NW, plan_extra_bytes(K));
  PlanShared* sh = reinterpret_cast<PlanShared*>(smem + L.extra);
  SplitX* xs = K > 1 ? reinterpret_cast<SplitX*>(smem + L.extra + plan_extra_bytes(1)) : nullptr;
  const CcShared S = cc_shared(smem, L, warp);
  float4* s_obs = reinterpret_cast<float4*>(smem + L.obs);
  WorkCount wc{};
  const size_t MN = (size_t)a.max_nodes, ew = (size_t)b.max_W * 8;  // edge floats (max)
  const size_t slot = blockIdx.x;
  for (;;) {
    __syncthreads();  // the previous problem is done with shared memory
    if (threadIdx.x == 0) s_t = (int)atomicAdd(b.counter, 1u);
    __syncthreads();
    const int t = s_t;
    if (t >= b.n_class) break;
    const int p = b.order[t];
    if (threadIdx.x == 0) {
      const int4 d = b.problems[p];
      s_robot = d.x;
      s_cons = d.y;
      const int4 sd = a.scenes[d.z];
      s_sc = SceneDev{a.scene_obs + sd.x, sd.y, sd.z, sd.w};
      ProblemView& P = sh->pv;
      P.p = p;
      P.start = a.start + (size_t)p * 8;
      P.goal = a.goal + (size_t)p * 8;
      P.W = d.w;
      P.nodes = b.nodes + slot * 2 * MN * 8;
      P.parent = b.parent + slot * 2 * MN;
      P.edges = b.edges + slot * 2 * MN * ew;
      P.pend = b.pend + slot * B * 8;
      P.pend_edges = b.pend_edges + slot * B * 2 * ew;
      const size_t oew = (size_t)b.out_max_W * 8;  // output edge floats: the batch's largest W
      P.path = a.path + (size_t)p * a.max_path * 8;
      P.path_edges = a.path_edges ? a.path_edges + (size_t)p * (a.max_path - 1) * oew : nullptr;
      P.ostride = 8;
      P.estride = (int)oew;
    }
    __syncthreads();
    // robot and constraint tables are read from the constant bank (kernel parameter)
    const RobotDev& rb = T.robots[s_robot];
    const ConsDev& cs = T.cons[s_cons];
    const int n4 = s_sc.n_float4();
    if (a.stage_obs)
      for (int i = threadIdx.x; i < n4; i += blockDim.x) s_obs[i] = s_sc.obs[i];
    stage_robot(rb, smem, L);
    __syncthreads();
    const SceneDev sc = s_sc;  // in registers: the collision walk reads it in its inner loops
    const SelfMask self = T.self[s_robot];
    const MlpView* net = WARM && T.nets[s_robot][s_cons].dof ? &T.nets[s_robot][s_cons] : nullptr;
    plan_problem<CT, WPL, false, WARM, SPLIT>(rb, sc, a.stage_obs ? s_obs : sc.obs, cs, a, sh->pv, S,
                                              sh, wc, self, net, xs);
  }
  wc.flush(a.work_counters);
}

template <int CT, int WPL>
__global__ void plan_batch_kernel(BatchArgs b, const __grid_constant__ BatchTables T) {
  plan_batch_body<CT, WPL, false>(b, T);
}

// The learned form of a class, held to two CTAs of 8 warps per SM like plan_warm_kernel.
template <int CT, int WPL>
__global__ void __launch_bounds__(256, 2) plan_batch_warm_kernel(BatchArgs b,
                                                                 const __grid_constant__ BatchTables T) {
  plan_batch_body<CT, WPL, true>(b, T);
}

// A class with a warp pair per worker, split by waypoints (33..64 waypoints, one per lane) or
// by obstacles (up to 32 waypoints): up to 16 warps, held to the 128 registers that let them
// share one SM.
template <int CT, int SPLIT>
__global__ void __launch_bounds__(512, 1) plan_batch_pair_kernel(BatchArgs b,
                                                                 const __grid_constant__ BatchTables T) {
  plan_batch_body<CT, 1, false, SPLIT>(b, T);
}

static const void* plan_batch_fn(int cls, bool warm = false, int K = 1) {
  if (K == 2) {  // warp pairs, plain form
    switch (cls) {
      case 0: return (const void*)plan_batch_pair_kernel<kConsNone, kSplitObstacles>;
      case 1: return (const void*)plan_batch_pair_kernel<kConsNone, kSplitWaypoints>;
      case 2: return (const void*)plan_batch_pair_kernel<kConsRollPitch, kSplitObstacles>;
      case 3: return (const void*)plan_batch_pair_kernel<kConsRollPitch, kSplitWaypoints>;
      case 4: return (const void*)plan_batch_pair_kernel<kConsZPlane, kSplitObstacles>;
      default: return (const void*)plan_batch_pair_kernel<kConsZPlane, kSplitWaypoints>;
    }
  }
  if (warm) {  // the learned form of the roll-pitch and z-plane classes
    switch (cls) {
      case 2: return (const void*)plan_batch_warm_kernel<kConsRollPitch, 1>;
      case 3: return (const void*)plan_batch_warm_kernel<kConsRollPitch, 2>;
      case 4: return (const void*)plan_batch_warm_kernel<kConsZPlane, 1>;
      case 5: return (const void*)plan_batch_warm_kernel<kConsZPlane, 2>;
      default: break;
    }
  }
  switch (cls) {
    case 0: return (const void*)plan_batch_kernel<kConsNone, 1>;
    case 1: return (const void*)plan_batch_kernel<kConsNone, 2>;
    case 2: return (const void*)plan_batch_kernel<kConsRollPitch, 1>;
    case 3: return (const void*)plan_batch_kernel<kConsRollPitch, 2>;
    case 4: return (const void*)plan_batch_kernel<kConsZPlane, 1>;
    default: return (const void*)plan_batch_kernel<kConsZPlane, 2>;
  }
}

size_t plan_batch_smem_bytes(int max_scene_f4, int max_S, int max_W, int workers, bool stage, int K) {
  return SmemLayout(stage ? max_scene_f4 : 0, max_S, max_W, workers * K, plan_extra_bytes(K)).total;
}

int plan_batch_occupancy(int cls, int workers, size_t smem, bool warm, int K) {
  const void* fn = plan_batch_fn(cls, warm, K);
  int per_sm = 0;
  if (!fn) return 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * workers * K, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm;
}

cudaError_t launch_plan_batch(int cls, BatchArgs b, const BatchTables& T, int grid, size_t smem,
                              int K, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(b.counter, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  const void* fn = plan_batch_fn(cls, b.a.warm_refine > 0, K);
  if (!fn) return cudaErrorNotSupported;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {&b, const_cast<BatchTables*>(&T)};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(32 * b.a.workers * K), args, smem, stream);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

static const void* plan_fn(int ct, int W, bool sequential = false, bool warm = false) {
  const bool two = W > 32;
  if (warm) {  // the learned form: roll-pitch and z-plane
    if (ct == kConsRollPitch)
      return two ? (const void*)plan_warm_kernel<kConsRollPitch, 2>
                 : (const void*)plan_warm_kernel<kConsRollPitch, 1>;
    if (ct == kConsZPlane)
      return two ? (const void*)plan_warm_kernel<kConsZPlane, 2>
                 : (const void*)plan_warm_kernel<kConsZPlane, 1>;
    return nullptr;
  }
  if (sequential) {  // the naive baseline's projection: roll-pitch and z-plane, W <= 32
    if (two) return nullptr;
    if (ct == kConsRollPitch) return (const void*)plan_kernel<kConsRollPitch, 1, true>;
    if (ct == kConsZPlane) return (const void*)plan_kernel<kConsZPlane, 1, true>;
    return nullptr;
  }
  switch (ct) {
    case kConsRollPitch:
      return two ? (const void*)plan_kernel<kConsRollPitch, 2> : (const void*)plan_kernel<kConsRollPitch, 1>;
    case kConsZPlane:
      return two ? (const void*)plan_kernel<kConsZPlane, 2> : (const void*)plan_kernel<kConsZPlane, 1>;
    case kConsLine:
      return two ? (const void*)plan_kernel<kConsLine, 2> : (const void*)plan_kernel<kConsLine, 1>;
    case kConsOrientPlane:
      return two ? (const void*)plan_kernel<kConsOrientPlane, 2> : (const void*)plan_kernel<kConsOrientPlane, 1>;
    case kConsOrientLine:
      return two ? (const void*)plan_kernel<kConsOrientLine, 2> : (const void*)plan_kernel<kConsOrientLine, 1>;
    default:
      return two ? (const void*)plan_kernel<kConsNone, 2> : (const void*)plan_kernel<kConsNone, 1>;
  }
}

int plan_max_workers(int cons_type, int W, bool sequential, bool warm) {
  cudaFuncAttributes attr;
  const void* fn = plan_fn(cons_type, W, sequential, warm);
  if (!fn) return 0;
  if (cudaFuncGetAttributes(&attr, fn) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return attr.maxThreadsPerBlock / 32 < kMaxWorkers ? attr.maxThreadsPerBlock / 32 : kMaxWorkers;
}

size_t plan_smem_bytes(const RobotDev& rb, int max_scene_f4, int W, int workers, bool stage) {
  return SmemLayout(stage ? max_scene_f4 : 0, rb.n_spheres, W, workers, sizeof(PlanShared)).total;
}

cudaError_t launch_plan(const RobotDev& rb, const SceneDev& sc, const ConsDev& cs, PlanArgs a,
                        const DeviceInfo& dev, cudaStream_t stream) {
  if (a.n <= 0) return cudaSuccess;
  size_t smem = plan_smem_bytes(rb, a.max_scene_f4, a.W, a.workers, true);
  a.stage_obs = smem <= dev.smem_optin ? 1 : 0;
  if (!a.stage_obs) smem = plan_smem_bytes(rb, a.max_scene_f4, a.W, a.workers, false);
  if (smem > dev.smem_optin) return cudaErrorInvalidConfiguration;
  const void* fn = plan_fn(cs.type, a.W, a.sequential != 0, a.warm_refine > 0);
  if (!fn) return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = a.n;
  if (a.queue) {  // persistent CTAs: as many as fit the GPU at once, at most one per problem
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * a.workers, smem);
    if (e != cudaSuccess) return e;
    const long long slots = (long long)(per_sm > 0 ? per_sm : 1) * dev.sm_count;
    grid = slots < a.n ? (int)slots : a.n;
    e = cudaMemsetAsync(a.queue, 0, plan_queue_bytes(a.n), stream);
    if (e != cudaSuccess) return e;
  }
  void* args[] = {const_cast<RobotDev*>(&rb), const_cast<SceneDev*>(&sc),
                  const_cast<ConsDev*>(&cs), &a};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(32 * a.workers), args, smem, stream);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace cprrtc

namespace cprrtc {

__global__ void philox_kernel(uint32_t k0, uint32_t k1, const uint4* __restrict__ ctr, int n,
                              uint4* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = ctr[i];
  const U32x4 r = philox4x32_10(U32x4{c.x, c.y, c.z, c.w}, k0, k1);
  out[i] = make_uint4(r.x, r.y, r.z, r.w);
}

cudaError_t launch_philox(uint32_t k0, uint32_t k1, const uint32_t* ctr, int n, uint32_t* out,
                          cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  philox_kernel<<<(n + 255) / 256, 256, 0, stream>>>(k0, k1, reinterpret_cast<const uint4*>(ctr),
                                                     n, reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

}  // namespace cprrtc
