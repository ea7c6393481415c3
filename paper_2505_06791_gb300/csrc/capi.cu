// C-ABI layer: context lifecycle, robot / scene / constraint upload, pointer staging and
// the exported entry points declared in include/cprrtc.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cprrtc.h"
#include "launch.h"

using namespace cprrtc;

namespace {

struct TimingRec {
  std::string name;
  cudaEvent_t a, b;
};

}  // namespace

struct cprrtc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  DeviceInfo dev{};
  bool has_robot = false;
  RobotDev rb{};
  float4* d_spheres = nullptr;
  int* d_sframe = nullptr;
  SceneDev sc{};
  float4* d_obs = nullptr;
  size_t obs_cap = 0;  // float4 slots
  ConsDev cs{};
  char* d_stage = nullptr;
  size_t stage_cap = 0;
  // scene batch for planning
  float4* d_batch_obs = nullptr;
  size_t batch_obs_cap = 0;
  int4* d_batch_tab = nullptr;
  size_t batch_tab_cap = 0;
  int n_scenes = 0;
  int max_scene_f4 = 0;
  // planner trees and per-worker pending buffers
  char* d_plan = nullptr;
  size_t plan_cap = 0;
  // executed-work totals (validate and plan kernels)
  unsigned long long* d_work = nullptr;
  bool timing = false;
  std::vector<TimingRec> pending;
  std::map<std::string, std::pair<double, long long>> acc;
  std::vector<cudaEvent_t> events;
};

namespace {

int fail(cprrtc_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(cprrtc_ctx* ctx, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(ctx, e == cudaErrorMemoryAllocation ? CPRRTC_E_OOM : CPRRTC_E_CUDA, m);
}

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaEvent_t take_event(cprrtc_ctx* ctx) {
  if (!ctx->events.empty()) {
    cudaEvent_t e = ctx->events.back();
    ctx->events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel launch with events when timing is enabled.
struct LaunchTimer {
  cprrtc_ctx* ctx;
  TimingRec rec{};
  bool on;
  LaunchTimer(cprrtc_ctx* c, const char* name) : ctx(c), on(c->timing) {
    if (!on) return;
    rec.name = name;
    rec.a = take_event(ctx);
    rec.b = take_event(ctx);
    cudaEventRecord(rec.a, ctx->stream);
  }
  void done() {
    if (!on) return;
    cudaEventRecord(rec.b, ctx->stream);
    ctx->pending.push_back(rec);
    on = false;
  }
};

// Host <-> device staging of the array arguments of one call. Device pointers are used as
// they are; host arrays get a slot in the context's staging buffer.
struct Staging {
  struct Item {
    const void* host_in;
    void* host_out;
    size_t bytes;
    size_t off;
    void** dev;
  };
  std::vector<Item> items;
  size_t total = 0;
  bool any_host = false;

  template <class T>
  void input(const T* p, size_t bytes, const T** dev) {
    if (!p || bytes == 0 || is_device_ptr(p)) {
      *dev = p;
      return;
    }
    any_host = true;
    items.push_back({p, nullptr, bytes, total, reinterpret_cast<void**>(const_cast<T**>(dev))});
    total += (bytes + 255) & ~size_t(255);
  }
  template <class T>
  void output(T* p, size_t bytes, T** dev) {
    if (!p || bytes == 0 || is_device_ptr(p)) {
      *dev = p;
      return;
    }
    any_host = true;
    items.push_back({nullptr, p, bytes, total, reinterpret_cast<void**>(dev)});
    total += (bytes + 255) & ~size_t(255);
  }
  // Allocates, assigns device pointers and uploads inputs.
  int begin(cprrtc_ctx* ctx) {
    if (total > ctx->stage_cap) {
      const size_t cap = std::max(total, ctx->stage_cap * 2);
      if (ctx->d_stage) cudaFree(ctx->d_stage);
      ctx->d_stage = nullptr;
      ctx->stage_cap = 0;
      cudaError_t e = cudaMalloc(&ctx->d_stage, cap);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "staging allocation");
      ctx->stage_cap = cap;
    }
    for (auto& it : items) {
      *it.dev = ctx->d_stage + it.off;
      if (it.host_in) {
        cudaError_t e = cudaMemcpyAsync(ctx->d_stage + it.off, it.host_in, it.bytes,
                                        cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "host-to-device copy");
      }
    }
    return CPRRTC_OK;
  }
  // Downloads outputs and waits for them when any argument was host memory.
  int end(cprrtc_ctx* ctx) {
    for (auto& it : items) {
      if (it.host_out) {
        cudaError_t e = cudaMemcpyAsync(it.host_out, ctx->d_stage + it.off, it.bytes,
                                        cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "device-to-host copy");
      }
    }
    if (any_host) {
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    }
    return CPRRTC_OK;
  }
};

template <class T>
int upload(cprrtc_ctx* ctx, T** dst, size_t* cap, const std::vector<T>& src) {
  if (src.size() > *cap || !*dst) {
    if (*dst) cudaFree(*dst);
    *dst = nullptr;
    *cap = 0;
    size_t n = std::max<size_t>(src.size(), 1);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), n * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device allocation");
    *cap = n;
  }
  if (!src.empty()) {
    cudaError_t e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T),
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upload");
  }
  return CPRRTC_OK;
}

bool is_finite(double x) { return std::isfinite(x); }

// Packs obstacles into the float4 stream the kernels read, component arrays per primitive:
// spheres [n] {x,y,z,r}; boxes 4 x [n]: {c, hx} {R col 0, hy} {R col 1, hz} {R col 2, 0};
// capsules 2 x [n]: {p0, r} {p1 - p0, 1/|p1-p0|^2}.
int pack_obstacles(cprrtc_ctx* ctx, const cprrtc_obs_sphere* sph, int n_sph,
                   const cprrtc_obs_box* box, int n_box, const cprrtc_obs_capsule* cap, int n_cap,
                   std::vector<float4>& v) {
  const size_t s0 = v.size();
  v.resize(s0 + (size_t)n_sph + 4 * (size_t)n_box + 2 * (size_t)n_cap);
  float4* out = v.data() + s0;
  for (int i = 0; i < n_sph; ++i) {
    const cprrtc_obs_sphere& o = sph[i];
    if (!is_finite(o.x) || !is_finite(o.y) || !is_finite(o.z) || !is_finite(o.r) || o.r < 0)
      return fail(ctx, CPRRTC_E_INVALID_ARG, "obstacles: bad sphere " + std::to_string(i));
    out[i] = make_float4((float)o.x, (float)o.y, (float)o.z, (float)o.r);
  }
  float4* bx = out + n_sph;
  for (int i = 0; i < n_box; ++i) {
    const cprrtc_obs_box& b = box[i];
    for (int k = 0; k < 3; ++k)
      if (!is_finite(b.c[k]) || !is_finite(b.h[k]) || b.h[k] < 0)
        return fail(ctx, CPRRTC_E_INVALID_ARG, "obstacles: bad box " + std::to_string(i));
    for (int k = 0; k < 9; ++k)
      if (!is_finite(b.R[k])) return fail(ctx, CPRRTC_E_INVALID_ARG, "obstacles: bad box rotation");
    bx[i] = make_float4((float)b.c[0], (float)b.c[1], (float)b.c[2], (float)b.h[0]);
    bx[n_box + i] = make_float4((float)b.R[0], (float)b.R[3], (float)b.R[6], (float)b.h[1]);
    bx[2 * n_box + i] = make_float4((float)b.R[1], (float)b.R[4], (float)b.R[7], (float)b.h[2]);
    bx[3 * n_box + i] = make_float4((float)b.R[2], (float)b.R[5], (float)b.R[8], 0.f);
  }
  float4* cp = bx + 4 * n_box;
  for (int i = 0; i < n_cap; ++i) {
    const cprrtc_obs_capsule& c = cap[i];
    for (int k = 0; k < 3; ++k)
      if (!is_finite(c.p0[k]) || !is_finite(c.p1[k]))
        return fail(ctx, CPRRTC_E_INVALID_ARG, "obstacles: bad capsule " + std::to_string(i));
    if (!is_finite(c.r) || c.r < 0) return fail(ctx, CPRRTC_E_INVALID_ARG, "obstacles: bad capsule radius");
    const double u[3] = {c.p1[0] - c.p0[0], c.p1[1] - c.p0[1], c.p1[2] - c.p0[2]};
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    cp[i] = make_float4((float)c.p0[0], (float)c.p0[1], (float)c.p0[2], (float)c.r);
    cp[n_cap + i] = make_float4((float)u[0], (float)u[1], (float)u[2], uu > 0 ? (float)(1.0 / uu) : 0.f);
  }
  return CPRRTC_OK;
}

}  // namespace

extern "C" {

int cprrtc_create(cprrtc_ctx** out, int device, void* stream) {
  if (!out) return CPRRTC_E_INVALID_ARG;
  *out = nullptr;
  int n_dev = 0;
  cudaError_t e = cudaGetDeviceCount(&n_dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CPRRTC_E_CUDA;
  }
  if (device < 0 || device >= n_dev) return CPRRTC_E_INVALID_ARG;
  cprrtc_ctx* ctx = new (std::nothrow) cprrtc_ctx();
  if (!ctx) return CPRRTC_E_OOM;
  ctx->device = device;
  ctx->stream = reinterpret_cast<cudaStream_t>(stream);
  DeviceGuard g(device);
  int smem = 0;
  if (cudaDeviceGetAttribute(&ctx->dev.sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return CPRRTC_E_CUDA;
  }
  ctx->dev.smem_optin = (size_t)smem;
  if (cudaMalloc(&ctx->d_work, kWorkCounters * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(ctx->d_work, 0, kWorkCounters * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ctx->d_work);
    delete ctx;
    return CPRRTC_E_OOM;
  }
  ctx->cs = ConsDev{kConsNone, 0.f, 1e-4f, 2.f, 1e-3f, 1e-4f, 1.f, 1e-6f, 20};
  ctx->sc = SceneDev{nullptr, 0, 0, 0};
  *out = ctx;
  return CPRRTC_OK;
}

int cprrtc_destroy(cprrtc_ctx* ctx) {
  if (!ctx) return CPRRTC_OK;
  DeviceGuard g(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  cudaFree(ctx->d_spheres);
  cudaFree(ctx->d_sframe);
  cudaFree(ctx->d_obs);
  cudaFree(ctx->d_stage);
  cudaFree(ctx->d_batch_obs);
  cudaFree(ctx->d_batch_tab);
  cudaFree(ctx->d_plan);
  cudaFree(ctx->d_work);
  for (auto& r : ctx->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->events) cudaEventDestroy(e);
  delete ctx;
  return CPRRTC_OK;
}

int cprrtc_set_stream(cprrtc_ctx* ctx, void* stream) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  ctx->stream = reinterpret_cast<cudaStream_t>(stream);
  return CPRRTC_OK;
}

const char* cprrtc_last_error(const cprrtc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int cprrtc_set_robot(cprrtc_ctx* ctx, const cprrtc_joint* joints, int dof,
                     const cprrtc_sphere* spheres, int n_spheres, const double ee[3]) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!joints || !spheres || !ee) return fail(ctx, CPRRTC_E_INVALID_ARG, "set_robot: null pointer");
  if (dof < 1 || dof > CPRRTC_MAX_DOF)
    return fail(ctx, dof < 1 ? CPRRTC_E_INVALID_ARG : CPRRTC_E_UNSUPPORTED, "set_robot: dof must be in [1, 8]");
  if (n_spheres < 1 || n_spheres > CPRRTC_MAX_SPHERES)
    return fail(ctx, n_spheres < 1 ? CPRRTC_E_INVALID_ARG : CPRRTC_E_UNSUPPORTED,
                "set_robot: n_spheres must be in [1, 256]");
  RobotDev rb{};
  rb.dof = dof;
  rb.n_spheres = n_spheres;
  for (int k = 0; k < dof; ++k) {
    const cprrtc_joint& j = joints[k];
    if ((j.type != CPRRTC_JOINT_REVOLUTE && j.type != CPRRTC_JOINT_PRISMATIC) || !is_finite(j.d) ||
        !is_finite(j.a) || !is_finite(j.alpha) || !is_finite(j.theta0) || !is_finite(j.lo) || !is_finite(j.hi) || j.lo > j.hi)
      return fail(ctx, CPRRTC_E_INVALID_ARG, "set_robot: bad joint " + std::to_string(k));
    JointDev& d = rb.j[k];
    d.ca = (float)std::cos(j.alpha);
    d.sa = (float)std::sin(j.alpha);
    d.a = (float)j.a;
    d.d = (float)j.d;
    d.theta0 = (float)j.theta0;
    d.ct0 = (float)std::cos(j.theta0);
    d.st0 = (float)std::sin(j.theta0);
    d.lo = (float)j.lo;
    d.hi = (float)j.hi;
    d.prismatic = j.type == CPRRTC_JOINT_PRISMATIC;
  }
  for (int i = 0; i < 3; ++i) {
    if (!is_finite(ee[i])) return fail(ctx, CPRRTC_E_INVALID_ARG, "set_robot: bad ee");
    rb.ee[i] = (float)ee[i];
  }
  // spheres sorted by frame (stable): lanes of one frame read the same transform
  std::vector<int> order(n_spheres);
  for (int i = 0; i < n_spheres; ++i) {
    const cprrtc_sphere& s = spheres[i];
    if (s.frame < 0 || s.frame > dof || !is_finite(s.x) || !is_finite(s.y) || !is_finite(s.z) || !(s.r > 0) || !is_finite(s.r))
      return fail(ctx, CPRRTC_E_INVALID_ARG, "set_robot: bad sphere " + std::to_string(i));
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return spheres[a].frame < spheres[b].frame; });
  std::vector<float4> loc(n_spheres);
  std::vector<int> frm(n_spheres);
  for (int i = 0; i < n_spheres; ++i) {
    const cprrtc_sphere& s = spheres[order[i]];
    loc[i] = make_float4((float)s.x, (float)s.y, (float)s.z, (float)s.r);
    frm[i] = s.frame;
  }
  // Bounding sphere of each frame's spheres, from the FP32 values the kernels use: centre at
  // the middle of their bounding box, radius max(|c - b| + r) padded by 1e-5 m and rounded
  // up, so a miss of the bound proves a miss of every sphere under FP32 evaluation.
  for (int f = 0; f <= CPRRTC_MAX_DOF; ++f) {
    rb.bound[f] = make_float4(0.f, 0.f, 0.f, -1.f);
    rb.n_per_frame[f] = 0;
  }
  for (int i = 0; i < n_spheres; ++i) rb.n_per_frame[frm[i]]++;
  rb.bound_count = 0;
  for (int f = 0; f <= dof; ++f) rb.bound_count += rb.n_per_frame[f] > 0;
  for (int f = 0; f <= dof; ++f) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    bool any = false;
    for (int i = 0; i < n_spheres; ++i) {
      if (frm[i] != f) continue;
      any = true;
      const double c[3] = {loc[i].x, loc[i].y, loc[i].z};
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], c[k]);
        hi[k] = std::max(hi[k], c[k]);
      }
    }
    if (!any) continue;
    const float b[3] = {(float)(0.5 * (lo[0] + hi[0])), (float)(0.5 * (lo[1] + hi[1])),
                        (float)(0.5 * (lo[2] + hi[2]))};
    double R = 0.0;
    for (int i = 0; i < n_spheres; ++i) {
      if (frm[i] != f) continue;
      const double dx = (double)loc[i].x - b[0], dy = (double)loc[i].y - b[1], dz = (double)loc[i].z - b[2];
      R = std::max(R, std::sqrt(dx * dx + dy * dy + dz * dz) + (double)loc[i].w);
    }
    rb.bound[f] = make_float4(b[0], b[1], b[2], std::nextafter((float)(R + 1e-5), 1e30f));
  }
  DeviceGuard g(ctx->device);
  size_t cap1 = 0, cap2 = 0;
  if (ctx->d_spheres) { cudaFree(ctx->d_spheres); ctx->d_spheres = nullptr; }
  if (ctx->d_sframe) { cudaFree(ctx->d_sframe); ctx->d_sframe = nullptr; }
  int rc = upload(ctx, &ctx->d_spheres, &cap1, loc);
  if (rc) return rc;
  rc = upload(ctx, &ctx->d_sframe, &cap2, frm);
  if (rc) return rc;
  rb.spheres = ctx->d_spheres;
  rb.sphere_frame = ctx->d_sframe;
  ctx->rb = rb;
  ctx->has_robot = true;
  return CPRRTC_OK;
}

int cprrtc_set_obstacles(cprrtc_ctx* ctx, const cprrtc_obs_sphere* sph, int n_sph,
                         const cprrtc_obs_box* box, int n_box, const cprrtc_obs_capsule* cap,
                         int n_cap) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (n_sph < 0 || n_box < 0 || n_cap < 0 || (n_sph && !sph) || (n_box && !box) || (n_cap && !cap))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_obstacles: bad counts or null pointer");
  if ((long long)n_sph + 4LL * n_box + 2LL * n_cap > (1LL << 26))
    return fail(ctx, CPRRTC_E_UNSUPPORTED, "set_obstacles: too many obstacles");
  std::vector<float4> v;
  int rc = pack_obstacles(ctx, sph, n_sph, box, n_box, cap, n_cap, v);
  if (rc) return rc;
  DeviceGuard g(ctx->device);
  rc = upload(ctx, &ctx->d_obs, &ctx->obs_cap, v);
  if (rc) return rc;
  ctx->sc = SceneDev{ctx->d_obs, n_sph, n_box, n_cap};
  return CPRRTC_OK;
}

int cprrtc_set_scene_batch(cprrtc_ctx* ctx, int n_scenes, const cprrtc_obs_sphere* sph,
                           const int32_t* sph_off, const cprrtc_obs_box* box,
                           const int32_t* box_off, const cprrtc_obs_capsule* cap,
                           const int32_t* cap_off) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (n_scenes < 1 || !sph_off || !box_off || !cap_off)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_scene_batch: n_scenes < 1 or null offsets");
  const int32_t* offs[3] = {sph_off, box_off, cap_off};
  for (int t = 0; t < 3; ++t) {
    if (offs[t][0] != 0) return fail(ctx, CPRRTC_E_INVALID_ARG, "set_scene_batch: offsets must start at 0");
    for (int i = 0; i < n_scenes; ++i)
      if (offs[t][i + 1] < offs[t][i])
        return fail(ctx, CPRRTC_E_INVALID_ARG, "set_scene_batch: offsets must not decrease");
  }
  if ((sph_off[n_scenes] && !sph) || (box_off[n_scenes] && !box) || (cap_off[n_scenes] && !cap))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_scene_batch: null obstacle array");
  if ((long long)sph_off[n_scenes] + 4LL * box_off[n_scenes] + 2LL * cap_off[n_scenes] > (1LL << 28))
    return fail(ctx, CPRRTC_E_UNSUPPORTED, "set_scene_batch: too many obstacles");
  std::vector<float4> all;
  std::vector<int4> tab(n_scenes);
  int max_f4 = 0;
  for (int s_ = 0; s_ < n_scenes; ++s_) {
    const int ns = sph_off[s_ + 1] - sph_off[s_], nb = box_off[s_ + 1] - box_off[s_],
              nc = cap_off[s_ + 1] - cap_off[s_];
    std::vector<float4> v;
    int rc = pack_obstacles(ctx, sph + sph_off[s_], ns, box + box_off[s_], nb, cap + cap_off[s_], nc, v);
    if (rc) return rc;
    tab[s_] = make_int4((int)all.size(), ns, nb, nc);
    max_f4 = std::max(max_f4, (int)v.size());
    all.insert(all.end(), v.begin(), v.end());
  }
  DeviceGuard g(ctx->device);
  int rc = upload(ctx, &ctx->d_batch_obs, &ctx->batch_obs_cap, all);
  if (rc) return rc;
  rc = upload(ctx, &ctx->d_batch_tab, &ctx->batch_tab_cap, tab);
  if (rc) return rc;
  ctx->n_scenes = n_scenes;
  ctx->max_scene_f4 = max_f4;
  return CPRRTC_OK;
}

int cprrtc_set_constraint(cprrtc_ctx* ctx, const cprrtc_constraint* c) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!c) return fail(ctx, CPRRTC_E_INVALID_ARG, "set_constraint: null pointer");
  if (c->type < CPRRTC_CONSTRAINT_NONE || c->type > CPRRTC_CONSTRAINT_Z_PLANE)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_constraint: unknown type");
  if (c->max_iters < 1 || c->max_iters > 255)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_constraint: max_iters must be in [1, 255]");
  if (!is_finite(c->target) || !(c->tol_task > 0) || !(c->tol_sm > 0) || !(c->c_sm > 0) ||
      !(c->tau_floor >= 0) || !is_finite(c->alpha) || !(c->lambda >= 0) || !is_finite(c->lambda) ||
      !is_finite(c->tol_task) || !is_finite(c->tol_sm) || !is_finite(c->c_sm) || !is_finite(c->tau_floor))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_constraint: bad parameter");
  ctx->cs = ConsDev{c->type,          (float)c->target, (float)c->tol_task,
                    (float)c->c_sm,   (float)c->tau_floor, (float)c->tol_sm,
                    (float)c->alpha,  (float)(c->lambda * c->lambda), c->max_iters};
  return CPRRTC_OK;
}

int cprrtc_validate(cprrtc_ctx* ctx, const float* q_start, const float* q_end, int n, int W,
                    float* out_q, uint8_t* status, int32_t* first_fail, uint8_t* iters,
                    float* resid) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!ctx->has_robot) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "validate: set_robot first");
  if (n < 0) return fail(ctx, CPRRTC_E_INVALID_ARG, "validate: n < 0");
  if (W < 2 || W > CPRRTC_MAX_W)
    return fail(ctx, W < 2 ? CPRRTC_E_INVALID_ARG : CPRRTC_E_UNSUPPORTED, "validate: W must be in [2, 64]");
  if (n == 0) return CPRRTC_OK;
  if (!q_start || !q_end || !status) return fail(ctx, CPRRTC_E_INVALID_ARG, "validate: null pointer");
  DeviceGuard g(ctx->device);
  const size_t dof = ctx->rb.dof, N = (size_t)n;
  ValidateArgs a{};
  a.n = n;
  a.W = W;
  a.cc_skip_first = 0;
  a.work_counters = ctx->d_work;
  Staging st;
  st.input(q_start, N * dof * sizeof(float), &a.q_start);
  st.input(q_end, N * dof * sizeof(float), &a.q_end);
  st.output(out_q, N * W * dof * sizeof(float), &a.out_q);
  st.output(status, N, &a.status);
  st.output(first_fail, N * sizeof(int32_t), &a.first_fail);
  st.output(iters, N, &a.iters);
  st.output(resid, N * sizeof(float), &a.resid);
  int rc = st.begin(ctx);
  if (rc) return rc;
  LaunchTimer tm(ctx, "validate");
  cudaError_t e = launch_validate(ctx->rb, ctx->sc, ctx->cs, a, ctx->dev, ctx->stream);
  tm.done();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "validate launch");
  return st.end(ctx);
}

int cprrtc_project_configs(cprrtc_ctx* ctx, const float* q_in, int n, int max_iters,
                           float* q_out, uint8_t* ok, float* resid) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!ctx->has_robot) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "project_configs: set_robot first");
  if (ctx->cs.type == kConsNone)
    return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "project_configs: constraint is NONE");
  if (n < 0 || max_iters < 0 || max_iters > 100000)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "project_configs: bad n or max_iters");
  if (n == 0) return CPRRTC_OK;
  if (!q_in || !q_out) return fail(ctx, CPRRTC_E_INVALID_ARG, "project_configs: null pointer");
  DeviceGuard g(ctx->device);
  const size_t dof = ctx->rb.dof, N = (size_t)n;
  const float* d_in;
  float *d_out, *d_res;
  uint8_t* d_ok;
  Staging st;
  st.input(q_in, N * dof * sizeof(float), &d_in);
  st.output(q_out, N * dof * sizeof(float), &d_out);
  st.output(ok, N, &d_ok);
  st.output(resid, N * sizeof(float), &d_res);
  int rc = st.begin(ctx);
  if (rc) return rc;
  LaunchTimer tm(ctx, "project");
  cudaError_t e = launch_project_configs(ctx->rb, ctx->cs, d_in, n, max_iters, d_out, d_ok, d_res, ctx->stream);
  tm.done();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "project launch");
  return st.end(ctx);
}

int cprrtc_plan(cprrtc_ctx* ctx, const float* start, const float* goal, int n,
                const cprrtc_plan_params* pp, int32_t* path_len, float* path, float* path_edges,
                int32_t* rounds, int64_t* waypoints, float* plan_ms, int64_t* work) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!ctx->has_robot) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "plan: set_robot first");
  if (!pp) return fail(ctx, CPRRTC_E_INVALID_ARG, "plan: null params");
  if (n < 0) return fail(ctx, CPRRTC_E_INVALID_ARG, "plan: n < 0");
  if (pp->W < 2 || pp->W > CPRRTC_MAX_W || !(pp->range > 0) || !is_finite(pp->range) ||
      pp->max_rounds < 1 || pp->workers < 1 || pp->workers > kMaxWorkers || pp->max_nodes < 2 ||
      pp->max_connect < 0 || pp->max_path < 2)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "plan: bad parameters");
  if (pp->use_scene_batch && ctx->n_scenes != n)
    return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "plan: scene batch must hold one scene per problem");
  if (n == 0) return CPRRTC_OK;
  if (!start || !goal || !path_len || !path) return fail(ctx, CPRRTC_E_INVALID_ARG, "plan: null pointer");
  DeviceGuard g(ctx->device);
  const size_t dof = ctx->rb.dof, N = (size_t)n, W = (size_t)pp->W;
  const size_t B = (size_t)pp->workers, MN = (size_t)pp->max_nodes;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_nodes = al(N * 2 * MN * 8 * sizeof(float));
  const size_t b_parent = al(N * 2 * MN * sizeof(int));
  const size_t b_edges = al(N * 2 * MN * W * dof * sizeof(float));
  const size_t b_pend = al(N * B * 8 * sizeof(float));
  const size_t b_pedge = al(N * B * 2 * W * dof * sizeof(float));
  const size_t need = b_nodes + b_parent + b_edges + b_pend + b_pedge;
  if (need > ctx->plan_cap) {
    if (ctx->d_plan) cudaFree(ctx->d_plan);
    ctx->d_plan = nullptr;
    ctx->plan_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->d_plan, need);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plan: tree allocation");
    ctx->plan_cap = need;
  }
  PlanArgs a{};
  a.n = n;
  a.range = (float)pp->range;
  a.W = pp->W;
  a.max_rounds = pp->max_rounds;
  a.workers = pp->workers;
  a.max_nodes = pp->max_nodes;
  a.max_connect = pp->max_connect;
  a.max_path = pp->max_path;
  a.seed = pp->seed;
  a.work_counters = ctx->d_work;
  if (pp->use_scene_batch) {
    a.scene_obs = ctx->d_batch_obs;
    a.scenes = ctx->d_batch_tab;
    a.max_scene_f4 = ctx->max_scene_f4;
  } else {
    a.scene_obs = nullptr;
    a.scenes = nullptr;
    a.max_scene_f4 = ctx->sc.n_float4();
  }
  char* base = ctx->d_plan;
  a.nodes = reinterpret_cast<float*>(base);
  a.parent = reinterpret_cast<int*>(base + b_nodes);
  a.edges = reinterpret_cast<float*>(base + b_nodes + b_parent);
  a.pend = reinterpret_cast<float*>(base + b_nodes + b_parent + b_edges);
  a.pend_edges = reinterpret_cast<float*>(base + b_nodes + b_parent + b_edges + b_pend);
  Staging st;
  st.input(start, N * dof * sizeof(float), &a.start);
  st.input(goal, N * dof * sizeof(float), &a.goal);
  st.output(path_len, N * sizeof(int32_t), &a.path_len);
  st.output(path, N * (size_t)pp->max_path * dof * sizeof(float), &a.path);
  st.output(path_edges, N * (size_t)(pp->max_path - 1) * W * dof * sizeof(float), &a.path_edges);
  st.output(rounds, N * sizeof(int32_t), &a.rounds);
  st.output(reinterpret_cast<long long*>(waypoints), N * sizeof(int64_t), &a.waypoints);
  st.output(plan_ms, N * sizeof(float), &a.plan_ms);
  st.output(reinterpret_cast<long long*>(work), N * 2 * sizeof(int64_t), &a.work);
  int rc = st.begin(ctx);
  if (rc) return rc;
  LaunchTimer tm(ctx, "plan");
  cudaError_t e = launch_plan(ctx->rb, ctx->sc, ctx->cs, a, ctx->dev, ctx->stream);
  tm.done();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "plan launch");
  return st.end(ctx);
}

int cprrtc_philox(cprrtc_ctx* ctx, uint32_t key0, uint32_t key1, const uint32_t* counters, int n,
                  uint32_t* out) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (n < 0) return fail(ctx, CPRRTC_E_INVALID_ARG, "philox: n < 0");
  if (n == 0) return CPRRTC_OK;
  if (!counters || !out) return fail(ctx, CPRRTC_E_INVALID_ARG, "philox: null pointer");
  DeviceGuard g(ctx->device);
  const uint32_t* d_in;
  uint32_t* d_out;
  Staging st;
  st.input(counters, (size_t)n * 4 * sizeof(uint32_t), &d_in);
  st.output(out, (size_t)n * 4 * sizeof(uint32_t), &d_out);
  int rc = st.begin(ctx);
  if (rc) return rc;
  cudaError_t e = launch_philox(key0, key1, d_in, n, d_out, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "philox launch");
  return st.end(ctx);
}

int cprrtc_work_counters(cprrtc_ctx* ctx, int64_t* out, int reset) {
  if (!ctx || !out) return CPRRTC_E_INVALID_ARG;
  DeviceGuard g(ctx->device);
  unsigned long long h[kWorkCounters];
  cudaError_t e = cudaMemcpyAsync(h, ctx->d_work, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(ctx->d_work, 0, sizeof(h), ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "work counters");
  for (int i = 0; i < kWorkCounters; ++i) out[i] = (int64_t)h[i];
  return CPRRTC_OK;
}

int cprrtc_set_timing(cprrtc_ctx* ctx, int enabled) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  ctx->timing = enabled != 0;
  return CPRRTC_OK;
}

int cprrtc_kernel_time(cprrtc_ctx* ctx, const char* name, double* ms, long long* launches) {
  if (!ctx || !name || !ms || !launches) return CPRRTC_E_INVALID_ARG;
  DeviceGuard g(ctx->device);
  for (auto& r : ctx->pending) {
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event synchronize");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event elapsed");
    auto& slot = ctx->acc[r.name];
    slot.first += t;
    slot.second += 1;
    ctx->events.push_back(r.a);
    ctx->events.push_back(r.b);
  }
  ctx->pending.clear();
  auto it = ctx->acc.find(name);
  *ms = it == ctx->acc.end() ? 0.0 : it->second.first;
  *launches = it == ctx->acc.end() ? 0 : it->second.second;
  return CPRRTC_OK;
}

int cprrtc_reset_timing(cprrtc_ctx* ctx) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  double ms;
  long long l;
  cprrtc_kernel_time(ctx, "", &ms, &l);
  ctx->acc.clear();
  return CPRRTC_OK;
}

}  // extern "C"

// ---- planning from a fixed device array (no allocation) ----------------------------------
//
// The trees of cprrtc_plan_static live here, one array per device that loads the library.
// Host code must not use the symbol as an address: the kernel receives the device address
// looked up with cudaGetSymbolAddress, once per device.
namespace {

static __device__ __align__(256) unsigned char g_plan_scratch[CPRRTC_STATIC_SCRATCH_BYTES];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kStaticMaxDevices] = {};

// Device address of g_plan_scratch on `device` (which must be current); nullptr on error.
void* static_scratch(int device, cudaError_t* err) {
  *err = cudaSuccess;
  if (device < 0 || device >= kStaticMaxDevices) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[device]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_plan_scratch);
    if (*err != cudaSuccess) return nullptr;
    g_static_ptr[device] = p;
  }
  return g_static_ptr[device];
}

}  // namespace

extern "C" int cprrtc_plan_static(cprrtc_ctx* ctx, const float* start, const float* goal, int n,
                                  const cprrtc_plan_params* pp, int32_t* path_len, float* path,
                                  float* path_edges, int32_t* rounds, int64_t* waypoints,
                                  float* plan_ms, int64_t* work) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!ctx->has_robot) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "plan_static: set_robot first");
  if (!pp) return fail(ctx, CPRRTC_E_INVALID_ARG, "plan_static: null params");
  if (n < 0) return fail(ctx, CPRRTC_E_INVALID_ARG, "plan_static: n < 0");
  if (pp->W < 2 || pp->W > CPRRTC_MAX_W || !(pp->range > 0) || !is_finite(pp->range) ||
      pp->max_rounds < 1 || pp->workers < 1 || pp->workers > kMaxWorkers || pp->max_nodes < 2 ||
      pp->max_connect < 0 || pp->max_path < 2)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "plan_static: bad parameters");
  if (pp->use_scene_batch && ctx->n_scenes != n)
    return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "plan_static: scene batch must hold one scene per problem");
  if (n == 0) return CPRRTC_OK;
  if (!start || !goal || !path_len || !path)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "plan_static: null pointer");
  DeviceGuard g(ctx->device);
  const void* arrays[] = {start, goal, path_len, path, path_edges, rounds, waypoints, plan_ms, work};
  for (const void* a : arrays)
    if (a && !is_device_ptr(a))
      return fail(ctx, CPRRTC_E_INVALID_ARG, "plan_static: every array must be device memory");
  const size_t dof = ctx->rb.dof, N = (size_t)n, W = (size_t)pp->W;
  const size_t B = (size_t)pp->workers, MN = (size_t)pp->max_nodes;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_nodes = al(N * 2 * MN * 8 * sizeof(float));
  const size_t b_parent = al(N * 2 * MN * sizeof(int));
  const size_t b_edges = al(N * 2 * MN * W * dof * sizeof(float));
  const size_t b_pend = al(N * B * 8 * sizeof(float));
  const size_t b_pedge = al(N * B * 2 * W * dof * sizeof(float));
  const size_t need = b_nodes + b_parent + b_edges + b_pend + b_pedge;
  if (need > (size_t)CPRRTC_STATIC_SCRATCH_BYTES)
    return fail(ctx, CPRRTC_E_CAPACITY,
                "plan_static: needs " + std::to_string(need) + " bytes of scratch, the fixed array holds " +
                    std::to_string((size_t)CPRRTC_STATIC_SCRATCH_BYTES) +
                    " (reduce n, max_nodes, W or workers)");
  cudaError_t e;
  char* base = static_cast<char*>(static_scratch(ctx->device, &e));
  if (!base) return cuda_fail(ctx, e, "plan_static: cudaGetSymbolAddress");
  PlanArgs a{};
  a.start = start;
  a.goal = goal;
  a.n = n;
  a.range = (float)pp->range;
  a.W = pp->W;
  a.max_rounds = pp->max_rounds;
  a.workers = pp->workers;
  a.max_nodes = pp->max_nodes;
  a.max_connect = pp->max_connect;
  a.max_path = pp->max_path;
  a.seed = pp->seed;
  if (pp->use_scene_batch) {
    a.scene_obs = ctx->d_batch_obs;
    a.scenes = ctx->d_batch_tab;
    a.max_scene_f4 = ctx->max_scene_f4;
  } else {
    a.scene_obs = nullptr;
    a.scenes = nullptr;
    a.max_scene_f4 = ctx->sc.n_float4();
  }
  a.nodes = reinterpret_cast<float*>(base);
  a.parent = reinterpret_cast<int*>(base + b_nodes);
  a.edges = reinterpret_cast<float*>(base + b_nodes + b_parent);
  a.pend = reinterpret_cast<float*>(base + b_nodes + b_parent + b_edges);
  a.pend_edges = reinterpret_cast<float*>(base + b_nodes + b_parent + b_edges + b_pend);
  a.path_len = path_len;
  a.path = path;
  a.path_edges = path_edges;
  a.rounds = rounds;
  a.waypoints = reinterpret_cast<long long*>(waypoints);
  a.plan_ms = plan_ms;
  a.work = reinterpret_cast<long long*>(work);
  e = launch_plan(ctx->rb, ctx->sc, ctx->cs, a, ctx->dev, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "plan_static launch");
  return CPRRTC_OK;
}
