// C-ABI layer: context lifecycle, robot / scene / constraint upload, pointer staging and
// the exported entry points declared in include/cprrtc.h.
#include <algorithm>
#include <array>
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

// Device buffers one batch launch references (kept alive while a captured graph exists).
struct BatchRes {
  int4* d_probs = nullptr;
  size_t probs_cap = 0;
  int* d_order = nullptr;
  size_t order_cap = 0;
  unsigned* d_counters = nullptr;
  char* d_scratch = nullptr;
  size_t scratch_cap = 0;
  long long* d_span = nullptr;  // [n][2] each problem's start and end on the global timer
  size_t span_cap = 0;
  int n = 0;                    // problems of the batch these buffers last served
};

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
  // batch tables
  std::vector<RobotDev> tab_robots;
  std::vector<SelfMask> tab_self;  // each table robot's self-collision frame pairs
  // the uneven batch's learned form: a copy of a trained network per (table robot,
  // constraint) pair, [robot * kBatchMaxCons + constraint] (buffer null: none)
  void* batch_net_buf[kBatchMaxRobots * kBatchMaxCons] = {};
  MlpView batch_net[kBatchMaxRobots * kBatchMaxCons] = {};
  float4* d_tab_sph = nullptr;
  size_t tab_sph_cap = 0;
  int* d_tab_frm = nullptr;
  size_t tab_frm_cap = 0;
  std::vector<ConsDev> tab_cons;
  cprrtc_tuning tuned{};
  bool has_tuned = false;
  BatchRes batch_res, graph_res;
  const BatchRes* last_batch = nullptr;  // the buffers of the last batch run (for its spans)
  cudaStream_t side[2 * kBatchClasses] = {};  // one per batch part (two per class)
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[2 * kBatchClasses] = {};
  cudaGraphExec_t graph_exec = nullptr;
  // collision checking in GEMM form
  int cc_mode = CPRRTC_CC_EXACT;
  int early_exit = 1;  // 0: collision checking skips nothing (ablation)
  bool self_on = false;                   // self-collision after cprrtc_validate
  unsigned short self_rows[kMaxDof + 1] = {};
  int projection = CPRRTC_PROJECTION_PARALLEL;
  double cc_guard = 0.005;
  std::vector<float4> host_sph;  // sphere obstacles as staged (FP32), image row order
  std::vector<float4> host_robot_sph;  // robot spheres {x, y, z, r} in their frames
  uint8_t* d_bimage = nullptr;
  size_t bimage_cap = 0;
  int cc_tiles = 0;
  float4 cc_origin{};
  double cc_bound = 0.0;
  unsigned long long* d_cc_counters = nullptr;  // [2]
  int* d_cc_error = nullptr;
  float* d_cc_q = nullptr;  // projected waypoints when the caller does not ask for them
  size_t cc_q_cap = 0;
  int32_t* d_cc_ff = nullptr;
  size_t cc_ff_cap = 0;
  // learned warm start
  MlpDev* mlp = nullptr;
  bool mlp_fp32 = false;    // the network's FP32 checking mode
  unsigned long long wait_ns = 0;  // bounded-wait limit of the tensor-core kernels (0: 1 s)
  int plan_warm = 0;               // planner's learned form: refine iterations (0: off)
  int plan_first_slice = 100;      // planner's time-sliced schedule (0: one CTA per problem)
  int plan_slice = 50;
  float* d_warm = nullptr;  // corrections [n*W][16]
  size_t warm_cap = 0;      // bytes
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
  // a failed launch (resources, configuration) leaves the runtime's last-error state set; a
  // later call's launch check would report it again, so it is consumed here (sticky errors,
  // which end the context, are not cleared by this)
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return fail(ctx, CPRRTC_E_OOM, m);
  return fail(ctx, CPRRTC_E_CUDA, m);
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

// Where an array argument lives, seen from `device`: host memory (pageable or pinned),
// device memory of `device` or managed memory (usable as it is), or device memory of
// another GPU (rejected: the kernels would read or write peer memory nobody mapped).
enum PtrWhere { kPtrHost = 0, kPtrHere = 1, kPtrOtherDevice = 2 };

PtrWhere ptr_where(const void* p, int device) {
  if (!p) return kPtrHost;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return kPtrHost;
  }
  if (a.type == cudaMemoryTypeManaged) return kPtrHere;
  if (a.type == cudaMemoryTypeDevice) return a.device == device ? kPtrHere : kPtrOtherDevice;
  return kPtrHost;
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
  bool foreign = false;  // some array is device memory of another GPU
  int device = -1;       // the context's device (current while a call runs)

  // Classifies p against the current device: true if it is used as it is (null, empty,
  // device memory of this GPU or managed memory); a foreign device pointer is recorded and
  // makes begin() fail.
  bool usable(const void* p, size_t bytes) {
    if (!p || bytes == 0) return true;
    if (device < 0 && cudaGetDevice(&device) != cudaSuccess) device = -1;
    const PtrWhere w = ptr_where(p, device);
    if (w == kPtrOtherDevice) foreign = true;
    return w != kPtrHost;
  }

  template <class T>
  void input(const T* p, size_t bytes, const T** dev) {
    if (usable(p, bytes)) {
      *dev = p;
      return;
    }
    any_host = true;
    items.push_back({p, nullptr, bytes, total, reinterpret_cast<void**>(const_cast<T**>(dev))});
    total += (bytes + 255) & ~size_t(255);
  }
  template <class T>
  void output(T* p, size_t bytes, T** dev) {
    if (usable(p, bytes)) {
      *dev = p;
      return;
    }
    any_host = true;
    items.push_back({nullptr, p, bytes, total, reinterpret_cast<void**>(dev)});
    total += (bytes + 255) & ~size_t(255);
  }
  // Allocates, assigns device pointers and uploads inputs.
  int begin(cprrtc_ctx* ctx) {
    if (foreign)
      return fail(ctx, CPRRTC_E_INVALID_ARG,
                  "an array argument is device memory of another GPU than the context's");
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

// 3-bit interleave helper of a 30-bit Morton code.
uint32_t spread10(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Order of `centres` along a Morton curve over their bounding box (ties keep input order).
std::vector<int> morton_order(const std::vector<std::array<double, 3>>& centres) {
  const size_t n = centres.size();
  std::vector<int> idx(n);
  for (size_t i = 0; i < n; ++i) idx[i] = (int)i;
  if (n < 2) return idx;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (auto& c : centres)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], c[k]);
      hi[k] = std::max(hi[k], c[k]);
    }
  std::vector<uint32_t> code(n);
  for (size_t i = 0; i < n; ++i) {
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
      const double span = hi[k] - lo[k];
      const double t = span > 0 ? (centres[i][k] - lo[k]) / span : 0.0;
      q[k] = (uint32_t)std::min(1023.0, std::max(0.0, std::floor(t * 1024.0)));
    }
    code[i] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
  }
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return code[a] < code[b]; });
  return idx;
}

// The planner kernel's registers bound its CTA size: with two waypoints per lane (W > 32)
// fewer than the maximum 16 workers fit.
int check_plan_workers(cprrtc_ctx* ctx, const cprrtc_plan_params* pp, const char* who) {
  const bool seq = ctx->projection == CPRRTC_PROJECTION_SEQUENTIAL;
  if (seq && (pp->W > 32 || (ctx->cs.type != kConsRollPitch && ctx->cs.type != kConsZPlane)))
    return fail(ctx, CPRRTC_E_UNSUPPORTED,
                std::string(who) + ": the sequential projection plans with ROLL_PITCH or Z_PLANE and W <= 32");
  const bool warm = ctx->plan_warm > 0;
  if (warm) {
    if (seq || (ctx->cs.type != kConsRollPitch && ctx->cs.type != kConsZPlane))
      return fail(ctx, CPRRTC_E_UNSUPPORTED,
                  std::string(who) + ": the learned form plans with ROLL_PITCH or Z_PLANE and the parallel projection");
    if (!ctx->mlp || mlp_dof(ctx->mlp) != ctx->rb.dof)
      return fail(ctx, CPRRTC_E_NOT_CONFIGURED,
                  std::string(who) + ": the learned form needs a network for the robot (mlp_init or mlp_load)");
  }
  const int mw = plan_max_workers(ctx->cs.type, pp->W, seq, warm);
  if (pp->workers > mw)
    return fail(ctx, CPRRTC_E_UNSUPPORTED, std::string(who) + ": at most " + std::to_string(mw) +
                                               " workers fit one CTA at W = " + std::to_string(pp->W));
  return CPRRTC_OK;
}

float round_down(double x) {
  float f = (float)x;
  return (double)f > x ? std::nextafter(f, -INFINITY) : f;
}
float round_up(double x) {
  float f = (float)x;
  return (double)f < x ? std::nextafter(f, INFINITY) : f;
}

// Packs obstacles into the float4 stream the kernels read. Each primitive kind is sorted
// along a Morton curve (neighbours in the stream are neighbours in space; collision results
// do not depend on the order) and stored as component arrays: spheres [n] {x,y,z,r}; boxes
// 4 x [n]: {c, hx} {R col 0, hy} {R col 1, hz} {R col 2, bounding radius}; capsules 2 x [n]:
// {p0, r} {p1 - p0, 1/|p1-p0|^2}. Then, per chunk (kChunk consecutive obstacles of one
// kind), an axis-aligned box containing every obstacle of the chunk (rounded outward to
// FP32).
int pack_obstacles(cprrtc_ctx* ctx, const cprrtc_obs_sphere* sph, int n_sph,
                   const cprrtc_obs_box* box, int n_box, const cprrtc_obs_capsule* cap, int n_cap,
                   std::vector<float4>& v) {
  const int n_obs = n_sph + n_box + n_cap;
  const SceneDev layout{nullptr, n_sph, n_box, n_cap};
  const int n_chunks = layout.n_chunks();
  const size_t s0 = v.size();
  v.resize(s0 + (size_t)n_sph + 4 * (size_t)n_box + 2 * (size_t)n_cap + 2 * (size_t)n_chunks);
  float4* out = v.data() + s0;
  std::vector<std::array<double, 6>> aabb(n_obs);  // per obstacle, in stream order
  std::vector<std::array<double, 3>> cen;
  cen.resize(n_sph);
  for (int i = 0; i < n_sph; ++i) {
    const cprrtc_obs_sphere& o = sph[i];
    if (!is_finite(o.x) || !is_finite(o.y) || !is_finite(o.z) || !is_finite(o.r) || o.r < 0)
      return fail(ctx, CPRRTC_E_INVALID_ARG, "obstacles: bad sphere " + std::to_string(i));
    cen[i] = {o.x, o.y, o.z};
  }
  std::vector<int> ord = morton_order(cen);
  for (int j = 0; j < n_sph; ++j) {
    const cprrtc_obs_sphere& o = sph[ord[j]];
    out[j] = make_float4((float)o.x, (float)o.y, (float)o.z, (float)o.r);
    aabb[j] = {o.x - o.r, o.y - o.r, o.z - o.r, o.x + o.r, o.y + o.r, o.z + o.r};
  }
  cen.resize(n_box);
  for (int i = 0; i < n_box; ++i) {
    const cprrtc_obs_box& b = box[i];
    for (int k = 0; k < 3; ++k)
      if (!is_finite(b.c[k]) || !is_finite(b.h[k]) || b.h[k] < 0)
        return fail(ctx, CPRRTC_E_INVALID_ARG, "obstacles: bad box " + std::to_string(i));
    for (int k = 0; k < 9; ++k)
      if (!is_finite(b.R[k])) return fail(ctx, CPRRTC_E_INVALID_ARG, "obstacles: bad box rotation");
    cen[i] = {b.c[0], b.c[1], b.c[2]};
  }
  ord = morton_order(cen);
  float4* bx = out + n_sph;
  for (int j = 0; j < n_box; ++j) {
    const cprrtc_obs_box& b = box[ord[j]];
    bx[j] = make_float4((float)b.c[0], (float)b.c[1], (float)b.c[2], (float)b.h[0]);
    bx[n_box + j] = make_float4((float)b.R[0], (float)b.R[3], (float)b.R[6], (float)b.h[1]);
    bx[2 * n_box + j] = make_float4((float)b.R[1], (float)b.R[4], (float)b.R[7], (float)b.h[2]);
    // w: radius of a ball about the centre containing the box (padded beyond FP32 error)
    const double rbox = std::sqrt(b.h[0] * b.h[0] + b.h[1] * b.h[1] + b.h[2] * b.h[2]);
    bx[3 * n_box + j] = make_float4((float)b.R[2], (float)b.R[5], (float)b.R[8],
                                    round_up(rbox * (1.0 + 1e-6) + 1e-6));
    std::array<double, 6> a;
    for (int r = 0; r < 3; ++r) {  // world half-extent along axis r: sum_k |R[r][k]| h_k
      const double ext = std::fabs(b.R[3 * r]) * b.h[0] + std::fabs(b.R[3 * r + 1]) * b.h[1] +
                         std::fabs(b.R[3 * r + 2]) * b.h[2];
      a[r] = b.c[r] - ext;
      a[3 + r] = b.c[r] + ext;
    }
    aabb[n_sph + j] = a;
  }
  cen.resize(n_cap);
  for (int i = 0; i < n_cap; ++i) {
    const cprrtc_obs_capsule& c = cap[i];
    for (int k = 0; k < 3; ++k)
      if (!is_finite(c.p0[k]) || !is_finite(c.p1[k]))
        return fail(ctx, CPRRTC_E_INVALID_ARG, "obstacles: bad capsule " + std::to_string(i));
    if (!is_finite(c.r) || c.r < 0) return fail(ctx, CPRRTC_E_INVALID_ARG, "obstacles: bad capsule radius");
    cen[i] = {0.5 * (c.p0[0] + c.p1[0]), 0.5 * (c.p0[1] + c.p1[1]), 0.5 * (c.p0[2] + c.p1[2])};
  }
  ord = morton_order(cen);
  float4* cp = bx + 4 * n_box;
  for (int j = 0; j < n_cap; ++j) {
    const cprrtc_obs_capsule& c = cap[ord[j]];
    const double u[3] = {c.p1[0] - c.p0[0], c.p1[1] - c.p0[1], c.p1[2] - c.p0[2]};
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    cp[j] = make_float4((float)c.p0[0], (float)c.p0[1], (float)c.p0[2], (float)c.r);
    cp[n_cap + j] = make_float4((float)u[0], (float)u[1], (float)u[2], uu > 0 ? (float)(1.0 / uu) : 0.f);
    std::array<double, 6> a;
    for (int k = 0; k < 3; ++k) {
      a[k] = std::min(c.p0[k], c.p1[k]) - c.r;
      a[3 + k] = std::max(c.p0[k], c.p1[k]) + c.r;
    }
    aabb[n_sph + n_box + j] = a;
  }
  // chunk boxes, padded by 1e-5 m beyond the FP32 values the kernels test against
  float4* cb = cp + 2 * n_cap;
  for (int ch = 0; ch < n_chunks; ++ch) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int o = layout.chunk_first(ch); o < layout.chunk_end(ch); ++o)
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], aabb[o][k]);
        hi[k] = std::max(hi[k], aabb[o][3 + k]);
      }
    cb[2 * ch] = make_float4(round_down(lo[0] - 1e-5), round_down(lo[1] - 1e-5), round_down(lo[2] - 1e-5), 0.f);
    cb[2 * ch + 1] = make_float4(round_up(hi[0] + 1e-5), round_up(hi[1] + 1e-5), round_up(hi[2] + 1e-5), 0.f);
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
  ctx->cs = ConsDev{kConsNone, 0.f, 0.f, 0.f, 1e-4f, 2.f, 1e-3f, 1e-4f, 1.f, 1e-6f, 20};
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
  cudaFree(ctx->d_tab_sph);
  for (void* b : ctx->batch_net_buf) cudaFree(b);
  cudaFree(ctx->d_tab_frm);
  mlp_destroy(ctx->mlp);
  cudaFree(ctx->d_warm);
  cudaFree(ctx->d_bimage);
  cudaFree(ctx->d_cc_counters);
  cudaFree(ctx->d_cc_error);
  cudaFree(ctx->d_cc_q);
  cudaFree(ctx->d_cc_ff);
  for (BatchRes* r : {&ctx->batch_res, &ctx->graph_res}) {
    cudaFree(r->d_probs);
    cudaFree(r->d_order);
    cudaFree(r->d_counters);
    cudaFree(r->d_scratch);
    cudaFree(r->d_span);
  }
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  for (int c = 0; c < 2 * kBatchClasses; ++c) {
    if (ctx->side[c]) cudaStreamDestroy(ctx->side[c]);
    if (ctx->ev_join[c]) cudaEventDestroy(ctx->ev_join[c]);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
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

}  // extern "C"

namespace {

// Validates one robot and converts it to the kernels' form: FP32 joint table, spheres sorted
// by frame (loc, frm) and per-frame bounding spheres. Device pointers are left unset.
int build_robot(cprrtc_ctx* ctx, const cprrtc_joint* joints, int dof, const cprrtc_sphere* spheres,
                int n_spheres, const double ee[3], RobotDev& rb, std::vector<float4>& loc,
                std::vector<int>& frm) {
  if (!joints || !spheres || !ee) return fail(ctx, CPRRTC_E_INVALID_ARG, "set_robot: null pointer");
  if (dof < 1 || dof > CPRRTC_MAX_DOF)
    return fail(ctx, dof < 1 ? CPRRTC_E_INVALID_ARG : CPRRTC_E_UNSUPPORTED, "set_robot: dof must be in [1, 8]");
  if (n_spheres < 1 || n_spheres > CPRRTC_MAX_SPHERES)
    return fail(ctx, n_spheres < 1 ? CPRRTC_E_INVALID_ARG : CPRRTC_E_UNSUPPORTED,
                "set_robot: n_spheres must be in [1, 256]");
  rb = RobotDev{};
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
  loc.assign(n_spheres, make_float4(0.f, 0.f, 0.f, 0.f));
  frm.assign(n_spheres, 0);
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
  return CPRRTC_OK;
}

}  // namespace

extern "C" {

static int build_cc_image(cprrtc_ctx* ctx);

int cprrtc_set_robot(cprrtc_ctx* ctx, const cprrtc_joint* joints, int dof,
                     const cprrtc_sphere* spheres, int n_spheres, const double ee[3]) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  RobotDev rb;
  std::vector<float4> loc;
  std::vector<int> frm;
  int rc0 = build_robot(ctx, joints, dof, spheres, n_spheres, ee, rb, loc, frm);
  if (rc0) return rc0;
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
  ctx->self_on = false;  // frame pairs belong to a robot: set them again for a new one
  ctx->host_robot_sph = loc;
  if (ctx->cc_mode != CPRRTC_CC_EXACT) return build_cc_image(ctx);  // the bound depends on the robot
  return CPRRTC_OK;
}

// ---- collision checking in GEMM form: the obstacle operand and its error bound ----

namespace {

// Round-to-nearest-even of an FP32 value to `bits` significant bits (BF16 8, TF32 11).
float round_bits(float x, int bits) {
  uint32_t u;
  memcpy(&u, &x, 4);
  const int drop = 24 - bits;
  const uint32_t half = (1u << (drop - 1)) - 1u + ((u >> drop) & 1u);
  u = (u + half) & ~((1u << drop) - 1u);
  float r;
  memcpy(&r, &u, 4);
  return r;
}

// Byte offset of byte `kb` (< 128) of row r in the 128-byte-swizzle layout.
size_t sw128_host(int r, int kb) {
  return (size_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((kb >> 4) & 7) ^ (r & 7)) << 4) + (kb & 15));
}

}  // namespace

// Builds the obstacle operand B' of the GEMM-form check for the current mode (layout and
// columns as described in gemm_cc.cu) and the bound E on the contraction's error.
static int build_cc_image(cprrtc_ctx* ctx) {
  const bool tf32 = ctx->cc_mode == CPRRTC_CC_GEMM_TF32;
  const int bits = tf32 ? 11 : 8, elem = tf32 ? 4 : 2, slice = 16 * elem, tpr = 128 / slice;
  const int n = (int)ctx->host_sph.size();
  const int tiles = std::max(1, (n + 255) / 256);
  const int chunks = (tiles + tpr - 1) / tpr;
  // origin: centre of the obstacles' bounding box
  double lo[3] = {1e30, 1e30, 1e30}, hi[3] = {-1e30, -1e30, -1e30};
  double rho_max = 0.0;
  for (const float4& o : ctx->host_sph) {
    const double c[3] = {o.x, o.y, o.z};
    for (int k = 0; k < 3; ++k) lo[k] = std::min(lo[k], c[k]), hi[k] = std::max(hi[k], c[k]);
    rho_max = std::max(rho_max, (double)o.w);
  }
  float4 ori = make_float4(0.f, 0.f, 0.f, (float)(0.5 * ctx->cc_guard));
  if (n > 0) ori = make_float4((float)(0.5 * (lo[0] + hi[0])), (float)(0.5 * (lo[1] + hi[1])),
                               (float)(0.5 * (lo[2] + hi[2])), (float)(0.5 * ctx->cc_guard));
  const double g2 = ori.w;
  std::vector<uint8_t> img((size_t)chunks * 32768, 0);
  auto put = [&](int j, int col, double v) {
    const int t = j / 256, r = j % 256;
    const size_t off = (size_t)(t / tpr) * 32768 + sw128_host(r, (t % tpr) * slice + col * elem);
    const float f = round_bits((float)v, bits);
    if (tf32) {
      memcpy(&img[off], &f, 4);
    } else {
      uint32_t u;
      memcpy(&u, &f, 4);
      const uint16_t h = (uint16_t)(u >> 16);  // exact: f has 8 significant bits
      memcpy(&img[off], &h, 2);
    }
  };
  auto split = [&](double v, double& h, double& l) {
    h = round_bits((float)v, bits);
    l = (double)round_bits((float)(v - h), bits);
  };
  double lb = 0.0;
  for (int j = 0; j < tiles * 256; ++j) {
    if (j >= n) {  // padding obstacle: s = 1e4
      put(j, 12, 1e4);
      continue;
    }
    const float4 o = ctx->host_sph[j];
    const double b[3] = {(double)o.x - ori.x, (double)o.y - ori.y, (double)o.z - ori.z};
    const double rp = (double)o.w + g2;
    double h, l;
    for (int k = 0; k < 3; ++k) {
      split(b[k], h, l);
      put(j, 3 * k, h);
      put(j, 3 * k + 1, l);
      put(j, 3 * k + 2, h);
    }
    put(j, 9, 1.0);
    put(j, 10, 1.0);
    put(j, 11, rp);
    const double beta = b[0] * b[0] + b[1] * b[1] + b[2] * b[2] - rp * rp;
    split(beta, h, l);
    put(j, 12, h);
    put(j, 13, l);
    lb = std::max(lb, std::sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]));
  }
  // reach of the robot spheres from the origin: |base - origin| + sum of link lengths,
  // offsets and prismatic travel + largest sphere offset in its frame
  double reach = std::sqrt((double)ori.x * ori.x + (double)ori.y * ori.y + (double)ori.z * ori.z);
  for (int k = 0; k < ctx->rb.dof; ++k) {
    const JointDev& J = ctx->rb.j[k];
    reach += std::fabs(J.a) + std::fabs(J.d) +
             (J.prismatic ? std::max(std::fabs(J.lo), std::fabs(J.hi)) : 0.0);
  }
  double off_max = 0.0, r_max = 0.0;
  for (const float4& sp : ctx->host_robot_sph) {
    off_max = std::max(off_max, std::sqrt((double)sp.x * sp.x + (double)sp.y * sp.y + (double)sp.z * sp.z));
    r_max = std::max(r_max, (double)sp.w);
  }
  const double la = reach + off_max, u = std::ldexp(1.0, -bits);
  const double rpm = r_max + g2, rhom = rho_max + g2;
  const double cross = 2.0 * la * lb, amax = la * la + rpm * rpm, bmax = lb * lb + rhom * rhom, rr = 2.0 * rpm * rhom;
  // dropped lo*lo terms and the rounding of every split part (lo parts of TF32 operands may
  // be truncated by the hardware), -2r' and rho' rounded once each, alpha evaluated in FP32,
  // and the FP32 accumulation of 16 products (allowing 8x the textbook summation bound)
  const double e_split = 5.0 * u * u * cross + 2.0 * u * u * (amax + bmax) + 2.01 * u * rr;
  const double e_fp32 = std::ldexp(1.0, -21) * amax;
  const double e_acc = 16.0 * std::ldexp(1.0, -21) * (3.0 * cross + amax + bmax + rr);
  ctx->cc_bound = 1.5 * (e_split + e_fp32 + e_acc);
  ctx->cc_origin = ori;
  ctx->cc_tiles = tiles;
  DeviceGuard gd(ctx->device);
  if (img.size() > ctx->bimage_cap) {
    cudaFree(ctx->d_bimage);
    ctx->d_bimage = nullptr;
    ctx->bimage_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->d_bimage, img.size());
    if (e != cudaSuccess) return cuda_fail(ctx, e, "GEMM-form obstacle image");
    ctx->bimage_cap = img.size();
  }
  cudaError_t e = cudaMemcpy(ctx->d_bimage, img.data(), img.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "GEMM-form obstacle image upload");
  return CPRRTC_OK;
}

int cprrtc_set_cc_mode(cprrtc_ctx* ctx, int mode, double guard_m) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (mode != CPRRTC_CC_EXACT && mode != CPRRTC_CC_GEMM_TF32 && mode != CPRRTC_CC_GEMM_BF16)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_cc_mode: unknown mode");
  if (!(guard_m >= 0.0) || !(guard_m <= 0.1))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_cc_mode: guard must be in [0, 0.1] m");
  if (mode != CPRRTC_CC_EXACT && !ctx->has_robot)
    return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "set_cc_mode: set_robot first");
  ctx->cc_mode = mode;
  ctx->cc_guard = guard_m;
  if (mode == CPRRTC_CC_EXACT) return CPRRTC_OK;
  DeviceGuard g(ctx->device);
  if (!ctx->d_cc_counters) {
    // word 0: rechecks, word 1: unused, word 2: the kernel's motion counter
    cudaError_t e = cudaMalloc(&ctx->d_cc_counters, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_cc_counters, 0, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_cc_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_cc_error, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set_cc_mode");
  }
  return build_cc_image(ctx);
}

int cprrtc_cc_stats(cprrtc_ctx* ctx, double* bound_m2, int64_t* counters, int reset) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (bound_m2) *bound_m2 = ctx->cc_mode == CPRRTC_CC_EXACT ? 0.0 : ctx->cc_bound;
  if (!ctx->d_cc_counters) {
    if (counters) counters[0] = counters[1] = 0;
    return CPRRTC_OK;
  }
  DeviceGuard g(ctx->device);
  unsigned long long h[2] = {0, 0};
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpy(h, ctx->d_cc_counters, sizeof(h), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && reset) e = cudaMemset(ctx->d_cc_counters, 0, sizeof(h));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cc_stats");
  if (counters) {
    counters[0] = (int64_t)h[0];
    counters[1] = (int64_t)h[1];
  }
  return CPRRTC_OK;
}

int cprrtc_set_obstacles(cprrtc_ctx* ctx, const cprrtc_obs_sphere* sph, int n_sph,
                         const cprrtc_obs_box* box, int n_box, const cprrtc_obs_capsule* cap,
                         int n_cap) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (n_sph < 0 || n_box < 0 || n_cap < 0 || (n_sph && !sph) || (n_box && !box) || (n_cap && !cap))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_obstacles: bad counts or null pointer");
  if ((long long)n_sph + 4LL * n_box + 2LL * n_cap > (1LL << 26) || (long long)n_sph + n_box + n_cap > (1LL << 20))
    return fail(ctx, CPRRTC_E_UNSUPPORTED, "set_obstacles: too many obstacles");
  std::vector<float4> v;
  int rc = pack_obstacles(ctx, sph, n_sph, box, n_box, cap, n_cap, v);
  if (rc) return rc;
  DeviceGuard g(ctx->device);
  rc = upload(ctx, &ctx->d_obs, &ctx->obs_cap, v);
  if (rc) return rc;
  ctx->sc = SceneDev{ctx->d_obs, n_sph, n_box, n_cap};
  ctx->host_sph.assign(v.begin(), v.begin() + n_sph);
  if (ctx->cc_mode != CPRRTC_CC_EXACT) return build_cc_image(ctx);
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
  if (c->type < CPRRTC_CONSTRAINT_NONE || c->type > CPRRTC_CONSTRAINT_ORIENT_LINE)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_constraint: unknown type");
  if (c->max_iters < 1 || c->max_iters > 255)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_constraint: max_iters must be in [1, 255]");
  if (!is_finite(c->target) || !is_finite(c->line_y) || !is_finite(c->yaw) ||
      !(c->tol_task > 0) || !(c->tol_sm > 0) || !(c->c_sm > 0) ||
      !(c->tau_floor >= 0) || !is_finite(c->alpha) || !(c->lambda >= 0) || !is_finite(c->lambda) ||
      !is_finite(c->tol_task) || !is_finite(c->tol_sm) || !is_finite(c->c_sm) || !is_finite(c->tau_floor))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_constraint: bad parameter");
  ctx->cs = ConsDev{c->type,          (float)c->target,    (float)c->line_y,
                    (float)c->yaw,    (float)c->tol_task,  (float)c->c_sm,
                    (float)c->tau_floor, (float)c->tol_sm, (float)c->alpha,
                    (float)(c->lambda * c->lambda), c->max_iters};
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
  a.no_early_exit = !ctx->early_exit;
  a.sequential = ctx->projection == CPRRTC_PROJECTION_SEQUENTIAL;
  if (a.sequential && ctx->cs.type != kConsNone && ctx->cs.type != kConsRollPitch &&
      ctx->cs.type != kConsZPlane)
    return fail(ctx, CPRRTC_E_UNSUPPORTED, "validate: the sequential projection takes ROLL_PITCH or Z_PLANE");
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
  const bool gemm = ctx->cc_mode != CPRRTC_CC_EXACT;
  if (gemm || ctx->self_on) {
    // the GEMM-form check and the self-collision pass need the projected waypoints and a
    // first-failure array even when the caller does not ask for them
    if (!a.out_q) {
      const size_t need = N * W * dof * sizeof(float);
      if (need > ctx->cc_q_cap) {
        cudaFree(ctx->d_cc_q);
        ctx->d_cc_q = nullptr;
        ctx->cc_q_cap = 0;
        cudaError_t e = cudaMalloc(&ctx->d_cc_q, need);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "validate: waypoint buffer");
        ctx->cc_q_cap = need;
      }
      a.out_q = ctx->d_cc_q;
    }
    if (!a.first_fail) {
      const size_t need = N * sizeof(int32_t);
      if (need > ctx->cc_ff_cap) {
        cudaFree(ctx->d_cc_ff);
        ctx->d_cc_ff = nullptr;
        ctx->cc_ff_cap = 0;
        cudaError_t e = cudaMalloc(&ctx->d_cc_ff, need);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "validate: first-failure buffer");
        ctx->cc_ff_cap = need;
      }
      a.first_fail = ctx->d_cc_ff;
    }
  }
  if (gemm) {
    // projection only here
    if (ctx->sc.n_box || ctx->sc.n_cap)
      return fail(ctx, CPRRTC_E_UNSUPPORTED, "validate: the GEMM-form check takes sphere obstacles only");
    if (ctx->rb.n_spheres > 128)
      return fail(ctx, CPRRTC_E_UNSUPPORTED, "validate: the GEMM-form check takes at most 128 robot spheres");
    a.skip_cc = 1;
  }
  LaunchTimer tm(ctx, "validate");
  cudaError_t e = launch_validate(ctx->rb, ctx->sc, ctx->cs, a, ctx->dev, ctx->stream);
  tm.done();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "validate launch");
  if (gemm) {
    GemmCcArgs g{};
    g.q = a.out_q;
    g.n = n;
    g.W = W;
    g.status = a.status;
    g.first_fail = a.first_fail;
    g.bimage = ctx->d_bimage;
    g.n_tiles = ctx->cc_tiles;
    g.obs = ctx->sc.obs;
    g.n_obs = ctx->sc.n_sph;
    g.origin = ctx->cc_origin;
    g.bound = (float)ctx->cc_bound;
    g.counters = ctx->d_cc_counters;
    g.error = ctx->d_cc_error;
    g.next = reinterpret_cast<int*>(ctx->d_cc_counters + 2);
    g.wait_ns = ctx->wait_ns;
    e = cudaMemsetAsync(g.next, 0, sizeof(int), ctx->stream);
    // a timeout of an earlier call must not be reported again
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_cc_error, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "validate: GEMM-form scheduling counter");
    LaunchTimer tg(ctx, "gemm_cc");
    e = launch_gemm_cc(ctx->cc_mode == CPRRTC_CC_GEMM_TF32, ctx->rb, g, ctx->dev.sm_count, ctx->stream);
    tg.done();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "validate: GEMM-form check launch");
  }
  if (ctx->self_on) {
    SelfArgs sa{};
    sa.q = a.out_q;
    sa.n = n;
    sa.W = W;
    sa.i0 = a.cc_skip_first;
    sa.status = a.status;
    sa.first_fail = a.first_fail;
    for (int f = 0; f <= kMaxDof; ++f) sa.rows[f] = ctx->self_rows[f];
    LaunchTimer ts(ctx, "self_collide");
    e = launch_self_collide(ctx->rb, sa, ctx->stream);
    ts.done();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "validate: self-collision launch");
  }
  rc = st.end(ctx);
  if (rc == CPRRTC_OK && gemm && st.any_host) {
    int flag = 0;
    e = cudaMemcpy(&flag, ctx->d_cc_error, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "validate: GEMM-form status");
    if (flag) return fail(ctx, CPRRTC_E_TIMEOUT, "validate: a wait of the GEMM-form check timed out");
  }
  return rc;
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

// ---- learned warm start ----

int64_t cprrtc_mlp_param_count(int dof) {
  if (dof < 1 || dof > CPRRTC_MAX_DOF) return 0;
  return (int64_t)mlp_compact_count(dof);
}

int cprrtc_mlp_init(cprrtc_ctx* ctx, uint64_t seed) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!ctx->has_robot) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "mlp_init: set_robot first");
  DeviceGuard g(ctx->device);
  if (ctx->mlp) {
    cudaStreamSynchronize(ctx->stream);
    mlp_destroy(ctx->mlp);
    ctx->mlp = nullptr;
  }
  cudaError_t e = mlp_create(&ctx->mlp, ctx->rb.dof);
  if (e == cudaSuccess) {
    mlp_set_fp32(ctx->mlp, ctx->mlp_fp32);
    mlp_set_wait_ns(ctx->mlp, ctx->wait_ns);
  }
  if (e == cudaSuccess) e = mlp_init(ctx->mlp, seed, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_init");
  return CPRRTC_OK;
}

int cprrtc_set_plan_warm_start(cprrtc_ctx* ctx, int refine_iters) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (refine_iters < 0 || refine_iters > 20)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_plan_warm_start: refine_iters 0..20");
  ctx->plan_warm = refine_iters;
  return CPRRTC_OK;
}

int cprrtc_set_plan_slicing(cprrtc_ctx* ctx, int first_slice, int slice) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (first_slice < 0 || (first_slice > 0 && slice < 1))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_plan_slicing: first_slice >= 0, slice >= 1");
  ctx->plan_first_slice = first_slice;
  ctx->plan_slice = first_slice > 0 ? slice : 0;
  return CPRRTC_OK;
}

int cprrtc_set_wait_limit(cprrtc_ctx* ctx, double seconds) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!(seconds == 0.0 || (seconds >= 1e-6 && seconds <= 10.0)))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_wait_limit: 0 (default) or 1e-6 .. 10 seconds");
  ctx->wait_ns = (unsigned long long)(seconds * 1e9);
  if (ctx->mlp) mlp_set_wait_ns(ctx->mlp, ctx->wait_ns);
  return CPRRTC_OK;
}

int cprrtc_mlp_set_precision(cprrtc_ctx* ctx, int precision) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (precision != CPRRTC_MLP_BF16 && precision != CPRRTC_MLP_FP32)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_set_precision: CPRRTC_MLP_BF16 or CPRRTC_MLP_FP32");
  ctx->mlp_fp32 = precision == CPRRTC_MLP_FP32;
  if (ctx->mlp) mlp_set_fp32(ctx->mlp, ctx->mlp_fp32);
  return CPRRTC_OK;
}

static int mlp_ready(cprrtc_ctx* ctx, const char* who) {
  if (!ctx->mlp) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, std::string(who) + ": call mlp_init first");
  if (!ctx->has_robot || mlp_dof(ctx->mlp) != ctx->rb.dof)
    return fail(ctx, CPRRTC_E_NOT_CONFIGURED, std::string(who) + ": network dof differs from the robot's");
  return CPRRTC_OK;
}

int cprrtc_mlp_set_params(cprrtc_ctx* ctx, const float* params, int64_t count) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!ctx->mlp) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "mlp_set_params: call mlp_init first");
  if (!params || count != (int64_t)mlp_compact_count(mlp_dof(ctx->mlp)) || is_device_ptr(params))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_set_params: host array of mlp_param_count(dof) floats");
  DeviceGuard g(ctx->device);
  cudaError_t e = mlp_set_params(ctx->mlp, params, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_set_params");
  return CPRRTC_OK;
}

int cprrtc_mlp_get_params(cprrtc_ctx* ctx, float* params, int64_t count) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!ctx->mlp) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "mlp_get_params: call mlp_init first");
  if (!params || count != (int64_t)mlp_compact_count(mlp_dof(ctx->mlp)) || is_device_ptr(params))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_get_params: host array of mlp_param_count(dof) floats");
  DeviceGuard g(ctx->device);
  cudaError_t e = mlp_get_params(ctx->mlp, params, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_get_params");
  return CPRRTC_OK;
}

// ---- warm-start network checkpoints ----

namespace {

// CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320), bitwise.
uint32_t crc32_update(uint32_t crc, const uint8_t* p, size_t n) {
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) {
    crc ^= p[i];
    for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
  }
  return ~crc;
}

const char kCkptMagic[8] = {'C', 'P', 'R', 'M', 'L', 'P', '0', '1'};
constexpr uint32_t kCkptVersion = 1;

struct CkptHeader {
  char magic[8];
  uint32_t version, dof, hidden, layers;
  int32_t step;
  uint32_t reserved;
  uint64_t count;
};

}  // namespace

int cprrtc_mlp_save(cprrtc_ctx* ctx, const char* path) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!ctx->mlp) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "mlp_save: call mlp_init first");
  if (!path) return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_save: null path");
  DeviceGuard g(ctx->device);
  const int dof = mlp_dof(ctx->mlp);
  const size_t n = mlp_compact_count(dof);
  std::vector<float> p(n), m(n), v(n);
  CkptHeader h{};
  memcpy(h.magic, kCkptMagic, 8);
  h.version = kCkptVersion;
  h.dof = (uint32_t)dof;
  h.hidden = (uint32_t)kMlpHidden;
  h.layers = (uint32_t)kMlpLayers;
  h.count = n;
  int step = 0;
  cudaError_t e = mlp_get_state(ctx->mlp, p.data(), m.data(), v.data(), &step, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_save");
  h.step = step;
  std::vector<uint8_t> buf(sizeof(h) + 3 * n * 4 + 4);
  uint8_t* o = buf.data();
  memcpy(o, &h, sizeof(h));
  memcpy(o + sizeof(h), p.data(), n * 4);
  memcpy(o + sizeof(h) + n * 4, m.data(), n * 4);
  memcpy(o + sizeof(h) + 2 * n * 4, v.data(), n * 4);
  const uint32_t crc = crc32_update(0u, o, buf.size() - 4);
  memcpy(o + buf.size() - 4, &crc, 4);
  FILE* f = fopen(path, "wb");
  if (!f) return fail(ctx, CPRRTC_E_INVALID_ARG, std::string("mlp_save: cannot open ") + path);
  const size_t w = fwrite(buf.data(), 1, buf.size(), f);
  const int closed = fclose(f);
  if (w != buf.size() || closed != 0) return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_save: write failed");
  return CPRRTC_OK;
}

int cprrtc_mlp_load(cprrtc_ctx* ctx, const char* path) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!ctx->has_robot) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "mlp_load: set_robot first");
  if (!path) return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_load: null path");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(ctx, CPRRTC_E_INVALID_ARG, std::string("mlp_load: cannot open ") + path);
  std::vector<uint8_t> buf;
  uint8_t chunk[65536];
  size_t r;
  while ((r = fread(chunk, 1, sizeof(chunk), f)) > 0) buf.insert(buf.end(), chunk, chunk + r);
  fclose(f);
  CkptHeader h{};
  if (buf.size() < sizeof(h) + 4) return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_load: truncated file");
  memcpy(&h, buf.data(), sizeof(h));
  if (memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != kCkptVersion)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_load: not a warm-start checkpoint of this version");
  if (h.dof != (uint32_t)ctx->rb.dof || h.hidden != (uint32_t)kMlpHidden || h.layers != (uint32_t)kMlpLayers ||
      h.count != mlp_compact_count(ctx->rb.dof))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_load: network shape differs from the robot's");
  const size_t n = (size_t)h.count;
  if (buf.size() != sizeof(h) + 3 * n * 4 + 4) return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_load: bad size");
  uint32_t crc;
  memcpy(&crc, buf.data() + buf.size() - 4, 4);
  if (crc != crc32_update(0u, buf.data(), buf.size() - 4))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_load: checksum mismatch");
  DeviceGuard g(ctx->device);
  if (!ctx->mlp || mlp_dof(ctx->mlp) != ctx->rb.dof) {
    if (ctx->mlp) {
      cudaStreamSynchronize(ctx->stream);
      mlp_destroy(ctx->mlp);
      ctx->mlp = nullptr;
    }
    cudaError_t e = mlp_create(&ctx->mlp, ctx->rb.dof);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_load");
    mlp_set_fp32(ctx->mlp, ctx->mlp_fp32);
    mlp_set_wait_ns(ctx->mlp, ctx->wait_ns);
  }
  std::vector<float> p(n), m(n), v(n);
  memcpy(p.data(), buf.data() + sizeof(h), n * 4);
  memcpy(m.data(), buf.data() + sizeof(h) + n * 4, n * 4);
  memcpy(v.data(), buf.data() + sizeof(h) + 2 * n * 4, n * 4);
  cudaError_t e = mlp_set_state(ctx->mlp, p.data(), m.data(), v.data(), h.step, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_load");
  return CPRRTC_OK;
}

int cprrtc_mlp_grad(cprrtc_ctx* ctx, const float* q, const float* t, int rows, float* grads,
                    float* loss) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (int rc = mlp_ready(ctx, "mlp_grad")) return rc;
  if (rows < 1 || !q || !t) return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_grad: rows >= 1 and data required");
  if ((grads && is_device_ptr(grads)) || (loss && is_device_ptr(loss)))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_grad: grads and loss are host arrays");
  DeviceGuard g(ctx->device);
  const size_t bytes = (size_t)rows * ctx->rb.dof * sizeof(float);
  const float *dq, *dt;
  Staging st;
  st.input(q, bytes, &dq);
  st.input(t, bytes, &dt);
  int rc = st.begin(ctx);
  if (rc) return rc;
  cudaError_t e = mlp_grad(ctx->mlp, dq, dt, rows, grads, loss, ctx->stream);
  if (e == cudaErrorTimeout)
    return fail(ctx, CPRRTC_E_TIMEOUT, "mlp_grad: a wait of a tensor-core GEMM timed out");
  if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_grad");
  return st.end(ctx);
}

int cprrtc_mlp_train(cprrtc_ctx* ctx, const float* q, const float* t, int n, int batch,
                     int epochs, float lr, uint64_t seed, float* loss_per_epoch) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (int rc = mlp_ready(ctx, "mlp_train")) return rc;
  if (batch < 1 || n < batch || epochs < 0 || !is_finite(lr) || !q || !t)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_train: need 1 <= batch <= n, epochs >= 0, finite lr");
  if (loss_per_epoch && is_device_ptr(loss_per_epoch))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_train: loss_per_epoch is a host array");
  if (epochs == 0) return CPRRTC_OK;
  DeviceGuard g(ctx->device);
  const size_t bytes = (size_t)n * ctx->rb.dof * sizeof(float);
  const float *dq, *dt;
  Staging st;
  st.input(q, bytes, &dq);
  st.input(t, bytes, &dt);
  int rc = st.begin(ctx);
  if (rc) return rc;
  LaunchTimer tm(ctx, "mlp_train");
  cudaError_t e = mlp_train(ctx->mlp, dq, dt, n, batch, epochs, lr, seed, loss_per_epoch, ctx->stream);
  tm.done();
  if (e == cudaErrorTimeout)
    return fail(ctx, CPRRTC_E_TIMEOUT, "mlp_train: a wait of a tensor-core GEMM timed out");
  if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_train");
  return st.end(ctx);
}

// q_out = q + correction, rows of [rows][dof]
__global__ void add_correction_kernel(const float* __restrict__ q, const float* __restrict__ y, int rows,
                                      int dof, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * dof) return;
  const int r = i / dof, k = i - r * dof;
  out[i] = q[i] + y[(size_t)r * 16 + k];
}

static int ensure_warm(cprrtc_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->warm_cap) return CPRRTC_OK;
  if (ctx->d_warm) cudaFree(ctx->d_warm);
  ctx->d_warm = nullptr;
  ctx->warm_cap = 0;
  cudaError_t e = cudaMalloc(&ctx->d_warm, bytes);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "warm-start buffer");
  ctx->warm_cap = bytes;
  return CPRRTC_OK;
}

int cprrtc_mlp_infer(cprrtc_ctx* ctx, const float* q, int rows, float* q_out) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (int rc = mlp_ready(ctx, "mlp_infer")) return rc;
  if (rows < 0) return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_infer: rows < 0");
  if (rows == 0) return CPRRTC_OK;
  if (!q || !q_out) return fail(ctx, CPRRTC_E_INVALID_ARG, "mlp_infer: null pointer");
  DeviceGuard g(ctx->device);
  const int dof = ctx->rb.dof;
  const size_t bytes = (size_t)rows * dof * sizeof(float);
  if (int rc = ensure_warm(ctx, (size_t)rows * 16 * sizeof(float))) return rc;
  const float* dq;
  float* dout;
  Staging st;
  st.input(q, bytes, &dq);
  st.output(q_out, bytes, &dout);
  int rc = st.begin(ctx);
  if (rc) return rc;
  LaunchTimer tm(ctx, "mlp_infer");
  cudaError_t e = mlp_infer(ctx->mlp, dq, dof, rows, ctx->d_warm, ctx->stream);
  if (e == cudaSuccess) {
    const int tot = rows * dof;
    add_correction_kernel<<<(tot + 255) / 256, 256, 0, ctx->stream>>>(dq, ctx->d_warm, rows, dof, dout);
    e = cudaGetLastError();
  }
  tm.done();
  if (e != cudaSuccess) return cuda_fail(ctx, e, (std::string("mlp_infer ") + mlp_fused_diag()).c_str());
  rc = st.end(ctx);
  if (rc == CPRRTC_OK && st.any_host) {
    int flag = 0;
    e = cudaMemcpy(&flag, mlp_error_flag(ctx->mlp), sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_infer status");
    if (flag) return fail(ctx, CPRRTC_E_TIMEOUT, "mlp_infer: a wait of the inference kernel timed out");
  }
  return rc;
}

int cprrtc_validate_ws(cprrtc_ctx* ctx, const float* q_start, const float* q_end, int n, int W,
                       int refine_iters, float* out_q, uint8_t* status, int32_t* first_fail,
                       uint8_t* iters, float* resid, uint8_t* warm_used) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!ctx->has_robot) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "validate_ws: set_robot first");
  if (ctx->cs.type == kConsNone)
    return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "validate_ws: constraint is NONE");
  if (int rc = mlp_ready(ctx, "validate_ws")) return rc;
  if (n < 0) return fail(ctx, CPRRTC_E_INVALID_ARG, "validate_ws: n < 0");
  if (refine_iters < 1 || refine_iters > 20)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "validate_ws: refine_iters must be in [1, 20]");
  if (W < 2 || W > CPRRTC_MAX_W)
    return fail(ctx, W < 2 ? CPRRTC_E_INVALID_ARG : CPRRTC_E_UNSUPPORTED, "validate_ws: W must be in [2, 64]");
  if (n == 0) return CPRRTC_OK;
  if (!q_start || !q_end || !status) return fail(ctx, CPRRTC_E_INVALID_ARG, "validate_ws: null pointer");
  DeviceGuard g(ctx->device);
  const size_t dof = ctx->rb.dof, N = (size_t)n;
  if (int rc = ensure_warm(ctx, N * W * 16 * sizeof(float))) return rc;
  ValidateArgs a{};
  a.n = n;
  a.W = W;
  a.cc_skip_first = 0;
  a.no_early_exit = !ctx->early_exit;
  a.work_counters = ctx->d_work;
  a.warm = ctx->d_warm;
  a.warm_error = mlp_error_flag(ctx->mlp);
  a.refine_iters = refine_iters;
  Staging st;
  st.input(q_start, N * dof * sizeof(float), &a.q_start);
  st.input(q_end, N * dof * sizeof(float), &a.q_end);
  st.output(out_q, N * W * dof * sizeof(float), &a.out_q);
  st.output(status, N, &a.status);
  st.output(first_fail, N * sizeof(int32_t), &a.first_fail);
  st.output(iters, N, &a.iters);
  st.output(resid, N * sizeof(float), &a.resid);
  st.output(warm_used, N, &a.warm_used);
  int rc = st.begin(ctx);
  if (rc) return rc;
  {
    LaunchTimer tm(ctx, "mlp_infer");
    cudaError_t e = mlp_infer_motions(ctx->mlp, a.q_start, a.q_end, n, W, ctx->d_warm, ctx->stream);
    tm.done();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "validate_ws inference");
  }
  LaunchTimer tm(ctx, "validate");
  cudaError_t e = launch_validate(ctx->rb, ctx->sc, ctx->cs, a, ctx->dev, ctx->stream);
  tm.done();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "validate_ws launch");
  return st.end(ctx);
}

namespace {
bool mul_within(size_t a, size_t b, size_t limit, size_t* out);  // a * b <= limit, no wrap-around
}  // namespace

int cprrtc_plan(cprrtc_ctx* ctx, const float* start, const float* goal, int n,
                const cprrtc_plan_params* pp, int32_t* path_len, float* path, float* path_edges,
                int32_t* rounds, int64_t* waypoints, float* plan_ms, int64_t* work) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!ctx->has_robot) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "plan: set_robot first");
  if (!pp) return fail(ctx, CPRRTC_E_INVALID_ARG, "plan: null params");
  if (n < 0) return fail(ctx, CPRRTC_E_INVALID_ARG, "plan: n < 0");
  if (pp->W < 2 || pp->W > CPRRTC_MAX_W || !(pp->range > 0) || !is_finite(pp->range) ||
      pp->max_rounds < 1 || pp->workers < 1 || pp->workers > kMaxWorkers || pp->max_nodes < 2 ||
      pp->max_connect < 0 || pp->max_path < 2 || !(pp->time_budget_ms >= 0.0) || !is_finite(pp->time_budget_ms))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "plan: bad parameters");
  if (pp->use_scene_batch && ctx->n_scenes != n)
    return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "plan: scene batch must hold one scene per problem");
  if (n == 0) return CPRRTC_OK;
  if (!start || !goal || !path_len || !path) return fail(ctx, CPRRTC_E_INVALID_ARG, "plan: null pointer");
  DeviceGuard g(ctx->device);
  if (int rc = check_plan_workers(ctx, pp, "plan")) return rc;
  const size_t dof = ctx->rb.dof, N = (size_t)n, W = (size_t)pp->W;
  const size_t B = (size_t)pp->workers, MN = (size_t)pp->max_nodes;
  {  // every product below stays far from wrapping around 2^64 (larger requests cannot be met)
    const size_t lim = (size_t)1 << 56;
    size_t trees = 0, tree_bytes = 0, worker_bytes = 0;
    if (!mul_within(N, 2 * MN, lim, &trees) ||
        !mul_within(trees, (W * dof + 9) * sizeof(float), lim, &tree_bytes) ||
        !mul_within(N, B * (2 * W * dof + 8) * sizeof(float), lim, &worker_bytes))
      return fail(ctx, CPRRTC_E_OOM, "plan: the trees of n problems of max_nodes exceed any device memory");
  }
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_nodes = al(N * 2 * MN * 8 * sizeof(float));
  const size_t b_parent = al(N * 2 * MN * sizeof(int));
  const size_t b_edges = al(N * 2 * MN * W * dof * sizeof(float));
  const size_t b_pend = al(N * B * 8 * sizeof(float));
  const size_t b_pedge = al(N * B * 2 * W * dof * sizeof(float));
  const bool sliced = ctx->plan_first_slice > 0;
  const size_t b_state = sliced ? al(N * sizeof(PlanState)) : 0;
  const size_t b_queue = sliced ? al(plan_queue_bytes(n)) : 0;
  const size_t b_status = sliced ? 256 : 0;
  const size_t need = b_nodes + b_parent + b_edges + b_pend + b_pedge + b_state + b_queue + b_status;
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
  a.budget_ns = pp->time_budget_ms > 0.0 ? (unsigned long long)(pp->time_budget_ms * 1e6) : 0ull;
  a.sequential = ctx->projection == CPRRTC_PROJECTION_SEQUENTIAL;
  a.work_counters = ctx->d_work;
  if (ctx->plan_warm > 0) {
    a.net = mlp_view(ctx->mlp);
    a.warm_refine = ctx->plan_warm;
  }
  a.self_on = ctx->self_on ? 1 : 0;
  for (int f = 0; f <= kMaxDof; ++f) a.self_rows[f] = ctx->self_rows[f];
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
  if (sliced) {
    char* sb = base + b_nodes + b_parent + b_edges + b_pend + b_pedge;
    a.state = reinterpret_cast<PlanState*>(sb);
    a.queue = reinterpret_cast<PlanQueue*>(sb + b_state);
    a.status = reinterpret_cast<int*>(sb + b_state + b_queue);
    a.first_slice = ctx->plan_first_slice;
    a.slice = ctx->plan_slice;
    cudaError_t e = cudaMemsetAsync(a.status, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plan: status");
  }
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
  rc = st.end(ctx);
  if (rc == CPRRTC_OK && sliced && st.any_host) {
    int flag = 0;
    e = cudaMemcpy(&flag, a.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plan status");
    if (flag) return fail(ctx, CPRRTC_E_TIMEOUT, "plan: a wait of the time-sliced queue timed out");
  }
  return rc;
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

int cprrtc_set_self_collision(cprrtc_ctx* ctx, const uint8_t* frame_pairs, int n) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (n == 0 || !frame_pairs) {
    ctx->self_on = false;
    return CPRRTC_OK;
  }
  if (!ctx->has_robot) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "set_self_collision: set_robot first");
  const int nf = ctx->rb.dof + 1;
  if (n != nf * nf)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_self_collision: n must be (dof + 1)^2");
  for (int f = 0; f <= kMaxDof; ++f) ctx->self_rows[f] = 0;
  bool any = false;
  for (int i = 0; i < nf; ++i)
    for (int j = i + 1; j < nf; ++j)
      if (frame_pairs[i * nf + j] || frame_pairs[j * nf + i]) {
        ctx->self_rows[i] |= (unsigned short)(1u << j);
        any = true;
      }
  ctx->self_on = any;
  return CPRRTC_OK;
}

int cprrtc_set_projection(cprrtc_ctx* ctx, int mode) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (mode != CPRRTC_PROJECTION_PARALLEL && mode != CPRRTC_PROJECTION_SEQUENTIAL)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_projection: unknown mode");
  ctx->projection = mode;
  return CPRRTC_OK;
}

int cprrtc_set_early_exit(cprrtc_ctx* ctx, int enabled) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  ctx->early_exit = enabled ? 1 : 0;
  return CPRRTC_OK;
}

int cprrtc_measure_fp32_peak(cprrtc_ctx* ctx, double* tflops) {
  if (!ctx || !tflops) return CPRRTC_E_INVALID_ARG;
  DeviceGuard g(ctx->device);
  cudaError_t e = measure_fp32_peak(ctx->dev, ctx->stream, tflops);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "measure_fp32_peak");
  return CPRRTC_OK;
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
unsigned long long g_static_ctx[kStaticMaxDevices] = {};  // context id the address belongs to

// Unique id of the current CUDA context (driver entry points looked up through the runtime,
// so the library does not link the driver library). 0 when unavailable.
unsigned long long current_context_id() {
  typedef int (*GetCurrentFn)(void**);
  typedef int (*GetIdFn)(void*, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrentFn>(f1);
      get_id = reinterpret_cast<GetIdFn>(f2);
    } else {
      cudaGetLastError();
    }
    looked_up = true;
  }
  void* c = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&c) != 0 || !c || get_id(c, &id) != 0) return 0;
  return id;
}

// Device address of g_plan_scratch on `device` (which must be current); nullptr on error.
// The address is looked up once per device and context: a device reset (cudaDeviceReset,
// or a reset of the primary context) creates a new context, whose id no longer matches, and
// the next call looks the address up again. Without the context id (an old driver) the
// address is looked up on every call.
void* static_scratch(int device, cudaError_t* err) {
  *err = cudaSuccess;
  if (device < 0 || device >= kStaticMaxDevices) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  const unsigned long long id = current_context_id();
  if (!g_static_ptr[device] || id == 0 || id != g_static_ctx[device]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_plan_scratch);
    if (*err != cudaSuccess) {
      g_static_ptr[device] = nullptr;
      return nullptr;
    }
    g_static_ptr[device] = p;
    g_static_ctx[device] = id;
  }
  return g_static_ptr[device];
}

// a * b into *out unless it exceeds `limit` (or overflows); false then.
bool mul_within(size_t a, size_t b, size_t limit, size_t* out) {
  if (a != 0 && b > limit / a) return false;
  *out = a * b;
  return *out <= limit;
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
      pp->max_connect < 0 || pp->max_path < 2 || !(pp->time_budget_ms >= 0.0) || !is_finite(pp->time_budget_ms))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "plan_static: bad parameters");
  if (pp->use_scene_batch && ctx->n_scenes != n)
    return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "plan_static: scene batch must hold one scene per problem");
  if (n == 0) return CPRRTC_OK;
  if (!start || !goal || !path_len || !path)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "plan_static: null pointer");
  DeviceGuard g(ctx->device);
  if (int rc = check_plan_workers(ctx, pp, "plan_static")) return rc;
  const void* arrays[] = {start, goal, path_len, path, path_edges, rounds, waypoints, plan_ms, work};
  for (const void* a : arrays)
    if (a && ptr_where(a, ctx->device) != kPtrHere)
      return fail(ctx, CPRRTC_E_INVALID_ARG,
                  "plan_static: every array must be device memory of the context's GPU");
  const size_t dof = ctx->rb.dof, N = (size_t)n, W = (size_t)pp->W;
  const size_t B = (size_t)pp->workers, MN = (size_t)pp->max_nodes;
  // Every product is bounded by the array's size before it is formed, so that no size wraps
  // around to a small value and passes the capacity check (the array is this call's only
  // guard: no allocation can fail first).
  const size_t cap = (size_t)CPRRTC_STATIC_SCRATCH_BYTES;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  size_t trees = 0, per_node = 0, b_tree_part = 0, workers_n = 0, per_worker = 0, b_w = 0;
  const bool fits = mul_within(N, 2 * MN, cap, &trees) &&         // tree nodes of all problems
                    mul_within(W * dof + 9, sizeof(float), cap, &per_node) &&
                    mul_within(trees, per_node, cap, &b_tree_part) &&
                    mul_within(N, B, cap, &workers_n) &&
                    mul_within(2 * W * dof + 8, sizeof(float), cap, &per_worker) &&
                    mul_within(workers_n, per_worker, cap, &b_w);
  size_t need = cap + 1;
  size_t b_nodes = 0, b_parent = 0, b_edges = 0, b_pend = 0, b_pedge = 0;
  if (fits) {
    b_nodes = al(trees * 8 * sizeof(float));
    b_parent = al(trees * sizeof(int));
    b_edges = al(trees * W * dof * sizeof(float));
    b_pend = al(workers_n * 8 * sizeof(float));
    b_pedge = al(workers_n * 2 * W * dof * sizeof(float));
    need = b_nodes + b_parent + b_edges + b_pend + b_pedge;
  }
  if (need > cap)
    return fail(ctx, CPRRTC_E_CAPACITY,
                std::string("plan_static: needs ") + (fits ? std::to_string(need) : std::string("more")) +
                    " bytes of scratch, the fixed array holds " + std::to_string(cap) +
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
  a.budget_ns = pp->time_budget_ms > 0.0 ? (unsigned long long)(pp->time_budget_ms * 1e6) : 0ull;
  a.sequential = ctx->projection == CPRRTC_PROJECTION_SEQUENTIAL;
  if (ctx->plan_warm > 0) {
    a.net = mlp_view(ctx->mlp);
    a.warm_refine = ctx->plan_warm;
  }
  a.self_on = ctx->self_on ? 1 : 0;
  for (int f = 0; f <= kMaxDof; ++f) a.self_rows[f] = ctx->self_rows[f];
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
  a.work_counters = ctx->d_work;  // allocated with the context: nothing is allocated here
  e = launch_plan(ctx->rb, ctx->sc, ctx->cs, a, ctx->dev, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "plan_static launch");
  return CPRRTC_OK;
}


// ---- batches of uneven problems ------------------------------------------------------------

namespace {

// Host-side preparation of a batch: problem descriptors, classes and dequeue orders.
struct BatchPlan {
  int n = 0;
  std::vector<int4> probs;
  std::vector<int> order;            // per class, concatenated
  std::vector<double> cost;          // estimated cost of order[i] (see prepare_batch)
  int off[kBatchClasses + 1] = {};   // class c: order[off[c] .. off[c + 1])
  int max_W[kBatchClasses] = {}, max_S[kBatchClasses] = {}, max_f4[kBatchClasses] = {};
  int max_W_all = 0;
  double work[kBatchClasses] = {};  // estimated cost of the class's problems (see prepare_batch)
  double work_all = 0.0;
};

int prepare_batch(cprrtc_ctx* ctx, const cprrtc_problem* probs, int n, BatchPlan& bp) {
  if (ctx->tab_robots.empty() || ctx->tab_cons.empty())
    return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "batch: set the robot and constraint tables first");
  if (ctx->n_scenes < 1) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "batch: set a scene batch first");
  if (!probs || n < 0) return fail(ctx, CPRRTC_E_INVALID_ARG, "batch: bad problems");
  if (is_device_ptr(probs)) return fail(ctx, CPRRTC_E_INVALID_ARG, "batch: problems must be host memory");
  std::vector<int4> scene_tab(ctx->n_scenes);
  if (cudaMemcpy(scene_tab.data(), ctx->d_batch_tab, sizeof(int4) * ctx->n_scenes,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_fail(ctx, cudaGetLastError(), "batch: scene table");
  bp = BatchPlan{};
  bp.n = n;
  bp.probs.resize(n);
  std::vector<std::pair<double, int>> cls[kBatchClasses];
  for (int p = 0; p < n; ++p) {
    const cprrtc_problem& q = probs[p];
    if (q.robot < 0 || q.robot >= (int)ctx->tab_robots.size() || q.constraint < 0 ||
        q.constraint >= (int)ctx->tab_cons.size() || q.scene < 0 || q.scene >= ctx->n_scenes ||
        q.W < 2 || q.W > CPRRTC_MAX_W)
      return fail(ctx, CPRRTC_E_INVALID_ARG, "batch: bad problem " + std::to_string(p));
    bp.probs[p] = make_int4(q.robot, q.constraint, q.scene, q.W);
    const RobotDev& r = ctx->tab_robots[q.robot];
    const int ct = ctx->tab_cons[q.constraint].type;
    const int c = 2 * ct + (q.W > 32 ? 1 : 0);
    const int4 sd = scene_tab[q.scene];
    const int n_obs = sd.y + sd.z + sd.w;
    const int f4 = SceneDev{nullptr, sd.y, sd.z, sd.w}.n_float4();
    // expected cost for longest-first ordering: waypoints x (obstacles + robot spheres)
    const double cost = (double)q.W * (n_obs + r.n_spheres) * (ct != kConsNone ? 2.0 : 1.0);
    cls[c].push_back({cost, p});
    bp.work[c] += cost;
    bp.work_all += cost;
    bp.max_W[c] = std::max(bp.max_W[c], q.W);
    bp.max_S[c] = std::max(bp.max_S[c], r.n_spheres);
    bp.max_f4[c] = std::max(bp.max_f4[c], f4);
    bp.max_W_all = std::max(bp.max_W_all, q.W);
  }
  for (int c = 0; c < kBatchClasses; ++c) {
    std::stable_sort(cls[c].begin(), cls[c].end(),
                     [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
                       return a.first > b.first;
                     });
    bp.off[c] = (int)bp.order.size();
    for (auto& e : cls[c]) {
      bp.order.push_back(e.second);
      bp.cost.push_back(e.first);
    }
  }
  bp.off[kBatchClasses] = (int)bp.order.size();
  return CPRRTC_OK;
}

cprrtc_tuning default_tuning() {
  cprrtc_tuning t{};
  for (int c = 0; c < kBatchClasses; ++c) {
    t.ctas_per_sm[c] = 0;
    t.stage_obstacles[c] = 1;
    t.warps_per_motion[c] = 1;
    t.pair_problems[c] = 0;
  }
  return t;
}

// Whether class c may run warp pairs: plain form, at most 8 workers (16 warps).
bool pairs_allowed(cprrtc_ctx* ctx, int workers) {
  return ctx->plan_warm <= 0 && 2 * workers <= kMaxWorkers;
}

// One launch of a batch: part 0 of class c plans its first n problems in longest-first
// order with warp pairs (the whole class with warps_per_motion = 2, else its pair_problems
// heaviest), part 1 the others with one warp per motion. Each part has its own queue
// counter, side stream and scratch slots.
constexpr int kBatchParts = 2 * kBatchClasses;
struct PartLaunch {
  bool on = false;
  int cls = 0, first = 0, n = 0;  // problems order[off[cls] + first .. + n)
  int workers = 8, grid = 0, stage = 0, K = 1, per_sm = 0;
  size_t smem = 0, slot_bytes = 0;
  double work = 0.0;
};

// Plans the parts of the classes in cls_mask under tuning t. A part that cannot be launched
// (shared memory or registers beyond an SM) is E_UNSUPPORTED.
int batch_parts(cprrtc_ctx* ctx, const BatchPlan& bp, const cprrtc_tuning& t, int workers,
                size_t max_nodes, unsigned cls_mask, PartLaunch (&P)[kBatchParts]) {
  for (auto& q : P) q = PartLaunch{};
  for (int c = 0; c < kBatchClasses; ++c) {
    const int nc = bp.off[c + 1] - bp.off[c];
    if (!((cls_mask >> c) & 1u) || nc == 0) continue;
    const bool pairs = pairs_allowed(ctx, workers);
    const int n_pair = !pairs ? 0 : t.warps_per_motion[c] == 2 ? nc : std::max(0, std::min(nc, t.pair_problems[c]));
    for (int part = 0; part < 2; ++part) {
      PartLaunch& L = P[2 * c + part];
      L.cls = c;
      L.first = part == 0 ? 0 : n_pair;
      L.n = part == 0 ? n_pair : nc - n_pair;
      if (L.n == 0) continue;
      for (int i = L.first; i < L.first + L.n; ++i) L.work += bp.cost[bp.off[c] + i];
      L.workers = workers;
      L.K = part == 0 ? 2 : 1;
      L.stage = t.stage_obstacles[c] ? 1 : 0;
      L.smem = plan_batch_smem_bytes(bp.max_f4[c], bp.max_S[c], bp.max_W[c], workers, L.stage, L.K);
      if (L.smem > ctx->dev.smem_optin) {
        L.stage = 0;
        L.smem = plan_batch_smem_bytes(bp.max_f4[c], bp.max_S[c], bp.max_W[c], workers, false, L.K);
      }
      const int occ = L.smem > ctx->dev.smem_optin
                          ? 0
                          : plan_batch_occupancy(c, workers, L.smem, ctx->plan_warm > 0, L.K);
      if (occ < 1)
        return fail(ctx, CPRRTC_E_UNSUPPORTED, "batch: class " + std::to_string(c) + " does not fit an SM");
      L.per_sm = part == 1 && t.ctas_per_sm[c] > 0 ? std::min(t.ctas_per_sm[c], occ) : occ;
      const size_t ew = (size_t)bp.max_W[c] * 8;
      L.slot_bytes = 2 * max_nodes * 8 * 4 + 2 * max_nodes * 4 + 2 * max_nodes * ew * 4 +
                     (size_t)workers * 8 * 4 + (size_t)workers * 2 * ew * 4;
    }
  }
  // The parts run concurrently, so each gets the share of the SMs that its estimated work is
  // of the batch's: every part's CTAs are resident from the start and begin with their
  // longest problems (a part given every SM would hold them until its queue is empty, and
  // the parts launched after it would start their longest problems late).
  for (auto& L : P) {
    if (L.n == 0) continue;
    const double share = bp.work_all > 0.0 ? L.work / bp.work_all : 1.0;
    const int sms = std::max(1, (int)std::floor(share * ctx->dev.sm_count));
    L.grid = std::min(L.n, L.per_sm * sms);
    L.on = L.grid > 0;
  }
  return CPRRTC_OK;
}

// Scratch of the parts, each part's slots 256-byte aligned, in part order.
size_t parts_scratch(const PartLaunch (&P)[kBatchParts], size_t (*off)[kBatchParts + 1] = nullptr) {
  size_t total = 0;
  for (int i = 0; i < kBatchParts; ++i) {
    if (off) (*off)[i] = total;
    if (P[i].on) total += (P[i].slot_bytes * P[i].grid + 255) & ~size_t(255);
  }
  if (off) (*off)[kBatchParts] = total;
  return total;
}

template <class T>
int ensure(cprrtc_ctx* ctx, T** p, size_t* cap, size_t count) {
  if (count <= *cap && *p) return CPRRTC_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch allocation");
  *cap = std::max<size_t>(count, 1);
  return CPRRTC_OK;
}

// Uploads the problems and orders, sizes the per-CTA scratch and launches the parts of the
// classes in cls_mask concurrently on side streams joined back into the context's stream.
int run_batch(cprrtc_ctx* ctx, const BatchPlan& bp, BatchRes& res, PlanArgs base,
              const cprrtc_tuning& t, unsigned cls_mask, bool capturing) {
  PartLaunch P[kBatchParts];
  const size_t MN = (size_t)base.max_nodes;
  int rc = batch_parts(ctx, bp, t, base.workers, MN, cls_mask, P);
  if (rc) return rc;
  size_t scratch_off[kBatchParts + 1];
  parts_scratch(P, &scratch_off);
  if (!capturing) {
    rc = ensure(ctx, &res.d_probs, &res.probs_cap, bp.probs.size());
    if (!rc) rc = ensure(ctx, &res.d_order, &res.order_cap, bp.order.size());
    if (!rc && !res.d_counters) {
      cudaError_t e = cudaMalloc(&res.d_counters, kBatchParts * sizeof(unsigned));
      if (e != cudaSuccess) rc = cuda_fail(ctx, e, "batch counters");
    }
    if (!rc) rc = ensure(ctx, &res.d_scratch, &res.scratch_cap, scratch_off[kBatchParts]);
    if (!rc) rc = ensure(ctx, &res.d_span, &res.span_cap, 2 * (size_t)bp.n);
    if (!rc && bp.n > 0) {
      cudaError_t e = cudaMemsetAsync(res.d_span, 0, 2 * (size_t)bp.n * sizeof(long long), ctx->stream);
      if (e != cudaSuccess) rc = cuda_fail(ctx, e, "batch spans");
    }
    if (rc) return rc;
    res.n = bp.n;
    if (!bp.probs.empty()) {
      cudaError_t e = cudaMemcpyAsync(res.d_probs, bp.probs.data(), bp.probs.size() * sizeof(int4),
                                      cudaMemcpyHostToDevice, ctx->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(res.d_order, bp.order.data(), bp.order.size() * sizeof(int),
                            cudaMemcpyHostToDevice, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "batch upload");
    }
  }
  BatchTables T{};
  for (size_t i = 0; i < ctx->tab_robots.size(); ++i) T.robots[i] = ctx->tab_robots[i];
  for (size_t i = 0; i < ctx->tab_self.size() && i < (size_t)kBatchMaxRobots; ++i) T.self[i] = ctx->tab_self[i];
  if (ctx->plan_warm > 0)
    for (int r = 0; r < kBatchMaxRobots; ++r)
      for (int c = 0; c < kBatchMaxCons; ++c) T.nets[r][c] = ctx->batch_net[r * kBatchMaxCons + c];
  for (size_t i = 0; i < ctx->tab_cons.size(); ++i) T.cons[i] = ctx->tab_cons[i];
  if (!ctx->ev_fork) {
    if (cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(ctx, cudaGetLastError(), "batch events");
    for (int i = 0; i < kBatchParts; ++i)
      if (cudaStreamCreateWithFlags(&ctx->side[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ctx->ev_join[i], cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(ctx, cudaGetLastError(), "batch streams");
  }
  cudaError_t e = cudaEventRecord(ctx->ev_fork, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch fork");
  // Launch order: parts whose CTAs take a whole SM first, then by estimated work. The block
  // scheduler spreads a grid's CTAs over the SMs; CTAs that hold half an SM, placed first,
  // would leave no whole SM free for the others until they finish.
  int order[kBatchParts];
  for (int i = 0; i < kBatchParts; ++i) order[i] = i;
  std::stable_sort(order, order + kBatchParts, [&](int x, int y) {
    if (P[x].per_sm != P[y].per_sm) return P[x].per_sm < P[y].per_sm;
    return P[x].work > P[y].work;
  });
  for (int i : order) {
    const PartLaunch& L = P[i];
    if (!L.on) continue;
    const int c = L.cls;
    BatchArgs b{};
    b.a = base;
    b.a.span = res.d_span;
    b.a.stage_obs = L.stage;
    b.a.max_scene_f4 = bp.max_f4[c];
    b.problems = res.d_probs;
    b.order = res.d_order + bp.off[c] + L.first;
    b.n_class = L.n;
    b.counter = res.d_counters + i;
    b.max_S = bp.max_S[c];
    b.max_W = bp.max_W[c];
    b.out_max_W = bp.max_W_all;
    const size_t ew = (size_t)bp.max_W[c] * 8, B = (size_t)L.workers, G = (size_t)L.grid;
    char* base_p = res.d_scratch + scratch_off[i];
    b.nodes = reinterpret_cast<float*>(base_p);
    b.parent = reinterpret_cast<int*>(b.nodes + G * 2 * MN * 8);
    b.edges = reinterpret_cast<float*>(b.parent + G * 2 * MN);
    b.pend = b.edges + G * 2 * MN * ew;
    b.pend_edges = b.pend + G * B * 8;
    if ((e = cudaStreamWaitEvent(ctx->side[i], ctx->ev_fork, 0)) != cudaSuccess ||
        (e = launch_plan_batch(c, b, T, L.grid, L.smem, L.K, ctx->side[i])) != cudaSuccess ||
        (e = cudaEventRecord(ctx->ev_join[i], ctx->side[i])) != cudaSuccess ||
        (e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join[i], 0)) != cudaSuccess)
      return cuda_fail(ctx, e, "batch launch");
  }
  return CPRRTC_OK;
}

PlanArgs batch_base(cprrtc_ctx* ctx, const cprrtc_plan_params* pp, int n) {
  PlanArgs a{};
  a.n = n;
  a.range = (float)pp->range;
  a.W = 0;
  a.max_rounds = pp->max_rounds;
  a.workers = pp->workers;
  a.max_nodes = pp->max_nodes;
  a.max_connect = pp->max_connect;
  a.max_path = pp->max_path;
  a.seed = pp->seed;
  a.budget_ns = pp->time_budget_ms > 0.0 ? (unsigned long long)(pp->time_budget_ms * 1e6) : 0ull;
  a.scene_obs = ctx->d_batch_obs;
  a.scenes = ctx->d_batch_tab;
  a.work_counters = ctx->d_work;
  a.warm_refine = ctx->plan_warm;
  return a;
}

int check_batch_params(cprrtc_ctx* ctx, const cprrtc_plan_params* pp) {
  if (!pp || !(pp->range > 0) || !is_finite(pp->range) || pp->max_rounds < 1 || pp->max_nodes < 2 ||
      pp->max_connect < 0 || pp->max_path < 2 || pp->workers < 1 || pp->workers > kMaxWorkers ||
      !(pp->time_budget_ms >= 0.0) || !is_finite(pp->time_budget_ms))
    return fail(ctx, CPRRTC_E_INVALID_ARG, "batch: bad parameters");
  return CPRRTC_OK;
}

// Stages the batch's arrays (host or device) and fills base's pointers.
void stage_batch_io(Staging& st, PlanArgs& a, size_t N, int max_path, int max_W, const float* start,
                    const float* goal, int32_t* path_len, float* path, float* path_edges,
                    int32_t* rounds, int64_t* waypoints, float* plan_ms, int64_t* work) {
  st.input(start, N * 8 * sizeof(float), &a.start);
  st.input(goal, N * 8 * sizeof(float), &a.goal);
  st.output(path_len, N * sizeof(int32_t), &a.path_len);
  st.output(path, N * (size_t)max_path * 8 * sizeof(float), &a.path);
  st.output(path_edges, N * (size_t)(max_path - 1) * max_W * 8 * sizeof(float), &a.path_edges);
  st.output(rounds, N * sizeof(int32_t), &a.rounds);
  st.output(reinterpret_cast<long long*>(waypoints), N * sizeof(int64_t), &a.waypoints);
  st.output(plan_ms, N * sizeof(float), &a.plan_ms);
  st.output(reinterpret_cast<long long*>(work), N * 2 * sizeof(int64_t), &a.work);
}

}  // namespace

extern "C" {

// Drops the uneven batch's networks (their buffers are kept for reuse).
static void clear_batch_nets(cprrtc_ctx* ctx) {
  for (auto& v : ctx->batch_net) v = MlpView{};
}

int cprrtc_set_robot_table(cprrtc_ctx* ctx, const cprrtc_robot_desc* robots, int n) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!robots || n < 1) return fail(ctx, CPRRTC_E_INVALID_ARG, "robot table: empty");
  if (n > CPRRTC_BATCH_MAX_ROBOTS) return fail(ctx, CPRRTC_E_UNSUPPORTED, "robot table: too many robots");
  std::vector<RobotDev> tab(n);
  std::vector<float4> all_loc;
  std::vector<int> all_frm;
  std::vector<size_t> off(n);
  for (int i = 0; i < n; ++i) {
    std::vector<float4> loc;
    std::vector<int> frm;
    int rc = build_robot(ctx, robots[i].joints, robots[i].dof, robots[i].spheres, robots[i].n_spheres,
                         robots[i].ee, tab[i], loc, frm);
    if (rc) return rc;
    off[i] = all_loc.size();
    all_loc.insert(all_loc.end(), loc.begin(), loc.end());
    all_frm.insert(all_frm.end(), frm.begin(), frm.end());
  }
  DeviceGuard g(ctx->device);
  int rc = upload(ctx, &ctx->d_tab_sph, &ctx->tab_sph_cap, all_loc);
  if (!rc) rc = upload(ctx, &ctx->d_tab_frm, &ctx->tab_frm_cap, all_frm);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    tab[i].spheres = ctx->d_tab_sph + off[i];
    tab[i].sphere_frame = ctx->d_tab_frm + off[i];
  }
  ctx->tab_robots = tab;
  ctx->tab_self.assign(n, SelfMask{});  // frame pairs belong to the robots: set them again
  clear_batch_nets(ctx);                // so do the networks
  return CPRRTC_OK;
}

// Frame pairs of an (n_frames x n_frames) 0/1 matrix as row masks (bit b of rows[a], a < b).
static bool self_mask_of(const uint8_t* frame_pairs, int nf, SelfMask& m) {
  m = SelfMask{};
  for (int i = 0; i < nf; ++i)
    for (int j = i + 1; j < nf; ++j)
      if (frame_pairs[i * nf + j] || frame_pairs[j * nf + i]) {
        m.rows[i] |= (unsigned short)(1u << j);
        m.on = 1;
      }
  return m.on != 0;
}

int cprrtc_set_table_self_collision(cprrtc_ctx* ctx, int robot, const uint8_t* frame_pairs, int n) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (robot < 0 || robot >= (int)ctx->tab_robots.size())
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_table_self_collision: no such robot in the table");
  if (n == 0 || !frame_pairs) {
    ctx->tab_self[robot] = SelfMask{};
    return CPRRTC_OK;
  }
  const int nf = ctx->tab_robots[robot].dof + 1;
  if (n != nf * nf)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "set_table_self_collision: n must be (dof + 1)^2");
  self_mask_of(frame_pairs, nf, ctx->tab_self[robot]);
  return CPRRTC_OK;
}

int cprrtc_set_constraint_table(cprrtc_ctx* ctx, const cprrtc_constraint* cons, int n) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!cons || n < 1) return fail(ctx, CPRRTC_E_INVALID_ARG, "constraint table: empty");
  if (n > CPRRTC_BATCH_MAX_CONSTRAINTS)
    return fail(ctx, CPRRTC_E_UNSUPPORTED, "constraint table: too many constraints");
  const ConsDev saved = ctx->cs;
  std::vector<ConsDev> tab(n);
  for (int i = 0; i < n; ++i) {
    int rc = cprrtc_set_constraint(ctx, &cons[i]);  // validates and converts
    if (rc == CPRRTC_OK && cons[i].type > CPRRTC_CONSTRAINT_Z_PLANE)
      rc = fail(ctx, CPRRTC_E_UNSUPPORTED, "constraint table: the uneven batch takes NONE, ROLL_PITCH and Z_PLANE");
    if (rc) {
      ctx->cs = saved;
      return rc;
    }
    tab[i] = ctx->cs;
  }
  ctx->cs = saved;
  ctx->tab_cons = tab;
  clear_batch_nets(ctx);  // networks belong to (robot, constraint) pairs of the tables
  return CPRRTC_OK;
}

int cprrtc_batch_adopt_network(cprrtc_ctx* ctx, int robot, int constraint) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (robot < 0 || robot >= (int)ctx->tab_robots.size() || constraint < 0 ||
      constraint >= (int)ctx->tab_cons.size())
    return fail(ctx, CPRRTC_E_INVALID_ARG, "batch_adopt_network: no such robot or constraint in the tables");
  const int ct = ctx->tab_cons[constraint].type;
  if (ct != kConsRollPitch && ct != kConsZPlane)
    return fail(ctx, CPRRTC_E_UNSUPPORTED, "batch_adopt_network: the learned form plans with ROLL_PITCH or Z_PLANE");
  if (!ctx->mlp || mlp_dof(ctx->mlp) != ctx->tab_robots[robot].dof)
    return fail(ctx, CPRRTC_E_NOT_CONFIGURED,
                "batch_adopt_network: the context's network must be for the table robot's dof");
  DeviceGuard g(ctx->device);
  const MlpView src = mlp_view(ctx->mlp);
  // one buffer: layer 0..2 transposes (BF16 [16][256], [256][256] x 2), layer 3 (BF16 [16][256]),
  // biases (FP32 3 x 256 + 16)
  const size_t b0 = 16 * 256 * 2, b1 = 256 * 256 * 2, b3 = 16 * 256 * 2, bb = (3 * 256 + 16) * 4;
  const size_t total = b0 + 2 * b1 + b3 + bb;
  const int slot = robot * kBatchMaxCons + constraint;
  char* buf = static_cast<char*>(ctx->batch_net_buf[slot]);
  cudaError_t e = cudaSuccess;
  if (!buf) {
    e = cudaMalloc(reinterpret_cast<void**>(&buf), total);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch_adopt_network: allocation");
    ctx->batch_net_buf[slot] = buf;
  }
  MlpView v{};
  v.wt[0] = buf;
  v.wt[1] = buf + b0;
  v.wt[2] = buf + b0 + b1;
  v.w3 = buf + b0 + 2 * b1;
  float* bias = reinterpret_cast<float*>(buf + b0 + 2 * b1 + b3);
  v.b[0] = bias;
  v.b[1] = bias + 256;
  v.b[2] = bias + 512;
  v.b[3] = bias + 768;
  v.dof = src.dof;
  const void* from[4] = {src.wt[0], src.wt[1], src.wt[2], src.w3};
  const void* to[4] = {v.wt[0], v.wt[1], v.wt[2], v.w3};
  const size_t bytes[4] = {b0, b1, b1, b3};
  for (int i = 0; i < 4 && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(const_cast<void*>(to[i]), from[i], bytes[i], cudaMemcpyDeviceToDevice, ctx->stream);
  for (int l = 0; l < 4 && e == cudaSuccess; ++l)
    e = cudaMemcpyAsync(const_cast<float*>(v.b[l]), src.b[l], (l < 3 ? 256 : src.dof) * sizeof(float),
                        cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch_adopt_network: copy");
  ctx->batch_net[slot] = v;
  return CPRRTC_OK;
}

int cprrtc_plan_batch(cprrtc_ctx* ctx, const cprrtc_problem* problems, int n, const float* start,
                      const float* goal, const cprrtc_plan_params* pp, const cprrtc_tuning* tuning,
                      int32_t* path_len, float* path, float* path_edges, int32_t* rounds,
                      int64_t* waypoints, float* plan_ms, int64_t* work) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  int rc = check_batch_params(ctx, pp);
  if (rc) return rc;
  if (n == 0) return CPRRTC_OK;
  if (!start || !goal || !path_len || !path) return fail(ctx, CPRRTC_E_INVALID_ARG, "batch: null pointer");
  DeviceGuard g(ctx->device);
  BatchPlan bp;
  rc = prepare_batch(ctx, problems, n, bp);
  if (rc) return rc;
  PlanArgs a = batch_base(ctx, pp, n);
  Staging st;
  stage_batch_io(st, a, (size_t)n, pp->max_path, bp.max_W_all, start, goal, path_len, path,
                 path_edges, rounds, waypoints, plan_ms, work);
  rc = st.begin(ctx);
  if (rc) return rc;
  const cprrtc_tuning t = tuning ? *tuning : (ctx->has_tuned ? ctx->tuned : default_tuning());
  LaunchTimer tm(ctx, "plan_batch");
  rc = run_batch(ctx, bp, ctx->batch_res, a, t, (1u << kBatchClasses) - 1u, false);
  tm.done();
  if (rc) return rc;
  ctx->last_batch = &ctx->batch_res;
  return st.end(ctx);
}

int cprrtc_autotune_batch(cprrtc_ctx* ctx, const cprrtc_problem* problems, int n, const float* start,
                          const float* goal, const cprrtc_plan_params* pp, int trial_rounds,
                          cprrtc_tuning* out) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  int rc = check_batch_params(ctx, pp);
  if (rc) return rc;
  if (trial_rounds < 1) return fail(ctx, CPRRTC_E_INVALID_ARG, "autotune: trial_rounds < 1");
  if (n < 1 || !start || !goal) return fail(ctx, CPRRTC_E_INVALID_ARG, "autotune: no problems");
  DeviceGuard g(ctx->device);
  BatchPlan bp;
  rc = prepare_batch(ctx, problems, n, bp);
  if (rc) return rc;
  cprrtc_plan_params trial = *pp;
  trial.max_rounds = trial_rounds;
  PlanArgs a = batch_base(ctx, &trial, n);
  a.work_counters = nullptr;
  // device outputs of the trials (the tuner allocates; plan calls do not need to)
  const size_t N = (size_t)n;
  float *d_path = nullptr, *d_ms = nullptr;
  int32_t *d_len = nullptr, *d_rounds = nullptr;
  long long* d_wp = nullptr;
  cudaError_t e = cudaMalloc(&d_path, N * trial.max_path * 8 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_len, N * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&d_rounds, N * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&d_wp, N * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&d_ms, N * sizeof(float));
  auto release = [&]() {
    cudaFree(d_path);
    cudaFree(d_len);
    cudaFree(d_rounds);
    cudaFree(d_wp);
    cudaFree(d_ms);
  };
  if (e != cudaSuccess) {
    release();
    return cuda_fail(ctx, e, "autotune allocation");
  }
  a.path = d_path;
  a.path_len = d_len;
  a.rounds = d_rounds;
  a.waypoints = d_wp;
  a.plan_ms = d_ms;
  Staging st;
  st.input(start, N * 8 * sizeof(float), &a.start);
  st.input(goal, N * 8 * sizeof(float), &a.goal);
  rc = st.begin(ctx);
  if (rc) {
    release();
    return rc;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cprrtc_tuning best = ctx->has_tuned ? ctx->tuned : default_tuning();
  std::vector<long long> wp(N);
  for (int c = 0; c < kBatchClasses && !rc; ++c) {
    if (bp.off[c + 1] == bp.off[c]) continue;
    double best_rate = -1.0;
    const int nc = bp.off[c + 1] - bp.off[c];
    // shapes: one warp per worker with none, 4 or 16 of the class's heaviest problems on warp
    // pairs, or the whole class on warp pairs (pairs = -1); obstacles staged or through L1;
    // CTAs per SM of the one-warp part
    const int pair_shapes[] = {0, 4, 16, -1};
    for (int si = 0; si < 4 * 2 && !rc; ++si) {
      const int pairs = pair_shapes[si / 2], stage = 1 - si % 2;
      if (pairs != 0 && !pairs_allowed(ctx, pp->workers)) continue;
      if (pairs > 0 && pairs >= nc) continue;  // the whole class: the pairs = -1 shape
      cprrtc_tuning t = best;
      t.warps_per_motion[c] = pairs < 0 ? 2 : 1;
      t.pair_problems[c] = pairs < 0 ? 0 : pairs;
      t.stage_obstacles[c] = stage;
      t.ctas_per_sm[c] = 0;
      PartLaunch P[kBatchParts];
      if (batch_parts(ctx, bp, t, pp->workers, (size_t)pp->max_nodes, 1u << c, P)) continue;  // does not fit
      const PartLaunch &P0 = P[2 * c], &P1 = P[2 * c + 1];
      if ((P0.n && P0.stage != stage) || (P1.n && P1.stage != stage)) continue;  // staging did not fit: tried as L1
      const int max_ctas = P1.n ? std::min(P1.per_sm, 4) : 1;
      for (int ctas = 1; ctas <= max_ctas && !rc; ++ctas) {
        t.ctas_per_sm[c] = P1.n ? ctas : 0;
        cudaEventRecord(e0, ctx->stream);
        rc = run_batch(ctx, bp, ctx->batch_res, a, t, 1u << c, false);
        if (rc) break;
        ctx->last_batch = &ctx->batch_res;
        cudaEventRecord(e1, ctx->stream);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
          rc = cuda_fail(ctx, e, "autotune trial");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaMemcpy(wp.data(), d_wp, N * sizeof(long long), cudaMemcpyDeviceToHost);
        double total = 0.0;
        for (int i = bp.off[c]; i < bp.off[c + 1]; ++i) total += (double)wp[bp.order[i]];
        const double rate = ms > 0.f ? total / ms : 0.0;
        if (rate > best_rate) {
          best_rate = rate;
          best.stage_obstacles[c] = stage;
          best.ctas_per_sm[c] = t.ctas_per_sm[c];
          best.warps_per_motion[c] = t.warps_per_motion[c];
          best.pair_problems[c] = t.pair_problems[c];
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release();
  if (rc) return rc;
  ctx->tuned = best;
  ctx->has_tuned = true;
  if (out) *out = best;
  return CPRRTC_OK;
}

int cprrtc_batch_capture(cprrtc_ctx* ctx, const cprrtc_problem* problems, int n, const float* start,
                         const float* goal, const cprrtc_plan_params* pp, const cprrtc_tuning* tuning,
                         int32_t* path_len, float* path, float* path_edges, int32_t* rounds,
                         int64_t* waypoints, float* plan_ms, int64_t* work) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  int rc = check_batch_params(ctx, pp);
  if (rc) return rc;
  if (n < 1 || !start || !goal || !path_len || !path)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "batch capture: null pointer or no problems");
  DeviceGuard g(ctx->device);
  const void* arrays[] = {start, goal, path_len, path, path_edges, rounds, waypoints, plan_ms, work};
  for (const void* ptr : arrays)
    if (ptr && ptr_where(ptr, ctx->device) != kPtrHere)
      return fail(ctx, CPRRTC_E_INVALID_ARG,
                  "batch capture: every array must be device memory of the context's GPU");
  BatchPlan bp;
  rc = prepare_batch(ctx, problems, n, bp);
  if (rc) return rc;
  PlanArgs a = batch_base(ctx, pp, n);
  Staging st;  // device pointers only: no copies
  stage_batch_io(st, a, (size_t)n, pp->max_path, bp.max_W_all, start, goal, path_len, path,
                 path_edges, rounds, waypoints, plan_ms, work);
  const cprrtc_tuning t = tuning ? *tuning : (ctx->has_tuned ? ctx->tuned : default_tuning());
  // buffers and attributes first (no allocation while capturing), then record the launches
  if (ctx->graph_exec) {
    cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
  }
  rc = run_batch(ctx, bp, ctx->graph_res, a, t, 0u, false);  // uploads, no launch
  if (rc) return rc;
  BatchRes& res = ctx->graph_res;
  {
    // scratch for every part (run_batch with an empty mask sized nothing)
    PartLaunch P[kBatchParts];
    rc = batch_parts(ctx, bp, t, pp->workers, (size_t)pp->max_nodes, (1u << kBatchClasses) - 1u, P);
    if (!rc) rc = ensure(ctx, &res.d_scratch, &res.scratch_cap, parts_scratch(P));
    if (rc) return rc;
  }
  if (!ctx->stream) return fail(ctx, CPRRTC_E_INVALID_ARG, "batch capture: needs a non-default stream");
  cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch capture begin");
  rc = run_batch(ctx, bp, res, a, t, (1u << kBatchClasses) - 1u, true);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(ctx->stream, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch capture end");
  e = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch graph instantiate");
  return CPRRTC_OK;
}

int cprrtc_batch_replay(cprrtc_ctx* ctx) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  if (!ctx->graph_exec) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "batch replay: nothing captured");
  DeviceGuard g(ctx->device);
  LaunchTimer tm(ctx, "plan_batch");
  cudaError_t e = cudaGraphLaunch(ctx->graph_exec, ctx->stream);
  tm.done();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch replay");
  ctx->last_batch = &ctx->graph_res;
  return CPRRTC_OK;
}

int cprrtc_batch_spans(cprrtc_ctx* ctx, int64_t* span, int n) {
  if (!ctx) return CPRRTC_E_INVALID_ARG;
  const BatchRes* r = ctx->last_batch;
  if (!r || !r->d_span) return fail(ctx, CPRRTC_E_NOT_CONFIGURED, "batch spans: no batch has run");
  if (!span || n != r->n) return fail(ctx, CPRRTC_E_INVALID_ARG, "batch spans: n must be the last batch's problem count");
  if (ptr_where(span, ctx->device) != kPtrHost)
    return fail(ctx, CPRRTC_E_INVALID_ARG, "batch spans: span must be host memory");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaMemcpyAsync(span, r->d_span, 2 * (size_t)n * sizeof(long long), cudaMemcpyDeviceToHost,
                                  ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch spans");
  return CPRRTC_OK;
}

}  // extern "C"
