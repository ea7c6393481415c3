// Collision checking of sphere obstacles in GEMM form on the 5th-generation tensor cores,
// with an exact FP32 recheck of every pair the contraction cannot clear.
//
// For a robot sphere (centre c, radius r) and an obstacle sphere (centre p, radius rho),
// with a = c - o and b = p - o about a fixed origin o and radii inflated by a guard
// (r' = r + g/2, rho' = rho + g/2):
//   s = |a - b|^2 - (r' + rho')^2 = -2 a.b + (|a|^2 - r'^2) - 2 r' rho' + (|b|^2 - rho'^2),
// a dot product of A' (one row per robot sphere) and B' (one row per obstacle) over K = 16
// columns. Every FP32 value is split into hi + lo in the MMA precision (BF16 or TF32), and
// each coordinate product is kept to hi*hi + hi*lo + lo*hi:
//   A' = [(-2a_k)hi, (-2a_k)hi, (-2a_k)lo]_k=0..2, alpha_hi, alpha_lo, -2r', 1, 1, 0, 0
//   B' = [ b_k hi,    b_k lo,    b_k hi  ]_k=0..2, 1,        1,        rho', beta_hi, beta_lo, 0, 0
// with alpha = |a|^2 - r'^2 - E and beta = |b|^2 - rho'^2. The host derives a bound E on
// |s_tensor - s| from the unit roundoff of the precision and the coordinate ranges; folding
// -E into alpha makes the contraction s - E. A pair with s_tensor - E >= 0 has s >= 0, i.e.
// clearance >= g > 0: no collision, and no FP32 rounding can turn it into one. An epilogue
// warp reads its block of accumulator columns with tensor-memory loads that also return the
// minimum of what they load: a positive minimum clears all its pairs; otherwise (rarely) the
// row is rechecked against the block's obstacles with the same FP32 test as the exact
// collision kernel, on sphere centres computed by the same FK arithmetic, so the verdicts,
// and each motion's first colliding waypoint, are those of the exact kernel.
//
// One persistent CTA per SM takes motions from a global counter (the FK group fetches them,
// skipping motions that did not project, into a small ring every role reads in the same
// order) and their waypoints in order.
// A waypoint is one M = 128 tile (robot spheres, padding rows never collide); the obstacles
// are N tiles of 256, and every N tile is one (BF16) or two (TF32) tcgen05.mma into an FP32
// accumulator in tensor memory (two accumulators, so the epilogue of one tile overlaps the
// MMA of the next). The obstacle matrix B' is a pre-swizzled image of 32 KB chunks; each
// 128-byte row of a chunk carries the K slices of 4 (BF16) or 2 (TF32) N tiles, and a tile is
// addressed by its byte offset inside the row, the same K stepping the MMA uses. Up to four
// chunks stay resident in shared memory (4096 obstacles in BF16); larger images stream
// through a four-stage ring filled by bulk (TMA) copies.
//
// Warp roles (kCcThreads threads):
//   warps 0-3   FK: the chain of the waypoint (one thread, Frame::advance from the base),
//               then one thread per robot sphere: FP32 centre (Frame::world), the A' row in
//               the operand layout, and the centre kept for the recheck.
//   kEpiWarpsCc epilogue warps from warp 4: warp w reads accumulator lanes 32 (w % 4) .. + 31
//               and column block (w - 4) / 4 (kEpiCols columns) of each N tile in pairs of
//               32-column loads, releases the accumulator, takes the loads' minima, and in
//               the rare case of a minimum <= 0 rechecks the block's pairs exactly.
//   then        the producer of B' chunks, and a warp that allocates tensor memory and
//               issues the MMAs.
// Early termination: after each waypoint the epilogue publishes a verdict. Waypoint w of a
// motion is issued only while waypoint w - 2 was collision-free, so after the first
// colliding waypoint h exactly one more (h + 1, if it exists) is in flight and is drained.
// Every wait is bounded in time; on expiry the CTA raises a flag, drains what it issued,
// frees tensor memory and exits.
#include <cuda_bf16.h>
#include <stdint.h>

#include "collide.cuh"
#include "launch.h"
#include "motion.cuh"

namespace cprrtc {

namespace {

#ifndef CPRRTC_CC_EPI_WARPS
#define CPRRTC_CC_EPI_WARPS 16
#endif
constexpr int kFkWarps = 4;
// epilogue warps: 4 lane quarters x (kEpiWarpsCc / 4) column blocks of kEpiCols columns
constexpr int kEpiFirst = 4, kEpiWarpsCc = CPRRTC_CC_EPI_WARPS;
constexpr int kEpiCols = 256 / (kEpiWarpsCc / 4);
constexpr int kProdWarp = kEpiFirst + kEpiWarpsCc, kMmaWarpCc = kProdWarp + 1;
constexpr int kCcThreads = 32 * (kMmaWarpCc + 1);
static_assert(kEpiWarpsCc % 4 == 0 && kEpiCols % 64 == 0, "epilogue loads go in pairs of 32 columns");
constexpr int kCcStages = 4;
constexpr int kChunkBytes = 32768;
constexpr int kATile = 128 * 128;  // one waypoint's A' (SW128, 128 rows x 128 B)

constexpr int kOffRingCc = 0;
constexpr int kOffA = kOffRingCc + kCcStages * kChunkBytes;
constexpr int kOffCentre = kOffA + 2 * kATile;       // float4 [2][128]
constexpr int kOffFrames = kOffCentre + 2 * 128 * 16;  // float [2][9][12]
constexpr int kOffBarCc = kOffFrames + 2 * 9 * 12 * 4 + 16;  // + a control word
// barriers: b_full[4] b_empty[4] a_full[2] acc_full[2] acc_empty[2] verdict[2]
constexpr int kBFull = 0, kBEmpty = 4, kAFull = 8, kAccF = 10, kAccE = 12, kVerdict = 14;
constexpr int kNumBarsCc = 16;
constexpr int kOffHit = kOffBarCc + kNumBarsCc * 8;  // int [2]
constexpr int kOffTmemCc = kOffHit + 8;
constexpr int kOffAbortCc = kOffTmemCc + 4;
constexpr int kOffRechk = kOffAbortCc + 4;  // unsigned long long
constexpr int kOffRing8 = kOffRechk + 8;    // int [8] motion ring, int fetched, int done
constexpr int kRingM = 8;
// Work items are runs of kWpRun waypoints of one motion, handed out run-major (every
// motion's first run, then every second run, ...), so the long collision-free motions
// spread over the SMs instead of ending the launch on a few of them.
constexpr int kWpRun = 16;
constexpr int kSmemCc = kOffRing8 + (kRingM + 2) * 4;
constexpr uint64_t kWaitNs = 1000000000ull;  // default limit of a bounded wait: 1 s
constexpr uint64_t kDrainNs = 20000000ull;
// this launch's limit of a bounded wait (set by thread 0 before the first barrier)
__shared__ uint64_t s_wait_ns;
static_assert(kOffBarCc % 8 == 0 && kOffRechk % 8 == 0, "alignment");

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mb_init(uint32_t b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(n) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint32_t b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}
__device__ __forceinline__ void mb_expect(uint32_t b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mb_try(uint32_t b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(b), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait; false when another role aborted or the limit expired (then raises the flag).
__device__ bool mb_wait(uint32_t b, uint32_t parity, volatile int* abort_flag) {
  if (mb_try(b, parity)) return true;
  const uint64_t t0 = gtime();
  for (;;) {
    for (int i = 0; i < 32; ++i)
      if (mb_try(b, parity)) return true;
    if (*abort_flag) return false;
    if (gtime() - t0 > s_wait_ns) {
      *abort_flag = 1;
      return false;
    }
  }
}
__device__ void mb_drain(uint32_t b, uint32_t parity) {
  const uint64_t t0 = gtime();
  while (!mb_try(b, parity) && gtime() - t0 < kDrainNs) {
  }
}
__device__ __forceinline__ void fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tcb() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tca() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ uint32_t sw128b(int r, int kbyte) {  // byte kbyte (< 128) of row r, 128-row... any rows
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((kbyte >> 4) & 7) ^ (r & 7)) << 4) + (kbyte & 15));
}
__device__ __forceinline__ uint64_t sdesc(uint32_t a) {
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}
// kind::f16 (BF16, format 1) or kind::tf32 (format 2), FP32 accumulator, K-major, M=128, N=256
template <int TF32>
__device__ __forceinline__ void mma_cc(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  constexpr uint32_t fmt = TF32 ? 2u : 1u;
  constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  if (TF32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void commit_to(uint32_t b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b) : "memory");
}
// Loads 32 accumulator columns of this thread's lane and returns their minimum (the load's
// own min reduction); the loaded values themselves are not needed. Valid after tld_wait.
__device__ __forceinline__ float tld32_min(uint32_t taddr) {
  float r[32], m;
  asm volatile(
      "tcgen05.ld.red.sync.aligned.32x32b.x32.min.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, %32, [%33];"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]),
        "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15]), "=f"(r[16]),
        "=f"(r[17]), "=f"(r[18]), "=f"(r[19]), "=f"(r[20]), "=f"(r[21]), "=f"(r[22]), "=f"(r[23]), "=f"(r[24]),
        "=f"(r[25]), "=f"(r[26]), "=f"(r[27]), "=f"(r[28]), "=f"(r[29]), "=f"(r[30]), "=f"(r[31]), "=f"(m)
      : "r"(taddr)
      : "memory");
  return m;
}
__device__ __forceinline__ void tld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Round-to-nearest-even to the MMA precision (BF16: 8 significant bits, TF32: 11).
template <int TF32>
__device__ __forceinline__ float round_prec(float x) {
  if (TF32) {
    uint32_t u = __float_as_uint(x);
    u = (u + 0xFFFu + ((u >> 13) & 1u)) & ~0x1FFFu;
    return __uint_as_float(u);
  }
  return __bfloat162float(__float2bfloat16(x));
}
template <int TF32>
__device__ __forceinline__ void put(uint8_t* tile, int row, int col, float v) {
  if (TF32)
    *reinterpret_cast<float*>(tile + sw128b(row, 4 * col)) = v;
  else
    *reinterpret_cast<__nv_bfloat16*>(tile + sw128b(row, 2 * col)) = __float2bfloat16(v);
}

template <int TF32>
// 80 registers (the compiler's choice, with a small spill): an SM splits its registers between
// four sub-partitions of 16,384 each, and the 22 warps of a CTA put six warps on two of them,
// so 6 x 32 x R <= 16,384 bounds R at 85, i.e. 80 in 8-register steps (88 fails to launch).
__global__ void __launch_bounds__(kCcThreads, 1) gemm_cc_kernel(RobotDev rb, GemmCcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sb = saddr(sm);
  auto bar = [&](int i) { return sb + kOffBarCc + 8u * (uint32_t)i; };
  volatile int* s_abort = reinterpret_cast<volatile int*>(sm + kOffAbortCc);
  volatile int* s_hit = reinterpret_cast<volatile int*>(sm + kOffHit);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + kOffTmemCc);
  unsigned long long* s_rechk = reinterpret_cast<unsigned long long*>(sm + kOffRechk);
  float4* s_centre = reinterpret_cast<float4*>(sm + kOffCentre);
  float* s_frames = reinterpret_cast<float*>(sm + kOffFrames);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kTilesPerRow = TF32 ? 2 : 4;     // N tiles sharing one 128-byte row
  constexpr int kSliceBytes = TF32 ? 64 : 32;   // K = 16 values
  constexpr int kMmasPerTile = TF32 ? 2 : 1;    // K = 8 (TF32) or 16 (BF16) per instruction
  const int n_tiles = a.n_tiles;
  const int n_chunks = (n_tiles + kTilesPerRow - 1) / kTilesPerRow;
  const bool resident = n_chunks <= kCcStages;
  const int W = a.W, dof = rb.dof;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kCcStages; ++s) {
      mb_init(bar(kBFull + s), 1);
      mb_init(bar(kBEmpty + s), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mb_init(bar(kAFull + i), kFkWarps * 32);
      mb_init(bar(kAccF + i), 1);
      mb_init(bar(kAccE + i), kEpiWarpsCc);
      mb_init(bar(kVerdict + i), kEpiWarpsCc);
      s_hit[i] = 0;
    }
    *s_abort = 0;
    s_wait_ns = a.wait_ns ? a.wait_ns : kWaitNs;
    *s_rechk = 0ull;
    *reinterpret_cast<volatile int*>(sm + kOffRing8 + kRingM * 4) = 0;
    *reinterpret_cast<volatile int*>(sm + kOffRing8 + kRingM * 4 + 4) = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarpCc) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(saddr(s_tmem)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tcb();
  __syncthreads();
  tca();
  const uint32_t tmem = *s_tmem;

  int* s_mring = reinterpret_cast<int*>(sm + kOffRing8);
  volatile int* s_fetched = reinterpret_cast<volatile int*>(sm + kOffRing8 + kRingM * 4);
  volatile int* s_done = s_fetched + 1;
  // bounded wait on a shared counter written by another role
  auto wait_count = [&](volatile int* cnt, int need) -> bool {  // until *cnt >= need
    const uint64_t t0 = gtime();
    while (*cnt < need) {
      if (*s_abort) return false;
      if (gtime() - t0 > s_wait_ns) {
        *s_abort = 1;
        return false;
      }
      __nanosleep(64);
    }
    return true;
  };
  // the k-th work item of this CTA (-1: none left; -2: aborted): motion item % n, waypoints
  // [w0, w1) with w0 = (item / n) * kWpRun
  auto motion = [&](int k) -> int {
    if (!wait_count(s_fetched, k + 1)) return -2;
    return *reinterpret_cast<volatile int*>(&s_mring[k % kRingM]);
  };
  const int n_runs = (W + kWpRun - 1) / kWpRun;
  auto run_of = [&](int item, int& m, int& w0, int& w1) {
    const int j = item / a.n;
    m = item - j * a.n;
    w0 = j * kWpRun;
    w1 = min(W, w0 + kWpRun);
  };
  // verdict of global waypoint g: the epilogue stores g + 1 into s_hit[g % 2] when it collided
  auto verdict_hit = [&](uint32_t g) { return s_hit[g & 1] == (int)(g + 1); };
  // per item: issue(w) = w < w1 and (w - w0 < 2 or the item is still active after
  // verdict(w - 2))

  if (warp == kProdWarp) {
    if (lane == 0) {
      bool ok = true;
      if (resident) {
        for (int c = 0; c < n_chunks; ++c) {
          mb_expect(bar(kBFull + c), kChunkBytes);
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                           sb + kOffRingCc + c * kChunkBytes),
                       "l"(a.bimage + (size_t)c * kChunkBytes), "r"(kChunkBytes), "r"(bar(kBFull + c))
                       : "memory");
        }
        for (int c = 0; c < n_chunks; ++c) mb_drain(bar(kBFull + c), 0);
      } else {
        uint32_t fill = 0, g = 0;
        for (int k = 0; ok; ++k) {
          const int item = motion(k);
          if (item == -2) ok = false;
          if (item < 0) break;
          int m, w0, w1;
          run_of(item, m, w0, w1);
          bool active = true;
          for (int w = w0; ok && w < w1; ++w, ++g) {
            if (g >= 2) {
              if (!mb_wait(bar(kVerdict + (g & 1)), ((g - 2) >> 1) & 1, s_abort)) { ok = false; break; }
              if (w - w0 >= 2 && verdict_hit(g - 2)) active = false;
            }
            if (!active) break;
            for (int c = 0; c < n_chunks; ++c, ++fill) {
              const int s = fill % kCcStages;
              if (fill >= (uint32_t)kCcStages &&
                  !mb_wait(bar(kBEmpty + s), ((fill / kCcStages) - 1) & 1, s_abort)) {
                ok = false;
                break;
              }
              mb_expect(bar(kBFull + s), kChunkBytes);
              asm volatile(
                  "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                      sb + kOffRingCc + s * kChunkBytes),
                  "l"(a.bimage + (size_t)c * kChunkBytes), "r"(kChunkBytes), "r"(bar(kBFull + s))
                  : "memory");
            }
          }
        }
        for (uint32_t f = fill > (uint32_t)kCcStages ? fill - kCcStages : 0; f < fill; ++f)
          mb_drain(bar(kBFull + f % kCcStages), (f / kCcStages) & 1);
      }
    }
  } else if (warp == kMmaWarpCc) {
    if (lane == 0) {
      bool ok = true, loaded = false;
      uint32_t g = 0, tcount = 0, use = 0;
      for (int k = 0; ok; ++k) {
        const int item = motion(k);
        if (item == -2) ok = false;
        if (item < 0) break;
        int m, w0, w1;
        run_of(item, m, w0, w1);
        bool active = true;
        for (int w = w0; ok && w < w1; ++w, ++g) {
          if (g >= 2) {
            if (!mb_wait(bar(kVerdict + (g & 1)), ((g - 2) >> 1) & 1, s_abort)) { ok = false; break; }
            if (w - w0 >= 2 && verdict_hit(g - 2)) active = false;
          }
          if (!active) break;
          if (!mb_wait(bar(kAFull + (g & 1)), (g >> 1) & 1, s_abort)) { ok = false; break; }
          if (resident && !loaded) {
            for (int c = 0; c < n_chunks && ok; ++c) ok = mb_wait(bar(kBFull + c), 0, s_abort);
            loaded = true;
            if (!ok) break;
          }
          tca();
          const uint32_t a_addr = sb + kOffA + (g & 1) * kATile;
          for (int t = 0; t < n_tiles; ++t, ++tcount) {
            const int c = t / kTilesPerRow;
            uint32_t stage_addr;
            if (resident) {
              stage_addr = sb + kOffRingCc + c * kChunkBytes;
            } else {
              if (t % kTilesPerRow == 0) {
                const int s = use % kCcStages;
                if (!mb_wait(bar(kBFull + s), (use / kCcStages) & 1, s_abort)) { ok = false; break; }
                tca();
              }
              stage_addr = sb + kOffRingCc + (use % kCcStages) * kChunkBytes;
            }
            const uint32_t slot = tcount & 1;
            if (tcount >= 2 && !mb_wait(bar(kAccE + slot), ((tcount >> 1) - 1) & 1, s_abort)) { ok = false; break; }
            tca();
            const uint32_t b_addr = stage_addr + (t % kTilesPerRow) * kSliceBytes;
#pragma unroll
            for (int kk = 0; kk < kMmasPerTile; ++kk)
              mma_cc<TF32>(tmem + slot * 256, sdesc(a_addr + kk * 32), sdesc(b_addr + kk * 32), kk > 0 ? 1u : 0u);
            commit_to(bar(kAccF + slot));
            if (!resident && (t % kTilesPerRow == kTilesPerRow - 1 || t == n_tiles - 1)) {
              commit_to(bar(kBEmpty + use % kCcStages));
              ++use;
            }
          }
        }
      }
      if (tcount > 0) mb_drain(bar(kAccF + ((tcount - 1) & 1)), ((tcount - 1) >> 1) & 1);
    }
  } else if (warp < kFkWarps) {
    // FK warps: one thread per A' row; thread 0 takes the waits and decisions and shares them
    // (with the frames) through shared memory, so the group stays in step
    const int row = threadIdx.x;
    const float4 ori = a.origin;  // {ox, oy, oz, guard / 2}
    volatile int* s_ctl = reinterpret_cast<volatile int*>(s_frames + 2 * 9 * 12);  // control word
    uint32_t g = 0;
    bool ok = true;
    for (int k = 0; ok; ++k) {
      if (threadIdx.x == 0) {  // fetch the next work item of a projected motion into the ring
        int m = -1;
        if (wait_count(s_done, k - kRingM + 1)) {  // slot k % 8 no longer read
          // skip motions that did not project, and runs after a collision already found
          // (run-major order: the earlier runs of a motion were handed out before)
          for (;;) {
            const int item = atomicAdd(a.next, 1);
            if (item >= a.n * n_runs) break;
            int mm, w0, w1;
            run_of(item, mm, w0, w1);
            const int st = *reinterpret_cast<volatile const uint8_t*>(&a.status[mm]);
            const unsigned ff = (unsigned)*reinterpret_cast<volatile const int*>(&a.first_fail[mm]);
            if ((st == kValid || st == kCollision) && ff >= (unsigned)w0) {
              m = item;
              break;
            }
          }
        } else {
          m = -2;
        }
        *reinterpret_cast<volatile int*>(&s_mring[k % kRingM]) = m;
        __threadfence_block();
        *s_fetched = k + 1;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(kFkWarps * 32) : "memory");
      const int item = *reinterpret_cast<volatile int*>(&s_mring[k % kRingM]);
      if (item == -2) ok = false;
      if (item < 0) break;
      int m, w0, w1;
      run_of(item, m, w0, w1);
      bool active = true;
      for (int w = w0; ok && w < w1; ++w, ++g) {
        const int buf = g & 1;
        float* fr = s_frames + buf * 9 * 12;
        if (threadIdx.x == 0) {
          int ctl = 1;
          if (g >= 2) {  // buffer g % 2 is free once waypoint g - 2 has its verdict
            if (!mb_wait(bar(kVerdict + (g & 1)), ((g - 2) >> 1) & 1, s_abort)) ctl = -1;
            else if (w - w0 >= 2 && verdict_hit(g - 2)) ctl = 0;
          }
          if (ctl == 1) {  // the chain, with the exact kernel's arithmetic
            const float* q = a.q + ((size_t)m * W + w) * dof;
            Frame F;
            F.identity();
            for (int f = 0; f <= dof; ++f) {
              if (f > 0) F.advance(rb.j[f - 1], q[f - 1]);
              float* o = fr + f * 12;
              o[0] = F.x0; o[1] = F.x1; o[2] = F.x2; o[3] = F.y0; o[4] = F.y1; o[5] = F.y2;
              o[6] = F.z0; o[7] = F.z1; o[8] = F.z2; o[9] = F.p0; o[10] = F.p1; o[11] = F.p2;
            }
          }
          *s_ctl = ctl;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kFkWarps * 32) : "memory");
        const int ctl = *s_ctl;
        // every thread has read the decision before thread 0 may overwrite it
        asm volatile("bar.sync 1, %0;" ::"r"(kFkWarps * 32) : "memory");
        if (ctl < 0) { ok = false; break; }
        if (ctl == 0) { active = false; break; }
        uint8_t* tile = sm + kOffA + buf * kATile;
        float v[16];
        if (row < rb.n_spheres) {
          const float4 l = rb.spheres[row];
          const float* o = fr + rb.sphere_frame[row] * 12;
          Frame F;
          F.x0 = o[0]; F.x1 = o[1]; F.x2 = o[2]; F.y0 = o[3]; F.y1 = o[4]; F.y2 = o[5];
          F.z0 = o[6]; F.z1 = o[7]; F.z2 = o[8]; F.p0 = o[9]; F.p1 = o[10]; F.p2 = o[11];
          float cx, cy, cz;
          F.world(l.x, l.y, l.z, cx, cy, cz);
          s_centre[buf * 128 + row] = make_float4(cx, cy, cz, l.w);
          const float ax = cx - ori.x, ay = cy - ori.y, az = cz - ori.z;
          const float rp = l.w + ori.w;
          // alpha less the bound: a candidate pair is then simply s - E <= 0
          const float al = fmaf(ax, ax, fmaf(ay, ay, fmaf(az, az, -rp * rp))) - a.bound;
          const float m2[3] = {-2.f * ax, -2.f * ay, -2.f * az};
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float hi = round_prec<TF32>(m2[k]);
            v[3 * k] = hi;
            v[3 * k + 1] = hi;
            v[3 * k + 2] = m2[k] - hi;
          }
          const float ah = round_prec<TF32>(al);
          v[9] = ah;
          v[10] = al - ah;
          v[11] = -2.f * rp;
          v[12] = 1.f;
          v[13] = 1.f;
        } else {  // padding row: s = 1e4
#pragma unroll
          for (int k = 0; k < 14; ++k) v[k] = 0.f;
          v[9] = 1e4f;
          s_centre[buf * 128 + row] = make_float4(0.f, 0.f, 0.f, -1.f);
        }
        v[14] = 0.f;
        v[15] = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) put<TF32>(tile, row, k, v[k]);
        fence_async();
        mb_arrive(bar(kAFull + buf));
      }
    }
  } else if (warp >= kEpiFirst && warp < kEpiFirst + kEpiWarpsCc) {
    const int e = warp - kEpiFirst;
    const int lq = warp & 3, qc = e >> 2;  // lane quarter, column block of each tile
    const int row = lq * 32 + lane;
    bool ok = true;
    uint32_t g = 0, tcount = 0;
    unsigned rechecks = 0;
    for (int k = 0; ok; ++k) {
      const int item = motion(k);
      if (item == -2) ok = false;
      if (item < 0) break;
      int m, w0, w1;
      run_of(item, m, w0, w1);
      int first_hit = -1;
      for (int w = w0; ok && w < w1; ++w, ++g) {
        const int buf = g & 1;
        const bool drain = first_hit >= 0;  // the one waypoint issued after the first hit
        // the FK warps' centres for this waypoint (a_full cannot move on before this verdict)
        if (!__all_sync(0xffffffffu, mb_wait(bar(kAFull + buf), (g >> 1) & 1, s_abort))) { ok = false; break; }
        // the FK warps' centre of this row is read only when a recheck needs it
        const float4* cen_p = s_centre + buf * 128 + row;
        bool hit = false;
        // per N tile: this warp's columns, two loads at a time; the accumulator is released
        // as soon as they land, so the next tile's MMA overlaps the tests
        for (int t = 0; ok && t < n_tiles; ++t) {
          const uint32_t tc = tcount + (uint32_t)t, slot = tc & 1;
          if (!__all_sync(0xffffffffu, mb_wait(bar(kAccF + slot), (tc >> 1) & 1, s_abort))) {
            ok = false;
            break;
          }
          tca();
          const uint32_t base = tmem + ((uint32_t)(lq * 32) << 16) + slot * 256 + (uint32_t)qc * kEpiCols;
          float mn = INFINITY;  // loads in pairs, each pair's minima read after its wait
#pragma unroll
          for (int u = 0; u < kEpiCols / 32; u += 2) {
            const float ma = tld32_min(base + 32 * u), mb = tld32_min(base + 32 * u + 32);
            tld_wait();
            mn = fminf(mn, fminf(ma, mb));
          }
          // some s - E <= 0 among this warp's columns (a NaN would also count)
          const bool any = !(mn > 0.f);
          tcb();
          __syncwarp();
          if (lane == 0) mb_arrive(bar(kAccE + slot));
          if (any && !drain && cen_p->w >= 0.f) {
            // rare: recheck this row against the block's obstacles exactly
            const float4 cen = *cen_p;
            const int j0 = t * 256 + qc * kEpiCols;
            for (int i = 0; i < kEpiCols && !hit; ++i) {
              if (j0 + i < a.n_obs) {
                ++rechecks;
                hit = hit_sphere(cen.x, cen.y, cen.z, cen.w, a.obs[j0 + i]);
              }
            }
          }
        }
        tcount += (uint32_t)n_tiles;
        if (!ok) break;
        // verdict of waypoint g: s_hit[g % 2] = g + 1 when any row collided
        const bool any = __any_sync(0xffffffffu, hit);
        if (lane == 0 && any) atomicMax((int*)&s_hit[buf], (int)(g + 1));
        __syncwarp();
        if (lane == 0) mb_arrive(bar(kVerdict + buf));
        if (!__all_sync(0xffffffffu, mb_wait(bar(kVerdict + buf), (g >> 1) & 1, s_abort))) { ok = false; break; }
        if (drain) {
          ++g;
          break;
        }
        if (s_hit[buf] == (int)(g + 1)) {
          first_hit = w;
          if (e == 0 && lane == 0) {
            // runs of one motion may finish in any order: the smallest colliding waypoint
            // wins (a projected motion enters with first_fail = -1, the largest unsigned)
            a.status[m] = (uint8_t)kCollision;
            atomicMin(reinterpret_cast<unsigned*>(&a.first_fail[m]), (unsigned)w);
          }
          if (w + 1 >= w1) {
            ++g;
            break;
          }
        }
      }
      // every epilogue warp has passed this motion's last verdict: its ring slot is free
      if (ok && e == 0 && lane == 0) *s_done = k + 1;
    }
    if (rechecks) atomicAdd(s_rechk, (unsigned long long)rechecks);
  }
  tcb();
  __syncthreads();
  if (warp == kMmaWarpCc) {
    __syncwarp();
    tca();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
  if (threadIdx.x == 0) {
    if (*s_abort) atomicExch(a.error, 1);
    if (a.counters) {
      atomicAdd(&a.counters[0], *s_rechk);
    }
  }
}

}  // namespace

size_t gemm_cc_smem_bytes() { return (size_t)kSmemCc + 1024; }

cudaError_t launch_gemm_cc(int tf32, const RobotDev& rb, const GemmCcArgs& a, int sm_count, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int smem = (int)gemm_cc_smem_bytes();
  const void* fn = tf32 ? (const void*)gemm_cc_kernel<1> : (const void*)gemm_cc_kernel<0>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int grid = a.n < sm_count ? a.n : sm_count;
  GemmCcArgs args = a;
  RobotDev r = rb;
  void* params[] = {&r, &args};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(kCcThreads), params, smem, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace cprrtc
