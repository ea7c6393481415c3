// Fused inference of the warm-start network on the 5th-generation tensor cores.
//
// One persistent CTA per SM walks 128-row tiles. For each tile the four layers run back to
// back without leaving the SM: activations stay in shared memory (BF16, two 64 KB
// buffers used in turn), each layer's output is produced in chunks of 64 columns by
// tcgen05.mma (M = 128, N = 64, K = 16 per instruction, FP32 accumulators in tensor
// memory), and the weights stream from L2 through a two-stage ring filled by bulk (TMA)
// copies of a pre-swizzled image, so no thread formats operands on the way in.
//
// Warp roles (320 threads):
//   warps 0-7  epilogue: build the input tile, then per chunk read the accumulator from
//              tensor memory (warp w reads lanes 32 (w % 4) .. + 31, column half w / 4),
//              add the bias, apply GELU, and store BF16 into the next activation buffer in
//              the operand layout; the last layer writes FP32 corrections to global memory.
//   warp 8     producer: one lane issues the bulk copies of weight chunks into the ring.
//   warp 9     MMA: allocates tensor memory; one lane issues the MMAs and commits them to
//              the mbarriers that release the ring stage and publish the accumulator.
//
// Operand layout (A = activations [128][K], B = a weight chunk [N][K], both K-major): the
// 128-byte swizzle of the tensor cores. K is split into atoms of 64 BF16 (128 bytes); an
// atom holds rows in groups of 8 (1024 bytes per group), and within a group the 16-byte
// piece c of row r sits at slot c ^ (r % 8).
//
// Every wait has a time limit; on expiry the CTA raises a flag, drains what it issued,
// frees tensor memory and exits, and the host-visible error word is set.
#include <cuda_bf16.h>
#include <stdint.h>

#include "launch.h"
#include "mlp_common.cuh"

namespace cprrtc {

namespace {

constexpr int kTileRows = 128;
constexpr int kEpiWarps = 8;
constexpr int kProducerWarp = 8;
constexpr int kMmaWarp = 9;
constexpr int kFusedThreads = 320;
constexpr int kStages = 2;
constexpr int kStageBytes = 32768;
constexpr int kActBytes = kTileRows * 256 * 2;  // one activation buffer
constexpr int kChunks = 13;                     // weight chunks per tile: 4 + 4 + 4 + 1
constexpr int kAccSlots = 4;                    // 64-column accumulators in tensor memory
constexpr uint32_t kTmemCols = 256;
constexpr int kBiasFloats = 3 * 256 + 16;

constexpr int kOffAct0 = 0;
constexpr int kOffAct1 = kActBytes;
constexpr int kOffRing = 2 * kActBytes;
constexpr int kOffBias = kOffRing + kStages * kStageBytes;
constexpr int kOffBar = kOffBias + kBiasFloats * 4;  // 8-byte aligned
// barriers: w_full[2] w_empty[2] acc_full[4] acc_empty[4] act_full
constexpr int kBarWFull = 0, kBarWEmpty = 2, kBarAccFull = 4, kBarAccEmpty = 8, kBarAct = 12;
constexpr int kNumBars = 13;
constexpr int kOffTmem = kOffBar + kNumBars * 8;
constexpr int kOffAbort = kOffTmem + 4;
constexpr int kSmemUsed = kOffAbort + 4;
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s: every wait here is microseconds
constexpr uint64_t kDrainLimitNs = 20000000ull;

static_assert(kOffBar % 8 == 0, "mbarriers need 8-byte alignment");

// Weight chunk c of a tile: layer, chunk index within the layer, rows (= MMA N), K, offset
// and size in the packed image.
struct Chunk {
  int layer, j, n, k, off, bytes;
};

__host__ __device__ __forceinline__ Chunk chunk_of(int c) {
  if (c < 4) return {0, c, 64, 64, c * 8192, 8192};
  if (c < 8) return {1, c - 4, 64, 256, 32768 + (c - 4) * 32768, 32768};
  if (c < 12) return {2, c - 8, 64, 256, 163840 + (c - 8) * 32768, 32768};
  return {3, 0, 16, 256, 294912, 8192};
}

// Byte offset of element (r, k) of a K-major operand with R rows, 128-byte swizzle.
__host__ __device__ __forceinline__ uint32_t sw128(int r, int k, int R) {
  return (uint32_t)((k >> 6) * (R * 128) + (r >> 3) * 1024 + (r & 7) * 128 +
                    ((((k >> 3) & 7) ^ (r & 7)) << 4) + (k & 7) * 2);
}

// Shared-memory matrix descriptor of tcgen05.mma for the layout above: start address,
// leading offset (unused by swizzled K-major operands), 1024-byte stride between 8-row
// groups, descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase of `parity` to complete. Gives up (false) when another role raised
// the abort flag, or after kWaitLimitNs, raising it.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  for (;;) {
    for (int i = 0; i < 32; ++i)
      if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (now_ns() - t0 > kWaitLimitNs) {
      *abort_flag = 1;
      return false;
    }
  }
}

// Bounded wait that ignores the abort flag (draining on the way out).
__device__ void mbar_drain(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = now_ns();
  while (!mbar_try(bar, parity) && now_ns() - t0 < kDrainLimitNs) {
  }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
        "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
        "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
        "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
        "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Input value k of tile row `row`: q / pi of a configuration row, or of waypoint i of
// motion m when rows are motions x W waypoints.
__device__ __forceinline__ float input_value(const FusedMlpArgs& a, int row, int k) {
  if (a.q) return a.q[(size_t)row * a.ldq + k] * kMlpInvPi;
  const int m = row / a.W, i = row - m * a.W;
  const float x0 = a.q0[(size_t)m * a.dof + k], x1 = a.q1[(size_t)m * a.dof + k];
  return fmaf((float)i / (float)(a.W - 1), x1 - x0, x0) * kMlpInvPi;
}

__global__ void __launch_bounds__(kFusedThreads, 1) mlp_fused_kernel(FusedMlpArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_addr(smem);
  float* s_bias = reinterpret_cast<float*>(smem + kOffBias);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + kOffTmem);
  volatile int* s_abort = reinterpret_cast<volatile int*>(smem + kOffAbort);
  auto bar = [&](int i) { return sbase + kOffBar + 8u * (uint32_t)i; };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = (a.rows + kTileRows - 1) / kTileRows;

  for (int i = threadIdx.x; i < kBiasFloats; i += blockDim.x) s_bias[i] = a.bias[i];
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(bar(kBarWFull + s), 1);
      mbar_init(bar(kBarWEmpty + s), 1);
    }
    for (int s = 0; s < kAccSlots; ++s) {
      mbar_init(bar(kBarAccFull + s), 1);
      mbar_init(bar(kBarAccEmpty + s), kEpiWarps);
    }
    mbar_init(bar(kBarAct), kEpiWarps * 32);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *s_tmem;

  if (warp == kProducerWarp) {
    if (lane == 0) {
      uint32_t fill = 0;
      bool ok = true;
      for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x) {
        for (int c = 0; c < kChunks; ++c, ++fill) {
          const int s = fill % kStages;
          if (fill >= (uint32_t)kStages && !mbar_wait(bar(kBarWEmpty + s), ((fill / kStages) - 1) & 1, s_abort)) {
            ok = false;
            break;
          }
          const Chunk ch = chunk_of(c);
          mbar_expect_tx(bar(kBarWFull + s), (uint32_t)ch.bytes);
          bulk_g2s(sbase + kOffRing + s * kStageBytes, a.wpack + ch.off, (uint32_t)ch.bytes, bar(kBarWFull + s));
        }
      }
      // no copy may still be landing when the CTA exits
      for (uint32_t f = fill > (uint32_t)kStages ? fill - kStages : 0; f < fill; ++f)
        mbar_drain(bar(kBarWFull + f % kStages), (f / kStages) & 1);
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      uint32_t use = 0, acc = 0, actw = 0;
      bool ok = true;
      for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x) {
        for (int c = 0; c < kChunks; ++c) {
          const Chunk ch = chunk_of(c);
          if (ch.j == 0) {  // the layer's input activations complete
            if (!mbar_wait(bar(kBarAct), actw & 1, s_abort)) { ok = false; break; }
            ++actw;
          }
          const int s = use % kStages, slot = acc % kAccSlots;
          if (!mbar_wait(bar(kBarWFull + s), (use / kStages) & 1, s_abort)) { ok = false; break; }
          if (acc >= (uint32_t)kAccSlots &&
              !mbar_wait(bar(kBarAccEmpty + slot), ((acc / kAccSlots) - 1) & 1, s_abort)) {
            ok = false;
            break;
          }
          tc_after();
          const uint32_t a_base = sbase + ((ch.layer & 1) ? kOffAct1 : kOffAct0);
          const uint32_t b_base = sbase + kOffRing + s * kStageBytes;
          const uint32_t d = tmem + (uint32_t)slot * 64;
          const uint32_t idesc = mma_idesc(kTileRows, ch.n);
          for (int kk = 0; kk < ch.k / 16; ++kk) {
            const uint32_t a_addr = a_base + (kk >> 2) * (kTileRows * 128) + (kk & 3) * 32;
            const uint32_t b_addr = b_base + (kk >> 2) * (ch.n * 128) + (kk & 3) * 32;
            umma_bf16(d, sw128_desc(a_addr), sw128_desc(b_addr), idesc, kk > 0 ? 1u : 0u);
          }
          umma_commit(bar(kBarWEmpty + s));
          umma_commit(bar(kBarAccFull + slot));
          ++use;
          ++acc;
        }
      }
      if (acc > 0) mbar_drain(bar(kBarAccFull + (acc - 1) % kAccSlots), ((acc - 1) / kAccSlots) & 1);
    }
  } else {
    // epilogue warps
    const int wq = warp & 3, h = warp >> 2;
    const int r = wq * 32 + lane;  // tile row = tensor-memory lane
    const uint32_t lane_addr = tmem + ((uint32_t)(wq * 32) << 16);
    uint32_t acc = 0;
    bool ok = true;
    for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x) {
      const int row = t * kTileRows + r;
      {  // input tile: columns h*32 .. h*32+31 of row r (dof used, zero padding to 64)
        uint8_t* dst = smem + kOffAct0;
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
          uint32_t w[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int k0 = h * 32 + c4 * 8 + 2 * e;
            const float lo = (row < a.rows && k0 < a.dof) ? input_value(a, row, k0) : 0.f;
            const float hi = (row < a.rows && k0 + 1 < a.dof) ? input_value(a, row, k0 + 1) : 0.f;
            w[e] = pack_bf16x2(lo, hi);
          }
          *reinterpret_cast<uint4*>(dst + sw128(r, h * 32 + c4 * 8, kTileRows)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        fence_async_smem();
        mbar_arrive(bar(kBarAct));
      }
      for (int c = 0; c < kChunks; ++c, ++acc) {
        const Chunk ch = chunk_of(c);
        const int slot = acc % kAccSlots;
        // warp-uniform outcome: the tensor-memory loads below are warp-collective
        if (!__all_sync(0xffffffffu, mbar_wait(bar(kBarAccFull + slot), (acc / kAccSlots) & 1, s_abort))) {
          ok = false;
          break;
        }
        tc_after();
        if (ch.layer < 3) {
          uint32_t v[32];
          tmem_ld32(lane_addr + (uint32_t)slot * 64 + (uint32_t)h * 32, v);
          tmem_wait_ld();
          tc_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(kBarAccEmpty + slot));
          const int col0 = ch.j * 64 + h * 32;  // output column = next layer's K index
          const float* b = s_bias + ch.layer * 256 + col0;
          uint8_t* dst = smem + ((ch.layer & 1) ? kOffAct0 : kOffAct1);
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int i = c4 * 8 + 2 * e;
              w[e] = pack_bf16x2(mlp_gelu(__uint_as_float(v[i]) + b[i]), mlp_gelu(__uint_as_float(v[i + 1]) + b[i + 1]));
            }
            *reinterpret_cast<uint4*>(dst + sw128(r, col0 + c4 * 8, kTileRows)) = make_uint4(w[0], w[1], w[2], w[3]);
          }
          if (ch.j == 3) {
            fence_async_smem();
            mbar_arrive(bar(kBarAct));
          }
        } else {
          uint32_t v[16];
          if (h == 0) {
            tmem_ld16(lane_addr + (uint32_t)slot * 64, v);
            tmem_wait_ld();
          }
          tc_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(kBarAccEmpty + slot));
          if (h == 0 && row < a.rows) {
            float4* o = reinterpret_cast<float4*>(a.out + (size_t)row * 16);
            const float* b = s_bias + 768;
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4)
              o[q4] = make_float4(__uint_as_float(v[4 * q4]) + b[4 * q4], __uint_as_float(v[4 * q4 + 1]) + b[4 * q4 + 1],
                                  __uint_as_float(v[4 * q4 + 2]) + b[4 * q4 + 2],
                                  __uint_as_float(v[4 * q4 + 3]) + b[4 * q4 + 3]);
          }
        }
      }
    }
  }
  tc_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    __syncwarp();
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  if (threadIdx.x == 0 && *s_abort) atomicExch(a.error, 1);
}

// Packs the BF16 weights (padded [out][in] per layer: [256][16], [256][256] x 2, [16][256])
// into the image the kernel streams: per chunk, the swizzled operand layout.
__global__ void mlp_pack_kernel(const __nv_bfloat16* __restrict__ w0, const __nv_bfloat16* __restrict__ w1,
                                const __nv_bfloat16* __restrict__ w2, const __nv_bfloat16* __restrict__ w3,
                                uint8_t* __restrict__ image) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  int layer, rg, k;
  if (e < 256 * 64) {
    layer = 0; rg = e / 64; k = e % 64;
  } else if (e < 256 * 64 + 2 * 65536) {
    const int f = e - 256 * 64;
    layer = 1 + f / 65536; rg = (f % 65536) / 256; k = f % 256;
  } else if (e < 256 * 64 + 2 * 65536 + 16 * 256) {
    const int f = e - 256 * 64 - 2 * 65536;
    layer = 3; rg = f / 256; k = f % 256;
  } else {
    return;
  }
  __nv_bfloat16 v = __float2bfloat16(0.f);
  int c, r, R;
  if (layer == 0) {
    if (k < kMlpIO) v = w0[rg * kMlpIO + k];
    c = rg / 64; r = rg % 64; R = 64;
  } else if (layer < 3) {
    v = (layer == 1 ? w1 : w2)[rg * 256 + k];
    c = 4 * layer + rg / 64; r = rg % 64; R = 64;
  } else {
    v = w3[rg * 256 + k];
    c = 12; r = rg; R = 16;
  }
  *reinterpret_cast<__nv_bfloat16*>(image + chunk_of(c).off + sw128(r, k, R)) = v;
}

}  // namespace

size_t mlp_fused_image_bytes() { return (size_t)chunk_of(12).off + chunk_of(12).bytes; }
int mlp_fused_bias_floats() { return kBiasFloats; }
size_t mlp_fused_smem_bytes() { return (size_t)kSmemUsed + 1024; }

cudaError_t launch_mlp_pack(const void* w0, const void* w1, const void* w2, const void* w3,
                            uint8_t* image, cudaStream_t s) {
  const int n = 256 * 64 + 2 * 65536 + 16 * 256;
  mlp_pack_kernel<<<(n + 255) / 256, 256, 0, s>>>(
      static_cast<const __nv_bfloat16*>(w0), static_cast<const __nv_bfloat16*>(w1),
      static_cast<const __nv_bfloat16*>(w2), static_cast<const __nv_bfloat16*>(w3), image);
  return cudaGetLastError();
}

cudaError_t launch_mlp_fused(const FusedMlpArgs& a, int sm_count, cudaStream_t s) {
  if (a.rows <= 0) return cudaSuccess;
  const int smem = (int)mlp_fused_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int tiles = (a.rows + kTileRows - 1) / kTileRows;
  const int grid = tiles < sm_count ? tiles : sm_count;
  mlp_fused_kernel<<<grid, kFusedThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace cprrtc
