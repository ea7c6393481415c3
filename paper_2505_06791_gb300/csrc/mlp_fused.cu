// Fused inference of the warm-start network on the 5th-generation tensor cores.
//
// One persistent CTA per SM walks pairs of 128-row tiles. Each tile's activations stay in
// shared memory (BF16, one 64 KB buffer per tile, updated in place: a layer's epilogue
// overwrites its input only after all of that layer's MMAs have completed) and each layer's
// output accumulates in tensor memory (FP32, 128 lanes x 256 columns per tile). The two
// tiles of a pair alternate layer by layer, so the tensor cores run one tile's next layer
// while the epilogue warps work on the other tile. tcgen05.mma runs at its full width,
// M = 128, N = 256, K = 16 per instruction: narrower N re-reads the activation tile from
// shared memory once per output chunk and the tensor cores then wait on shared-memory
// bandwidth. The weights stream from L2 in K slabs (all 256 output rows x 64 inputs,
// 32 KB) through a two-stage ring filled by bulk (TMA) copies of a pre-swizzled image.
//
// Warp roles (576 threads):
//   warps 0-15 epilogue, one group of 8 per tile of the pair (the groups drift apart, so
//              one computes while the other waits): build the group's input tile; per layer
//              read the accumulator from tensor memory (warp w reads lanes 32 (w % 4) .. + 31
//              and the 32-column half (w / 4) % 2 of each 64-column block, 16 columns at a
//              time with the next load in flight), add the bias, apply GELU, and store BF16
//              back into the tile's activation buffer in the operand layout, publishing each
//              64-column block as soon as it is written; the last layer writes FP32
//              corrections to global memory.
//   warp 16    producer: one lane issues the bulk copies of weight slabs into the ring.
//   warp 17    MMA: allocates tensor memory; one lane issues the MMAs, starting each K atom
//              of a layer as soon as its activation block is published, and commits them to
//              the mbarriers that release the ring stage and publish the accumulator.
//
// Operand layout (A = activations [128][K], B = a weight slab [N][K], both K-major): the
// 128-byte swizzle of the tensor cores. K is split into atoms of 64 BF16 (128 bytes); an
// atom holds rows in groups of 8 (1024 bytes per group), and within a group the 16-byte
// piece c of row r sits at slot c ^ (r % 8).
//
// Every wait has a time limit; on expiry the CTA raises a flag, drains what it issued,
// frees tensor memory and exits, and the host-visible error word is set.
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include "launch.h"
#include "mlp_common.cuh"
#include "tcgen05.cuh"

namespace cprrtc {

namespace {

using namespace tc;

constexpr int kTileRows = 128;
constexpr int kEpiWarps = 16;
constexpr int kGroupWarps = 8;  // epilogue warps per tile of the pair
static_assert(kEpiWarps == 2 * kGroupWarps, "one epilogue group per tile of a pair");
constexpr int kProducerWarp = 16;
constexpr int kMmaWarp = 17;
constexpr int kFusedThreads = 576;
constexpr int kStages = 2;
constexpr int kStageBytes = 32768;
constexpr int kActBytes = kTileRows * 256 * 2;  // one activation buffer
constexpr uint32_t kTmemCols = 512;             // two 256-column accumulators
constexpr int kBiasFloats = 3 * 256 + 16;

constexpr int kOffAct0 = 0;          // tile 0 of a pair
constexpr int kOffAct1 = kActBytes;  // tile 1
constexpr int kOffRing = 2 * kActBytes;
constexpr int kOffBias = kOffRing + kStages * kStageBytes;
constexpr int kOffBar = kOffBias + kBiasFloats * 4;  // 8-byte aligned
// barriers: w_full[stages] w_empty[stages] acc_full[2] acc_empty[2] (per tile of the pair)
// act_full[2][4] (per tile and 64-column block) drain (the MMA issuer's last commit)
constexpr int kBarWFull = 0, kBarWEmpty = kStages, kBarAccFull = 2 * kStages;
constexpr int kBarAccEmpty = kBarAccFull + 2, kBarAct = kBarAccEmpty + 2;
constexpr int kBarDrain = kBarAct + 8;
constexpr int kNumBars = kBarDrain + 1;
constexpr int kOffTmem = kOffBar + kNumBars * 8;
constexpr int kOffAbort = kOffTmem + 4;
constexpr int kSmemUsed = kOffAbort + 4;
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // default 1 s: every wait here is microseconds
constexpr uint64_t kDrainLimitNs = 20000000ull;
// this launch's limit of a bounded wait (set by thread 0 before the first barrier)
__shared__ uint64_t s_wait_limit_ns;

static_assert(kOffBar % 8 == 0, "mbarriers need 8-byte alignment");

// Weight slab c of a tile: layer, first K atom, K atoms, rows (= MMA N), offset and size in
// the packed image. Layers 0-2 stream one K atom per slab; layer 3 (16 rows) fits in one.
struct Chunk {
  int layer, atom0, atoms, n, off, bytes;
};

__host__ __device__ __forceinline__ Chunk chunk_of(int c) {
  if (c == 0) return {0, 0, 1, 256, 0, 32768};
  if (c < 5) return {1, c - 1, 1, 256, 32768 + (c - 1) * 32768, 32768};
  if (c < 9) return {2, c - 5, 1, 256, 163840 + (c - 5) * 32768, 32768};
  return {3, 0, 4, 16, 294912, 8192};
}

// Slabs [first_chunk(l), first_chunk(l + 1)) belong to layer l.
__host__ __device__ __forceinline__ int first_chunk(int layer) { return layer == 0 ? 0 : layer == 1 ? 1 : layer == 2 ? 5 : layer == 3 ? 9 : 10; }

// Waits for the phase of `parity` to complete. Gives up (false) when another role raised
// the abort flag, or after the launch's wait limit, raising it.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  return mbar_wait_for(bar, parity, abort_flag, s_wait_limit_ns);
}

// Bounded wait that ignores the abort flag (draining on the way out).
__device__ void mbar_drain(uint32_t bar, uint32_t parity) { mbar_drain_for(bar, parity, kDrainLimitNs); }

// Inputs of tile row `row` (q / pi, zero past dof): a configuration row, or waypoint i of
// motion m when rows are motions x W waypoints.
__device__ __forceinline__ void input_row(const FusedMlpArgs& a, int row, float (&x)[kMaxDof]) {
  if (a.q) {
    const float* src = a.q + (size_t)row * a.ldq;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) x[k] = k < a.dof ? src[k] * kMlpInvPi : 0.f;
  } else {
    const int m = row / a.W, i = row - m * a.W;
    const float f = (float)i / (float)(a.W - 1);
    const float* p0 = a.q0 + (size_t)m * a.dof;
    const float* p1 = a.q1 + (size_t)m * a.dof;
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) x[k] = k < a.dof ? fmaf(f, p1[k] - p0[k], p0[k]) * kMlpInvPi : 0.f;
  }
}

// 18 warps: registers are split between the SM's four sub-partitions, and the two that
// hold five warps allow 96 registers per thread.
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
  const int pairs = (tiles + 1) / 2;  // pair p = tiles 2p and 2p + 1 (the latter may not exist)

  for (int i = threadIdx.x; i < kBiasFloats; i += blockDim.x) s_bias[i] = a.bias[i];
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(bar(kBarWFull + s), 1);
      mbar_init(bar(kBarWEmpty + s), 1);
    }
    for (int u = 0; u < 2; ++u) {
      mbar_init(bar(kBarAccFull + u), 1);
      mbar_init(bar(kBarAccEmpty + u), kGroupWarps);
    }
    for (int b = 0; b < 8; ++b) mbar_init(bar(kBarAct + b), kGroupWarps);
    mbar_init(bar(kBarDrain), 1);
    *s_abort = 0;
    s_wait_limit_ns = a.wait_ns ? a.wait_ns : kWaitLimitNs;
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
      for (int p = blockIdx.x; ok && p < pairs; p += gridDim.x) {
        const int nt = (2 * p + 1 < tiles) ? 2 : 1;
        for (int layer = 0; ok && layer < 4; ++layer)
          for (int u = 0; ok && u < nt; ++u)
            for (int c = first_chunk(layer); c < first_chunk(layer + 1); ++c, ++fill) {
              const int s = fill % kStages;
              if (fill >= (uint32_t)kStages &&
                  !mbar_wait(bar(kBarWEmpty + s), ((fill / kStages) - 1) & 1, s_abort)) {
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
      uint32_t use = 0;
      uint32_t layers = 0;  // layers issued per tile slot u, 16-bit field u
      uint32_t act_par = 0;            // bit 4u + b: parity of the next phase of block b of tile u
      bool ok = true;
      for (int p = blockIdx.x; ok && p < pairs; p += gridDim.x) {
        const int nt = (2 * p + 1 < tiles) ? 2 : 1;
        for (int layer = 0; ok && layer < 4; ++layer) {
          for (int u = 0; ok && u < nt; ++u) {
            // the tile's accumulator must have been read out by the previous layer's epilogue
            const uint32_t lu = (layers >> (16 * u)) & 0xffffu;
            if (lu >= 1 && !mbar_wait(bar(kBarAccEmpty + u), (lu - 1) & 1, s_abort)) { ok = false; break; }
            const uint32_t a_base = sbase + (u ? kOffAct1 : kOffAct0);
            const uint32_t d = tmem + (uint32_t)u * 256;
            for (int c = first_chunk(layer); ok && c < first_chunk(layer + 1); ++c) {
              const Chunk ch = chunk_of(c);
              const int s = use % kStages;
              if (!mbar_wait(bar(kBarWFull + s), (use / kStages) & 1, s_abort)) { ok = false; break; }
              tc_after();
              const uint32_t b_base = sbase + kOffRing + s * kStageBytes;
              const uint32_t idesc = mma_idesc(kTileRows, ch.n);
              for (int q = 0; q < ch.atoms; ++q) {
                const int blk = ch.atom0 + q;  // K atom = activation block
                const int bit = 4 * u + blk;
                if (!mbar_wait(bar(kBarAct + bit), (act_par >> bit) & 1u, s_abort)) { ok = false; break; }
                act_par ^= 1u << bit;
                tc_after();
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                  const uint32_t a_addr = a_base + blk * (kTileRows * 128) + kk * 32;
                  const uint32_t b_addr = b_base + q * (ch.n * 128) + kk * 32;
                  umma_bf16(d, sw128_desc(a_addr), sw128_desc(b_addr), idesc, (blk > 0 || kk > 0) ? 1u : 0u);
                }
              }
              if (!ok) break;
              umma_commit(bar(kBarWEmpty + s));
              ++use;
            }
            if (!ok) break;
            umma_commit(bar(kBarAccFull + u));
            layers += 1u << (16 * u);
          }
        }
      }
      // every MMA this thread issued has completed before tensor memory is freed, also when
      // it gave up in the middle of a slab (MMAs issued but not yet committed elsewhere): a
      // commit tracks all of the thread's earlier tcgen05 operations
      umma_commit(bar(kBarDrain));
      mbar_drain(bar(kBarDrain), 0);
    }
  } else {
    // epilogue warps: group u serves tile u of each pair
    const int u = warp >> 3, wq = warp & 3, h = (warp >> 2) & 1;  // tile slot, lane quarter, column half
    const int r = wq * 32 + lane;                                   // tile row = tensor-memory lane
    const uint32_t acc_base = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)u * 256 + (uint32_t)h * 32;
    uint8_t* act = smem + (u ? kOffAct1 : kOffAct0);
    uint32_t lu = 0;  // layers of this tile slot consumed
    bool ok = true;
    // makes this warp's shared-memory stores visible to the tensor cores, then counts the
    // warp in on block b of the group's tile
    auto publish = [&](int b) {
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(kBarAct + 4 * u + b));
    };
    auto release = [&]() {  // this warp has read the tile's accumulator
      tc_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(kBarAccEmpty + u));
    };
    for (int p = blockIdx.x; ok && p < pairs; p += gridDim.x) {
      if (2 * p + u >= tiles) continue;  // this pair has no tile for the group
      const int row = (2 * p + u) * kTileRows + r;
      {  // input tile: dof <= 8, so only the first 16 bytes of a row are nonzero
        uint32_t w0[4] = {0u, 0u, 0u, 0u};
        if (h == 0 && row < a.rows) {
          float x[kMaxDof];
          input_row(a, row, x);
#pragma unroll
          for (int e = 0; e < 4; ++e) w0[e] = pack_bf16x2(x[2 * e], x[2 * e + 1]);
        }
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4)
          *reinterpret_cast<uint4*>(act + sw128(r, h * 32 + c4 * 8, kTileRows)) =
              c4 == 0 ? make_uint4(w0[0], w0[1], w0[2], w0[3]) : make_uint4(0u, 0u, 0u, 0u);
        publish(0);
      }
      for (int layer = 0; layer < 4; ++layer, ++lu) {
        // warp-uniform outcome: the tensor-memory loads below are warp-collective
        if (!__all_sync(0xffffffffu, mbar_wait(bar(kBarAccFull + u), lu & 1, s_abort))) {
          ok = false;
          break;
        }
        tc_after();
        if (layer < 3) {
          const float* bl = s_bias + layer * 256;
          uint32_t v[16], nv[16];
          tmem_ld16(acc_base, v);
          tmem_wait_ld();
          // 8 pieces of 16 columns: piece j = block j / 2, half j % 2 of this warp's 32
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            if (j < 7) tmem_ld16(acc_base + (uint32_t)((j + 1) >> 1) * 64 + (uint32_t)((j + 1) & 1) * 16, nv);
            const int col0 = (j >> 1) * 64 + h * 32 + (j & 1) * 16;  // next layer's K index
            const float4* b4 = reinterpret_cast<const float4*>(bl + col0);
#pragma unroll
            for (int c2 = 0; c2 < 2; ++c2) {
              const float4 bA = b4[2 * c2], bB = b4[2 * c2 + 1];
              const float bb[8] = {bA.x, bA.y, bA.z, bA.w, bB.x, bB.y, bB.z, bB.w};
              uint32_t w[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int i = c2 * 8 + 2 * e;
                float g0, g1;
                mlp_gelu2(__uint_as_float(v[i]) + bb[2 * e], __uint_as_float(v[i + 1]) + bb[2 * e + 1], g0, g1);
                w[e] = pack_bf16x2(g0, g1);
              }
              // in place: all of this layer's MMAs have completed
              *reinterpret_cast<uint4*>(act + sw128(r, col0 + c2 * 8, kTileRows)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
            if (j < 7) {
              tmem_wait_ld();
              if (j == 6) release();  // the whole accumulator is in registers or consumed
#pragma unroll
              for (int i = 0; i < 16; ++i) v[i] = nv[i];
            }
            if (j & 1) publish(j >> 1);
          }
        } else {
          uint32_t v[16];
          if (h == 0) {
            tmem_ld16(acc_base, v);
            tmem_wait_ld();
          }
          release();
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
// into the image the kernel streams: per slab, the swizzled operand layout.
__global__ void mlp_pack_kernel(const __nv_bfloat16* __restrict__ w0, const __nv_bfloat16* __restrict__ w1,
                                const __nv_bfloat16* __restrict__ w2, const __nv_bfloat16* __restrict__ w3,
                                uint8_t* __restrict__ image) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  __nv_bfloat16 v = __float2bfloat16(0.f);
  uint32_t dst;
  if (e < 256 * 64) {  // layer 0: one slab, K padded to 64
    const int r = e / 64, k = e % 64;
    if (k < kMlpIO) v = w0[r * kMlpIO + k];
    dst = chunk_of(0).off + sw128(r, k, 256);
  } else if (e < 256 * 64 + 2 * 65536) {  // layers 1, 2: four slabs of 64 inputs each
    const int f = e - 256 * 64;
    const int layer = 1 + f / 65536, r = (f % 65536) / 256, k = f % 256;
    v = (layer == 1 ? w1 : w2)[r * 256 + k];
    dst = chunk_of((layer == 1 ? 1 : 5) + k / 64).off + sw128(r, k % 64, 256);
  } else if (e < 256 * 64 + 2 * 65536 + 16 * 256) {  // layer 3: one slab, 16 rows x 256
    const int f = e - 256 * 64 - 2 * 65536;
    const int r = f / 256, k = f % 256;
    v = w3[r * 256 + k];
    dst = chunk_of(9).off + sw128(r, k, 16);
  } else {
    return;
  }
  *reinterpret_cast<__nv_bfloat16*>(image + dst) = v;
}

}  // namespace

size_t mlp_fused_image_bytes() { return (size_t)chunk_of(9).off + chunk_of(9).bytes; }
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

static char g_fused_diag[256];

const char* mlp_fused_diag() { return g_fused_diag; }

cudaError_t launch_mlp_fused(const FusedMlpArgs& a, int sm_count, cudaStream_t s) {
  if (a.rows <= 0) return cudaSuccess;
  const int smem = (int)mlp_fused_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_fused_kernel, kFusedThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, mlp_fused_kernel);
    snprintf(g_fused_diag, sizeof(g_fused_diag),
             "fused MLP kernel does not fit an SM: %d registers/thread, max %d threads/block, "
             "%zu B static + %d B dynamic shared memory, %d threads",
             fa.numRegs, fa.maxThreadsPerBlock, fa.sharedSizeBytes, smem, kFusedThreads);
    return cudaErrorLaunchOutOfResources;
  }
  const int pairs = ((a.rows + kTileRows - 1) / kTileRows + 1) / 2;
  const int grid = pairs < sm_count ? pairs : sm_count;
  mlp_fused_kernel<<<grid, kFusedThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace cprrtc
