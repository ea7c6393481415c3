// Learned projection warm start: a 4-layer MLP (dof -> 256 -> 256 -> 256 -> dof, GELU),
// BF16 weights and activations, FP32 accumulation on the tensor cores, trained with Adam
// by the kernels below (forward, backward, optimiser), and evaluated in batches to give
// Alg. 1 a starting segment closer to the manifold.
//
// GEMM: C[M,N] = A'[M,K] B'[K,N] in BF16 x BF16 -> FP32 on the 5th-generation tensor cores
// (tcgen05.mma, kind::f16, accumulator in tensor memory). A' is A ([M][K], or [K][M] when
// transposed) and B' is B ([K][N], or [N][K] when transposed), all row-major with given
// leading dimensions. A CTA computes a 128 x BN output tile (BN = 32, or 16 for the 16-wide
// input and output layers): its 8 warps stage K chunks of 64 of both operands into shared
// memory in the 128-byte-swizzled K-major layout (transposed on the way in when needed, zero
// past the matrix), two chunks in flight, while one thread issues the chunk's MMAs (K = 16
// each) and commits them to the chunk's mbarrier. The epilogue reads the accumulator with
// tensor-memory loads (warp w: lanes 32 (w % 4) .., 16-column groups of parity w / 4) and
// fuses the bias, GELU, GELU's derivative or split-K accumulation.
//
// FP32 checking mode: the same network, forward pass and gradient with FP32 weights and
// activations (no rounding to BF16 anywhere) on a plain FP32 FMA GEMM with the same
// epilogues. It separates the arithmetic of the layers from the BF16 rounding when the
// kernels are compared with an FP64 evaluation; inference in this mode skips the fused
// tensor-core kernel.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>

#include "launch.h"
#include "mlp_common.cuh"
#include "tcgen05.cuh"

namespace cprrtc {

namespace {

constexpr int kTM = 64, kTN = 64;  // output tile of the FP32 checking mode's GEMM
constexpr int kTcM = 128, kTcK = 64, kTcThreads = 256;
constexpr uint64_t kTcWaitNs = 1000000000ull, kTcDrainNs = 20000000ull;

}  // namespace

// Epilogue kinds.
enum : int {
  kEpiStore = 0,     // C (FP32) = acc
  kEpiBiasGelu = 1,  // Z (FP32) = acc + bias; H (BF16) = gelu(Z)
  kEpiBias = 2,      // C (FP32) = acc + bias
  kEpiGeluBwd = 3,   // H (BF16) = acc * gelu'(Z)   (Z read, FP32)
  kEpiAtomic = 4,    // C (FP32) += acc  (split-K)
};

// Operands of one GEMM; T is the element type of A, B and the activation output H (BF16, or
// FP32 in the checking mode).
template <class T>
struct GemmArgsT {
  int M, N, K;
  const T* A;
  int lda, transA;
  const T* B;
  int ldb, transB;
  float* C;  // FP32 output / Z (ldc)
  int ldc;
  T* H;      // activation output (ldh)
  int ldh;
  const float* bias;
  const float* Z;  // pre-activation for the GELU backward (ldc)
  int k_split;     // K range per blockIdx.z
  int* error;      // set to 1 when a bounded wait of the tensor-core GEMM ran out (may be null)
  unsigned long long wait_ns;  // limit of its bounded waits (0: 1 s)
  int vec_a, vec_b;  // set by the launcher: the operand's rows are 16-byte aligned
};
using GemmArgs = GemmArgsT<__nv_bfloat16>;
using GemmArgsF = GemmArgsT<float>;

template <class T>
__device__ __forceinline__ T to_act(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to_act<__nv_bfloat16>(float x) { return __float2bfloat16(x); }
template <>
__device__ __forceinline__ float to_act<float>(float x) { return x; }
__device__ __forceinline__ float act_f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float act_f(float x) { return x; }

// The epilogue of one accumulated element (row gm, column gn), shared by both GEMMs.
template <int EPI, class T>
__device__ __forceinline__ void epilogue(const GemmArgsT<T>& g, int gm, int gn, float v) {
  const size_t ci = (size_t)gm * g.ldc + gn;
  if (EPI == kEpiStore) {
    g.C[ci] = v;
  } else if (EPI == kEpiAtomic) {
    atomicAdd(&g.C[ci], v);
  } else if (EPI == kEpiBias) {
    g.C[ci] = v + g.bias[gn];
  } else if (EPI == kEpiBiasGelu) {
    const float z = v + g.bias[gn];
    if (g.C) g.C[ci] = z;
    g.H[(size_t)gm * g.ldh + gn] = to_act<T>(mlp_gelu(z));
  } else {  // kEpiGeluBwd
    g.H[(size_t)gm * g.ldh + gn] = to_act<T>(v * mlp_gelu_grad(g.Z[ci]));
  }
}

// Shared memory of gemm_tc_kernel: two stages of (A' 128 x 64, B' up to 64 x 64) BF16
// chunks, then two mbarriers (the chunk's MMAs done), the tensor-memory address and the
// abort flag; 1024-byte alignment slack for the swizzled operands.
constexpr int kTcStageA = kTcM * 128, kTcStage = kTcStageA + 64 * 128;
constexpr int kTcOffBar = 2 * kTcStage;
constexpr size_t kTcSmem = kTcOffBar + 32 + 1024;

// One operand of a K chunk: rows r0.. (R rows: 128, or BN) x K [k0, k0 + 64) of a source that
// is K-contiguous ([rows][K], KMAJOR) or row-contiguous ([K][rows]) with leading dimension ld
// and `nrows` valid rows, staged into `dst` (swizzled), zero past the matrix and past ke.
// With `vec` (16-byte aligned source rows) a thread moves 8 elements at a time: 8 consecutive
// k of one row (K-contiguous), or 8 consecutive rows of one k (row-contiguous, written to 8
// rows of the tile). Every thread loads its share into registers first (all loads in flight)
// and then stores it.
__device__ __forceinline__ unsigned short bits_or_zero(const __nv_bfloat16* p, bool ok) {
  return ok ? __bfloat16_as_ushort(*p) : (unsigned short)0;
}

template <int R, bool KMAJOR>
__device__ __forceinline__ void stage_operand(const __nv_bfloat16* __restrict__ src, int ld, bool vec,
                                              int r0, int nrows, int k0, int ke, uint8_t* dst) {
  if (vec) {
    constexpr int kPieces = R * kTcK / 8, kPer = (kPieces + kTcThreads - 1) / kTcThreads;
    uint4 v[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int p = threadIdx.x + i * kTcThreads;
      // K-contiguous: row p / 8, k 8 (p % 8) ..; row-contiguous: k p / (R / 8), rows 8 (p % (R / 8)) ..
      const int r = KMAJOR ? p >> 3 : 8 * (p % (R / 8)), k = KMAJOR ? 8 * (p & 7) : p / (R / 8);
      const int gr = r0 + r, gk = k0 + k;
      v[i] = make_uint4(0u, 0u, 0u, 0u);
      if (p >= kPieces) continue;
      if (KMAJOR ? (gr < nrows && gk + 8 <= ke) : (gk < ke && gr + 8 <= nrows)) {
        v[i] = *reinterpret_cast<const uint4*>(KMAJOR ? src + (size_t)gr * ld + gk : src + (size_t)gk * ld + gr);
      } else if (KMAJOR ? gr < nrows : gk < ke) {  // a ragged piece, element by element
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int j0 = 2 * j, j1 = 2 * j + 1;
          const unsigned short lo = KMAJOR ? bits_or_zero(src + (size_t)gr * ld + gk + j0, gk + j0 < ke)
                                           : bits_or_zero(src + (size_t)gk * ld + gr + j0, gr + j0 < nrows);
          const unsigned short hi = KMAJOR ? bits_or_zero(src + (size_t)gr * ld + gk + j1, gk + j1 < ke)
                                           : bits_or_zero(src + (size_t)gk * ld + gr + j1, gr + j1 < nrows);
          w[j] = (uint32_t)lo | ((uint32_t)hi << 16);
        }
        v[i] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int p = threadIdx.x + i * kTcThreads;
      if (p >= kPieces) continue;
      if (KMAJOR) {
        *reinterpret_cast<uint4*>(dst + tc::sw128(p >> 3, 8 * (p & 7), R)) = v[i];
      } else {
        const int r = 8 * (p % (R / 8)), k = p / (R / 8);
        const uint32_t w[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
#pragma unroll
        for (int j = 0; j < 8; ++j)
          *reinterpret_cast<unsigned short*>(dst + tc::sw128(r + j, k, R)) =
              (unsigned short)(w[j >> 1] >> (16 * (j & 1)));
      }
    }
    return;
  }
  constexpr int kPer = R * kTcK / kTcThreads;
  static_assert(R * kTcK % kTcThreads == 0, "whole elements per thread");
  __nv_bfloat16 v[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int e = threadIdx.x + i * kTcThreads;
    // K-contiguous: consecutive threads walk k; row-contiguous: consecutive threads walk rows
    const int r = KMAJOR ? e / kTcK : e % R, k = KMAJOR ? e % kTcK : e / R;
    const int gr = r0 + r, gk = k0 + k;
    v[i] = __float2bfloat16(0.f);
    if (gr < nrows && gk < ke) v[i] = KMAJOR ? src[(size_t)gr * ld + gk] : src[(size_t)gk * ld + gr];
  }
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int e = threadIdx.x + i * kTcThreads;
    const int r = KMAJOR ? e / kTcK : e % R, k = KMAJOR ? e % kTcK : e / R;
    *reinterpret_cast<__nv_bfloat16*>(dst + tc::sw128(r, k, R)) = v[i];
  }
}

// Stages K chunk [k0, k0 + 64) of the tile's A' rows m0.. (128) and B' rows n0.. (BN, the
// output columns) into sa / sb.
template <int BN>
__device__ __forceinline__ void stage_tc(const GemmArgs& g, int m0, int n0, int k0, int ke,
                                         uint8_t* sa, uint8_t* sb) {
  if (g.transA)
    stage_operand<kTcM, false>(g.A, g.lda, g.vec_a, m0, g.M, k0, ke, sa);
  else
    stage_operand<kTcM, true>(g.A, g.lda, g.vec_a, m0, g.M, k0, ke, sa);
  if (g.transB)
    stage_operand<BN, true>(g.B, g.ldb, g.vec_b, n0, g.N, k0, ke, sb);
  else
    stage_operand<BN, false>(g.B, g.ldb, g.vec_b, n0, g.N, k0, ke, sb);
}

// One 128 x BN output tile (BN 16 or 32) over the K range of split blockIdx.z. Every wait is
// bounded; on expiry the CTA raises its abort flag, skips the rest, waits (bounded) for the
// MMAs it issued, frees tensor memory, exits and sets *g.error.
template <int EPI, int BN>
__global__ void __launch_bounds__(kTcThreads, 1) gemm_tc_kernel(GemmArgs g) {
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 64, "MMA N of an M = 128 tile");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = tc::smem_addr(smem);
  auto bar = [&](int i) { return sbase + kTcOffBar + 8u * (uint32_t)i; };
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + kTcOffBar + 16);
  volatile int* s_abort = reinterpret_cast<volatile int*>(smem + kTcOffBar + 20);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTcM, n0 = blockIdx.y * BN;
  const int kb = blockIdx.z * g.k_split, ke = min(g.K, kb + g.k_split);
  const int nchunks = (ke - kb + kTcK - 1) / kTcK;
  constexpr uint32_t cols = BN <= 32 ? 32u : 64u;  // tensor-memory columns (a power of 2, >= 32)
  const uint64_t limit = g.wait_ns ? g.wait_ns : kTcWaitNs;
  if (threadIdx.x == 0) {
    tc::mbar_init(bar(0), 1);
    tc::mbar_init(bar(1), 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_addr(s_tmem)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::tc_before();
  __syncthreads();
  tc::tc_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t idesc = tc::mma_idesc(kTcM, BN);
  int issued = 0;  // thread 0: chunks whose MMAs were committed
  for (int c = 0; c < nchunks; ++c) {
    const int s = c & 1;
    // stage s was read by the MMAs of chunk c - 2 (phase (c - 2) / 2 of its barrier)
    if (c >= 2) tc::mbar_wait_for(bar(s), ((c - 2) >> 1) & 1, s_abort, limit);
    __syncthreads();
    if (*s_abort) break;
    const int k0 = kb + c * kTcK;
    stage_tc<BN>(g, m0, n0, k0, ke, smem + s * kTcStage, smem + s * kTcStage + kTcStageA);
    tc::fence_async_smem();  // the staged operands are visible to the tensor cores
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::tc_after();
      const int steps = (min(kTcK, ke - k0) + 15) / 16;
      const uint32_t a_addr = sbase + (uint32_t)(s * kTcStage), b_addr = a_addr + kTcStageA;
      for (int kk = 0; kk < steps; ++kk)
        tc::umma_bf16(tmem, tc::sw128_desc(a_addr + 32u * kk), tc::sw128_desc(b_addr + 32u * kk), idesc,
                      (c > 0 || kk > 0) ? 1u : 0u);
      tc::umma_commit(bar(s));
      issued = c + 1;
    }
  }
  // the accumulator is complete once the last chunk's MMAs are
  if (!*s_abort) tc::mbar_wait_for(bar((nchunks - 1) & 1), ((nchunks - 1) >> 1) & 1, s_abort, limit);
  tc::tc_after();
  __syncthreads();
  if (!*s_abort) {
    const int q = warp & 3, h = warp >> 2;  // lane quarter, column-group parity
    const int gm = m0 + 32 * q + lane;
    for (int j = h; 16 * j < BN; j += 2) {
      uint32_t v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * j), v);
      tc::tmem_wait_ld();
      if (gm < g.M) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int gn = n0 + 16 * j + i;
          if (gn < g.N) epilogue<EPI>(g, gm, gn, __uint_as_float(v[i]));
        }
      }
    }
  } else if (threadIdx.x == 0) {  // no MMA may still be running when tensor memory is freed
    for (int c = issued > 2 ? issued - 2 : 0; c < issued; ++c)
      tc::mbar_drain_for(bar(c & 1), (c >> 1) & 1, kTcDrainNs);
  }
  tc::tc_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc::tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
  }
  if (threadIdx.x == 0 && *s_abort && g.error) atomicExch(g.error, 1);
}

// The FP32 checking mode's GEMM: 64 x 64 output tiles, K steps of 16, 256 threads with 4 x 4
// outputs each; operands staged in shared memory as [k][row] (transposed on the way in
// when needed); FP32 FMA accumulation in k order within a split.
constexpr int kFK = 16;
template <int EPI>
__global__ void __launch_bounds__(256) gemm_f32_kernel(GemmArgsF g) {
  __shared__ float As[kFK][kTM + 4];
  __shared__ float Bs[kFK][kTN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * kTN;
  const int kb = blockIdx.z * g.k_split, ke = min(g.K, kb + g.k_split);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += kFK) {
    for (int e = tid; e < kTM * kFK; e += 256) {
      int r, k;
      if (g.transA) {  // source [K][M]
        r = e % kTM;
        k = e / kTM;
      } else {         // source [M][K]
        r = e / kFK;
        k = e % kFK;
      }
      const int gm = m0 + r, gk = k0 + k;
      float v = 0.f;
      if (gm < g.M && gk < ke) v = g.transA ? g.A[(size_t)gk * g.lda + gm] : g.A[(size_t)gm * g.lda + gk];
      As[k][r] = v;
    }
    for (int e = tid; e < kTN * kFK; e += 256) {
      int c, k;
      if (g.transB) {  // source [N][K]
        c = e / kFK;
        k = e % kFK;
      } else {         // source [K][N]
        c = e % kTN;
        k = e / kTN;
      }
      const int gn = n0 + c, gk = k0 + k;
      float v = 0.f;
      if (gn < g.N && gk < ke) v = g.transB ? g.B[(size_t)gn * g.ldb + gk] : g.B[(size_t)gk * g.ldb + gn];
      Bs[k][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kFK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
      if (gm < g.M && gn < g.N) epilogue<EPI>(g, gm, gn, acc[i][j]);
    }
}

// Grid of one GEMM: output tiles of tm x tn, and for the split-K epilogue enough splits of
// the reduction to cover the GPU (each a multiple of k_step).
template <class T>
static dim3 gemm_grid(int epi, GemmArgsT<T>& g, int tm, int tn, int k_step, int k_min = 256) {
  int splits = 1;
  if (epi == kEpiAtomic) {  // splits of at least k_min
    const int tiles = ((g.M + tm - 1) / tm) * ((g.N + tn - 1) / tn);
    splits = std::max(1, std::min((g.K + k_min - 1) / k_min, (4 * 152 + tiles - 1) / tiles));
  }
  g.k_split = ((g.K + splits - 1) / splits + k_step - 1) / k_step * k_step;
  splits = (g.K + g.k_split - 1) / g.k_split;
  return dim3((g.M + tm - 1) / tm, (g.N + tn - 1) / tn, splits);
}

template <int EPI, int BN>
static cudaError_t launch_tc(const GemmArgs& g, dim3 grid, cudaStream_t stream) {
  // the kernel's shared memory is above the 48 KB default: set once per device
  static std::atomic<unsigned long long> set_on{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(set_on.load() & bit)) {
    e = cudaFuncSetAttribute(gemm_tc_kernel<EPI, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e != cudaSuccess) return e;
    set_on.fetch_or(bit);
  }
  gemm_tc_kernel<EPI, BN><<<grid, kTcThreads, kTcSmem, stream>>>(g);
  return cudaGetLastError();
}

template <int EPI>
static cudaError_t launch_tc_n(const GemmArgs& g, dim3 grid, int BN, cudaStream_t stream) {
  return BN == 16 ? launch_tc<EPI, 16>(g, grid, stream) : launch_tc<EPI, 32>(g, grid, stream);
}

cudaError_t launch_gemm(int epi, const GemmArgs& g0, cudaStream_t stream) {
  GemmArgs g = g0;
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
  // narrow tiles and short splits: these GEMMs are small, so more CTAs finish sooner
  const int BN = g.N <= 16 ? 16 : 32;
  const dim3 grid = gemm_grid(epi, g, kTcM, BN, kTcK, 2 * kTcK);
  auto rows16 = [](const void* p, int ld) { return ((uintptr_t)p & 15) == 0 && ld % 8 == 0; };
  g.vec_a = rows16(g.A, g.lda);
  g.vec_b = rows16(g.B, g.ldb);
  switch (epi) {
    case kEpiStore: return launch_tc_n<kEpiStore>(g, grid, BN, stream);
    case kEpiBiasGelu: return launch_tc_n<kEpiBiasGelu>(g, grid, BN, stream);
    case kEpiBias: return launch_tc_n<kEpiBias>(g, grid, BN, stream);
    case kEpiGeluBwd: return launch_tc_n<kEpiGeluBwd>(g, grid, BN, stream);
    default: return launch_tc_n<kEpiAtomic>(g, grid, BN, stream);
  }
}

cudaError_t launch_gemm(int epi, const GemmArgsF& g0, cudaStream_t stream) {
  GemmArgsF g = g0;
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
  const dim3 grid = gemm_grid(epi, g, kTM, kTN, kFK);
  switch (epi) {
    case kEpiStore: gemm_f32_kernel<kEpiStore><<<grid, 256, 0, stream>>>(g); break;
    case kEpiBiasGelu: gemm_f32_kernel<kEpiBiasGelu><<<grid, 256, 0, stream>>>(g); break;
    case kEpiBias: gemm_f32_kernel<kEpiBias><<<grid, 256, 0, stream>>>(g); break;
    case kEpiGeluBwd: gemm_f32_kernel<kEpiGeluBwd><<<grid, 256, 0, stream>>>(g); break;
    default: gemm_f32_kernel<kEpiAtomic><<<grid, 256, 0, stream>>>(g); break;
  }
  return cudaGetLastError();
}

// ---- elementwise kernels ---------------------------------------------------------------

// X[r][0..in) = q[r][k] / pi (k < dof), zero padding; rows of the input to layer 1.
template <class T>
__global__ void mlp_input_kernel(const float* __restrict__ q, int ldq, int rows, int dof, int in, T* X) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * in) return;
  const int r = i / in, k = i - r * in;
  X[i] = to_act<T>(k < dof ? q[(size_t)r * ldq + k] * kMlpInvPi : 0.f);
}

// Interpolated waypoints of each motion as MLP input rows (row m * W + i).
template <class T>
__global__ void mlp_interp_input_kernel(const float* __restrict__ q0, const float* __restrict__ q1,
                                        int n, int W, int dof, int in, T* X) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * W * in) return;
  const int r = i / in, k = i - r * in;
  const int m = r / W, w = r - m * W;
  float v = 0.f;
  if (k < dof) {
    const float a = q0[(size_t)m * dof + k], b = q1[(size_t)m * dof + k];
    v = fmaf((float)w / (float)(W - 1), b - a, a) * kMlpInvPi;
  }
  X[i] = to_act<T>(v);
}

// dY = (Y - T) / rows on the dof used outputs (zero on padding), and the loss 0.5 |Y-T|^2 / rows.
template <class A>
__global__ void mse_grad_kernel(const float* __restrict__ Y, int ldy, const float* __restrict__ T,
                                int ldt, int rows, int dof, int out, A* dY, float* loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < rows * out) {
    const int r = i / out, k = i - r * out;
    float d = 0.f;
    if (k < dof) {
      d = Y[(size_t)r * ldy + k] - T[(size_t)r * ldt + k];
      l = 0.5f * d * d / (float)rows;
    }
    dY[i] = to_act<A>(d / (float)rows);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
}

// db[n] = sum_r D[r][n]  (D [rows][ld])
template <class T>
__global__ void bias_grad_kernel(const T* __restrict__ D, int ld, int rows, int N, float* db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) s += act_f(D[(size_t)r * ld + n]);
  atomicAdd(&db[n], s);
}

// Adam on one tensor (FP32 master p, moments m v, gradient g), then its BF16 copies:
// wt [rows][cols] (the tensor itself) and, if w_t is set, its transpose [cols][rows].
// Entries outside [rows_used, cols_used) (padding) stay zero.
__global__ void adam_kernel(float* p, float* m, float* v, const float* g, int rows, int cols,
                            int rows_used, int cols_used, float lr, float b1, float b2, float eps,
                            float c1, float c2, __nv_bfloat16* wt, __nv_bfloat16* w_t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int r = i / cols, c = i - r * cols;
  float x = 0.f;
  if (r < rows_used && c < cols_used) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    x = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = x;
  }
  if (wt) wt[i] = __float2bfloat16(x);
  if (w_t) w_t[(size_t)c * rows + r] = __float2bfloat16(x);
}

// BF16 copies of an FP32 tensor [rows][cols] (and of its transpose).
__global__ void to_bf16_kernel(const float* p, int rows, int cols, __nv_bfloat16* wt,
                               __nv_bfloat16* w_t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int r = i / cols, c = i - r * cols;
  if (wt) wt[i] = __float2bfloat16(p[i]);
  if (w_t) w_t[(size_t)c * rows + r] = __float2bfloat16(p[i]);
}

// T[r][k] = t[r][k] - q[r][k] (k < dof), zero padding to 16.
__global__ void residual_target_kernel(const float* __restrict__ q, const float* __restrict__ t, int rows,
                                       int dof, float* T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * kMlpIO) return;
  const int r = i / kMlpIO, k = i - r * kMlpIO;
  T[i] = k < dof ? t[(size_t)r * dof + k] - q[(size_t)r * dof + k] : 0.f;
}

__global__ void accumulate_kernel(float* dst, const float* src) { *dst += *src; }

cudaError_t launch_residual_target(const float* q, const float* t, int rows, int dof, float* T,
                                   cudaStream_t s) {
  const int n = rows * kMlpIO;
  if (n <= 0) return cudaSuccess;
  residual_target_kernel<<<(n + 255) / 256, 256, 0, s>>>(q, t, rows, dof, T);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(float* dst, const float* src, cudaStream_t s) {
  accumulate_kernel<<<1, 1, 0, s>>>(dst, src);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_mlp_input(const float* q, int ldq, int rows, int dof, int in, T* X, cudaStream_t s) {
  const int n = rows * in;
  if (n <= 0) return cudaSuccess;
  mlp_input_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(q, ldq, rows, dof, in, X);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_mlp_interp_input(const float* q0, const float* q1, int n, int W, int dof, int in, T* X,
                                    cudaStream_t s) {
  const long long tot = (long long)n * W * in;
  if (tot <= 0) return cudaSuccess;
  mlp_interp_input_kernel<T><<<(int)((tot + 255) / 256), 256, 0, s>>>(q0, q1, n, W, dof, in, X);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_mse_grad(const float* Y, int ldy, const float* Tg, int ldt, int rows, int dof, int out,
                            T* dY, float* loss, cudaStream_t s) {
  const int n = rows * out;
  if (n <= 0) return cudaSuccess;
  mse_grad_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(Y, ldy, Tg, ldt, rows, dof, out, dY, loss);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_bias_grad(const T* D, int ld, int rows, int N, float* db, cudaStream_t s) {
  if (rows <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + 127) / 128, std::min(rows, 256));
  bias_grad_kernel<T><<<grid, 128, 0, s>>>(D, ld, rows, N, db);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, float* m, float* v, const float* g, int rows, int cols, int rows_used,
                        int cols_used, float lr, float b1, float b2, float eps, int step,
                        __nv_bfloat16* wt, __nv_bfloat16* w_t, cudaStream_t s) {
  const int n = rows * cols;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(p, m, v, g, rows, cols, rows_used, cols_used, lr, b1, b2,
                                              eps, c1, c2, wt, w_t);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* p, int rows, int cols, __nv_bfloat16* wt, __nv_bfloat16* w_t,
                           cudaStream_t s) {
  const int n = rows * cols;
  to_bf16_kernel<<<(n + 255) / 256, 256, 0, s>>>(p, rows, cols, wt, w_t);
  return cudaGetLastError();
}

// ---- the network and its training -----------------------------------------------------
//
// Layers l = 0..3: in_l -> out_l with in = (16, 256, 256, 256), out = (256, 256, 256, 16);
// dof inputs and outputs are used, the rest is zero padding. Parameters (FP32 master copy)
// are laid out flat as, per layer, the weight [out][in] then the bias [out].

namespace {

constexpr int kIn[kMlpLayers] = {kMlpIO, kMlpHidden, kMlpHidden, kMlpHidden};
constexpr int kOut[kMlpLayers] = {kMlpHidden, kMlpHidden, kMlpHidden, kMlpIO};

size_t w_off(int l) {
  size_t o = 0;
  for (int i = 0; i < l; ++i) o += (size_t)kOut[i] * kIn[i] + kOut[i];
  return o;
}

}  // namespace

size_t mlp_param_count() { return w_off(kMlpLayers); }

struct MlpDev {
  int dof = 0;
  int step = 0;
  float* p = nullptr;   // FP32 master parameters
  float* m = nullptr;   // Adam moments
  float* v = nullptr;
  float* g = nullptr;   // gradients
  __nv_bfloat16* wb = nullptr;  // BF16 weights [out][in] per layer (biases stay FP32)
  // BF16 transposes [in][out] of layers 0..2, for the planner's per-warp evaluation (a warp's
  // lanes read consecutive outputs of one input)
  __nv_bfloat16* wbt = nullptr;
  // fused inference: packed weight image, padded biases, timeout flag
  uint8_t* wpack = nullptr;
  float* bias_pad = nullptr;
  int* err = nullptr;
  bool packed = false;
  int sm_count = 0;
  bool fp32 = false;  // checking mode: FP32 weights and activations, unfused inference
  unsigned long long wait_ns = 0;  // bounded-wait limit of the fused kernel (0: its default)
  // workspace
  char* ws = nullptr;
  size_t ws_bytes = 0;
};

static cudaError_t ensure_ws(MlpDev* d, size_t bytes) {
  if (bytes <= d->ws_bytes) return cudaSuccess;
  if (d->ws) cudaFree(d->ws);
  d->ws = nullptr;
  d->ws_bytes = 0;
  cudaError_t e = cudaMalloc(&d->ws, bytes);
  if (e == cudaSuccess) d->ws_bytes = bytes;
  return e;
}

cudaError_t mlp_create(MlpDev** out, int dof) {
  *out = nullptr;
  MlpDev* d = new MlpDev();
  d->dof = dof;
  const size_t n = mlp_param_count();
  size_t nw = 0;
  for (int l = 0; l < kMlpLayers; ++l) nw += (size_t)kOut[l] * kIn[l];
  cudaError_t e = cudaMalloc(&d->p, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d->m, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d->v, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d->g, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d->wb, nw * 2);
  if (e == cudaSuccess) e = cudaMalloc(&d->wbt, (nw - (size_t)kOut[3] * kIn[3]) * 2);
  if (e == cudaSuccess) e = cudaMemset(d->p, 0, n * 4);
  if (e == cudaSuccess) e = cudaMemset(d->m, 0, n * 4);
  if (e == cudaSuccess) e = cudaMemset(d->v, 0, n * 4);
  if (e == cudaSuccess) e = cudaMemset(d->wb, 0, nw * 2);
  if (e == cudaSuccess) e = cudaMalloc(&d->wpack, mlp_fused_image_bytes());
  if (e == cudaSuccess) e = cudaMalloc(&d->bias_pad, (size_t)mlp_fused_bias_floats() * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d->err, 0, sizeof(int));
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    mlp_destroy(d);
    return e;
  }
  *out = d;
  return cudaSuccess;
}

void mlp_destroy(MlpDev* d) {
  if (!d) return;
  cudaFree(d->p);
  cudaFree(d->m);
  cudaFree(d->v);
  cudaFree(d->g);
  cudaFree(d->wb);
  cudaFree(d->wbt);
  cudaFree(d->ws);
  cudaFree(d->wpack);
  cudaFree(d->bias_pad);
  cudaFree(d->err);
  delete d;
}

int mlp_dof(const MlpDev* d) { return d->dof; }
void mlp_set_fp32(MlpDev* d, bool on) { d->fp32 = on; }

void mlp_set_wait_ns(MlpDev* d, unsigned long long ns) { d->wait_ns = ns; }
bool mlp_fp32(const MlpDev* d) { return d->fp32; }
const int* mlp_error_flag(const MlpDev* d) { return d->err; }
int mlp_step(const MlpDev* d) { return d->step; }

static __nv_bfloat16* wbt_of(MlpDev* d, int l) {  // layers 0..2
  size_t o = 0;
  for (int i = 0; i < l; ++i) o += (size_t)kOut[i] * kIn[i];
  return d->wbt + o;
}

static __nv_bfloat16* wb_of(MlpDev* d, int l) {
  size_t o = 0;
  for (int i = 0; i < l; ++i) o += (size_t)kOut[i] * kIn[i];
  return d->wb + o;
}

MlpView mlp_view(MlpDev* d) {
  MlpView v{};
  for (int l = 0; l < kMlpLayers - 1; ++l) v.wt[l] = wbt_of(d, l);
  v.w3 = wb_of(d, kMlpLayers - 1);
  for (int l = 0; l < kMlpLayers; ++l) v.b[l] = d->p + w_off(l) + (size_t)kOut[l] * kIn[l];
  v.dof = d->dof;
  return v;
}

// Refreshes the BF16 weight copies from the FP32 master parameters.
static cudaError_t refresh_bf16(MlpDev* d, cudaStream_t s) {
  d->packed = false;
  for (int l = 0; l < kMlpLayers; ++l) {
    cudaError_t e = launch_to_bf16(d->p + w_off(l), kOut[l], kIn[l], wb_of(d, l),
                                   l < kMlpLayers - 1 ? wbt_of(d, l) : nullptr, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Public (compact) layout for a robot with dof joints: per layer l, W_l [out_l][in_l] then
// b_l [out_l], with in = (dof, 256, 256, 256) and out = (256, 256, 256, dof).
size_t mlp_compact_count(int dof) {
  return (size_t)kMlpHidden * dof + kMlpHidden + 2 * ((size_t)kMlpHidden * kMlpHidden + kMlpHidden) +
         (size_t)dof * kMlpHidden + dof;
}

static void compact_dims(int dof, int l, int& rows, int& cols) {
  rows = l == kMlpLayers - 1 ? dof : kOut[l];
  cols = l == 0 ? dof : kIn[l];
}

// The padded device layout of a host array in the compact layout (padding zero).
static std::vector<float> from_compact(const MlpDev* d, const float* host) {
  std::vector<float> p(mlp_param_count(), 0.f);
  const float* src = host;
  for (int l = 0; l < kMlpLayers; ++l) {
    int rows, cols;
    compact_dims(d->dof, l, rows, cols);
    float* w = p.data() + w_off(l);
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) w[(size_t)r * kIn[l] + c] = *src++;
    float* b = w + (size_t)kOut[l] * kIn[l];
    for (int r = 0; r < rows; ++r) b[r] = *src++;
  }
  return p;
}

// Sets parameters, Adam moments (null: zero) and step from host arrays in the compact layout.
static cudaError_t set_state(MlpDev* d, const float* params, const float* m, const float* v, int step,
                             cudaStream_t s) {
  const size_t n = mlp_param_count();
  const std::vector<float> p = from_compact(d, params);
  cudaError_t e = cudaMemcpyAsync(d->p, p.data(), n * 4, cudaMemcpyHostToDevice, s);
  std::vector<float> mm, vv;
  if (e == cudaSuccess) {
    if (m) {
      mm = from_compact(d, m);
      e = cudaMemcpyAsync(d->m, mm.data(), n * 4, cudaMemcpyHostToDevice, s);
    } else {
      e = cudaMemsetAsync(d->m, 0, n * 4, s);
    }
  }
  if (e == cudaSuccess) {
    if (v) {
      vv = from_compact(d, v);
      e = cudaMemcpyAsync(d->v, vv.data(), n * 4, cudaMemcpyHostToDevice, s);
    } else {
      e = cudaMemsetAsync(d->v, 0, n * 4, s);
    }
  }
  if (e == cudaSuccess) e = refresh_bf16(d, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors must outlive the copies
  d->step = step;
  return e;
}

// Sets the parameters from a host array in the compact layout (padding stays zero) and
// resets the optimiser state.
cudaError_t mlp_set_params(MlpDev* d, const float* host, cudaStream_t s) {
  return set_state(d, host, nullptr, nullptr, 0, s);
}

cudaError_t mlp_set_state(MlpDev* d, const float* params, const float* m, const float* v, int step,
                          cudaStream_t s) {
  return set_state(d, params, m, v, step, s);
}

// Copies a padded device parameter-shaped array (parameters or gradients) to a host array
// in the compact layout.
static cudaError_t to_compact(MlpDev* d, const float* dev, float* host, cudaStream_t s) {
  std::vector<float> p(mlp_param_count());
  cudaError_t e = cudaMemcpyAsync(p.data(), dev, p.size() * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  float* dst = host;
  for (int l = 0; l < kMlpLayers; ++l) {
    int rows, cols;
    compact_dims(d->dof, l, rows, cols);
    const float* w = p.data() + w_off(l);
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) *dst++ = w[(size_t)r * kIn[l] + c];
    const float* b = w + (size_t)kOut[l] * kIn[l];
    for (int r = 0; r < rows; ++r) *dst++ = b[r];
  }
  return cudaSuccess;
}

cudaError_t mlp_get_params(MlpDev* d, float* host, cudaStream_t s) { return to_compact(d, d->p, host, s); }

cudaError_t mlp_get_state(MlpDev* d, float* params, float* m, float* v, int* step, cudaStream_t s) {
  cudaError_t e = to_compact(d, d->p, params, s);
  if (e == cudaSuccess) e = to_compact(d, d->m, m, s);
  if (e == cudaSuccess) e = to_compact(d, d->v, v, s);
  *step = d->step;
  return e;
}

// He-normal weights (the last layer scaled by 0.1: the corrections it predicts are small),
// zero biases; Gaussian draws from a splitmix64 stream with the Box-Muller transform.
cudaError_t mlp_init(MlpDev* d, uint64_t seed, cudaStream_t s) {
  std::vector<float> p(mlp_compact_count(d->dof), 0.f);
  uint64_t st = seed * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull;
  auto next = [&]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto normal = [&]() {
    const double u1 = ((next() >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (next() >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  float* w = p.data();
  for (int l = 0; l < kMlpLayers; ++l) {
    int rows, cols;
    compact_dims(d->dof, l, rows, cols);
    const double sd = std::sqrt(2.0 / cols) * (l == kMlpLayers - 1 ? 0.1 : 1.0);
    for (size_t i = 0; i < (size_t)rows * cols; ++i) *w++ = (float)(sd * normal());
    w += rows;  // zero biases
  }
  return mlp_set_params(d, p.data(), s);
}

// Workspace layout for `rows` rows: X (16) | H ping-pong (256 x 2) | Z x 3 (f32 256, training
// only) | Y (f32 16) | dY (16) | dZ ping-pong (256 x 2) | loss (f32); X, H, dY and dZ in the
// activation type T (BF16, or FP32 in the checking mode).
template <class T>
struct MlpWs {
  T *X, *H[2], *dY, *dZ[2];
  float *Z[3], *Y, *loss;
};

template <class T>
static size_t ws_layout(char* base, int rows, bool train, MlpWs<T>* w) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + o : nullptr;
    o += (bytes + 255) & ~size_t(255);
    return p;
  };
  const size_t R = (size_t)rows, e = sizeof(T);
  w->X = (T*)take(R * kMlpIO * e);
  w->H[0] = (T*)take(R * kMlpHidden * e);
  w->H[1] = (T*)take(R * kMlpHidden * e);
  for (int i = 0; i < 3; ++i) w->Z[i] = train ? (float*)take(R * kMlpHidden * 4) : nullptr;
  w->Y = (float*)take(R * kMlpIO * 4);
  w->dY = train ? (T*)take(R * kMlpIO * e) : nullptr;
  w->dZ[0] = train ? (T*)take(R * kMlpHidden * e) : nullptr;
  w->dZ[1] = train ? (T*)take(R * kMlpHidden * e) : nullptr;
  w->loss = (float*)take(4);
  return o;
}

// Layer l's weight [out][in] in the arithmetic's type: the BF16 copy, or the FP32 master.
template <class T>
static const T* weights_of(MlpDev* d, int l);
template <>
const __nv_bfloat16* weights_of<__nv_bfloat16>(MlpDev* d, int l) { return wb_of(d, l); }
template <>
const float* weights_of<float>(MlpDev* d, int l) { return d->p + w_off(l); }

// Forward pass of rows of X already in w.X; Y (FP32 [rows][16], `y` or else w.Y) =
// corrections. In training mode the activations H_l (kept in a 3-deep set for the backward)
// and Z_l are stored.
template <class T>
static cudaError_t forward(MlpDev* d, const MlpWs<T>& w, int rows, T* Hkeep[3], float* y,
                           cudaStream_t s) {
  const T* in = w.X;
  int ld_in = kMlpIO;
  for (int l = 0; l < kMlpLayers; ++l) {
    GemmArgsT<T> g{};
    g.error = d->err;
    g.wait_ns = d->wait_ns;
    g.M = rows;
    g.N = kOut[l];
    g.K = kIn[l];
    g.A = in;
    g.lda = ld_in;
    g.transA = 0;
    g.B = weights_of<T>(d, l);  // [out][in] = [N][K]
    g.ldb = kIn[l];
    g.transB = 1;
    g.bias = d->p + w_off(l) + (size_t)kOut[l] * kIn[l];
    cudaError_t e;
    if (l < kMlpLayers - 1) {
      T* out = Hkeep ? Hkeep[l] : w.H[l & 1];
      g.C = w.Z[0] && Hkeep ? w.Z[l] : nullptr;
      g.ldc = kMlpHidden;
      g.H = out;
      g.ldh = kMlpHidden;
      e = launch_gemm(kEpiBiasGelu, g, s);
      in = out;
      ld_in = kMlpHidden;
    } else {
      g.C = y ? y : w.Y;
      g.ldc = kMlpIO;
      e = launch_gemm(kEpiBias, g, s);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Packs the current weights for the fused kernel when they changed since the last pack.
static cudaError_t ensure_packed(MlpDev* d, cudaStream_t s) {
  if (d->packed) return cudaSuccess;
  cudaError_t e = launch_mlp_pack(wb_of(d, 0), wb_of(d, 1), wb_of(d, 2), wb_of(d, 3), d->wpack, s);
  for (int l = 0; l < kMlpLayers && e == cudaSuccess; ++l)
    e = cudaMemcpyAsync(d->bias_pad + 256 * l, d->p + w_off(l) + (size_t)kOut[l] * kIn[l],
                        (size_t)kOut[l] * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) d->packed = true;
  return e;
}

static cudaError_t run_fused(MlpDev* d, FusedMlpArgs a, cudaStream_t s) {
  cudaError_t e = ensure_packed(d, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d->err, 0, sizeof(int), s);
  a.dof = d->dof;
  a.wpack = d->wpack;
  a.bias = d->bias_pad;
  a.error = d->err;
  a.wait_ns = d->wait_ns;
  if (e == cudaSuccess) e = launch_mlp_fused(a, d->sm_count, s);
  return e;
}

// The checking mode's inference: the unfused FP32 forward pass on rows of q (or of the
// interpolated motions when q0 is set) into Y [rows][16].
static cudaError_t infer_f32(MlpDev* d, const float* q, int ldq, const float* q0, const float* q1, int W,
                             int rows, float* Y, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  MlpWs<float> w;
  cudaError_t e = ensure_ws(d, ws_layout<float>(nullptr, rows, false, &w));
  if (e != cudaSuccess) return e;
  ws_layout<float>(d->ws, rows, false, &w);
  e = q0 ? launch_mlp_interp_input<float>(q0, q1, rows / W, W, d->dof, kMlpIO, w.X, s)
         : launch_mlp_input<float>(q, ldq, rows, d->dof, kMlpIO, w.X, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d->err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = forward<float>(d, w, rows, nullptr, Y, s);
  return e;
}

// Inference: corrections Y [rows][16] for rows of q ([rows][ldq], first dof used).
cudaError_t mlp_infer(MlpDev* d, const float* q, int ldq, int rows, float* Y, cudaStream_t s) {
  if (d->fp32) return infer_f32(d, q, ldq, nullptr, nullptr, 1, rows, Y, s);
  FusedMlpArgs a{};
  a.q = q;
  a.ldq = ldq;
  a.rows = rows;
  a.out = Y;
  return run_fused(d, a, s);
}

// Inference on the interpolated waypoints of n motions (row m * W + i) into Y [n*W][16].
cudaError_t mlp_infer_motions(MlpDev* d, const float* q0, const float* q1, int n, int W, float* Y,
                              cudaStream_t s) {
  if (d->fp32) return infer_f32(d, nullptr, 0, q0, q1, W, n * W, Y, s);
  FusedMlpArgs a{};
  a.q0 = q0;
  a.q1 = q1;
  a.W = W;
  a.rows = n * W;
  a.out = Y;
  return run_fused(d, a, s);
}

// Loss 0.5 |MLP(q) - (t - q)|^2 averaged over rows and its gradient into d->g.
// q, t: [rows][dof] device arrays. *loss_dev (device float) receives the loss.
template <class T>
static cudaError_t loss_and_grad(MlpDev* d, const float* q, const float* t, int rows, cudaStream_t s,
                                 MlpWs<T>& w) {
  const size_t need = ws_layout<T>(nullptr, rows, true, &w) + (size_t)rows * kMlpIO * 4;
  cudaError_t e = ensure_ws(d, need);
  if (e != cudaSuccess) return e;
  const size_t used = ws_layout<T>(d->ws, rows, true, &w);
  float* target = reinterpret_cast<float*>(d->ws + used);  // t - q, [rows][16]
  e = launch_mlp_input<T>(q, d->dof, rows, d->dof, kMlpIO, w.X, s);
  if (e != cudaSuccess) return e;
  e = launch_residual_target(q, t, rows, d->dof, target, s);
  if (e != cudaSuccess) return e;
  T* H[3] = {w.H[0], w.H[1], w.dZ[1]};  // three stored activations
  // a third activation buffer: reuse dZ[1] for H3 during the forward; the backward below
  // writes dZ only into buffers whose activation is no longer needed
  e = forward<T>(d, w, rows, H, nullptr, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(w.loss, 0, 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d->g, 0, mlp_param_count() * 4, s);
  if (e == cudaSuccess)
    e = launch_mse_grad<T>(w.Y, kMlpIO, target, kMlpIO, rows, d->dof, kMlpIO, w.dY, w.loss, s);
  if (e != cudaSuccess) return e;
  // backward, layer 3 .. 0: D_l = dL/dZ_l (BF16), previous activation A_{l} = H[l-1] or X
  const T* D = w.dY;
  int ldD = kMlpIO;
  T* dz_out[3] = {w.dZ[0], w.H[1], w.dZ[0]};  // dZ_2 -> dZ[0], dZ_1 -> H[1], dZ_0 -> dZ[0]
  for (int l = kMlpLayers - 1; l >= 0; --l) {
    const T* Aprev = l == 0 ? w.X : H[l - 1];
    const int ldA = l == 0 ? kMlpIO : kMlpHidden;
    // weight gradient dW_l [out][in] = D^T Aprev  (split-K over rows, atomics)
    GemmArgsT<T> gw{};
    gw.error = d->err;
    gw.wait_ns = d->wait_ns;
    gw.M = kOut[l];
    gw.N = kIn[l];
    gw.K = rows;
    gw.A = D;
    gw.lda = ldD;
    gw.transA = 1;  // D is [rows][out] = [K][M]
    gw.B = Aprev;
    gw.ldb = ldA;
    gw.transB = 0;  // Aprev is [rows][in] = [K][N]
    gw.C = d->g + w_off(l);
    gw.ldc = kIn[l];
    e = launch_gemm(kEpiAtomic, gw, s);
    if (e == cudaSuccess)
      e = launch_bias_grad<T>(D, ldD, rows, kOut[l], d->g + w_off(l) + (size_t)kOut[l] * kIn[l], s);
    if (e != cudaSuccess) return e;
    if (l == 0) break;
    // dZ_{l-1} = (D W_l) * gelu'(Z_{l-1})
    GemmArgsT<T> gd{};
    gd.error = d->err;
    gd.wait_ns = d->wait_ns;
    gd.M = rows;
    gd.N = kIn[l];
    gd.K = kOut[l];
    gd.A = D;
    gd.lda = ldD;
    gd.transA = 0;
    gd.B = weights_of<T>(d, l);  // [out][in] = [K][N]
    gd.ldb = kIn[l];
    gd.transB = 0;
    gd.Z = w.Z[l - 1];
    gd.ldc = kMlpHidden;
    gd.H = dz_out[l - 1];
    gd.ldh = kMlpHidden;
    e = launch_gemm(kEpiGeluBwd, gd, s);
    if (e != cudaSuccess) return e;
    D = dz_out[l - 1];
    ldD = kMlpHidden;
  }
  return cudaSuccess;
}

// After the stream synchronised: cudaErrorTimeout when a tensor-core GEMM gave up a wait.
static cudaError_t gemm_status(MlpDev* d) {
  int flag = 0;
  const cudaError_t e = cudaMemcpy(&flag, d->err, sizeof(int), cudaMemcpyDeviceToHost);
  return e != cudaSuccess ? e : flag ? cudaErrorTimeout : cudaSuccess;
}

cudaError_t mlp_grad(MlpDev* d, const float* q, const float* t, int rows, float* grads_host,
                     float* loss_host, cudaStream_t s) {
  float* loss_dev = nullptr;
  cudaError_t e = cudaMemsetAsync(d->err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (d->fp32) {
    MlpWs<float> w;
    e = loss_and_grad<float>(d, q, t, rows, s, w);
    loss_dev = w.loss;
  } else {
    MlpWs<__nv_bfloat16> w;
    e = loss_and_grad<__nv_bfloat16>(d, q, t, rows, s, w);
    loss_dev = w.loss;
  }
  if (e == cudaSuccess && loss_host) e = cudaMemcpyAsync(loss_host, loss_dev, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = gemm_status(d);
  if (e == cudaSuccess && grads_host) e = to_compact(d, d->g, grads_host, s);
  return e;
}

// One Adam step on the batch; the batch loss is added to *loss_dev (device) if given.
cudaError_t mlp_train_step(MlpDev* d, const float* q, const float* t, int rows, float lr,
                           float* loss_dev, cudaStream_t s) {
  float* batch_loss = nullptr;
  cudaError_t e;
  if (d->fp32) {
    MlpWs<float> w;
    e = loss_and_grad<float>(d, q, t, rows, s, w);
    batch_loss = w.loss;
  } else {
    MlpWs<__nv_bfloat16> w;
    e = loss_and_grad<__nv_bfloat16>(d, q, t, rows, s, w);
    batch_loss = w.loss;
  }
  if (e != cudaSuccess) return e;
  d->step++;
  for (int l = 0; l < kMlpLayers; ++l) {
    const int rows_used = l == kMlpLayers - 1 ? d->dof : kOut[l];
    const int cols_used = l == 0 ? d->dof : kIn[l];
    const size_t o = w_off(l);
    e = launch_adam(d->p + o, d->m + o, d->v + o, d->g + o, kOut[l], kIn[l], rows_used, cols_used, lr,
                    0.9f, 0.999f, 1e-8f, d->step, wb_of(d, l),
                    l < kMlpLayers - 1 ? wbt_of(d, l) : nullptr, s);
    if (e == cudaSuccess) {
      const size_t ob = o + (size_t)kOut[l] * kIn[l];
      e = launch_adam(d->p + ob, d->m + ob, d->v + ob, d->g + ob, 1, kOut[l], 1, rows_used, lr, 0.9f,
                      0.999f, 1e-8f, d->step, nullptr, nullptr, s);
    }
    if (e != cudaSuccess) return e;
  }
  if (loss_dev) e = launch_accumulate(loss_dev, batch_loss, s);
  return e;
}

// rows of q and t picked by idx into contiguous batch arrays
__global__ void gather_rows_kernel(const float* __restrict__ q, const float* __restrict__ t,
                                   const int* __restrict__ idx, int rows, int dof, float* qb, float* tb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * dof) return;
  const int r = i / dof, k = i - r * dof;
  const size_t src = (size_t)idx[r] * dof + k;
  qb[i] = q[src];
  tb[i] = t[src];
}

// Epochs of minibatch Adam over n pairs (q, t) in device memory, in an order drawn per epoch
// (Fisher-Yates over a splitmix64 stream). loss_host[epoch] (optional) = mean batch loss.
cudaError_t mlp_train(MlpDev* d, const float* q, const float* t, int n, int batch, int epochs,
                      float lr, uint64_t seed, float* loss_host, cudaStream_t s) {
  const int dof = d->dof;
  const int nb = n / batch;  // full batches only
  if (nb < 1) return cudaErrorInvalidValue;
  int* idx = nullptr;
  float *qb = nullptr, *tb = nullptr, *loss = nullptr;
  cudaError_t e = cudaMalloc(&idx, (size_t)n * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&qb, (size_t)batch * dof * 4);
  if (e == cudaSuccess) e = cudaMalloc(&tb, (size_t)batch * dof * 4);
  if (e == cudaSuccess) e = cudaMalloc(&loss, (size_t)std::max(epochs, 1) * 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, (size_t)std::max(epochs, 1) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d->err, 0, sizeof(int), s);
  std::vector<int> perm(n);
  for (int i = 0; i < n; ++i) perm[i] = i;
  uint64_t st = seed ^ 0xD1B54A32D192ED03ull;
  auto next = [&]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (int i = n - 1; i > 0; --i) std::swap(perm[i], perm[(int)(next() % (uint64_t)(i + 1))]);
    e = cudaMemcpyAsync(idx, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, s);
    // the host order must not change while the copy is in flight
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
      const int tot = batch * dof;
      gather_rows_kernel<<<(tot + 255) / 256, 256, 0, s>>>(q, t, idx + (size_t)b * batch, batch, dof, qb, tb);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = mlp_train_step(d, qb, tb, batch, lr, loss + ep, s);
    }
  }
  if (e == cudaSuccess && loss_host) {
    std::vector<float> l(std::max(epochs, 1));
    e = cudaMemcpyAsync(l.data(), loss, l.size() * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int ep = 0; ep < epochs; ++ep) loss_host[ep] = l[ep] / nb;
  }
  cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = gemm_status(d);
  cudaFree(idx);
  cudaFree(qb);
  cudaFree(tb);
  cudaFree(loss);
  return e;
}

}  // namespace cprrtc
