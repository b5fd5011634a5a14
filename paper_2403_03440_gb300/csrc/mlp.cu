// Chemistry surrogate network on the 5th-generation tensor cores (no counterpart in the paper:
// a 14-128-128-128-22 multilayer perceptron that stands in for the Arrhenius source and
// Jacobian-diagonal evaluation of Sec. 2.1 / Sec. 2.3.2 inside the implicit operator only).
//
// Every matrix product is one tile GEMM, C = A B^T with A [M][K] and B [N][K] in bfloat16
// (K contiguous), accumulated in FP32 in tensor memory: a CTA of 4 warps owns 128 rows of C,
// stages K in chunks of 64 columns into shared memory in the canonical K-major layout without
// swizzle (8-row x 16-byte core matrices), one thread issues tcgen05.mma (M = 128, N <= 256,
// K = 16 per instruction), tcgen05.commit signals an mbarrier, and each warp reads its 32
// accumulator lanes back with tcgen05.ld for the epilogue.  Weight gradients reduce over the
// batch (K = samples) split across CTAs and added atomically.  Forward, backward, Adam and the
// solver coupling (features in, species Jacobian diagonal out) are small kernels around it.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "../../include/cs.h"

namespace csmlp {

using bf16 = __nv_bfloat16;

constexpr int kThreads = 128;            // 4 warps, one tensor-memory lane quarter each
constexpr int kTileM = 128;              // rows of C per CTA (MMA M)
constexpr int kChunkK = 64;              // K columns staged per step (4 MMAs of K = 16)
constexpr int kMaxN = 256;
constexpr long kSpinLimit = 1L << 22;    // bounded mbarrier waits
// shared memory: A chunk, B chunk, then slack so that every address an MMA forms from these
// descriptors stays inside the allocation, then the mbarrier and the tensor-memory address
constexpr int kSmemA = kTileM * kChunkK * 2;
constexpr int kSmemB = kMaxN * kChunkK * 2;
constexpr int kSmemSlack = 48 * 1024;
constexpr int kSmemBytes = kSmemA + kSmemB + kSmemSlack + 64;

enum { EPI_STORE = 0, EPI_SILU = 1, EPI_ATOMIC = 2 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of tcgen05: start address, leading-dimension byte offset
// (between core matrices adjacent in K), stride-dimension byte offset (between core matrices
// adjacent in M/N), all in units of 16 bytes; descriptor version 1; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of tcgen05.mma.kind::f16: D FP32, A and B bfloat16, both K-major,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t phase) {
  for (long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(bar), "r"(phase) : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t ta, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t ta, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// C (+)= A[M][K] B[N][K]^T for the 128 rows of this CTA and the K range of blockIdx.y
// (klen columns each).  M is a multiple of 128, N a multiple of 16 in [16, 256], K and klen
// multiples of 16.  Epilogues: EPI_STORE C = acc (+ bias); EPI_SILU Z = acc + bias into C and
// bf16(silu(Z)) into Cb (and transposed into CbT when given); EPI_ATOMIC C += acc.
template <int EPI>
__global__ void __launch_bounds__(kThreads) k_gemm(const bf16* __restrict__ A, int lda,
                                                   const bf16* __restrict__ B, int ldb, int N, int K,
                                                   int klen, const float* __restrict__ bias, float* C,
                                                   int ldc, bf16* Cb, int ldcb, bf16* CbT, int ldt,
                                                   int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* sA = smem;
  unsigned char* sB = smem + kSmemA;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kSmemA + kSmemB + kSmemSlack);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * kTileM;
  const int kbeg = blockIdx.y * klen;
  const int kend = min(K, kbeg + klen);
  const uint32_t ncols = N <= 32 ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u));
  const uint32_t barA = smem_u32(bar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 ::"r"(smem_u32(tslot)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(barA) : "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = instr_desc(kTileM, N);
  uint32_t phase = 0;
  bool failed = false;
  for (int k0 = kbeg; k0 < kend; k0 += kChunkK) {
    const int kc = min(kChunkK, kend - k0);
    const int c8n = kc / 8;
    // stage the chunk: element (r, k) at core matrix (k/8, r/8), row r%8, column k%8
    for (int v = tid; v < kTileM * c8n; v += kThreads) {
      const int r = v / c8n, c8 = v - r * c8n;
      const uint4 x = *reinterpret_cast<const uint4*>(A + (size_t)(row0 + r) * lda + k0 + c8 * 8);
      *reinterpret_cast<uint4*>(sA + (c8 * (kTileM / 8) + (r >> 3)) * 128 + (r & 7) * 16) = x;
    }
    for (int v = tid; v < N * c8n; v += kThreads) {
      const int r = v / c8n, c8 = v - r * c8n;
      const uint4 x = *reinterpret_cast<const uint4*>(B + (size_t)r * ldb + k0 + c8 * 8);
      *reinterpret_cast<uint4*>(sB + (c8 * (N / 8) + (r >> 3)) * 128 + (r & 7) * 16) = x;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      for (int j = 0; j < kc / 16; ++j) {
        const uint64_t ad = smem_desc(a0 + 2 * j * (kTileM / 8) * 128, (kTileM / 8) * 128, 128);
        const uint64_t bd = smem_desc(b0 + 2 * j * (N / 8) * 128, (N / 8) * 128, 128);
        const uint32_t acc = (k0 > kbeg || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                   ::"r"(barA) : "memory");
    }
    // the MMAs read the staged chunk: wait for them before staging the next one
    const bool ok = wait_parity(barA, phase);
    phase ^= 1;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
  } else if (kend > kbeg) {
    const int r = row0 + warp * 32 + lane;
    for (int c0 = 0; c0 < N; c0 += 32) {
      float v[32];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      const int nc = min(32, N - c0);
      if (nc == 32) tmem_ld32(ta, v);
      else tmem_ld16(ta, v);
      for (int i = 0; i < nc; ++i) {
        const int n = c0 + i;
        if (EPI == EPI_ATOMIC) {
          atomicAdd(&C[(size_t)r * ldc + n], v[i]);
        } else {
          const float z = v[i] + (bias ? bias[n] : 0.f);
          C[(size_t)r * ldc + n] = z;
          if (EPI == EPI_SILU) {
            const bf16 h = __float2bfloat16_rn(z / (1.f + __expf(-z)));
            Cb[(size_t)r * ldcb + n] = h;
            if (CbT) CbT[(size_t)n * ldt + r] = h;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
}

// Layer sizes (the flat FP32 parameter layout is described with the elementwise kernels below).
constexpr int LNH = CS_MLP_HIDDEN, LKIN = 16, LNOUTP = 32;

// Fused inference: the whole network on 128-row tiles of a persistent grid.  Each CTA stages
// the bfloat16 weights and the biases into shared memory once (canonical K-major layout,
// 76 KB + 1.6 KB), then per tile: inputs -> bf16 tile, and for each layer one tcgen05.mma group
// into tensor memory, tcgen05.ld, bias (+ SiLU), bf16 back into shared memory as the next
// layer's A operand; the last layer's FP32 outputs go to Y [n][22].  No activation leaves the
// SM.  8 warps: warp w reads tensor-memory lanes 32 (w % 4) .. +31 (the rows it may access)
// and columns 64 (w / 4) .. +63 of the accumulator.  The input tile lives in the first 4 KB of
// the activation tile: layer 1's MMA has completed (mbarrier) before its epilogue overwrites
// it, and the next tile's inputs are written after layer 4's MMA has completed.  Two CTAs fit
// on an SM (shared memory), so one CTA's MMAs overlap the other's epilogue.
constexpr int kFuseThreads = 256;
constexpr int kFuseSmemW = (LNH * LKIN + 2 * LNH * LNH + LNOUTP * LNH) * 2;   // 77824 B
constexpr int kFuseSmemA = kTileM * LNH * 2;                                   // 32768 B
constexpr int kFuseSmemB = (3 * LNH + LNOUTP) * 4;                             // 1664 B
constexpr int kFuseSmemBytes = kFuseSmemW + kFuseSmemA + kFuseSmemB + 64;
static_assert(kTileM * LKIN * 2 <= kFuseSmemA, "input tile inside the activation tile");
static_assert(2 * (kFuseSmemBytes + 1024) <= 228 * 1024, "two CTAs per SM");

// stage rows [0, rows) x [0, K) of a row-major bf16 matrix into the canonical K-major layout
__device__ __forceinline__ void stage_kmajor(const bf16* src, int rows, int K, unsigned char* dst) {
  const int c8n = K / 8;
  for (int v = threadIdx.x; v < rows * c8n; v += blockDim.x) {
    const int r = v / c8n, c8 = v - r * c8n;
    const uint4 x = *reinterpret_cast<const uint4*>(src + (size_t)r * K + c8 * 8);
    *reinterpret_cast<uint4*>(dst + (c8 * (rows / 8) + (r >> 3)) * 128 + (r & 7) * 16) = x;
  }
}

// one layer: D[128 x N] = A[128 x K] W[N x K]^T into tensor memory; returns false on timeout
__device__ __forceinline__ bool fused_layer(uint32_t tmem, uint32_t a0, uint32_t w0, int N, int K,
                                            uint32_t bar, uint32_t& phase) {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t idesc = instr_desc(kTileM, N);
    for (int j = 0; j < K / 16; ++j) {
      const uint64_t ad = smem_desc(a0 + 2 * j * (kTileM / 8) * 128, (kTileM / 8) * 128, 128);
      const uint64_t bd = smem_desc(w0 + 2 * j * (N / 8) * 128, (N / 8) * 128, 128);
      const uint32_t acc = j > 0 ? 1u : 0u;
      asm volatile(
          "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
          ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 ::"r"(bar) : "memory");
  }
  const bool ok = wait_parity(bar, phase);
  phase ^= 1;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  return !__syncthreads_or(!ok);
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// hidden-layer epilogue of this warp's 32 rows x 64 columns: bias + SiLU -> bf16 into the A tile
__device__ __forceinline__ void fused_hidden_epilogue(uint32_t tmem, const float* bias, unsigned char* A) {
  const int warp = threadIdx.x >> 5, q = warp & 3, h = warp >> 2;
  const int r = 32 * q + (threadIdx.x & 31);
#pragma unroll
  for (int cc = 0; cc < 2; ++cc) {
    const int c0 = 64 * h + 32 * cc;
    float v[32];
    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
#pragma unroll
    for (int g8 = 0; g8 < 4; ++g8) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int n0 = c0 + g8 * 8 + 2 * e;
        const float z0 = v[g8 * 8 + 2 * e] + bias[n0], z1 = v[g8 * 8 + 2 * e + 1] + bias[n0 + 1];
        // silu(z) = z sigma(z) = (z/2)(1 + tanh(z/2)): one special-function op per value
        // (tanh.approx, relative error ~2^-11, below the bfloat16 rounding that follows)
        const float h0 = 0.5f * z0, h1 = 0.5f * z1;
        const bf16 o0 = __float2bfloat16_rn(fmaf(h0, tanh_approx(h0), h0));
        const bf16 o1 = __float2bfloat16_rn(fmaf(h1, tanh_approx(h1), h1));
        w[e] = (uint32_t)__bfloat16_as_ushort(o0) | ((uint32_t)__bfloat16_as_ushort(o1) << 16);
      }
      const int c8 = (c0 >> 3) + g8;
      *reinterpret_cast<uint4*>(A + (c8 * (kTileM / 8) + (r >> 3)) * 128 + (r & 7) * 16) =
          make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

__global__ void __launch_bounds__(kFuseThreads) k_mlp_infer(const float* __restrict__ X, int n,
                                                            const bf16* __restrict__ W1, const bf16* __restrict__ W2,
                                                            const bf16* __restrict__ W3, const bf16* __restrict__ W4,
                                                            const float* __restrict__ b1, const float* __restrict__ b2,
                                                            const float* __restrict__ b3, const float* __restrict__ b4,
                                                            float* __restrict__ Y, int* err) {
  extern __shared__ __align__(128) unsigned char fsm[];
  unsigned char* sW1 = fsm;
  unsigned char* sW2 = sW1 + LNH * LKIN * 2;
  unsigned char* sW3 = sW2 + LNH * LNH * 2;
  unsigned char* sW4 = sW3 + LNH * LNH * 2;
  unsigned char* sA = fsm + kFuseSmemW;
  unsigned char* sX = sA;                     // the input tile aliases the activation tile
  float* sB = reinterpret_cast<float*>(sA + kFuseSmemA);   // b1 | b2 | b3 | b4 (padded to 32)
  uint64_t* bar = reinterpret_cast<uint64_t*>(sA + kFuseSmemA + kFuseSmemB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t barA = smem_u32(bar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 ::"r"(smem_u32(tslot)), "r"(128u) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(barA) : "memory");
  stage_kmajor(W1, LNH, LKIN, sW1);
  stage_kmajor(W2, LNH, LNH, sW2);
  stage_kmajor(W3, LNH, LNH, sW3);
  stage_kmajor(W4, LNOUTP, LNH, sW4);
  for (int k = tid; k < 3 * LNH + LNOUTP; k += kFuseThreads) {
    const int l = k / LNH, o = k - l * LNH;
    sB[k] = l == 0 ? b1[o] : (l == 1 ? b2[o] : (l == 2 ? b3[o] : (o < 22 ? b4[o] : 0.f)));
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t sAu = smem_u32(sA), sXu = smem_u32(sX);
  uint32_t phase = 0;
  bool failed = false;
  const int ntiles = (n + kTileM - 1) / kTileM;
  // inputs: thread (row r, half h) converts features 8h .. 8h+7 of row r (14 features and 2
  // zero columns) to bf16, one 16-byte core-matrix row of the canonical layout.  The next
  // tile's features are loaded into registers while the current tile's layers run.
  const int xr = tid & (kTileM - 1), xh = tid >> 7;
  float xin[8];
  auto load_x = [&](int tile) {
    const int gr = tile * kTileM + xr;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = 8 * xh + e;
      xin[e] = (tile < ntiles && gr < n && k < 14) ? X[(size_t)gr * 14 + k] : 0.f;
    }
  };
  load_x(blockIdx.x);
  for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int row0 = tile * kTileM;
    {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e)
        w[e] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(xin[2 * e])) |
               ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(xin[2 * e + 1])) << 16);
      *reinterpret_cast<uint4*>(sX + (xh * (kTileM / 8) + (xr >> 3)) * 128 + (xr & 7) * 16) =
          make_uint4(w[0], w[1], w[2], w[3]);
    }
    load_x(tile + gridDim.x);
    if (!fused_layer(tmem, sXu, smem_u32(sW1), LNH, LKIN, barA, phase)) { failed = true; break; }
    fused_hidden_epilogue(tmem, sB, sA);
    if (!fused_layer(tmem, sAu, smem_u32(sW2), LNH, LNH, barA, phase)) { failed = true; break; }
    fused_hidden_epilogue(tmem, sB + LNH, sA);
    if (!fused_layer(tmem, sAu, smem_u32(sW3), LNH, LNH, barA, phase)) { failed = true; break; }
    fused_hidden_epilogue(tmem, sB + 2 * LNH, sA);
    if (!fused_layer(tmem, sAu, smem_u32(sW4), LNOUTP, LNH, barA, phase)) { failed = true; break; }
    if (warp < 4) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
      const int gr = row0 + tid;
      if (gr < n)
#pragma unroll
        for (int o = 0; o < 22; ++o) Y[(size_t)gr * 22 + o] = v[o] + sB[3 * LNH + o];
    }
    // the next tile's first MMA overwrites the accumulators: every warp has read them
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
  }
  if (failed && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(128u) : "memory");
}

// ---------------------------------------------------------------------------------------
// Elementwise kernels of the network
// ---------------------------------------------------------------------------------------

// Layer sizes and the flat FP32 parameter vector: W1 [128][14], b1, W2 [128][128], b2, W3, b3,
// W4 [22][128], b4.
constexpr int NIN = CS_MLP_IN, NH = CS_MLP_HIDDEN, NOUT = CS_MLP_OUT;
constexpr int KIN = 16, NOUTP = 32;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NH, OFF_W4 = OFF_B3 + NH,
              OFF_B4 = OFF_W4 + NOUT * NH, NPARAM = OFF_B4 + NOUT;
static_assert(NPARAM == CS_MLP_NPARAM, "parameter count");

struct Weights {   // bfloat16 operands (padded) and FP32 biases (padded)
  bf16 *W1, *W2, *W3, *W4, *W2T, *W3T, *W4T;   // W1 [128][16], W4 [32][128], W4T [128][32]
  float *b1, *b2, *b3, *b4;                    // b4 [32]
};

__global__ void k_cast_params(const float* __restrict__ p, Weights w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NH * KIN) {   // W1 padded from 14 to 16 input columns
    const int o = i / KIN, k = i % KIN;
    w.W1[i] = __float2bfloat16_rn(k < NIN ? p[OFF_W1 + o * NIN + k] : 0.f);
  }
  if (i < NH * NH) {
    const int o = i / NH, k = i % NH;
    const bf16 a = __float2bfloat16_rn(p[OFF_W2 + i]), b = __float2bfloat16_rn(p[OFF_W3 + i]);
    w.W2[i] = a;
    w.W3[i] = b;
    w.W2T[k * NH + o] = a;
    w.W3T[k * NH + o] = b;
  }
  if (i < NOUTP * NH) {   // W4 padded from 22 to 32 output rows
    const int o = i / NH, k = i % NH;
    const bf16 a = __float2bfloat16_rn(o < NOUT ? p[OFF_W4 + o * NH + k] : 0.f);
    w.W4[i] = a;
    w.W4T[k * NOUTP + o] = a;
  }
  if (i < NH) {
    w.b1[i] = p[OFF_B1 + i];
    w.b2[i] = p[OFF_B2 + i];
    w.b3[i] = p[OFF_B3 + i];
  }
  if (i < NOUTP) w.b4[i] = i < NOUT ? p[OFF_B4 + i] : 0.f;
}

// inputs [n][14] FP32 -> bf16 [npad][16] (zero padding in columns and rows)
__global__ void k_pack_input(const float* __restrict__ X, int n, int npad, bf16* Xb, bf16* XbT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad * KIN) return;
  const int r = i / KIN, k = i % KIN;
  const bf16 v = __float2bfloat16_rn(r < n && k < NIN ? X[(size_t)r * NIN + k] : 0.f);
  Xb[i] = v;
  if (XbT) XbT[(size_t)k * npad + r] = v;
}

// outputs [npad][32] -> [n][22]
__global__ void k_unpack_output(const float* __restrict__ Y, int n, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * NOUT) return;
  out[i] = Y[(size_t)(i / NOUT) * NOUTP + i % NOUT];
}

// dY = 2 (Y - T) / (n * 22) for the real rows and outputs (0 elsewhere), as bf16 [npad][32]
// and transposed bf16 [128][npad] (rows >= 22 stay zero); loss partial sums in FP64
__global__ void k_loss_grad(const float* __restrict__ Y, const float* __restrict__ T, int n, int npad,
                            bf16* dZ, bf16* dZT, float* dZf, double* loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double e2 = 0.0;
  if (i < npad * NOUTP) {
    const int r = i / NOUTP, o = i % NOUTP;
    float g = 0.f;
    if (r < n && o < NOUT) {
      const float d = Y[i] - T[(size_t)r * NOUT + o];
      e2 = (double)d * (double)d;
      g = 2.f * d / (float)((double)n * NOUT);
    }
    const bf16 b = __float2bfloat16_rn(g);
    dZ[i] = b;
    dZf[i] = g;
    dZT[(size_t)o * npad + r] = b;
  }
  __shared__ double red[256];
  red[threadIdx.x] = e2;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// dZ = dH * silu'(Z) for the real rows (0 in padding rows), bf16 copies and transposed copy
__global__ void k_silu_bwd(const float* __restrict__ dH, const float* __restrict__ Z, int n, int npad,
                           bf16* dZ, bf16* dZT, float* dZf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad * NH) return;
  const int r = i / NH, o = i % NH;
  float g = 0.f;
  if (r < n) {
    const float z = Z[i];
    const float s = 1.f / (1.f + __expf(-z));
    g = dH[i] * s * (1.f + z * (1.f - s));
  }
  const bf16 b = __float2bfloat16_rn(g);
  dZ[i] = b;
  dZf[i] = g;
  dZT[(size_t)o * npad + r] = b;
}

// column sums of dZ [npad][ncol] (FP32) into db (atomic)
__global__ void k_colsum(const float* __restrict__ dZ, int npad, int ncol, float* db) {
  const int c = blockIdx.x;
  float s = 0.f;
  for (int r = threadIdx.x; r < npad; r += blockDim.x) s += dZ[(size_t)r * ncol + c];
  __shared__ float red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] = red[0];
}

// gradient buffers (padded layouts) -> flat gradient in parameter order
struct Grads {
  float *gW1, *gW2, *gW3, *gW4, *gb1, *gb2, *gb3, *gb4;   // gW1 [128][16], gW4 [128 rows][128]
};
__global__ void k_flatten_grads(Grads g, float* flat) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  float v;
  if (i < OFF_B1) v = g.gW1[(i / NIN) * KIN + i % NIN];
  else if (i < OFF_W2) v = g.gb1[i - OFF_B1];
  else if (i < OFF_B2) v = g.gW2[i - OFF_W2];
  else if (i < OFF_W3) v = g.gb2[i - OFF_B2];
  else if (i < OFF_B3) v = g.gW3[i - OFF_W3];
  else if (i < OFF_W4) v = g.gb3[i - OFF_B3];
  else if (i < OFF_B4) v = g.gW4[i - OFF_W4];
  else v = g.gb4[i - OFF_B4];
  flat[i] = v;
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 master parameters; bc1 = 1 - beta1^t,
// bc2 = 1 - beta2^t
__global__ void k_adam(float* p, const float* __restrict__ g, float* m, float* v, float lr, float bc1,
                       float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
static int blocks(long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace csmlp

using namespace csmlp;

struct cs_mlp_s {
  int max_batch = 0, npad_max = 0;
  std::vector<void*> allocs;
  float *p = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;   // FP32 [NPARAM]
  Weights w{};
  // activations [npad][...]
  bf16 *X = nullptr, *XT = nullptr, *H1 = nullptr, *H2 = nullptr, *H3 = nullptr;
  bf16 *H1T = nullptr, *H2T = nullptr, *H3T = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *Y = nullptr, *dH = nullptr, *dZf = nullptr;
  bf16 *dZ = nullptr, *dZT = nullptr;        // [npad][128], [128][npad]
  Grads g{};
  double* loss = nullptr;
  int* err = nullptr;
  double* h_loss = nullptr;
  int* h_err = nullptr;
  int step = 0;
  cudaStream_t st = nullptr;
  char msg[256] = {0};
};

static cs_status mfail(cs_mlp m, cs_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(m->msg, sizeof m->msg, fmt, ap);
  va_end(ap);
  return s;
}

template <class T>
static cudaError_t malloc0(cs_mlp m, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, n * sizeof(T));
  if (e != cudaSuccess) return e;
  m->allocs.push_back(q);
  *p = (T*)q;
  return cudaMemset(q, 0, n * sizeof(T));
}

static bool g_attr_done = false;
static cudaError_t gemm_attrs() {
  if (g_attr_done) return cudaSuccess;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_gemm<EPI_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes)) ||
      (e = cudaFuncSetAttribute(k_gemm<EPI_SILU>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes)) ||
      (e = cudaFuncSetAttribute(k_gemm<EPI_ATOMIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes)) ||
      (e = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, kFuseSmemBytes)))
    return e;
  g_attr_done = true;
  return cudaSuccess;
}

// C = A B^T (+ epilogue) over npad rows (multiple of 128); split: K ranges per CTA column
template <int EPI>
static void gemm(cs_mlp m, const bf16* A, int lda, const bf16* B, int ldb, int rows, int N, int K,
                 const float* bias, float* C, int ldc, bf16* Cb = nullptr, int ldcb = 0,
                 bf16* CbT = nullptr, int ldt = 0, int ksplit = 1) {
  const int klen = ((K / ksplit + 15) / 16) * 16;
  dim3 grid(rows / kTileM, (K + klen - 1) / klen);
  k_gemm<EPI><<<grid, kThreads, kSmemBytes, m->st>>>(A, lda, B, ldb, N, K, klen, bias, C, ldc, Cb,
                                                      ldcb, CbT, ldt, m->err);
}

// forward on the first n rows of the packed input m->X (npad rows); save = keep transposed
// activations for the weight gradients
static void forward(cs_mlp m, int npad, bool save) {
  Weights& w = m->w;
  gemm<EPI_SILU>(m, m->X, KIN, w.W1, KIN, npad, NH, KIN, w.b1, m->Z1, NH, m->H1, NH, save ? m->H1T : nullptr, npad);
  gemm<EPI_SILU>(m, m->H1, NH, w.W2, NH, npad, NH, NH, w.b2, m->Z2, NH, m->H2, NH, save ? m->H2T : nullptr, npad);
  gemm<EPI_SILU>(m, m->H2, NH, w.W3, NH, npad, NH, NH, w.b3, m->Z3, NH, m->H3, NH, save ? m->H3T : nullptr, npad);
  gemm<EPI_STORE>(m, m->H3, NH, w.W4, NH, npad, NOUTP, NH, w.b4, m->Y, NOUTP);
}

static int g_num_sms = 0;
static void infer(cs_mlp m, const float* X, int n, float* Y, cudaStream_t st) {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms < 1) g_num_sms = 1;
  }
  const int ntiles = (n + kTileM - 1) / kTileM;
  const int grid = ntiles < 2 * g_num_sms ? ntiles : 2 * g_num_sms;
  const Weights& w = m->w;
  k_mlp_infer<<<grid, kFuseThreads, kFuseSmemBytes, st>>>(X, n, w.W1, w.W2, w.W3, w.W4, w.b1, w.b2,
                                                      w.b3, w.b4, Y, m->err);
}
static cs_status check_err(cs_mlp m, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mfail(m, CS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  if (cudaMemcpyAsync(m->h_err, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
      cudaMemcpyAsync(m->h_loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
      cudaStreamSynchronize(m->st) != cudaSuccess)
    return mfail(m, CS_ERR_CUDA, "%s: synchronise", what);
  if (*m->h_err) return mfail(m, CS_ERR_TIMEOUT, "%s: tensor-core wait timed out", what);
  return CS_OK;
}

// loss and flat gradient of a batch already packed into m->X (n real rows)
static cs_status backward(cs_mlp m, const float* T, int n, int npad) {
  Weights& w = m->w;
  Grads& g = m->g;
  cudaMemsetAsync(m->loss, 0, sizeof(double), m->st);
  forward(m, npad, true);
  // output layer
  k_loss_grad<<<blocks((long)npad * NOUTP, 256), 256, 0, m->st>>>(m->Y, T, n, npad, m->dZ, m->dZT, m->dZf, m->loss);
  const int ks = npad / kTileM;   // one 128-sample K slice per CTA column
  cudaMemsetAsync(g.gW4, 0, sizeof(float) * kTileM * NH, m->st);
  gemm<EPI_ATOMIC>(m, m->dZT, npad, m->H3T, npad, kTileM, NH, npad, nullptr, g.gW4, NH, nullptr, 0, nullptr, 0, ks);
  k_colsum<<<NOUTP, 256, 0, m->st>>>(m->dZf, npad, NOUTP, g.gb4);
  gemm<EPI_STORE>(m, m->dZ, NOUTP, w.W4T, NOUTP, npad, NH, NOUTP, nullptr, m->dH, NH);
  // hidden layer 3
  k_silu_bwd<<<blocks((long)npad * NH, 256), 256, 0, m->st>>>(m->dH, m->Z3, n, npad, m->dZ, m->dZT, m->dZf);
  cudaMemsetAsync(g.gW3, 0, sizeof(float) * NH * NH, m->st);
  gemm<EPI_ATOMIC>(m, m->dZT, npad, m->H2T, npad, kTileM, NH, npad, nullptr, g.gW3, NH, nullptr, 0, nullptr, 0, ks);
  k_colsum<<<NH, 256, 0, m->st>>>(m->dZf, npad, NH, g.gb3);
  gemm<EPI_STORE>(m, m->dZ, NH, w.W3T, NH, npad, NH, NH, nullptr, m->dH, NH);
  // hidden layer 2
  k_silu_bwd<<<blocks((long)npad * NH, 256), 256, 0, m->st>>>(m->dH, m->Z2, n, npad, m->dZ, m->dZT, m->dZf);
  cudaMemsetAsync(g.gW2, 0, sizeof(float) * NH * NH, m->st);
  gemm<EPI_ATOMIC>(m, m->dZT, npad, m->H1T, npad, kTileM, NH, npad, nullptr, g.gW2, NH, nullptr, 0, nullptr, 0, ks);
  k_colsum<<<NH, 256, 0, m->st>>>(m->dZf, npad, NH, g.gb2);
  gemm<EPI_STORE>(m, m->dZ, NH, w.W2T, NH, npad, NH, NH, nullptr, m->dH, NH);
  // hidden layer 1
  k_silu_bwd<<<blocks((long)npad * NH, 256), 256, 0, m->st>>>(m->dH, m->Z1, n, npad, m->dZ, m->dZT, m->dZf);
  cudaMemsetAsync(g.gW1, 0, sizeof(float) * NH * KIN, m->st);
  gemm<EPI_ATOMIC>(m, m->dZT, npad, m->XT, npad, kTileM, KIN, npad, nullptr, g.gW1, KIN, nullptr, 0, nullptr, 0, ks);
  k_colsum<<<NH, 256, 0, m->st>>>(m->dZf, npad, NH, g.gb1);
  k_flatten_grads<<<blocks(NPARAM, 256), 256, 0, m->st>>>(g, m->grad);
  return check_err(m, "backward");
}

static cs_status pack(cs_mlp m, const float* X, int n, int* npad, bool transposed) {
  if (!X || n < 1 || n > m->max_batch) return mfail(m, CS_ERR_ARG, "batch of %d rows (1..%d)", n, m->max_batch);
  *npad = ((n + kTileM - 1) / kTileM) * kTileM;
  k_pack_input<<<blocks((long)*npad * KIN, 256), 256, 0, m->st>>>(X, n, *npad, m->X, transposed ? m->XT : nullptr);
  return CS_OK;
}

extern "C" cs_status cs_mlp_create(int max_batch, const float* params_host, cs_mlp* out) {
  if (!out || !params_host || max_batch < 1 || max_batch > (1 << 24)) return CS_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<cs_mlp_s> m(new cs_mlp_s);
  m->max_batch = max_batch;
  const size_t np = ((size_t)(max_batch + kTileM - 1) / kTileM) * kTileM;
  m->npad_max = (int)np;
  cudaError_t e = gemm_attrs();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking);
#define MA(p, n) if (e == cudaSuccess) e = malloc0(m.get(), &(p), (n))
  MA(m->p, NPARAM); MA(m->m, NPARAM); MA(m->v, NPARAM); MA(m->grad, NPARAM);
  MA(m->w.W1, NH * KIN); MA(m->w.W2, NH * NH); MA(m->w.W3, NH * NH); MA(m->w.W4, NOUTP * NH);
  MA(m->w.W2T, NH * NH); MA(m->w.W3T, NH * NH); MA(m->w.W4T, NH * NOUTP);
  MA(m->w.b1, NH); MA(m->w.b2, NH); MA(m->w.b3, NH); MA(m->w.b4, NOUTP);
  MA(m->X, np * KIN); MA(m->XT, np * KIN);
  MA(m->H1, np * NH); MA(m->H2, np * NH); MA(m->H3, np * NH);
  MA(m->H1T, np * NH); MA(m->H2T, np * NH); MA(m->H3T, np * NH);
  MA(m->Z1, np * NH); MA(m->Z2, np * NH); MA(m->Z3, np * NH); MA(m->Y, np * NOUTP);
  MA(m->dH, np * NH); MA(m->dZf, np * NH); MA(m->dZ, np * NH); MA(m->dZT, np * NH);
  MA(m->g.gW1, NH * KIN); MA(m->g.gW2, NH * NH); MA(m->g.gW3, NH * NH); MA(m->g.gW4, kTileM * NH);
  MA(m->g.gb1, NH); MA(m->g.gb2, NH); MA(m->g.gb3, NH); MA(m->g.gb4, NOUTP);
  MA(m->loss, 1); MA(m->err, 1);
#undef MA
  if (e == cudaSuccess && cudaMallocHost(&m->h_loss, sizeof(double)) != cudaSuccess) e = cudaErrorMemoryAllocation;
  if (e == cudaSuccess && cudaMallocHost(&m->h_err, sizeof(int)) != cudaSuccess) e = cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = cudaMemcpy(m->p, params_host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_cast_params<<<blocks(NH * NH, 256), 256, 0, m->st>>>(m->p, m->w);
    e = cudaStreamSynchronize(m->st);
  }
  if (e != cudaSuccess) {
    cs_mlp_destroy(m.release());
    return e == cudaErrorMemoryAllocation ? CS_ERR_OOM : CS_ERR_CUDA;
  }
  *out = m.release();
  return CS_OK;
}

extern "C" cs_status cs_mlp_destroy(cs_mlp m) {
  if (!m) return CS_ERR_ARG;
  if (m->st) cudaStreamSynchronize(m->st);
  for (void* p : m->allocs) cudaFree(p);
  if (m->h_loss) cudaFreeHost(m->h_loss);
  if (m->h_err) cudaFreeHost(m->h_err);
  if (m->st) cudaStreamDestroy(m->st);
  delete m;
  return CS_OK;
}

extern "C" cs_status cs_mlp_get_params(cs_mlp m, float* params_host) {
  if (!m || !params_host) return CS_ERR_ARG;
  if (cudaMemcpyAsync(params_host, m->p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
      cudaStreamSynchronize(m->st) != cudaSuccess)
    return mfail(m, CS_ERR_CUDA, "get_params");
  return CS_OK;
}

extern "C" cs_status cs_mlp_forward(cs_mlp m, const float* X_dev, int n, float* Y_dev) {
  if (!m || !Y_dev) return CS_ERR_ARG;
  if (!X_dev || n < 1 || n > m->max_batch) return mfail(m, CS_ERR_ARG, "batch of %d rows (1..%d)", n, m->max_batch);
  cudaMemsetAsync(m->err, 0, sizeof(int), m->st);
  infer(m, X_dev, n, Y_dev, m->st);
  return check_err(m, "cs_mlp_forward");
}

extern "C" cs_status cs_mlp_grad(cs_mlp m, const float* X_dev, const float* T_dev, int n, float* grad_host,
                                 double* loss_out) {
  if (!m || !T_dev) return CS_ERR_ARG;
  int npad;
  cs_status s = pack(m, X_dev, n, &npad, true);
  if (s) return s;
  cudaMemsetAsync(m->err, 0, sizeof(int), m->st);
  if ((s = backward(m, T_dev, n, npad))) return s;
  if (loss_out) *loss_out = *m->h_loss / ((double)n * NOUT);
  if (grad_host &&
      (cudaMemcpy(grad_host, m->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess))
    return mfail(m, CS_ERR_CUDA, "grad copy");
  return CS_OK;
}

extern "C" cs_status cs_mlp_train_step(cs_mlp m, const float* X_dev, const float* T_dev, int n, float lr,
                                       double* loss_out) {
  if (!m || !T_dev || !(lr > 0.f)) return CS_ERR_ARG;
  int npad;
  cs_status s = pack(m, X_dev, n, &npad, true);
  if (s) return s;
  cudaMemsetAsync(m->err, 0, sizeof(int), m->st);
  if ((s = backward(m, T_dev, n, npad))) return s;
  m->step++;
  const float bc1 = (float)(1.0 - std::pow(0.9, m->step)), bc2 = (float)(1.0 - std::pow(0.999, m->step));
  k_adam<<<blocks(NPARAM, 256), 256, 0, m->st>>>(m->p, m->grad, m->m, m->v, lr, bc1, bc2);
  k_cast_params<<<blocks(NH * NH, 256), 256, 0, m->st>>>(m->p, m->w);
  if (loss_out) *loss_out = *m->h_loss / ((double)n * NOUT);
  // the updated weights are complete when the call returns (another stream may use them next)
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(m->st) != cudaSuccess)
    return mfail(m, CS_ERR_CUDA, "adam");
  return CS_OK;
}

extern "C" const char* cs_mlp_last_error(cs_mlp m) { return m ? m->msg : "null network"; }

// Solver coupling (C++ linkage, called by the grid code): the network on n rows of
// standardised FP32 inputs X into Y [n][22], enqueued on stream st without synchronisation.
// A network must not serve two streams at once (its activation buffers are shared).
int mlp_max_batch(cs_mlp m) { return m ? m->max_batch : 0; }
void mlp_forward_on(cs_mlp m, const float* X, int n, float* Y, cudaStream_t st) { infer(m, X, n, Y, st); }
int mlp_error(cs_mlp m) {
  int e = 0;
  cudaMemcpy(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost);
  return e;
}
