// Weight-gradient reduction of the reduced-precision training step on the
// 5th-generation tensor cores (tcgen05 + TMA + TMEM), sm_103a.
//
// The per-sample backward writes its recomputed activations and (loss-scaled)
// gradients into one fp16/bf16 array X of kWgRows rows (a row per channel, a
// column per sample; chunk-contiguous, see wg_index), so every operand is
// K-major with K = samples:
//
//   rows   0.. 63  dH2        rows 128..191  H1        rows 240..303  H2
//   rows  64..127  dH1        rows 192..223  F         row  304       1
//                             row  224       1         rows 305..367  0
//                             rows 225..239  0         rows 368..371  dO
//                                                      rows 372..383  0
//
//   GEMM 1: D1 [128 x 112] = X[0:128] X[128:240]^T  -> dW2 (rows 0..63, cols 0..63),
//           db2 (rows 0..63, col 96), dW1 (rows 64..127, cols 64..95), db1 (col 96)
//   GEMM 2: D2 [128 x 16]  = X[240:368] X[368:384]^T -> dW3^T (rows 0..63, cols 0..3),
//           db3 (row 64, cols 0..3)
//
// X is chunk-contiguous (wg_index): each CTA reduces a contiguous range of
// 64-sample chunks, each one sequential 48 KiB block.  The work is split by
// role: lane 0 of warp 0 streams the chunks with TMA (three 128-row boxes per
// chunk, 128-byte swizzle) into a four-stage ring, lane 0 of
// warp 1 waits for each stage, issues its MMAs (M = 128, K = 16 per
// instruction, fp32 accumulation in 128 TMEM columns) and commits them to the
// stage's "empty" barrier, which hands the stage back to the producer; so up
// to four chunks are in flight per SM while the tensor cores consume the
// oldest.  After the last commit all four warps read the accumulators with
// tcgen05.ld, unscale them and add them to the fp32 gradients.
//
// Every mbarrier wait is bounded in time (WgradArgs::wait_ns, from the
// global nanosecond timer).  When a wait expires, or the other role gave up,
// the thread stops issuing and raises kStepPipelineError in the step's flags
// (the step is then skipped: its gradients are zeroed and the host call
// reports the error).  Before the CTA frees its TMEM and exits it waits, again
// with a bound, for what it already put in flight: the producer for each TMA
// load it issued, the MMA thread for a final commit that tracks every MMA it
// issued.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "ia_profile.h"
#include "ia_wgrad.h"

namespace ia {

constexpr int kWgStageBytes = kWgRows * kWgChunk * 2;  // 48 KiB
constexpr int kWgStages = 4;
constexpr int kWgThreads = 128;
constexpr int kWgBoxRows = 128;                         // rows per TMA box
constexpr uint64_t kWgDrainNs = 1000000000ull;          // 1 s bound on waiting for work in flight

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(a), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the phase of `bar` with the given parity.  False when it has not
// completed within limit_ns, or when *abort (if given) was raised meanwhile.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns,
                                          const volatile int* abort) {
  const uint32_t a = smem_u32(bar);
  uint64_t t0 = 0;
  for (uint32_t i = 0;; ++i) {
    if (mbar_try(a, parity)) return true;
    if ((i & 31) == 0) {
      const uint64_t t = global_ns();
      if (i == 0) t0 = t;
      else if (t - t0 > limit_ns) return false;
      if (abort && *abort) return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// K-major operand, 128-byte swizzle: 8-row atoms of 1024 B (stride-dimension
// byte offset 1024), descriptor version 1, layout type 2 (SWIZZLE_128B).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);         // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused within one atom)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset
  d |= (uint64_t)1 << 46;                        // version
  d |= (uint64_t)2 << 61;                        // SWIZZLE_128B
  return d;
}

// kind::f16 instruction descriptor: fp32 accumulator, fp16 or bf16 operands,
// both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, int bf16) {
  return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrives on `bar` once every tcgen05 operation this thread issued before it has completed
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// four consecutive gradient entries: one vector atomic where the address allows it
__device__ __forceinline__ void add4(float* p, float a, float b, float c, float d) {
  if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
    atomicAdd(reinterpret_cast<float4*>(p), make_float4(a, b, c, d));
  } else {
    atomicAdd(p, a);
    atomicAdd(p + 1, b);
    atomicAdd(p + 2, c);
    atomicAdd(p + 3, d);
  }
}

__global__ void __launch_bounds__(kWgThreads, 1) wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmap,
                                                               const WgradArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kWgStages * kWgStageBytes);  // stage loaded
  uint64_t* empty = full + kWgStages;                                              // stage consumed
  uint64_t* done = empty + kWgStages;                                              // every MMA completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ volatile int s_abort;

  const int n = *a.count;
  const int chunks = (n + kWgChunk - 1) / kWgChunk;
  const int per = (chunks + gridDim.x - 1) / gridDim.x;
  const int c0 = blockIdx.x * per, c1 = min(chunks, c0 + per);
  if (c0 >= c1) return;  // uniform over the CTA
  const int nch = c1 - c0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kWgStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t tD1 = tmem, tD2 = tmem + 112;

  if (warp == 0 && lane == 0) {
    // ---- producer: chunk i into stage i % kWgStages once its previous chunk's MMAs are done
    int issued = 0;
    for (int i = 0; i < nch; ++i) {
      const int st = i % kWgStages;
      if (i >= kWgStages && !mbar_wait(&empty[st], ((i / kWgStages) - 1) & 1, a.wait_ns, &s_abort)) {
        s_abort = 1;
        break;
      }
      if (a.withhold_last && i == nch - 1) break;  // injected stall: the consumer's wait must expire
      uint8_t* base = smem + st * kWgStageBytes;
      mbar_expect_tx(&full[st], kWgStageBytes);
      for (int r = 0; r < kWgRows; r += kWgBoxRows) tma_load_3d(base + r * 128, &tmap, 0, r, c0 + i, &full[st]);
      ++issued;
    }
    // every load issued has landed before the CTA may exit (the last load of
    // each stage: no later load was issued to it, so its phase is the one to wait for)
    bool drained = true;
    for (int i = issued > kWgStages ? issued - kWgStages : 0; i < issued; ++i)
      drained &= mbar_wait(&full[i % kWgStages], (i / kWgStages) & 1, kWgDrainNs, nullptr);
    if (!drained) s_abort = 1;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t id1 = idesc_f16(128, 112, a.bf16), id2 = idesc_f16(128, 16, a.bf16);
    for (int i = 0; i < nch; ++i) {
      const int st = i % kWgStages;
      if (!mbar_wait(&full[st], (i / kWgStages) & 1, a.wait_ns, &s_abort)) {
        s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t b = smem_u32(smem + st * kWgStageBytes);
#pragma unroll
      for (int kk = 0; kk < kWgChunk / 16; ++kk) {
        const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
        umma_f16(tD1, smem_desc_sw128(b + kk * 32), smem_desc_sw128(b + 128 * 128 + kk * 32), id1, acc);
        umma_f16(tD2, smem_desc_sw128(b + 240 * 128 + kk * 32), smem_desc_sw128(b + 368 * 128 + kk * 32), id2, acc);
      }
      umma_commit(&empty[st]);
    }
    // tracks every MMA issued above, on the normal path and after giving up alike
    umma_commit(done);
    if (!mbar_wait(done, 0, kWgDrainNs, nullptr)) s_abort = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (s_abort) {
    if (threadIdx.x == 0) atomicOr(a.flags, kStepPipelineError);
  } else {
    const float inv = 1.f / *a.scale;
    const int row = warp * 32 + lane;  // TMEM lane = accumulator row
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    float v[16];
    // D1 columns in blocks of 16: 0..63 H1, 64..95 F, 96 ones
#pragma unroll 1
    for (int cb = 0; cb < 112; cb += 16) {
      tmem_ld16(tD1 + lane_base + cb, v);
#pragma unroll
      for (int j = 0; j < 16; j += 4) {
        const int col = cb + j;
        if (row < 64) {
          if (col < 64) add4(a.gW2 + row * 64 + col, v[j] * inv, v[j + 1] * inv, v[j + 2] * inv, v[j + 3] * inv);
          else if (col == 96) atomicAdd(a.gb2 + row, v[j] * inv);
        } else {
          const int r = row - 64;
          if (col >= 64 && col + 3 < 64 + a.n_in) {
            add4(a.gW1 + r * a.n_in + (col - 64), v[j] * inv, v[j + 1] * inv, v[j + 2] * inv, v[j + 3] * inv);
          } else if (col >= 64 && col < 64 + a.n_in) {
            for (int q = 0; q < 4 && col + q < 64 + a.n_in; ++q) atomicAdd(a.gW1 + r * a.n_in + (col + q - 64), v[j + q] * inv);
          } else if (col == 96) {
            atomicAdd(a.gb1 + r, v[j] * inv);
          }
        }
      }
    }
    tmem_ld16(tD2 + lane_base, v);
    if (row < 64) {
#pragma unroll
      for (int o = 0; o < 4; ++o) atomicAdd(a.gW3 + o * 64 + row, v[o] * inv);
    } else if (row == 64) {
      add4(a.gb3, v[0] * inv, v[1] * inv, v[2] * inv, v[3] * inv);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(tmem));
}

static size_t wgrad_smem_bytes() { return (size_t)kWgStages * kWgStageBytes + 8 * (2 * kWgStages + 1) + 16 + 1024; }

cudaError_t make_wgrad_map(CUtensorMap* map, void* X, int64_t ld, int bf16) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  if (ld % kWgChunk != 0 || ld <= 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0) return cudaErrorInvalidValue;
  const cuuint64_t dims[3] = {(cuuint64_t)kWgChunk, (cuuint64_t)kWgRows, (cuuint64_t)(ld / kWgChunk)};
  const cuuint64_t strides[2] = {(cuuint64_t)kWgChunk * 2, (cuuint64_t)kWgRows * kWgChunk * 2};
  const cuuint32_t box[3] = {(cuuint32_t)kWgChunk, (cuuint32_t)kWgBoxRows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, X, dims,
                      strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_wgrad_tc(const CUtensorMap& map, const WgradArgs& a, int grid, cudaStream_t s) {
  const size_t smem = wgrad_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  {
    KernelSpan span("wgrad_tc_kernel", s);
    wgrad_tc_kernel<<<grid, kWgThreads, smem, s>>>(map, a);
  }
  return cudaGetLastError();
}

}  // namespace ia
