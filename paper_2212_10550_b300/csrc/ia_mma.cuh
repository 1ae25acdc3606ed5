// Reduced-precision canonical field: fp16 hash features and a tensor-core MLP
// (fp16 or bf16 operands, fp32 accumulation), evaluated for the 32 samples of a
// warp at once.
//
// The fused render kernel schedules work per warp (32 samples in flight), so the
// MLP runs as two 16-row tiles of m16n8k16 warp MMAs: the layer-1 accumulator
// fragments (16 x 64, fp32) are rectified and packed in registers straight into
// the A fragments of layer 2, and likewise into layer 3; only the features go
// through shared memory (lane -> row), and only the 4 outputs come back.  Weights
// live in shared memory as [out][in] rows, padded so the B-fragment loads of the
// 32 lanes hit 32 different banks.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ia_device.cuh"

namespace ia {

enum class Prec { F32 = 0, F16 = 1, BF16 = 2 };

// shared-memory layout of the reduced-precision MLP (32-bit words)
constexpr int kW1Stride = kIn / 2 + 4;      // 20 words per W1 row (32 halves + pad)
constexpr int kW2Stride = kWidth / 2 + 4;   // 36 words per W2 / W3 row
constexpr int kXStride = kIn / 2 + 4;       // 20 words per staged feature row
constexpr int kOffHW1 = 0;
constexpr int kOffHW2 = kOffHW1 + kWidth * kW1Stride;
constexpr int kOffHW3 = kOffHW2 + kWidth * kW2Stride;     // 8 rows, rows 4..7 zero
constexpr int kOffHB = kOffHW3 + 8 * kW2Stride;            // fp32 biases b1 [64], b2 [64], b3 [8]
constexpr int kMlpHWords = kOffHB + kWidth + kWidth + 8;
constexpr int kWarpXWords = 32 * kXStride + 32 * 4;         // staged features + outputs per warp

template <Prec P>
struct HalfOf;
template <>
struct HalfOf<Prec::F16> {
  using T = __half;
  __device__ static uint32_t pack(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  __device__ static float round(float x) { return __half2float(__float2half_rn(x)); }
  __device__ static uint16_t bits(float x) { return __half_as_ushort(__float2half_rn(x)); }
  static constexpr float kMax = 65504.f;
};
template <>
struct HalfOf<Prec::BF16> {
  using T = __nv_bfloat16;
  __device__ static uint32_t pack(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  __device__ static float round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
  __device__ static uint16_t bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
  static constexpr float kMax = 3.38e38f;
};

// Stage the packed fp32 MLP into the reduced-precision shared layout.
template <Prec P>
__device__ __forceinline__ void stage_mlp_h(const float* __restrict__ g, int n_in, uint32_t* sw) {
  const int nW1 = kWidth * n_in;
  const float* b1 = g + nW1;
  const float* W2 = b1 + kWidth;
  const float* b2 = W2 + kWidth * kWidth;
  const float* W3 = b2 + kWidth;
  const float* b3 = W3 + 4 * kWidth;
  for (int t = threadIdx.x; t < kMlpHWords; t += blockDim.x) {
    uint32_t v = 0;
    if (t < kOffHW2) {
      const int r = t / kW1Stride, c = t % kW1Stride;
      if (c < kIn / 2) {
        const int i = 2 * c;
        v = HalfOf<P>::pack(i < n_in ? g[r * n_in + i] : 0.f, i + 1 < n_in ? g[r * n_in + i + 1] : 0.f);
      }
    } else if (t < kOffHW3) {
      const int q = t - kOffHW2, r = q / kW2Stride, c = q % kW2Stride;
      if (c < kWidth / 2) v = HalfOf<P>::pack(W2[r * kWidth + 2 * c], W2[r * kWidth + 2 * c + 1]);
    } else if (t < kOffHB) {
      const int q = t - kOffHW3, r = q / kW2Stride, c = q % kW2Stride;
      if (c < kWidth / 2 && r < 4) v = HalfOf<P>::pack(W3[r * kWidth + 2 * c], W3[r * kWidth + 2 * c + 1]);
    } else {
      const int q = t - kOffHB;
      float f = 0.f;
      if (q < kWidth) f = b1[q];
      else if (q < 2 * kWidth) f = b2[q - kWidth];
      else if (q < 2 * kWidth + 4) f = b3[q - 2 * kWidth];
      v = __float_as_uint(f);
    }
    sw[t] = v;
  }
}

template <Prec P>
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  if constexpr (P == Prec::F16) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
}

// The warp's 32 feature rows (one per lane) -> 32 output rows of 4, one per lane.
// All 32 lanes must call; xs: this warp's staging area (kWarpXWords words).
template <Prec P, bool kRolled = false>
__device__ __forceinline__ void mlp_mma_warp_staged(const uint32_t* __restrict__ sw, uint32_t* xs, float out[4]);

template <Prec P>
__device__ __forceinline__ void mlp_mma_warp(const uint32_t* __restrict__ sw, uint32_t* xs, const float feat[kIn],
                                             float out[4]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < kIn / 2; ++c) xs[lane * kXStride + c] = HalfOf<P>::pack(feat[2 * c], feat[2 * c + 1]);
  mlp_mma_warp_staged<P>(sw, xs, out);
}

// The same chain with the feature rows already staged in xs (row = lane, word c
// = the operand pair of inputs 2c, 2c + 1).  kRolled runs the two 16-row halves
// rolled: the chain runs once per list, and in the proposal kernels, whose code
// is largest, the search loop beside it must stay in the instruction cache.
template <Prec P, bool kRolled>
__device__ __forceinline__ void mlp_mma_warp_staged(const uint32_t* __restrict__ sw, uint32_t* xs, float out[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t* X = xs;
  float* O = reinterpret_cast<float*>(xs + 32 * kXStride);
  __syncwarp();
  const float* bias = reinterpret_cast<const float*>(sw + kOffHB);
#pragma unroll(kRolled ? 1 : 2)
  for (int mt = 0; mt < 2; ++mt) {
    const int r0 = 16 * mt + g, r1 = r0 + 8;
    // ---- layer 1: [16 x 32] x W1^T -> [16 x 64]
    uint32_t A[2][4];
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) {
      A[kt][0] = X[r0 * kXStride + 8 * kt + t];
      A[kt][1] = X[r1 * kXStride + 8 * kt + t];
      A[kt][2] = X[r0 * kXStride + 8 * kt + 4 + t];
      A[kt][3] = X[r1 * kXStride + 8 * kt + 4 + t];
    }
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float b0 = bias[8 * nt + 2 * t], b1 = bias[8 * nt + 2 * t + 1];
      acc[nt][0] = b0; acc[nt][1] = b1; acc[nt][2] = b0; acc[nt][3] = b1;
      const uint32_t* Wr = sw + kOffHW1 + (8 * nt + g) * kW1Stride;
#pragma unroll
      for (int kt = 0; kt < 2; ++kt) mma16816<P>(acc[nt], A[kt], Wr[8 * kt + t], Wr[8 * kt + 4 + t]);
    }
    // ---- ReLU, pack to A fragments of layer 2 (accumulator layout == A layout)
    uint32_t A2[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      A2[kt][0] = HalfOf<P>::pack(fmaxf(acc[2 * kt][0], 0.f), fmaxf(acc[2 * kt][1], 0.f));
      A2[kt][1] = HalfOf<P>::pack(fmaxf(acc[2 * kt][2], 0.f), fmaxf(acc[2 * kt][3], 0.f));
      A2[kt][2] = HalfOf<P>::pack(fmaxf(acc[2 * kt + 1][0], 0.f), fmaxf(acc[2 * kt + 1][1], 0.f));
      A2[kt][3] = HalfOf<P>::pack(fmaxf(acc[2 * kt + 1][2], 0.f), fmaxf(acc[2 * kt + 1][3], 0.f));
    }
    // ---- layer 2: [16 x 64] x W2^T -> [16 x 64]
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float b0 = bias[kWidth + 8 * nt + 2 * t], b1 = bias[kWidth + 8 * nt + 2 * t + 1];
      acc[nt][0] = b0; acc[nt][1] = b1; acc[nt][2] = b0; acc[nt][3] = b1;
      const uint32_t* Wr = sw + kOffHW2 + (8 * nt + g) * kW2Stride;
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) mma16816<P>(acc[nt], A2[kt], Wr[8 * kt + t], Wr[8 * kt + 4 + t]);
    }
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      A2[kt][0] = HalfOf<P>::pack(fmaxf(acc[2 * kt][0], 0.f), fmaxf(acc[2 * kt][1], 0.f));
      A2[kt][1] = HalfOf<P>::pack(fmaxf(acc[2 * kt][2], 0.f), fmaxf(acc[2 * kt][3], 0.f));
      A2[kt][2] = HalfOf<P>::pack(fmaxf(acc[2 * kt + 1][0], 0.f), fmaxf(acc[2 * kt + 1][1], 0.f));
      A2[kt][3] = HalfOf<P>::pack(fmaxf(acc[2 * kt + 1][2], 0.f), fmaxf(acc[2 * kt + 1][3], 0.f));
    }
    // ---- layer 3: [16 x 64] x W3^T -> [16 x 8] (outputs 4..7 are padding)
    float o[4];
    {
      const float b0 = bias[2 * kWidth + 2 * t], b1 = bias[2 * kWidth + 2 * t + 1];
      o[0] = b0; o[1] = b1; o[2] = b0; o[3] = b1;
      const uint32_t* Wr = sw + kOffHW3 + g * kW2Stride;
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) mma16816<P>(o, A2[kt], Wr[8 * kt + t], Wr[8 * kt + 4 + t]);
    }
    if (t < 2) {
      O[r0 * 4 + 2 * t] = o[0];
      O[r0 * 4 + 2 * t + 1] = o[1];
      O[r1 * 4 + 2 * t] = o[2];
      O[r1 * 4 + 2 * t + 1] = o[3];
    }
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 4; ++q) out[q] = O[lane * 4 + q];
  __syncwarp();
}

// The same network for one lane alone (the distinct root beyond a sample's
// list, evaluated where it is found), from the weights stage_mlp_h staged in
// shared memory: operands rounded to the reduced precision exactly as the
// tensor-core path rounds them, products and sums in fp32.
template <Prec P>
__device__ __forceinline__ float2 unpack_h(uint32_t w) {
  if constexpr (P == Prec::F16) return __half22float2(*reinterpret_cast<const __half2*>(&w));
  else return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
}

template <Prec P>
__device__ __forceinline__ void mlp_lane_hs(const uint32_t* __restrict__ sw, const float feat[kIn], float out[4]) {
  using H = HalfOf<P>;
  const float* bias = reinterpret_cast<const float*>(sw + kOffHB);
  float h1[kWidth];
  for (int j = 0; j < kWidth; ++j) {
    float acc = bias[j];
    const uint32_t* row = sw + kOffHW1 + j * kW1Stride;
#pragma unroll
    for (int c = 0; c < kIn / 2; ++c) {
      const float2 w = unpack_h<P>(row[c]);
      acc = fmaf(w.x, H::round(feat[2 * c]), acc);
      acc = fmaf(w.y, H::round(feat[2 * c + 1]), acc);
    }
    h1[j] = H::round(fmaxf(acc, 0.f));
  }
  float o[4] = {bias[2 * kWidth], bias[2 * kWidth + 1], bias[2 * kWidth + 2], bias[2 * kWidth + 3]};
  for (int j = 0; j < kWidth; ++j) {
    float acc = bias[kWidth + j];
    const uint32_t* row = sw + kOffHW2 + j * kW2Stride;
#pragma unroll
    for (int c = 0; c < kWidth / 2; ++c) {
      const float2 w = unpack_h<P>(row[c]);
      acc = fmaf(w.x, h1[2 * c], acc);
      acc = fmaf(w.y, h1[2 * c + 1], acc);
    }
    const float h = H::round(fmaxf(acc, 0.f));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 w = unpack_h<P>(sw[kOffHW3 + q * kW2Stride + j / 2]);
      o[q] = fmaf((j & 1) ? w.y : w.x, h, o[q]);
    }
  }
  for (int q = 0; q < 4; ++q) out[q] = o[q];
}

// fp16 hash features: the same encoding as encode(), reading the fp16 shadow table
// Hash encoding from the fp16 shadow table, written as the MLP chain's operand
// pairs straight into the staging row (word l = level l's two features), with
// the level loop rolled (small code; encode_h keeps every level's gathers in
// flight at once).  Same values as encode_h followed by the packing of
// mlp_mma_warp.
template <Prec P>
__device__ __forceinline__ void encode_h_staged(const FieldDev& F, const __half2* __restrict__ th, float3 x,
                                                uint32_t* row) {
  const float u[3] = {(x.x - F.cmin[0]) * F.inv_ext[0], (x.y - F.cmin[1]) * F.inv_ext[1],
                      (x.z - F.cmin[2]) * F.inv_ext[2]};
#pragma unroll 1
  for (int l = 0; l < kMaxLevels; ++l) {
    float a0 = 0.f, a1 = 0.f;
    if (l < F.L) {
      const Level lv = F.lv[l];
      int p0[3];
      float f[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        float pos = u[a] * (float)lv.res;
        int c = (int)floorf(pos);
        c = min(max(c, 0), lv.res - 1);
        p0[a] = c;
        f[a] = pos - (float)c;
      }
#pragma unroll
      for (int corner = 0; corner < 8; ++corner) {
        const int cx = corner & 1, cy = (corner >> 1) & 1, cz = (corner >> 2) & 1;
        const float w = (cx ? f[0] : 1.f - f[0]) * (cy ? f[1] : 1.f - f[1]) * (cz ? f[2] : 1.f - f[2]);
        const uint32_t e = lv.offset + vertex_index(lv, p0[0] + cx, p0[1] + cy, p0[2] + cz);
        const float2 t = __half22float2(th[e]);
        a0 = fmaf(w, t.x, a0);
        a1 = fmaf(w, t.y, a1);
      }
    }
    row[l] = HalfOf<P>::pack(a0, a1);
  }
}

__device__ __forceinline__ void encode_h(const FieldDev& F, const __half2* __restrict__ th, float3 x,
                                         float feat[kIn]) {
  const float u[3] = {(x.x - F.cmin[0]) * F.inv_ext[0], (x.y - F.cmin[1]) * F.inv_ext[1],
                      (x.z - F.cmin[2]) * F.inv_ext[2]};
#pragma unroll
  for (int l = 0; l < kMaxLevels; ++l) {
    feat[2 * l] = 0.f;
    feat[2 * l + 1] = 0.f;
    if (l < F.L) {
      const Level lv = F.lv[l];
      int p0[3];
      float f[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        float pos = u[a] * (float)lv.res;
        int c = (int)floorf(pos);
        c = min(max(c, 0), lv.res - 1);
        p0[a] = c;
        f[a] = pos - (float)c;
      }
      float a0 = 0.f, a1 = 0.f;
#pragma unroll
      for (int corner = 0; corner < 8; ++corner) {
        const int cx = corner & 1, cy = (corner >> 1) & 1, cz = (corner >> 2) & 1;
        const float w = (cx ? f[0] : 1.f - f[0]) * (cy ? f[1] : 1.f - f[1]) * (cz ? f[2] : 1.f - f[2]);
        const uint32_t e = lv.offset + vertex_index(lv, p0[0] + cx, p0[1] + cy, p0[2] + cz);
        const float2 t = __half22float2(th[e]);
        a0 = fmaf(w, t.x, a0);
        a1 = fmaf(w, t.y, a1);
      }
      feat[2 * l] = a0;
      feat[2 * l + 1] = a1;
    }
  }
}

}  // namespace ia
