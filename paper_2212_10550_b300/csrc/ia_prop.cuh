// Learned correspondence proposal (not part of the paper): device side.
//
// A small network maps a posed point x' (hash features of the normalised box)
// and the pose (axis-angles of all bones) to bone logits and a start offset; the
// correspondence search then begins from the top-k bones instead of all of them,
// and falls back to every bone-wise start when the proposed ones find no valid
// root.  Layer 1 is split: its pose columns are the same for every sample of a
// pose, so b1' = b1 + W1[:, pose] theta is computed once per block and each
// sample only multiplies its 2L hash features.
#pragma once

#include "ia_mma.cuh"

namespace ia {

constexpr int kPropMaxOut = 32;                 // logits + offset, padded to 4 n-tiles
constexpr int kPW1Stride = 8 + 4;               // 16 features = 8 words + pad
constexpr int kPOffW1 = 0;
constexpr int kPOffW2 = kPOffW1 + kWidth * kPW1Stride;
constexpr int kPOffW3 = kPOffW2 + kWidth * kW2Stride;
constexpr int kPOffW4 = kPOffW3 + kWidth * kW2Stride;
constexpr int kPOffB = kPOffW4 + kPropMaxOut * kW2Stride;  // fp32 b1' [64], b2 [64], b3 [64], b4 [32]
constexpr int kPropWords = kPOffB + 3 * kWidth + kPropMaxOut;
constexpr int kPropStageWords = 32 * kPW1Stride + 32 * (kPropMaxOut + 1);
constexpr int kStageWords = kPropStageWords > kWarpXWords ? kPropStageWords : kWarpXWords;

struct PropDev {
  const float2* table;     // fp32 [entries] (F = 2)
  int L;                   // levels (<= 8: 16 features)
  Level lv[kMaxLevels];
  float nmin[3];
  float inv_ext[3];        // 1 / (norm_max - norm_min)
  const float* mlp;        // packed fp32: W1 [64][n_in], b1, W2, b2, W3, b3, W4 [nb+3][64], b4
  int n_in;                // 2L + 3 nb
  int top_k;               // 1 or 2
  const float* b1p;        // [n_poses][64] per-pose layer-1 bias b1' (kernels whose
                           // lanes hold different poses), or null: b1' staged per block
};

// hash features of x' over the normalised box (2L values, zero-padded to 16)
__device__ __forceinline__ void prop_encode(const PropDev& Q, float3 x, float feat[16]) {
  const float u[3] = {(x.x - Q.nmin[0]) * Q.inv_ext[0], (x.y - Q.nmin[1]) * Q.inv_ext[1],
                      (x.z - Q.nmin[2]) * Q.inv_ext[2]};
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    feat[2 * l] = 0.f;
    feat[2 * l + 1] = 0.f;
    if (l < Q.L) {
      const Level lv = Q.lv[l];
      int p0[3];
      float f[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float pos = u[a] * (float)lv.res;
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
        const float2 t = __ldg(Q.table + e);
        a0 = fmaf(w, t.x, a0);
        a1 = fmaf(w, t.y, a1);
      }
      feat[2 * l] = a0;
      feat[2 * l + 1] = a1;
    }
  }
}

// prop_encode written as the network's operand pairs straight into the staging
// row (word l = level l's two features), with the level loop rolled.
template <Prec P>
__device__ __forceinline__ void prop_encode_staged(const PropDev& Q, float3 x, uint32_t* row) {
  const float u[3] = {(x.x - Q.nmin[0]) * Q.inv_ext[0], (x.y - Q.nmin[1]) * Q.inv_ext[1],
                      (x.z - Q.nmin[2]) * Q.inv_ext[2]};
#pragma unroll 1
  for (int l = 0; l < 8; ++l) {
    float a0 = 0.f, a1 = 0.f;
    if (l < Q.L) {
      const Level lv = Q.lv[l];
      int p0[3];
      float f[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float pos = u[a] * (float)lv.res;
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
        const float2 t = __ldg(Q.table + e);
        a0 = fmaf(w, t.x, a0);
        a1 = fmaf(w, t.y, a1);
      }
    }
    row[l] = HalfOf<P>::pack(a0, a1);
  }
}

// Stage the proposal weights (reduced precision) and the per-pose bias
// b1' = b1 + W1[:, 2L:] theta into shared memory.  theta: [nb * 3] fp64.
template <Prec P>
__device__ __forceinline__ void stage_prop_h(const PropDev& Q, int nb, const double* __restrict__ theta,
                                             uint32_t* sw) {
  const float* g = Q.mlp;
  const int nin = Q.n_in, nf = 2 * Q.L, nout = nb + 3;
  const float* b1 = g + kWidth * nin;
  const float* W2 = b1 + kWidth;
  const float* b2 = W2 + kWidth * kWidth;
  const float* W3 = b2 + kWidth;
  const float* b3 = W3 + kWidth * kWidth;
  const float* W4 = b3 + kWidth;
  const float* b4 = W4 + nout * kWidth;
  for (int t = threadIdx.x; t < kPropWords; t += blockDim.x) {
    uint32_t v = 0;
    if (t < kPOffW2) {
      const int r = t / kPW1Stride, c = t % kPW1Stride;
      if (c < 8) {
        const int i = 2 * c;
        v = HalfOf<P>::pack(i < nf ? g[r * nin + i] : 0.f, i + 1 < nf ? g[r * nin + i + 1] : 0.f);
      }
    } else if (t < kPOffW3) {
      const int q = t - kPOffW2, r = q / kW2Stride, c = q % kW2Stride;
      if (c < kWidth / 2) v = HalfOf<P>::pack(W2[r * kWidth + 2 * c], W2[r * kWidth + 2 * c + 1]);
    } else if (t < kPOffW4) {
      const int q = t - kPOffW3, r = q / kW2Stride, c = q % kW2Stride;
      if (c < kWidth / 2) v = HalfOf<P>::pack(W3[r * kWidth + 2 * c], W3[r * kWidth + 2 * c + 1]);
    } else if (t < kPOffB) {
      const int q = t - kPOffW4, r = q / kW2Stride, c = q % kW2Stride;
      if (c < kWidth / 2 && r < nout) v = HalfOf<P>::pack(W4[r * kWidth + 2 * c], W4[r * kWidth + 2 * c + 1]);
    } else {
      const int q = t - kPOffB;
      float f = 0.f;
      if (q < kWidth) {  // b1' = b1 + W1[:, pose part] theta (fp32)
        f = b1[q];
        if (theta)
          for (int i = 0; i < 3 * nb; ++i) f = fmaf(g[q * nin + nf + i], (float)theta[i], f);
      } else if (q < 2 * kWidth) {
        f = b2[q - kWidth];
      } else if (q < 3 * kWidth) {
        f = b3[q - 2 * kWidth];
      } else if (q - 3 * kWidth < nout) {
        f = b4[q - 3 * kWidth];
      }
      v = __float_as_uint(f);
    }
    sw[t] = v;
  }
}

// One hidden layer of 64 on a 16-row tile: A (4 k-tiles) -> rectified A'.
template <Prec P>
__device__ __forceinline__ void prop_hidden(const uint32_t* __restrict__ W, const float* __restrict__ b,
                                            uint32_t A[4][4], int g, int t) {
  float acc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = b[8 * nt + 2 * t], b1 = b[8 * nt + 2 * t + 1];
    acc[nt][0] = b0; acc[nt][1] = b1; acc[nt][2] = b0; acc[nt][3] = b1;
    const uint32_t* Wr = W + (8 * nt + g) * kW2Stride;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) mma16816<P>(acc[nt], A[kt], Wr[8 * kt + t], Wr[8 * kt + 4 + t]);
  }
#pragma unroll
  for (int kt = 0; kt < 4; ++kt) {
    A[kt][0] = HalfOf<P>::pack(fmaxf(acc[2 * kt][0], 0.f), fmaxf(acc[2 * kt][1], 0.f));
    A[kt][1] = HalfOf<P>::pack(fmaxf(acc[2 * kt][2], 0.f), fmaxf(acc[2 * kt][3], 0.f));
    A[kt][2] = HalfOf<P>::pack(fmaxf(acc[2 * kt + 1][0], 0.f), fmaxf(acc[2 * kt + 1][1], 0.f));
    A[kt][3] = HalfOf<P>::pack(fmaxf(acc[2 * kt + 1][2], 0.f), fmaxf(acc[2 * kt + 1][3], 0.f));
  }
}

// The warp's 32 feature rows -> 32 output rows (logits, offset) in the staging
// area O [32][kPropMaxOut + 1]; all 32 lanes call.  Returns O.  With b1p, each
// row takes the layer-1 bias of its own lane's pose (b1p + 64 * pose).
// (kRolled: the feature rows are already staged in xs, row = lane, word c = the
// operand pair of inputs 2c, 2c + 1, and the two 16-row halves run rolled, for
// the kernels whose code overflows the instruction cache.)
template <Prec P, bool kRolled = false>
__device__ __forceinline__ const float* prop_mma_warp(const uint32_t* __restrict__ sw, uint32_t* xs,
                                                      const float feat[16], const float* __restrict__ b1p = nullptr,
                                                      int pose = 0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t* X = xs;
  float* O = reinterpret_cast<float*>(xs + 32 * kPW1Stride);
  if constexpr (!kRolled) {
#pragma unroll
    for (int c = 0; c < 8; ++c) X[lane * kPW1Stride + c] = HalfOf<P>::pack(feat[2 * c], feat[2 * c + 1]);
  }
  __syncwarp();
  const float* bias = reinterpret_cast<const float*>(sw + kPOffB);
#pragma unroll(kRolled ? 1 : 2)
  for (int mt = 0; mt < 2; ++mt) {
    const int r0 = 16 * mt + g, r1 = r0 + 8;
    uint32_t A1[4] = {X[r0 * kPW1Stride + t], X[r1 * kPW1Stride + t], X[r0 * kPW1Stride + 4 + t],
                      X[r1 * kPW1Stride + 4 + t]};
    const float* bias0 = bias;  // layer-1 bias of rows r0 and r1
    const float* bias1 = bias;
    if (b1p) {
      bias0 = b1p + kWidth * __shfl_sync(kFull, pose, r0);
      bias1 = b1p + kWidth * __shfl_sync(kFull, pose, r1);
    }
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float2 c0 = *reinterpret_cast<const float2*>(bias0 + 8 * nt + 2 * t);
      const float2 c1 = *reinterpret_cast<const float2*>(bias1 + 8 * nt + 2 * t);
      acc[nt][0] = c0.x; acc[nt][1] = c0.y; acc[nt][2] = c1.x; acc[nt][3] = c1.y;
      const uint32_t* Wr = sw + kPOffW1 + (8 * nt + g) * kPW1Stride;
      mma16816<P>(acc[nt], A1, Wr[t], Wr[4 + t]);
    }
    uint32_t A[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      A[kt][0] = HalfOf<P>::pack(fmaxf(acc[2 * kt][0], 0.f), fmaxf(acc[2 * kt][1], 0.f));
      A[kt][1] = HalfOf<P>::pack(fmaxf(acc[2 * kt][2], 0.f), fmaxf(acc[2 * kt][3], 0.f));
      A[kt][2] = HalfOf<P>::pack(fmaxf(acc[2 * kt + 1][0], 0.f), fmaxf(acc[2 * kt + 1][1], 0.f));
      A[kt][3] = HalfOf<P>::pack(fmaxf(acc[2 * kt + 1][2], 0.f), fmaxf(acc[2 * kt + 1][3], 0.f));
    }
    prop_hidden<P>(sw + kPOffW2, bias + kWidth, A, g, t);
    prop_hidden<P>(sw + kPOffW3, bias + 2 * kWidth, A, g, t);
#pragma unroll
    for (int nt = 0; nt < kPropMaxOut / 8; ++nt) {
      const float b0 = bias[3 * kWidth + 8 * nt + 2 * t], b1 = bias[3 * kWidth + 8 * nt + 2 * t + 1];
      float o[4] = {b0, b1, b0, b1};
      const uint32_t* Wr = sw + kPOffW4 + (8 * nt + g) * kW2Stride;
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) mma16816<P>(o, A[kt], Wr[8 * kt + t], Wr[8 * kt + 4 + t]);
      const int c = 8 * nt + 2 * t;
      O[r0 * (kPropMaxOut + 1) + c] = o[0];
      O[r0 * (kPropMaxOut + 1) + c + 1] = o[1];
      O[r1 * (kPropMaxOut + 1) + c] = o[2];
      O[r1 * (kPropMaxOut + 1) + c + 1] = o[3];
    }
  }
  __syncwarp();
  return O;
}

}  // namespace ia
