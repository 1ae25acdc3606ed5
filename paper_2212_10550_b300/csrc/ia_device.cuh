// Device building blocks of the articulated radiance-field render path (sm_103a).
//
//   blend_value / blend_value_jac   LBS in normalised space through the blended
//                                   transform grid M(v) = sum_i W(v,i) N_i
//                                   (Sec. 3.1, Eq. 7)
//   posed_field_warp                Fast-SNARF style correspondence search: bone-wise
//                                   Broyden starts, one sample per lane, flattened
//                                   so that all lanes gather M at the same step,
//                                   then one Newton polish and a field evaluation
//                                   per distinct root, max-density selection
//   encode / mlp_fp32               multiresolution hash encoding + MLP (Eq. 1-2)
//
// Everything here is fp32 (the root-finding and skinning precision); the bone
// chain is fp64 in the pose kernel.  Indexing arithmetic that decides which
// samples exist lives in ia_index.cuh and uses explicitly rounded intrinsics.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ia {

constexpr int kMaxBones = 32;
constexpr int kMaxLevels = 16;
constexpr int kWidth = 64;
constexpr int kIn = 32;          // MLP input, zero-padded to 16 levels x 2 features
constexpr int kMaxRoots = 8;     // distinct roots remembered per sample for merging (measured on the
                                 // full-size frame against 4 / 6 / 12 / 16: fastest; a list that overflows
                                 // evaluates its roots to keep the best, which 4 did often)
constexpr unsigned kFull = 0xffffffffu;

// MLP weights staged in shared memory (fp32): W1 [64][32] (zero-padded
// columns), b1 [64], W2 [64][64], b2 [64], W3^T [64][4], b3 [4].
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kWidth * kIn;
constexpr int kOffW2 = kOffB1 + kWidth;
constexpr int kOffB2 = kOffW2 + kWidth * kWidth;
constexpr int kOffW3T = kOffB2 + kWidth;
constexpr int kOffB3 = kOffW3T + kWidth * 4;
constexpr int kMlpSmemFloats = kOffB3 + 4;

struct Level {
  int res;          // grid resolution N_l
  int dense;        // (N_l + 1)^3 <= T: row-major vertex index, else spatial hash
  uint32_t size;    // entries in the level
  uint32_t offset;  // first entry of the level
};

struct FieldDev {
  const float2* table;  // [entries] (F = 2)
  int L;
  Level lv[kMaxLevels];
  float cmin[3];
  float inv_ext[3];     // 1 / (cmax - cmin)
};

struct SkinDev {
  const float4* M;      // blended grid of one pose: [Rw^3][3] float4 = rows of N(v)
  int Rw;
  float cmin[3], cmax[3];
  float scale[3];       // (Rw - 1) / (cmax - cmin)
};

struct SolveCfg {
  int nb;
  int max_iter;
  float tol2;           // tol^2
};

// per-lane counters (32-bit: a lane's share of one launch stays far below 2^32)
struct SampleStats {
  unsigned starts = 0, iters = 0, converged = 0, roots = 0, proposed = 0, fallbacks = 0;
};

// ---------------------------------------------------------------------------
// LBS through the blended grid
// ---------------------------------------------------------------------------

struct CellCoord {
  int base;       // linear index of the lower corner
  float f[3];     // fractional position in the cell
  float live[3];  // 0 where the coordinate was clamped to the border
};

__device__ __forceinline__ CellCoord skin_cell(const SkinDev& S, float3 x) {
  CellCoord c;
  const float xs[3] = {x.x, x.y, x.z};
  int i0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float u = (xs[a] - S.cmin[a]) * S.scale[a];
    float hi = (float)(S.Rw - 1);
    c.live[a] = 1.f;
    if (!(u >= 0.f)) { u = 0.f; c.live[a] = 0.f; }
    if (u > hi) { u = hi; c.live[a] = 0.f; }
    int q = (int)floorf(u);
    q = min(q, S.Rw - 2);
    i0[a] = q;
    c.f[a] = u - (float)q;
  }
  c.base = (i0[2] * S.Rw + i0[1]) * S.Rw + i0[0];
  return c;
}

__device__ __forceinline__ int corner_index(const SkinDev& S, int base, int corner) {
  return base + (corner & 1) + S.Rw * (((corner >> 1) & 1) + S.Rw * ((corner >> 2) & 1));
}

// trilinear weight of a cell corner (bit 0: +x, bit 1: +y, bit 2: +z)
__device__ __forceinline__ float corner_weight(const CellCoord& c, int corner) {
  return ((corner & 1) ? c.f[0] : 1.f - c.f[0]) * (((corner >> 1) & 1) ? c.f[1] : 1.f - c.f[1]) *
         (((corner >> 2) & 1) ? c.f[2] : 1.f - c.f[2]);
}

// Mx += w * (one corner's three rows)
__device__ __forceinline__ void accumulate_corner(float Mx[12], float w, float4 r0, float4 r1, float4 r2) {
  Mx[0] = fmaf(w, r0.x, Mx[0]); Mx[1] = fmaf(w, r0.y, Mx[1]);
  Mx[2] = fmaf(w, r0.z, Mx[2]); Mx[3] = fmaf(w, r0.w, Mx[3]);
  Mx[4] = fmaf(w, r1.x, Mx[4]); Mx[5] = fmaf(w, r1.y, Mx[5]);
  Mx[6] = fmaf(w, r1.z, Mx[6]); Mx[7] = fmaf(w, r1.w, Mx[7]);
  Mx[8] = fmaf(w, r2.x, Mx[8]); Mx[9] = fmaf(w, r2.y, Mx[9]);
  Mx[10] = fmaf(w, r2.z, Mx[10]); Mx[11] = fmaf(w, r2.w, Mx[11]);
}

// M(x) = sum_c w_c M_c  (12 values, rows of a 3x4 matrix); M = one pose's grid
__device__ __forceinline__ void blend_value(const SkinDev& S, const float4* __restrict__ M, float3 x,
                                            float Mx[12]) {
  CellCoord c = skin_cell(S, x);
#pragma unroll
  for (int q = 0; q < 12; ++q) Mx[q] = 0.f;
#pragma unroll
  for (int corner = 0; corner < 8; ++corner) {
    const float4* p = M + 3 * corner_index(S, c.base, corner);
    accumulate_corner(Mx, corner_weight(c, corner), __ldg(p), __ldg(p + 1), __ldg(p + 2));
  }
}

// blend_value for a sequence of points of one pose (a Broyden iteration): the
// 8 corner records of the cell gathered last stay in registers (96 floats),
// and a point in the same cell evaluates M(x) without gathering (about half
// of the Broyden steps on the full-size frame stay in their cell).  The same
// weights and multiply-adds in the same order as blend_value.
struct CornerCache {
  float4 C[8][3];
  int base = -1;
  // returns whether it gathered
  __device__ __forceinline__ bool blend(const SkinDev& S, const float4* __restrict__ M, float3 x, float Mx[12]) {
    const CellCoord c = skin_cell(S, x);
    const bool gather = c.base != base;
    if (gather) {
      base = c.base;
#pragma unroll
      for (int corner = 0; corner < 8; ++corner) {
        const float4* p = M + 3 * corner_index(S, c.base, corner);
        C[corner][0] = __ldg(p);
        C[corner][1] = __ldg(p + 1);
        C[corner][2] = __ldg(p + 2);
      }
    }
#pragma unroll
    for (int q = 0; q < 12; ++q) Mx[q] = 0.f;
#pragma unroll
    for (int corner = 0; corner < 8; ++corner)
      accumulate_corner(Mx, corner_weight(c, corner), C[corner][0], C[corner][1], C[corner][2]);
    return gather;
  }
};

__device__ __forceinline__ float3 apply34(const float A[12], float3 x) {
  return make_float3(fmaf(A[0], x.x, fmaf(A[1], x.y, fmaf(A[2], x.z, A[3]))),
                     fmaf(A[4], x.x, fmaf(A[5], x.y, fmaf(A[6], x.z, A[7]))),
                     fmaf(A[8], x.x, fmaf(A[9], x.y, fmaf(A[10], x.z, A[11]))));
}

// M(x) and the full Jacobian J = M(x)[:, :3] + sum_c (M_c [x;1]) grad(w_c)^T
__device__ __forceinline__ void blend_value_jac(const SkinDev& S, const float4* __restrict__ M, float3 x,
                                                float Mx[12], float J[9]) {
  CellCoord c = skin_cell(S, x);
#pragma unroll
  for (int q = 0; q < 12; ++q) Mx[q] = 0.f;
  float G[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) G[q] = 0.f;
#pragma unroll
  for (int corner = 0; corner < 8; ++corner) {
    int v = corner_index(S, c.base, corner);
    const int cx = corner & 1, cy = (corner >> 1) & 1, cz = (corner >> 2) & 1;
    float wx = cx ? c.f[0] : 1.f - c.f[0];
    float wy = cy ? c.f[1] : 1.f - c.f[1];
    float wz = cz ? c.f[2] : 1.f - c.f[2];
    float w = wx * wy * wz;
    float gx = (cx ? 1.f : -1.f) * wy * wz * S.scale[0] * c.live[0];
    float gy = (cy ? 1.f : -1.f) * wx * wz * S.scale[1] * c.live[1];
    float gz = (cz ? 1.f : -1.f) * wx * wy * S.scale[2] * c.live[2];
    const float4* p = M + 3 * v;
    float4 r[3] = {__ldg(p), __ldg(p + 1), __ldg(p + 2)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Mx[4 * a + 0] = fmaf(w, r[a].x, Mx[4 * a + 0]);
      Mx[4 * a + 1] = fmaf(w, r[a].y, Mx[4 * a + 1]);
      Mx[4 * a + 2] = fmaf(w, r[a].z, Mx[4 * a + 2]);
      Mx[4 * a + 3] = fmaf(w, r[a].w, Mx[4 * a + 3]);
      float mc = fmaf(r[a].x, x.x, fmaf(r[a].y, x.y, fmaf(r[a].z, x.z, r[a].w)));
      G[3 * a + 0] = fmaf(mc, gx, G[3 * a + 0]);
      G[3 * a + 1] = fmaf(mc, gy, G[3 * a + 1]);
      G[3 * a + 2] = fmaf(mc, gz, G[3 * a + 2]);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) J[3 * a + b] = Mx[4 * a + b] + G[3 * a + b];
}

// 3x3 inverse by the adjugate; false if |det| < 1e-6 (treated as singular)
// The search's arithmetic below spells every multiply-add out (fmaf) and keeps
// every other product and sum apart (__fmul_rn, __fadd_rn), so that each
// kernel that runs the search computes bit-for-bit the same iterates, whatever
// contractions the compiler would choose in its surroundings.
__device__ __forceinline__ float dot3(float a0, float a1, float a2, float b0, float b1, float b2) {
  return fmaf(a0, b0, fmaf(a1, b1, __fmul_rn(a2, b2)));
}

// a * b - c * d
__device__ __forceinline__ float cross2(float a, float b, float c, float d) { return fmaf(a, b, -__fmul_rn(c, d)); }

__device__ __forceinline__ bool inv3(const float J[9], float H[9]) {
  const float c00 = cross2(J[4], J[8], J[5], J[7]);
  const float c01 = cross2(J[5], J[6], J[3], J[8]);
  const float c02 = cross2(J[3], J[7], J[4], J[6]);
  const float det = dot3(J[0], J[1], J[2], c00, c01, c02);
  if (!(fabsf(det) >= 1e-6f)) return false;
  const float id = 1.f / det;
  H[0] = __fmul_rn(c00, id);
  H[1] = __fmul_rn(cross2(J[2], J[7], J[1], J[8]), id);
  H[2] = __fmul_rn(cross2(J[1], J[5], J[2], J[4]), id);
  H[3] = __fmul_rn(c01, id);
  H[4] = __fmul_rn(cross2(J[0], J[8], J[2], J[6]), id);
  H[5] = __fmul_rn(cross2(J[2], J[3], J[0], J[5]), id);
  H[6] = __fmul_rn(c02, id);
  H[7] = __fmul_rn(cross2(J[1], J[6], J[0], J[7]), id);
  H[8] = __fmul_rn(cross2(J[0], J[4], J[1], J[3]), id);
  return true;
}

// ---- one bone-wise Broyden search (Sec. 3.1, Eq. 7), shared by every kernel
//      that searches: start, residual, step direction, rank-one update

// x0 = N_k^-1 [x'; 1] (+ the proposal's start offset)
__device__ __forceinline__ float3 search_start(const float A[12], float3 xn, bool shift, float3 off) {
  float3 x = make_float3(fmaf(A[0], xn.x, fmaf(A[1], xn.y, fmaf(A[2], xn.z, A[3]))),
                         fmaf(A[4], xn.x, fmaf(A[5], xn.y, fmaf(A[6], xn.z, A[7]))),
                         fmaf(A[8], xn.x, fmaf(A[9], xn.y, fmaf(A[10], xn.z, A[11]))));
  if (shift) x = make_float3(__fadd_rn(x.x, off.x), __fadd_rn(x.y, off.y), __fadd_rn(x.z, off.z));
  return x;
}

// r = M(x) [x; 1] - x'
__device__ __forceinline__ float3 search_residual(const float Mx[12], float3 x, float3 xn) {
  return make_float3(__fsub_rn(fmaf(Mx[0], x.x, fmaf(Mx[1], x.y, fmaf(Mx[2], x.z, Mx[3]))), xn.x),
                     __fsub_rn(fmaf(Mx[4], x.x, fmaf(Mx[5], x.y, fmaf(Mx[6], x.z, Mx[7]))), xn.y),
                     __fsub_rn(fmaf(Mx[8], x.x, fmaf(Mx[9], x.y, fmaf(Mx[10], x.z, Mx[11]))), xn.z));
}

__device__ __forceinline__ float search_norm2(float3 r) { return dot3(r.x, r.y, r.z, r.x, r.y, r.z); }

// dx = -H r
__device__ __forceinline__ float3 search_dir(const float H[9], float3 r) {
  return make_float3(-dot3(H[0], H[1], H[2], r.x, r.y, r.z), -dot3(H[3], H[4], H[5], r.x, r.y, r.z),
                     -dot3(H[6], H[7], H[8], r.x, r.y, r.z));
}

__device__ __forceinline__ float3 add3(float3 a, float3 b) {
  return make_float3(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z));
}

// good Broyden: H += (dx - H dr)(dx^T H) / (dx^T H dr), skipped when the
// denominator vanishes
__device__ __forceinline__ void broyden_update(float H[9], float3 dx, float3 dr) {
  const float u0 = dot3(H[0], H[1], H[2], dr.x, dr.y, dr.z);
  const float u1 = dot3(H[3], H[4], H[5], dr.x, dr.y, dr.z);
  const float u2 = dot3(H[6], H[7], H[8], dr.x, dr.y, dr.z);
  const float den = dot3(dx.x, dx.y, dx.z, u0, u1, u2);
  if (fabsf(den) > 1e-12f) {
    const float rden = 1.f / den;  // one reciprocal for the three quotients
    const float a0 = __fmul_rn(__fsub_rn(dx.x, u0), rden), a1 = __fmul_rn(__fsub_rn(dx.y, u1), rden),
                a2 = __fmul_rn(__fsub_rn(dx.z, u2), rden);
    const float b0 = dot3(dx.x, dx.y, dx.z, H[0], H[3], H[6]);
    const float b1 = dot3(dx.x, dx.y, dx.z, H[1], H[4], H[7]);
    const float b2 = dot3(dx.x, dx.y, dx.z, H[2], H[5], H[8]);
    H[0] = fmaf(a0, b0, H[0]); H[1] = fmaf(a0, b1, H[1]); H[2] = fmaf(a0, b2, H[2]);
    H[3] = fmaf(a1, b0, H[3]); H[4] = fmaf(a1, b1, H[4]); H[5] = fmaf(a1, b2, H[5]);
    H[6] = fmaf(a2, b0, H[6]); H[7] = fmaf(a2, b1, H[7]); H[8] = fmaf(a2, b2, H[8]);
  }
}

__device__ __forceinline__ bool in_box(const SkinDev& S, float3 x) {
  return x.x >= S.cmin[0] && x.x <= S.cmax[0] && x.y >= S.cmin[1] && x.y <= S.cmax[1] &&
         x.z >= S.cmin[2] && x.z <= S.cmax[2];
}

// ---------------------------------------------------------------------------
// Canonical field: hash encoding + MLP (fp32)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t vertex_index(const Level& lv, int i, int j, int k) {
  if (lv.dense) {
    uint32_t r1 = (uint32_t)lv.res + 1u;
    return (uint32_t)i + r1 * ((uint32_t)j + r1 * (uint32_t)k);
  }
  uint32_t h = (uint32_t)i ^ ((uint32_t)j * 2654435761u) ^ ((uint32_t)k * 805459861u);
  return h & (lv.size - 1u);  // hashed levels hold T = 2^log2_table entries
}

__device__ __forceinline__ void encode(const FieldDev& F, float3 x, float feat[kIn]) {
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
        float w = (cx ? f[0] : 1.f - f[0]) * (cy ? f[1] : 1.f - f[1]) * (cz ? f[2] : 1.f - f[2]);
        uint32_t e = lv.offset + vertex_index(lv, p0[0] + cx, p0[1] + cy, p0[2] + cz);
        float2 t = __ldg(F.table + e);
        a0 = fmaf(w, t.x, a0);
        a1 = fmaf(w, t.y, a1);
      }
      feat[2 * l] = a0;
      feat[2 * l + 1] = a1;
    }
  }
}

// [32] -> 64 -> ReLU -> 64 -> ReLU -> 4, weights broadcast from shared memory
__device__ __forceinline__ void mlp_fp32(const float* __restrict__ sw, const float feat[kIn], float out[4]) {
  float h1[kWidth];
#pragma unroll
  for (int j = 0; j < kWidth; ++j) {
    float acc = sw[kOffB1 + j];
    const float4* row = reinterpret_cast<const float4*>(sw + kOffW1 + j * kIn);
#pragma unroll
    for (int i = 0; i < kIn / 4; ++i) {
      float4 w = row[i];
      acc = fmaf(w.x, feat[4 * i], acc);
      acc = fmaf(w.y, feat[4 * i + 1], acc);
      acc = fmaf(w.z, feat[4 * i + 2], acc);
      acc = fmaf(w.w, feat[4 * i + 3], acc);
    }
    h1[j] = fmaxf(acc, 0.f);
  }
  float o0 = sw[kOffB3], o1 = sw[kOffB3 + 1], o2 = sw[kOffB3 + 2], o3 = sw[kOffB3 + 3];
#pragma unroll 4
  for (int j = 0; j < kWidth; ++j) {
    float acc = sw[kOffB2 + j];
    const float4* row = reinterpret_cast<const float4*>(sw + kOffW2 + j * kWidth);
#pragma unroll
    for (int i = 0; i < kWidth / 4; ++i) {
      float4 w = row[i];
      acc = fmaf(w.x, h1[4 * i], acc);
      acc = fmaf(w.y, h1[4 * i + 1], acc);
      acc = fmaf(w.z, h1[4 * i + 2], acc);
      acc = fmaf(w.w, h1[4 * i + 3], acc);
    }
    float h = fmaxf(acc, 0.f);
    float4 w3 = reinterpret_cast<const float4*>(sw + kOffW3T)[j];
    o0 = fmaf(w3.x, h, o0);
    o1 = fmaf(w3.y, h, o1);
    o2 = fmaf(w3.z, h, o2);
    o3 = fmaf(w3.w, h, o3);
  }
  out[0] = o0; out[1] = o1; out[2] = o2; out[3] = o3;
}

// density = exp(clamp(o0, -15, 15)), colour = sigmoid(o1..3)
__device__ __forceinline__ void activate(const float o[4], float& sigma, float3& rgb) {
  sigma = expf(fminf(fmaxf(o[0], -15.f), 15.f));
  rgb = make_float3(1.f / (1.f + expf(-o[1])), 1.f / (1.f + expf(-o[2])), 1.f / (1.f + expf(-o[3])));
}

__device__ __forceinline__ void field_fp32(const FieldDev& F, const float* sw, float3 x, float& sigma,
                                           float3& rgb) {
  float feat[kIn], o[4];
  encode(F, x, feat);
  mlp_fp32(sw, feat, o);
  activate(o, sigma, rgb);
}

// Stage the packed MLP (W1 [64][n_in], b1, W2, b2, W3 [4][64], b3) into the
// shared-memory layout above.
__device__ __forceinline__ void stage_mlp(const float* __restrict__ g, int n_in, float* sw) {
  const int nW1 = kWidth * n_in;
  for (int t = threadIdx.x; t < kMlpSmemFloats; t += blockDim.x) {
    float v = 0.f;
    if (t < kOffB1) {
      int j = t / kIn, i = t % kIn;
      v = (i < n_in) ? g[j * n_in + i] : 0.f;
    } else if (t < kOffW2) {
      v = g[nW1 + (t - kOffB1)];
    } else if (t < kOffB2) {
      v = g[nW1 + kWidth + (t - kOffW2)];
    } else if (t < kOffW3T) {
      v = g[nW1 + kWidth + kWidth * kWidth + (t - kOffB2)];
    } else if (t < kOffB3) {
      int q = t - kOffW3T, j = q / 4, o = q % 4;  // W3^T[j][o] = W3[o][j]
      v = g[nW1 + 2 * kWidth + kWidth * kWidth + o * kWidth + j];
    } else {
      v = g[nW1 + 2 * kWidth + kWidth * kWidth + 4 * kWidth + (t - kOffB3)];
    }
    sw[t] = v;
  }
}

// ---------------------------------------------------------------------------
// Posed field f'(x') = f(x*): one sample per lane, all 32 lanes must call.
// ---------------------------------------------------------------------------

struct PosedOut {
  float sigma;   // 0 when no valid root
  float3 rgb;
  float3 xstar;
  int start;     // -1 when no valid root
};

// One Newton step x <- x - J(x)^-1 (LBS(x) - x') with the analytic Jacobian.
__device__ __forceinline__ float3 polish_root(const SkinDev& S, const float4* __restrict__ M, float3 xs,
                                              float3 xn) {
  float Mx[12], J[9], Hn[9];
  blend_value_jac(S, M, xs, Mx, J);
  float3 y = apply34(Mx, xs);
  float3 rr = make_float3(y.x - xn.x, y.y - xn.y, y.z - xn.z);
  if (inv3(J, Hn)) {
    xs.x -= Hn[0] * rr.x + Hn[1] * rr.y + Hn[2] * rr.z;
    xs.y -= Hn[3] * rr.x + Hn[4] * rr.y + Hn[5] * rr.z;
    xs.z -= Hn[6] * rr.x + Hn[7] * rr.y + Hn[8] * rr.z;
  }
  return xs;
}

// keep the root with the highest density; equal densities keep the earlier start
__device__ __forceinline__ void take_best(PosedOut& out, float sig, float3 rgb, float3 xs, int start) {
  if (sig > out.sigma || (sig == out.sigma && out.start >= 0 && start < out.start) || out.start < 0) {
    out.sigma = sig;
    out.rgb = rgb;
    out.xstar = xs;
    out.start = start;
  }
}

}  // namespace ia
