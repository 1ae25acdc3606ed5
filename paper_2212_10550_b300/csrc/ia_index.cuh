// Sample and ray indexing (Sec. 3.2 ray samples, Sec. 3.3 occupancy cells).
//
// These functions decide WHICH samples exist: the pixel ray, its clip interval
// against the normalised box, the slot positions and the occupancy cell of each
// slot.  They are written with explicitly rounded intrinsics (__fmul_rn,
// __fadd_rn, __fdiv_rn, __fsqrt_rn), which the compiler never contracts or
// reorders, so the library's sample set is a fixed, documented sequence of
// IEEE fp32 operations:
//   dc   = ((u + 1/2) - cx) / fx, ((v + 1/2) - cy) / fy, 1
//   d_w  = normalize(R_c dc)            (sums left to right)
//   o, d = B_0^-1 applied to the camera centre and d_w
//   slab clip against [norm_min, norm_max], t_n >= 0
//   delta = (t_f - t_n) / N,  t_i = t_n + (i + 1/2) delta,  x_i = o + t_i d
//   cell = floor((x - norm_min) * (R / (norm_max - norm_min))), clamped
#pragma once

#include <cuda_runtime.h>

namespace ia {

struct CamDev {
  float fx, fy, cx, cy;
  int width, height;
  float c2w[12];
};

struct BoxDev {
  float nmin[3], nmax[3];
  float cell_scale[3];  // R / (nmax - nmin)
  float cell_size[3];   // (nmax - nmin) / R
  float sub_scale[3];   // kSub R / (nmax - nmin)
  int R;
};

// Sub-cells of the occupancy grid, kSub^3 per cell, for the root-culling masks:
// the global sub-cell index of x along axis a is floor((x_a - nmin_a) *
// sub_scale_a) in fp32 (monotone in x), and bit sx + kSub (sy + kSub sz) of
// sub[c] stands for sub-cell (kSub c + s) of cell c.
constexpr int kSub = 4;

// False only when the sub-cell holding x meets none of the boxes the culling
// kernel marked, i.e. when no root is possible at x; points outside the grid
// are never excluded.
__device__ __forceinline__ bool sub_marked(const unsigned long long* __restrict__ sub, const BoxDev& bx, float3 x) {
  const float xs[3] = {x.x, x.y, x.z};
  int g[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float f = floorf(__fmul_rn(__fsub_rn(xs[a], bx.nmin[a]), bx.sub_scale[a]));
    if (!(f >= 0.f && f <= (float)(kSub * bx.R - 1))) return true;
    g[a] = (int)f;
  }
  const int cell = g[0] / kSub + bx.R * (g[1] / kSub + bx.R * (g[2] / kSub));
  const int bit = g[0] % kSub + kSub * (g[1] % kSub + kSub * (g[2] % kSub));
  return (__ldg(sub + cell) >> bit) & 1ull;
}

__device__ __forceinline__ float dot3_rn(float a0, float a1, float a2, float b0, float b1, float b2) {
  return __fadd_rn(__fadd_rn(__fmul_rn(a0, b0), __fmul_rn(a1, b1)), __fmul_rn(a2, b2));
}

// World ray (ow, dw) -> normalised space through B_0^-1, then the slab clip
// against the normalised box; returns true if the ray meets the box.
__device__ __forceinline__ bool normalise_and_clip(const float* __restrict__ B0inv, const BoxDev& bx,
                                                   const float ow[3], const float dw[3], float o[3], float d[3],
                                                   float& tn, float& tf) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    o[i] = __fadd_rn(dot3_rn(B0inv[i * 4 + 0], B0inv[i * 4 + 1], B0inv[i * 4 + 2], ow[0], ow[1], ow[2]),
                     B0inv[i * 4 + 3]);
    d[i] = dot3_rn(B0inv[i * 4 + 0], B0inv[i * 4 + 1], B0inv[i * 4 + 2], dw[0], dw[1], dw[2]);
  }
  float tmin = 0.0f, tmax = __int_as_float(0x7f800000);  // +inf
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float inv = __fdiv_rn(1.0f, d[a]);
    const float t0 = __fmul_rn(__fsub_rn(bx.nmin[a], o[a]), inv);
    const float t1 = __fmul_rn(__fsub_rn(bx.nmax[a], o[a]), inv);
    tmin = fmaxf(tmin, fminf(t0, t1));
    tmax = fminf(tmax, fmaxf(t0, t1));
  }
  tn = tmin;
  tf = tmax;
  return tmax > tmin;
}

// Normalised-space ray of pixel (u, v); returns true if it meets the box.
__device__ __forceinline__ bool make_ray(const CamDev& c, const float* __restrict__ B0inv, const BoxDev& bx,
                                         int u, int v, float o[3], float d[3], float& tn, float& tf) {
  const float dc0 = __fdiv_rn(__fsub_rn(__fadd_rn((float)u, 0.5f), c.cx), c.fx);
  const float dc1 = __fdiv_rn(__fsub_rn(__fadd_rn((float)v, 0.5f), c.cy), c.fy);
  float dw[3], ow[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dw[i] = dot3_rn(c.c2w[i * 4 + 0], c.c2w[i * 4 + 1], c.c2w[i * 4 + 2], dc0, dc1, 1.0f);
    ow[i] = c.c2w[i * 4 + 3];
  }
  const float nrm = __fsqrt_rn(dot3_rn(dw[0], dw[1], dw[2], dw[0], dw[1], dw[2]));
#pragma unroll
  for (int i = 0; i < 3; ++i) dw[i] = __fdiv_rn(dw[i], nrm);
  return normalise_and_clip(B0inv, bx, ow, dw, o, d, tn, tf);
}

__device__ __forceinline__ float slot_delta(float tn, float tf, int n_slots) {
  return __fdiv_rn(__fsub_rn(tf, tn), (float)n_slots);
}

__device__ __forceinline__ float3 slot_position(const float o[3], const float d[3], float tn, float dt, int i) {
  const float t = __fadd_rn(tn, __fmul_rn(__fadd_rn((float)i, 0.5f), dt));
  return make_float3(__fadd_rn(o[0], __fmul_rn(t, d[0])), __fadd_rn(o[1], __fmul_rn(t, d[1])),
                     __fadd_rn(o[2], __fmul_rn(t, d[2])));
}

__device__ __forceinline__ int cell_of(const BoxDev& bx, float3 x) {
  const float xs[3] = {x.x, x.y, x.z};
  int c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int q = (int)floorf(__fmul_rn(__fsub_rn(xs[a], bx.nmin[a]), bx.cell_scale[a]));
    c[a] = min(max(q, 0), bx.R - 1);
  }
  return c[0] + bx.R * (c[1] + bx.R * c[2]);
}

__device__ __forceinline__ float3 cell_center(const BoxDev& bx, int cell) {
  const int c[3] = {cell % bx.R, (cell / bx.R) % bx.R, cell / (bx.R * bx.R)};
  float x[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    x[a] = __fadd_rn(bx.nmin[a], __fmul_rn(__fadd_rn((float)c[a], 0.5f), bx.cell_size[a]));
  return make_float3(x[0], x[1], x[2]);
}

// a point inside the cell: norm_min + (c + u) * cell size, u in [0, 1)^3 (fp32,
// the operation order of cell_center, which is u = 1/2)
__device__ __forceinline__ float3 cell_point(const BoxDev& bx, int cell, const float* __restrict__ u) {
  const int c[3] = {cell % bx.R, (cell / bx.R) % bx.R, cell / (bx.R * bx.R)};
  float x[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) x[a] = __fadd_rn(bx.nmin[a], __fmul_rn(__fadd_rn((float)c[a], u[a]), bx.cell_size[a]));
  return make_float3(x[0], x[1], x[2]);
}

}  // namespace ia
