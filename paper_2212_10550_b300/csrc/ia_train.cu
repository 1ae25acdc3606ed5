// Training step of the articulated radiance-field path: L2 photometric loss and
// its hand-written backward (sm_103a; fp32, or fp16 / bf16 operands with fp32
// accumulation and master gradients).
//
//   train_count_kernel,     world rays -> normalised space of each ray's pose,
//   pose_scan_kernel,       occupied slots; samples compacted and grouped by
//   train_emit_kernel       pose (count, per-pose offsets, emit); the density
//   (reg_*_kernel)          regulariser's points in empty cells join them
//   train_sample_kernel     posed field f'(x') at every sample (same warp-level
//                           correspondence search as rendering, per-lane pose)
//   train_composite_kernel  per ray: front-to-back compositing, loss, and its
//                           reverse: dL/dsigma_i, dL/dc_i (Sec. 3.2, Eq. 8)
//   train_backward_kernel   per sample: recomputed hash encoding and MLP
//                           activations, MLP backward to the features, hash-table
//                           scatter-add, canonical-position gradient, and the
//                           implicit-function gradient through the root
//                           (lambda = J^-T dL/dx*) to bone transforms and the
//                           skinning-weight grid
//   mlp_grad_kernel         weight gradients dW = sum_s dH_s^T A_s as split-K
//                           reductions over the samples
//
// In fp16 / bf16 the forward runs the tensor-core field, train_backward_h_kernel
// replaces the per-sample backward (loss-scaled, channel-major operands), and
// the weight gradients come from the tcgen05 GEMM of wgrad_tc_kernel; a
// loss-scale update closes the step.
//
// Per-sample activations are recomputed from x* in the backward (nothing of the
// MLP is kept from the forward); the backward writes them once, next to their
// gradients, for the weight-gradient reduction.
#include "ia_internal.h"
#include "ia_tcgen05.cuh"

namespace ia {

constexpr int kActF = 0, kActH1 = kIn, kActH2 = kActH1 + kWidth, kActD1 = kActH2 + kWidth,
              kActD2 = kActD1 + kWidth, kActDO = kActD2 + kWidth;

// ---------------------------------------------------------------------------

// March of one training ray in the normalised space of its pose: the occupied
// slots in march order, except those whose point can have no root in that pose
// (the pose's root-culling masks, when present: density 0 and no gradient, so
// they change neither the ray's colour nor any gradient; counted in *culled).
// A warp per ray, its lanes over the slots (every 32nd slot per lane; the
// ballots keep march order).  Returns the count (all lanes); emit(j, x) is
// called by the lane holding the ray's j-th sample.  A ray per thread left the
// GPU mostly idle at training batch sizes (32768 rays: 1024 warps, each lane
// marching 128 slots in turn).
template <typename Emit>
__device__ __forceinline__ int march_train_ray_warp(const TrainArgs& a, int r, int& pose, int& hit, float& dt,
                                                    Emit emit, int* culled) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  pose = a.pose[r];
  hit = 0;
  dt = 0.f;
  *culled = 0;
  if (pose < 0 || pose >= a.n_poses) return 0;
  const float ow[3] = {a.origin[3 * r], a.origin[3 * r + 1], a.origin[3 * r + 2]};
  const float dw[3] = {a.direction[3 * r], a.direction[3 * r + 1], a.direction[3 * r + 2]};
  float o[3], d[3], tn, tf;
  if (!normalise_and_clip(a.B0inv + 12 * (size_t)pose, a.box, ow, dw, o, d, tn, tf)) return 0;
  hit = 1;
  dt = slot_delta(tn, tf, a.n_slots);
  const unsigned long long* sub =
      a.sub ? a.sub + (size_t)pose * a.box.R * a.box.R * a.box.R : nullptr;
  int n = 0, nc = 0;
  for (int i0 = 0; i0 < a.n_slots; i0 += 32) {
    const int i = i0 + lane;
    bool keep = false, cull = false;
    float3 x = make_float3(0.f, 0.f, 0.f);
    if (i < a.n_slots) {
      x = slot_position(o, d, tn, dt, i);
      const int cell = cell_of(a.box, x);
      if ((__ldg(a.occ + (cell >> 5)) >> (cell & 31)) & 1u) {
        if (sub && !sub_marked(sub, a.box, x)) cull = true;
        else keep = true;
      }
    }
    const unsigned m = __ballot_sync(kFull, keep);
    nc += __popc(__ballot_sync(kFull, cull));
    if (keep) emit(n + __popc(m & lt), x);
    n += __popc(m);
  }
  *culled = nc;
  return n;
}

// pass 1: per-ray sample counts and per-pose totals (a warp per ray; the
// counters are summed over the block first: one atomic per block and counter)
__global__ void __launch_bounds__(256) train_count_kernel(const TrainArgs a) {
  __shared__ int s_st[5][8];
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, warp = threadIdx.x >> 5;
  const bool l0 = (threadIdx.x & 31) == 0;
  int n = 0, hit = 0, culled = 0;
  if (r < a.n_rays) {
    int pose;
    float dt;
    n = march_train_ray_warp(a, r, pose, hit, dt, [](int, float3) {}, &culled);
    if (l0) {
      a.ray_n[r] = n;
      a.ray_dt[r] = dt;
      if (n > 0) atomicAdd(a.pose_tot + pose, n);
    }
  }
  if (l0) {
    s_st[0][warp] = r < a.n_rays ? 1 : 0;
    s_st[1][warp] = hit;
    s_st[2][warp] = hit ? a.n_slots : 0;
    s_st[3][warp] = n + culled;
    s_st[4][warp] = culled;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    unsigned long long v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += (unsigned long long)s_st[threadIdx.x][w];
    const int idx[5] = {ST_RAYS, ST_HIT, ST_MARCHED, ST_OCC, ST_CULLED};
    if (v) atomicAdd(a.stats + idx[threadIdx.x], v);
  }
}

// pass 2: per-pose totals -> first sample index of each pose; total count
__global__ void pose_scan_kernel(const TrainArgs a) {
  if (threadIdx.x != 0) return;
  int run = 0;
  for (int p = 0; p < a.n_poses; ++p) {
    const int t = a.pose_tot[p];
    a.pose_tot[p] = run;
    run += t;
  }
  *a.count = run;
}

// pass 3: samples written grouped by pose (so that concurrent warps of the
// sample kernels share one pose's blended grid in L2), each ray's list of its
// sample indices in march order (a warp per ray)
__global__ void __launch_bounds__(256) train_emit_kernel(const TrainArgs a) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= a.n_rays) return;  // whole warps
  const int n = a.ray_n[r];
  if (n == 0) return;
  const int pose = a.pose[r];
  int base = 0;
  if ((threadIdx.x & 31) == 0) base = a.pose_tot[pose] + atomicAdd(a.pose_fill + pose, n);
  base = __shfl_sync(kFull, base, 0);
  int p, hit, culled;
  float dt;
  int* idx = a.ray_idx + (size_t)r * a.n_slots;
  march_train_ray_warp(
      a, r, p, hit, dt,
      [&](int j, float3 x) {
        a.s_pos[base + j] = make_float4(x.x, x.y, x.z, __int_as_float(pose));
        idx[j] = base + j;
      },
      &culled);
}

// Regulariser points (Eq. 12): only points in empty cells of the step's grid
// are samples.  Pass 1 counts them per pose (with the rays' counts) ...
__global__ void reg_count_kernel(const TrainArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_reg) return;
  const int pose = a.reg_pose[i];
  bool keep = false;
  if (pose >= 0 && pose < a.n_poses) {
    const float3 x = make_float3(a.reg_x[3 * i], a.reg_x[3 * i + 1], a.reg_x[3 * i + 2]);
    const int cell = cell_of(a.box, x);
    keep = !((__ldg(a.occ + (cell >> 5)) >> (cell & 31)) & 1u);
    // a point that can have no root has density 0: no loss, no gradient
    if (keep && a.sub) keep = sub_marked(a.sub + (size_t)pose * a.box.R * a.box.R * a.box.R, a.box, x);
  }
  a.reg_idx[i] = keep ? 0 : -1;
  if (keep) atomicAdd(a.pose_tot + pose, 1);
}

// ... pass 3 places them among their pose's samples
__global__ void reg_emit_kernel(const TrainArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_reg || a.reg_idx[i] < 0) return;
  const int pose = a.reg_pose[i];
  const int j = a.pose_tot[pose] + atomicAdd(a.pose_fill + pose, 1);
  a.s_pos[j] = make_float4(a.reg_x[3 * i], a.reg_x[3 * i + 1], a.reg_x[3 * i + 2], __int_as_float(pose));
  a.reg_idx[i] = j;
}

// after the forward: the regulariser's loss, weight / n_reg * sum sigma, and the
// density gradient of its samples (sigma >= 0, so d|sigma| / d sigma = 1)
__global__ void reg_grad_kernel(const TrainArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = i < a.n_reg ? a.reg_idx[i] : -1;
  const float w = a.reg_weight / (float)a.n_reg;
  float l = 0.f;
  if (j >= 0) {
    const float4 o = a.s_out[j];
    l = w * o.x;
    a.s_grad[j] = make_float4(o.x > 0.f ? w : 0.f, 0.f, 0.f, 0.f);
  }
  for (int d = 16; d > 0; d >>= 1) l += __shfl_down_sync(kFull, l, d);
  if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(a.loss, l);
}

// The step's own loss for ray r (Sec. 3.4, Eq. 9-11), averaged over the rays
// and added to *a.loss (one atomic per warp; every lane of the warp calls), and
// its gradients g = dL/dC, ga = dL/dalpha.
__device__ __forceinline__ void composite_loss(const TrainArgs& a, int r, bool active, const float C[3], float depth,
                                               float g[3], float& ga) {
  const float inv_n = 1.f / (float)a.n_rays;
  float e[3], ee = 0.f;
  for (int k = 0; k < 3; ++k) {
    e[k] = active ? C[k] - a.target[3 * r + k] : 0.f;
    ee = fmaf(e[k], e[k], ee);
  }
  // colour term (Eq. 9): L2 over channels, or Huber of the colour error's norm
  float lr;
  if (!a.huber) {
    lr = ee;
    for (int k = 0; k < 3; ++k) g[k] = 2.f * e[k];
  } else {
    const float rn = sqrtf(ee);
    if (rn <= a.huber_delta) {
      lr = 0.5f * ee;
      for (int k = 0; k < 3; ++k) g[k] = e[k];
    } else {
      lr = a.huber_delta * (rn - 0.5f * a.huber_delta);
      for (int k = 0; k < 3; ++k) g[k] = a.huber_delta * e[k] / rn;
    }
  }
  for (int k = 0; k < 3; ++k) g[k] *= a.w_rgb * inv_n;
  // opacity terms of alpha = 1 - T_N: L1 to the mask (Eq. 10), hard surface (Eq. 11)
  const float alpha = -expm1f(-depth);
  float la = 0.f;
  ga = 0.f;
  if (active && a.w_alpha != 0.f) {
    const float da = alpha - a.alpha_target[r];
    la += a.w_alpha * fabsf(da);
    ga += a.w_alpha * (da > 0.f ? 1.f : (da < 0.f ? -1.f : 0.f));
  }
  if (active && a.w_hard != 0.f) {
    const float e0 = expf(-fabsf(alpha)), e1 = expf(-fabsf(alpha - 1.f));
    la += a.w_hard * (-logf(e0 + e1) + 0.31326169f);  // log(1 + e^-1): zero at alpha in {0, 1}
    const float s0 = alpha > 0.f ? 1.f : (alpha < 0.f ? -1.f : 0.f);
    const float s1 = alpha > 1.f ? 1.f : (alpha < 1.f ? -1.f : 0.f);
    ga += a.w_hard * (s0 * e0 + s1 * e1) / (e0 + e1);
  }
  ga *= inv_n;
  float lw = active ? (a.w_rgb * lr + la) * inv_n : 0.f;
  for (int o = 16; o > 0; o >>= 1) lw += __shfl_down_sync(kFull, lw, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(a.loss, lw);
}

// The reverse sweep over the ray's samples in march order: dL/dsigma_i and
// dL/dc_i into s_grad (zero for samples without a root).
__device__ __forceinline__ void reverse_sweep(const TrainArgs& a, int n, float dt, const int* idx, const float C[3],
                                              float TN, const float g[3], float ga) {
  float Cle[3] = {0.f, 0.f, 0.f}, depth = 0.f;
  for (int j = 0; j < n; ++j) {
    const int s = idx[j];
    const float4 o = a.s_out[s];
    if (!(o.x > 0.f)) {
      a.s_grad[s] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const float sd = o.x * dt;
    const float T = expf(-depth), Tn = expf(-(depth + sd)), w = T * -expm1f(-sd);
    Cle[0] = fmaf(w, o.y, Cle[0]);
    Cle[1] = fmaf(w, o.z, Cle[1]);
    Cle[2] = fmaf(w, o.w, Cle[2]);
    const float cg = o.y * g[0] + o.z * g[1] + o.w * g[2];
    const float rest = g[0] * (C[0] - Cle[0]) + g[1] * (C[1] - Cle[1]) + g[2] * (C[2] - Cle[2]);
    a.s_grad[s] = make_float4(dt * (Tn * cg - rest) + ga * dt * TN, w * g[0], w * g[1], w * g[2]);
    depth += sd;
  }
}

// Front-to-back compositing of one ray, the loss, and the reverse sweep
//   dL/dc_i = T_i alpha_i g,
//   dL/dsigma_i = delta (T_{i+1} c_i.g - g.(C - C_{<=i})) + g_alpha delta T_N
// with g = dL/dC and g_alpha = dL/dalpha for the ray's alpha = 1 - T_N
// (Sec. 3.2, Eq. 8; loss terms of Sec. 3.4, Eq. 9-11).  a.comp_mode selects
// where g and g_alpha come from: kCompLoss -- the step's loss; kCompUpstream --
// the caller's per-ray gradients (a.up_rgb, a.up_alpha: the reverse sweep of a
// loss computed elsewhere); kCompForward -- no reverse sweep, only the ray's
// colour and alpha are written.
__global__ void train_composite_kernel(const TrainArgs a) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = r < a.n_rays;
  const int n = active ? a.ray_n[r] : 0;
  const float dt = active ? a.ray_dt[r] : 0.f;
  const int* idx = a.ray_idx + (size_t)(active ? r : 0) * a.n_slots;
  float C[3] = {0.f, 0.f, 0.f}, depth = 0.f;
  for (int j = 0; j < n; ++j) {
    const float4 o = a.s_out[idx[j]];
    if (o.x > 0.f) {
      const float sd = o.x * dt;
      const float w = expf(-depth) * -expm1f(-sd);
      C[0] = fmaf(w, o.y, C[0]);
      C[1] = fmaf(w, o.z, C[1]);
      C[2] = fmaf(w, o.w, C[2]);
      depth += sd;
    }
  }
  if (active && a.rgb_out)
    for (int k = 0; k < 3; ++k) a.rgb_out[3 * r + k] = C[k];
  if (active && a.alpha_out) a.alpha_out[r] = -expm1f(-depth);
  if (a.comp_mode == kCompForward) return;
  float g[3], ga;
  if (a.comp_mode == kCompUpstream) {
    if (!active) return;
    for (int k = 0; k < 3; ++k) g[k] = a.up_rgb[3 * r + k];
    ga = a.up_alpha ? a.up_alpha[r] : 0.f;
  } else {
    composite_loss(a, r, active, C, depth, g, ga);
    if (!active) return;
  }
  const float TN = expf(-depth);
  reverse_sweep(a, n, dt, idx, C, TN, g, ga);
}
// ---------------------------------------------------------------------------
// Per-sample backward
// ---------------------------------------------------------------------------

// Warp-wide sums of 16 per-lane values, scattered: lane l returns the sum over
// all 32 lanes of v[(l >> 1) & 15] (reduce-scatter by recursive halving, 16
// shuffles instead of 80).  All 32 lanes call; v is clobbered.
__device__ __forceinline__ float warp_reduce_scatter16(float v[16], int lane) {
#pragma unroll
  for (int step = 0; step < 4; ++step) {
    const int half = 8 >> step, off = 16 >> step;
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = upper ? v[i] : v[half + i];
      const float keep = upper ? v[half + i] : v[i];
      v[i] = keep + __shfl_xor_sync(kFull, send, off);
    }
  }
  return v[0] + __shfl_xor_sync(kFull, v[0], 1);
}

// dL/dx* -> lambda = J(x*)^-T dL/dx* -> bone-transform and skinning-grid
// gradients.  All 32 lanes call (has = this lane carries a sample with a root).
// When every contributing lane of the warp holds the same pose (the usual case:
// samples are grouped by pose), the bone-transform gradient is summed over the
// warp first and added with one atomic per entry.
__device__ __forceinline__ void ift_scatter_warp(const TrainArgs& a, bool has, int pose, float3 xs, float gx,
                                                 float gy, float gz) {
  const int nb = a.P.cfg.nb, lane = threadIdx.x & 31;
  float l0 = 0.f, l1 = 0.f, l2 = 0.f;
  bool ok = false;
  if (has) {
    const float4* M = a.P.S.M + (size_t)pose * a.V * 3;
    float Mx[12], J[9], Hi[9];
    blend_value_jac(a.P.S, M, xs, Mx, J);
    ok = inv3(J, Hi);
    if (ok) {
      l0 = Hi[0] * gx + Hi[3] * gy + Hi[6] * gz;
      l1 = Hi[1] * gx + Hi[4] * gy + Hi[7] * gz;
      l2 = Hi[2] * gx + Hi[5] * gy + Hi[8] * gz;
    }
  }
  const unsigned okm = __ballot_sync(kFull, ok);
  if (okm == 0) return;
  const int p0 = __shfl_sync(kFull, pose, __ffs(okm) - 1);
  const bool uniform = __all_sync(kFull, !ok || pose == p0);
  const float xb[4] = {xs.x, xs.y, xs.z, 1.f};
  // trilinear coefficients of x* in the skinning grid (as the forward blends them)
  CellCoord cc = skin_cell(a.P.S, ok ? xs : make_float3(a.P.S.cmin[0], a.P.S.cmin[1], a.P.S.cmin[2]));
  const float* Np = a.N + (size_t)(ok ? pose : p0) * nb * 12;
  float cwc[8];
  int vc[8];
#pragma unroll
  for (int corner = 0; corner < 8; ++corner) {
    vc[corner] = corner_index(a.P.S, cc.base, corner);
    cwc[corner] = ((corner & 1) ? cc.f[0] : 1.f - cc.f[0]) * (((corner >> 1) & 1) ? cc.f[1] : 1.f - cc.f[1]) *
                  (((corner >> 2) & 1) ? cc.f[2] : 1.f - cc.f[2]);
  }
  // bones in groups of four: with a.skin_vec (nb % 4 == 0 and 16-byte aligned
  // grids, checked by the host) one float4 load and one float4 atomic per corner
  // serve four bones of the [v][nb] layout; otherwise one bone at a time
  for (int k0 = 0; k0 < nb; k0 += 4) {
    float wk4[4] = {0.f, 0.f, 0.f, 0.f};
    if (ok) {
#pragma unroll
      for (int corner = 0; corner < 8; ++corner) {
        const float* src = a.skin + (size_t)vc[corner] * nb + k0;
        float4 w4;
        if (a.skin_vec) {
          w4 = __ldg(reinterpret_cast<const float4*>(src));
        } else {
          w4.x = __ldg(src);
          w4.y = k0 + 1 < nb ? __ldg(src + 1) : 0.f;
          w4.z = k0 + 2 < nb ? __ldg(src + 2) : 0.f;
          w4.w = k0 + 3 < nb ? __ldg(src + 3) : 0.f;
        }
        wk4[0] = fmaf(cwc[corner], w4.x, wk4[0]);
        wk4[1] = fmaf(cwc[corner], w4.y, wk4[1]);
        wk4[2] = fmaf(cwc[corner], w4.z, wk4[2]);
        wk4[3] = fmaf(cwc[corner], w4.w, wk4[3]);
      }
    }
    float ln4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int k = k0 + kk;
      if (k >= nb) break;  // uniform across the warp
      const float wk = wk4[kk];
      // dL/dN_k[a][b] = -lambda_a w_k [x*;1]_b
      if (uniform) {
        float v[16];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          v[b] = -l0 * wk * xb[b];
          v[4 + b] = -l1 * wk * xb[b];
          v[8 + b] = -l2 * wk * xb[b];
          v[12 + b] = 0.f;
        }
        const float sum = warp_reduce_scatter16(v, lane);
        const int idx = (lane >> 1) & 15;
        if ((lane & 1) == 0 && idx < 12) atomicAdd(a.g_bones + ((size_t)p0 * nb + k) * 12 + idx, sum);
      } else if (ok) {
        float* gB = a.g_bones + ((size_t)pose * nb + k) * 12;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          atomicAdd(gB + b, -l0 * wk * xb[b]);
          atomicAdd(gB + 4 + b, -l1 * wk * xb[b]);
          atomicAdd(gB + 8 + b, -l2 * wk * xb[b]);
        }
      }
      // dL/dW(v, k) = -c_v lambda . (N_k [x*;1])
      const float* Nk = Np + 12 * k;
      ln4[kk] = l0 * (Nk[0] * xb[0] + Nk[1] * xb[1] + Nk[2] * xb[2] + Nk[3]) +
                l1 * (Nk[4] * xb[0] + Nk[5] * xb[1] + Nk[6] * xb[2] + Nk[7]) +
                l2 * (Nk[8] * xb[0] + Nk[9] * xb[1] + Nk[10] * xb[2] + Nk[11]);
    }
    if (ok) {
#pragma unroll
      for (int corner = 0; corner < 8; ++corner) {
        const float c = -cwc[corner];
        float* dst = a.g_skin + (size_t)vc[corner] * nb + k0;
        if (a.skin_vec) {
          atomicAdd(reinterpret_cast<float4*>(dst), make_float4(c * ln4[0], c * ln4[1], c * ln4[2], c * ln4[3]));
        } else {
          for (int kk = 0; kk < 4 && k0 + kk < nb; ++kk) atomicAdd(dst + kk, c * ln4[kk]);
        }
      }
    }
  }
}

// hash-table scatter of dL/dfeatures and the canonical-position gradient dL/dx*
template <bool kHalfTable>
__device__ __forceinline__ void hash_backward(const TrainArgs& a, float3 xs, const float dfeat[kIn], float& gx,
                                              float& gy, float& gz) {
  const FieldDev& F = a.P.F;
  gx = gy = gz = 0.f;
  const float u[3] = {(xs.x - F.cmin[0]) * F.inv_ext[0], (xs.y - F.cmin[1]) * F.inv_ext[1],
                      (xs.z - F.cmin[2]) * F.inv_ext[2]};
#pragma unroll
  for (int l = 0; l < kMaxLevels; ++l) {
    if (l < F.L) {
      const Level lv = F.lv[l];
      int p0[3];
      float f[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float pos = u[q] * (float)lv.res;
        int c = (int)floorf(pos);
        c = min(max(c, 0), lv.res - 1);
        p0[q] = c;
        f[q] = pos - (float)c;
      }
      const float d0 = dfeat[2 * l], d1 = dfeat[2 * l + 1];
      const float sx = (float)lv.res * F.inv_ext[0], sy = (float)lv.res * F.inv_ext[1],
                  sz = (float)lv.res * F.inv_ext[2];
#pragma unroll
      for (int corner = 0; corner < 8; ++corner) {
        const int cx = corner & 1, cy = (corner >> 1) & 1, cz = (corner >> 2) & 1;
        const float wx = cx ? f[0] : 1.f - f[0], wy = cy ? f[1] : 1.f - f[1], wz = cz ? f[2] : 1.f - f[2];
        const uint32_t e = lv.offset + vertex_index(lv, p0[0] + cx, p0[1] + cy, p0[2] + cz);
        const float w = wx * wy * wz;
        // one 8-byte vector atomic per entry (the host checks the alignment)
        atomicAdd(reinterpret_cast<float2*>(a.g_table) + e, make_float2(w * d0, w * d1));
        float2 t;
        if constexpr (kHalfTable) t = __half22float2(a.P.table_h[e]);
        else t = __ldg(F.table + e);
        const float proj = t.x * d0 + t.y * d1;
        gx = fmaf(proj * (cx ? 1.f : -1.f) * wy * wz, sx, gx);
        gy = fmaf(proj * (cy ? 1.f : -1.f) * wx * wz, sy, gy);
        gz = fmaf(proj * (cz ? 1.f : -1.f) * wx * wy, sz, gz);
      }
    }
  }
}


// The backward's scatter, in two kernels so that each one's working set stays
// in L2 (one kernel reading the hash table, the skinning grid and the poses'
// blended grids while scatter-adding into the table and skinning-grid
// gradients re-read its lines from DRAM about four times over):
//  train_hash_grad_kernel: hash-table gradient (trilinear weights of
//    dL/dfeatures) and dL/dx*, one thread per sample, dL/dx* into s_gx;
//  train_ift_kernel: the implicit-function gradient to the bone transforms
//    and the skinning grid, warps walking the samples in order (grouped by
//    pose, so a pose's blended grid stays in L2).
template <bool kHalfTable>
__global__ void __launch_bounds__(256) train_hash_grad_kernel(const TrainArgs a) {
  const int n = *a.count;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const float4 x4 = a.s_x[s];
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (x4.w > 0.f) {
      float dfeat[kIn];
      const float4* src = a.s_dfeat + (size_t)s * (kIn / 4);
#pragma unroll
      for (int i = 0; i < kIn / 4; ++i) {
        const float4 v = src[i];
        dfeat[4 * i] = v.x;
        dfeat[4 * i + 1] = v.y;
        dfeat[4 * i + 2] = v.z;
        dfeat[4 * i + 3] = v.w;
      }
      hash_backward<kHalfTable>(a, make_float3(x4.x, x4.y, x4.z), dfeat, g.x, g.y, g.z);
    }
    a.s_gx[s] = g;
  }
}

__global__ void __launch_bounds__(256) train_ift_kernel(const TrainArgs a) {
  const int n = *a.count;
  const int lane = threadIdx.x & 31;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int s = base + lane;
    bool has = false;
    float3 xs = make_float3(0.f, 0.f, 0.f);
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    int pose = 0;
    if (s < n) {
      const float4 x4 = a.s_x[s];
      has = x4.w > 0.f;
      xs = make_float3(x4.x, x4.y, x4.z);
      pose = __float_as_int(a.s_pos[s].w);
      g = a.s_gx[s];
    }
    ift_scatter_warp(a, has, pose, xs, g.x, g.y, g.z);
  }
}

static cudaError_t launch_scatter(const TrainArgs& a, bool half_table, int num_sms, cudaStream_t s) {
  cudaError_t e;
  {
    KernelSpan span("train_hash_grad_kernel", s);
    if (half_table) train_hash_grad_kernel<true><<<num_sms * 8, 256, 0, s>>>(a);
    else train_hash_grad_kernel<false><<<num_sms * 8, 256, 0, s>>>(a);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    KernelSpan span("train_ift_kernel", s);
    train_ift_kernel<<<num_sms * 8, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// The 64-wide loops run rolled (a fully unrolled body does not fit the
// instruction cache); a vector that a rolled loop indexes by its counter lives
// in this thread's column of a shared array (vec[j * 128 + thread]: lanes hit
// consecutive banks), which each thread reuses for h1, then dH2, then dH1.
// Sums keep the order of the plain definition (inputs ascending).
constexpr int kBwdThreads = 256;  // threads of the fp32 backward (two blocks of eight warps per SM)

__global__ void __launch_bounds__(kBwdThreads) train_backward_kernel(const TrainArgs a) {
  __shared__ __align__(16) float sw[kMlpPadT];
  extern __shared__ float vec[];  // [kWidth * kBwdThreads], dynamic (static shared memory stops at 48 KB)
  stage_mlp(a.P.mlp, a.P.n_in, sw);
  __syncthreads();
  const int n = *a.count;
  const FieldDev& F = a.P.F;
  float* my = vec + threadIdx.x;  // my[j * kBwdThreads]: entry j of this thread's vector
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    // this sample's column of the channel-major activations: act[c * ld] is
    // channel c (consecutive lanes write consecutive addresses)
    float* act = a.act + s;
    const int64_t ld = a.act_ld;
    const float4 xs4 = a.s_x[s];
    if (!(xs4.w > 0.f)) {  // no root: no gradient; zero columns keep the reduction exact
      for (int q = 0; q < kActStride; ++q) act[q * ld] = 0.f;
      continue;
    }
    const float3 xs = make_float3(xs4.x, xs4.y, xs4.z);
    const float4 gr = a.s_grad[s];
    // ---- recompute the forward activations
    float feat[kIn];
    encode(F, xs, feat);
#pragma unroll
    for (int i = 0; i < kIn; ++i) act[(kActF + i) * ld] = feat[i];
    uint64_t m1 = 0;  // h1 > 0 mask
#pragma unroll 1
    for (int j = 0; j < kWidth; ++j) {
      float acc = sw[kOffB1 + j];
      const float4* row = reinterpret_cast<const float4*>(sw + kOffW1 + j * kIn);
#pragma unroll
      for (int i = 0; i < kIn / 4; ++i) {
        float4 w = row[i];
        acc = fmaf(w.x, feat[4 * i], fmaf(w.y, feat[4 * i + 1], fmaf(w.z, feat[4 * i + 2], fmaf(w.w, feat[4 * i + 3], acc))));
      }
      const float h = fmaxf(acc, 0.f);
      if (acc > 0.f) m1 |= 1ull << j;
      my[j * kBwdThreads] = h;
      act[(kActH1 + j) * ld] = h;
    }
    float h1[kWidth];
#pragma unroll
    for (int i = 0; i < kWidth; ++i) h1[i] = my[i * kBwdThreads];
    float o0 = sw[kOffB3], o1 = sw[kOffB3 + 1], o2 = sw[kOffB3 + 2], o3 = sw[kOffB3 + 3];
    uint64_t m2 = 0;  // h2 > 0 mask
#pragma unroll 1
    for (int j = 0; j < kWidth; ++j) {
      float acc = sw[kOffB2 + j];
      const float4* row = reinterpret_cast<const float4*>(sw + kOffW2 + j * kWidth);
#pragma unroll
      for (int i = 0; i < kWidth / 4; ++i) {
        float4 w = row[i];
        acc = fmaf(w.x, h1[4 * i], fmaf(w.y, h1[4 * i + 1], fmaf(w.z, h1[4 * i + 2], fmaf(w.w, h1[4 * i + 3], acc))));
      }
      const float h = fmaxf(acc, 0.f);
      act[(kActH2 + j) * ld] = h;
      if (acc > 0.f) m2 |= 1ull << j;
      const float4 w3 = reinterpret_cast<const float4*>(sw + kOffW3T)[j];
      o0 = fmaf(w3.x, h, o0);
      o1 = fmaf(w3.y, h, o1);
      o2 = fmaf(w3.z, h, o2);
      o3 = fmaf(w3.w, h, o3);
    }
    // ---- activations: sigma = exp(clamp(o0)), c = sigmoid
    float dO[4];
    {
      const float sig = expf(fminf(fmaxf(o0, -15.f), 15.f));
      dO[0] = (o0 > -15.f && o0 < 15.f) ? gr.x * sig : 0.f;
      const float oc[3] = {o1, o2, o3}, gc[3] = {gr.y, gr.z, gr.w};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float sg = 1.f / (1.f + expf(-oc[c]));
        dO[1 + c] = gc[c] * sg * (1.f - sg);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) act[(kActDO + q) * ld] = dO[q];
    // ---- MLP backward to the features
#pragma unroll 1
    for (int j = 0; j < kWidth; ++j) {
      const float4 w3 = reinterpret_cast<const float4*>(sw + kOffW3T)[j];
      const float v = w3.x * dO[0] + w3.y * dO[1] + w3.z * dO[2] + w3.w * dO[3];
      const float d = ((m2 >> j) & 1ull) ? v : 0.f;
      my[j * kBwdThreads] = d;  // dH2 (h1 is in registers now)
      act[(kActD2 + j) * ld] = d;
    }
    float dh1[kWidth];
#pragma unroll
    for (int i = 0; i < kWidth; ++i) dh1[i] = 0.f;
#pragma unroll 1
    for (int j = 0; j < kWidth; ++j) {
      const float4* row = reinterpret_cast<const float4*>(sw + kOffW2 + j * kWidth);
      const float d = my[j * kBwdThreads];
#pragma unroll
      for (int i = 0; i < kWidth / 4; ++i) {
        float4 w = row[i];
        dh1[4 * i] = fmaf(w.x, d, dh1[4 * i]);
        dh1[4 * i + 1] = fmaf(w.y, d, dh1[4 * i + 1]);
        dh1[4 * i + 2] = fmaf(w.z, d, dh1[4 * i + 2]);
        dh1[4 * i + 3] = fmaf(w.w, d, dh1[4 * i + 3]);
      }
    }
#pragma unroll
    for (int i = 0; i < kWidth; ++i) my[i * kBwdThreads] = dh1[i];
    float dfeat[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) dfeat[i] = 0.f;
#pragma unroll 1
    for (int j = 0; j < kWidth; ++j) {
      const float d = ((m1 >> j) & 1ull) ? my[j * kBwdThreads] : 0.f;
      act[(kActD1 + j) * ld] = d;
      const float4* row = reinterpret_cast<const float4*>(sw + kOffW1 + j * kIn);
#pragma unroll
      for (int i = 0; i < kIn / 4; ++i) {
        float4 w = row[i];
        dfeat[4 * i] = fmaf(w.x, d, dfeat[4 * i]);
        dfeat[4 * i + 1] = fmaf(w.y, d, dfeat[4 * i + 1]);
        dfeat[4 * i + 2] = fmaf(w.z, d, dfeat[4 * i + 2]);
        dfeat[4 * i + 3] = fmaf(w.w, d, dfeat[4 * i + 3]);
      }
    }
    // ---- dL/dfeatures for the scatter kernel
    float4* dst = a.s_dfeat + (size_t)s * (kIn / 4);
#pragma unroll
    for (int i = 0; i < kIn / 4; ++i) dst[i] = make_float4(dfeat[4 * i], dfeat[4 * i + 1], dfeat[4 * i + 2], dfeat[4 * i + 3]);
  }
}

// ---------------------------------------------------------------------------
// Weight gradients: gW1 = sum_s dH1_s^T F_s, gW2 = sum_s dH2_s^T H1_s,
// gW3 = sum_s dO_s^T H2_s, biases = sums of dH1, dH2, dO.  Split-K over samples:
// each block reduces a contiguous chunk in registers (32-sample tiles staged in
// shared memory) and adds its partial sums to the gradient once.
// ---------------------------------------------------------------------------

constexpr int kTileS = 32;

constexpr int kTilePitch = kActStride + 4;  // 16-byte rows: the operands are read as float4 / float2

__global__ void __launch_bounds__(256) mlp_grad_kernel(const TrainArgs a) {
  __shared__ __align__(16) float tile[kTileS][kTilePitch];
  const int n = *a.count;
  const int chunk = (n + gridDim.x - 1) / gridDim.x;
  const int s0 = blockIdx.x * chunk, s1 = min(n, s0 + chunk);
  const int t = threadIdx.x;
  const int n_in = a.P.n_in;
  // ownership: gW2 4x4 block, gW1 4x2 block, gW3 one entry, one bias entry
  const int i2 = (t / 16) * 4, j2 = (t % 16) * 4;
  const int i1 = (t / 16) * 4, j1 = (t % 16) * 2;
  const int o3 = t / 64, j3 = t % 64;
  float acc2[16], acc1[8], acc3 = 0.f, accb = 0.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) acc2[q] = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) acc1[q] = 0.f;
  for (int base = s0; base < s1; base += kTileS) {
    const int m = min(kTileS, s1 - base);
    __syncthreads();
    // channel-major source: warp w stages channel quads w, w + 8, ...; lane r
    // reads sample base + r of the quad's four channels (128-byte rows) and
    // stores them as one float4 of its sample's row
    {
      const int lane = t & 31;
      static_assert(kActStride % 4 == 0, "channel quads");
      for (int c = 4 * (t >> 5); c < kActStride; c += 4 * (blockDim.x >> 5))
        if (lane < m) {
          const float* src = a.act + (size_t)c * a.act_ld + base + lane;
          *reinterpret_cast<float4*>(&tile[lane][c]) =
              make_float4(__ldg(src), __ldg(src + a.act_ld), __ldg(src + 2 * a.act_ld), __ldg(src + 3 * a.act_ld));
        }
    }
    __syncthreads();
    for (int r = 0; r < m; ++r) {
      const float* T = tile[r];
      const float4 d2 = *reinterpret_cast<const float4*>(T + kActD2 + i2);
      const float4 h1 = *reinterpret_cast<const float4*>(T + kActH1 + j2);
      const float4 d1v = *reinterpret_cast<const float4*>(T + kActD1 + i1);
      const float2 fv = *reinterpret_cast<const float2*>(T + kActF + j1);
      const float dd[4] = {d2.x, d2.y, d2.z, d2.w}, hh[4] = {h1.x, h1.y, h1.z, h1.w};
      const float ee[4] = {d1v.x, d1v.y, d1v.z, d1v.w}, ff[2] = {fv.x, fv.y};
#pragma unroll
      for (int x = 0; x < 4; ++x) {
#pragma unroll
        for (int y = 0; y < 4; ++y) acc2[4 * x + y] = fmaf(dd[x], hh[y], acc2[4 * x + y]);
#pragma unroll
        for (int y = 0; y < 2; ++y) acc1[2 * x + y] = fmaf(ee[x], ff[y], acc1[2 * x + y]);
      }
      acc3 = fmaf(T[kActDO + o3], T[kActH2 + j3], acc3);
      if (t < kWidth) accb += T[kActD1 + t];
      else if (t < 2 * kWidth) accb += T[kActD2 + t - kWidth];
      else if (t < 2 * kWidth + 4) accb += T[kActDO + t - 2 * kWidth];
    }
  }
  if (s0 >= s1) return;
  float* gW1 = a.g_mlp;
  float* gb1 = gW1 + kWidth * n_in;
  float* gW2 = gb1 + kWidth;
  float* gb2 = gW2 + kWidth * kWidth;
  float* gW3 = gb2 + kWidth;
  float* gb3 = gW3 + 4 * kWidth;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
#pragma unroll
    for (int y = 0; y < 4; ++y) atomicAdd(gW2 + (i2 + x) * kWidth + j2 + y, acc2[4 * x + y]);
#pragma unroll
    for (int y = 0; y < 2; ++y)
      if (j1 + y < n_in) atomicAdd(gW1 + (i1 + x) * n_in + j1 + y, acc1[2 * x + y]);
  }
  atomicAdd(gW3 + o3 * kWidth + j3, acc3);
  if (t < kWidth) atomicAdd(gb1 + t, accb);
  else if (t < 2 * kWidth) atomicAdd(gb2 + t - kWidth, accb);
  else if (t < 2 * kWidth + 4) atomicAdd(gb3 + t - 2 * kWidth, accb);
}

// ---------------------------------------------------------------------------
// Reduced-precision backward (fp16 / bf16 operands, fp32 accumulation).
//
// The MLP is recomputed with the operands the tensor-core forward used (weights,
// features and hidden activations rounded to the operand type, biases and
// accumulation fp32), and run backward like a reduced-precision GEMM chain: the
// output gradient is multiplied by the loss scale S, and every gradient that a
// later product consumes (dO, dH2, dH1) is rounded to the operand type.  These
// rounded operands and activations are written channel-major into X for the
// tensor-core weight-gradient reduction; dL/dfeatures is unscaled to fp32 before
// the hash-table scatter and the implicit-function gradient.  A scaled gradient
// or a hidden activation outside the operand type's range, or a non-finite
// dL/dfeatures, sets the overflow flag (the step is then skipped).
// ---------------------------------------------------------------------------

constexpr int kXdH2 = 0, kXdH1 = 64, kXH1 = 128, kXF = 192, kXOne = 224, kXH2 = 240, kXOne2 = 304, kXdO = 368;

// Shared memory of the reduced-precision backward: the forward's MLP layout
// (stage_mlp_h), the transposed weights the backward products need
// (W2T[i][j] = W2[j][i], W1T[f][i] = W1[i][f], rows padded like the forward's),
// W3 rounded to the operand type in fp32, then per warp: staged features and
// outputs, the scaled output gradients, and a [64 channel][32 sample] buffer
// that turns fragment-ordered values into coalesced rows of X.
constexpr int kBwThreads = 256;
constexpr int kBwOffW2T = (kMlpHWords + 3) / 4 * 4;
constexpr int kBwOffW1T = kBwOffW2T + kWidth * kW2Stride;
constexpr int kBwOffW3F = kBwOffW1T + kIn * kW2Stride;
constexpr int kBwShared = kBwOffW3F + 4 * kWidth;
constexpr int kTrStride = 20;  // words per channel row of the transposition buffer (32 samples + pad)
constexpr int kBwWarpWords = kWarpXWords + 32 * 4 + kWidth * kTrStride;
constexpr size_t kBwSmemBytes = sizeof(uint32_t) * (kBwShared + (kBwThreads / 32) * kBwWarpWords);

template <Prec P>
__device__ __forceinline__ void stage_backward_h(const float* __restrict__ g, int n_in, uint32_t* sw) {
  stage_mlp_h<P>(g, n_in, sw);
  const float* W2 = g + kWidth * n_in + kWidth;
  const float* W3 = W2 + kWidth * kWidth + kWidth;
  for (int t = threadIdx.x; t < kBwShared - kBwOffW2T; t += blockDim.x) {
    if (t < kWidth * kW2Stride) {  // W2T
      const int i = t / kW2Stride, c = t % kW2Stride;
      sw[kBwOffW2T + t] = c < kWidth / 2 ? HalfOf<P>::pack(W2[(2 * c) * kWidth + i], W2[(2 * c + 1) * kWidth + i]) : 0u;
    } else if (t < (kWidth + kIn) * kW2Stride) {  // W1T (feature rows past n_in are zero)
      const int q = t - kWidth * kW2Stride, f = q / kW2Stride, c = q % kW2Stride;
      sw[kBwOffW2T + t] =
          (c < kWidth / 2 && f < n_in) ? HalfOf<P>::pack(g[(2 * c) * n_in + f], g[(2 * c + 1) * n_in + f]) : 0u;
    } else {  // W3 [4][64], rounded as the forward's operand
      const int q = t - (kWidth + kIn) * kW2Stride;
      reinterpret_cast<float*>(sw)[kBwOffW2T + t] = HalfOf<P>::round(W3[q]);
    }
  }
}

// fragment (rows r0 / r0 + 8, columns 8 nt + 2t, + 1) -> transposition buffer
__device__ __forceinline__ void tr_put(uint16_t* tr16, int ch, int r, uint16_t v) { tr16[ch * 2 * kTrStride + r] = v; }

// transposition buffer (64 channels x 32 samples) -> rows row0 .. row0 + 63 of X
// at columns s0 .. s0 + 31 (two samples per 32-bit store, 64 B per row)
__device__ __forceinline__ void tr_flush(const uint32_t* tr32, uint16_t* X, int row0, int s0, int lane) {
  __syncwarp();
  uint32_t* X32 = reinterpret_cast<uint32_t*>(X + wg_index(row0, s0));
#pragma unroll 4
  for (int c2 = 0; c2 < kWidth / 2; ++c2) {
    const int ch = 2 * c2 + (lane >> 4);
    X32[ch * (kWgChunk / 2) + (lane & 15)] = tr32[ch * kTrStride + (lane & 15)];
  }
  __syncwarp();
}

template <Prec P>
__device__ __forceinline__ float rnd_bits(float v, uint16_t& b) {
  b = HalfOf<P>::bits(v);
  if constexpr (P == Prec::F16) return __half2float(__ushort_as_half(b));
  else return __bfloat162float(__ushort_as_bfloat16(b));
}

// One warp, 32 samples (one per lane): the forward recomputed with tensor-core
// MMAs (m16n8k16, fp32 accumulation, operands as the forward rounded them), the
// backward as two more MMA chains: dH1 = (dH2 W2) o [h1 > 0], dF = dH1 W1, with
// dH2 = (dO W3) o [h2 > 0] done in fp32 (K = 4).  Operands and gradients are
// written channel-major into X for the weight-gradient GEMM, dL/dfeatures
// (unscaled, fp32) into s_dfeat for the scatter kernel.
template <Prec P>
__global__ void __launch_bounds__(kBwThreads) train_backward_h_kernel(const TrainArgs a) {
  extern __shared__ uint32_t bw_smem[];
  uint32_t* sw = bw_smem;
  stage_backward_h<P>(a.P.mlp, a.P.n_in, sw);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t* wbase = bw_smem + kBwShared + warp * kBwWarpWords;
  uint32_t* Xs = wbase;                                                   // [32][kXStride] features
  float* Os = reinterpret_cast<float*>(wbase + 32 * kXStride);            // [32][4] outputs
  float* Ds = reinterpret_cast<float*>(wbase + kWarpXWords);              // [32][4] scaled dO (rounded)
  uint32_t* tr32 = wbase + kWarpXWords + 32 * 4;                          // [64][kTrStride]
  uint16_t* tr16 = reinterpret_cast<uint16_t*>(tr32);
  const float* bias = reinterpret_cast<const float*>(sw + kOffHB);
  const float* W3f = reinterpret_cast<const float*>(sw + kBwOffW3F);
  const uint32_t* W2T = sw + kBwOffW2T;
  const uint32_t* W1T = sw + kBwOffW1T;

  const int n = *a.count;
  const int n_pad = (n + kWgChunk - 1) / kWgChunk * kWgChunk;
  const float S = *a.scale, inv_S = 1.f / S;
  bool overflow = false;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int s0 = (blockIdx.x * (blockDim.x >> 5) + warp) * 32; s0 < n_pad; s0 += warps * 32) {
    const int s = s0 + lane;
    // ---- this lane's sample: features (zero without a root), compositing gradient
    bool valid = false;
    float3 xs = make_float3(0.f, 0.f, 0.f);
    float4 gr = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s < n) {
      const float4 x4 = a.s_x[s];
      valid = x4.w > 0.f;
      xs = make_float3(x4.x, x4.y, x4.z);
      if (valid) gr = a.s_grad[s];
    }
    {
      float feat[kIn];
      if (valid) encode_h(a.P.F, a.P.table_h, xs, feat);
      uint16_t* col = a.X + wg_index(0, s);  // this sample's entries, kWgChunk apart row to row
#pragma unroll
      for (int c = 0; c < kIn / 2; ++c) {
        uint16_t b0 = 0, b1 = 0;
        if (valid) {
          rnd_bits<P>(feat[2 * c], b0);
          rnd_bits<P>(feat[2 * c + 1], b1);
        }
        Xs[lane * kXStride + c] = (uint32_t)b0 | ((uint32_t)b1 << 16);
        col[(kXF + 2 * c) * kWgChunk] = b0;
        col[(kXF + 2 * c + 1) * kWgChunk] = b1;
      }
      const uint16_t one = HalfOf<P>::bits(1.f);
      col[kXOne * kWgChunk] = one;
      col[kXOne2 * kWgChunk] = one;
    }
    __syncwarp();
    // ---- layer 1: h1 = relu(W1 f + b1); masks and rounded A fragments of layer 2
    uint32_t A2[2][4][4], m1[2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int r0 = 16 * mt + g, r1 = r0 + 8;
      uint32_t A[2][4];
#pragma unroll
      for (int kt = 0; kt < 2; ++kt) {
        A[kt][0] = Xs[r0 * kXStride + 8 * kt + t];
        A[kt][1] = Xs[r1 * kXStride + 8 * kt + t];
        A[kt][2] = Xs[r0 * kXStride + 8 * kt + 4 + t];
        A[kt][3] = Xs[r1 * kXStride + 8 * kt + 4 + t];
      }
      m1[mt] = 0;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const float b0 = bias[8 * nt + 2 * t], b1 = bias[8 * nt + 2 * t + 1];
        float acc[4] = {b0, b1, b0, b1};
        const uint32_t* Wr = sw + kOffHW1 + (8 * nt + g) * kW1Stride;
#pragma unroll
        for (int kt = 0; kt < 2; ++kt) mma16816<P>(acc, A[kt], Wr[8 * kt + t], Wr[8 * kt + 4 + t]);
        uint16_t hb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (acc[q] > 0.f) m1[mt] |= 1u << (4 * nt + q);
          overflow |= !(acc[q] <= HalfOf<P>::kMax);  // an operand out of range (or NaN) spoils the GEMM
          rnd_bits<P>(fmaxf(acc[q], 0.f), hb[q]);
        }
        const int ch = 8 * nt + 2 * t;
        tr_put(tr16, ch, r0, hb[0]);
        tr_put(tr16, ch + 1, r0, hb[1]);
        tr_put(tr16, ch, r1, hb[2]);
        tr_put(tr16, ch + 1, r1, hb[3]);
        // accumulator (cols 8nt..8nt+7) -> A fragment of k-tile nt / 2
        const uint32_t lo = (uint32_t)hb[0] | ((uint32_t)hb[1] << 16), hi = (uint32_t)hb[2] | ((uint32_t)hb[3] << 16);
        A2[mt][nt >> 1][(nt & 1) * 2] = lo;
        A2[mt][nt >> 1][(nt & 1) * 2 + 1] = hi;
      }
    }
    tr_flush(tr32, a.X, kXH1, s0, lane);
    // ---- layer 2: h2 = relu(W2 h1 + b2); layer 3: o = W3 h2 + b3
    uint32_t m2[2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int r0 = 16 * mt + g, r1 = r0 + 8;
      uint32_t A3[4][4];
      m2[mt] = 0;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const float b0 = bias[kWidth + 8 * nt + 2 * t], b1 = bias[kWidth + 8 * nt + 2 * t + 1];
        float acc[4] = {b0, b1, b0, b1};
        const uint32_t* Wr = sw + kOffHW2 + (8 * nt + g) * kW2Stride;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) mma16816<P>(acc, A2[mt][kt], Wr[8 * kt + t], Wr[8 * kt + 4 + t]);
        uint16_t hb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (acc[q] > 0.f) m2[mt] |= 1u << (4 * nt + q);
          overflow |= !(acc[q] <= HalfOf<P>::kMax);
          rnd_bits<P>(fmaxf(acc[q], 0.f), hb[q]);
        }
        const int ch = 8 * nt + 2 * t;
        tr_put(tr16, ch, r0, hb[0]);
        tr_put(tr16, ch + 1, r0, hb[1]);
        tr_put(tr16, ch, r1, hb[2]);
        tr_put(tr16, ch + 1, r1, hb[3]);
        A3[nt >> 1][(nt & 1) * 2] = (uint32_t)hb[0] | ((uint32_t)hb[1] << 16);
        A3[nt >> 1][(nt & 1) * 2 + 1] = (uint32_t)hb[2] | ((uint32_t)hb[3] << 16);
      }
      const float b0 = bias[2 * kWidth + 2 * t], b1 = bias[2 * kWidth + 2 * t + 1];
      float o[4] = {b0, b1, b0, b1};
      const uint32_t* Wr = sw + kOffHW3 + g * kW2Stride;
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) mma16816<P>(o, A3[kt], Wr[8 * kt + t], Wr[8 * kt + 4 + t]);
      if (t < 2) {
        Os[r0 * 4 + 2 * t] = o[0];
        Os[r0 * 4 + 2 * t + 1] = o[1];
        Os[r1 * 4 + 2 * t] = o[2];
        Os[r1 * 4 + 2 * t + 1] = o[3];
      }
    }
    tr_flush(tr32, a.X, kXH2, s0, lane);  // (also orders the Os writes before the reads below)
    // ---- scaled output gradient of this lane's sample (zero without a root)
    {
      const float o0 = Os[lane * 4], o1 = Os[lane * 4 + 1], o2 = Os[lane * 4 + 2], o3 = Os[lane * 4 + 3];
      float dO[4];
      const float sig = expf(fminf(fmaxf(o0, -15.f), 15.f));
      dO[0] = (o0 > -15.f && o0 < 15.f) ? gr.x * sig : 0.f;
      const float oc[3] = {o1, o2, o3}, gc[3] = {gr.y, gr.z, gr.w};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float sg = 1.f / (1.f + expf(-oc[c]));
        dO[1 + c] = gc[c] * sg * (1.f - sg);
      }
      uint16_t* col = a.X + wg_index(0, s);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float v = dO[q] * S;
        overflow |= !(fabsf(v) <= HalfOf<P>::kMax);
        uint16_t b;
        Ds[lane * 4 + q] = rnd_bits<P>(v, b);
        col[(kXdO + q) * kWgChunk] = b;
      }
    }
    __syncwarp();
    // ---- dH2 = (dO W3) o [h2 > 0], fp32 (K = 4), rounded: A fragments of the next product
    uint32_t B2[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int r0 = 16 * mt + g, r1 = r0 + 8;
      const float4 d0 = reinterpret_cast<const float4*>(Ds)[r0], d1 = reinterpret_cast<const float4*>(Ds)[r1];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        uint16_t hb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 8 * nt + 2 * t + (q & 1);
          const float4 d = (q < 2) ? d0 : d1;
          float v = W3f[j] * d.x + W3f[kWidth + j] * d.y + W3f[2 * kWidth + j] * d.z + W3f[3 * kWidth + j] * d.w;
          v = ((m2[mt] >> (4 * nt + q)) & 1u) ? v : 0.f;
          overflow |= !(fabsf(v) <= HalfOf<P>::kMax);
          rnd_bits<P>(v, hb[q]);
        }
        const int ch = 8 * nt + 2 * t;
        tr_put(tr16, ch, r0, hb[0]);
        tr_put(tr16, ch + 1, r0, hb[1]);
        tr_put(tr16, ch, r1, hb[2]);
        tr_put(tr16, ch + 1, r1, hb[3]);
        B2[mt][nt >> 1][(nt & 1) * 2] = (uint32_t)hb[0] | ((uint32_t)hb[1] << 16);
        B2[mt][nt >> 1][(nt & 1) * 2 + 1] = (uint32_t)hb[2] | ((uint32_t)hb[3] << 16);
      }
    }
    tr_flush(tr32, a.X, kXdH2, s0, lane);
    // ---- dH1 = (dH2 W2) o [h1 > 0] on tensor cores, rounded
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int r0 = 16 * mt + g, r1 = r0 + 8;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const uint32_t* Wr = W2T + (8 * nt + g) * kW2Stride;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) mma16816<P>(acc, B2[mt][kt], Wr[8 * kt + t], Wr[8 * kt + 4 + t]);
        uint16_t hb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float v = ((m1[mt] >> (4 * nt + q)) & 1u) ? acc[q] : 0.f;
          overflow |= !(fabsf(v) <= HalfOf<P>::kMax);
          rnd_bits<P>(v, hb[q]);
        }
        const int ch = 8 * nt + 2 * t;
        tr_put(tr16, ch, r0, hb[0]);
        tr_put(tr16, ch + 1, r0, hb[1]);
        tr_put(tr16, ch, r1, hb[2]);
        tr_put(tr16, ch + 1, r1, hb[3]);
        // reuse A2 for the dH1 fragments (layer 1's are no longer needed)
        A2[mt][nt >> 1][(nt & 1) * 2] = (uint32_t)hb[0] | ((uint32_t)hb[1] << 16);
        A2[mt][nt >> 1][(nt & 1) * 2 + 1] = (uint32_t)hb[2] | ((uint32_t)hb[3] << 16);
      }
    }
    tr_flush(tr32, a.X, kXdH1, s0, lane);
    // ---- dF = dH1 W1 on tensor cores, unscaled to fp32
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int r0 = 16 * mt + g, r1 = r0 + 8;
#pragma unroll
      for (int nt = 0; nt < kIn / 8; ++nt) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const uint32_t* Wr = W1T + (8 * nt + g) * kW2Stride;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) mma16816<P>(acc, A2[mt][kt], Wr[8 * kt + t], Wr[8 * kt + 4 + t]);
        const int c = 8 * nt + 2 * t;
        overflow |= !(isfinite(acc[0]) && isfinite(acc[1]) && isfinite(acc[2]) && isfinite(acc[3]));
        float* df = reinterpret_cast<float*>(a.s_dfeat);
        if (s0 + r0 < n)
          *reinterpret_cast<float2*>(df + (size_t)(s0 + r0) * kIn + c) = make_float2(acc[0] * inv_S, acc[1] * inv_S);
        if (s0 + r1 < n)
          *reinterpret_cast<float2*>(df + (size_t)(s0 + r1) * kIn + c) = make_float2(acc[2] * inv_S, acc[3] * inv_S);
      }
    }
  }
  if (overflow) atomicOr(a.overflow, kStepOverflow);
}

// After an overflow the step's gradients are meaningless: zero them (the step is
// skipped) -- the flag is read on the device, so nothing waits for the host.
__global__ void zero_on_overflow_kernel(const int* overflow, float* p, size_t n) {
  if (!*overflow) return;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = 0.f;
}

// Dynamic loss scale: halve on overflow, double after kScaleWindow clean steps
// (fp16 only; bf16 has fp32's exponent range and keeps S = 1).
constexpr int kScaleWindow = 1000;
constexpr float kScaleMax = 16777216.f;  // 2^24

__global__ void loss_scale_kernel(const TrainArgs a, int dynamic) {
  if (*a.overflow & kStepOverflow) {
    *a.scale = fmaxf(*a.scale * 0.5f, 1.f);
    *a.good_steps = 0;
  } else if (*a.overflow) {
    // skipped for another reason (the weight-gradient pipeline gave up): the scale stays
  } else if (dynamic && ++*a.good_steps >= kScaleWindow) {
    *a.scale = fminf(*a.scale * 2.f, kScaleMax);
    *a.good_steps = 0;
  }
}

cudaError_t launch_train_forward(const TrainArgs& a, int num_sms, cudaStream_t s) {
  cudaError_t e;
  const int gb = (a.n_reg + 127) / 128;
  const int wb = (a.n_rays + 7) / 8;  // a warp per ray
  {
    KernelSpan span("train_count_kernel", s);
    train_count_kernel<<<wb, 256, 0, s>>>(a);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.n_reg > 0) {
    {
      KernelSpan span("reg_count_kernel", s);
      reg_count_kernel<<<gb, 128, 0, s>>>(a);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    KernelSpan span("pose_scan_kernel", s);
    pose_scan_kernel<<<1, 32, 0, s>>>(a);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    KernelSpan span("train_emit_kernel", s);
    train_emit_kernel<<<wb, 256, 0, s>>>(a);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.n_reg > 0) {
    {
      KernelSpan span("reg_emit_kernel", s);
      reg_emit_kernel<<<gb, 128, 0, s>>>(a);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const Prec P = (Prec)a.prec;
  if (a.P.search) {
    if ((e = launch_prop_bias(a.P.prop, a.P.cfg.nb, a.theta_all, a.n_poses, const_cast<float*>(a.P.prop.b1p), s)) !=
        cudaSuccess)
      return e;
  }
  // search and field at the emitted samples: the render's wavefront kernels
  // (proposal, search waves, field) with each sample's pose
  RenderArgs ra{};
  ra.P = a.P;
  ra.box = a.box;  // the fallback's point test locates each sample's occupancy cell
  ra.P.theta = nullptr;  // the proposal's layer-1 bias per pose comes from P.prop.b1p
  if (P == Prec::F32) ra.P.search = 0;
  ra.stats = a.stats;
  return launch_wf_chunk(ra, a.wf, num_sms, s);
}

cudaError_t launch_train_composite(const TrainArgs& a, cudaStream_t s) {
  cudaError_t e;
  const int rb = (a.n_rays + 127) / 128;
  const int gb = (a.n_reg + 127) / 128;
  {
    KernelSpan span("train_composite_kernel", s);
    train_composite_kernel<<<rb, 128, 0, s>>>(a);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.n_reg > 0 && a.comp_mode == kCompLoss) {
    {
      KernelSpan span("reg_grad_kernel", s);
      reg_grad_kernel<<<gb, 128, 0, s>>>(a);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_train(const TrainArgs& a, const CUtensorMap* map, int num_sms, cudaStream_t s) {
  cudaError_t e;
  if ((e = launch_train_forward(a, num_sms, s)) != cudaSuccess) return e;
  if ((e = launch_train_composite(a, s)) != cudaSuccess) return e;
  return launch_train_backward(a, map, num_sms, s);
}

cudaError_t launch_train_backward(const TrainArgs& a, const CUtensorMap* map, int num_sms, cudaStream_t s) {
  cudaError_t e;
  const Prec P = (Prec)a.prec;
  if (P == Prec::F32) {
    const size_t vec_bytes = sizeof(float) * kWidth * kBwdThreads;
    if ((e = set_smem(train_backward_kernel, vec_bytes, kBwdThreads)) != cudaSuccess) return e;
    {
      KernelSpan span("train_backward_kernel", s);
      train_backward_kernel<<<num_sms * 2, kBwdThreads, vec_bytes, s>>>(a);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_scatter(a, false, num_sms, s)) != cudaSuccess) return e;
    {
      KernelSpan span("mlp_grad_kernel", s);
      mlp_grad_kernel<<<num_sms * 4, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
  }
  if (P == Prec::F16) {
    if ((e = set_smem(train_backward_h_kernel<Prec::F16>, kBwSmemBytes, kBwThreads)) != cudaSuccess) return e;
    {
      KernelSpan span("train_backward_h_kernel<fp16>", s);
      train_backward_h_kernel<Prec::F16><<<num_sms * 2, kBwThreads, kBwSmemBytes, s>>>(a);
    }
  } else {
    if ((e = set_smem(train_backward_h_kernel<Prec::BF16>, kBwSmemBytes, kBwThreads)) != cudaSuccess) return e;
    {
      KernelSpan span("train_backward_h_kernel<bf16>", s);
      train_backward_h_kernel<Prec::BF16><<<num_sms * 2, kBwThreads, kBwSmemBytes, s>>>(a);
    }
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_scatter(a, true, num_sms, s)) != cudaSuccess) return e;
  WgradArgs w{};
  w.count = a.count;
  w.scale = a.scale;
  w.gW1 = a.g_mlp;
  w.gb1 = w.gW1 + kWidth * a.P.n_in;
  w.gW2 = w.gb1 + kWidth;
  w.gb2 = w.gW2 + kWidth * kWidth;
  w.gW3 = w.gb2 + kWidth;
  w.gb3 = w.gW3 + 4 * kWidth;
  w.n_in = a.P.n_in;
  w.bf16 = P == Prec::BF16 ? 1 : 0;
  w.flags = a.overflow;
  w.wait_ns = a.wait_ns;
  w.withhold_last = (a.inject & 1) ? 1 : 0;
  if ((e = launch_wgrad_tc(*map, w, num_sms, s)) != cudaSuccess) return e;
  const size_t sizes[4] = {a.n_table_f, a.n_mlp_f, a.n_skin_f, a.n_bones_f};
  float* bufs[4] = {a.g_table, a.g_mlp, a.g_skin, a.g_bones};
  for (int q = 0; q < 4; ++q) {
    {
      KernelSpan span("zero_on_overflow_kernel", s);
      zero_on_overflow_kernel<<<num_sms * 4, 256, 0, s>>>(a.overflow, bufs[q], sizes[q]);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    KernelSpan span("loss_scale_kernel", s);
    loss_scale_kernel<<<1, 1, 0, s>>>(a, P == Prec::F16 ? 1 : 0);
  }
  return cudaGetLastError();
}

}  // namespace ia
