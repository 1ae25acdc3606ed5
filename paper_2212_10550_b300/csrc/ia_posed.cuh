// Precision-generic canonical field evaluation and the multi-start
// correspondence search built on it (Sec. 3.1, Eq. 1-4 and 7).
#pragma once

#include "ia_device.cuh"
#include "ia_mma.cuh"
#include "ia_prop.cuh"

namespace ia {

// Where a kernel keeps what the field evaluation reads.
struct FieldSmem {
  const float* sw;           // fp32 MLP in the layout of stage_mlp (Prec::F32)
  const uint32_t* swh;       // reduced-precision MLP in the layout of stage_mlp_h
  uint32_t* xstage;          // this warp's staging area (kStageWords words)
  const uint32_t* pw;        // proposal network in the layout of stage_prop_h (or null)
  const float* gmlp;         // packed fp32 MLP in global memory
  int n_in;
  const __half2* table_h;    // fp16 shadow of the hash table (reduced precision)
};

// Field at one point per lane; all 32 lanes call (tensor cores need the warp).
template <Prec P>
__device__ __forceinline__ void field_eval_warp(const FieldDev& F, const FieldSmem& fs, float3 x, float& sigma,
                                                float3& rgb) {
  float feat[kIn], o[4];
  if constexpr (P == Prec::F32) {
    encode(F, x, feat);
    mlp_fp32(fs.sw, feat, o);
  } else {
    encode_h(F, fs.table_h, x, feat);
    mlp_mma_warp<P>(fs.swh, fs.xstage, feat, o);
  }
  activate(o, sigma, rgb);
}

// Field at one point for a single lane (numerically the same network).
template <Prec P>
__device__ __forceinline__ void field_eval_lane(const FieldDev& F, const FieldSmem& fs, float3 x, float& sigma,
                                                float3& rgb) {
  float feat[kIn], o[4];
  if constexpr (P == Prec::F32) {
    encode(F, x, feat);
    mlp_fp32(fs.sw, feat, o);
  } else {
    encode_h(F, fs.table_h, x, feat);
    mlp_lane_h<P>(fs.gmlp, fs.n_in, feat, o);
  }
  activate(o, sigma, rgb);
}

// Multi-start correspondence search and field evaluation for NS samples per
// lane (NS independent Broyden chains interleaved, so that each loop step has
// NS gathers of the blended grid in flight per lane).  All 32 lanes must call.
//   M[s]: sample s's pose's blended grid; Ninv[s]: that pose's N_k^-1 ([nb][12]);
//   roots: this CTA's float4 scratch of kMaxRoots * NS * blockDim.x entries
//   (x, y, z, start bits).
// The first kMaxRoots distinct roots of a sample are evaluated together by the
// warp after the search; any further distinct root (rare) is evaluated on the
// spot so that no root is ever dropped.
// With use_prop (warp-uniform; reduced precision only) the proposal network
// picks each sample's first starts: the top_k bones by logit (ties to the lower
// bone), the first shifted by the predicted offset; when none of them yields a
// valid root the search continues over every bone-wise start (the fallback).
// With Q.b1p set, lane_pose[s] names sample s's pose (its layer-1 bias row).
template <int NS, Prec P>
__device__ __forceinline__ void posed_field_warp_n(const SkinDev& S, const float4* const* M, const FieldDev& F,
                                                   const SolveCfg& cfg, const float* const* Ninv, const FieldSmem& fs,
                                                   float4* roots, const bool* active, const float3* xn,
                                                   PosedOut* out, SampleStats& st, const PropDev& Q = PropDev{},
                                                   bool use_prop = false, const int* lane_pose = nullptr) {
  const int tid = threadIdx.x, stride = blockDim.x;
  // ---- proposed starts
  int nprop[NS], pk[NS][2];
  float3 poff[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    nprop[s] = 0;
    pk[s][0] = pk[s][1] = 0;
    poff[s] = make_float3(0.f, 0.f, 0.f);
  }
  if constexpr (P != Prec::F32) {
    if (use_prop) {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        float f16[16];
        prop_encode(Q, active[s] ? xn[s] : make_float3(Q.nmin[0], Q.nmin[1], Q.nmin[2]), f16);
        const float* O = prop_mma_warp<P>(fs.pw, fs.xstage, f16, Q.b1p, lane_pose ? lane_pose[s] : 0) +
                         (threadIdx.x & 31) * (kPropMaxOut + 1);
        if (active[s]) {
          int b0 = 0, b1 = -1;
          float v0 = O[0], v1 = -3.0e38f;
          for (int i = 1; i < cfg.nb; ++i) {
            const float v = O[i];
            if (v > v0) { b1 = b0; v1 = v0; b0 = i; v0 = v; }
            else if (v > v1) { b1 = i; v1 = v; }
          }
          pk[s][0] = b0;
          pk[s][1] = b1 < 0 ? b0 : b1;
          nprop[s] = min(Q.top_k, cfg.nb);
          poff[s] = make_float3(O[cfg.nb], O[cfg.nb + 1], O[cfg.nb + 2]);
          st.proposed++;
        }
        __syncwarp();  // every lane has read its row before the staging area is reused
      }
    }
  }
  int k[NS], it[NS], nroots[NS], phase[NS];  // phase 0 = start k, 1 = iterate, 2 = done
  int label[NS];
  float3 x[NS], r[NS], dx[NS];
  float H[NS][9];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    out[s].sigma = 0.f;
    out[s].rgb = make_float3(0.f, 0.f, 0.f);
    out[s].xstar = out[s].rgb;
    out[s].start = -1;
    k[s] = 0; it[s] = 0; nroots[s] = 0; label[s] = 0;
    phase[s] = active[s] ? 0 : 2;
    x[s] = make_float3(0.f, 0.f, 0.f); r[s] = x[s]; dx[s] = x[s];
#pragma unroll
    for (int q = 0; q < 9; ++q) H[s][q] = 0.f;
  }
  auto busy = [&]() {
    bool b = false;
#pragma unroll
    for (int s = 0; s < NS; ++s) b |= phase[s] != 2;
    return b;
  };
  // ---- flattened multi-start Broyden: every loop step evaluates M once per chain
  while (__any_sync(kFull, busy())) {
    float3 q[NS];
    float Mx[NS][12];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      q[s] = x[s];
      if (phase[s] == 0) {
        // starts 0 .. nprop-1 are proposed bones, the rest every bone in order
        const bool proposed = k[s] < nprop[s];
        label[s] = proposed ? (k[s] == 0 ? pk[s][0] : pk[s][1]) : k[s] - nprop[s];
        const float* A = Ninv[s] + 12 * label[s];
        const float3 p = xn[s];
        q[s] = make_float3(A[0] * p.x + A[1] * p.y + A[2] * p.z + A[3], A[4] * p.x + A[5] * p.y + A[6] * p.z + A[7],
                           A[8] * p.x + A[9] * p.y + A[10] * p.z + A[11]);
        if (proposed && k[s] == 0) q[s] = make_float3(q[s].x + poff[s].x, q[s].y + poff[s].y, q[s].z + poff[s].z);
      } else if (phase[s] == 1) {
        q[s] = make_float3(x[s].x + dx[s].x, x[s].y + dx[s].y, x[s].z + dx[s].z);
      }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (phase[s] != 2) blend_value(S, M[s], q[s], Mx[s]);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      bool finish = false, conv = false;
      if (phase[s] == 0) {
        st.starts++;
        const float3 y = apply34(Mx[s], q[s]);
        x[s] = q[s];
        r[s] = make_float3(y.x - xn[s].x, y.y - xn[s].y, y.z - xn[s].z);
        // initial inverse Jacobian: LBS with the weights frozen at x0, (sum_i w_i R_i)^-1
        const float J0[9] = {Mx[s][0], Mx[s][1], Mx[s][2], Mx[s][4], Mx[s][5], Mx[s][6], Mx[s][8], Mx[s][9], Mx[s][10]};
        it[s] = 0;
        if (!inv3(J0, H[s])) finish = true;
      } else if (phase[s] == 1) {
        const float3 y = apply34(Mx[s], q[s]);
        const float3 rn = make_float3(y.x - xn[s].x, y.y - xn[s].y, y.z - xn[s].z);
        const float3 dr = make_float3(rn.x - r[s].x, rn.y - r[s].y, rn.z - r[s].z);
        x[s] = q[s];
        r[s] = rn;
        ++it[s];
        st.iters++;
        // good Broyden: H += (dx - H dr)(dx^T H) / (dx^T H dr)
        float* h = H[s];
        const float3 d = dx[s];
        const float u0 = h[0] * dr.x + h[1] * dr.y + h[2] * dr.z;
        const float u1 = h[3] * dr.x + h[4] * dr.y + h[5] * dr.z;
        const float u2 = h[6] * dr.x + h[7] * dr.y + h[8] * dr.z;
        const float den = d.x * u0 + d.y * u1 + d.z * u2;
        if (fabsf(den) > 1e-12f) {
          const float rden = 1.f / den;  // one reciprocal for the three quotients
          const float a0 = (d.x - u0) * rden, a1 = (d.y - u1) * rden, a2 = (d.z - u2) * rden;
          const float b0 = d.x * h[0] + d.y * h[3] + d.z * h[6];
          const float b1 = d.x * h[1] + d.y * h[4] + d.z * h[7];
          const float b2 = d.x * h[2] + d.y * h[5] + d.z * h[8];
          h[0] += a0 * b0; h[1] += a0 * b1; h[2] += a0 * b2;
          h[3] += a1 * b0; h[4] += a1 * b1; h[5] += a1 * b2;
          h[6] += a2 * b0; h[7] += a2 * b1; h[8] += a2 * b2;
        }
      }
      if (phase[s] != 2 && !finish) {
        const float rr = r[s].x * r[s].x + r[s].y * r[s].y + r[s].z * r[s].z;
        if (rr < cfg.tol2) {
          conv = true;
          finish = true;
        } else if (it[s] >= cfg.max_iter) {
          finish = true;
        } else {
          const float* h = H[s];
          dx[s] = make_float3(-(h[0] * r[s].x + h[1] * r[s].y + h[2] * r[s].z),
                              -(h[3] * r[s].x + h[4] * r[s].y + h[5] * r[s].z),
                              -(h[6] * r[s].x + h[7] * r[s].y + h[8] * r[s].z));
          phase[s] = 1;
        }
      }
      if (finish) {
        if (conv && in_box(S, x[s])) {
          st.converged++;
          bool dup = false;
          for (int j = 0; j < min(nroots[s], kMaxRoots); ++j) {
            const float4 o = roots[((s * kMaxRoots) + j) * stride + tid];
            const float ddx = x[s].x - o.x, ddy = x[s].y - o.y, ddz = x[s].z - o.z;
            if (ddx * ddx + ddy * ddy + ddz * ddz < 1e-8f) { dup = true; break; }
          }
          if (!dup) {
            st.roots++;
            if (nroots[s] < kMaxRoots) {
              roots[((s * kMaxRoots) + nroots[s]) * stride + tid] =
                  make_float4(x[s].x, x[s].y, x[s].z, __int_as_float(label[s]));
            } else {
              const float3 xs = polish_root(S, M[s], x[s], xn[s]);
              float sig;
              float3 rgb;
              field_eval_lane<P>(F, fs, xs, sig, rgb);
              take_best(out[s], sig, rgb, xs, label[s]);
            }
            nroots[s]++;
          }
        }
        ++k[s];
        if (nprop[s] > 0 && k[s] == nprop[s]) {
          if (nroots[s] > 0) k[s] = nprop[s] + cfg.nb;  // a proposed start found a root: done
          else st.fallbacks++;                            // none did: every bone-wise start follows
        }
        phase[s] = (k[s] < nprop[s] + cfg.nb) ? 0 : 2;
      }
    }
  }
  // ---- one Newton polish per stored root, field evaluation, max-density root;
  //      the lane's (sample, root) pairs are evaluated one per warp step
  int nr[NS], total = 0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    nr[s] = min(nroots[s], kMaxRoots);
    total += nr[s];
  }
  const int nmax = __reduce_max_sync(kFull, total);
  for (int e = 0; e < nmax; ++e) {
    const bool has = e < total;
    int si = 0, j = e;
#pragma unroll
    for (int s = 0; s + 1 < NS; ++s)
      if (si == s && j >= nr[s]) { j -= nr[s]; si = s + 1; }
    float3 xs = make_float3(S.cmin[0], S.cmin[1], S.cmin[2]);
    int start = -1;
    float3 xq = xn[0];
    const float4* Mq = M[0];
#pragma unroll
    for (int s = 1; s < NS; ++s)
      if (si == s) { xq = xn[s]; Mq = M[s]; }
    if (has) {
      const float4 o = roots[((si * kMaxRoots) + j) * stride + tid];
      start = __float_as_int(o.w);
      xs = polish_root(S, Mq, make_float3(o.x, o.y, o.z), xq);
    }
    float sig;
    float3 rgb;
    field_eval_warp<P>(F, fs, xs, sig, rgb);
    if (has) {
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (si == s) take_best(out[s], sig, rgb, xs, start);
    }
  }
}

// ---------------------------------------------------------------------------
// Shared-memory layout of kernels that evaluate the posed field:
//   MLP (fp32 layout, or reduced-precision layout + proposal + per-warp
//   staging), a pose's N_k^-1, and the per-lane root lists.
// ---------------------------------------------------------------------------

struct PosedStage {
  const float* mlp;      // packed fp32 MLP (global)
  int n_in;
  const __half2* table_h;
  int search;            // stage the proposal network too (the host sizes the
                         // shared memory with the same flag: mlp_smem_words)
  PropDev prop;
  const double* theta;   // pose axis-angles (proposal input)
  const float* Ninv;     // [nb][12]
  int nb;
};

constexpr int kMlpPad = (kMlpSmemFloats + 3) / 4 * 4;

// 32-bit words of the MLP area; the proposal's weights and its larger per-warp
// staging are reserved only when the proposal is staged (prop), so that kernels
// without it leave more of the SM's unified memory to L1
__host__ __device__ constexpr int mlp_smem_words(Prec P, int threads, bool prop) {
  return P == Prec::F32 ? kMlpPad
                        : ((kMlpHWords + 3) / 4 * 4 + (prop ? (kPropWords + 3) / 4 * 4 : 0) +
                           (threads / 32) * (prop ? kStageWords : kWarpXWords));
}

struct PosedSmem {
  FieldSmem fs;
  float* sNinv;
  float4* roots;
};

template <Prec P>
__device__ __forceinline__ PosedSmem stage_posed(const PosedStage& a, float4* smem4) {
  PosedSmem p;
  float* base = reinterpret_cast<float*>(smem4);
  p.fs.gmlp = a.mlp;
  p.fs.n_in = a.n_in;
  p.fs.table_h = a.table_h;
  if constexpr (P == Prec::F32) {
    p.fs.sw = base;
    p.fs.swh = nullptr;
    p.fs.xstage = nullptr;
    p.fs.pw = nullptr;
    stage_mlp(a.mlp, a.n_in, base);
  } else {
    uint32_t* w = reinterpret_cast<uint32_t*>(base);
    uint32_t* pw = w + (kMlpHWords + 3) / 4 * 4;
    p.fs.sw = nullptr;
    p.fs.swh = w;
    p.fs.pw = a.search ? pw : nullptr;
    p.fs.xstage = a.search ? pw + (kPropWords + 3) / 4 * 4 + (threadIdx.x >> 5) * kStageWords
                           : pw + (threadIdx.x >> 5) * kWarpXWords;
    stage_mlp_h<P>(a.mlp, a.n_in, w);
    if (a.search) stage_prop_h<P>(a.prop, a.nb, a.theta, pw);
  }
  p.sNinv = base + mlp_smem_words(P, blockDim.x, a.search != 0);
  p.roots = reinterpret_cast<float4*>(p.sNinv + kMaxBones * 12);
  for (int t = threadIdx.x; t < a.nb * 12; t += blockDim.x) p.sNinv[t] = a.Ninv[t];
  __syncthreads();
  return p;
}

}  // namespace ia
