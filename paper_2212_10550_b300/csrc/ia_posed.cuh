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

// ---------------------------------------------------------------------------
// Multi-start correspondence search and field evaluation (Sec. 3.1, Eq. 3-4, 7)
// for a warp's list of m <= 32 samples, one per lane.  The bone-wise Broyden
// chains are flattened: every loop step evaluates the blended grid once per
// lane, whatever start or iteration the lane is on.  Each sample's distinct
// roots go to the warp's shared-memory list; once the search is done the warp
// evaluates the field at the roots (the tensor-core MLP needs the whole warp)
// and keeps each sample's max-density root.
//   src(i, xn, M, Ninv, pose): sample i's normalised point, blended grid, N^-1
//   rows and pose index;  dst(i, out): its result.
// With use_prop (reduced precision only) the proposal network picks each
// sample's first starts: the top_k bones by logit (ties to the lower bone), the
// first shifted by the predicted offset; when none of them yields a valid root
// the search continues over every bone-wise start (the fallback).
// Kernels hand their warps lists from a counter shared by the grid, since lists
// differ a lot in cost (a sample without a root runs every start to the cap).
// (Longer lists with lanes refilled from them were measured: no faster, and
// their root lists cost L1 capacity.)
// ---------------------------------------------------------------------------

constexpr int kList = 32;

struct ListSmem {
  float4* roots;     // [kMaxRoots][kList]  (x, y, z, start bone), slot-major: conflict-free rows
  uint8_t* nroots;   // [kList]
  float4* prop;      // [kList]  (bones b0 | b1 << 8, offset xyz), or null
};

__host__ __device__ constexpr int list_smem_words(bool prop) {
  return kList * kMaxRoots * 4 + kList / 4 + (prop ? kList * 4 : 0);
}

__device__ __forceinline__ ListSmem list_smem(uint32_t* base, bool prop) {
  ListSmem q;
  q.roots = reinterpret_cast<float4*>(base);
  q.prop = prop ? reinterpret_cast<float4*>(base + kList * kMaxRoots * 4) : nullptr;
  q.nroots = reinterpret_cast<uint8_t*>(base + kList * kMaxRoots * 4 + (prop ? kList * 4 : 0));
  return q;
}

// A sample found more distinct roots than its list holds: evaluate the list and
// the new root now and keep only the max-density one (ties to the earlier
// start), so that no root is ever dropped from the selection.
template <Prec P>
__device__ __noinline__ void compress_roots(const SkinDev& S, const float4* M, const FieldDev& F, const FieldSmem& fs,
                                            float4* list, float3 xn, float3 xnew, int label_new) {
  // list[j * kList]: root j of this sample
  PosedOut best;
  best.sigma = 0.f;
  best.rgb = best.xstar = make_float3(0.f, 0.f, 0.f);
  best.start = -1;
  for (int j = 0; j <= kMaxRoots; ++j) {
    const float4 o =
        j < kMaxRoots ? list[j * kList] : make_float4(xnew.x, xnew.y, xnew.z, __int_as_float(label_new));
    const float3 xs = polish_root(S, M, make_float3(o.x, o.y, o.z), xn);
    float sig;
    float3 rgb;
    field_eval_lane<P>(F, fs, xs, sig, rgb);
    take_best(best, sig, rgb, xs, __float_as_int(o.w));
  }
  list[0] = make_float4(best.xstar.x, best.xstar.y, best.xstar.z, __int_as_float(best.start));
}

template <Prec P, class Src, class Dst>
__device__ __forceinline__ void posed_field_list(const SkinDev& S, const FieldDev& F, const SolveCfg& cfg,
                                                  const FieldSmem& fs, const ListSmem& qs, int m, Src src, Dst dst,
                                                  SampleStats& st, const PropDev& Q = PropDev{},
                                                  bool use_prop = false) {
  const int lane = threadIdx.x & 31;
  // ---- proposed starts of every sample of the list (warp MMA)
  if constexpr (P != Prec::F32) {
    if (use_prop) {
      const bool act = lane < m;
      float3 xn = make_float3(Q.nmin[0], Q.nmin[1], Q.nmin[2]);
      const float4* Mi;
      const float* Ni;
      int pose = 0;
      if (act) src(lane, xn, Mi, Ni, pose);
      float f16[16];
      prop_encode(Q, xn, f16);
      const float* O = prop_mma_warp<P>(fs.pw, fs.xstage, f16, Q.b1p, pose) + lane * (kPropMaxOut + 1);
      if (act) {
        int b0 = 0, b1 = -1;
        float v0 = O[0], v1 = -3.0e38f;
        for (int k = 1; k < cfg.nb; ++k) {
          const float v = O[k];
          if (v > v0) { b1 = b0; v1 = v0; b0 = k; v0 = v; }
          else if (v > v1) { b1 = k; v1 = v; }
        }
        if (b1 < 0) b1 = b0;
        qs.prop[lane] = make_float4(__int_as_float(b0 | (b1 << 8)), O[cfg.nb], O[cfg.nb + 1], O[cfg.nb + 2]);
        st.proposed++;
      }
      __syncwarp();  // every lane has read its row before the staging area is reused
    }
  }
  // ---- search: lane i takes sample i
  int k = 0, it = 0, nr = 0, label = 0, phase = 2, nprop = 0, pk0 = 0, pk1 = 0;
  const int cur = lane;
  float3 xn = make_float3(0.f, 0.f, 0.f), x = xn, r = xn, dx = xn, poff = xn;
  const float4* M = nullptr;
  const float* Ninv = nullptr;
  float H[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) H[q] = 0.f;
  if (lane < m) {
    int pose;
    src(lane, xn, M, Ninv, pose);
    phase = 0;
    if (use_prop) {
      nprop = min(Q.top_k, cfg.nb);
      const float4 pp = qs.prop[lane];
      const int bb = __float_as_int(pp.x);
      pk0 = bb & 0xff;
      pk1 = (bb >> 8) & 0xff;
      poff = make_float3(pp.y, pp.z, pp.w);
    }
  }
  while (__any_sync(kFull, phase != 2)) {
    float3 q = x;
    if (phase == 0) {
      // starts 0 .. nprop-1 are proposed bones, the rest every bone in order
      const bool proposed = k < nprop;
      label = proposed ? (k == 0 ? pk0 : pk1) : k - nprop;
      const float* A = Ninv + 12 * label;
      q = make_float3(A[0] * xn.x + A[1] * xn.y + A[2] * xn.z + A[3], A[4] * xn.x + A[5] * xn.y + A[6] * xn.z + A[7],
                      A[8] * xn.x + A[9] * xn.y + A[10] * xn.z + A[11]);
      if (proposed && k == 0) q = make_float3(q.x + poff.x, q.y + poff.y, q.z + poff.z);
    } else if (phase == 1) {
      q = make_float3(x.x + dx.x, x.y + dx.y, x.z + dx.z);
    }
    float Mx[12];
    if (phase != 2) blend_value(S, M, q, Mx);
    bool finish = false, conv = false;
    if (phase == 0) {
      st.starts++;
      const float3 y = apply34(Mx, q);
      x = q;
      r = make_float3(y.x - xn.x, y.y - xn.y, y.z - xn.z);
      // initial inverse Jacobian: LBS with the weights frozen at x0, (sum_i w_i R_i)^-1
      const float J0[9] = {Mx[0], Mx[1], Mx[2], Mx[4], Mx[5], Mx[6], Mx[8], Mx[9], Mx[10]};
      it = 0;
      if (!inv3(J0, H)) finish = true;
    } else if (phase == 1) {
      const float3 y = apply34(Mx, q);
      const float3 rn = make_float3(y.x - xn.x, y.y - xn.y, y.z - xn.z);
      const float3 dr = make_float3(rn.x - r.x, rn.y - r.y, rn.z - r.z);
      x = q;
      r = rn;
      ++it;
      st.iters++;
      // good Broyden: H += (dx - H dr)(dx^T H) / (dx^T H dr)
      const float3 d = dx;
      const float u0 = H[0] * dr.x + H[1] * dr.y + H[2] * dr.z;
      const float u1 = H[3] * dr.x + H[4] * dr.y + H[5] * dr.z;
      const float u2 = H[6] * dr.x + H[7] * dr.y + H[8] * dr.z;
      const float den = d.x * u0 + d.y * u1 + d.z * u2;
      if (fabsf(den) > 1e-12f) {
        const float rden = 1.f / den;  // one reciprocal for the three quotients
        const float a0 = (d.x - u0) * rden, a1 = (d.y - u1) * rden, a2 = (d.z - u2) * rden;
        const float b0 = d.x * H[0] + d.y * H[3] + d.z * H[6];
        const float b1 = d.x * H[1] + d.y * H[4] + d.z * H[7];
        const float b2 = d.x * H[2] + d.y * H[5] + d.z * H[8];
        H[0] += a0 * b0; H[1] += a0 * b1; H[2] += a0 * b2;
        H[3] += a1 * b0; H[4] += a1 * b1; H[5] += a1 * b2;
        H[6] += a2 * b0; H[7] += a2 * b1; H[8] += a2 * b2;
      }
    }
    if (phase != 2 && !finish) {
      const float rr = r.x * r.x + r.y * r.y + r.z * r.z;
      if (rr < cfg.tol2) {
        conv = true;
        finish = true;
      } else if (it >= cfg.max_iter) {
        finish = true;
      } else {
        dx = make_float3(-(H[0] * r.x + H[1] * r.y + H[2] * r.z), -(H[3] * r.x + H[4] * r.y + H[5] * r.z),
                         -(H[6] * r.x + H[7] * r.y + H[8] * r.z));
        phase = 1;
      }
    }
    if (finish) {
      float4* list = qs.roots + cur;
      if (conv && in_box(S, x)) {
        st.converged++;
        bool dup = false;
        for (int j = 0; j < nr; ++j) {
          const float4 o = list[j * kList];
          const float ddx = x.x - o.x, ddy = x.y - o.y, ddz = x.z - o.z;
          if (ddx * ddx + ddy * ddy + ddz * ddz < 1e-8f) { dup = true; break; }
        }
        if (!dup) {
          st.roots++;
          if (nr < kMaxRoots) {
            list[kList * nr++] = make_float4(x.x, x.y, x.z, __int_as_float(label));
          } else {
            compress_roots<P>(S, M, F, fs, list, xn, x, label);
            nr = 1;
          }
        }
      }
      ++k;
      if (nprop > 0 && k == nprop) {
        if (nr > 0) k = nprop + cfg.nb;  // a proposed start found a root: done
        else st.fallbacks++;             // none did: every bone-wise start follows
      }
      if (k < nprop + cfg.nb) {
        phase = 0;
      } else {
        qs.nroots[cur] = (uint8_t)nr;
        phase = 2;
      }
    }
  }
  __syncwarp();
  // ---- one Newton polish per stored root, field at the roots, max-density root
  {
    const int i = lane;  // the lane evaluates its own sample's roots
    const bool act = i < m;
    PosedOut out;
    out.sigma = 0.f;
    out.rgb = out.xstar = make_float3(0.f, 0.f, 0.f);
    out.start = -1;
    int n_r = 0;
    float3 xq = make_float3(0.f, 0.f, 0.f);
    const float4* Mq = nullptr;
    if (act) {
      const float* Nq;
      int pose;
      src(i, xq, Mq, Nq, pose);
      n_r = qs.nroots[i];
    }
    const int nmax = __reduce_max_sync(kFull, n_r);
    for (int e = 0; e < nmax; ++e) {
      const bool has = e < n_r;
      float3 xs = make_float3(S.cmin[0], S.cmin[1], S.cmin[2]);
      int start = -1;
      if (has) {
        const float4 o = qs.roots[e * kList + i];
        start = __float_as_int(o.w);
        xs = polish_root(S, Mq, make_float3(o.x, o.y, o.z), xq);
      }
      float sig;
      float3 rgb;
      field_eval_warp<P>(F, fs, xs, sig, rgb);
      if (has) take_best(out, sig, rgb, xs, start);
    }
    if (act) dst(i, out);
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Shared-memory layout of kernels that evaluate the posed field:
//   MLP (fp32 layout, or reduced-precision layout + proposal + per-warp
//   staging), a pose's N_k^-1, and each warp's search lists.
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
  ListSmem list;  // this warp's search list
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
  p.list = list_smem(reinterpret_cast<uint32_t*>(p.sNinv + kMaxBones * 12) +
                           (threadIdx.x >> 5) * list_smem_words(a.search != 0),
                       a.search != 0);
  for (int t = threadIdx.x; t < a.nb * 12; t += blockDim.x) p.sNinv[t] = a.Ninv[t];
  __syncthreads();
  return p;
}

}  // namespace ia
