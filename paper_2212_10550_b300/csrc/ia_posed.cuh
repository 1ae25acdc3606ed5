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
// kCompact (reduced precision): rolled encoding and MLP chain, for kernels
// whose code overflows the instruction cache (measured: the proposal render
// 3.09 -> 2.47 ms; the plain fp16 training forward is faster unrolled).
template <Prec P, bool kCompact = false>
__device__ __forceinline__ void field_eval_warp(const FieldDev& F, const FieldSmem& fs, float3 x, float& sigma,
                                                float3& rgb) {
  float feat[kIn], o[4];
  if constexpr (P == Prec::F32) {
    encode(F, x, feat);
    mlp_fp32(fs.sw, feat, o);
  } else if constexpr (kCompact) {
    encode_h_staged<P>(F, fs.table_h, x, fs.xstage + (threadIdx.x & 31) * kXStride);
    mlp_mma_warp_staged<P, true>(fs.swh, fs.xstage, o);
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
    mlp_lane_hs<P>(fs.swh, feat, o);
  }
  activate(o, sigma, rgb);
}

// ---------------------------------------------------------------------------
// Multi-start correspondence search and field evaluation (Sec. 3.1, Eq. 3-4, 7)
// for a warp's list of m <= 32 samples.
//
// The work items are (sample, start) pairs (ItemOrder below): with a shared
// queue a lane that finishes an item takes the next one, so a sample without a
// root (every start runs to the iteration cap) no longer holds a whole warp
// while the other lanes idle.  Every loop step evaluates the blended grid once per busy lane, whatever
// start or iteration the lane is on.  Converged roots inside the canonical box
// are merged into their sample's shared-memory list: a root within 1e-4 of a
// listed one is the same root, and the list keeps the earlier start's (code and
// position; found by each lane in parallel); new roots are appended one at a
// time by the whole warp.  Once the items are
// done the warp evaluates the field at the roots (the tensor-core MLP needs the
// whole warp), lane i for sample i, and keeps each sample's max-density root
// (ties to the lower start bone).
//   src(i, xn, M, Ninv, pose): sample i's normalised point, blended grid, N^-1
//   rows and pose index;  dst(i, out): its result.
// With use_prop (reduced precision only) the proposal network picks each
// sample's first starts: the top_k bones by logit (ties to the lower bone), the
// first shifted by the predicted offset.  Those items run first; the samples
// none of whose proposed starts yields a valid root then take every bone-wise
// start (the fallback).
// Kernels hand their warps lists from a counter shared by the grid, since lists
// differ a lot in cost.
// ---------------------------------------------------------------------------

constexpr int kList = 32;

struct ListSmem {
  float4* roots;     // [kMaxRoots][kList]  (x, y, z, order << 8 | start bone), slot-major rows
  uint8_t* nroots;   // [kList]
  uint8_t* fb;       // [kList] samples that fall back to every start
  float4* prop;      // [kList]  (bones b0 | b1 << 8, offset xyz), or null
};

__host__ __device__ constexpr int list_smem_words(bool prop) {
  return kList * kMaxRoots * 4 + kList / 4 + kList / 4 + (prop ? kList * 4 : 0);
}

__device__ __forceinline__ ListSmem list_smem(uint32_t* base, bool prop) {
  ListSmem q;
  q.roots = reinterpret_cast<float4*>(base);
  q.prop = prop ? reinterpret_cast<float4*>(base + kList * kMaxRoots * 4) : nullptr;
  q.nroots = reinterpret_cast<uint8_t*>(base + kList * kMaxRoots * 4 + (prop ? kList * 4 : 0));
  q.fb = q.nroots + kList;
  return q;
}

// A sample found more distinct roots than its list holds: evaluate the list and
// the new root now and keep only the max-density one (ties to the lower start
// bone), so that no root is ever dropped from the selection.  The kept entry
// is the root as found (position and start code), not its polished position:
// the final selection polishes it once like every other root, so the result
// does not depend on when (or whether) the list was compressed.
template <Prec P>
__device__ __noinline__ void compress_roots(const SkinDev& S, const float4* M, const FieldDev& F, const FieldSmem& fs,
                                            float4* list, float3 xn, float3 xnew, int code_new) {
  // list[j * kList]: root j of this sample
  PosedOut best;
  best.sigma = 0.f;
  best.rgb = best.xstar = make_float3(0.f, 0.f, 0.f);
  best.start = -1;
  int best_code = code_new;
  float3 best_raw = xnew;
  for (int j = 0; j <= kMaxRoots; ++j) {
    const float4 o =
        j < kMaxRoots ? list[j * kList] : make_float4(xnew.x, xnew.y, xnew.z, __int_as_float(code_new));
    const int code = __float_as_int(o.w), bone = code & 0xff;
    const float3 xs = polish_root(S, M, make_float3(o.x, o.y, o.z), xn);
    float sig;
    float3 rgb;
    field_eval_lane<P>(F, fs, xs, sig, rgb);
    // take_best's rule, with the list code kept alongside
    if (sig > best.sigma || (sig == best.sigma && best.start >= 0 && bone < best.start) || best.start < 0) {
      best.sigma = sig;
      best.rgb = rgb;
      best.xstar = xs;
      best.start = bone;
      best_code = code;
      best_raw = make_float3(o.x, o.y, o.z);
    }
  }
  list[0] = make_float4(best_raw.x, best_raw.y, best_raw.z, __int_as_float(best_code));
}

// The field phase of a list of m <= 32 samples whose distinct roots are in qs
// (qs.nroots, qs.roots): one Newton polish per root, the field at the roots,
// each sample's max-density root (ties to the lower start bone) to dst.
// The list's roots are spread over the lanes, 32 per warp-wide field
// evaluation: root e of sample i has the flat index first_i + e (first_i = the
// roots of samples 0..i-1); lane l of a round evaluates flat index base + l.
// The owner lane of each sample then takes its roots' results in root order
// (take_best), as if it had evaluated them itself.  All 32 lanes call.
template <Prec P, bool kCompact, class Src, class Dst>
__device__ __forceinline__ void list_field_phase(const SkinDev& S, const FieldDev& F, const FieldSmem& fs,
                                                 const ListSmem& qs, int m, Src src, Dst dst) {
  const int lane = threadIdx.x & 31;
  {
    const int i = lane;  // owner of sample i
    const bool act = i < m;
    PosedOut out;
    out.sigma = 0.f;
    out.rgb = out.xstar = make_float3(0.f, 0.f, 0.f);
    out.start = -1;
    const int n_r = act ? qs.nroots[i] : 0;
    int incl = n_r;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    const int first = incl - n_r;
    const int total = __shfl_sync(kFull, incl, 31);
    for (int base = 0; base < total; base += 32) {
      const int f = base + lane;
      const bool has = f < total;
      // the sample holding flat index f: the last lane whose first index is <= f
      // (a lane with no roots shares its first index with the next lane)
      int s_of = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int cand = s_of + step;
        const int fc = __shfl_sync(kFull, first, cand & 31);
        if (cand < 32 && fc <= f) s_of = cand;
      }
      const int e = f - __shfl_sync(kFull, first, s_of);
      float3 xs = make_float3(S.cmin[0], S.cmin[1], S.cmin[2]);
      int start = -1;
      if (has) {
        float3 xq;
        const float4* Mq;
        const float* Nq;
        int pose;
        src(s_of, xq, Mq, Nq, pose);
        const float4 o = qs.roots[e * kList + s_of];
        start = __float_as_int(o.w) & 0xff;
        xs = polish_root(S, Mq, make_float3(o.x, o.y, o.z), xq);
      }
      float sig;
      float3 rgb;
      field_eval_warp<P, kCompact>(F, fs, xs, sig, rgb);
      // each owner collects its sample's roots of this round, in root order
#pragma unroll
      for (int e2 = 0; e2 < kMaxRoots; ++e2) {
        const int fl = first + e2;
        const bool mine = act && e2 < n_r && fl >= base && fl < base + 32;
        const int from = mine ? fl - base : lane;
        const float g_sig = __shfl_sync(kFull, sig, from);
        const float3 g_rgb = make_float3(__shfl_sync(kFull, rgb.x, from), __shfl_sync(kFull, rgb.y, from),
                                         __shfl_sync(kFull, rgb.z, from));
        const float3 g_xs = make_float3(__shfl_sync(kFull, xs.x, from), __shfl_sync(kFull, xs.y, from),
                                        __shfl_sync(kFull, xs.z, from));
        const int g_start = __shfl_sync(kFull, start, from);
        if (mine) take_best(out, g_sig, g_rgb, g_xs, g_start);
      }
    }
    if (act) dst(i, out);
  }
  __syncwarp();
}

// How a list's (sample, start) items meet the lanes:
//   kPerLane      lane i runs sample i's starts in order (no sharing)
//   kSampleMajor  a shared queue, every start of sample 0, then of sample 1, ...
//   kStartMajor   a shared queue, start 0 of every sample, then start 1, ...
// (measured: the plain 24-start render keeps its L1 locality best per lane; the
// proposal's render, whose fallbacks are few but long, the culled occupancy
// grid, whose short lists leave few per warp, and the training forward gain from
// the shared queue, start-major, start-major and sample-major respectively).
// The queues run a sample's starts concurrently and in an order that depends on
// the other samples of the list; the selected root does not depend on it (the
// earliest start keeps a root's code and position, compressed lists keep roots
// as found), barring roots within the merge distance of two listed ones.
enum class ItemOrder { kPerLane, kSampleMajor, kStartMajor };

template <Prec P, ItemOrder kOrder, bool kCompact = false, ItemOrder kFallbackOrder = kOrder, class Src, class Dst>
__device__ __forceinline__ void posed_field_list(const SkinDev& S, const FieldDev& F, const SolveCfg& cfg,
                                                 const FieldSmem& fs, const ListSmem& qs, int m, Src src, Dst dst,
                                                 SampleStats& st, const PropDev& Q = PropDev{},
                                                 bool use_prop = false) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  // ---- proposed starts of every sample of the list (warp MMA)
  if constexpr (P != Prec::F32) {
    if (use_prop) {
      const bool act = lane < m;
      float3 xn = make_float3(Q.nmin[0], Q.nmin[1], Q.nmin[2]);
      const float4* Mi;
      const float* Ni;
      int pose = 0;
      if (act) src(lane, xn, Mi, Ni, pose);
      const float* O;
      if constexpr (kCompact) {
        prop_encode_staged<P>(Q, xn, fs.xstage + lane * kPW1Stride);
        O = prop_mma_warp<P, true>(fs.pw, fs.xstage, nullptr, Q.b1p, pose) + lane * (kPropMaxOut + 1);
      } else {
        float f16[16];
        prop_encode(Q, xn, f16);
        O = prop_mma_warp<P>(fs.pw, fs.xstage, f16, Q.b1p, pose) + lane * (kPropMaxOut + 1);
      }
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
  if (lane < m) qs.nroots[lane] = 0;
  __syncwarp();
  const int nprop = use_prop ? min(Q.top_k, cfg.nb) : 0;
  // ---- stage 0: the proposed starts (or every start without the proposal);
  //      stage 1: every start of the samples whose proposed starts found no root
  for (int stage = 0; stage < (use_prop ? 2 : 1); ++stage) {
    int per, n_items, ns;  // starts per sample, items, samples of the stage
    if (stage == 0) {
      per = use_prop ? nprop : cfg.nb;
      ns = m;
      n_items = m * per;
    } else {
      const bool fall = lane < m && qs.nroots[lane] == 0;
      const unsigned fm = __ballot_sync(kFull, fall);
      if (fall) {
        qs.fb[__popc(fm & lt)] = (uint8_t)lane;
        st.fallbacks++;
      }
      __syncwarp();
      per = cfg.nb;
      ns = __popc(fm);
      n_items = ns * per;
    }
    // this stage's order: kOrder for the first starts, kFallbackOrder for the fallback
    const ItemOrder ord = stage == 0 ? kOrder : kFallbackOrder;
    // shared queue: idx -> (sample, start) by a multiply-high division (exact
    // for idx < 2^16; ns == 1 and per == 1 need none: 2^32 does not fit)
    const int dv = ord == ItemOrder::kStartMajor ? ns : per;
    const unsigned magic = dv > 1 ? 0xFFFFFFFFu / (unsigned)dv + 1u : 0u;
    const bool mine = stage == 0 ? lane < m : (lane < m && qs.nroots[lane] == 0);  // kPerLane
    int next = 0;  // warp-uniform: items handed out so far
    int jl = -1;   // kPerLane: this lane's last start
    int loaded = -1;
    bool need = true;
    int phase = 2, cur = 0, label = 0, order = 0, it = 0;
    bool shift = false;
    float3 xn = make_float3(0.f, 0.f, 0.f), x = xn, r = xn, dx = xn, poff = xn;
    const float4* M = nullptr;
    const float* Ninv = nullptr;
    float H[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) H[q] = 0.f;
    while (true) {
      // lanes without an item take the next one
      bool got = false;
      int i = 0, j = 0;
      if (ord == ItemOrder::kPerLane) {
        if (need) {
          need = false;
          phase = 2;
          if (mine && jl + 1 < per) {
            got = true;
            i = lane;
            j = ++jl;
          }
        }
      } else {
        const unsigned needm = __ballot_sync(kFull, need);
        if (needm) {
          const int idx = next + __popc(needm & lt);
          next += __popc(needm);
          if (need) {
            need = false;
            phase = 2;
            if (idx < n_items) {
              got = true;
              const int q = dv > 1 ? (int)__umulhi((unsigned)idx, magic) : idx, rm = idx - q * dv;
              if (ord == ItemOrder::kStartMajor) { j = q; i = rm; }
              else { i = q; j = rm; }
            }
          }
        }
      }
      if (got) {
        cur = (stage == 0 || ord == ItemOrder::kPerLane) ? i : qs.fb[i];
        if (cur != loaded) {  // consecutive items of one sample reuse its point and grids
          int pose;
          src(cur, xn, M, Ninv, pose);
          loaded = cur;
        }
        if (stage == 0 && use_prop) {
          const float4 pp = qs.prop[cur];
          const int bb = __float_as_int(pp.x);
          label = j == 0 ? (bb & 0xff) : ((bb >> 8) & 0xff);
          shift = j == 0;
          poff = make_float3(pp.y, pp.z, pp.w);
          order = j;
        } else {
          label = j;
          shift = false;
          order = (stage == 0 ? 0 : nprop) + j;
        }
        phase = 0;
      }
      if (!__any_sync(kFull, phase != 2)) break;
      float3 q = x;
      if (phase == 0) q = search_start(Ninv + 12 * label, xn, shift, poff);
      else if (phase == 1) q = add3(x, dx);
      float Mx[12];
      if (phase != 2) blend_value(S, M, q, Mx);
      bool finish = false, conv = false;
      if (phase == 0) {
        st.starts++;
        x = q;
        r = search_residual(Mx, q, xn);
        // initial inverse Jacobian: LBS with the weights frozen at x0, (sum_i w_i R_i)^-1
        const float J0[9] = {Mx[0], Mx[1], Mx[2], Mx[4], Mx[5], Mx[6], Mx[8], Mx[9], Mx[10]};
        it = 0;
        if (!inv3(J0, H)) finish = true;
      } else if (phase == 1) {
        const float3 rn = search_residual(Mx, q, xn);
        const float3 dr = make_float3(__fsub_rn(rn.x, r.x), __fsub_rn(rn.y, r.y), __fsub_rn(rn.z, r.z));
        x = q;
        r = rn;
        ++it;
        st.iters++;
        broyden_update(H, dx, dr);
      }
      if (phase != 2 && !finish) {
        if (search_norm2(r) < cfg.tol2) {
          conv = true;
          finish = true;
        } else if (it >= cfg.max_iter) {
          finish = true;
        } else {
          dx = search_dir(H, r);
          phase = 1;
        }
      }
      if (ord == ItemOrder::kPerLane) {
        // the lane owns its sample and runs its starts in order: the first of
        // equal roots is the earlier start's
        if (finish) {
          if (conv && in_box(S, x)) {
            st.converged++;
            const int nr = qs.nroots[cur];
            bool dup = false;
            for (int j2 = 0; j2 < nr; ++j2) {
              const float4 o = qs.roots[j2 * kList + cur];
              const float ddx = x.x - o.x, ddy = x.y - o.y, ddz = x.z - o.z;
              if (ddx * ddx + ddy * ddy + ddz * ddz < 1e-8f) { dup = true; break; }
            }
            if (!dup) {
              st.roots++;
              const int code = (order << 8) | label;
              if (nr < kMaxRoots) {
                qs.roots[nr * kList + cur] = make_float4(x.x, x.y, x.z, __int_as_float(code));
                qs.nroots[cur] = (uint8_t)(nr + 1);
              } else {
                compress_roots<P>(S, M, F, fs, qs.roots + cur, xn, x, code);
                qs.nroots[cur] = 1;
              }
            }
          }
          phase = 2;
          need = true;
        }
      } else {
        bool fresh = false;
        int dupj = -1;
        const int code = (order << 8) | label;
        if (finish) {
          if (conv && in_box(S, x)) {
            st.converged++;
            // most converged starts find a root already listed: those only lower
            // the listed root's start code, in parallel
            const int nr = qs.nroots[cur];
            fresh = true;
            for (int j = 0; j < nr; ++j) {
              float4* o = qs.roots + j * kList + cur;
              const float ddx = x.x - o->x, ddy = x.y - o->y, ddz = x.z - o->z;
              if (ddx * ddx + ddy * ddy + ddz * ddz < 1e-8f) {
                atomicMin(reinterpret_cast<int*>(&o->w), code);
                fresh = false;
                dupj = j;
                break;
              }
            }
          }
          phase = 2;
          need = true;
        }
        __syncwarp();
        // the earliest start's position stays with the root (codes of a sample are distinct)
        if (dupj >= 0 && __float_as_int(qs.roots[dupj * kList + cur].w) == code) {
          float4* o = qs.roots + dupj * kList + cur;
          o->x = x.x;
          o->y = x.y;
          o->z = x.z;
        }
        __syncwarp();
        // the others are merged into their samples' lists one at a time (two of
        // this step's roots may be the same)
        unsigned ins = __ballot_sync(kFull, fresh);
        while (ins) {
          const int ld = __ffs(ins) - 1;
          ins &= ins - 1u;
          const int s_l = __shfl_sync(kFull, cur, ld);
          const float px = __shfl_sync(kFull, x.x, ld), py = __shfl_sync(kFull, x.y, ld),
                      pz = __shfl_sync(kFull, x.z, ld);
          const int code_l = (__shfl_sync(kFull, order, ld) << 8) | __shfl_sync(kFull, label, ld);
          const int nr = qs.nroots[s_l];
          bool dup = false;
          float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
          if (lane < nr) {
            o = qs.roots[lane * kList + s_l];
            const float ddx = px - o.x, ddy = py - o.y, ddz = pz - o.z;
            dup = ddx * ddx + ddy * ddy + ddz * ddz < 1e-8f;
          }
          const unsigned dupm = __ballot_sync(kFull, dup);
          if (dupm) {
            // the same root: the list keeps the earlier start's (its position too)
            if (lane == __ffs(dupm) - 1 && code_l < __float_as_int(o.w))
              qs.roots[lane * kList + s_l] = make_float4(px, py, pz, __int_as_float(code_l));
          } else if (lane == ld) {
            st.roots++;
            if (nr < kMaxRoots) {
              qs.roots[nr * kList + s_l] = make_float4(px, py, pz, __int_as_float(code_l));
              qs.nroots[s_l] = (uint8_t)(nr + 1);
            } else {
              compress_roots<P>(S, M, F, fs, qs.roots + s_l, xn, x, code_l);
              qs.nroots[s_l] = 1;
            }
          }
          __syncwarp();
        }
      }
    }
    __syncwarp();
  }
  list_field_phase<P, kCompact>(S, F, fs, qs, m, src, dst);
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
