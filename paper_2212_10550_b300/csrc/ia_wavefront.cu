// Wavefront render path (sm_103a): the frame as a sequence of kernels over
// arrays instead of one persistent kernel per ray batch.
//
//   wf_march_kernel      one thread per ray: the slots in occupied cells that
//                        root culling keeps, written contiguously per ray (Sec.
//                        3.2-3.3; the same fp32 indexing as the fused render)
//   wf_propose_kernel    (proposal search) the network's top-2 bones and start
//                        offset for every sample, 32 samples per warp MMA
//   wf_search_kernel     one thread per (sample, start) item: bone-wise Broyden
//                        from that start (Sec. 3.1, Eq. 7), its converged root
//                        inside the canonical box, or none
//   wf_fallback_kernel   (proposal search) the samples none of whose proposed
//                        starts found a root, less those whose point lies in
//                        no canonical cell's grown image box; a second search
//                        wave runs every bone-wise start of those samples only
//   wf_field_kernel      per sample: its item results merged in start order
//                        (a root within 1e-4 of an earlier one is that root),
//                        one Newton polish per root, the field at the roots,
//                        the max-density root (Sec. 3.1, Eq. 1-4)
//   wf_composite_kernel  one thread per ray: front-to-back compositing of its
//                        samples with early termination (Sec. 3.2, Eq. 8)
//
// Each sample's result is bit for bit the fused render's with the plain search
// (the same starts, the same explicitly rounded Broyden arithmetic of
// ia_device.cuh, merge rule, polish, field and selection; the difference is the
// schedule), and with the proposal search up to the fused kernel's fallback
// queue merging a sample's roots in another order.  The search
// items are independent and light (the Broyden state and the last cell's 8
// corner records: 158 registers, three blocks of four warps per SM against
// one block of eight warps for the fused kernel), and the
// proposal's fallback starts, a few per ray where they occur, form one dense
// wave instead of a tail per list.  Samples behind the point where a ray's
// transmittance falls below the threshold are searched too (the march does
// not know the densities yet): 3 % more samples on the full-size frame.  The
// training step's forward and the occupancy refresh run the same per-sample
// kernels over their own samples (each with its pose).
#include "ia_internal.h"

namespace ia {

namespace {

// warp-aggregated reservation of `count` consecutive entries of *counter; returns
// this lane's first entry (all 32 lanes call)
__device__ __forceinline__ int warp_reserve(unsigned* counter, int count) {
  const int lane = threadIdx.x & 31;
  int incl = count;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  int base = 0;
  if (lane == 31 && total > 0) base = (int)atomicAdd(counter, (unsigned)total);
  base = __shfl_sync(kFull, base, 31);
  return base + incl - count;
}

template <class F>
__device__ __forceinline__ void for_each_kept_slot(const RenderArgs& a, const float o[3], const float d[3], float tn,
                                                   float dt, unsigned& marched, unsigned& culled, F kept) {
  for (int i = 0; i < a.n_slots; ++i) {
    const float3 x = slot_position(o, d, tn, dt, i);
    const int cell = cell_of(a.box, x);
    ++marched;
    if ((__ldg(a.occ + (cell >> 5)) >> (cell & 31)) & 1u) {
      if (a.sub && !sub_marked(a.sub, a.box, x)) ++culled;
      else kept(x);
    }
  }
}

}  // namespace

// ---- march: count, reserve, emit (one thread per ray id, tile order).  With
//      at most kMaskSlots slots the count pass records the kept slots in a
//      register mask and the emit pass visits only those; above, it marches
//      again.  Measured against it: one warp per ray with its lanes over the
//      slots and one reservation per block (0.64 ms: the block's atomic on one
//      counter is on every block's critical path), and a warp marching 32 rays
//      in turn with its lanes over the slots (0.128 ms against 0.111 ms: the
//      ballots, broadcasts and mask bookkeeping cost as much as the second
//      pass saved).
constexpr int kMaskSlots = 128;

template <bool kMask>
__global__ void __launch_bounds__(256) wf_march_kernel(const RenderArgs a, const WfArgs w) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  const int W = a.cam.width, H = a.cam.height;
  int u = 0, v = 0;
  bool valid = false;
  if (id < a.n_ray_ids) tile_pixel(id, a.tiles_x, W, H, u, v, valid);
  float o[3], d[3], tn = 0.f, tf = 0.f;
  const bool hit = valid && make_ray(a.cam, a.B0inv, a.box, u, v, o, d, tn, tf);
  const float dt = hit ? slot_delta(tn, tf, a.n_slots) : 0.f;
  unsigned marched = 0, culled = 0;
  int cnt = 0;
  uint32_t mk[kMaskSlots / 32] = {};
  if (hit) {
    if constexpr (kMask) {
#pragma unroll
      for (int q = 0; q < kMaskSlots / 32; ++q) {
        for (int b = 0; b < 32; ++b) {
          const int i = 32 * q + b;
          if (i >= a.n_slots) break;
          const float3 x = slot_position(o, d, tn, dt, i);
          const int cell = cell_of(a.box, x);
          ++marched;
          if ((__ldg(a.occ + (cell >> 5)) >> (cell & 31)) & 1u) {
            if (a.sub && !sub_marked(a.sub, a.box, x)) {
              ++culled;
            } else {
              mk[q] |= 1u << b;
              ++cnt;
            }
          }
        }
      }
    } else {
      for_each_kept_slot(a, o, d, tn, dt, marched, culled, [&](float3) { ++cnt; });
    }
  }
  const int first = warp_reserve(w.n_samples, cnt);
  const int pix = v * W + u;
  if (valid) {
    w.ray_first[pix] = first;
    w.ray_cnt[pix] = cnt;
    w.ray_dt[pix] = dt;
  }
  if (cnt > 0 && first + cnt <= w.cap) {  // beyond the capacity the host grows it and marches again
    int k = first;
    if constexpr (kMask) {
#pragma unroll
      for (int q = 0; q < kMaskSlots / 32; ++q) {
        for (uint32_t m = mk[q]; m; m &= m - 1u) {
          const float3 x = slot_position(o, d, tn, dt, 32 * q + __ffs(m) - 1);
          w.xn[k++] = make_float4(x.x, x.y, x.z, 0.f);
        }
      }
    } else {
      unsigned m2 = 0, c2 = 0;
      for_each_kept_slot(a, o, d, tn, dt, m2, c2, [&](float3 x) { w.xn[k++] = make_float4(x.x, x.y, x.z, 0.f); });
    }
  }
  if (a.stats)
    flush_stats_block<5>(a.stats, {ST_RAYS, ST_HIT, ST_MARCHED, ST_OCC, ST_CULLED},
                         {valid ? 1 : 0, hit ? 1 : 0, marched, (long long)cnt + culled, culled});
}

// ---- the proposal's bones and start offset for every sample
// shared memory: the network's weights (reduced precision, the pose's inputs
// folded into the first layer's bias) and each warp's MMA staging area
constexpr int kPropPad = (kPropWords + 3) / 4 * 4;
constexpr size_t propose_smem_bytes(int threads) {
  return sizeof(uint32_t) * (kPropPad + (size_t)(threads / 32) * kPropStageWords);
}

template <Prec P>
__global__ void __launch_bounds__(256) wf_propose_kernel(const RenderArgs a, const WfArgs w) {
  extern __shared__ float4 smem4[];
  uint32_t* pw = reinterpret_cast<uint32_t*>(smem4);
  stage_prop_h<P>(a.P.prop, a.P.cfg.nb, a.P.theta, pw);
  __syncthreads();
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  uint32_t* xstage = pw + kPropPad + (threadIdx.x >> 5) * kPropStageWords;
  const int n = chunk_size(w);
  const PropDev& Q = a.P.prop;
  const int nb = a.P.cfg.nb;
  unsigned proposed = 0;
  for (int s0 = (blockIdx.x * warps + (threadIdx.x >> 5)) * 32; s0 < n; s0 += gridDim.x * warps * 32) {
    const int s = s0 + lane;
    const bool act = s < n;
    float3 xn = make_float3(Q.nmin[0], Q.nmin[1], Q.nmin[2]);
    int pose = 0;
    if (act) {
      const float4 p = w.xn[w.s0 + s];
      xn = make_float3(p.x, p.y, p.z);
      pose = __float_as_int(p.w);
    }
    prop_encode_staged<P>(Q, xn, xstage + lane * kPW1Stride);
    // with per-pose layer-1 biases (Q.b1p) each row takes its sample's pose's
    const float* O = prop_mma_warp<P, true>(pw, xstage, nullptr, Q.b1p, pose) + lane * (kPropMaxOut + 1);
    if (act) {
      // the top-2 bones by logit (ties to the lower bone), as the fused search
      int b0 = 0, b1 = -1;
      float v0 = O[0], v1 = -3.0e38f;
      for (int k = 1; k < nb; ++k) {
        const float v = O[k];
        if (v > v0) { b1 = b0; v1 = v0; b0 = k; v0 = v; }
        else if (v > v1) { b1 = k; v1 = v; }
      }
      if (b1 < 0) b1 = b0;
      w.prop[s] = make_float4(__int_as_float(b0 | (b1 << 8)), O[nb], O[nb + 1], O[nb + 2]);
      ++proposed;
    }
    __syncwarp();  // every lane has read its row before the staging area is reused
  }
  if (a.stats) flush_stats(a.stats, ST_PROP, proposed);
}

// ---- search items: wave 0 = every start of every sample (plain search) or the
//      proposed starts; wave 1 = every start of the fallback samples
// Items are handed out grid-stride in sample-major order, so a warp's lanes
// run the starts of one or two samples in step: as their iterations converge
// onto the same few roots, the lanes' gathers fall on the same grid cells and
// share cache lines.  Measured against it on the full-size frame: refilling
// each lane with the next item as it finishes (lanes busy but scattered) is
// 1.2x slower, start-major order (neighbouring samples' starts of one bone
// together) 1.7x slower.
// The inverse rest-to-pose transforms the items start from are staged in
// shared memory (w.n_ninv floats, 1.1 KB per pose at 24 bones) when they fit
// kNinvSmemFloats (one pose: the render, the occupancy refresh), else read
// from global memory (the training step's 16 poses: staging them, 18 KB per
// block, took L1 capacity from the gathers and was slower).
// Each item keeps the corner records of the cell it gathered last in registers
// (CornerCache): about half of the Broyden steps stay in their cell and skip
// the gather.  Measured on the full-size frame against gathering every step at
// 128 registers and 16 warps per SM: plain search 3.90 -> 3.61 ms, proposal
// wave 0.44 -> 0.33 ms.  Wider loads of the same records were slower: a corner
// pair (x, x + 1) as 256-bit loads, 4.5-4.8 ms.
constexpr int kNinvSmemFloats = 1024;

template <bool kProp>
__global__ void __launch_bounds__(128, 3) wf_search_kernel(const RenderArgs a, const WfArgs w, int wave) {
  extern __shared__ float4 sNinv4[];
  const int nb = a.P.cfg.nb;
  const SkinDev& S = a.P.S;
  const bool staged = w.n_ninv <= kNinvSmemFloats;
  if (staged) {
    const float4* g4 = reinterpret_cast<const float4*>(w.ninv);
    for (int t = threadIdx.x; t < w.n_ninv / 4; t += blockDim.x) sNinv4[t] = g4[t];
  }
  __syncthreads();
  const float4* ninv4 = staged ? sNinv4 : reinterpret_cast<const float4*>(w.ninv);
  const int nprop = kProp ? min(a.P.prop.top_k, nb) : 0;
  const int per = (kProp && wave == 0) ? nprop : nb;
  const int n = wave == 0 ? chunk_size(w) : (int)*w.n_fb;
  const int total = n * per;  // the host keeps samples x bones below 2^30
  float4* out = wave == 0 ? w.item0 : w.item1;
  const int max_iter = a.P.cfg.max_iter;
  const float tol2 = a.P.cfg.tol2;
  unsigned starts = 0, iters = 0, conv_n = 0, gathers = 0;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int q = (int)((unsigned)it / (unsigned)per), j = it - q * per;
    const int s = wave == 0 ? q : w.fb[q];
    const float4 p4 = w.xn[w.s0 + s];
    const float3 xn = make_float3(p4.x, p4.y, p4.z);
    const int pose = __float_as_int(p4.w);
    const float4* M = S.M + (size_t)pose * w.pose_stride;
    int label = j, order = (wave == 0 ? 0 : nprop) + j;
    float3 poff = make_float3(0.f, 0.f, 0.f);
    if (kProp && wave == 0) {
      const float4 pp = w.prop[s];
      const int bb = __float_as_int(pp.x);
      label = j == 0 ? (bb & 0xff) : ((bb >> 8) & 0xff);
      if (j == 0) poff = make_float3(pp.y, pp.z, pp.w);
      order = j;
    }
    float A[12];
    {
      const float4* r = ninv4 + ((size_t)pose * nb + label) * 3;
      const float4 r0 = r[0], r1 = r[1], r2 = r[2];
      A[0] = r0.x; A[1] = r0.y; A[2] = r0.z; A[3] = r0.w;
      A[4] = r1.x; A[5] = r1.y; A[6] = r1.z; A[7] = r1.w;
      A[8] = r2.x; A[9] = r2.y; A[10] = r2.z; A[11] = r2.w;
    }
    float3 x = search_start(A, xn, kProp && wave == 0 && j == 0, poff);
    float Mx[12];
    CornerCache cells;
    gathers += cells.blend(S, M, x, Mx);
    ++starts;
    float3 r = search_residual(Mx, x, xn);
    // initial inverse Jacobian: LBS with the weights frozen at x0, (sum_i w_i R_i)^-1
    const float J0[9] = {Mx[0], Mx[1], Mx[2], Mx[4], Mx[5], Mx[6], Mx[8], Mx[9], Mx[10]};
    float H[9];
    bool conv = false;
    if (inv3(J0, H)) {
      for (int k = 0;; ++k) {
        if (search_norm2(r) < tol2) {
          conv = true;
          break;
        }
        if (k >= max_iter) break;
        const float3 dx = search_dir(H, r);
        x = add3(x, dx);
        gathers += cells.blend(S, M, x, Mx);
        ++iters;
        const float3 rn = search_residual(Mx, x, xn);
        const float3 dr = make_float3(__fsub_rn(rn.x, r.x), __fsub_rn(rn.y, r.y), __fsub_rn(rn.z, r.z));
        r = rn;
        broyden_update(H, dx, dr);
      }
    }
    const bool valid = conv && in_box(S, x);
    conv_n += valid;
    out[it] = make_float4(x.x, x.y, x.z, __int_as_float(valid ? ((order << 8) | label) : -1));
  }
  if (a.stats)
    flush_stats_block<4>(a.stats, {ST_STARTS, ST_ITERS, ST_CONV, ST_GATHERS},
                         {(long long)starts, (long long)iters, (long long)conv_n, (long long)gathers});
}

// ---- the samples whose proposed starts found no root.  With box lists (the
//      render's, per occupied cell; the training step's, per pose and cell), a
//      point that lies in no grown image box of a skinning cell meeting its
//      occupancy cell has no root (the culling bound, point by point): it gets
//      density 0 without the fallback search, which would find none.  A list
//      is complete when its count is at most the cap, and tested when it is at
//      most blist_scan long (measured: the training lists, which hold every
//      cell a box meets, pay only when short; the render's are scanned whole).
constexpr int kShortBoxList = 16;  // lists scanned with all their loads issued at once

__global__ void __launch_bounds__(256) wf_fallback_kernel(const RenderArgs a, const WfArgs w) {
  const int n = chunk_size(w);
  const int nprop = min(a.P.prop.top_k, a.P.cfg.nb);
  unsigned fell = 0, pculled = 0;
  // whole warps step together (warp_reserve needs all 32 lanes)
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int s = base + threadIdx.x;
    bool fall = false;
    if (s < n) {
      fall = true;
      for (int j = 0; j < nprop; ++j) fall &= __float_as_int(w.item0[(size_t)s * nprop + j].w) < 0;
    }
    if (fall && w.blist) {
      const float4 p4 = w.xn[w.s0 + s];
      const int pose = __float_as_int(p4.w);
      const size_t c = (size_t)pose * w.blist_pose_cells + cell_of(a.box, make_float3(p4.x, p4.y, p4.z));
      const int nbox = w.blist_count[c];
      const float4* boxes = w.cell_box + 2 * (size_t)pose * w.box_pose_cells;
      auto inside = [&](int b) {
        const float4 lo = boxes[2 * (size_t)b], hi = boxes[2 * (size_t)b + 1];
        return p4.x >= lo.x && p4.x <= hi.x && p4.y >= lo.y && p4.y <= hi.y && p4.z >= lo.z && p4.z <= hi.z;
      };
      bool tested = false, in = false;
      if (nbox <= kShortBoxList) {  // every load issued at once
        int b[kShortBoxList];
#pragma unroll
        for (int k = 0; k < kShortBoxList; ++k) b[k] = k < nbox ? w.blist[c * w.blist_cap + k] : -1;
#pragma unroll
        for (int k = 0; k < kShortBoxList; ++k) in |= b[k] >= 0 && inside(b[k]);
        tested = true;
      } else if (nbox <= w.blist_scan) {  // a longer, complete list: box by box
        for (int k = 0; k < nbox && !in; ++k) in = inside(w.blist[c * w.blist_cap + k]);
        tested = true;
      }
      if (tested && !in) {
        fall = false;
        ++pculled;
      }
    }
    const int idx = warp_reserve(w.n_fb, fall ? 1 : 0);
    if (s < n) w.fbidx[s] = fall ? idx : -1;
    if (fall) w.fb[idx] = s;
    fell += fall;
  }
  if (a.stats) {
    flush_stats(a.stats, ST_FALLBACK, fell);
    flush_stats(a.stats, ST_PCULLED, pculled);
  }
}

// ---- per sample: merge the item results, polish, field, max-density root
template <Prec P, bool kProp>
__device__ __forceinline__ void field_body(const RenderArgs& a, const WfArgs& w, float4* smem4) {
  PosedStage ps = stage_of(a.P);
  ps.search = 0;  // the field only: no proposal staged here
  PosedSmem sm = stage_posed<P>(ps, smem4);
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  const SkinDev& S = a.P.S;
  const int nb = a.P.cfg.nb;
  const int nprop = kProp ? min(a.P.prop.top_k, nb) : 0;
  const int per0 = kProp ? nprop : nb;
  const int n = chunk_size(w);
  const ListSmem& qs = sm.list;
  unsigned roots = 0, rooted = 0;
  for (int s0 = (blockIdx.x * warps + (threadIdx.x >> 5)) * 32; s0 < n; s0 += gridDim.x * warps * 32) {
    const int m = min(32, n - s0);
    const int s = s0 + lane;
    if (lane < m) {
      const float4 p4 = w.xn[w.s0 + s];
      const float3 xn = make_float3(p4.x, p4.y, p4.z);
      const float4* M = S.M + (size_t)__float_as_int(p4.w) * w.pose_stride;
      int nr = 0;
      // items in start order: the first of equal roots keeps its position and code
      auto merge = [&](const float4 r) {
        const int code = __float_as_int(r.w);
        if (code < 0) return;
        for (int j2 = 0; j2 < nr; ++j2) {
          const float4 o = qs.roots[j2 * kList + lane];
          const float ddx = r.x - o.x, ddy = r.y - o.y, ddz = r.z - o.z;
          if (ddx * ddx + ddy * ddy + ddz * ddz < 1e-8f) return;
        }
        ++roots;
        if (nr < kMaxRoots) {
          qs.roots[nr * kList + lane] = r;
          ++nr;
        } else {
          compress_roots<P>(S, M, a.P.F, sm.fs, qs.roots + lane, xn, make_float3(r.x, r.y, r.z), code);
          nr = 1;
        }
      };
      for (int j = 0; j < per0; ++j) merge(w.item0[(size_t)s * per0 + j]);
      if (kProp) {
        const int fi = w.fbidx[s];
        if (fi >= 0)
          for (int k = 0; k < nb; ++k) merge(w.item1[(size_t)fi * nb + k]);
      }
      qs.nroots[lane] = (uint8_t)nr;
    }
    __syncwarp();
    list_field_phase<P, P != Prec::F32>(
        S, a.P.F, sm.fs, qs, m,
        [&](int i, float3& xq, const float4*& Mq, const float*& Nq, int& pose) {
          const float4 p4 = w.xn[w.s0 + s0 + i];
          xq = make_float3(p4.x, p4.y, p4.z);
          pose = __float_as_int(p4.w);
          Mq = S.M + (size_t)pose * w.pose_stride;
          Nq = w.ninv + (size_t)pose * nb * 12;
        },
        [&](int i, const PosedOut& o) {
          const bool has = o.start >= 0;
          rooted += has;
          w.res[w.s0 + s0 + i] = make_float4(has ? o.sigma : 0.f, o.rgb.x, o.rgb.y, o.rgb.z);
          if (w.xs) w.xs[w.s0 + s0 + i] = make_float4(o.xstar.x, o.xstar.y, o.xstar.z, has ? 1.f : 0.f);
        });
  }
  if (a.stats) {
    flush_stats(a.stats, ST_ROOTS, roots);
    flush_stats(a.stats, ST_ROOTED, rooted);
  }
}

// fp32: the per-lane MLP holds its activations in registers (one block of 8
// warps per SM; register caps for two blocks spill and gained at most 6 %)
__global__ void __launch_bounds__(256) wf_field_kernel_f32(const RenderArgs a, const WfArgs w) {
  extern __shared__ float4 smem4[];
  field_body<Prec::F32, false>(a, w, smem4);
}

// fp16 / bf16: the MLP runs on the warp MMA from staged operands; with the
// proposal (2 proposed items per sample to merge, and the fallback's) two
// blocks per SM, with the plain search (24 items per sample) one
template <Prec P, bool kProp>
__global__ void __launch_bounds__(256, kProp ? 2 : 1) wf_field_kernel(const RenderArgs a, const WfArgs w) {
  extern __shared__ float4 smem4[];
  field_body<P, kProp>(a, w, smem4);
}

template <Prec P, bool kProp>
static constexpr auto field_kernel() {
  if constexpr (P == Prec::F32) return wf_field_kernel_f32;
  else return wf_field_kernel<P, kProp>;
}

// ---- per ray: front-to-back compositing, alpha_i = 1 - exp(-sigma_i delta)
__global__ void __launch_bounds__(256) wf_composite_kernel(const RenderArgs a, const WfArgs w) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  const int npix = a.cam.width * a.cam.height;
  unsigned early = 0;
  if (pix < npix) {
    const float log_stop = a.early_T > 0.f ? -logf(a.early_T) : __int_as_float(0x7f800000);
    const int cnt = w.ray_cnt[pix], first = w.ray_first[pix];
    const float dt = w.ray_dt[pix];
    float depth = 0.f, cr = 0.f, cg = 0.f, cb = 0.f;
    for (int j = 0; j < cnt; ++j) {
      const float4 sres = w.res[first + j];
      if (sres.x > 0.f) {
        const float sd = sres.x * dt;
        const float wgt = expf(-depth) * -expm1f(-sd);  // T_i alpha_i
        cr = fmaf(wgt, sres.y, cr);
        cg = fmaf(wgt, sres.z, cg);
        cb = fmaf(wgt, sres.w, cb);
        depth += sd;
      }
      if (depth > log_stop) {  // transmittance below the threshold: the ray stops
        ++early;
        break;
      }
    }
    a.rgb[3 * pix] = cr;
    a.rgb[3 * pix + 1] = cg;
    a.rgb[3 * pix + 2] = cb;
    a.alpha[pix] = -expm1f(-depth);
  }
  if (a.stats) flush_stats_block<1>(a.stats, {ST_EARLY}, {(long long)early});
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// launch names for the traces, by caller: the render, the occupancy density,
// the training step's forward
#define IA_WF_NAMES(base) \
  { base, base " [occupancy]", base " [train]" }
constexpr const char* kNameSearch[3] = IA_WF_NAMES("wf_search_kernel");
constexpr const char* kNameSearchProp[3] = IA_WF_NAMES("wf_search_kernel<proposal>");
constexpr const char* kNameSearchFb[3] = IA_WF_NAMES("wf_search_kernel<fallback>");
constexpr const char* kNameFallback[3] = IA_WF_NAMES("wf_fallback_kernel");
constexpr const char* kNamePropose16[3] = IA_WF_NAMES("wf_propose_kernel<fp16>");
constexpr const char* kNamePropose16b[3] = IA_WF_NAMES("wf_propose_kernel<bf16>");
constexpr const char* kNameField32[3] = IA_WF_NAMES("wf_field_kernel<fp32>");
constexpr const char* kNameField16[3] = IA_WF_NAMES("wf_field_kernel<fp16>");
constexpr const char* kNameField16p[3] = IA_WF_NAMES("wf_field_kernel<fp16,proposal>");
constexpr const char* kNameFieldB[3] = IA_WF_NAMES("wf_field_kernel<bf16>");
constexpr const char* kNameFieldBp[3] = IA_WF_NAMES("wf_field_kernel<bf16,proposal>");
#undef IA_WF_NAMES

template <Prec P>
constexpr const char* wf_field_name(bool prop, int role) {
  return P == Prec::F32 ? kNameField32[role]
                        : (P == Prec::F16 ? (prop ? kNameField16p[role] : kNameField16[role])
                                          : (prop ? kNameFieldBp[role] : kNameFieldB[role]));
}

cudaError_t launch_wf_march(const RenderArgs& a, const WfArgs& w, cudaStream_t s) {
  KernelSpan span("wf_march_kernel", s);
  if (a.n_slots <= kMaskSlots) wf_march_kernel<true><<<(a.n_ray_ids + 255) / 256, 256, 0, s>>>(a, w);
  else wf_march_kernel<false><<<(a.n_ray_ids + 255) / 256, 256, 0, s>>>(a, w);
  return cudaGetLastError();
}

template <Prec P, bool kProp>
static cudaError_t launch_wf_chunk_p(const RenderArgs& a, const WfArgs& w, int num_sms, cudaStream_t s) {
  cudaError_t e;
  const int n = w.ns;
  if (n <= 0) return cudaSuccess;
  if constexpr (kProp) {
    if ((e = cudaMemsetAsync(w.n_fb, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    const size_t smem = propose_smem_bytes(256);
    if ((e = set_smem(wf_propose_kernel<P>, smem, 256)) != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wf_propose_kernel<P>, 256, smem)) != cudaSuccess)
      return e;
    const int blocks = min((n + 255) / 256, num_sms * max(per_sm, 1));
    {
      KernelSpan span(P == Prec::F16 ? kNamePropose16[w.role] : kNamePropose16b[w.role], s);
      wf_propose_kernel<P><<<blocks, 256, smem, s>>>(a, w);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int grid = num_sms * 4 * 8;  // items are handed out grid-stride
  const size_t ninv_smem = w.n_ninv <= kNinvSmemFloats ? sizeof(float) * w.n_ninv : 0;
  {
    KernelSpan span(kProp ? kNameSearchProp[w.role] : kNameSearch[w.role], s);
    wf_search_kernel<kProp><<<grid, 128, ninv_smem, s>>>(a, w, 0);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if constexpr (kProp) {
    {
      KernelSpan span(kNameFallback[w.role], s);
      wf_fallback_kernel<<<min((n + 255) / 256, num_sms * 8), 256, 0, s>>>(a, w);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
      KernelSpan span(kNameSearchFb[w.role], s);
      wf_search_kernel<kProp><<<grid, 128, ninv_smem, s>>>(a, w, 1);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  constexpr int kFT = 256;
  const size_t smem = posed_smem_bytes_p<P>(kFT, false);
  constexpr auto kField = field_kernel<P, kProp>();
  if ((e = set_smem(kField, smem, kFT)) != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kField, kFT, smem)) != cudaSuccess) return e;
  const int blocks = min((n + kFT - 1) / kFT, num_sms * max(per_sm, 1));
  {
    KernelSpan span(wf_field_name<P>(kProp, w.role), s);
    kField<<<blocks, kFT, smem, s>>>(a, w);
  }
  return cudaGetLastError();
}

cudaError_t launch_wf_chunk(const RenderArgs& a, const WfArgs& w, int num_sms, cudaStream_t s) {
  switch (a.P.prec) {
    case 1:
      return a.P.search ? launch_wf_chunk_p<Prec::F16, true>(a, w, num_sms, s)
                        : launch_wf_chunk_p<Prec::F16, false>(a, w, num_sms, s);
    case 2:
      return a.P.search ? launch_wf_chunk_p<Prec::BF16, true>(a, w, num_sms, s)
                        : launch_wf_chunk_p<Prec::BF16, false>(a, w, num_sms, s);
    default:
      return launch_wf_chunk_p<Prec::F32, false>(a, w, num_sms, s);
  }
}

// ---- occupancy density (Sec. 3.3) through the same kernels: each searched
//      cell's query point is a sample of pose 0, its density goes back to the
//      cell's entry of sigma
__global__ void wf_occ_points_kernel(const BoxDev box, const float* __restrict__ jitter,
                                     const int* __restrict__ cells, const unsigned* __restrict__ count, int n_all,
                                     float4* __restrict__ xn) {
  const int n = cells ? (int)*count : n_all;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = cells ? cells[i] : i;
    const float3 x = jitter ? cell_point(box, c, jitter + 3 * (size_t)c) : cell_center(box, c);
    xn[i] = make_float4(x.x, x.y, x.z, 0.f);  // pose 0 (int bits of 0.f)
  }
}

__global__ void wf_occ_scatter_kernel(const int* __restrict__ cells, const unsigned* __restrict__ count, int n_all,
                                      const float4* __restrict__ res, float* __restrict__ sigma) {
  const int n = cells ? (int)*count : n_all;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    sigma[cells ? cells[i] : i] = res[i].x;
}

cudaError_t launch_wf_occupancy(const PosedArgs& P, const BoxDev& box, const float* jitter, const int* cells,
                                const unsigned* count, float* sigma, unsigned long long* stats, WfArgs w, int num_sms,
                                cudaStream_t s) {
  const int n_all = box.R * box.R * box.R;
  RenderArgs ra{};
  ra.P = P;
  ra.stats = stats;
  w.s0 = 0;
  w.ns = n_all;
  w.ns_dev = cells ? count : nullptr;
  w.pose_stride = 0;
  w.ninv = P.Ninv;
  w.n_ninv = P.cfg.nb * 12;
  w.xs = nullptr;
  w.role = kWfOccupancy;
  const int blocks = min((n_all + 255) / 256, num_sms * 8);
  cudaError_t e;
  {
    KernelSpan span("wf_occ_points_kernel", s);
    wf_occ_points_kernel<<<blocks, 256, 0, s>>>(box, jitter, cells, count, n_all, w.xn);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_wf_chunk(ra, w, num_sms, s)) != cudaSuccess) return e;
  {
    KernelSpan span("wf_occ_scatter_kernel", s);
    wf_occ_scatter_kernel<<<blocks, 256, 0, s>>>(cells, count, n_all, w.res, sigma);
  }
  return cudaGetLastError();
}

cudaError_t launch_wf_composite(const RenderArgs& a, const WfArgs& w, cudaStream_t s) {
  const int npix = a.cam.width * a.cam.height;
  {
    KernelSpan span("wf_composite_kernel", s);
    wf_composite_kernel<<<(npix + 255) / 256, 256, 0, s>>>(a, w);
  }
  return cudaGetLastError();
}

}  // namespace ia
