// Kernels of the articulated radiance-field render path (sm_103a).
//
//   pose_chain_kernel     fp64 kinematic chain -> fp32 normalised-space transforms
//   blend_kernel          per-pose blended transform grid M(v) = sum_i W(v,i) N_i
//   occ_density_kernel    posed-field density at every occupancy cell centre
//   occ_bits_kernel       threshold + dilation + packing (+ union into the training grid)
//   query_*_kernel        posed / canonical field at caller points
//   render_kernel         persistent fused march -> correspondence search -> hash
//                         encoding -> MLP -> front-to-back compositing
#include <algorithm>
#include <cmath>

#include "ia_internal.h"

// minimum resident CTAs per SM the compiler must fit (a register cap)
#ifndef IA_RENDER_MIN_BLOCKS
#define IA_RENDER_MIN_BLOCKS 1
#endif
#ifndef IA_POSED_MIN_BLOCKS
#define IA_POSED_MIN_BLOCKS 1
#endif

namespace ia {

// ---------------------------------------------------------------------------
// Pose chain (fp64, explicitly rounded so the fp32 results are reproducible)
// ---------------------------------------------------------------------------

__device__ __forceinline__ double DM(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double DA(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double DS(double a, double b) { return __dsub_rn(a, b); }

// cos a and sin a of a joint's rotation angle, from their Maclaurin series:
// a is reduced once by the nearest multiple of 2 pi (an fp64 constant), then
// the terms t_{k+1} = t_k (-x^2) r_k, with r_k = 1 / ((2k+2)(2k+3)) for sin
// (from t_0 = x) and 1 / ((2k+1)(2k+2)) for cos (from t_0 = 1), are formed
// and added in order, 22 of them (the first omitted one is below pi^46 / 46!
// < 1e-32).  The reciprocals are correctly rounded fp64 divisions, made once
// per block (recip[0][k] sin, recip[1][k] cos); every other step is one
// correctly rounded fp64 multiply or add in a fixed order, so the values --
// and the fp32 transforms made from them -- are reproducible on any IEEE
// machine, which a library cos / sin (accurate to an ulp or two, by
// machine-specific methods) is not.
constexpr int kSeriesTerms = 22;

__device__ __forceinline__ void cos_sin_series(double a, const double (*recip)[kSeriesTerms], double& c, double& s) {
  const double two_pi = 6.283185307179586;
  const double x = DS(a, DM(rint(__ddiv_rn(a, two_pi)), two_pi));
  const double mx2 = -DM(x, x);
  double ts = x, tc = 1.0, sn = x, cs = 1.0;
#pragma unroll 1
  for (int k = 0; k < kSeriesTerms; ++k) {
    ts = DM(DM(ts, mx2), recip[0][k]);
    tc = DM(DM(tc, mx2), recip[1][k]);
    sn = DA(sn, ts);
    cs = DA(cs, tc);
  }
  c = cs;
  s = sn;
}

// One block per pose, twelve threads per joint, thread (k, e) owning element e
// of joint k's 3 x 4 matrices.  The chain is composed level by level down the
// tree, G_k = G_p(k) L_k, which is the same left-to-right product
// ((L_root L_a1) L_a2) ... L_k as composing parent-first; every element is
// formed with the same rounded operations in the same order as a sequential
// 3 x 4 product, so the fp64 results do not depend on the thread layout.
// (fp64 runs at a small fraction of the fp32 rate here: spreading the products
// over the elements shortens the chain of dependent fp64 instructions.)
__device__ __forceinline__ double mat34_elem_d(const double* a, const double* b, int e) {
  const int i = e >> 2, j = e & 3;
  double s = DA(DA(DM(a[i * 4 + 0], b[0 * 4 + j]), DM(a[i * 4 + 1], b[1 * 4 + j])), DM(a[i * 4 + 2], b[2 * 4 + j]));
  if (j == 3) s = DA(s, a[i * 4 + 3]);
  return s;
}

// element e of the inverse of the rigid transform a = [R | t]: [R^T | -R^T t]
__device__ __forceinline__ double rigid_inv_elem_d(const double* a, int e) {
  const int i = e >> 2, j = e & 3;
  if (j < 3) return a[j * 4 + i];
  return -DA(DA(DM(a[0 * 4 + i], a[3]), DM(a[1 * 4 + i], a[7])), DM(a[2 * 4 + i], a[11]));
}

__global__ void pose_chain_kernel(int P, int nb, const int* __restrict__ parent, const double* __restrict__ rest,
                                  const double* __restrict__ theta, const double* __restrict__ trans,
                                  float* __restrict__ N, float* __restrict__ Ninv, float* __restrict__ B0inv) {
  __shared__ double sL[kMaxBones][12];   // local transforms [R_k | j_k - j_p(k)]
  __shared__ double sG[kMaxBones][12];   // chain G_k, then rest-relative B_k
  __shared__ double sN[kMaxBones][12];   // B_0^-1 B_k
  __shared__ double sRod[kMaxBones][6];  // c, s, 1 - c, unit axis
  __shared__ double sB0i[12];
  __shared__ double sRecip[2][kSeriesTerms];  // series reciprocals (sin, cos)
  __shared__ int sDepth[kMaxBones];
  __shared__ bool sZero[kMaxBones];      // zero rotation angle
  __shared__ int sMaxDepth;
  const int p = blockIdx.x;
  if (p >= P) return;
  const int t = threadIdx.x, k = t / 12, e = t % 12;
  const bool own = k < nb;
  if (t == 0) sMaxDepth = 0;
  for (int j = t; j < kSeriesTerms; j += blockDim.x) {  // one warp: both reciprocals of term j
    sRecip[0][j] = __ddiv_rn(1.0, (double)((2 * j + 2) * (2 * j + 3)));
    sRecip[1][j] = __ddiv_rn(1.0, (double)((2 * j + 1) * (2 * j + 2)));
  }
  __syncthreads();
  // the angle's scalars, thread q for joint q: the first warp(s) alone issue
  // these long fp64 sequences (a warp instruction costs the fp64 pipe the same
  // with 1 or 32 lanes active; with the joints' first threads, spread over every
  // warp of the block, the kernel took 29-34 us per pose)
  for (int q = t; q < nb; q += blockDim.x) {
    const double* th = theta + ((size_t)p * nb + q) * 3;
    const double a2 = DA(DA(DM(th[0], th[0]), DM(th[1], th[1])), DM(th[2], th[2]));
    const double a = __dsqrt_rn(a2);
    sZero[q] = a2 == 0.0;
    if (a == 0.0) {
      sRod[q][0] = 1.0;  // identity rotation
    } else {
      double c, sn;
      cos_sin_series(a, sRecip, c, sn);
      sRod[q][0] = c;
      sRod[q][1] = sn;
      sRod[q][2] = DS(1.0, c);
      sRod[q][3] = __ddiv_rn(th[0], a);
      sRod[q][4] = __ddiv_rn(th[1], a);
      sRod[q][5] = __ddiv_rn(th[2], a);
    }
    int d = 0;
    for (int j = parent[q]; j >= 0; j = parent[j]) ++d;
    sDepth[q] = d;
    atomicMax(&sMaxDepth, d);
  }
  __syncthreads();
  const int i = e >> 2, j = e & 3;
  if (own) {
    // Rodrigues: R = c I + (1 - c) k k^T + s [k]_x
    const bool zero = sZero[k];
    const int par = parent[k];
    double v;
    if (j == 3) {
      v = (par < 0) ? rest[3 * k + i] : DS(rest[3 * k + i], rest[3 * par + i]);
    } else if (zero) {
      v = i == j ? 1.0 : 0.0;
    } else {
      const double c = sRod[k][0], sn = sRod[k][1], C = sRod[k][2];
      const double ki = sRod[k][3 + i], kj = sRod[k][3 + j];
      const double Ck = DM(DM(C, ki), kj);
      if (i == j) {
        v = DA(c, Ck);
      } else {
        // the cross-product term s k_m, m the third axis; its sign as in [k]_x
        const int m = 3 - i - j;
        const double sk = DM(sn, sRod[k][3 + m]);
        const bool plus = (i == 0 && j == 2) || (i == 1 && j == 0) || (i == 2 && j == 1);
        v = plus ? DA(Ck, sk) : DS(Ck, sk);
      }
    }
    sL[k][e] = v;
  }
  __syncthreads();
  const int depth = own ? sDepth[k] : -1;
  const int maxd = sMaxDepth;
  for (int d = 0; d <= maxd; ++d) {  // parents are final before their children read them
    if (depth == d) sG[k][e] = d == 0 ? sL[k][e] : mat34_elem_d(sG[parent[k]], sL[k], e);
    __syncthreads();
  }
  // rest-relative bone transform B_k = G_k [I | -j_k] + root translation
  double b = 0.0;
  if (own) {
    const double* G = sG[k];
    if (j < 3) {
      b = G[e];
    } else {
      const double Rj = DA(DA(DM(G[i * 4 + 0], rest[3 * k + 0]), DM(G[i * 4 + 1], rest[3 * k + 1])),
                           DM(G[i * 4 + 2], rest[3 * k + 2]));
      b = DA(DS(G[i * 4 + 3], Rj), trans[(size_t)p * 3 + i]);
    }
  }
  __syncthreads();  // every thread has read its G before B overwrites it
  if (own) sG[k][e] = b;
  __syncthreads();
  if (k == 0) sB0i[e] = rigid_inv_elem_d(sG[0], e);  // the root is bone 0 (parents precede children)
  __syncthreads();
  if (own) sN[k][e] = mat34_elem_d(sB0i, sG[k], e);
  __syncthreads();
  if (own) {
    N[((size_t)p * nb + k) * 12 + e] = (float)sN[k][e];
    Ninv[((size_t)p * nb + k) * 12 + e] = (float)rigid_inv_elem_d(sN[k], e);
    if (k == 0) B0inv[(size_t)p * 12 + e] = (float)sB0i[e];
  }
}

cudaError_t launch_pose_chain(int P, int nb, const int* parent, const double* rest, const double* theta,
                              const double* trans, float* N, float* Ninv, float* B0inv, cudaStream_t s) {
  {
    KernelSpan span("pose_chain_kernel", s);
    pose_chain_kernel<<<P, (nb * 12 + 31) / 32 * 32, 0, s>>>(P, nb, parent, rest, theta, trans, N, Ninv, B0inv);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Blended transform grid M(v) = sum_i W(v, i) N_i, one pose per blockIdx.y
// ---------------------------------------------------------------------------

// kVec: nb a multiple of 4, a voxel's weights read as float4 (W's rows are then
// 16-byte aligned); the bones are summed in the same order either way.
template <bool kVec>
__global__ void blend_kernel(int V, int nb, const float* __restrict__ W, const float* __restrict__ N,
                             float4* __restrict__ M) {
  __shared__ float4 sN4[kMaxBones * 3];
  float* sN = reinterpret_cast<float*>(sN4);
  const int p = blockIdx.y;
  for (int t = threadIdx.x; t < nb * 12; t += blockDim.x) sN[t] = N[(size_t)p * nb * 12 + t];
  __syncthreads();
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    float acc[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) acc[q] = 0.f;
    const float* w = W + (size_t)v * nb;
    auto add_bone = [&](int i, float wi) {
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float4 n = sN4[i * 3 + r];
        acc[4 * r] = fmaf(wi, n.x, acc[4 * r]);
        acc[4 * r + 1] = fmaf(wi, n.y, acc[4 * r + 1]);
        acc[4 * r + 2] = fmaf(wi, n.z, acc[4 * r + 2]);
        acc[4 * r + 3] = fmaf(wi, n.w, acc[4 * r + 3]);
      }
    };
    if constexpr (kVec) {
      const float4* w4 = reinterpret_cast<const float4*>(w);
      for (int i4 = 0; i4 < nb / 4; ++i4) {
        const float4 wq = __ldg(w4 + i4);
        add_bone(4 * i4, wq.x);
        add_bone(4 * i4 + 1, wq.y);
        add_bone(4 * i4 + 2, wq.z);
        add_bone(4 * i4 + 3, wq.w);
      }
    } else {
      for (int i = 0; i < nb; ++i) add_bone(i, __ldg(w + i));
    }
    float4* out = M + ((size_t)p * V + v) * 3;
    out[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    out[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    out[2] = make_float4(acc[8], acc[9], acc[10], acc[11]);
  }
}

cudaError_t launch_blend(int P, int V, int nb, const float* W, const float* N, float4* M, cudaStream_t s) {
  dim3 grid((V + 255) / 256, P);
  if (grid.x > 4096) grid.x = 4096;
  {
    KernelSpan span("blend_kernel", s);
    if (nb % 4 == 0 && reinterpret_cast<uintptr_t>(W) % 16 == 0) blend_kernel<true><<<grid, 256, 0, s>>>(V, nb, W, N, M);
    else blend_kernel<false><<<grid, 256, 0, s>>>(V, nb, W, N, M);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Shared-memory layout of kernels that evaluate the posed field:
//   MLP (fp32 layout, or reduced-precision layout + per-warp staging), the
//   pose's N_k^-1, and the per-lane root lists.
// ---------------------------------------------------------------------------


// ---------------------------------------------------------------------------
// Occupancy grid (Sec. 3.3, inference mode)
// ---------------------------------------------------------------------------

// The fused occupancy density, kept for the allocation-free entry (the other
// occupancy calls run the wavefront kernels over the candidate cells): per
// warp a list of kOccList cells from a shared counter, each lane running its
// cell's starts in order with the search arithmetic and merge rule of the
// wavefront search, so both give the same densities bit for bit.
// cells: the cells to search (occ_cand_kernel's list, *count of them), or null
// for every cell of the grid.
constexpr int kOccList = 32;
template <Prec P, bool kProp>
__global__ void __launch_bounds__(256, IA_POSED_MIN_BLOCKS)
    occ_density_kernel(const PosedArgs a, const BoxDev box, const float* __restrict__ jitter,
                       const int* __restrict__ cells, const unsigned* __restrict__ count,
                       float* __restrict__ sigma, unsigned long long* __restrict__ stats,
                       unsigned* __restrict__ work) {
  extern __shared__ float4 smem4[];
  PosedSmem sm = stage_posed<P>(stage_of(a), smem4);
  const int n = cells ? (int)*count : box.R * box.R * box.R;
  SampleStats st;
  for (int list = next_list(work); list * kOccList < n; list = next_list(work)) {
    const int base = list * kOccList;
    posed_field_list<P, ItemOrder::kPerLane, kProp>(
        a.S, a.F, a.cfg, sm.fs, sm.list, min(kOccList, n - base),
        [&](int i, float3& xn, const float4*& M, const float*& Ni, int& pose) {
          const int c = cells ? cells[base + i] : base + i;
          xn = jitter ? cell_point(box, c, jitter + 3 * (size_t)c) : cell_center(box, c);
          M = a.S.M;
          Ni = sm.sNinv;
          pose = 0;
        },
        [&](int i, const PosedOut& o) {
          const int c = cells ? cells[base + i] : base + i;
          sigma[c] = o.start >= 0 ? o.sigma : 0.f;
        },
        st, a.prop, kProp);  // the proposal code is compiled only into kProp variants
  }
  if (stats) {
    flush_stats(stats, ST_STARTS, st.starts);
    flush_stats(stats, ST_ITERS, st.iters);
    flush_stats(stats, ST_GATHERS, st.starts + st.iters);
    flush_stats(stats, ST_CONV, st.converged);
    flush_stats(stats, ST_ROOTS, st.roots);
    flush_stats(stats, ST_PROP, st.proposed);
    flush_stats(stats, ST_FALLBACK, st.fallbacks);
  }
}

template <Prec P, bool kProp>
constexpr const char* occ_density_name() {
  return kProp ? variant_name<P>("occ_density_kernel<fp32,proposal>", "occ_density_kernel<fp16,proposal>",
                                 "occ_density_kernel<bf16,proposal>")
               : variant_name<P>("occ_density_kernel<fp32>", "occ_density_kernel<fp16>", "occ_density_kernel<bf16>");
}

template <Prec P, bool kProp>
static cudaError_t launch_occ_density_k(const PosedArgs& a, const BoxDev& box, const float* jitter, const int* cells,
                                        const unsigned* count, float* sigma, unsigned long long* stats,
                                        unsigned* work, int num_sms, cudaStream_t s) {
  const int n = box.R * box.R * box.R;
  const size_t smem = posed_smem_bytes_p<P>(256, kProp);
  cudaError_t e = set_smem(occ_density_kernel<P, kProp>, smem, 256);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, occ_density_kernel<P, kProp>, 256, smem);
  if (e != cudaSuccess) return e;
  const int lists = (n + kOccList - 1) / kOccList;
  int blocks = num_sms * (per_sm < 1 ? 1 : per_sm);
  if (blocks > (lists + 7) / 8) blocks = (lists + 7) / 8;
  if ((e = cudaMemsetAsync(work, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
  {
    KernelSpan span(occ_density_name<P, kProp>(), s);
    occ_density_kernel<P, kProp><<<blocks, 256, smem, s>>>(a, box, jitter, cells, count, sigma, stats, work);
  }
  return cudaGetLastError();
}

template <Prec P>
static cudaError_t launch_occ_density_p(const PosedArgs& a, const BoxDev& box, const float* jitter, const int* cells,
                                        const unsigned* count, float* sigma, unsigned long long* stats,
                                        unsigned* work, int num_sms, cudaStream_t s) {
  if constexpr (P != Prec::F32) {
    if (a.search) return launch_occ_density_k<P, true>(a, box, jitter, cells, count, sigma, stats, work, num_sms, s);
  }
  return launch_occ_density_k<P, false>(a, box, jitter, cells, count, sigma, stats, work, num_sms, s);
}

cudaError_t launch_occ_density(const PosedArgs& a, const BoxDev& box, const float* jitter, const int* cells,
                               const unsigned* count, float* sigma, unsigned long long* stats, unsigned* work,
                               int num_sms, cudaStream_t s) {
  switch (a.prec) {
    case 1: return launch_occ_density_p<Prec::F16>(a, box, jitter, cells, count, sigma, stats, work, num_sms, s);
    case 2: return launch_occ_density_p<Prec::BF16>(a, box, jitter, cells, count, sigma, stats, work, num_sms, s);
    default: return launch_occ_density_p<Prec::F32>(a, box, jitter, cells, count, sigma, stats, work, num_sms, s);
  }
}

// ---------------------------------------------------------------------------
// Occupancy cells whose query point can have a root (exact culling)
//
// A valid root lies in the canonical box, which the cells of the skinning grid
// tile.  Inside one cell with corners v_c and trilinear weights w_c(x), which
// reproduce affine functions (sum_c w_c = 1, sum_c w_c v_c = x), the LBS map
// f(x) = M(x) [x; 1] with M_c = [A_c | t_c] splits, for any constant A0, as
//   f(x) = sum_c w_c (A_c v_c + t_c) + sum_c w_c (A_c - A0)(x - v_c).
// The first sum lies in the bounding box of the corner images; component k of
// the second is at most max_c sum_j |A_c - A0|_kj h_j (h_j the cell's edges;
// A0 = the corners' mean, so this is the variation of the blended rotation
// over one cell, mostly far below a cell).  A query point with a root is within
// the Broyden tolerance of f(cell) for some cell, so a point outside all these
// boxes, grown by `slack` (the tolerance plus a margin far above fp32
// rounding), has no root and density 0: the search would end with none.  The
// boxes are recorded at the resolution of kSub^3 sub-cells per occupancy cell
// (a 64-bit mask per cell), which the occupancy queries and the render's
// samples test.
// ---------------------------------------------------------------------------

// One thread per skinning-grid cell, a block per 8 x 8 x 4 of them: marks the
// occupancy sub-cells meeting the cell's image box (sub_marked's index of a
// point is monotone in x, so the range of the box's two corners holds the index
// of every point inside).  The block first ORs its masks into a shared window
// over the occupancy cells its boxes meet and then adds each touched word to
// the grid with one global OR; a block whose window would not fit writes
// straight to the grid.
// With cen (one pose only) it also marks, one bit per occupancy cell, the cells
// whose centre (cell_center's fp32 value) lies inside a grown box: the point
// test that the centre queries of the per-pose occupancy refresh use, finer
// than the sub-cell masks (a rootless centre in a marked sub-cell is dropped
// when no box holds the point itself).  The box's sub-cell range holds every
// such cell (the index arithmetic is monotone), so the loop below visits them.
constexpr int kCoverWin = 4096;  // 64-bit words of the shared window (32 KB)

// blockIdx.y: the pose (blended grid S.M + pose * V * 3, masks sub + pose * R^3).
__global__ void __launch_bounds__(256) occ_cover_kernel(SkinDev S, int V, const BoxDev box, float slack,
                                                        unsigned long long* __restrict__ sub,
                                                        unsigned* __restrict__ cen, float4* __restrict__ cell_box) {
  static_assert(kSub * kSub * kSub == 64, "one 64-bit word per occupancy cell");
  __shared__ unsigned long long win[kCoverWin];
  __shared__ unsigned char wcen[kCoverWin];  // centre flags of the window's cells
  __shared__ int wlo[3], whi[3];
  S.M += (size_t)blockIdx.y * V * 3;
  sub += (size_t)blockIdx.y * box.R * box.R * box.R;
  if (cell_box) cell_box += (size_t)blockIdx.y * 2 * (S.Rw - 1) * (S.Rw - 1) * (S.Rw - 1);
  const int nc = S.Rw - 1;  // cells per axis
  const int bx = (nc + 7) / 8, by = (nc + 7) / 8;
  const int tid = threadIdx.x;
  const int cx = (blockIdx.x % bx) * 8 + (tid & 7), cy = ((blockIdx.x / bx) % by) * 8 + ((tid >> 3) & 7),
            cz = (blockIdx.x / (bx * by)) * 4 + (tid >> 6);
  if (tid < 3) {
    wlo[tid] = 0x7fffffff;
    whi[tid] = -1;
  }
  __syncthreads();
  const int ns = kSub * box.R;  // sub-cells per axis
  int s0[3] = {0, 0, 0}, s1[3] = {-1, -1, -1};
  float blo[3] = {0.f, 0.f, 0.f}, bhi[3] = {-1.f, -1.f, -1.f};  // the grown box
  bool live = cx < nc && cy < nc && cz < nc;
  if (live) {
    float h[3], v0[3];
    const int ci[3] = {cx, cy, cz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      h[a] = (S.cmax[a] - S.cmin[a]) / (float)nc;
      v0[a] = S.cmin[a] + (float)ci[a] * h[a];
    }
    float A[8][9];
    float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
    float mean[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) mean[q] = 0.f;
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
      const int ox = corner & 1, oy = (corner >> 1) & 1, oz = (corner >> 2) & 1;
      const int v = (cz + oz) * S.Rw * S.Rw + (cy + oy) * S.Rw + (cx + ox);
      const float4* p = S.M + 3 * (size_t)v;
      const float4 r[3] = {__ldg(p), __ldg(p + 1), __ldg(p + 2)};
      const float x = ox ? v0[0] + h[0] : v0[0], y = oy ? v0[1] + h[1] : v0[1], z = oz ? v0[2] + h[2] : v0[2];
      const float img[3] = {fmaf(r[0].x, x, fmaf(r[0].y, y, fmaf(r[0].z, z, r[0].w))),
                            fmaf(r[1].x, x, fmaf(r[1].y, y, fmaf(r[1].z, z, r[1].w))),
                            fmaf(r[2].x, x, fmaf(r[2].y, y, fmaf(r[2].z, z, r[2].w)))};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        lo[a] = fminf(lo[a], img[a]);
        hi[a] = fmaxf(hi[a], img[a]);
        A[corner][3 * a + 0] = a == 0 ? r[0].x : a == 1 ? r[1].x : r[2].x;
        A[corner][3 * a + 1] = a == 0 ? r[0].y : a == 1 ? r[1].y : r[2].y;
        A[corner][3 * a + 2] = a == 0 ? r[0].z : a == 1 ? r[1].z : r[2].z;
      }
#pragma unroll
      for (int q = 0; q < 9; ++q) mean[q] += 0.125f * A[corner][q];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float m = 0.f;
#pragma unroll
      for (int corner = 0; corner < 8; ++corner)
        m = fmaxf(m, fabsf(A[corner][3 * a] - mean[3 * a]) * h[0] +
                         fabsf(A[corner][3 * a + 1] - mean[3 * a + 1]) * h[1] +
                         fabsf(A[corner][3 * a + 2] - mean[3 * a + 2]) * h[2]);
      // sub_marked's index arithmetic (fp32), clamped before the conversion
      const float g = m + slack;
      blo[a] = lo[a] - g;
      bhi[a] = hi[a] + g;
      const float f0 = floorf(__fmul_rn(__fsub_rn(blo[a], box.nmin[a]), box.sub_scale[a]));
      const float f1 = floorf(__fmul_rn(__fsub_rn(bhi[a], box.nmin[a]), box.sub_scale[a]));
      if (!(f1 >= 0.f) || !(f0 <= (float)(ns - 1))) live = false;  // the box misses the grid
      s0[a] = (int)fminf(fmaxf(f0, 0.f), (float)(ns - 1));
      s1[a] = (int)fmaxf(fminf(f1, (float)(ns - 1)), 0.f);
    }
  }
  if (cell_box && cx < nc && cy < nc && cz < nc) {  // the grown box, or an empty one
    const size_t ci = (size_t)cx + (size_t)nc * (cy + (size_t)nc * cz);
    cell_box[2 * ci] = live ? make_float4(blo[0], blo[1], blo[2], 0.f) : make_float4(1.f, 1.f, 1.f, 0.f);
    cell_box[2 * ci + 1] = live ? make_float4(bhi[0], bhi[1], bhi[2], 0.f) : make_float4(-1.f, -1.f, -1.f, 0.f);
  }
  if (live) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      atomicMin(&wlo[a], s0[a] / kSub);
      atomicMax(&whi[a], s1[a] / kSub);
    }
  }
  __syncthreads();
  const int ex = whi[0] - wlo[0] + 1, ey = whi[1] - wlo[1] + 1, ez = whi[2] - wlo[2] + 1;
  const bool any = whi[0] >= 0;
  const bool shared = any && ex * ey * ez <= kCoverWin;
  if (shared)
    for (int t = tid; t < ex * ey * ez; t += blockDim.x) {
      win[t] = 0ull;
      wcen[t] = 0;
    }
  __syncthreads();
  // cell_center's fp32 coordinate of cell index i on axis a, and the box test
  auto centre_in = [&](int a, int i) {
    const float xc = __fadd_rn(box.nmin[a], __fmul_rn(__fadd_rn((float)i, 0.5f), box.cell_size[a]));
    return xc >= blo[a] && xc <= bhi[a];
  };
  if (live) {
    for (int z = s0[2] / kSub; z <= s1[2] / kSub; ++z) {
      const int z0 = max(s0[2] - kSub * z, 0), z1 = min(s1[2] - kSub * z, kSub - 1);
      const bool in_z = cen && centre_in(2, z);
      // one bit (kSub sy + kSub^2 sz) per z-layer of the box: 0x0001000100010001 masked
      const unsigned long long zs = (z1 == kSub - 1 ? ~0ull : (1ull << (16 * (z1 + 1))) - 1ull) &
                                    ~((1ull << (16 * z0)) - 1ull) & 0x0001000100010001ull;
      for (int y = s0[1] / kSub; y <= s1[1] / kSub; ++y) {
        const int y0 = max(s0[1] - kSub * y, 0), y1 = min(s1[1] - kSub * y, kSub - 1);
        // one bit per row of the box within a layer (nibble sy), then per layer:
        // the products place disjoint copies of the x-row, so they add without carries
        const unsigned long long ys = ((1ull << (4 * (y1 + 1))) - 1ull) & ~((1ull << (4 * y0)) - 1ull) & 0x1111ull;
        const unsigned long long yz = ys * zs;
        const bool in_yz = in_z && centre_in(1, y);
        for (int x = s0[0] / kSub; x <= s1[0] / kSub; ++x) {
          const int x0 = max(s0[0] - kSub * x, 0), x1 = min(s1[0] - kSub * x, kSub - 1);
          const unsigned long long row = ((1ull << (x1 + 1)) - 1ull) & ~((1ull << x0) - 1ull);
          const unsigned long long m = row * yz;  // bits x + kSub (sy + kSub sz) of the box
          const bool in_c = in_yz && centre_in(0, x);
          if (shared) {
            const int w = (x - wlo[0]) + ex * ((y - wlo[1]) + ey * (z - wlo[2]));
            atomicOr(win + w, m);
            if (in_c) wcen[w] = 1;  // every writer stores the same value
          } else {
            const int cell = x + box.R * (y + box.R * z);
            atomicOr(sub + cell, m);
            if (in_c) atomicOr(cen + (cell >> 5), 1u << (cell & 31));
          }
        }
      }
    }
  }
  __syncthreads();
  if (shared)
    for (int t = tid; t < ex * ey * ez; t += blockDim.x) {
      const unsigned long long m = win[t];
      if (m) {
        const int x = wlo[0] + t % ex, y = wlo[1] + (t / ex) % ey, z = wlo[2] + t / (ex * ey);
        const int cell = x + box.R * (y + box.R * z);
        atomicOr(sub + cell, m);
        if (wcen[t]) atomicOr(cen + (cell >> 5), 1u << (cell & 31));
      }
    }
}

// One thread per occupancy cell: its query point (the density kernel's), that
// point's sub-cell mark and, for centre queries (cen), its centre flag.  Points
// that can have a root go to `cells` (one atomic per warp; order across warps
// is free, since each cell's search is independent of the others); the others
// get density 0.
__global__ void occ_cand_kernel(const BoxDev box, const float* __restrict__ jitter,
                                const unsigned long long* __restrict__ sub, const unsigned* __restrict__ cen,
                                int* __restrict__ cells, unsigned* __restrict__ count, float* __restrict__ sigma,
                                unsigned long long* __restrict__ stats) {
  const int n = box.R * box.R * box.R;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  bool cand = false;
  if (c < n) {
    const float3 x = jitter ? cell_point(box, c, jitter + 3 * (size_t)c) : cell_center(box, c);
    cand = sub_marked(sub, box, x) && (!cen || ((__ldg(cen + (c >> 5)) >> (c & 31)) & 1u));
    if (!cand) sigma[c] = 0.f;
  }
  const unsigned m = __ballot_sync(kFull, cand);
  const int lane = threadIdx.x & 31;
  unsigned base = 0;
  if (lane == 0 && m) base = atomicAdd(count, (unsigned)__popc(m));
  base = __shfl_sync(kFull, base, 0);
  if (cand) cells[base + __popc(m & ((1u << lane) - 1u))] = c;
  if (stats) flush_stats_block<1>(stats, {ST_CULLED}, {(long long)(c < n && !cand ? 1 : 0)});
}

// The root-culling masks of n_poses consecutive blended grids (S.M = the
// first, V vertices each) into sub [n_poses][R^3] (cleared here); with cen
// (n_poses == 1) also the centre flags [ceil(R^3 / 32)] (cleared here).
cudaError_t launch_occ_cover(const SkinDev& S, int V, int n_poses, const SolveCfg& cfg, const BoxDev& box,
                             unsigned long long* sub, unsigned* cen, cudaStream_t s, float4* cell_box) {
  const size_t n = (size_t)box.R * box.R * box.R;
  if (cen && n_poses != 1) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(sub, 0, n * n_poses * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (cen && (e = cudaMemsetAsync(cen, 0, (n + 31) / 32 * sizeof(unsigned), s)) != cudaSuccess) return e;
  // slack: the Broyden tolerance plus 1e-4 of the scene's largest coordinate
  // (fp32 rounding of the LBS map and of these bounds is below 1e-6 of it)
  float L = 0.f;
  for (int k = 0; k < 3; ++k)
    L = std::max({L, std::fabs(S.cmin[k]), std::fabs(S.cmax[k]), std::fabs(box.nmin[k]), std::fabs(box.nmax[k])});
  const float slack = std::sqrt(cfg.tol2) + 1e-4f * L;
  const int nc = S.Rw - 1;
  const int blocks = ((nc + 7) / 8) * ((nc + 7) / 8) * ((nc + 3) / 4);
  {
    KernelSpan span("occ_cover_kernel", s);
    occ_cover_kernel<<<dim3(blocks, n_poses), 256, 0, s>>>(S, V, box, slack, sub, cen, cell_box);
  }
  return cudaGetLastError();
}

// sub: [R^3] masks, cen: [ceil(R^3 / 32)] centre flags (both rebuilt here; the
// flags only serve centre queries, jitter == null); count: the candidate count
// (cleared here)
cudaError_t launch_occ_cull(const PosedArgs& a, const BoxDev& box, const float* jitter, unsigned long long* sub,
                            unsigned* cen, unsigned* count, int* cells, float* sigma, unsigned long long* stats,
                            cudaStream_t s, float4* cell_box) {
  const int n = box.R * box.R * box.R;
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  unsigned* c = jitter ? nullptr : cen;
  if ((e = launch_occ_cover(a.S, a.S.Rw * a.S.Rw * a.S.Rw, 1, a.cfg, box, sub, c, s, cell_box)) != cudaSuccess)
    return e;
  {
    KernelSpan span("occ_cand_kernel", s);
    occ_cand_kernel<<<(n + 255) / 256, 256, 0, s>>>(box, jitter, sub, c, cells, count, sigma, stats);
  }
  return cudaGetLastError();
}

// Per occupied cell of the render's grid (occ), or per cell of the grid
// (occ null: the training step's lists, independent of its changing grid), the
// skinning cells whose grown image box (cell_box, from occ_cover_kernel)
// meets it: one thread per skinning cell, its box's range of occupancy cells
// by cell_of's index arithmetic (monotone in the coordinates, so the range
// holds the cell of every point inside the box), one slot per listed cell of
// the range.  A cell with more than `cap` boxes keeps a count above cap: its
// points are not tested.  blockIdx.y: the pose (boxes [pose][n_cells][2],
// counts [pose][R^3], lists [pose][R^3][cap]).
__global__ void occ_boxlist_kernel(const float4* __restrict__ cell_box, int n_cells, const BoxDev box,
                                   const uint32_t* __restrict__ occ, int* __restrict__ count, int* __restrict__ list,
                                   int cap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cells) return;
  const size_t cells = (size_t)box.R * box.R * box.R;
  cell_box += (size_t)blockIdx.y * 2 * n_cells;
  count += blockIdx.y * cells;
  list += blockIdx.y * cells * cap;
  const float4 lo = cell_box[2 * (size_t)i], hi = cell_box[2 * (size_t)i + 1];
  if (!(lo.x <= hi.x)) return;  // no box
  const int c0 = cell_of(box, make_float3(lo.x, lo.y, lo.z)), c1 = cell_of(box, make_float3(hi.x, hi.y, hi.z));
  const int R = box.R;
  const int x0 = c0 % R, y0 = (c0 / R) % R, z0 = c0 / (R * R);
  const int x1 = c1 % R, y1 = (c1 / R) % R, z1 = c1 / (R * R);
  // a row of the range is a run of consecutive bits: its words are read once
  // and only the occupied cells visited
  for (int z = z0; z <= z1; ++z)
    for (int y = y0; y <= y1; ++y) {
      const int r0 = x0 + R * (y + R * z), r1 = x1 + R * (y + R * z);
      for (int wd = r0 >> 5; wd <= (r1 >> 5); ++wd) {
        uint32_t bits = occ ? __ldg(occ + wd) : ~0u;
        const int lo_bit = max(r0 - 32 * wd, 0), hi_bit = min(r1 - 32 * wd, 31);
        bits &= (hi_bit == 31 ? ~0u : (1u << (hi_bit + 1)) - 1u) & ~((1u << lo_bit) - 1u);
        while (bits) {
          const int c = 32 * wd + __ffs(bits) - 1;
          bits &= bits - 1u;
          const int slot = atomicAdd(count + c, 1);
          if (slot < cap) list[(size_t)c * cap + slot] = i;
        }
      }
    }
}

cudaError_t launch_occ_boxlist(const float4* cell_box, int n_cells, int n_poses, const BoxDev& box,
                               const uint32_t* occ, int* count, int* list, int cap, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)n_poses * box.R * box.R * box.R, s);
  if (e != cudaSuccess) return e;
  {
    KernelSpan span("occ_boxlist_kernel", s);
    occ_boxlist_kernel<<<dim3((n_cells + 255) / 256, n_poses), 256, 0, s>>>(cell_box, n_cells, box, occ, count, list,
                                                                         cap);
  }
  return cudaGetLastError();
}

// training-mode occupancy (Sec. 3.3): the sequence's running density
// d <- max(decay d, sigma) of one frame's query
__global__ void occ_ema_kernel(const float* __restrict__ sigma, float* __restrict__ d, int n, float decay) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = fmaxf(__fmul_rn(decay, d[i]), sigma[i]);
}

cudaError_t launch_occ_ema(const float* sigma, float* d, int n, float decay, cudaStream_t s) {
  {
    KernelSpan span("occ_ema_kernel", s);
    occ_ema_kernel<<<(n + 255) / 256, 256, 0, s>>>(sigma, d, n, decay);
  }
  return cudaGetLastError();
}

// occupied = sigma > tau, dilated by a (2 dilate + 1)^3 cube clipped to the grid;
// cell b = x + R (y + R z) is bit b % 32 of word b / 32.  One thread per cell, a
// warp per word (blocks of whole warps, so warp w holds cells 32 w .. 32 w + 31).
__global__ void occ_bits_kernel(const float* __restrict__ sigma, int R, int dilate, float tau,
                                uint32_t* __restrict__ bits, uint32_t* __restrict__ union_bits) {
  const int n = R * R * R;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  bool on = false;
  if (cell < n) {
    const int x = cell % R, y = (cell / R) % R, z = cell / (R * R);
    for (int dz = -dilate; dz <= dilate && !on; ++dz) {
      const int zz = z + dz;
      if (zz < 0 || zz >= R) continue;
      for (int dy = -dilate; dy <= dilate && !on; ++dy) {
        const int yy = y + dy;
        if (yy < 0 || yy >= R) continue;
        for (int dx = -dilate; dx <= dilate && !on; ++dx) {
          const int xx = x + dx;
          if (xx < 0 || xx >= R) continue;
          if (__ldg(sigma + xx + R * (yy + R * zz)) > tau) on = true;
        }
      }
    }
  }
  const unsigned word = __ballot_sync(kFull, on);
  if ((threadIdx.x & 31) == 0 && cell < n) {
    if (bits) bits[cell >> 5] = word;
    if (union_bits) union_bits[cell >> 5] |= word;
  }
}

cudaError_t launch_occ_bits(const float* sigma, int R, int dilate, float tau, uint32_t* bits, uint32_t* union_bits,
                            cudaStream_t s) {
  const int n = R * R * R;
  {
    KernelSpan span("occ_bits_kernel", s);
    occ_bits_kernel<<<(n + 255) / 256, 256, 0, s>>>(sigma, R, dilate, tau, bits, union_bits);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Queries
// ---------------------------------------------------------------------------

template <Prec P>
__global__ void __launch_bounds__(256, IA_POSED_MIN_BLOCKS)
    query_posed_kernel(const PosedArgs a, int n, const float* __restrict__ x, float* sigma, float* rgb, float* xc,
                       int* start) {
  extern __shared__ float4 smem4[];
  PosedSmem sm = stage_posed<P>(stage_of(a), smem4);
  SampleStats st;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kList; base < n;
       base += warps * kList) {
    posed_field_list<P, ItemOrder::kSampleMajor>(
        a.S, a.F, a.cfg, sm.fs, sm.list, min(kList, n - base),
        [&](int i, float3& xn, const float4*& M, const float*& Ni, int& pose) {
          const int j = base + i;
          xn = make_float3(x[3 * j], x[3 * j + 1], x[3 * j + 2]);
          M = a.S.M;
          Ni = sm.sNinv;
          pose = 0;
        },
        [&](int i, const PosedOut& o) {
          const int j = base + i;
          if (sigma) sigma[j] = o.start >= 0 ? o.sigma : 0.f;
          if (rgb) { rgb[3 * j] = o.rgb.x; rgb[3 * j + 1] = o.rgb.y; rgb[3 * j + 2] = o.rgb.z; }
          if (xc) { xc[3 * j] = o.xstar.x; xc[3 * j + 1] = o.xstar.y; xc[3 * j + 2] = o.xstar.z; }
          if (start) start[j] = o.start;
        },
        st, a.prop, a.search != 0);
  }
}

template <Prec P>
static cudaError_t launch_query_posed_p(const PosedArgs& a, int n, const float* x, float* sigma, float* rgb,
                                        float* xc, int* start, cudaStream_t s) {
  const size_t smem = posed_smem_bytes_p<P>(256, a.search != 0);
  cudaError_t e = set_smem(query_posed_kernel<P>, smem, 256);
  if (e != cudaSuccess) return e;
  {
    KernelSpan span("query_posed_kernel", s);
    query_posed_kernel<P><<<(n + 8 * kList - 1) / (8 * kList), 256, smem, s>>>(a, n, x, sigma, rgb, xc, start);
  }
  return cudaGetLastError();
}

cudaError_t launch_query_posed(const PosedArgs& a, int n, const float* x, float* sigma, float* rgb, float* xc,
                               int* start, cudaStream_t s) {
  switch (a.prec) {
    case 1: return launch_query_posed_p<Prec::F16>(a, n, x, sigma, rgb, xc, start, s);
    case 2: return launch_query_posed_p<Prec::BF16>(a, n, x, sigma, rgb, xc, start, s);
    default: return launch_query_posed_p<Prec::F32>(a, n, x, sigma, rgb, xc, start, s);
  }
}

// canonical field at caller points; whole warps iterate so the tensor-core
// path has all 32 lanes
template <Prec P>
__global__ void __launch_bounds__(256) query_canonical_kernel(const PosedArgs a, int n, const float* __restrict__ x,
                                                              float* sigma, float* rgb) {
  extern __shared__ float4 smem4[];
  PosedSmem sm = stage_posed<P>(stage_of(a), smem4);
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    const bool act = i < n;
    const float3 p = act ? make_float3(x[3 * i], x[3 * i + 1], x[3 * i + 2])
                         : make_float3(a.F.cmin[0], a.F.cmin[1], a.F.cmin[2]);
    float s;
    float3 c;
    field_eval_warp<P>(a.F, sm.fs, p, s, c);
    if (act) {
      sigma[i] = s;
      rgb[3 * i] = c.x;
      rgb[3 * i + 1] = c.y;
      rgb[3 * i + 2] = c.z;
    }
  }
}

template <Prec P>
static cudaError_t launch_query_canonical_p(const PosedArgs& a, int n, const float* x, float* sigma, float* rgb,
                                            cudaStream_t s) {
  const size_t smem = posed_smem_bytes_p<P>(256, a.search != 0);
  cudaError_t e = set_smem(query_canonical_kernel<P>, smem, 256);
  if (e != cudaSuccess) return e;
  {
    KernelSpan span("query_canonical_kernel", s);
    query_canonical_kernel<P><<<(n + 255) / 256, 256, smem, s>>>(a, n, x, sigma, rgb);
  }
  return cudaGetLastError();
}

cudaError_t launch_query_canonical(const PosedArgs& a, int n, const float* x, float* sigma, float* rgb,
                                   cudaStream_t s) {
  switch (a.prec) {
    case 1: return launch_query_canonical_p<Prec::F16>(a, n, x, sigma, rgb, s);
    case 2: return launch_query_canonical_p<Prec::BF16>(a, n, x, sigma, rgb, s);
    default: return launch_query_canonical_p<Prec::F32>(a, n, x, sigma, rgb, s);
  }
}

// ---------------------------------------------------------------------------
// Persistent fused render kernel
//
// Every warp runs on its own: it keeps a pool of 32 rays, one per lane, and
// loops over rounds with warp-level synchronisation only.  A round:
//  1. march: every ray advances its slot cursor until it has found up to K
//     slots in occupied cells (empty-space skipping) whose point can have a
//     root (the pose's root-culling masks, when present: the others have
//     density 0); exhausted rays write their pixel and take the next ray from
//     a global counter (one atomic per warp);
//  2. a warp scan packs the found (ray, slot) samples into shared memory;
//  3. the warp evaluates them 32 at a time: bone-wise Broyden search, polish,
//     hash encoding, MLP, max-density root;
//  4. every ray composites its own samples front to back and stops once its
//     transmittance is below the threshold.
// ---------------------------------------------------------------------------

template <Prec P>
size_t render_smem_bytes_p(int K, bool prop) {
  return posed_smem_bytes_p<P>(kRenderThreads, prop) + sizeof(float4) * (2 * kRenderThreads + K * kRenderThreads) +
         (sizeof(uint8_t) + sizeof(uint16_t)) * K * kRenderThreads;
}


constexpr int kMarchAhead = 4;  // slots whose occupancy words one march step fetches together

template <int K, Prec P, bool kProp>
__global__ void __launch_bounds__(kRenderThreads, IA_RENDER_MIN_BLOCKS) render_kernel(const RenderArgs a) {
  extern __shared__ float4 smem4[];
  PosedSmem sm = stage_posed<P>(stage_of(a.P), smem4);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // this warp's slices of the shared arrays
  float4* const after_roots = reinterpret_cast<float4*>(sm.sNinv + kMaxBones * 12) +
                              (kRenderThreads / 32) * list_smem_words(kProp) / 4;
  float4* ray_o = after_roots + warp * 32;                             // (o.xyz, delta)
  float4* ray_d = ray_o + kRenderThreads;                              // (d.xyz, t_near)
  float4* s_res = after_roots + 2 * kRenderThreads + warp * 32 * K;    // (sigma, r, g, b)
  uint8_t* const idx_area = reinterpret_cast<uint8_t*>(after_roots + (2 + K) * kRenderThreads);
  uint16_t* s_slot = reinterpret_cast<uint16_t*>(idx_area) + warp * 32 * K;              // [K * threads]
  uint8_t* s_ray = idx_area + sizeof(uint16_t) * K * kRenderThreads + warp * 32 * K;     // [K * threads]
  __shared__ float sB0inv[12];
  if (tid < 12) sB0inv[tid] = a.B0inv[tid];
  __syncthreads();

  const int W = a.cam.width, H = a.cam.height;
  const float log_stop = a.early_T > 0.f ? -logf(a.early_T) : __int_as_float(0x7f800000);

  // per-ray state of this lane's pool slot
  bool has_ray = false, queue_empty = false;
  int pix = 0, cursor = 0;
  float depth = 0.f;  // optical depth sum sigma_i delta
  float cr = 0.f, cg = 0.f, cb = 0.f;
  unsigned n_rays = 0, n_hit = 0, n_marched = 0, n_occ = 0, n_early = 0, n_culled = 0;
  SampleStats st;

  while (true) {
    // ---- 1. march
    int nfound = 0;
    int slots[K];
    while (true) {
      if (has_ray) {
        const float4 ro = ray_o[lane], rd = ray_d[lane];
        const float o[3] = {ro.x, ro.y, ro.z}, d[3] = {rd.x, rd.y, rd.z};
        // kMarchAhead slots at a time: their cells and occupancy words are
        // fetched together (independent loads in flight), then tested in slot
        // order, stopping at the K-th occupied one as a one-slot loop would
        while (cursor < a.n_slots && nfound < K) {
          int cl[kMarchAhead];
          uint32_t wd[kMarchAhead];
#pragma unroll
          for (int q = 0; q < kMarchAhead; ++q) {
            const int sl = min(cursor + q, a.n_slots - 1);
            cl[q] = cell_of(a.box, slot_position(o, d, rd.w, ro.w, sl));
            wd[q] = __ldg(a.occ + (cl[q] >> 5));
          }
#pragma unroll
          for (int q = 0; q < kMarchAhead; ++q) {
            if (cursor >= a.n_slots || nfound >= K) break;
            ++n_marched;
            if ((wd[q] >> (cl[q] & 31)) & 1u) {
              if (a.sub && !sub_marked(a.sub, a.box, slot_position(o, d, rd.w, ro.w, cursor))) {
                ++n_culled;  // no root possible: density 0, nothing to composite
              } else {
#pragma unroll
                for (int k = 0; k < K; ++k)
                  if (k == nfound) slots[k] = cursor;
                ++nfound;
              }
            }
            ++cursor;
          }
        }
        if (nfound == 0) {  // exhausted: write the pixel
          a.rgb[3 * pix] = cr;
          a.rgb[3 * pix + 1] = cg;
          a.rgb[3 * pix + 2] = cb;
          a.alpha[pix] = -expm1f(-depth);
          has_ray = false;
        }
      }
      const bool need = !has_ray && !queue_empty;
      const unsigned m = __ballot_sync(kFull, need);
      if (m == 0) break;
      unsigned base = 0;
      const int leader = __ffs(m) - 1;
      if (lane == leader) base = atomicAdd(a.counter, (unsigned)__popc(m));
      base = __shfl_sync(kFull, base, leader);
      if (need) {
        const int id = (int)(base + __popc(m & ((1u << lane) - 1u)));
        if (id >= a.n_ray_ids) {
          queue_empty = true;
        } else {
          int u, v;
          bool valid;
          tile_pixel(id, a.tiles_x, W, H, u, v, valid);
          if (valid) {
            ++n_rays;
            float o[3], d[3], tn, tf;
            pix = v * W + u;
            cr = cg = cb = 0.f;
            depth = 0.f;
            cursor = 0;
            if (make_ray(a.cam, sB0inv, a.box, u, v, o, d, tn, tf)) {
              ++n_hit;
              ray_o[lane] = make_float4(o[0], o[1], o[2], slot_delta(tn, tf, a.n_slots));
              ray_d[lane] = make_float4(d[0], d[1], d[2], tn);
              has_ray = true;
            } else {
              a.rgb[3 * pix] = 0.f;
              a.rgb[3 * pix + 1] = 0.f;
              a.rgb[3 * pix + 2] = 0.f;
              a.alpha[pix] = 0.f;
            }
          }
        }
      }
    }
    // ---- 2. pack samples (warp exclusive scan of nfound)
    int incl = nfound;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    const int offset = incl - nfound;
    if (total == 0) break;  // no ray of this warp has work and the queue is drained
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j < nfound) {
        s_ray[offset + j] = (uint8_t)lane;
        s_slot[offset + j] = (uint16_t)slots[j];  // n_slots <= 1024
      }
    n_occ += nfound;
    __syncwarp();
    // ---- 3. correspondence search and field at the round's samples (lists of kList)
    for (int base = 0; base < total; base += kList) {
      // each lane runs its own sample's starts in order (the proposed ones, or
      // all bones); the proposal's fallback starts, many for a few samples,
      // go through the warp's shared queue
      posed_field_list<P, ItemOrder::kPerLane, kProp, ItemOrder::kStartMajor>(
          a.P.S, a.P.F, a.P.cfg, sm.fs, sm.list, min(kList, total - base),
          [&](int i, float3& xn, const float4*& M, const float*& Ni, int& pose) {
            const int sidx = base + i;
            const int owner = s_ray[sidx];
            const float4 ro = ray_o[owner], rd = ray_d[owner];
            const float o[3] = {ro.x, ro.y, ro.z}, d[3] = {rd.x, rd.y, rd.z};
            xn = slot_position(o, d, rd.w, ro.w, s_slot[sidx]);
            M = a.P.S.M;
            Ni = sm.sNinv;
            pose = 0;
          },
          [&](int i, const PosedOut& o) {
            s_res[base + i] = make_float4(o.start >= 0 ? o.sigma : 0.f, o.rgb.x, o.rgb.y, o.rgb.z);
          },
          st, a.P.prop, kProp);  // the proposal code is compiled only into kProp variants
    }
    __syncwarp();
    // ---- 4. composite this ray's samples, alpha_i = 1 - exp(-sigma_i delta)
    if (nfound > 0) {
      const float dt = ray_o[lane].w;
      for (int j = 0; j < nfound; ++j) {
        const float4 sres = s_res[offset + j];
        if (sres.x > 0.f) {
          const float sd = sres.x * dt;
          const float w = expf(-depth) * -expm1f(-sd);  // T_i alpha_i
          cr = fmaf(w, sres.y, cr);
          cg = fmaf(w, sres.z, cg);
          cb = fmaf(w, sres.w, cb);
          depth += sd;
        }
        if (depth > log_stop) {  // transmittance below the threshold: stop the ray
          ++n_early;
          cursor = a.n_slots;
          break;
        }
      }
    }
    __syncwarp();
  }
  if (a.stats) {
    flush_stats(a.stats, ST_RAYS, n_rays);
    flush_stats(a.stats, ST_HIT, n_hit);
    flush_stats(a.stats, ST_MARCHED, n_marched);
    flush_stats(a.stats, ST_OCC, n_occ + n_culled);
    flush_stats(a.stats, ST_CULLED, n_culled);
    flush_stats(a.stats, ST_STARTS, st.starts);
    flush_stats(a.stats, ST_ITERS, st.iters);
    flush_stats(a.stats, ST_GATHERS, st.starts + st.iters);
    flush_stats(a.stats, ST_CONV, st.converged);
    flush_stats(a.stats, ST_ROOTS, st.roots);
    flush_stats(a.stats, ST_EARLY, n_early);
    flush_stats(a.stats, ST_PROP, st.proposed);
    flush_stats(a.stats, ST_FALLBACK, st.fallbacks);
  }
}

template <Prec P, bool kProp>
constexpr const char* render_name() {
  return kProp ? variant_name<P>("render_kernel<fp32,proposal>", "render_kernel<fp16,proposal>", "render_kernel<bf16,proposal>")
               : variant_name<P>("render_kernel<fp32>", "render_kernel<fp16>", "render_kernel<bf16>");
}

template <int K, Prec P, bool kProp>
static cudaError_t launch_render_k(const RenderArgs& a, int num_sms, cudaStream_t s) {
  const size_t smem = render_smem_bytes_p<P>(K, kProp);
  cudaError_t e = set_smem(render_kernel<K, P, kProp>, smem, kRenderThreads);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_kernel<K, P, kProp>, kRenderThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int want = (a.n_ray_ids + kRenderThreads - 1) / kRenderThreads;
  int grid = num_sms * per_sm;
  if (grid > want) grid = want;
  if (grid < 1) grid = 1;
  {
    KernelSpan span(render_name<P, kProp>(), s);
    render_kernel<K, P, kProp><<<grid, kRenderThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <Prec P, bool kProp>
static cudaError_t launch_render_pp(const RenderArgs& a, int num_sms, cudaStream_t s) {
  // with early termination, few samples per ray per round bound the work done
  // past the stopping sample; without it, larger rounds amortise the scans.
  // Measured (540^2 frames, early termination on): the plain fp32 render is
  // fastest with one sample per ray per round, i.e. lists of neighbouring rays
  // at like depths (8.4 ms against 8.7 ms with two; four and eight: 9.6 and
  // 10.9 ms), the fp16 + proposal render with two (2.73 ms against 2.87 ms)
  if (a.early_T > 0.f) return launch_render_k<P == Prec::F32 ? 1 : 2, P, kProp>(a, num_sms, s);
  return launch_render_k<8, P, kProp>(a, num_sms, s);
}

template <Prec P>
static cudaError_t launch_render_p(const RenderArgs& a, int num_sms, cudaStream_t s) {
  if constexpr (P == Prec::F32) {
    return launch_render_pp<P, false>(a, num_sms, s);  // the proposal search needs fp16 / bf16
  } else {
    if (a.P.search) return launch_render_pp<P, true>(a, num_sms, s);
    return launch_render_pp<P, false>(a, num_sms, s);
  }
}

cudaError_t launch_render(const RenderArgs& a, int num_sms, cudaStream_t s) {
  switch (a.P.prec) {
    case 1: return launch_render_p<Prec::F16>(a, num_sms, s);
    case 2: return launch_render_p<Prec::BF16>(a, num_sms, s);
    default: return launch_render_p<Prec::F32>(a, num_sms, s);
  }
}

// fp16 shadow of the fp32 master hash table (reduced-precision field)
__global__ void table_to_half_kernel(const float2* __restrict__ t, __half2* __restrict__ th, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    th[i] = __float22half2_rn(t[i]);
}

cudaError_t launch_table_to_half(const float* table, __half2* th, int64_t entries, cudaStream_t s) {
  {
    KernelSpan span("table_to_half_kernel", s);
    table_to_half_kernel<<<1184, 256, 0, s>>>(reinterpret_cast<const float2*>(table), th, entries);
  }
  return cudaGetLastError();
}

// One thread per pixel: the slots the render kernel's march would keep.
__global__ void march_mask_kernel(const RenderArgs a, uint32_t* __restrict__ mask) {
  const int W = a.cam.width, H = a.cam.height;
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= W * H) return;
  const int words = (a.n_slots + 31) / 32;
  uint32_t* m = mask + (size_t)pix * words;
  for (int w = 0; w < words; ++w) m[w] = 0u;
  float o[3], d[3], tn, tf;
  if (!make_ray(a.cam, a.B0inv, a.box, pix % W, pix / W, o, d, tn, tf)) return;
  const float dt = slot_delta(tn, tf, a.n_slots);
  for (int i = 0; i < a.n_slots; ++i) {
    const int cell = cell_of(a.box, slot_position(o, d, tn, dt, i));
    if ((__ldg(a.occ + (cell >> 5)) >> (cell & 31)) & 1u) m[i >> 5] |= 1u << (i & 31);
  }
}

cudaError_t launch_march_mask(const RenderArgs& a, uint32_t* mask, cudaStream_t s) {
  const int n = a.cam.width * a.cam.height;
  {
    KernelSpan span("march_mask_kernel", s);
    march_mask_kernel<<<(n + 127) / 128, 128, 0, s>>>(a, mask);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gather and atomic probes (measurement helpers, not part of the method).
// Every thread reads, or adds to, records at xorshift-random indices of a
// table: 48-byte records (three float4, one vertex of the blended grid: one
// corner of the LBS gather), 16, 8 or 4 bytes (an fp32 / fp16 hash entry).
// Their rates on tables the size of the kernels' own are the peaks the
// search, field and scatter kernels are compared against.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned probe_next(unsigned h) {
  h ^= h << 13;  // xorshift32 (Marsaglia): the record index
  h ^= h >> 17;
  h ^= h << 5;
  return h;
}

template <int kBytes>
__global__ void gather_probe_kernel(const float* __restrict__ table, unsigned n_records, int iters,
                                    float* __restrict__ sink) {
  unsigned h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
  float acc = 0.f;
  for (int i = 0; i < iters; ++i) {
    h = probe_next(h);
    const size_t r = h % n_records;
    if constexpr (kBytes == 4) {
      acc += __ldg(table + r);
    } else if constexpr (kBytes == 8) {
      const float2 a = __ldg(reinterpret_cast<const float2*>(table) + r);
      acc += a.x + a.y;
    } else if constexpr (kBytes == 16) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(table) + r);
      acc += a.x + a.w;
    } else {
      const float4* p = reinterpret_cast<const float4*>(table) + 3 * r;
      const float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
      acc += a.x + b.y + c.z;
    }
  }
  if (acc == 1.2345f) sink[0] = acc;  // keeps the loads; practically never taken
}

template <int kBytes>
__global__ void atomic_probe_kernel(float* __restrict__ table, unsigned n_records, int iters) {
  unsigned h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
  for (int i = 0; i < iters; ++i) {
    h = probe_next(h);
    const size_t r = h % n_records;
    if constexpr (kBytes == 8) atomicAdd(reinterpret_cast<float2*>(table) + r, make_float2(1e-7f, 1e-7f));
    else atomicAdd(reinterpret_cast<float4*>(table) + r, make_float4(1e-7f, 1e-7f, 1e-7f, 1e-7f));
  }
}

cudaError_t launch_gather_probe(const float* table, int64_t n_records, int record_bytes, int iters, int blocks,
                                float* sink, cudaStream_t s) {
  KernelSpan span("gather_probe_kernel", s);
  const unsigned n = (unsigned)n_records;
  switch (record_bytes) {
    case 4: gather_probe_kernel<4><<<blocks, 256, 0, s>>>(table, n, iters, sink); break;
    case 8: gather_probe_kernel<8><<<blocks, 256, 0, s>>>(table, n, iters, sink); break;
    case 16: gather_probe_kernel<16><<<blocks, 256, 0, s>>>(table, n, iters, sink); break;
    default: gather_probe_kernel<48><<<blocks, 256, 0, s>>>(table, n, iters, sink); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_atomic_probe(float* table, int64_t n_records, int record_bytes, int iters, int blocks,
                                cudaStream_t s) {
  KernelSpan span("atomic_probe_kernel", s);
  if (record_bytes == 8) atomic_probe_kernel<8><<<blocks, 256, 0, s>>>(table, (unsigned)n_records, iters);
  else atomic_probe_kernel<16><<<blocks, 256, 0, s>>>(table, (unsigned)n_records, iters);
  return cudaGetLastError();
}

}  // namespace ia
