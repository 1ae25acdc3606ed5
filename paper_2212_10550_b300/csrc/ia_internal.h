// Internal launch interface between the C ABI (ia_api.cu) and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ia_device.cuh"
#include "ia_index.cuh"
#include "ia_posed.cuh"
#include "ia_profile.h"
#include "ia_wgrad.h"

namespace ia {

// warp-reduce a per-lane count, one atomic per warp; all 32 lanes call
__device__ __forceinline__ void flush_stats(unsigned long long* stats, int idx, long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0) atomicAdd(stats + idx, (unsigned long long)v);
}

// The same summed over the block first (one atomic per block and counter, for
// short kernels with many blocks, whose per-warp atomics on the same counters
// would serialise); all threads of the block call, with the same N and idx.
template <int N>
__device__ __forceinline__ void flush_stats_block(unsigned long long* stats, const int (&idx)[N],
                                                  const long long (&v)[N]) {
  __shared__ unsigned long long s_sum[N];
  if (threadIdx.x < N) s_sum[threadIdx.x] = 0;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) {
    long long x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
    if ((threadIdx.x & 31) == 0 && x != 0) atomicAdd(s_sum + k, (unsigned long long)x);
  }
  __syncthreads();
  if (threadIdx.x < N && s_sum[threadIdx.x] != 0) atomicAdd(stats + idx[threadIdx.x], s_sum[threadIdx.x]);
}

// the next list index of a warp from a counter shared by the grid (zeroed by
// the host before the launch); all 32 lanes call
__device__ __forceinline__ int next_list(unsigned* work) {
  int w = 0;
  if ((threadIdx.x & 31) == 0) w = (int)atomicAdd(work, 1u);
  return __shfl_sync(kFull, w, 0);
}

enum StatIdx {
  ST_RAYS = 0, ST_HIT, ST_MARCHED, ST_OCC, ST_STARTS, ST_ITERS, ST_CONV, ST_ROOTS, ST_EARLY, ST_PROP, ST_FALLBACK,
  ST_CULLED, ST_GATHERS, ST_ROOTED, ST_PCULLED,
  ST_COUNT = 16
};

#ifndef IA_RENDER_THREADS
#define IA_RENDER_THREADS 256
#endif
constexpr int kRenderThreads = IA_RENDER_THREADS;
constexpr int kTile = 16;  // rays are handed out in 16 x 16 pixel tiles

struct PosedArgs {
  SkinDev S;
  FieldDev F;
  SolveCfg cfg;
  const float* Ninv;   // [nb][12] of the pose
  const float* mlp;    // packed MLP (fp32 master)
  int n_in;
  int prec;            // ia_precision of the field evaluation
  const __half2* table_h;  // fp16 shadow of the hash table (prec != fp32)
  int search;          // 1: proposal network picks the first starts (prec != fp32)
  PropDev prop;
  const double* theta; // [nb][3] axis-angles of the pose (proposal input)
};

__device__ __forceinline__ PosedStage stage_of(const PosedArgs& a) {
  PosedStage s;
  s.mlp = a.mlp;
  s.n_in = a.n_in;
  s.table_h = a.table_h;
  s.search = a.search;
  s.prop = a.prop;
  s.theta = a.theta;
  s.Ninv = a.Ninv;
  s.nb = a.cfg.nb;
  return s;
}

// ray id -> pixel: rays are numbered tile by tile (kTile x kTile pixels, row by row inside a tile)
__device__ __forceinline__ void tile_pixel(int id, int tiles_x, int W, int H, int& u, int& v, bool& valid) {
  const int tile = id / (kTile * kTile), i = id % (kTile * kTile);
  u = (tile % tiles_x) * kTile + i % kTile;
  v = (tile / tiles_x) * kTile + i / kTile;
  valid = u < W && v < H;
}

// dynamic shared memory of a kernel that stages the posed field (stage_posed)
template <Prec P>
size_t posed_smem_bytes_p(int threads, bool prop) {
  return sizeof(float) * (mlp_smem_words(P, threads, prop) + kMaxBones * 12) +
         sizeof(uint32_t) * (threads / 32) * list_smem_words(prop);
}

struct RenderArgs {
  PosedArgs P;
  const float* B0inv;  // [12]
  const uint32_t* occ;
  const unsigned long long* sub;  // root-culling masks of this pose, or null
  BoxDev box;
  CamDev cam;
  int n_slots;
  float early_T;       // <= 0: no early termination
  int tiles_x;
  int n_ray_ids;       // tiles_x * tiles_y * kTile^2
  unsigned int* counter;
  float* rgb;
  float* alpha;
  unsigned long long* stats;
};

// The march writes the frame's samples; the search and field kernels then run
// over chunks [s0, s0 + ns) of them (arrays marked "chunk" are indexed from
// s0).  The training step's forward runs the same kernels over its emitted
// samples (one chunk, its count on the device, one pose per sample).
struct WfArgs {
  unsigned* n_samples;  // kept samples of the frame (counter, zeroed by the host)
  int cap;              // samples xn and res hold
  float4* xn;           // [cap] normalised-space positions and pose (int bits of w), each ray's
                        // samples contiguous in slot order
  float4* res;          // [cap] sigma (0 without a root), rgb
  float4* xs;           // [cap] or null: the selected root x* and 1 (0 without a root)
  int pose_stride;      // float4s per pose of the blended grids S.M (3 V)
  const float* ninv;    // [poses][n_bones][12] inverse rest-to-pose transforms (16-byte aligned)
  int n_ninv;           // floats of ninv the items may read (poses x n_bones x 12)
  int* ray_first;       // [W * H] first sample of the pixel's ray
  int* ray_cnt;         // [W * H] its kept samples
  float* ray_dt;        // [W * H] its slot spacing
  int s0, ns;           // the chunk (ns: its size, or an upper bound of *ns_dev)
  const unsigned* ns_dev;  // or null: the chunk's size on the device (then s0 = 0)
  float4* prop;         // chunk [ns] proposal: bones b0 | b1 << 8, start offset
  float4* item0;        // chunk [ns * starts] first wave: root (x, y, z) and order << 8 | bone, or -1
  float4* item1;        // [n_fb * n_bones] fallback wave, indexed by the sample's fallback position
  int* fb;              // [ns] the chunk's fallback samples (chunk indices)
  int* fbidx;           // chunk [ns] a sample's fallback position, or -1
  unsigned* n_fb;       // the chunk's fallback samples (counter, zeroed per chunk)
  int role;             // the caller, for the launch names: kWfRender, kWfOccupancy, kWfTrain
  // or null: per occupied cell of the render's grid, the skinning cells whose
  // grown image box meets it (blist_count [R^3], blist [R^3][blist_cap],
  // cell_box [(Rw - 1)^3][2]); a sample whose proposed starts found no root
  // and whose point lies in none of its cell's boxes has no root: no fallback
  const int* blist_count;
  const int* blist;
  int blist_cap;
  int blist_scan;       // the longest list the test scans (<= blist_cap); longer: no test
  const float4* cell_box;
  int blist_pose_cells;  // per-pose strides (a sample's pose: the int bits of xn.w): R^3
  int box_pose_cells;    //   and (Rw - 1)^3
};
constexpr int kWfRender = 0, kWfOccupancy = 1, kWfTrain = 2;

__device__ __forceinline__ int chunk_size(const WfArgs& w) { return w.ns_dev ? (int)*w.ns_dev : w.ns; }

// Training step (ia_train.cu).  Per-sample workspace: one column of kActStride
// floats holds the recomputed features, hidden activations and their gradients
// (F [32], H1 [64], H2 [64], dH1 [64], dH2 [64], dO [4]).
constexpr int kActStride = kIn + 4 * kWidth + 4;
constexpr int kMlpPadT = (kMlpSmemFloats + 3) / 4 * 4;

struct TrainArgs {
  PosedArgs P;           // P.S.M and P.Ninv point at pose 0 of the per-pose arrays
  WfArgs wf;             // the forward's search and field over the emitted samples
  int V;                 // skinning-grid vertices (one pose's blended grid = 3V float4)
  const float* B0inv;    // [n_poses][12]
  const float* N;        // [n_poses][nb][12]
  const float* skin;     // [V][nb]
  const uint32_t* occ;
  const unsigned long long* sub;  // root-culling masks [n_poses][R^3], or null
  BoxDev box;
  int n_slots;
  int n_rays;
  const float* origin;   // [n][3] world
  const float* direction;
  const int* pose;       // [n]; indices outside [0, n_poses) make an empty ray
  int n_poses;
  const float* target;   // [n][3]
  int* count;            // device scalar: samples
  int* ray_n;            // [n] samples per ray
  float* ray_dt;         // [n] slot spacing
  int* ray_idx;          // [n][n_slots] sample index of the ray's j-th sample
  float4* s_pos;         // [cap] normalised position, pose bits
  float4* s_out;         // [cap] sigma (0 without a root), rgb
  float4* s_x;           // [cap] x*, has-root
  float4* s_grad;        // [cap] dL/dsigma, dL/dc
  float* act;            // [kActStride][act_ld], channel-major (a warp's samples are contiguous)
  int64_t act_ld;
  float* loss;           // device scalar (accumulated)
  float* rgb_out;        // [n][3] or null
  float* alpha_out;      // [n] or null: alpha = 1 - final transmittance
  int comp_mode;         // kCompLoss, kCompForward or kCompUpstream (train_composite_kernel)
  const float* up_rgb;   // [n][3] dL/dC from the caller (kCompUpstream)
  const float* up_alpha; // [n] dL/dalpha from the caller, or null (kCompUpstream)
  float* g_table;
  float* g_mlp;
  float* g_skin;
  float* g_bones;
  // reduced precision (prec != fp32): channel-major operands of the weight-gradient GEMM
  int prec;
  uint16_t* X;           // kWgRows x ld fp16 / bf16, chunk-contiguous (wg_index)
  int64_t ld;            // samples X holds (a multiple of 64; layout wg_index)
  float* scale;          // dynamic loss scale (device scalar)
  int* overflow;         // the step's skip flags (kStepOverflow, kStepPipelineError)
  int* good_steps;       // steps since the last overflow
  uint64_t wait_ns;      // bound on each wait of the tensor-core pipeline
  int inject;            // ia_set_fault_injection flags
  size_t n_table_f, n_mlp_f, n_skin_f, n_bones_f;  // gradient sizes (floats)
  const double* theta_all;  // [n_poses][nb][3] (proposal search: per-pose layer-1 bias)
  unsigned long long* stats;  // [ST_COUNT] counters of this step
  int* pose_tot;         // [n_poses] samples per pose, then the first index of each pose (zeroed by the host)
  int* pose_fill;        // [n_poses] fill counters (zeroed by the host)
  float4* s_dfeat;       // [samples][kIn / 4] dL/dfeatures (fp32, unscaled)
  float4* s_gx;          // [samples] dL/dx* of the hash encoding (between the scatter's two kernels)
  unsigned* work;        // list counter of the sample kernel (zeroed by the host)
  // occupancy-based density regulariser (Eq. 12)
  int n_reg;
  const float* reg_x;    // [n_reg][3] normalised space
  const int32_t* reg_pose;
  float reg_weight;
  int* reg_idx;          // [n_reg] sample index of each point in an empty cell, else -1
  // loss set (Sec. 3.4)
  int huber;
  float huber_delta, w_rgb, w_alpha, w_hard;
  const float* alpha_target;  // [n_rays] (w_alpha != 0)
  int skin_vec;          // skin / g_skin as float4 groups of bones (nb % 4 == 0, 16-byte aligned)
};

// b1p[pose][j] = b1[j] + W1[j, pose columns] . theta_pose for every pose
cudaError_t launch_prop_bias(const PropDev& Q, int nb, const double* theta_all, int n_poses, float* b1p,
                             cudaStream_t s);

// Names of the precision / search variants of a kernel, for launch tracing
template <Prec P>
constexpr const char* variant_name(const char* f32, const char* f16, const char* bf16) {
  return P == Prec::F32 ? f32 : (P == Prec::F16 ? f16 : bf16);
}

// Opt a kernel into `smem` bytes of dynamic shared memory and ask for the
// smallest shared-memory carveout that still fits as many blocks per SM as its
// registers allow, so that the rest of the SM's unified memory serves as L1
// (the correspondence search gathers the blended grid through L1).
template <typename Kern>
cudaError_t set_smem(Kern k, size_t smem, int threads) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, k)) != cudaSuccess) return e;
  int dev = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
    return e;
  const int regs = fa.numRegs > 0 ? fa.numRegs : 1;
  int blocks = 65536 / (regs * threads);
  blocks = blocks < 1 ? 1 : (blocks > 32 ? 32 : blocks);
  const size_t need = (size_t)blocks * (smem + fa.sharedSizeBytes + 1024);  // + per-block reserve
  int pct = (int)((100 * need + per_sm - 1) / per_sm);
  pct = pct > 100 ? 100 : pct;
  return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

constexpr float kInitialLossScale = 16384.f;  // 2^14
// default bound on each wait of the tensor-core pipeline: the whole reduction
// takes well under a millisecond, so a wait this long means it is stuck
constexpr uint64_t kDefaultWaitNs = 200000000ull;  // 200 ms

// Where the compositing kernel takes dL/dC and dL/dalpha from
constexpr int kCompLoss = 0;      // the step's own loss (ia_train_step)
constexpr int kCompForward = 1;   // none: colour and alpha only (ia_train_forward)
constexpr int kCompUpstream = 2;  // the caller's per-ray gradients (ia_train_backward)

// The whole step: forward, compositing (a.comp_mode), backward.
cudaError_t launch_train(const TrainArgs& a, const CUtensorMap* map, int num_sms, cudaStream_t s);
// Its parts: march + posed field of every sample; compositing (and the
// regulariser's density gradient with kCompLoss); the backward from s_grad.
cudaError_t launch_train_forward(const TrainArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_train_composite(const TrainArgs& a, cudaStream_t s);
cudaError_t launch_train_backward(const TrainArgs& a, const CUtensorMap* map, int num_sms, cudaStream_t s);

// Proposal network (ia_prop.cu).
constexpr int kPropMaxIn = 2 * 8 + 3 * kMaxBones;  // 8 levels x 2 features + 32 bones x 3
constexpr int kPropRow = kPropMaxIn + 3 * kWidth + 2 * kPropMaxOut + 3 * kWidth;

struct PropLabelArgs {
  SkinDev S;
  const float* skin;     // [V][nb]
  int nb;
  const float* Ninv;     // [nb][12] of the pose
  int n;
  const float* x;        // [n][3] normalised posed points
  const float* xc;       // [n][3] selected roots
  const int* start;      // [n] (-1: no root)
  int* label;            // [n] (-1: no root)
  float* offset;         // [n][3]
};

struct PropTrainArgs {
  PropDev Q;             // fp32 master table and MLP
  int nb;
  const double* theta;   // [n_poses][nb][3]
  int n;                 // pairs
  int first, batch;      // this step's pairs: (first + i) % n, i < batch
  const float* x;        // [n][3]
  const int* pose;       // [n]
  const int* label;      // [n]
  const float* target;   // [n][3]
  float offset_weight;
  float* rows;           // [batch][kPropRow]
  float* loss;           // device scalar (accumulated)
  float* g_table;        // [entries][2]
  float* g_mlp;          // packed
};

cudaError_t launch_prop_label(const PropLabelArgs& a, cudaStream_t s);
cudaError_t launch_prop_grad(const PropTrainArgs& a, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, int step, float b1,
                        float b2, float eps, const int* skip, cudaStream_t s);

cudaError_t launch_pose_chain(int P, int nb, const int* parent, const double* rest, const double* theta,
                              const double* trans, float* N, float* Ninv, float* B0inv, cudaStream_t s);
cudaError_t launch_blend(int P, int V, int nb, const float* W, const float* N, float4* M, cudaStream_t s);
cudaError_t launch_occ_density(const PosedArgs& a, const BoxDev& box, const float* jitter, const int* cells,
                               const unsigned* count, float* sigma, unsigned long long* stats, unsigned* work,
                               int num_sms, cudaStream_t s);
// cell_box: each skinning cell's grown image box, [n_poses][(Rw - 1)^3][2]
cudaError_t launch_occ_cover(const SkinDev& S, int V, int n_poses, const SolveCfg& cfg, const BoxDev& box,
                             unsigned long long* sub, unsigned* cen, cudaStream_t s, float4* cell_box = nullptr);
cudaError_t launch_occ_cull(const PosedArgs& a, const BoxDev& box, const float* jitter, unsigned long long* sub,
                            unsigned* cen, unsigned* count, int* cells, float* sigma, unsigned long long* stats,
                            cudaStream_t s, float4* cell_box = nullptr);
cudaError_t launch_occ_boxlist(const float4* cell_box, int n_cells, int n_poses, const BoxDev& box,
                               const uint32_t* occ, int* count, int* list, int cap, cudaStream_t s);
cudaError_t launch_gather_probe(const float* table, int64_t n_records, int record_bytes, int iters, int blocks,
                                float* sink, cudaStream_t s);
cudaError_t launch_atomic_probe(float* table, int64_t n_records, int record_bytes, int iters, int blocks,
                                cudaStream_t s);
cudaError_t launch_occ_ema(const float* sigma, float* d, int n, float decay, cudaStream_t s);
cudaError_t launch_occ_bits(const float* sigma, int R, int dilate, float tau, uint32_t* bits,
                            uint32_t* union_bits, cudaStream_t s);
cudaError_t launch_query_posed(const PosedArgs& a, int n, const float* x, float* sigma, float* rgb,
                               float* xc, int* start, cudaStream_t s);
cudaError_t launch_query_canonical(const PosedArgs& a, int n, const float* x, float* sigma, float* rgb,
                                   cudaStream_t s);
cudaError_t launch_table_to_half(const float* table, __half2* th, int64_t entries, cudaStream_t s);
cudaError_t launch_render(const RenderArgs& a, int num_sms, cudaStream_t s);

// Wavefront render path (ia_wavefront.cu): march -> [proposal] -> search waves
// -> field -> compositing, over these arrays (device, context-owned).
cudaError_t launch_wf_march(const RenderArgs& a, const WfArgs& w, cudaStream_t s);
// proposal, search waves and field of the chunk w.s0, w.ns
cudaError_t launch_wf_chunk(const RenderArgs& a, const WfArgs& w, int num_sms, cudaStream_t s);
cudaError_t launch_wf_composite(const RenderArgs& a, const WfArgs& w, cudaStream_t s);
// density at the occupancy cells' query points (cells/count: the candidates, or
// null for every cell) through the chunk kernels; w: xn, res with R^3 entries,
// the item arrays for R^3 samples, n_fb
cudaError_t launch_wf_occupancy(const PosedArgs& P, const BoxDev& box, const float* jitter, const int* cells,
                                const unsigned* count, float* sigma, unsigned long long* stats, WfArgs w, int num_sms,
                                cudaStream_t s);
cudaError_t launch_march_mask(const RenderArgs& a, uint32_t* mask, cudaStream_t s);

}  // namespace ia
