// Internal launch interface between the C ABI (ia_api.cu) and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ia_device.cuh"
#include "ia_index.cuh"

namespace ia {

enum StatIdx {
  ST_RAYS = 0, ST_HIT, ST_MARCHED, ST_OCC, ST_STARTS, ST_ITERS, ST_CONV, ST_ROOTS, ST_EARLY,
  ST_COUNT = 16
};

constexpr int kRenderThreads = 256;
constexpr int kTile = 16;  // rays are handed out in 16 x 16 pixel tiles

struct PosedArgs {
  SkinDev S;
  FieldDev F;
  SolveCfg cfg;
  const float* Ninv;   // [nb][12] of the pose
  const float* mlp;    // packed MLP (fp32)
  int n_in;
};

struct RenderArgs {
  PosedArgs P;
  const float* B0inv;  // [12]
  const uint32_t* occ;
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

size_t posed_smem_bytes(int threads);
size_t render_smem_bytes(int K);

cudaError_t launch_pose_chain(int P, int nb, const int* parent, const double* rest, const double* theta,
                              const double* trans, float* N, float* Ninv, float* B0inv, cudaStream_t s);
cudaError_t launch_blend(int P, int V, int nb, const float* W, const float* N, float4* M, cudaStream_t s);
cudaError_t launch_occ_density(const PosedArgs& a, const BoxDev& box, float* sigma,
                               unsigned long long* stats, cudaStream_t s);
cudaError_t launch_occ_bits(const float* sigma, int R, int dilate, float tau, uint32_t* bits,
                            uint32_t* union_bits, cudaStream_t s);
cudaError_t launch_query_posed(const PosedArgs& a, int n, const float* x, float* sigma, float* rgb,
                               float* xc, int* start, cudaStream_t s);
cudaError_t launch_query_canonical(const FieldDev& F, const float* mlp, int n_in, int n, const float* x,
                                   float* sigma, float* rgb, cudaStream_t s);
cudaError_t launch_render(const RenderArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_march_mask(const RenderArgs& a, uint32_t* mask, cudaStream_t s);

}  // namespace ia
