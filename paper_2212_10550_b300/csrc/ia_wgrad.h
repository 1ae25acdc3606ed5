// Host-visible part of the tensor-core weight-gradient reduction: the operand
// layout constants, its arguments, and the host entry points (defined with the
// kernel in the translation unit of the training step).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace ia {

constexpr int kWgRows = 384;   // channel rows of the operand array X
constexpr int kWgChunk = 64;   // samples per pipeline stage (128 B of fp16 / bf16)

// Layout of the operand array X: chunk-contiguous.  Row r of sample s sits at
//   (s / kWgChunk) * kWgRows * kWgChunk + r * kWgChunk + s % kWgChunk,
// so every 64-sample chunk of all 384 rows is one contiguous 48 KiB block (the
// GEMM streams whole blocks; a warp's 32 samples of one row are 64 contiguous
// bytes for the backward's stores).
__host__ __device__ __forceinline__ size_t wg_index(int row, int64_t s) {
  return (size_t)(s / kWgChunk) * (kWgRows * kWgChunk) + (size_t)row * kWgChunk + (size_t)(s % kWgChunk);
}

// Bits of a reduced-precision step's flags word (device int, zeroed at the start
// of every step); any bit set means the step is skipped (its gradients zeroed).
constexpr int kStepOverflow = 1;       // a scaled gradient or activation left the operand range
constexpr int kStepPipelineError = 2;  // the tensor-core reduction gave up waiting on its pipeline

struct WgradArgs {
  const int* count;    // samples (device scalar)
  const float* scale;  // loss scale (device scalar)
  float* gW1;          // [64][n_in]
  float* gb1;          // [64]
  float* gW2;          // [64][64]
  float* gb2;          // [64]
  float* gW3;          // [4][64]
  float* gb3;          // [4]
  int n_in;
  int bf16;            // operand type: 0 fp16, 1 bf16
  int* flags;          // the step's skip flags: kStepPipelineError is raised when a wait gives up
  uint64_t wait_ns;    // bound on each pipeline wait
  int withhold_last;   // failure injection: the producer never issues the copy of its last chunk
};

// Tensor map over X (ld samples in the layout of wg_index, 2-byte elements):
// dimensions (64 samples, 384 rows, ld / 64 chunks), 64 x 128 x 1 boxes,
// 128-byte swizzle.  ld must be a multiple of 64 and X 16-byte aligned.
cudaError_t make_wgrad_map(CUtensorMap* map, void* X, int64_t ld, int bf16);
cudaError_t launch_wgrad_tc(const CUtensorMap& map, const WgradArgs& a, int grid, cudaStream_t s);

}  // namespace ia
