// Learned correspondence proposal (not part of the paper): training kernels.
//
//   prop_label_kernel   training pairs from the plain search: the bone with the
//                       largest skinning weight at the selected root x*, and the
//                       start offset x* - N_label^-1 x'
//   prop_fwd_kernel     per pair: hash features of x' + pose vector -> MLP
//                       (3 x 64, ReLU) -> logits, offset; loss = cross-entropy +
//                       w |offset - target|^2; output gradient
//   prop_bwd_kernel     per pair: hidden-layer gradients and the hash-table
//                       scatter-add
//   dense_grad_kernel   dW = sum_s dH_s A_s^T, db = sum_s dH_s (split-K over pairs)
//   adam_kernel         Adam on the fp32 parameters
// Activations and their gradients are kept per pair in one row of the
// workspace; the network is small (about 30 k parameters) so everything is fp32.
#include "ia_internal.h"

namespace ia {

// row layout of the per-pair workspace
constexpr int kPX = 0;                      // input [2L hash features | 3 nb pose]
constexpr int kPH1 = kPX + kPropMaxIn;
constexpr int kPH2 = kPH1 + kWidth;
constexpr int kPH3 = kPH2 + kWidth;
constexpr int kPO = kPH3 + kWidth;          // outputs (nb logits, 3 offset)
constexpr int kPdO = kPO + kPropMaxOut;
constexpr int kPd3 = kPdO + kPropMaxOut;
constexpr int kPd2 = kPd3 + kWidth;
constexpr int kPd1 = kPd2 + kWidth;
static_assert(kPd1 + kWidth == kPropRow, "row layout");

// ---------------------------------------------------------------------------

__global__ void prop_label_kernel(const PropLabelArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  if (a.start[i] < 0) {  // no valid root: not a training pair
    a.label[i] = -1;
    a.offset[3 * i] = a.offset[3 * i + 1] = a.offset[3 * i + 2] = 0.f;
    return;
  }
  const float3 xs = make_float3(a.xc[3 * i], a.xc[3 * i + 1], a.xc[3 * i + 2]);
  const float3 xn = make_float3(a.x[3 * i], a.x[3 * i + 1], a.x[3 * i + 2]);
  const CellCoord cc = skin_cell(a.S, xs);
  int best = 0;
  float wbest = -1.f;
  for (int k = 0; k < a.nb; ++k) {
    float w = 0.f;
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
      const int v = corner_index(a.S, cc.base, corner);
      const float cw = ((corner & 1) ? cc.f[0] : 1.f - cc.f[0]) * (((corner >> 1) & 1) ? cc.f[1] : 1.f - cc.f[1]) *
                       (((corner >> 2) & 1) ? cc.f[2] : 1.f - cc.f[2]);
      w = fmaf(cw, __ldg(a.skin + (size_t)v * a.nb + k), w);
    }
    if (w > wbest) { wbest = w; best = k; }
  }
  const float* A = a.Ninv + 12 * best;
  a.label[i] = best;
  a.offset[3 * i] = xs.x - (A[0] * xn.x + A[1] * xn.y + A[2] * xn.z + A[3]);
  a.offset[3 * i + 1] = xs.y - (A[4] * xn.x + A[5] * xn.y + A[6] * xn.z + A[7]);
  a.offset[3 * i + 2] = xs.z - (A[8] * xn.x + A[9] * xn.y + A[10] * xn.z + A[11]);
}

cudaError_t launch_prop_label(const PropLabelArgs& a, cudaStream_t s) {
  {
    KernelSpan span("prop_label_kernel", s);
    prop_label_kernel<<<(a.n + 127) / 128, 128, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------

__device__ __forceinline__ void dense_row(const float* __restrict__ W, const float* __restrict__ b, const float* in,
                                          int nin, int nout, float* out, bool relu) {
  for (int j = 0; j < nout; ++j) {
    float acc = b[j];
    const float* w = W + (size_t)j * nin;
    for (int i = 0; i < nin; ++i) acc = fmaf(__ldg(w + i), in[i], acc);
    out[j] = relu ? fmaxf(acc, 0.f) : acc;
  }
}

__device__ __noinline__ float prop_fwd_one(const PropTrainArgs& a, int i);

__global__ void prop_fwd_kernel(const PropTrainArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = i < a.batch;
  float lw = 0.f;
  if (act) lw = prop_fwd_one(a, i);
  for (int off = 16; off > 0; off >>= 1) lw += __shfl_down_sync(kFull, lw, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(a.loss, lw);
}

__device__ __noinline__ float prop_fwd_one(const PropTrainArgs& a, int i) {
  const int s = (a.first + i) % a.n;
  float* row = a.rows + (size_t)i * kPropRow;
  const PropDev& Q = a.Q;
  const int nb = a.nb, nf = 2 * Q.L, nin = Q.n_in, nout = nb + 3;
  float f16[16];
  prop_encode(Q, make_float3(a.x[3 * s], a.x[3 * s + 1], a.x[3 * s + 2]), f16);
  for (int q = 0; q < nf; ++q) row[kPX + q] = f16[q];
  const double* th = a.theta + (size_t)a.pose[s] * nb * 3;
  for (int q = 0; q < 3 * nb; ++q) row[kPX + nf + q] = (float)th[q];
  const float* W1 = Q.mlp;
  const float* b1 = W1 + kWidth * nin;
  const float* W2 = b1 + kWidth;
  const float* b2 = W2 + kWidth * kWidth;
  const float* W3 = b2 + kWidth;
  const float* b3 = W3 + kWidth * kWidth;
  const float* W4 = b3 + kWidth;
  const float* b4 = W4 + nout * kWidth;
  dense_row(W1, b1, row + kPX, nin, kWidth, row + kPH1, true);
  dense_row(W2, b2, row + kPH1, kWidth, kWidth, row + kPH2, true);
  dense_row(W3, b3, row + kPH2, kWidth, kWidth, row + kPH3, true);
  dense_row(W4, b4, row + kPH3, kWidth, nout, row + kPO, false);
  // loss = logsumexp(logits) - logit[label] + w |offset - target|^2, averaged over the batch
  const float* o = row + kPO;
  float mx = o[0];
  for (int q = 1; q < nb; ++q) mx = fmaxf(mx, o[q]);
  float z = 0.f;
  for (int q = 0; q < nb; ++q) z += expf(o[q] - mx);
  const float lse = mx + logf(z);
  const int lab = a.label[s];
  float l = lse - o[lab];
  const float inv_b = 1.f / (float)a.batch;
  float* dO = row + kPdO;
  for (int q = 0; q < nb; ++q) dO[q] = (expf(o[q] - lse) - (q == lab ? 1.f : 0.f)) * inv_b;
  for (int c = 0; c < 3; ++c) {
    const float e = o[nb + c] - a.target[3 * s + c];
    l = fmaf(a.offset_weight * e, e, l);
    dO[nb + c] = 2.f * a.offset_weight * e * inv_b;
  }
  for (int q = nout; q < kPropMaxOut; ++q) dO[q] = 0.f;
  return l * inv_b;
}

__device__ __forceinline__ void back_row(const float* __restrict__ W, const float* dout, int nin, int nout,
                                         const float* act_in, float* din) {
  // din[i] = (sum_j W[j][i] dout[j]) * [act_in[i] > 0]
  for (int i = 0; i < nin; ++i) din[i] = 0.f;
  for (int j = 0; j < nout; ++j) {
    const float d = dout[j];
    const float* w = W + (size_t)j * nin;
    for (int i = 0; i < nin; ++i) din[i] = fmaf(__ldg(w + i), d, din[i]);
  }
  for (int i = 0; i < nin; ++i)
    if (!(act_in[i] > 0.f)) din[i] = 0.f;
}

__global__ void prop_bwd_kernel(const PropTrainArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.batch) return;
  const int s = (a.first + i) % a.n;
  float* row = a.rows + (size_t)i * kPropRow;
  const PropDev& Q = a.Q;
  const int nb = a.nb, nin = Q.n_in, nout = nb + 3;
  const float* W1 = Q.mlp;
  const float* W2 = W1 + kWidth * nin + kWidth;
  const float* W3 = W2 + kWidth * kWidth + kWidth;
  const float* W4 = W3 + kWidth * kWidth + kWidth;
  back_row(W4, row + kPdO, kWidth, nout, row + kPH3, row + kPd3);
  back_row(W3, row + kPd3, kWidth, kWidth, row + kPH2, row + kPd2);
  back_row(W2, row + kPd2, kWidth, kWidth, row + kPH1, row + kPd1);
  // hash features: dX[q] = sum_j W1[j][q] dH1[j], scattered to the 8 corners per level
  const float3 x = make_float3(a.x[3 * s], a.x[3 * s + 1], a.x[3 * s + 2]);
  const float u[3] = {(x.x - Q.nmin[0]) * Q.inv_ext[0], (x.y - Q.nmin[1]) * Q.inv_ext[1],
                      (x.z - Q.nmin[2]) * Q.inv_ext[2]};
  const float* d1 = row + kPd1;
  for (int l = 0; l < Q.L; ++l) {
    float g0 = 0.f, g1 = 0.f;
    for (int j = 0; j < kWidth; ++j) {
      g0 = fmaf(__ldg(W1 + (size_t)j * nin + 2 * l), d1[j], g0);
      g1 = fmaf(__ldg(W1 + (size_t)j * nin + 2 * l + 1), d1[j], g1);
    }
    const Level lv = Q.lv[l];
    int p0[3];
    float f[3];
    for (int c = 0; c < 3; ++c) {
      const float pos = u[c] * (float)lv.res;
      int q = (int)floorf(pos);
      q = min(max(q, 0), lv.res - 1);
      p0[c] = q;
      f[c] = pos - (float)q;
    }
    for (int corner = 0; corner < 8; ++corner) {
      const int cx = corner & 1, cy = (corner >> 1) & 1, cz = (corner >> 2) & 1;
      const float w = (cx ? f[0] : 1.f - f[0]) * (cy ? f[1] : 1.f - f[1]) * (cz ? f[2] : 1.f - f[2]);
      const uint32_t e = lv.offset + vertex_index(lv, p0[0] + cx, p0[1] + cy, p0[2] + cz);
      atomicAdd(a.g_table + 2 * (size_t)e, w * g0);
      atomicAdd(a.g_table + 2 * (size_t)e + 1, w * g1);
    }
  }
}

// dW[o][i] += sum_s D[s][o] A[s][i], db[o] += sum_s D[s][o] over a chunk of rows
constexpr int kDG = 32;

__global__ void __launch_bounds__(256) dense_grad_kernel(const float* __restrict__ rows, int batch, int offA, int nin,
                                                         int offD, int nout, float* gW, float* gb) {
  __shared__ float tA[kDG][kPropMaxIn + 1];
  __shared__ float tD[kDG][kWidth + 1];
  const int chunk = (batch + gridDim.x - 1) / gridDim.x;
  const int s0 = blockIdx.x * chunk, s1 = min(batch, s0 + chunk);
  const int n_out = nout * (nin + 1);  // the last column is the bias
  constexpr int kPer = (kWidth * (kPropMaxIn + 1) + 255) / 256;
  float acc[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) acc[q] = 0.f;
  for (int base = s0; base < s1; base += kDG) {
    const int m = min(kDG, s1 - base);
    __syncthreads();
    for (int q = threadIdx.x; q < m * nin; q += blockDim.x) tA[q / nin][q % nin] = rows[(size_t)(base + q / nin) * kPropRow + offA + q % nin];
    for (int q = threadIdx.x; q < m * nout; q += blockDim.x)
      tD[q / nout][q % nout] = rows[(size_t)(base + q / nout) * kPropRow + offD + q % nout];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = threadIdx.x + q * 256;
      if (e < n_out) {
        const int o = e / (nin + 1), i = e % (nin + 1);
        float a2 = acc[q];
        for (int r = 0; r < m; ++r) a2 = fmaf(tD[r][o], i < nin ? tA[r][i] : 1.f, a2);
        acc[q] = a2;
      }
    }
  }
  if (s0 >= s1) return;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int e = threadIdx.x + q * 256;
    if (e < n_out) {
      const int o = e / (nin + 1), i = e % (nin + 1);
      if (i < nin) atomicAdd(gW + (size_t)o * nin + i, acc[q]);
      else atomicAdd(gb + o, acc[q]);
    }
  }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float c1, float c2, float b1, float b2,
                            float eps, const int* __restrict__ skip) {
  if (skip && *skip) return;  // a skipped (overflowed) step leaves parameters and moments alone
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

cudaError_t launch_prop_grad(const PropTrainArgs& a, cudaStream_t s) {
  cudaError_t e;
  const int blocks = (a.batch + 127) / 128;
  {
    KernelSpan span("prop_fwd_kernel", s);
    prop_fwd_kernel<<<blocks, 128, 0, s>>>(a);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    KernelSpan span("prop_bwd_kernel", s);
    prop_bwd_kernel<<<blocks, 128, 0, s>>>(a);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nin = a.Q.n_in, nout = a.nb + 3;
  float* gW1 = a.g_mlp;
  float* gb1 = gW1 + kWidth * nin;
  float* gW2 = gb1 + kWidth;
  float* gb2 = gW2 + kWidth * kWidth;
  float* gW3 = gb2 + kWidth;
  float* gb3 = gW3 + kWidth * kWidth;
  float* gW4 = gb3 + kWidth;
  float* gb4 = gW4 + nout * kWidth;
  const int g = max(1, min(296, (a.batch + 63) / 64));
  {
    KernelSpan span("dense_grad_kernel", s);
    dense_grad_kernel<<<g, 256, 0, s>>>(a.rows, a.batch, kPX, nin, kPd1, kWidth, gW1, gb1);
  }
  {
    KernelSpan span("dense_grad_kernel", s);
    dense_grad_kernel<<<g, 256, 0, s>>>(a.rows, a.batch, kPH1, kWidth, kPd2, kWidth, gW2, gb2);
  }
  {
    KernelSpan span("dense_grad_kernel", s);
    dense_grad_kernel<<<g, 256, 0, s>>>(a.rows, a.batch, kPH2, kWidth, kPd3, kWidth, gW3, gb3);
  }
  {
    KernelSpan span("dense_grad_kernel", s);
    dense_grad_kernel<<<g, 256, 0, s>>>(a.rows, a.batch, kPH3, kWidth, kPdO, nout, gW4, gb4);
  }
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, int step, float b1,
                        float b2, float eps, const int* skip, cudaStream_t s) {
  // bias corrections of step t (1-based): 1 / (1 - b^t)
  const float c1 = 1.f / (1.f - powf(b1, (float)step)), c2 = 1.f / (1.f - powf(b2, (float)step));
  {
    KernelSpan span("adam_kernel", s);
    adam_kernel<<<592, 256, 0, s>>>(p, g, m, v, n, lr, c1, c2, b1, b2, eps, skip);
  }
  return cudaGetLastError();
}

// per-pose layer-1 bias of the proposal: one thread per (pose, hidden unit),
// fp32 accumulation in the order of the per-block fold (stage_prop_h)
__global__ void prop_bias_kernel(const PropDev Q, int nb, const double* __restrict__ theta_all, int n_poses,
                                 float* __restrict__ b1p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_poses * kWidth) return;
  const int pose = i / kWidth, q = i % kWidth;
  const int nin = Q.n_in, nf = 2 * Q.L;
  const float* g = Q.mlp;
  const double* th = theta_all + (size_t)pose * 3 * nb;
  float f = g[kWidth * nin + q];
  for (int j = 0; j < 3 * nb; ++j) f = fmaf(g[q * nin + nf + j], (float)th[j], f);
  b1p[i] = f;
}

cudaError_t launch_prop_bias(const PropDev& Q, int nb, const double* theta_all, int n_poses, float* b1p,
                             cudaStream_t s) {
  const int n = n_poses * kWidth;
  {
    KernelSpan span("prop_bias_kernel", s);
    prop_bias_kernel<<<(n + 255) / 256, 256, 0, s>>>(Q, nb, theta_all, n_poses, b1p);
  }
  return cudaGetLastError();
}

}  // namespace ia
