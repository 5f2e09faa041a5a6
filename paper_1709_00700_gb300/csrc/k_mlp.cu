// Cost-model network: fp32 multilayer perceptron that predicts a variant's
// log run time (a per-query variant choice, the run-time optimizer the paper
// leaves to future work, Section 9.4).
//
//   xh = (x - mu) / sigma            F features
//   z1 = xh W1 + b1, h1 = relu(z1)   H = 64 units
//   z2 = h1 W2 + b2, h2 = relu(z2)   H units
//   y  = h2 w3 + b3
//   L  = mean over the batch of (y - t)^2
//
// Parameters are one float vector: W1 (F x H, row-major), b1, W2 (H x H),
// b2, w3, b3.  Adam (Kingma and Ba, 2015, Algorithm 1) updates it in place.
// One thread per sample for the forward and per-sample backward passes
// (weights staged in shared memory, read as broadcasts); weight gradients are
// block partial sums over a tile of samples staged in shared memory, added to
// the gradient with atomics.
#include <algorithm>

#include "pv_internal.h"

namespace pv {

constexpr int kH = PV_MLP_HIDDEN;
constexpr int kMaxF = PV_MLP_MAX_FEATURES;
constexpr int kTile = 64;  // samples per block in the weight-gradient kernel

struct MlpArgs {
  const float* p;      // parameters
  const float* x;      // [B x F]
  const float* mu;     // [F]
  const float* sigma;  // [F]
  float* y;            // [B]
  float* act;          // [B x 2H]: z1 then z2 of every sample (may be null in forward)
  const float* t;      // [B] targets
  float* dz;           // [B x (2H + 1)]: dz1, dz2, dy per sample
  float* grad;         // same layout as p
  float* loss;         // [1]
  int B, F;
};

__host__ __device__ inline int64_t mlp_n_params(int F) { return static_cast<int64_t>(F) * kH + kH + kH * kH + kH + kH + 1; }

// Stages all parameters in shared memory.
__device__ __forceinline__ void stage_params(float* sp, const float* p, int F) {
  const int n = static_cast<int>(mlp_n_params(F));
  for (int i = threadIdx.x; i < n; i += blockDim.x) sp[i] = p[i];
  __syncthreads();
}

__global__ void __launch_bounds__(128) k_mlp_forward(const __grid_constant__ MlpArgs a) {
  extern __shared__ float sp[];
  stage_params(sp, a.p, a.F);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.B) return;
  const int F = a.F;
  const float* W1 = sp;
  const float* b1 = W1 + F * kH;
  const float* W2 = b1 + kH;
  const float* b2 = W2 + kH * kH;
  const float* w3 = b2 + kH;
  const float b3 = w3[kH];
  float z[kH];
#pragma unroll
  for (int j = 0; j < kH; ++j) z[j] = b1[j];
  for (int f = 0; f < F; ++f) {
    const float xh = (a.x[static_cast<int64_t>(i) * F + f] - a.mu[f]) / a.sigma[f];
#pragma unroll
    for (int j = 0; j < kH; ++j) z[j] = fmaf(xh, W1[f * kH + j], z[j]);
  }
  float z2[kH];
#pragma unroll
  for (int k = 0; k < kH; ++k) z2[k] = b2[k];
#pragma unroll
  for (int j = 0; j < kH; ++j) {
    const float h = fmaxf(z[j], 0.0f);
#pragma unroll
    for (int k = 0; k < kH; ++k) z2[k] = fmaf(h, W2[j * kH + k], z2[k]);
  }
  float y = b3;
#pragma unroll
  for (int k = 0; k < kH; ++k) y = fmaf(fmaxf(z2[k], 0.0f), w3[k], y);
  a.y[i] = y;
  if (a.act) {
    float* o = a.act + static_cast<int64_t>(i) * 2 * kH;
#pragma unroll
    for (int j = 0; j < kH; ++j) o[j] = z[j];
#pragma unroll
    for (int k = 0; k < kH; ++k) o[kH + k] = z2[k];
  }
}

// Per-sample backward: dy = 2 (y - t) / B, dz2 = dy w3 (z2 > 0),
// dz1 = (W2 dz2)(z1 > 0); also the loss.
__global__ void __launch_bounds__(128) k_mlp_backward_rows(const __grid_constant__ MlpArgs a) {
  extern __shared__ float sp[];
  stage_params(sp, a.p, a.F);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int F = a.F;
  const float* W2 = sp + F * kH + kH;
  const float* w3 = W2 + kH * kH + kH;
  float l = 0.0f;
  if (i < a.B) {
    const float d = a.y[i] - a.t[i];
    l = d * d / a.B;
    const float dy = 2.0f * d / a.B;
    const float* z = a.act + static_cast<int64_t>(i) * 2 * kH;
    float* o = a.dz + static_cast<int64_t>(i) * (2 * kH + 1);
    float dz2[kH];
#pragma unroll
    for (int k = 0; k < kH; ++k) dz2[k] = z[kH + k] > 0.0f ? dy * w3[k] : 0.0f;
#pragma unroll
    for (int j = 0; j < kH; ++j) {
      float s = 0.0f;
#pragma unroll
      for (int k = 0; k < kH; ++k) s = fmaf(W2[j * kH + k], dz2[k], s);
      o[j] = z[j] > 0.0f ? s : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < kH; ++k) o[kH + k] = dz2[k];
    o[2 * kH] = dy;
  }
  // loss: warp sums, one atomic per warp
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
  if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(a.loss, l);
}

// Weight gradients over a tile of kTile samples: the tile's inputs (xh),
// activations (h1, h2) and deltas (dz1, dz2, dy) are staged in shared memory;
// each thread accumulates a few parameters over the tile and adds them to the
// gradient with one atomic each.
__global__ void __launch_bounds__(256) k_mlp_backward_weights(const __grid_constant__ MlpArgs a) {
  extern __shared__ float sm[];
  const int F = a.F;
  float* xh = sm;                 // [kTile][F]
  float* h1 = xh + kTile * F;     // [kTile][H]
  float* h2 = h1 + kTile * kH;    // [kTile][H]
  float* d1 = h2 + kTile * kH;    // [kTile][H]
  float* d2 = d1 + kTile * kH;    // [kTile][H]
  float* dy = d2 + kTile * kH;    // [kTile]
  const int i0 = blockIdx.x * kTile;
  const int n = min(kTile, a.B - i0);
  for (int e = threadIdx.x; e < kTile * F; e += blockDim.x) {
    const int s = e / F, f = e % F;
    xh[e] = s < n ? (a.x[static_cast<int64_t>(i0 + s) * F + f] - a.mu[f]) / a.sigma[f] : 0.0f;
  }
  for (int e = threadIdx.x; e < kTile * kH; e += blockDim.x) {
    const int s = e / kH, j = e % kH;
    const bool v = s < n;
    const float* z = a.act + static_cast<int64_t>(i0 + s) * 2 * kH;
    const float* o = a.dz + static_cast<int64_t>(i0 + s) * (2 * kH + 1);
    h1[e] = v ? fmaxf(z[j], 0.0f) : 0.0f;
    h2[e] = v ? fmaxf(z[kH + j], 0.0f) : 0.0f;
    d1[e] = v ? o[j] : 0.0f;
    d2[e] = v ? o[kH + j] : 0.0f;
  }
  for (int s = threadIdx.x; s < kTile; s += blockDim.x)
    dy[s] = s < n ? a.dz[static_cast<int64_t>(i0 + s) * (2 * kH + 1) + 2 * kH] : 0.0f;
  __syncthreads();
  const int64_t np = mlp_n_params(F);
  const int64_t oW1 = 0, ob1 = F * kH, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, ow3 = ob2 + kH, ob3 = ow3 + kH;
  for (int64_t q = threadIdx.x; q < np; q += blockDim.x) {
    float g = 0.0f;
    if (q < ob1) {
      const int f = static_cast<int>(q / kH), j = static_cast<int>(q % kH);
      for (int s = 0; s < kTile; ++s) g = fmaf(xh[s * F + f], d1[s * kH + j], g);
    } else if (q < oW2) {
      const int j = static_cast<int>(q - ob1);
      for (int s = 0; s < kTile; ++s) g += d1[s * kH + j];
    } else if (q < ob2) {
      const int j = static_cast<int>((q - oW2) / kH), k = static_cast<int>((q - oW2) % kH);
      for (int s = 0; s < kTile; ++s) g = fmaf(h1[s * kH + j], d2[s * kH + k], g);
    } else if (q < ow3) {
      const int k = static_cast<int>(q - ob2);
      for (int s = 0; s < kTile; ++s) g += d2[s * kH + k];
    } else if (q < ob3) {
      const int k = static_cast<int>(q - ow3);
      for (int s = 0; s < kTile; ++s) g = fmaf(h2[s * kH + k], dy[s], g);
    } else {
      for (int s = 0; s < kTile; ++s) g += dy[s];
    }
    if (g != 0.0f) atomicAdd(a.grad + q, g);
  }
}

__global__ void k_mlp_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                           float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

pv_status mlp_forward(cudaStream_t s, int* launches, const float* params, const float* x, const float* mu,
                      const float* sigma, int B, int F, float* y, float* act) {
  if (B < 0 || F < 1 || F > kMaxF || !params || !x || !mu || !sigma || (B > 0 && !y)) return PV_ERR_INVALID_ARG;
  if (B == 0) return PV_OK;
  MlpArgs a{};
  a.p = params; a.x = x; a.mu = mu; a.sigma = sigma; a.y = y; a.act = act; a.B = B; a.F = F;
  const size_t smem = static_cast<size_t>(mlp_n_params(F)) * sizeof(float);
  if (cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
    return PV_ERR_CUDA;
  k_mlp_forward<<<(B + 127) / 128, 128, smem, s>>>(a);
  ++*launches;
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

pv_status mlp_backward(cudaStream_t s, int* launches, const float* params, const float* x, const float* mu,
                       const float* sigma, const float* act, const float* y, const float* t, int B, int F,
                       float* dz, float* grad, float* loss) {
  if (B < 1 || F < 1 || F > kMaxF || !params || !x || !mu || !sigma || !act || !y || !t || !dz || !grad || !loss)
    return PV_ERR_INVALID_ARG;
  MlpArgs a{};
  a.p = params; a.x = x; a.mu = mu; a.sigma = sigma; a.y = const_cast<float*>(y); a.act = const_cast<float*>(act);
  a.t = t; a.dz = dz; a.grad = grad; a.loss = loss; a.B = B; a.F = F;
  if (cudaMemsetAsync(grad, 0, static_cast<size_t>(mlp_n_params(F)) * sizeof(float), s) != cudaSuccess) return PV_ERR_CUDA;
  if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return PV_ERR_CUDA;
  const size_t smem1 = static_cast<size_t>(mlp_n_params(F)) * sizeof(float);
  if (cudaFuncSetAttribute(k_mlp_backward_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem1)) != cudaSuccess)
    return PV_ERR_CUDA;
  k_mlp_backward_rows<<<(B + 127) / 128, 128, smem1, s>>>(a);
  const size_t smem2 = static_cast<size_t>(kTile) * (F + 4 * kH + 1) * sizeof(float);
  if (cudaFuncSetAttribute(k_mlp_backward_weights, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem2)) != cudaSuccess)
    return PV_ERR_CUDA;
  k_mlp_backward_weights<<<(B + kTile - 1) / kTile, 256, smem2, s>>>(a);
  *launches += 2;
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

pv_status mlp_adam(cudaStream_t s, int* launches, float* p, const float* g, float* m, float* v, int64_t n, float lr,
                   float b1, float b2, float eps, int step) {
  if (!p || !g || !m || !v || n < 0 || step < 1 || !(b1 >= 0 && b1 < 1) || !(b2 >= 0 && b2 < 1)) return PV_ERR_INVALID_ARG;
  if (n == 0) return PV_OK;
  const float c1 = 1.0f - powf(b1, static_cast<float>(step));
  const float c2 = 1.0f - powf(b2, static_cast<float>(step));
  const int grid = static_cast<int>(std::min<int64_t>(1024, (n + 255) / 256));
  k_mlp_adam<<<grid, 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
  ++*launches;
  return cudaGetLastError() == cudaSuccess ? PV_OK : PV_ERR_CUDA;
}

}  // namespace pv
