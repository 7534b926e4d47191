// Training and evaluation kernels of the learned Newton guess (FP32).
//
// Network: 6 -> 64 -> 64 -> 1, tanh hidden layers, linear output; loss: mean
// squared error over a batch; optimiser: Adam.  Parameter layout (4673):
// W1[6][64], b1[64], W2[64][64], b2[64], w3[64], b3.
// Per batch of n samples the caller provides a work array of
// GRP_MLP_WORK_FLOATS(n) floats: h1[n][64], h2[n][64], dz1[n][64], dz2[n][64], dy[n].
#include <cuda_runtime.h>

#include "grp_device.cuh"
#include "grprec.h"

using grp::MLP_NH;
using grp::MLP_NIN;
using grp::MLP_NPARAM;

namespace {

constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + MLP_NIN * MLP_NH;
constexpr int OFF_W2 = OFF_B1 + MLP_NH;
constexpr int OFF_B2 = OFF_W2 + MLP_NH * MLP_NH;
constexpr int OFF_W3 = OFF_B2 + MLP_NH;
constexpr int OFF_B3 = OFF_W3 + MLP_NH;

// forward pass of one sample (accurate tanh, as in training)
__device__ __forceinline__ float forward_one(const float* __restrict__ w, const float* x, float* h1, float* h2)
{
#pragma unroll 8
  for (int j = 0; j < MLP_NH; ++j) {
    float z = w[OFF_B1 + j];
#pragma unroll
    for (int i = 0; i < MLP_NIN; ++i) z = fmaf(x[i], w[OFF_W1 + i * MLP_NH + j], z);
    h1[j] = tanhf(z);
  }
  float y = w[OFF_B3];
  for (int k = 0; k < MLP_NH; ++k) {
    float z = w[OFF_B2 + k];
#pragma unroll 16
    for (int j = 0; j < MLP_NH; ++j) z = fmaf(h1[j], w[OFF_W2 + j * MLP_NH + k], z);
    h2[k] = tanhf(z);
    y = fmaf(h2[k], w[OFF_W3 + k], y);
  }
  return y;
}

__global__ void k_mlp_forward(const float* __restrict__ w, const float* __restrict__ x, long long n,
                              float* __restrict__ y)
{
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  float xi[MLP_NIN], h1[MLP_NH], h2[MLP_NH];
#pragma unroll
  for (int i = 0; i < MLP_NIN; ++i) xi[i] = x[b * MLP_NIN + i];
  y[b] = forward_one(w, xi, h1, h2);
}

// forward + backward of one sample per thread; stores activations and
// back-propagated pre-activation gradients; accumulates the loss
__global__ void k_mlp_fb(const float* __restrict__ w, const float* __restrict__ x, const float* __restrict__ t,
                         long long n, float* __restrict__ work, float* __restrict__ loss)
{
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float* H1 = work;
  float* H2 = H1 + n * MLP_NH;
  float* DZ1 = H2 + n * MLP_NH;
  float* DZ2 = DZ1 + n * MLP_NH;
  float* DY = DZ2 + n * MLP_NH;
  float r2 = 0.0f;
  if (b < n) {
    float xi[MLP_NIN], h1[MLP_NH], h2[MLP_NH];
#pragma unroll
    for (int i = 0; i < MLP_NIN; ++i) xi[i] = x[b * MLP_NIN + i];
    const float y = forward_one(w, xi, h1, h2);
    const float r = y - t[b];
    r2 = r * r;
    const float dy = 2.0f * r / (float)n;
    DY[b] = dy;
    float dz2[MLP_NH];
    for (int k = 0; k < MLP_NH; ++k) {
      dz2[k] = dy * w[OFF_W3 + k] * (1.0f - h2[k] * h2[k]);
      H2[b * MLP_NH + k] = h2[k];
      DZ2[b * MLP_NH + k] = dz2[k];
    }
    for (int j = 0; j < MLP_NH; ++j) {
      float s = 0.0f;
#pragma unroll 16
      for (int k = 0; k < MLP_NH; ++k) s = fmaf(dz2[k], w[OFF_W2 + j * MLP_NH + k], s);
      H1[b * MLP_NH + j] = h1[j];
      DZ1[b * MLP_NH + j] = s * (1.0f - h1[j] * h1[j]);
    }
  }
  // block sum of the squared residuals, one atomic per block
  __shared__ float red[256];
  red[threadIdx.x] = r2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / (float)n);
}

// Weight gradients: reductions over the batch.  Block `blk` handles one row of
// 64 outputs; 256 threads = 64 outputs x 4 partial sums over the samples.
//   blk 0..63 : W2[j][.] = sum_b h1[b][j] dz2[b][.]
//   blk 64..69: W1[i][.] = sum_b x[b][i] dz1[b][.]
//   blk 70    : b1 = sum_b dz1[b][.];  71: b2 = sum_b dz2[b][.]
//   blk 72    : w3 = sum_b h2[b][.] dy[b], and b3 = sum_b dy[b]
__global__ void k_mlp_wgrad(const float* __restrict__ x, long long n, const float* __restrict__ work,
                            float* __restrict__ grad)
{
  const float* H1 = work;
  const float* H2 = H1 + n * MLP_NH;
  const float* DZ1 = H2 + n * MLP_NH;
  const float* DZ2 = DZ1 + n * MLP_NH;
  const float* DY = DZ2 + n * MLP_NH;
  const int blk = blockIdx.x, k = threadIdx.x & 63, part = threadIdx.x >> 6;
  float acc = 0.0f, acc3 = 0.0f;
  for (long long b = part; b < n; b += 4) {
    if (blk < 64) acc = fmaf(H1[b * MLP_NH + blk], DZ2[b * MLP_NH + k], acc);
    else if (blk < 70) acc = fmaf(x[b * MLP_NIN + (blk - 64)], DZ1[b * MLP_NH + k], acc);
    else if (blk == 70) acc += DZ1[b * MLP_NH + k];
    else if (blk == 71) acc += DZ2[b * MLP_NH + k];
    else {
      acc = fmaf(H2[b * MLP_NH + k], DY[b], acc);
      if (k == 0) acc3 += DY[b];
    }
  }
  __shared__ float red[256], red3[4];
  red[threadIdx.x] = acc;
  if (k == 0) red3[part] = acc3;
  __syncthreads();
  if (part == 0) {
    const float s = red[k] + red[64 + k] + red[128 + k] + red[192 + k];
    int dst;
    if (blk < 64) dst = OFF_W2 + blk * MLP_NH + k;
    else if (blk < 70) dst = OFF_W1 + (blk - 64) * MLP_NH + k;
    else if (blk == 70) dst = OFF_B1 + k;
    else if (blk == 71) dst = OFF_B2 + k;
    else dst = OFF_W3 + k;
    grad[dst] = s;
    if (blk == 72 && k == 0) grad[OFF_B3] = red3[0] + red3[1] + red3[2] + red3[3];
  }
}

__global__ void k_mlp_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int n, float lr, float beta1, float beta2, float eps,
                           float c1, float c2)
{
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
  const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

extern "C" {

int grp_mlp_forward(const float* weights, const float* x, long long n, float* y, void* stream)
{
  if (!weights || !x || !y || n < 0) return GRP_E_INVALID_ARG;
  if (n == 0) return GRP_OK;
  k_mlp_forward<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(weights, x, n, y);
  return cudaGetLastError() == cudaSuccess ? GRP_OK : GRP_E_CUDA;
}

int grp_mlp_loss_grad(const float* weights, const float* x, const float* target, long long n, float* grad,
                      float* loss, float* work, void* stream)
{
  if (!weights || !x || !target || !grad || !loss || !work || n < 1) return GRP_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return GRP_E_CUDA;
  k_mlp_fb<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(weights, x, target, n, work, loss);
  k_mlp_wgrad<<<73, 256, 0, s>>>(x, n, work, grad);
  return cudaGetLastError() == cudaSuccess ? GRP_OK : GRP_E_CUDA;
}

int grp_mlp_adam(float* weights, const float* grad, float* m, float* v, int step, float lr, float beta1,
                 float beta2, float eps, void* stream)
{
  if (!weights || !grad || !m || !v || step < 1) return GRP_E_INVALID_ARG;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(weights, grad, m, v, MLP_NPARAM, lr,
                                                                          beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? GRP_OK : GRP_E_CUDA;
}

}  // extern "C"
