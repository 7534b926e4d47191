// FP64 throughput probe (roofline denominator): independent FMA chains.
#include <cuda_runtime.h>
#include <stdio.h>

#include "grprec.h"

namespace {

constexpr int CHAINS = 8;

__global__ void k_dfma_chains(double* out, int iters, double a, double b)
{
  double x[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += x[k];
  if (s == 12345.678) out[0] = s;   // keeps the chains live; practically never taken
}

}  // namespace

extern "C" int grp_probe_fp64_peak(int device, double* flops_per_s)
{
  if (!flops_per_s) return GRP_E_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return GRP_E_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return GRP_E_CUDA;
  double* out = nullptr;
  if (cudaMalloc((void**)&out, sizeof(double)) != cudaSuccess) return GRP_E_CUDA;
  const int threads = 256, blocks = prop.multiProcessorCount * 8;
  const double a = 0.999999999, b = 1e-9;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_dfma_chains<<<blocks, threads>>>(out, 256, a, b);   // warm-up
  int iters = 4096;
  float ms = 0.f;
  for (int rep = 0; rep < 6; ++rep) {
    cudaEventRecord(e0);
    k_dfma_chains<<<blocks, threads>>>(out, iters, a, b);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 150.f) break;
    iters *= 2;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return GRP_E_CUDA;
  *flops_per_s = 2.0 * CHAINS * (double)iters * threads * (double)blocks / (ms * 1e-3);
  return GRP_OK;
}
