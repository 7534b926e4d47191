// Flux and persistent batched kernels of the Euler equations, M = 2
// (gamma = 7/5 fast path and generic gamma).
#include "grp_kernels.cuh"
#include "grp_launch.h"

namespace grp {
cudaError_t launch_flux_euler_m2(const StepArgs& a, cudaStream_t s)
{
  const unsigned g = (unsigned)((a.nif + 127) / 128);
  if (a.ph.gamma == 1.4) k_flux<SYS_EULER, 2, true><<<g, 128, 0, s>>>(a);
  else k_flux<SYS_EULER, 2, false><<<g, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_batch_euler_m2(const BatchLaunch& L, cudaStream_t s)
{
  if (L.a.ph.gamma == 1.4)
    k_batch<SYS_EULER, 2, true><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp, L.nsteps, L.parity, L.A0, L.A1, L.I0, L.I1);
  else
    k_batch<SYS_EULER, 2, false><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp, L.nsteps, L.parity, L.A0, L.A1, L.I0, L.I1);
  return cudaGetLastError();
}
cudaError_t launch_post_euler(const BatchLaunch& L, cudaStream_t s)
{
  if (L.a.ph.gamma == 1.4) k_post<SYS_EULER, true><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp);
  else k_post<SYS_EULER, false><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp);
  return cudaGetLastError();
}
}  // namespace grp
