// Flux kernels of the Euler equations, M = 2 (gamma = 7/5 fast path and generic gamma).
#include "grp_kernels.cuh"

namespace grp {
cudaError_t launch_flux_euler_m2(const StepArgs& a, cudaStream_t s)
{
  const unsigned g = (unsigned)((a.nif + 127) / 128);
  if (a.ph.gamma == 1.4) k_flux<SYS_EULER, 2, true><<<g, 128, 0, s>>>(a);
  else k_flux<SYS_EULER, 2, false><<<g, 128, 0, s>>>(a);
  return cudaGetLastError();
}
}  // namespace grp
