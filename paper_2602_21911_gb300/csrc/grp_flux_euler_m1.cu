// Flux kernel of the Euler equations, M = 1.
#include "grp_kernels.cuh"

namespace grp {
cudaError_t launch_flux_euler_m1(const StepArgs& a, cudaStream_t s)
{
  const unsigned g = (unsigned)((a.nif + 127) / 128);
  k_flux<SYS_EULER, 1><<<g, 128, 0, s>>>(a);
  return cudaGetLastError();
}
}  // namespace grp
