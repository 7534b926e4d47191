// Flux kernels of linear advection, M = 1..4.
#include "grp_kernels.cuh"
#include "grp_launch.h"

namespace grp {
cudaError_t launch_flux_adv(const StepArgs& a, cudaStream_t s)
{
  const unsigned g = (unsigned)((a.nif + 127) / 128);
  switch (a.M) {
    case 1: k_flux<SYS_ADV, 1, false><<<g, 128, 0, s>>>(a); break;
    case 2: k_flux<SYS_ADV, 2, false><<<g, 128, 0, s>>>(a); break;
    case 3: k_flux<SYS_ADV, 3, false><<<g, 128, 0, s>>>(a); break;
    case 4: k_flux<SYS_ADV, 4, false><<<g, 128, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
}  // namespace grp
