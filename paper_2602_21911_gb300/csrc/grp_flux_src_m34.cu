// Euler flux kernels with the constant-acceleration source term, M = 3, 4
// (a translation unit of their own, compiled in parallel with the rest).
#include "grp_kernels.cuh"
#include "grp_launch.h"

namespace grp {
cudaError_t launch_flux_src_m34(const StepArgs& a, cudaStream_t s)
{
  const unsigned g = (unsigned)((flux_threads(a.nif) + GRP_FLUX_TPB - 1) / GRP_FLUX_TPB);
  const bool g75 = a.ph.gamma == 1.4;
  switch (a.M) {
    case 3:
      if (g75) k_flux<SYS_EULER, 3, true, false, true><<<g, GRP_FLUX_TPB, 0, s>>>(a);
      else k_flux<SYS_EULER, 3, false, false, true><<<g, GRP_FLUX_TPB, 0, s>>>(a);
      break;
    case 4:
      if (g75) k_flux<SYS_EULER, 4, true, false, true><<<g, GRP_FLUX_TPB, 0, s>>>(a);
      else k_flux<SYS_EULER, 4, false, false, true><<<g, GRP_FLUX_TPB, 0, s>>>(a);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
}  // namespace grp
