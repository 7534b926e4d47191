// Flux kernels with a source term (Section 2: the balance law with S(Q), the
// GRP with the source, the numerical source of eq. eq:source), linear GRPrec
// reconstruction: advection with S = k q and the Euler equations with a
// constant acceleration, M = 1..4 (gamma = 7/5 fast path and generic gamma).
#include "grp_kernels.cuh"
#include "grp_launch.h"

namespace grp {
cudaError_t launch_flux_src(const StepArgs& a, cudaStream_t s)
{
  const unsigned g = (unsigned)((flux_threads(a.nif) + GRP_FLUX_TPB - 1) / GRP_FLUX_TPB);
  const bool g75 = a.ph.gamma == 1.4;
  if (a.sys == SYS_ADV) {
    switch (a.M) {
      case 1: k_flux<SYS_ADV, 1, false, false, true><<<g, GRP_FLUX_TPB, 0, s>>>(a); break;
      case 2: k_flux<SYS_ADV, 2, false, false, true><<<g, GRP_FLUX_TPB, 0, s>>>(a); break;
      case 3: k_flux<SYS_ADV, 3, false, false, true><<<g, GRP_FLUX_TPB, 0, s>>>(a); break;
      case 4: k_flux<SYS_ADV, 4, false, false, true><<<g, GRP_FLUX_TPB, 0, s>>>(a); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  switch (a.M) {
    case 1:
      if (g75) k_flux<SYS_EULER, 1, true, false, true><<<g, GRP_FLUX_TPB, 0, s>>>(a);
      else k_flux<SYS_EULER, 1, false, false, true><<<g, GRP_FLUX_TPB, 0, s>>>(a);
      break;
    case 2:
      if (g75) k_flux<SYS_EULER, 2, true, false, true><<<g, GRP_FLUX_TPB, 0, s>>>(a);
      else k_flux<SYS_EULER, 2, false, false, true><<<g, GRP_FLUX_TPB, 0, s>>>(a);
      break;
    default: return launch_flux_src_m34(a, s);
  }
  return cudaGetLastError();
}
}  // namespace grp
