// Flux and persistent batched kernels of the Euler equations, M = 2, GRPrec
// reconstruction (gamma = 7/5 fast path and generic gamma).
#include "grp_flux_inst.cuh"

namespace grp {
GRP_DEFINE_EULER_LAUNCHERS(2, false, m2)

cudaError_t launch_post_euler(const BatchLaunch& L, cudaStream_t s)
{
  if (L.a.ph.gamma == 1.4) k_post<SYS_EULER, true><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp);
  else k_post<SYS_EULER, false><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp);
  return cudaGetLastError();
}
}  // namespace grp
