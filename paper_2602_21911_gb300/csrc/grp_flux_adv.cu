// Flux and persistent batched kernels of linear advection, M = 1..4, GRPrec
// reconstruction; the post kernel of the split form.
#include "grp_flux_inst.cuh"

namespace grp {
GRP_DEFINE_ADV_LAUNCHERS(false, )

cudaError_t launch_post_adv(const BatchLaunch& L, cudaStream_t s)
{
  k_post<SYS_ADV, false><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp);
  return cudaGetLastError();
}
}  // namespace grp
