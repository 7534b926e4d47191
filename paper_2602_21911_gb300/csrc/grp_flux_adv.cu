// Flux and persistent batched kernels of linear advection, M = 1..4.
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

cudaError_t launch_batch_adv(const BatchLaunch& L, cudaStream_t s)
{
#define GRP_BATCH_ADV(MM) \
  k_batch<SYS_ADV, MM, false><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp, L.nsteps, L.parity, L.A0, L.A1, L.I0, L.I1)
  switch (L.a.M) {
    case 1: GRP_BATCH_ADV(1); break;
    case 2: GRP_BATCH_ADV(2); break;
    case 3: GRP_BATCH_ADV(3); break;
    case 4: GRP_BATCH_ADV(4); break;
    default: return cudaErrorInvalidValue;
  }
#undef GRP_BATCH_ADV
  return cudaGetLastError();
}
cudaError_t launch_post_adv(const BatchLaunch& L, cudaStream_t s)
{
  k_post<SYS_ADV, false><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp);
  return cudaGetLastError();
}
}  // namespace grp
