// Launchers of the flux and persistent batched kernels for one system, degree
// and reconstruction, defined by macro so that each (degree, reconstruction)
// instantiation sits in a translation unit of its own and they compile in
// parallel.  gamma = 7/5 takes the fast-path instantiation.
#pragma once
#include "grp_kernels.cuh"
#include "grp_launch.h"

namespace grp {
// the second pass of the flux kernel, where the first defers interfaces
template <int MM, bool NLV>
inline void launch_flux_hard(const StepArgs& a, cudaStream_t s)
{
  if constexpr (flux_defers_at<SYS_EULER, MM, NLV, false>()) {
    if (a.hard_cap > 0) {
      static int sms[64] = {0};
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev < 0 || dev >= 64) dev = 0;
      if (!sms[dev]) cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
      const unsigned gh = hard_blocks(a.hard_cap, sms[dev] > 0 ? sms[dev] : 1);
      const bool net = flux_hard_net(a);
      if (a.ph.gamma == 1.4) {
        if (net) k_flux_hard<MM, true, true><<<gh, GRP_HARD_TPB, 0, s>>>(a);
        else k_flux_hard<MM, true, false><<<gh, GRP_HARD_TPB, 0, s>>>(a);
      } else {
        if (net) k_flux_hard<MM, false, true><<<gh, GRP_HARD_TPB, 0, s>>>(a);
        else k_flux_hard<MM, false, false><<<gh, GRP_HARD_TPB, 0, s>>>(a);
      }
    }
  }
}
}  // namespace grp

#define GRP_DEFINE_EULER_LAUNCHERS(MM, NLV, SUFFIX)                                                          \
  cudaError_t launch_flux_euler_##SUFFIX(const StepArgs& a, cudaStream_t s)                                  \
  {                                                                                                          \
    const unsigned g = (unsigned)((flux_threads(a.nif) + GRP_FLUX_TPB - 1) / GRP_FLUX_TPB);                  \
    if (a.ph.gamma == 1.4) k_flux<SYS_EULER, MM, true, NLV><<<g, GRP_FLUX_TPB, 0, s>>>(a);                   \
    else k_flux<SYS_EULER, MM, false, NLV><<<g, GRP_FLUX_TPB, 0, s>>>(a);                                    \
    launch_flux_hard<MM, NLV>(a, s);                                                                         \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  cudaError_t launch_batch_euler_##SUFFIX(const BatchLaunch& L, cudaStream_t s)                              \
  {                                                                                                          \
    if (L.a.ph.gamma == 1.4)                                                                                 \
      k_batch<SYS_EULER, MM, true, NLV><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp, L.nsteps, L.parity, L.A0, \
                                                                       L.A1, L.I0, L.I1);                    \
    else                                                                                                     \
      k_batch<SYS_EULER, MM, false, NLV><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp, L.nsteps, L.parity,      \
                                                                        L.A0, L.A1, L.I0, L.I1);             \
    return cudaGetLastError();                                                                               \
  }

#define GRP_DEFINE_ADV_LAUNCHERS(NLV, SUFFIX)                                                                \
  cudaError_t launch_flux_adv##SUFFIX(const StepArgs& a, cudaStream_t s)                                     \
  {                                                                                                          \
    const unsigned g = (unsigned)((flux_threads(a.nif) + GRP_FLUX_TPB - 1) / GRP_FLUX_TPB);                                         \
    switch (a.M) {                                                                                           \
      case 1: k_flux<SYS_ADV, 1, false, NLV><<<g, GRP_FLUX_TPB, 0, s>>>(a); break;                                    \
      case 2: k_flux<SYS_ADV, 2, false, NLV><<<g, GRP_FLUX_TPB, 0, s>>>(a); break;                                    \
      case 3: k_flux<SYS_ADV, 3, false, NLV><<<g, GRP_FLUX_TPB, 0, s>>>(a); break;                                    \
      case 4: k_flux<SYS_ADV, 4, false, NLV><<<g, GRP_FLUX_TPB, 0, s>>>(a); break;                                    \
      default: return cudaErrorInvalidValue;                                                                 \
    }                                                                                                        \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  cudaError_t launch_batch_adv##SUFFIX(const BatchLaunch& L, cudaStream_t s)                                 \
  {                                                                                                          \
    switch (L.a.M) {                                                                                         \
      case 1: k_batch<SYS_ADV, 1, false, NLV><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp, L.nsteps, L.parity, \
                                                                             L.A0, L.A1, L.I0, L.I1); break; \
      case 2: k_batch<SYS_ADV, 2, false, NLV><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp, L.nsteps, L.parity, \
                                                                             L.A0, L.A1, L.I0, L.I1); break; \
      case 3: k_batch<SYS_ADV, 3, false, NLV><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp, L.nsteps, L.parity, \
                                                                             L.A0, L.A1, L.I0, L.I1); break; \
      case 4: k_batch<SYS_ADV, 4, false, NLV><<<L.blocks, L.threads, 0, s>>>(L.a, L.grp, L.nsteps, L.parity, \
                                                                             L.A0, L.A1, L.I0, L.I1); break; \
      default: return cudaErrorInvalidValue;                                                                 \
    }                                                                                                        \
    return cudaGetLastError();                                                                               \
  }
