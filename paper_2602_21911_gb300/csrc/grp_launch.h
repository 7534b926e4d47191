// Host-side launchers of the templated flux kernels (one translation unit per
// system so the heavy FP64 instantiations compile in parallel).
#pragma once
#include <cuda_runtime.h>

namespace grp {
struct StepArgs;
cudaError_t launch_flux_adv(const StepArgs& a, cudaStream_t s);
cudaError_t launch_flux_euler_m1(const StepArgs& a, cudaStream_t s);
cudaError_t launch_flux_euler_m2(const StepArgs& a, cudaStream_t s);
cudaError_t launch_flux_euler_m3(const StepArgs& a, cudaStream_t s);
cudaError_t launch_flux_euler_m4(const StepArgs& a, cudaStream_t s);
}  // namespace grp
