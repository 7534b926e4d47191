// Host-side launchers of the templated kernels (one translation unit per
// system, degree and reconstruction, so the heavy FP64 instantiations compile
// in parallel).
#pragma once
#include <cuda_runtime.h>

namespace grp {
struct StepArgs;

// One launch of the persistent batched kernel.
struct BatchLaunch {
  const StepArgs& a;
  const int* grp;        // [blocks + 1] first domain of each block
  unsigned blocks, threads;
  int nsteps, parity;
  double *A0, *A1, *I0, *I1;
};

cudaError_t launch_flux_adv(const StepArgs& a, cudaStream_t s);
cudaError_t launch_flux_adv_nl(const StepArgs& a, cudaStream_t s);
cudaError_t launch_batch_adv_nl(const BatchLaunch& L, cudaStream_t s);
cudaError_t launch_flux_euler_m1_nl(const StepArgs& a, cudaStream_t s);
cudaError_t launch_flux_euler_m2_nl(const StepArgs& a, cudaStream_t s);
cudaError_t launch_flux_euler_m3_nl(const StepArgs& a, cudaStream_t s);
cudaError_t launch_flux_euler_m4_nl(const StepArgs& a, cudaStream_t s);
cudaError_t launch_batch_euler_m1_nl(const BatchLaunch& L, cudaStream_t s);
cudaError_t launch_batch_euler_m2_nl(const BatchLaunch& L, cudaStream_t s);
cudaError_t launch_batch_euler_m3_nl(const BatchLaunch& L, cudaStream_t s);
cudaError_t launch_batch_euler_m4_nl(const BatchLaunch& L, cudaStream_t s);
cudaError_t launch_flux_euler_m1(const StepArgs& a, cudaStream_t s);
cudaError_t launch_flux_euler_m2(const StepArgs& a, cudaStream_t s);
cudaError_t launch_flux_euler_m3(const StepArgs& a, cudaStream_t s);
cudaError_t launch_flux_euler_m4(const StepArgs& a, cudaStream_t s);
cudaError_t launch_batch_adv(const BatchLaunch& L, cudaStream_t s);
cudaError_t launch_batch_euler_m1(const BatchLaunch& L, cudaStream_t s);
cudaError_t launch_batch_euler_m2(const BatchLaunch& L, cudaStream_t s);
cudaError_t launch_batch_euler_m3(const BatchLaunch& L, cudaStream_t s);
cudaError_t launch_batch_euler_m4(const BatchLaunch& L, cudaStream_t s);
cudaError_t launch_post_adv(const BatchLaunch& L, cudaStream_t s);
// temporally blocked tiles (grp_tile.cu, grp_tile_m34.cu)
struct TileArgs;
cudaError_t launch_tile(const StepArgs& a, const TileArgs& T, unsigned blocks, size_t smem, cudaStream_t s);
cudaError_t launch_tile_m34(const StepArgs& a, const TileArgs& T, unsigned blocks, size_t smem, cudaStream_t s);
cudaError_t launch_tile_finish(const StepArgs& a, int* dflag, int nsteps, cudaStream_t s);
// flux kernels with a source term (grp_flux_src.cu, grp_flux_src_m34.cu)
cudaError_t launch_flux_src(const StepArgs& a, cudaStream_t s);
cudaError_t launch_flux_src_m34(const StepArgs& a, cudaStream_t s);

// DET solver (grp_det.cu): constant tables of the device (once), the size of
// the edge-value scratch, and the two launches of a step's GRP phase
int det_prepare(int device);
size_t det_doubles_per_cell(int M, int C);
size_t det_doubles(int M, int C, long long ncell);   // the whole DET buffer: edge values and the resume area
cudaError_t launch_det_step(const StepArgs& a, double* ed, cudaStream_t s);
cudaError_t launch_post_euler(const BatchLaunch& L, cudaStream_t s);
}  // namespace grp
