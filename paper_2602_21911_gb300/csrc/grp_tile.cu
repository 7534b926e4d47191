// Launchers of the temporally blocked tile kernel (grp_tile.cuh): linear
// advection and the Euler equations, degrees 1-4, GRPrec and GRPrecNL
// reconstructions (gamma = 7/5 fast path and generic gamma).
#include "grp_launch.h"
#include "grp_tile.cuh"

namespace grp {
namespace {
template <int SYS, int M, bool G75, bool NL>
cudaError_t go(const StepArgs& a, const TileArgs& T, unsigned blocks, size_t smem, cudaStream_t s)
{
  // blocks == 0: only raise the kernel's dynamic shared-memory limit (done
  // once per tiling, outside stream capture, before the first launch)
  if (blocks == 0) return cudaFuncSetAttribute(k_tile<SYS, M, G75, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_tile<SYS, M, G75, NL><<<blocks, TILE_THREADS, smem, s>>>(a, T);
  return cudaGetLastError();
}

template <int M, bool NL>
cudaError_t euler(const StepArgs& a, const TileArgs& T, unsigned blocks, size_t smem, cudaStream_t s)
{
  return a.ph.gamma == 1.4 ? go<SYS_EULER, M, true, NL>(a, T, blocks, smem, s)
                           : go<SYS_EULER, M, false, NL>(a, T, blocks, smem, s);
}
}  // namespace

cudaError_t launch_tile(const StepArgs& a, const TileArgs& T, unsigned blocks, size_t smem, cudaStream_t s)
{
  const bool nl = a.recon != 0;
  if (a.sys == SYS_ADV) {
    switch (a.M) {
      case 1: return nl ? go<SYS_ADV, 1, false, true>(a, T, blocks, smem, s) : go<SYS_ADV, 1, false, false>(a, T, blocks, smem, s);
      case 2: return nl ? go<SYS_ADV, 2, false, true>(a, T, blocks, smem, s) : go<SYS_ADV, 2, false, false>(a, T, blocks, smem, s);
      case 3: return nl ? go<SYS_ADV, 3, false, true>(a, T, blocks, smem, s) : go<SYS_ADV, 3, false, false>(a, T, blocks, smem, s);
      case 4: return nl ? go<SYS_ADV, 4, false, true>(a, T, blocks, smem, s) : go<SYS_ADV, 4, false, false>(a, T, blocks, smem, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (a.M) {
    case 1: return nl ? euler<1, true>(a, T, blocks, smem, s) : euler<1, false>(a, T, blocks, smem, s);
    case 2: return nl ? euler<2, true>(a, T, blocks, smem, s) : euler<2, false>(a, T, blocks, smem, s);
    default: return launch_tile_m34(a, T, blocks, smem, s);
  }
}

cudaError_t launch_tile_finish(const StepArgs& a, int* dflag, int nsteps, cudaStream_t s)
{
  k_tile_finish<<<(a.n_domains + 127) / 128, 128, 0, s>>>(a, dflag, nsteps);
  return cudaGetLastError();
}
}  // namespace grp
