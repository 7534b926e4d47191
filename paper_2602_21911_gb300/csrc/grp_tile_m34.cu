// Launchers of the tile kernel for the Euler equations at degrees 3 and 4 (a
// translation unit of their own, compiled in parallel with the rest).
#include "grp_launch.h"
#include "grp_tile.cuh"

namespace grp {
namespace {
template <int M, bool G75, bool NL>
cudaError_t go(const StepArgs& a, const TileArgs& T, unsigned blocks, size_t smem, cudaStream_t s)
{
  // blocks == 0: only raise the kernel's dynamic shared-memory limit (done
  // once per tiling, outside stream capture, before the first launch)
  if (blocks == 0) return cudaFuncSetAttribute(k_tile<SYS_EULER, M, G75, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_tile<SYS_EULER, M, G75, NL><<<blocks, TILE_THREADS, smem, s>>>(a, T);
  return cudaGetLastError();
}

template <int M>
cudaError_t euler(const StepArgs& a, const TileArgs& T, unsigned blocks, size_t smem, cudaStream_t s)
{
  const bool nl = a.recon != 0, g75 = a.ph.gamma == 1.4;
  if (g75) return nl ? go<M, true, true>(a, T, blocks, smem, s) : go<M, true, false>(a, T, blocks, smem, s);
  return nl ? go<M, false, true>(a, T, blocks, smem, s) : go<M, false, false>(a, T, blocks, smem, s);
}
}  // namespace

cudaError_t launch_tile_m34(const StepArgs& a, const TileArgs& T, unsigned blocks, size_t smem, cudaStream_t s)
{
  return a.M == 3 ? euler<3>(a, T, blocks, smem, s) : a.M == 4 ? euler<4>(a, T, blocks, smem, s)
                                                                  : cudaErrorInvalidValue;
}
}  // namespace grp
