// Flux and persistent batched kernels of linear advection, M = 1..4, GRPrecNL
// reconstruction.
#include "grp_flux_inst.cuh"

namespace grp {
GRP_DEFINE_ADV_LAUNCHERS(true, _nl)
}  // namespace grp
