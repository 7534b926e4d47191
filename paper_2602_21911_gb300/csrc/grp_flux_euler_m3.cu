// Flux and persistent batched kernels of the Euler equations, M = 3, GRPrec
// reconstruction (gamma = 7/5 fast path and generic gamma).
#include "grp_flux_inst.cuh"

namespace grp {
GRP_DEFINE_EULER_LAUNCHERS(3, false, m3)
}  // namespace grp
