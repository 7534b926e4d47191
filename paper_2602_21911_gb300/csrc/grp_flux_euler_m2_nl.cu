// Flux and persistent batched kernels of the Euler equations, M = 2, GRPrecNL
// reconstruction in characteristic variables (gamma = 7/5 fast path and
// generic gamma).
#include "grp_flux_inst.cuh"

namespace grp {
GRP_DEFINE_EULER_LAUNCHERS(2, true, m2_nl)
}  // namespace grp
