// Flux and persistent batched kernels of the Euler equations, M = 1, GRPrecNL
// reconstruction in characteristic variables (gamma = 7/5 fast path and
// generic gamma).
#include "grp_flux_inst.cuh"

namespace grp {
GRP_DEFINE_EULER_LAUNCHERS(1, true, m1_nl)
}  // namespace grp
