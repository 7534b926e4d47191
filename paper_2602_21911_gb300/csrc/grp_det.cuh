// The DET GRP solver (the solver of the paper's computations, Section 4.1):
// a local space-time Galerkin predictor evolves each cell's reconstruction
// over the step; classical Riemann problems of the evolved edge values at the
// time integration points give the flux, the one at the end of the step the
// interface datum.  The predictor: tensor-product nodal basis of degree M in
// space and time on the M+1 Gauss-Legendre points of [0, 1], the time
// derivative integrated by parts with upwinding from the reconstruction at
// t^n, nodal quadrature; for each spatial node k and time node l
//   sum_b T_lb q_kb = phi_l(0) w_k - nu w_l sum_a phi_a'(x_k) f(q_al),
//   T_lb = phi_l(1) phi_b(1) - w_b phi_l'(x_b),
// solved by Picard iteration until the largest update is below 1e-13 of the
// largest nodal value (at most 64 iterations).  Riemann problems: exact
// (upwind for advection), at the M+1 time nodes and at the end of the step.
#pragma once
#include "grp_kernels.cuh"

namespace grp {

constexpr int DET_MAXN = 5;

// basis tables of one degree (host-built, in constant memory)
struct DetTab {
  double x[DET_MAXN], w[DET_MAXN];     // nodes, weights on [0, 1]
  double D[DET_MAXN][DET_MAXN];        // D[k][a] = phi_a'(x_k)
  double e0[DET_MAXN], e1[DET_MAXN];   // phi_a(0), phi_a(1)
  double Ti[DET_MAXN][DET_MAXN];       // T^{-1}
  double Te[DET_MAXN];                 // T^{-1} phi(0): sum_b Ti[l][b] e0[b]
  double Tw[DET_MAXN][DET_MAXN];       // T^{-1} diag(w): Ti[l][b] w[b]
};

// ed layout: ed[((side * (M + 2) + g) * C + c) * ncell + cell], side 0 the
// left edge, 1 the right edge; g = 0..M the time nodes, g = M+1 the end.
__device__ __forceinline__ long long det_idx(int M, int C, long long ncell, int side, int g, int c, long long cell)
{
  return ((long long)((side * (M + 2) + g) * C + c)) * ncell + cell;
}

}  // namespace grp
