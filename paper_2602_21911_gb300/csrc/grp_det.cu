// DET solver kernels: the per-cell space-time predictor and the per-interface
// Riemann problems at the time integration points (see grp_det.cuh).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "grp_det.cuh"
#include "grp_launch.h"
#include "grprec.h"

namespace grp {

__constant__ DetTab c_det[4];          // degrees 1..4 at [M - 1]

namespace {

// Gauss-Legendre nodes and weights on [0, 1] in closed form (n <= 5)
void gauss01(int n, double* x, double* w)
{
  double z[5], v[5];
  if (n == 1) { z[0] = 0.0; v[0] = 2.0; }
  else if (n == 2) { const double a = 1.0 / sqrt(3.0); z[0] = -a; z[1] = a; v[0] = v[1] = 1.0; }
  else if (n == 3) { const double a = sqrt(0.6); z[0] = -a; z[1] = 0.0; z[2] = a; v[0] = v[2] = 5.0 / 9.0; v[1] = 8.0 / 9.0; }
  else if (n == 4) {
    const double a = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(1.2)), b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(1.2));
    const double wa = (18.0 + sqrt(30.0)) / 36.0, wb = (18.0 - sqrt(30.0)) / 36.0;
    z[0] = -b; z[1] = -a; z[2] = a; z[3] = b; v[0] = v[3] = wb; v[1] = v[2] = wa;
  } else {
    const double a = sqrt(5.0 - 2.0 * sqrt(10.0 / 7.0)) / 3.0, b = sqrt(5.0 + 2.0 * sqrt(10.0 / 7.0)) / 3.0;
    const double wa = (322.0 + 13.0 * sqrt(70.0)) / 900.0, wb = (322.0 - 13.0 * sqrt(70.0)) / 900.0;
    z[0] = -b; z[1] = -a; z[2] = 0.0; z[3] = a; z[4] = b;
    v[0] = v[4] = wb; v[1] = v[3] = wa; v[2] = 128.0 / 225.0;
  }
  for (int k = 0; k < n; ++k) { x[k] = 0.5 * (z[k] + 1.0); w[k] = 0.5 * v[k]; }
}

// barycentric Lagrange basis on the nodes x[0..n-1]
double bary_w(int n, const double* x, int a)
{
  double p = 1.0;
  for (int j = 0; j < n; ++j) if (j != a) p *= x[a] - x[j];
  return 1.0 / p;
}
double basis_at(int n, const double* x, int a, double s)
{
  double num = bary_w(n, x, a);
  for (int j = 0; j < n; ++j) if (j != a) num *= s - x[j];
  return num;
}
// phi_a'(x_k): the differentiation matrix of the nodes
double diff_at_node(int n, const double* x, int a, int k)
{
  if (a != k) return bary_w(n, x, a) / bary_w(n, x, k) / (x[k] - x[a]);
  double s = 0.0;
  for (int j = 0; j < n; ++j) if (j != k) s += 1.0 / (x[k] - x[j]);
  return s;
}

bool g_det_ready[64];                  // per device

int det_tables(int dev)
{
  if (dev < 0 || dev >= 64) return -1;
  if (g_det_ready[dev]) return 0;
  DetTab t[4];
  memset(t, 0, sizeof(t));
  for (int M = 1; M <= 4; ++M) {
    DetTab& T = t[M - 1];
    const int n = M + 1;
    gauss01(n, T.x, T.w);
    for (int a = 0; a < n; ++a) {
      T.e0[a] = basis_at(n, T.x, a, 0.0);
      T.e1[a] = basis_at(n, T.x, a, 1.0);
      for (int k = 0; k < n; ++k) T.D[k][a] = diff_at_node(n, T.x, a, k);
    }
    // T_lb = phi_l(1) phi_b(1) - w_b phi_l'(x_b), inverted by Gauss-Jordan
    double A[DET_MAXN][2 * DET_MAXN];
    for (int l = 0; l < n; ++l)
      for (int b = 0; b < 2 * n; ++b)
        A[l][b] = b < n ? T.e1[l] * T.e1[b] - T.w[b] * T.D[b][l] : (b - n == l ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
      int piv = col;
      for (int r = col + 1; r < n; ++r) if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
      for (int b = 0; b < 2 * n; ++b) { const double tmp = A[col][b]; A[col][b] = A[piv][b]; A[piv][b] = tmp; }
      const double inv = 1.0 / A[col][col];
      for (int b = 0; b < 2 * n; ++b) A[col][b] *= inv;
      for (int r = 0; r < n; ++r) {
        if (r == col) continue;
        const double f = A[r][col];
        for (int b = 0; b < 2 * n; ++b) A[r][b] -= f * A[col][b];
      }
    }
    for (int l = 0; l < n; ++l) for (int b = 0; b < n; ++b) T.Ti[l][b] = A[l][n + b];
    for (int l = 0; l < n; ++l) {
      T.Te[l] = 0.0;
      for (int b = 0; b < n; ++b) {
        T.Te[l] += T.Ti[l][b] * T.e0[b];
        T.Tw[l][b] = T.Ti[l][b] * T.w[b];
      }
    }
  }
  if (cudaMemcpyToSymbol(c_det, t, sizeof(t)) != cudaSuccess) return -1;
  g_det_ready[dev] = true;
  return 0;
}

template <int SYS>
__device__ __forceinline__ void phys_flux(const Phys& ph, const double* Q, double* F)
{
  if (SYS == SYS_ADV) { F[0] = ph.lambda * Q[0]; return; }
  const double u = Q[1] * rcp64(Q[0]);
  const double p = ph.gm1 * (Q[2] - 0.5 * Q[1] * u);
  F[0] = Q[1];
  F[1] = Q[1] * u + p;
  F[2] = u * (Q[2] + p);
}

// The predictor's Picard iteration runs in two phases.  Most cells converge
// in a few iterations (constant states in one, smooth flow in three), a few
// near strong waves take tens; one thread per cell would hold every warp with
// such a cell for all of them.  Phase 1 runs at most DET_PHASE1 iterations in
// every cell; a cell still iterating saves its nodal values and joins a list
// that phase 2 resumes on a fixed grid, with the same iteration and the same
// limit, so the results are those of one uninterrupted iteration.
constexpr int DET_PHASE1 = 4, DET_MAXIT = 64;

// resume area after the edge values: slot s holds w[n][C] then q[n][n][C]
struct DetResume {
  double* state;       // [cap][(n + n n) C]
  int* list;           // [cap] cells
  int* count;          // cells offered to phase 2 (may exceed cap)
  int cap;
};

// Picard iterations it0 <= it < it1 of one cell.  Returns 1 when converged,
// -1 on an inadmissible nodal state, 0 when it1 was reached first.
template <int SYS, int M>
__device__ __forceinline__ int det_picard(const StepArgs& a, const DetTab& T, double nu, const double w[][SYS == SYS_EULER ? 3 : 1],
                                          double q[][M + 1][SYS == SYS_EULER ? 3 : 1], int it0, int it1)
{
  constexpr int n = M + 1, C = SYS == SYS_EULER ? 3 : 1;
  for (int it = it0; it < it1; ++it) {
    double f[n][n][C];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int l = 0; l < n; ++l) {
        if (SYS == SYS_EULER && !admissible(a.ph.gamma, q[k][l][0], q[k][l][1], q[k][l][2])) ok = false;
        phys_flux<SYS>(a.ph, q[k][l], f[k][l]);
      }
    if (!ok) return -1;
    // q_kl = T^{-1} (phi(0) w_k - nu diag(w) df_k) = Te w_k - nu Tw df_k.  The
    // largest update and value are maxima of non-negative doubles, taken on
    // their bit patterns (integer max, the same order) off the FP64 pipe.
    long long diff = 0, scale = 0;
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int c = 0; c < C; ++c) {
        double df[n];
#pragma unroll
        for (int l = 0; l < n; ++l) {
          double acc = 0.0;
#pragma unroll
          for (int aa = 0; aa < n; ++aa) acc += T.D[k][aa] * f[aa][l][c];
          df[l] = nu * acc;
        }
#pragma unroll
        for (int l = 0; l < n; ++l) {
          double v = T.Te[l] * w[k][c];
#pragma unroll
          for (int bb = 0; bb < n; ++bb) v -= T.Tw[l][bb] * df[bb];
          diff = max(diff, __double_as_longlong(v - q[k][l][c]) & 0x7fffffffffffffffll);
          scale = max(scale, __double_as_longlong(v) & 0x7fffffffffffffffll);
          q[k][l][c] = v;
        }
      }
    if (__longlong_as_double(diff) <= 1e-13 * __longlong_as_double(scale)) return 1;
  }
  return 0;
}

// Edge values of cell gi from its converged nodal values (or, after an
// inadmissible nodal state, its cell average, unevolved).
template <int SYS, int M>
__device__ __forceinline__ void det_finish(const StepArgs& a, const DetTab& T, long long gi, int d, bool ok,
                                           const double q[][M + 1][SYS == SYS_EULER ? 3 : 1], double* ed)
{
  constexpr int n = M + 1, C = SYS == SYS_EULER ? 3 : 1;
  if (SYS == SYS_EULER && ok) {
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int l = 0; l < n; ++l)
        if (!admissible(a.ph.gamma, q[k][l][0], q[k][l][1], q[k][l][2])) ok = false;
  }
  if (!ok) {
    // an inadmissible predictor state: the cell keeps its average, unevolved
    atomicAdd(a.stats + (long long)d * NSTATS + S_RECON_FB, 1ull);
#pragma unroll
    for (int side = 0; side < 2; ++side)
#pragma unroll
      for (int g = 0; g <= n; ++g)
#pragma unroll
        for (int c = 0; c < C; ++c) ed[det_idx(M, C, a.ncell, side, g, c, gi)] = a.avg[c * a.ncell + gi];
    return;
  }
#pragma unroll
  for (int side = 0; side < 2; ++side) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
      for (int g = 0; g < n; ++g) {
        double v = 0.0;
#pragma unroll
        for (int aa = 0; aa < n; ++aa) v += (side ? T.e1[aa] : T.e0[aa]) * q[aa][g][c];
        ed[det_idx(M, C, a.ncell, side, g, c, gi)] = v;
      }
      double v = 0.0;
#pragma unroll
      for (int aa = 0; aa < n; ++aa)
#pragma unroll
        for (int bb = 0; bb < n; ++bb) v += (side ? T.e1[aa] : T.e0[aa]) * T.e1[bb] * q[aa][bb][c];
      ed[det_idx(M, C, a.ncell, side, n, c, gi)] = v;
    }
  }
}

// Phase 1, one thread per cell: reconstruction (GRPrec or GRPrecNL), the
// first DET_PHASE1 Picard iterations, edge values or a place on the list.
template <int SYS, int M, bool NL>
__global__ void __launch_bounds__(128) k_det_predict(StepArgs a, double* __restrict__ ed, DetResume r)
{
  constexpr int n = M + 1, C = SYS == SYS_EULER ? 3 : 1;
  const long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= a.ncell) return;
  const int d = a.cell_dom[gi];
  const DomStep& ds = a.ds[d];
  if (!ds.active) return;
  const long long c0 = a.cell_off[d], i0 = a.if_off[d];
  const int N = (int)(a.cell_off[d + 1] - c0);
  const int i = (int)(gi - c0);
  const DetTab& T = c_det[M - 1];
  double b[3][5];
  bool fb = false;
  cell_coeffs<SYS, M, NL>(a, c0, i0, N, a.bc[d], i, b, fb);
  if (fb) atomicAdd(a.stats + (long long)d * NSTATS + S_RECON_FB, 1ull);
  double w[n][C], q[n][n][C];
#pragma unroll
  for (int k = 0; k < n; ++k) {
    const double xi = T.x[k] - 0.5, x2 = xi * xi;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const double v = b[c][0] + b[c][1] * xi + b[c][2] * (x2 - 1.0 / 12.0) + b[c][3] * x2 * xi +
                       b[c][4] * (x2 * x2 - 1.0 / 80.0);
      w[k][c] = v;
#pragma unroll
      for (int l = 0; l < n; ++l) q[k][l][c] = v;
    }
  }
  const double nu = ds.nu;
  int st, it0 = 0, it1 = DET_PHASE1;
  while (true) {                     // one Picard call site (twice at most: the list may be full)
    st = det_picard<SYS, M>(a, T, nu, w, q, it0, it1);
    if (st != 0 || it1 == DET_MAXIT) break;
    const int slot = atomicAdd(r.count, 1);
    if (slot < r.cap) {
      double* z = r.state + (long long)slot * ((n + n * n) * C);
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int c = 0; c < C; ++c) z[k * C + c] = w[k][c];
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int l = 0; l < n; ++l)
#pragma unroll
          for (int c = 0; c < C; ++c) z[n * C + (k * n + l) * C + c] = q[k][l][c];
      r.list[slot] = (int)gi;
      return;
    }
    it0 = DET_PHASE1;                // the list is full: go on here
    it1 = DET_MAXIT;
  }
  det_finish<SYS, M>(a, T, gi, d, st >= 0, q, ed);
}

// Phase 2: the listed cells resume their iteration, one thread per slot.
template <int SYS, int M>
__global__ void __launch_bounds__(128) k_det_resume(StepArgs a, double* __restrict__ ed, DetResume r)
{
  constexpr int n = M + 1, C = SYS == SYS_EULER ? 3 : 1;
  const int cnt = *r.count < r.cap ? *r.count : r.cap;
  const DetTab& T = c_det[M - 1];
  for (int k0 = blockIdx.x * blockDim.x + threadIdx.x; k0 < cnt; k0 += gridDim.x * blockDim.x) {
    const long long gi = r.list[k0];
    const int d = a.cell_dom[gi];
    const double* z = r.state + (long long)k0 * ((n + n * n) * C);
    double w[n][C], q[n][n][C];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int c = 0; c < C; ++c) w[k][c] = z[k * C + c];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int l = 0; l < n; ++l)
#pragma unroll
        for (int c = 0; c < C; ++c) q[k][l][c] = z[n * C + (k * n + l) * C + c];
    const int st = det_picard<SYS, M>(a, T, a.ds[d].nu, w, q, DET_PHASE1, DET_MAXIT);
    det_finish<SYS, M>(a, T, gi, d, st >= 0, q, ed);
  }
}

// Riemann problems of the evolved edge values at interface gj: the flux
// (Gauss quadrature over the M+1 time nodes) and the interface datum (the
// state at the end of the step).  One thread per interface, full warps at the
// statistics.
template <int SYS, int M, bool G75>
__global__ void __launch_bounds__(128) k_det_flux(StepArgs a, const double* __restrict__ ed)
{
  constexpr int n = M + 1, C = SYS == SYS_EULER ? 3 : 1;
  const long long gj = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned st[5] = {0u, 0u, 0u, 0u, 0u};   // newton sum, newton max, RS calls, first order
  int d = -1;
  if (gj < a.nif) {
    d = a.if_dom[gj];
    const DomStep& ds = a.ds[d];
    if (!ds.active) {
#pragma unroll
      for (int c = 0; c < C; ++c) a.ifc_new[c * a.nif + gj] = a.ifc[c * a.nif + gj];
    } else {
      const long long i0 = a.if_off[d], c0 = a.cell_off[d];
      const int j = (int)(gj - i0), N = (int)(a.cell_off[d + 1] - c0), bc = a.bc[d];
      int cl, cr;
      if (bc == 0) { cl = j == 0 ? N - 1 : j - 1; cr = j; }
      else { cl = j - 1; cr = j == N ? -1 : j; }
      a.low[gj] = 0;
      const DetTab& T = c_det[M - 1];
      double Fs[3] = {0.0, 0.0, 0.0}, gnew[3] = {0.0, 0.0, 0.0};
      bool fo = false;
      int iters = 0;
      for (int g = 0; g <= n && !fo; ++g) {
        double QL[3] = {0.0, 0.0, 0.0}, QR[3] = {0.0, 0.0, 0.0}, Q0[3], F[3];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          QL[c] = cl < 0 ? a.avg[c * a.ncell + c0] : ed[det_idx(M, C, a.ncell, 1, g, c, c0 + cl)];
          QR[c] = cr < 0 ? a.avg[c * a.ncell + c0 + N - 1] : ed[det_idx(M, C, a.ncell, 0, g, c, c0 + cr)];
        }
        if (SYS == SYS_ADV) {
          const double lam = a.ph.lambda;
          Q0[0] = lam > 0.0 ? QL[0] : (lam < 0.0 ? QR[0] : 0.5 * (QL[0] + QR[0]));
        } else {
          const double gm = a.ph.gamma;
          if (!admissible(gm, QL[0], QL[1], QL[2]) || !admissible(gm, QR[0], QR[1], QR[2])) { fo = true; break; }
          Prim W;
          int it = 0;
          const int rs = riemann_state<G75>(a.ph, QL, QR, false, Q0, W, it);
          iters += it;
          st[2] += 1;
          if (rs != ST_OK) { fo = true; break; }
        }
        if (g < n) {
          phys_flux<SYS>(a.ph, Q0, F);
#pragma unroll
          for (int c = 0; c < C; ++c) Fs[c] += T.w[g] * F[c];
        } else {
#pragma unroll
          for (int c = 0; c < C; ++c) gnew[c] = Q0[c];
        }
      }
      if (fo) {
        int it2 = 0;
        const int r = first_order<G75>(a, c0, N, bc, j, Fs, gnew, it2);
        iters += it2;
        st[2] += 1;
        st[3] = 1;
        a.low[gj] = 1;
        if (r != ST_OK) atomicExch(a.fail + d, r);
      }
      st[0] = (unsigned)iters;
      st[1] = (unsigned)iters;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        a.flux[c * a.nif + gj] = Fs[c];
        a.ifc_new[c * a.nif + gj] = gnew[c];
      }
    }
  }
  __syncwarp();
  if (SYS == SYS_EULER) {
    warp_stat_add(a.stats, d, S_NEWTON_SUM, st[0]);
    warp_stat_max(a.stats, d, S_NEWTON_MAX, st[1]);
    warp_stat_add(a.stats, d, S_RS_CALLS, st[2]);
    warp_stat_add(a.stats, d, S_LOW, st[3]);
  }
}

// The resume area follows the edge values in the same buffer (det_doubles).
long long det_cap(long long ncell) { return ncell / 4 + 1024; }

DetResume det_resume(int M, int C, long long ncell, double* ed)
{
  const long long n = M + 1;
  DetResume r;
  r.cap = (int)det_cap(ncell);
  r.state = ed + (long long)det_doubles_per_cell(M, C) * ncell;
  r.list = reinterpret_cast<int*>(r.state + (long long)r.cap * (n + n * n) * C);
  r.count = r.list + r.cap;
  return r;
}

template <int SYS, int M, bool NL>
cudaError_t predict_launch(const StepArgs& a, double* ed, cudaStream_t s)
{
  constexpr int C = SYS == SYS_EULER ? 3 : 1;
  const DetResume r = det_resume(M, C, a.ncell, ed);
  cudaError_t e = cudaMemsetAsync(r.count, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_det_predict<SYS, M, NL><<<(unsigned)((a.ncell + 127) / 128), 128, 0, s>>>(a, ed, r);
  // one thread per slot of the list (its capacity fixes the grid, so a
  // captured graph serves every step; blocks past the count exit at once):
  // the listed cells iterate side by side, not one after another
  k_det_resume<SYS, M><<<(unsigned)((r.cap + 127) / 128), 128, 0, s>>>(a, ed, r);
  return cudaGetLastError();
}

template <int SYS, int M>
cudaError_t flux_launch(const StepArgs& a, const double* ed, cudaStream_t s)
{
  const unsigned g = (unsigned)((a.nif + 127) / 128);
  if (SYS == SYS_EULER && a.ph.gamma == 1.4) k_det_flux<SYS, M, true><<<g, 128, 0, s>>>(a, ed);
  else k_det_flux<SYS, M, false><<<g, 128, 0, s>>>(a, ed);
  return cudaGetLastError();
}

}  // namespace

int det_prepare(int device) { return det_tables(device); }

size_t det_doubles_per_cell(int M, int C) { return (size_t)2 * (M + 2) * C; }

size_t det_doubles(int M, int C, long long ncell)
{
  const long long n = M + 1, cap = det_cap(ncell);
  // edge values, resume states, then the list and its counter as ints
  return (size_t)(det_doubles_per_cell(M, C) * ncell + cap * (n + n * n) * C + (cap + 2) / 2 + 1);
}

cudaError_t launch_det_step(const StepArgs& a, double* ed, cudaStream_t s)
{
  const bool nl = a.recon == GRP_RECON_GRPRECNL;
  cudaError_t e = cudaSuccess;
#define GRP_DET_CASE(SYS, MM)                                                                  \
  case MM:                                                                                     \
    e = nl ? predict_launch<SYS, MM, true>(a, ed, s) : predict_launch<SYS, MM, false>(a, ed, s); \
    if (e == cudaSuccess) e = flux_launch<SYS, MM>(a, ed, s);                                   \
    break;
  if (a.sys == SYS_ADV) {
    switch (a.M) { GRP_DET_CASE(SYS_ADV, 1) GRP_DET_CASE(SYS_ADV, 2) GRP_DET_CASE(SYS_ADV, 3) GRP_DET_CASE(SYS_ADV, 4)
      default: return cudaErrorInvalidValue; }
  } else {
    switch (a.M) { GRP_DET_CASE(SYS_EULER, 1) GRP_DET_CASE(SYS_EULER, 2) GRP_DET_CASE(SYS_EULER, 3)
      GRP_DET_CASE(SYS_EULER, 4) default: return cudaErrorInvalidValue; }
  }
#undef GRP_DET_CASE
  return e;
}

}  // namespace grp
