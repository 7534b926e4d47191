// Device arithmetic of the FV+GRPrec step (arXiv 2602.21911), FP64 throughout.
//
// Scaled variables: every interface GRP is solved in X = x/dx, T = tau/dx.
// The equations are invariant under this scaling, so the Taylor coefficients
// of a reconstructed polynomial in xi = (x - x_i)/dx feed the Cauchy-Kovalevskaya
// recursion directly, with no powers of dx, and tau/dx = nu (1 + s)/2 at a
// Gauss node s.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#ifndef GRP_HD
#define GRP_HD __host__ __device__
#endif

namespace grp {

enum { SYS_ADV = 0, SYS_EULER = 1 };
enum { ST_OK = 0, ST_NO_CONV = 1, ST_VACUUM = 2, ST_NONPHYS = 3 };

// Speeds within TIE x (wave-speed scale) of zero count as zero when a sign
// picks a side (contact sampling, upwinding of derivative Riemann problems):
// a stationary contact must not be decided by rounding noise.
constexpr double TIE = 1e-10;

struct Phys {
  double lambda, gamma;
  double rtol;
  int max_iter;
  int guess;  // 0 PVRS, 1 TRRS, 2 learned
};

// ---------------------------------------------------------------------------
// Section 3.1, GRPrec: closed forms of the four constrained fits in the
// zero-mean basis phi_1 = xi, phi_2 = xi^2 - 1/12, phi_3 = xi^3,
// phi_4 = xi^4 - 1/80 (each has zero cell average, so conservation in cell i
// holds by construction).  Degrees 1 and 3 are the least-squares minimisers
// (normal equations solved by hand), degrees 2 and 4 the interpolants.
// Output: Taylor coefficients of p at xi = -1/2 (tm) and xi = +1/2 (tp),
// t_a = p^{(a)}(xi0)/a!.
// ---------------------------------------------------------------------------
template <int M>
GRP_HD __forceinline__ void grprec_coeffs(double qm, double q0, double qp, double gL, double gR,
                                              double b[5])
{
  b[0] = q0; b[1] = b[2] = b[3] = b[4] = 0.0;
  const double dg = gR - gL, sg = gL + gR, dq = qp - qm;
  if (M <= 2) b[1] = dg;
  if (M == 2) b[2] = 3.0 * (sg - 2.0 * q0);
  if (M >= 3) {
    b[1] = (10.0 * dg - dq) * 0.125;
    b[3] = 0.5 * dq - dg;
  }
  if (M == 3) b[2] = 3.0 * (sg - 14.0 * q0 + 6.0 * (qm + qp)) * (1.0 / 37.0);
  if (M == 4) {
    const double sq = qm + qp;
    b[2] = (30.0 * sg - 58.0 * q0 - sq) * 0.125;
    b[4] = -5.0 * (6.0 * sg - 10.0 * q0 - sq) * (1.0 / 12.0);
  }
}

// Taylor coefficients at the right edge (side = +1) or left edge (side = -1).
template <int M>
GRP_HD __forceinline__ void edge_taylor(const double b[5], double side, double t[M + 1])
{
  // p(xi) = b0 + b1 xi + b2 (xi^2 - 1/12) + b3 xi^3 + b4 (xi^4 - 1/80)
  t[0] = b[0] + side * 0.5 * b[1] + b[2] * (1.0 / 6.0) + side * 0.125 * b[3] + b[4] * 0.05;
  if (M >= 1) t[1] = b[1] + side * b[2] + 0.75 * b[3] + side * 0.5 * b[4];
  if (M >= 2) t[2] = b[2] + side * 1.5 * b[3] + 1.5 * b[4];
  if (M >= 3) t[3] = b[3] + side * 2.0 * b[4];
  if (M >= 4) t[4] = b[4];
}

// ---------------------------------------------------------------------------
// Ideal gas (Section 4.3)
// ---------------------------------------------------------------------------
struct Prim { double r, u, p; };

GRP_HD __forceinline__ Prim to_prim(double g, double r, double m, double E)
{
  Prim w;
  w.r = r;
  w.u = m / r;
  w.p = (g - 1.0) * (E - 0.5 * m * w.u);
  return w;
}

GRP_HD __forceinline__ void to_cons(double g, Prim w, double Q[3])
{
  Q[0] = w.r;
  Q[1] = w.r * w.u;
  Q[2] = w.p / (g - 1.0) + 0.5 * w.r * w.u * w.u;
}

GRP_HD __forceinline__ bool admissible(double g, double r, double m, double E)
{
  if (!(r > 0.0)) return false;
  const double p = (g - 1.0) * (E - 0.5 * m * (m / r));
  return p > 0.0;
}

GRP_HD __forceinline__ void euler_flux(double g, double r, double m, double E, double F[3])
{
  const double u = m / r;
  const double p = (g - 1.0) * (E - 0.5 * m * u);
  F[0] = m;
  F[1] = m * u + p;
  F[2] = u * (E + p);
}

// ---------------------------------------------------------------------------
// Exact Riemann solver of the ideal gas: Newton on the star pressure.
// ---------------------------------------------------------------------------
GRP_HD __forceinline__ void pressure_fn(double g, double p, Prim K, double c, double& f, double& df)
{
  if (p > K.p) {
    const double A = 2.0 / ((g + 1.0) * K.r);
    const double B = (g - 1.0) / (g + 1.0) * K.p;
    const double s = sqrt(A / (p + B));
    f = (p - K.p) * s;
    df = s * (1.0 - (p - K.p) / (2.0 * (B + p)));
  } else {
    const double ratio = p / K.p;
    f = 2.0 * c / (g - 1.0) * (pow(ratio, (g - 1.0) / (2.0 * g)) - 1.0);
    df = 1.0 / (K.r * c) * pow(ratio, -(g + 1.0) / (2.0 * g));
  }
}

// Returns ST_OK / ST_NO_CONV / ST_VACUUM.  p0 > 0 is used as the start when
// given (learned guess), otherwise PVRS or TRRS per ph.guess.
static GRP_HD int star_pressure(const Phys& ph, Prim L, Prim R, double cL, double cR, double p0,
                             double& ps, double& us, int& iters)
{
  const double g = ph.gamma;
  const double du = R.u - L.u;
  iters = 0;
  if (2.0 * (cL + cR) / (g - 1.0) <= du) return ST_VACUUM;
  const double pfloor = 1e-14 * fmax(L.p, R.p);
  double p;
  if (p0 > 0.0 && isfinite(p0)) {
    p = p0;
  } else if (ph.guess == 1) {
    const double z = (g - 1.0) / (2.0 * g);
    const double num = cL + cR - 0.5 * (g - 1.0) * du;
    const double den = cL * pow(L.p, -z) + cR * pow(R.p, -z);
    p = pow(num / den, 1.0 / z);
  } else {
    const double ppv = 0.5 * (L.p + R.p) - 0.125 * du * (L.r + R.r) * (cL + cR);
    p = fmax(ppv, pfloor);
  }
  if (!(p > pfloor)) p = pfloor;
  bool conv = false;
  int it = 0;
  while (it < ph.max_iter) {
    double fL, dfL, fR, dfR;
    pressure_fn(g, p, L, cL, fL, dfL);
    pressure_fn(g, p, R, cR, fR, dfR);
    double step = -(fL + fR + du) / (dfL + dfR);
    double pn = p + step;
    for (int h = 0; h < 64 && !(pn > 0.0); ++h) { step *= 0.5; pn = p + step; }
    ++it;
    const double change = 2.0 * fabs(pn - p) / (pn + p);
    p = pn;
    if (conv) break;
    if (change < ph.rtol) conv = true;
  }
  iters = it;
  if (!conv) return ST_NO_CONV;
  double fL, dfL, fR, dfR;
  pressure_fn(g, p, L, cL, fL, dfL);
  pressure_fn(g, p, R, cR, fR, dfR);
  ps = p;
  us = 0.5 * (L.u + R.u) + 0.5 * (fR - fL);
  return ST_OK;
}

// Left of the contact when u* >= 0, sampled on the ray x/t = 0.  A contact
// speed within TIE of the sound-speed scale is stationary and goes left.
static GRP_HD Prim sample_zero(double g, Prim L, Prim R, double cL, double cR, double ps, double us)
{
  const double g1 = (g - 1.0) / (2.0 * g), g6 = (g - 1.0) / (g + 1.0);
  if (us >= -TIE * (cL + cR)) {
    const double ratio = ps / L.p;
    if (ps > L.p) {
      const double S = L.u - cL * sqrt((g + 1.0) / (2.0 * g) * ratio + g1);
      if (S >= 0.0) return L;
      return Prim{L.r * (ratio + g6) / (g6 * ratio + 1.0), us, ps};
    }
    if (L.u - cL >= 0.0) return L;
    const double cs = cL * pow(ratio, g1);
    if (us - cs < 0.0) return Prim{L.r * pow(ratio, 1.0 / g), us, ps};
    const double c0 = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * L.u);
    return Prim{L.r * pow(c0 / cL, 2.0 / (g - 1.0)), c0, L.p * pow(c0 / cL, 2.0 * g / (g - 1.0))};
  }
  const double ratio = ps / R.p;
  if (ps > R.p) {
    const double S = R.u + cR * sqrt((g + 1.0) / (2.0 * g) * ratio + g1);
    if (S <= 0.0) return R;
    return Prim{R.r * (ratio + g6) / (g6 * ratio + 1.0), us, ps};
  }
  if (R.u + cR <= 0.0) return R;
  const double cs = cR * pow(ratio, g1);
  if (us + cs > 0.0) return Prim{R.r * pow(ratio, 1.0 / g), us, ps};
  const double c0 = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * R.u);
  return Prim{R.r * pow(c0 / cR, 2.0 / (g - 1.0)), -c0, R.p * pow(c0 / cR, 2.0 * g / (g - 1.0))};
}

// Vacuum-generating data: two rarefactions around a vacuum, sampled at x/t = 0.
static GRP_HD Prim sample_vacuum_zero(double g, Prim L, Prim R, double cL, double cR)
{
  if (L.u - cL >= 0.0) return L;
  if (L.u + 2.0 * cL / (g - 1.0) > 0.0) {
    const double c0 = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * L.u);
    return Prim{L.r * pow(c0 / cL, 2.0 / (g - 1.0)), c0, L.p * pow(c0 / cL, 2.0 * g / (g - 1.0))};
  }
  if (R.u + cR <= 0.0) return R;
  if (R.u - 2.0 * cR / (g - 1.0) < 0.0) {
    const double c0 = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * R.u);
    return Prim{R.r * pow(c0 / cR, 2.0 / (g - 1.0)), -c0, R.p * pow(c0 / cR, 2.0 * g / (g - 1.0))};
  }
  return Prim{0.0, 0.0, 0.0};
}

// Conserved Godunov state at x/t = 0 of conserved data QL | QR.
// allow_vacuum: vacuum data are sampled and ST_VACUUM returned with Q valid.
static GRP_HD int riemann_state(const Phys& ph, const double QL[3], const double QR[3], double p0,
                             bool allow_vacuum, double Q[3], int& iters)
{
  const double g = ph.gamma;
  const Prim L = to_prim(g, QL[0], QL[1], QL[2]);
  const Prim R = to_prim(g, QR[0], QR[1], QR[2]);
  const double cL = sqrt(g * L.p / L.r), cR = sqrt(g * R.p / R.r);
  double ps = 0.0, us = 0.0;
  const int st = star_pressure(ph, L, R, cL, cR, p0, ps, us, iters);
  if (st == ST_VACUUM && allow_vacuum) {
    to_cons(g, sample_vacuum_zero(g, L, R, cL, cR), Q);
    return ST_VACUUM;
  }
  if (st != ST_OK) return st;
  to_cons(g, sample_zero(g, L, R, cL, cR, ps, us), Q);
  return ST_OK;
}

// ---------------------------------------------------------------------------
// Derivative Riemann problem (Toro-Titarev, Section 2): the linear system
// d_t D + A(Q0) d_x D = 0 with data DL | DR; Godunov value at x/t = 0 by
// upwinding in the eigenbasis of A(Q0) (an eigenvalue within TIE of zero
// averages the two sides).
// Eigenvectors of the ideal-gas Jacobian in conserved variables, with
// H = (E + p)/rho, b1 = (g-1)/c^2, b2 = b1 u^2/2.
// ---------------------------------------------------------------------------
struct Eig {
  double u, c, H, b1, b2, ic, tie;
  double lam[3];
};

GRP_HD __forceinline__ Eig make_eig(double g, const double Q0[3])
{
  Eig e;
  const Prim w = to_prim(g, Q0[0], Q0[1], Q0[2]);
  e.u = w.u;
  e.c = sqrt(g * w.p / w.r);
  e.H = (Q0[2] + w.p) / w.r;
  e.ic = 1.0 / e.c;
  e.b1 = (g - 1.0) * e.ic * e.ic;
  e.b2 = 0.5 * e.u * e.u * e.b1;
  e.lam[0] = e.u - e.c; e.lam[1] = e.u; e.lam[2] = e.u + e.c;
  e.tie = TIE * (fabs(e.u) + e.c);
  return e;
}

GRP_HD __forceinline__ void char_proj(const Eig& e, const double D[3], double w[3])
{
  // rows of R^{-1}
  const double uc = e.u * e.ic;
  w[0] = 0.5 * ((e.b2 + uc) * D[0] - (e.b1 * e.u + e.ic) * D[1] + e.b1 * D[2]);
  w[1] = (1.0 - e.b2) * D[0] + e.b1 * e.u * D[1] - e.b1 * D[2];
  w[2] = 0.5 * ((e.b2 - uc) * D[0] - (e.b1 * e.u - e.ic) * D[1] + e.b1 * D[2]);
}

GRP_HD __forceinline__ void deriv_rp(const Eig& e, const double DL[3], const double DR[3], double D[3])
{
  double wl[3], wr[3], w[3];
  char_proj(e, DL, wl);
  char_proj(e, DR, wr);
#pragma unroll
  for (int j = 0; j < 3; ++j)
    w[j] = e.lam[j] > e.tie ? wl[j] : (e.lam[j] < -e.tie ? wr[j] : 0.5 * (wl[j] + wr[j]));
  D[0] = w[0] + w[1] + w[2];
  D[1] = (e.u - e.c) * w[0] + e.u * w[1] + (e.u + e.c) * w[2];
  D[2] = (e.H - e.u * e.c) * w[0] + 0.5 * e.u * e.u * w[1] + (e.H + e.u * e.c) * w[2];
}

// ---------------------------------------------------------------------------
// Cauchy-Kovalevskaya by truncated bivariate series (total degree M) in
// scaled variables: Q(X,T) = sum q[a][b] X^a T^b with
// q[a][b+1] = -(a+1)/(b+1) F[a+1][b]; F's series from series products and
// the series quotient u = m / rho.  Triangular storage idx(a,b).
// ---------------------------------------------------------------------------
template <int M>
struct Tri {
  static constexpr int N = (M + 1) * (M + 2) / 2;
  __host__ __device__ static constexpr int idx(int a, int b) { return (a + b) * (a + b + 1) / 2 + b; }
};

// In: q0[c][idx(a,0)] filled for a = 0..M (others ignored).  Out: s[c][b] = q[0][b].
template <int M>
GRP_HD __forceinline__ void ck_euler(double g, double rho[Tri<M>::N], double m[Tri<M>::N],
                                         double E[Tri<M>::N], double s[3][M + 1])
{
  using T = Tri<M>;
  double u[T::N], mu[T::N], Ep[T::N], F1[T::N], F2[T::N];
  const double irho = 1.0 / rho[0];
  const double gm1 = g - 1.0;
#pragma unroll
  for (int b = 0; b < M; ++b) {
#pragma unroll
    for (int a = 0; a + b <= M; ++a) {
      const int k = T::idx(a, b);
      double acc = m[k];
#pragma unroll
      for (int i = 0; i <= a; ++i)
#pragma unroll
        for (int j = 0; j <= b; ++j)
          if (i || j) acc -= rho[T::idx(i, j)] * u[T::idx(a - i, b - j)];
      u[k] = acc * irho;
      double mm = 0.0;
#pragma unroll
      for (int i = 0; i <= a; ++i)
#pragma unroll
        for (int j = 0; j <= b; ++j) mm += m[T::idx(i, j)] * u[T::idx(a - i, b - j)];
      mu[k] = mm;
      const double p = gm1 * (E[k] - 0.5 * mm);
      Ep[k] = E[k] + p;
      F1[k] = mm + p;
      double f3 = 0.0;
#pragma unroll
      for (int i = 0; i <= a; ++i)
#pragma unroll
        for (int j = 0; j <= b; ++j) f3 += u[T::idx(i, j)] * Ep[T::idx(a - i, b - j)];
      F2[k] = f3;
    }
#pragma unroll
    for (int a = 0; a + b + 1 <= M; ++a) {
      const double f = -double(a + 1) / double(b + 1);
      const int src = T::idx(a + 1, b), dst = T::idx(a, b + 1);
      rho[dst] = f * m[src];
      m[dst] = f * F1[src];
      E[dst] = f * F2[src];
    }
  }
#pragma unroll
  for (int b = 0; b <= M; ++b) {
    s[0][b] = rho[T::idx(0, b)];
    s[1][b] = m[T::idx(0, b)];
    s[2][b] = E[T::idx(0, b)];
  }
}

// Gauss-Legendre rule with G = ceil((M+1)/2) points on [0, 1]: nodes
// (1 + s)/2 and weights summing to 1.
template <int M>
struct Gauss {
  static constexpr int G = (M + 2) / 2;
  GRP_HD static __forceinline__ double node(int a)
  {
    if (G == 1) return 0.5;
    if (G == 2) return a == 0 ? 0.5 - 0.28867513459481288225 : 0.5 + 0.28867513459481288225;
    return a == 0 ? 0.5 - 0.38729833462074168852 : (a == 1 ? 0.5 : 0.5 + 0.38729833462074168852);
  }
  GRP_HD static __forceinline__ double weight(int a)
  {
    if (G == 1) return 1.0;
    if (G == 2) return 0.5;
    return a == 1 ? 8.0 / 18.0 : 5.0 / 18.0;
  }
};

// ---------------------------------------------------------------------------
// One GRP_M at an interface (Toro-Titarev structure, Section 2) and its flux
// time integral over [0, dt] (numerical flux, Section 2), in scaled
// variables: t[c][k] are the Taylor coefficients p^{(k)}/k! of the
// reconstructions at the interface, nu = dt/dx.  The interface datum for the
// next step is the series at tau = dt.
// ---------------------------------------------------------------------------
template <int M>
GRP_HD __forceinline__ void grp_adv(double lam, double nu, const double tL[M + 1], const double tR[M + 1],
                                    double& F, double& gnew)
{
  double s[M + 1];
#pragma unroll
  for (int k = 0; k <= M; ++k) s[k] = lam > 0.0 ? tL[k] : (lam < 0.0 ? tR[k] : 0.5 * (tL[k] + tR[k]));
  // CK for q_t + lam q_x = 0: q[0][b] = (-lam)^b q[b][0]
  double sc = 1.0;
#pragma unroll
  for (int k = 0; k <= M; ++k) { s[k] *= sc; sc *= -lam; }
  double acc = 0.0;
#pragma unroll
  for (int al = 0; al < Gauss<M>::G; ++al) {
    const double T = nu * Gauss<M>::node(al);
    double v = s[M];
#pragma unroll
    for (int k = M - 1; k >= 0; --k) v = v * T + s[k];
    acc += Gauss<M>::weight(al) * v;
  }
  F = lam * acc;
  double v = s[M];
#pragma unroll
  for (int k = M - 1; k >= 0; --k) v = v * nu + s[k];
  gnew = v;
}

// Returns ST_OK, or the failure of the leading Riemann problem (the caller
// then takes the first-order flux).  truncated: a state of the series at a
// Gauss node or at dt was inadmissible, so the series was cut to its
// leading term.
template <int M>
GRP_HD __forceinline__ int grp_euler(const Phys& ph, double nu, const double tL[3][M + 1],
                                     const double tR[3][M + 1], double F[3], double gnew[3], int& iters,
                                     bool& truncated)
{
  const double g = ph.gamma;
  const double QL[3] = {tL[0][0], tL[1][0], tL[2][0]}, QR[3] = {tR[0][0], tR[1][0], tR[2][0]};
  double Q0[3];
  truncated = false;
  const int st = riemann_state(ph, QL, QR, 0.0, false, Q0, iters);
  if (st != ST_OK) return st;
  using T = Tri<M>;
  double rho[T::N], m[T::N], E[T::N];
  rho[0] = Q0[0]; m[0] = Q0[1]; E[0] = Q0[2];
  {
    const Eig e = make_eig(g, Q0);
#pragma unroll
    for (int k = 1; k <= M; ++k) {
      const double DL[3] = {tL[0][k], tL[1][k], tL[2][k]}, DR[3] = {tR[0][k], tR[1][k], tR[2][k]};
      double D[3];
      deriv_rp(e, DL, DR, D);
      rho[T::idx(k, 0)] = D[0]; m[T::idx(k, 0)] = D[1]; E[T::idx(k, 0)] = D[2];
    }
  }
  double s[3][M + 1];
  ck_euler<M>(g, rho, m, E, s);
  // states at the Gauss nodes and at tau = dt
  double Qg[Gauss<M>::G + 1][3];
  bool ok = true;
#pragma unroll
  for (int al = 0; al <= Gauss<M>::G; ++al) {
    const double Tn = al < Gauss<M>::G ? nu * Gauss<M>::node(al) : nu;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double v = s[c][M];
#pragma unroll
      for (int k = M - 1; k >= 0; --k) v = v * Tn + s[c][k];
      Qg[al][c] = v;
    }
    ok = ok && admissible(g, Qg[al][0], Qg[al][1], Qg[al][2]);
  }
  if (!ok) {
    truncated = true;
#pragma unroll
    for (int al = 0; al <= Gauss<M>::G; ++al) { Qg[al][0] = Q0[0]; Qg[al][1] = Q0[1]; Qg[al][2] = Q0[2]; }
  }
  F[0] = F[1] = F[2] = 0.0;
#pragma unroll
  for (int al = 0; al < Gauss<M>::G; ++al) {
    double Fa[3];
    euler_flux(g, Qg[al][0], Qg[al][1], Qg[al][2], Fa);
    const double w = Gauss<M>::weight(al);
    F[0] += w * Fa[0]; F[1] += w * Fa[1]; F[2] += w * Fa[2];
  }
  gnew[0] = Qg[Gauss<M>::G][0]; gnew[1] = Qg[Gauss<M>::G][1]; gnew[2] = Qg[Gauss<M>::G][2];
  return ST_OK;
}

}  // namespace grp
