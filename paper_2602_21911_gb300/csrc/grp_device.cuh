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
  // gamma-dependent constants, computed once on the host (make_phys)
  double gm1, i_gm1, c2_gm1, c2_gp1, gm1_gp1, gm1_2g, gp1_2g, c2g_gm1, i_g, sqrt_c2_gp1, h_gm1;
  // learned Newton guess: FP32 weights (MLP_NPARAM) and input box lo[6], hi[6]
  const float* mlp_w;
  const float* mlp_box;
  int features;          // the learned-guess path for strong data: 0 off; 1 the learned start; 2 harvest
                         // (the records' targets in FP64)
  // source term S(Q) of the balance law (Section 2): 0 none; 1 S = src_k q
  // (advection); 2 S = (0, -src_k rho, -src_k m) (Euler, acceleration -src_k)
  int src;
  double src_k;
};

inline Phys make_phys(double lambda, double gamma, double rtol, int max_iter, int guess)
{
  Phys p;
  p.lambda = lambda; p.gamma = gamma; p.rtol = rtol; p.max_iter = max_iter; p.guess = guess;
  const double g = gamma;
  p.gm1 = g - 1.0;
  p.i_gm1 = 1.0 / (g - 1.0);
  p.c2_gm1 = 2.0 / (g - 1.0);
  p.c2_gp1 = 2.0 / (g + 1.0);
  p.gm1_gp1 = (g - 1.0) / (g + 1.0);
  p.gm1_2g = (g - 1.0) / (2.0 * g);
  p.gp1_2g = (g + 1.0) / (2.0 * g);
  p.c2g_gm1 = 2.0 * g / (g - 1.0);
  p.i_g = 1.0 / g;
  p.sqrt_c2_gp1 = sqrt(2.0 / (g + 1.0));
  p.h_gm1 = 0.5 * (g - 1.0);
  p.mlp_w = nullptr;
  p.mlp_box = nullptr;
  p.features = 0;
  p.src = 0;
  p.src_k = 0.0;
  return p;
}

// ---------------------------------------------------------------------------
// Arithmetic helpers.  FP64 is the scarce pipe on this GPU; seeds come from
// the FP32 special-function unit and are refined by FP64 Newton steps.
// ---------------------------------------------------------------------------
GRP_HD __forceinline__ float f32_log2(float x)
{
#ifdef __CUDA_ARCH__
  return __log2f(x);
#else
  return log2f(x);
#endif
}

GRP_HD __forceinline__ float f32_exp2(float x)
{
#ifdef __CUDA_ARCH__
  return exp2f(x);
#else
  return exp2f(x);
#endif
}

// 1/y to ~1e-14 relative: FP32 reciprocal seed, one FP64 Newton step.  Used
// only for the Newton update of the star pressure, whose next iterate corrects
// any residual of the step.
GRP_HD __forceinline__ double rcp_newton_step(double y)
{
  const float yf = (float)y;
  const float af = fabsf(yf);
  if (!(af > 1e-30f && af < 1e30f)) return 1.0 / y;
  double r = (double)(1.0f / yf);
  const double e = fma(-y, r, 1.0);
  return fma(r, e, r);
}

// 1/y for a positive normal y, correct to about an ulp: the hardware
// reciprocal approximation (rcp.approx.ftz.f64, about 2^-22 relative) and two
// Newton steps r <- r + r (1 - y r), each squaring the relative error.  Half
// the FP64 instructions of a correctly rounded division; used where the result
// feeds further arithmetic, not a comparison with the oracle's rounding.
GRP_HD __forceinline__ double rcp64(double y)
{
#ifdef __CUDA_ARCH__
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(y));
  double e = fma(-y, r, 1.0);
  r = fma(r, e, r);
  e = fma(-y, r, 1.0);
  return fma(r, e, r);
#else
  return 1.0 / y;
#endif
}

// x^(-1/7) for x > 0: FP32 seed 2^(-log2(x)/7), then two FP64 Newton steps on
// w^-7 = x, w <- w (8 - x w^7)/7, each squaring the relative error
// (2^-21 -> 2^-40 -> rounding).  Outside the FP32 normal range: pow.
GRP_HD __forceinline__ double inv_root7(double x)
{
  const float xf = (float)x;
  if (!(xf > 1e-36f && xf < 1e36f)) return pow(x, -1.0 / 7.0);
  double w = (double)f32_exp2(-f32_log2(xf) * (1.0f / 7.0f));
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double w2 = w * w, w4 = w2 * w2;
    const double w7 = w4 * w2 * w;
    w = w * fma(-x, w7, 8.0) * (1.0 / 7.0);
  }
  return w;
}

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

// ---------------------------------------------------------------------------
// Sections 3.3-3.4, GRPrecNL: the convex combination beta_L p_L + beta_C p_C
// + beta_R p_R of the one-sided polynomials and the linear GRPrec one, with
// beta_k = omega_k / sum omega, omega_k = lambda_k / (eps + OI_k)^4,
// eps = 1e-14, lambda_L = lambda_R = 1, lambda_C = 1e9, and
// OI_k = dx * sum_{l<=M} int_{-1/2}^{1/2} (d^l p_k / dxi^l)^2 dxi (the printed
// indicator, dx^{2l} with the measure dx).  Data
// d = {q_{i-1}, q_i, q_{i+1}, g_{i-3/2}, g_{i-1/2}, g_{i+1/2}, g_{i+3/2}}.
// One-sided polynomials in the zero-mean basis (all conserve cell i):
//   degree 1: p_L through g_{i-1/2}, p_R through g_{i+1/2};
//   degree 2: p_L conserves cell i-1 and passes through g_{i+1/2}, p_R
//             conserves cell i+1 and passes through g_{i-1/2};
//   degree 3: both conserve cells i-1, i+1; p_L through g_{i-1/2}, p_R
//             through g_{i+1/2};
//   degree 4: both conserve cells i-1, i+1; p_L through g_{i-1/2}, g_{i-3/2},
//             p_R through g_{i+1/2}, g_{i+3/2}.
// The closed forms solve those square systems in the zero-mean basis.
// ---------------------------------------------------------------------------
constexpr double NL_EPS = 1e-14, NL_LAMBDA_C = 1e9;

template <int M>
GRP_HD __forceinline__ void nl_sides(const double d[7], double bl[5], double br[5])
{
  const double qm = d[0], q0 = d[1], qp = d[2], gmm = d[3], gm = d[4], gp = d[5], gpp = d[6];
  bl[0] = br[0] = q0;
  bl[1] = bl[2] = bl[3] = bl[4] = br[1] = br[2] = br[3] = br[4] = 0.0;
  if (M == 1) {
    bl[1] = 2.0 * (q0 - gm);
    br[1] = 2.0 * (gp - q0);
  } else if (M == 2) {
    bl[1] = 1.5 * gp - 1.25 * q0 - 0.25 * qm;
    bl[2] = 1.5 * gp - 2.25 * q0 + 0.75 * qm;
    br[1] = -1.5 * gm + 1.25 * q0 + 0.25 * qp;
    br[2] = 1.5 * gm - 2.25 * q0 + 0.75 * qp;
  } else if (M == 3) {
    bl[1] = -2.5 * gm + (25.0 / 12.0) * q0 + (1.0 / 3.0) * qm + (1.0 / 12.0) * qp;
    bl[2] = 0.5 * (qm + qp) - q0;
    bl[3] = 2.0 * gm - (5.0 / 3.0) * q0 - (2.0 / 3.0) * qm + (1.0 / 3.0) * qp;
    br[1] = 2.5 * gp - (25.0 / 12.0) * q0 - (1.0 / 12.0) * qm - (1.0 / 3.0) * qp;
    br[2] = bl[2];
    br[3] = -2.0 * gp + (5.0 / 3.0) * q0 - (1.0 / 3.0) * qm + (2.0 / 3.0) * qp;
  } else {
    bl[1] = -3.75 * gm - (5.0 / 12.0) * gmm + (95.0 / 36.0) * q0 + (109.0 / 72.0) * qm + (1.0 / 72.0) * qp;
    bl[2] = -3.75 * gm - 1.25 * gmm + (2.0 / 3.0) * q0 + (97.0 / 24.0) * qm + (7.0 / 24.0) * qp;
    bl[3] = 3.0 * gm + (1.0 / 3.0) * gmm - (19.0 / 9.0) * q0 - (29.0 / 18.0) * qm + (7.0 / 18.0) * qp;
    bl[4] = 2.5 * gm + (5.0 / 6.0) * gmm - (10.0 / 9.0) * q0 - (85.0 / 36.0) * qm + (5.0 / 36.0) * qp;
    br[1] = 3.75 * gp + (5.0 / 12.0) * gpp - (95.0 / 36.0) * q0 - (1.0 / 72.0) * qm - (109.0 / 72.0) * qp;
    br[2] = -3.75 * gp - 1.25 * gpp + (2.0 / 3.0) * q0 + (7.0 / 24.0) * qm + (97.0 / 24.0) * qp;
    br[3] = -3.0 * gp - (1.0 / 3.0) * gpp + (19.0 / 9.0) * q0 - (7.0 / 18.0) * qm + (29.0 / 18.0) * qp;
    br[4] = 2.5 * gp + (5.0 / 6.0) * gpp - (10.0 / 9.0) * q0 + (5.0 / 36.0) * qm - (85.0 / 36.0) * qp;
  }
}

// sum_{l<=M} int_{-1/2}^{1/2} (p^{(l)})^2 dxi for p with zero-mean coefficients b
template <int M>
GRP_HD __forceinline__ double nl_indicator(const double b[5])
{
  double s = b[1] * b[1];
  if (M >= 2) s += (13.0 / 3.0) * b[2] * b[2];
  if (M >= 3) s += 0.5 * b[1] * b[3] + (3129.0 / 80.0) * b[3] * b[3];
  if (M >= 4) s += (21.0 / 5.0) * b[2] * b[4] + (87617.0 / 140.0) * b[4] * b[4];
  return s;
}

// GRPrecNL coefficients b (zero-mean basis) of one scalar component
template <int M>
GRP_HD __forceinline__ void grprec_nl_coeffs(const double d[7], double dx, double b[5])
{
  double p[3][5];
  nl_sides<M>(d, p[0], p[2]);
  grprec_coeffs<M>(d[0], d[1], d[2], d[4], d[5], p[1]);
  // beta_k = (lambda_k / s_k) / sum_j (lambda_j / s_j), s_k = (eps + OI_k)^4,
  // with numerator and denominator multiplied by s_L s_C s_R: products and
  // one reciprocal instead of four divisions (s_k >= eps^4 = 1e-56, so the
  // products of two stay far inside the double range)
  double sk[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double o = NL_EPS + dx * nl_indicator<M>(p[k]);
    const double o2 = o * o;
    sk[k] = o2 * o2;
  }
  const double om[3] = {sk[1] * sk[2], NL_LAMBDA_C * (sk[0] * sk[2]), sk[0] * sk[1]};
  const double is = rcp64(om[0] + om[1] + om[2]);
  b[0] = d[1];
#pragma unroll
  for (int q = 1; q <= 4; ++q) b[q] = q <= M ? (om[0] * p[0][q] + om[1] * p[1][q] + om[2] * p[2][q]) * is : 0.0;
}

// Taylor coefficients at the right edge (side = +1) or left edge (side = -1).
template <int M>
GRP_HD __forceinline__ void edge_taylor(const double b[5], double side, double t[M + 1])
{
  // p(xi) = b0 + b1 xi + b2 (xi^2 - 1/12) + b3 xi^3 + b4 (xi^4 - 1/80).
  // Coefficients above the degree M are zero and their terms are left out
  // (adding a +0.0 is an instruction the compiler must keep).
  double t0 = b[0] + side * 0.5 * b[1];
  if (M >= 2) t0 = t0 + b[2] * (1.0 / 6.0);
  if (M >= 3) t0 = t0 + side * 0.125 * b[3];
  if (M >= 4) t0 = t0 + b[4] * 0.05;
  t[0] = t0;
  if (M >= 1) {
    double t1 = b[1];
    if (M >= 2) t1 = t1 + side * b[2];
    if (M >= 3) t1 = t1 + 0.75 * b[3];
    if (M >= 4) t1 = t1 + side * 0.5 * b[4];
    t[1] = t1;
  }
  if (M >= 2) {
    double t2 = b[2];
    if (M >= 3) t2 = t2 + side * 1.5 * b[3];
    if (M >= 4) t2 = t2 + 1.5 * b[4];
    t[2] = t2;
  }
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

GRP_HD __forceinline__ void to_cons(const Phys& ph, Prim w, double Q[3])
{
  Q[0] = w.r;
  Q[1] = w.r * w.u;
  Q[2] = w.p * ph.i_gm1 + 0.5 * w.r * w.u * w.u;
}

// x > 0 for a double x, exactly (+inf included, NaN excluded).  On the GPU a
// signed-integer test of the bits, off the FP64 pipe: positive doubles order
// as their bit patterns, and negative values have negative patterns.
GRP_HD __forceinline__ bool positive(double x)
{
#ifdef __CUDA_ARCH__
  const long long b = __double_as_longlong(x);
  return b > 0ll && b <= 0x7ff0000000000000ll;
#else
  return x > 0.0;
#endif
}

// More tests on the bits (integer pipe), equal to the IEEE comparisons for
// arguments that are not NaN (-0 included): x >= 0, x <= 0, x < 0, and
// a > b, a < b, max(a, b) for a, b >= 0 (non-negative doubles order as their
// bit patterns do; max(a, b) also when only b is known to be positive).
GRP_HD __forceinline__ bool ge0(double x)
{
#ifdef __CUDA_ARCH__
  const long long b = __double_as_longlong(x);
  return b >= 0ll || b == (long long)0x8000000000000000ull;
#else
  return x >= 0.0;
#endif
}
GRP_HD __forceinline__ bool le0(double x)
{
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x) <= 0ll;
#else
  return x <= 0.0;
#endif
}
GRP_HD __forceinline__ bool lt0(double x)
{
#ifdef __CUDA_ARCH__
  const long long b = __double_as_longlong(x);
  return b < 0ll && b != (long long)0x8000000000000000ull;
#else
  return x < 0.0;
#endif
}
GRP_HD __forceinline__ bool gt_nn(double a, double b)
{
#ifdef __CUDA_ARCH__
  return __double_as_longlong(a) > __double_as_longlong(b);
#else
  return a > b;
#endif
}
GRP_HD __forceinline__ bool finite_positive(double x)
{
#ifdef __CUDA_ARCH__
  const long long b = __double_as_longlong(x);
  return b > 0ll && b < 0x7ff0000000000000ll;
#else
  return x > 0.0 && isfinite(x);
#endif
}
GRP_HD __forceinline__ double max_nn(double a, double b)
{
#ifdef __CUDA_ARCH__
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x > y ? x : y);
#else
  return fmax(a, b);
#endif
}

// rho > 0 and p = (g-1)(E - m^2/(2 rho)) > 0, written without a division:
// rho > 0 and 2 E rho - m^2 > 0 (one fused multiply-add; its sign is that of
// the exact 2 E rho - fl(m^2)), both sign tests on the integer pipe.
GRP_HD __forceinline__ bool admissible(double g, double r, double m, double E)
{
  (void)g;
#ifdef __CUDA_ARCH__
  return positive(r) && positive(fma(E + E, r, -(m * m)));
#else
  return r > 0.0 && 2.0 * E * r > m * m;
#endif
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
// G75 selects gamma = 7/5, where every power of the solver has exponent
// k/7 or an integer and comes from one x^(-1/7); otherwise pow() is used.
// ---------------------------------------------------------------------------
struct Side {
  double r, u, p, c;     // primitive state and sound speed
  double ir, ic;         // 1/rho, 1/c
  double sA, B;          // shock branch: sqrt(2/((g+1) rho)), (g-1)/(g+1) p
  double ip;             // 1/p
  double k;              // rarefaction branch: 2 c/(g-1)
  double d;              // rarefaction branch: 1/(rho c)
};

// One side of a Riemann problem from its conserved state: two reciprocal
// square roots and one division (1/p) replace the divisions of the textbook
// expressions.
GRP_HD __forceinline__ Side make_side(const Phys& ph, const double Q[3])
{
  Side s;
  const double tr = rsqrt(Q[0]);                 // rho^(-1/2)
  s.r = Q[0];
  s.ir = tr * tr;
  s.u = Q[1] * s.ir;
  s.p = ph.gm1 * (Q[2] - 0.5 * Q[1] * s.u);
  const double c2 = ph.gamma * s.p * s.ir;
  s.ic = rsqrt(c2);
  s.c = c2 * s.ic;
  s.sA = ph.sqrt_c2_gp1 * tr;
  s.B = ph.gm1_gp1 * s.p;
  s.ip = rcp64(s.p);
  s.k = ph.c2_gm1 * s.c;
  s.d = s.ir * s.ic;
  return s;
}

// pressure function f_K(p) and its derivative
template <bool G75>
GRP_HD __forceinline__ void pressure_fn(const Phys& ph, double p, const Side& K, double& f, double& df)
{
  if (gt_nn(p, K.p)) {                            // p, pK > 0
    const double t = rsqrt(p + K.B);             // (p + B)^(-1/2)
    const double s = K.sA * t;                    // sqrt(A / (p + B))
    f = (p - K.p) * s;
    df = s * (1.0 - 0.5 * (p - K.p) * (t * t));
  } else if (G75) {
    const double x = p * K.ip;
    const double w = inv_root7(x);
    const double w2 = w * w, w6 = w2 * w2 * w2;
    f = K.k * fma(x, w6, -1.0);          // (p/pK)^(1/7) = x * x^(-6/7)
    df = K.d * w6;                        // (p/pK)^(-6/7)
  } else {
    const double x = p * K.ip;
    f = K.k * (pow(x, ph.gm1_2g) - 1.0);
    df = K.d * pow(x, -ph.gp1_2g);
  }
}

// Two-rarefaction estimate of the star pressure (exact when both waves are
// rarefactions); 0 when the data generate vacuum.
template <bool G75>
GRP_HD __forceinline__ double trrs(const Phys& ph, const Side& L, const Side& R)
{
  const double num = L.c + R.c - 0.5 * ph.gm1 * (R.u - L.u);
  if (!positive(num)) return 0.0;
  if (G75) {                                        // z = 1/7: p^-z by a 7th root, ^(1/z) = ^7
    const double q = num / (L.c * inv_root7(L.p) + R.c * inv_root7(R.p));
    const double q2 = q * q, q4 = q2 * q2;
    return q4 * q2 * q;
  }
  const double z = ph.gm1_2g;
  return pow(num / (L.c * pow(L.p, -z) + R.c * pow(R.p, -z)), 1.0 / z);
}

// PVRS estimate of the star pressure, floored at 1e-14 max(pL, pR)
GRP_HD __forceinline__ double pvrs(const Side& L, const Side& R)
{
  const double ppv = 0.5 * (L.p + R.p) - 0.125 * (R.u - L.u) * (L.r + R.r) * (L.c + R.c);
  return max_nn(ppv, 1e-14 * max_nn(L.p, R.p));    // the floor is positive
}

// Two-shock estimate of the star pressure from the pressure p0 (the PVRS
// estimate): the shock branches linearised at p0.
GRP_HD __forceinline__ double tsrs(const Side& L, const Side& R, double p0)
{
  const double gL = L.sA * rsqrt(p0 + L.B), gR = R.sA * rsqrt(p0 + R.B);
  return (gL * L.p + gR * R.p - (R.u - L.u)) * rcp64(gL + gR);
}

// Internal start for the repair (first-order) Riemann problems of cell
// averages, whose data are strong: the textbook adaptive choice of PVRS when
// the pressures are close and its estimate lies between them, the
// two-rarefaction estimate when it falls below both, the two-shock estimate
// otherwise.
constexpr int GUESS_ADAPTIVE = 3;

// Returns ST_OK / ST_NO_CONV / ST_VACUUM.  p0 > 0 is used as the start when
// given (learned guess), otherwise PVRS, TRRS or the adaptive choice per
// ph.guess.
template <bool G75>
static GRP_HD int star_pressure(const Phys& ph, const Side& L, const Side& R, double p0, double& ps, double& us,
                                int& iters)
{
  const double du = R.u - L.u;
  iters = 0;
  if (ph.c2_gm1 * (L.c + R.c) <= du) return ST_VACUUM;
  const double pfloor = 1e-14 * max_nn(L.p, R.p);
  double p;
  if (finite_positive(p0)) {
    p = p0;
  } else if (ph.guess == 1) {
    p = trrs<G75>(ph, L, R);
  } else if (ph.guess == GUESS_ADAPTIVE) {
    // pL, pR > 0 and ppv is floored at a positive value: integer tests
    const double ppv = pvrs(L, R), pmax = max_nn(L.p, R.p);
    const double pmin = gt_nn(L.p, R.p) ? R.p : L.p;
    if (gt_nn(2.0 * pmin, pmax) && !gt_nn(pmin, ppv) && !gt_nn(ppv, pmax)) p = ppv;
    else if (gt_nn(pmin, ppv)) p = trrs<G75>(ph, L, R);
    else p = tsrs(L, R, ppv);
  } else {
    p = pvrs(L, R);
  }
  if (!gt_nn(p, pfloor) || !positive(p)) p = pfloor;
  bool conv = false, done = false;
  int it = 0;
  while (it < ph.max_iter) {
    double fL, dfL, fR, dfR;
    pressure_fn<G75>(ph, p, L, fL, dfL);
    pressure_fn<G75>(ph, p, R, fR, dfR);
    double step = -(fL + fR + du) * rcp_newton_step(dfL + dfR);
    double pn = p + step;
    for (int h = 0; h < 64 && !positive(pn); ++h) { step *= 0.5; pn = p + step; }
    ++it;
    const bool small = gt_nn(ph.rtol * (pn + p), 2.0 * fabs(pn - p));   // relative change < rtol
    if (conv) {
      // the extra iteration after convergence: its step is at the rounding
      // level, so the pressure functions at the new iterate are those at p
      // carried along the tangent (the error is of the step squared), and
      // u* needs no further evaluation
      us = 0.5 * (L.u + R.u) + 0.5 * ((fR - fL) + (dfR - dfL) * (pn - p));
      p = pn;
      done = true;
      break;
    }
    p = pn;
    if (small) conv = true;
  }
  iters = it;
  if (!conv) return ST_NO_CONV;
  if (!done) {          // converged on the last allowed iteration: evaluate at p
    double fL, dfL, fR, dfR;
    pressure_fn<G75>(ph, p, L, fL, dfL);
    pressure_fn<G75>(ph, p, R, fR, dfR);
    us = 0.5 * (L.u + R.u) + 0.5 * (fR - fL);
  }
  ps = p;
  return ST_OK;
}

// Density behind a rarefaction from K to pressure ratio x = p/pK, and the
// sound speed there: rho = rhoK x^(1/g), c = cK x^((g-1)/(2g)).
template <bool G75>
GRP_HD __forceinline__ void rarefied(const Phys& ph, const Side& K, double x, double& rho, double& c)
{
  if (G75) {
    const double w = inv_root7(x), w2 = w * w;
    rho = K.r * x * w2;                  // x^(5/7)
    c = K.c * x * (w2 * w2 * w2);        // x^(1/7)
  } else {
    rho = K.r * pow(x, ph.i_g);
    c = K.c * pow(x, ph.gm1_2g);
  }
}

// Sonic state inside a fan: rho = rhoK q^(2/(g-1)), p = pK q^(2g/(g-1)), q = c0/cK.
template <bool G75>
GRP_HD __forceinline__ Prim sonic(const Phys& ph, const Side& K, double c0, double u0)
{
  const double q = c0 * K.ic;
  if (G75) {
    const double q2 = q * q, q5 = q2 * q2 * q;
    return Prim{K.r * q5, u0, K.p * q5 * q2};
  }
  return Prim{K.r * pow(q, ph.c2_gm1), u0, K.p * pow(q, ph.c2g_gm1)};
}

// Left of the contact when u* >= 0, sampled on the ray x/t = 0.  A contact
// speed within TIE of the sound-speed scale is stationary and goes left.
template <bool G75>
static GRP_HD Prim sample_zero(const Phys& ph, const Side& L, const Side& R, double ps, double us)
{
  const double g1 = ph.gm1_2g, g6 = ph.gm1_gp1;
  const Prim WL{L.r, L.u, L.p}, WR{R.r, R.u, R.p};
  if (us >= -TIE * (L.c + R.c)) {
    const double ratio = ps * L.ip;
    if (gt_nn(ps, L.p)) {
      const double S = L.u - L.c * sqrt(ph.gp1_2g * ratio + g1);
      if (ge0(S)) return WL;
      return Prim{L.r * (ratio + g6) / (g6 * ratio + 1.0), us, ps};
    }
    if (ge0(L.u - L.c)) return WL;
    double rho, cs;
    rarefied<G75>(ph, L, ratio, rho, cs);
    if (lt0(us - cs)) return Prim{rho, us, ps};
    const double c0 = ph.c2_gp1 * (L.c + 0.5 * ph.gm1 * L.u);
    return sonic<G75>(ph, L, c0, c0);
  }
  const double ratio = ps * R.ip;
  if (gt_nn(ps, R.p)) {
    const double S = R.u + R.c * sqrt(ph.gp1_2g * ratio + g1);
    if (le0(S)) return WR;
    return Prim{R.r * (ratio + g6) / (g6 * ratio + 1.0), us, ps};
  }
  if (le0(R.u + R.c)) return WR;
  double rho, cs;
  rarefied<G75>(ph, R, ratio, rho, cs);
  if (positive(us + cs)) return Prim{rho, us, ps};
  const double c0 = ph.c2_gp1 * (R.c - 0.5 * ph.gm1 * R.u);
  return sonic<G75>(ph, R, c0, -c0);
}

// Vacuum-generating data: two rarefactions around a vacuum, sampled at x/t = 0.
template <bool G75>
static GRP_HD Prim sample_vacuum_zero(const Phys& ph, const Side& L, const Side& R)
{
  if (L.u - L.c >= 0.0) return Prim{L.r, L.u, L.p};
  if (L.u + ph.c2_gm1 * L.c > 0.0) {
    const double c0 = ph.c2_gp1 * (L.c + 0.5 * ph.gm1 * L.u);
    return sonic<G75>(ph, L, c0, c0);
  }
  if (R.u + R.c <= 0.0) return Prim{R.r, R.u, R.p};
  if (R.u - ph.c2_gm1 * R.c < 0.0) {
    const double c0 = ph.c2_gp1 * (R.c - 0.5 * ph.gm1 * R.u);
    return sonic<G75>(ph, R, c0, -c0);
  }
  return Prim{0.0, 0.0, 0.0};
}

// ---------------------------------------------------------------------------
// Learned Newton initial guess (FP32): a 6 -> 64 -> 64 -> 1 tanh network on
// features invariant under the scaling and Galilean symmetries of the Riemann
// problem, predicting the correction of the two-rarefaction estimate p_TR.
// With the shock strength s = ln(p_TR / min(pL, pR)) the correction
// ln(p*/p_TR) vanishes like s^3 (the Hugoniot and the isentrope agree to
// second order), so the network predicts the normalised correction
// v = ln(p*/p_TR) / (MLP_T_SCALE s^3), of order one at every strength, and the
// guess is p_TR exp(MLP_T_SCALE s^3 v).  Only strong data use it: with
// s >= MLP_S_MIN the network, below it (two rarefactions: s <= 0, p_TR is p*)
// p_TR itself; PVRS starts the rest and is the fallback.
// Parameter layout: W1[6][64], b1[64], W2[64][64], b2[64], w3[64], b3.
// ---------------------------------------------------------------------------
constexpr int MLP_NIN = 6, MLP_NH = 64;
constexpr int MLP_NPARAM = MLP_NIN * MLP_NH + MLP_NH + MLP_NH * MLP_NH + MLP_NH + MLP_NH + 1;
constexpr int MLP_GUESS_MAX_ITER = 8;     // Newton from the learned guess gives up after this
constexpr float MLP_GATE = 0.5f;          // |ln(pL/pR)| or |du|/cbar above this: strong data
constexpr double MLP_GATE_EXP = 1.6487212707001282;   // e^MLP_GATE
constexpr double MLP_S_MIN = 1e-3;        // shock strength below which p_TR is the start
constexpr double MLP_T_SCALE = -0.005;    // output scale: ln(p*/p_TR) = MLP_T_SCALE s^3 v
constexpr float MLP_VMAX = 50.0f;         // |v| above this: prediction rejected
constexpr double MLP_YMAX = 18.420681;    // |ln(p*/p_TR)| <= ln 1e8

GRP_HD __forceinline__ float fast_tanh(float x)
{
#ifdef __CUDA_ARCH__
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
#else
  return tanhf(x);
#endif
}

// Strong data, decided without transcendental functions:
// |ln(pL/pR)| > g  <=>  pL/pR outside [e^-g, e^g], and
// |du|/cbar > g    <=>  du^4 rhoL rhoR > g^4 gamma^2 pL pR.
GRP_HD __forceinline__ bool strong_data(const Phys& ph, const Side& L, const Side& R)
{
  const double pr = L.p * R.ip, dun = R.u - L.u, du2 = dun * dun;
  const double g2 = (double)MLP_GATE * (double)MLP_GATE;
  // all three compare non-negative doubles: integer tests of the bits
  return gt_nn(pr, MLP_GATE_EXP) || gt_nn(1.0, pr * MLP_GATE_EXP) ||
         gt_nn(du2 * du2 * (L.r * R.r), g2 * g2 * ph.gamma * ph.gamma * (L.p * R.p));
}

// Features x[6] of strong data, in FP32 (the network's precision; off the
// FP64 pipe, which the lanes around this one keep busy).
GRP_HD __forceinline__ void mlp_features(const Phys& ph, const Side& L, const Side& R, float x[6])
{
  const float pl = (float)L.p, pr = (float)R.p, rl = (float)L.r, rr = (float)R.r;
  const float lp = logf(pl / pr);
  const float lr = logf(rl / rr);
  const float cbar = sqrtf((float)ph.gamma * sqrtf(pl) * sqrtf(pr) / (sqrtf(rl) * sqrtf(rr)));
  const float du = ((float)R.u - (float)L.u) / cbar;
  x[0] = 0.5f * lr; x[1] = -0.5f * lr;
  x[2] = 0.5f * lp; x[3] = -0.5f * lp;
  x[4] = -0.5f * du; x[5] = 0.5f * du;
}

// The two-rarefaction estimate in FP32, as a Newton start (Newton takes any
// start to the same p*; the network's correction multiplies it).  0 when the
// data generate vacuum.
GRP_HD __forceinline__ float trrs_f32(const Phys& ph, const Side& L, const Side& R)
{
  const float cl = (float)L.c, cr = (float)R.c, gm1 = (float)ph.gm1, z = (float)ph.gm1_2g;
  const float num = cl + cr - 0.5f * gm1 * ((float)R.u - (float)L.u);
  if (!(num > 0.0f)) return 0.0f;
  const float q = num / (cl * powf((float)L.p, -z) + cr * powf((float)R.p, -z));
  return powf(q, 1.0f / z);
}

// The hidden activations live in local memory (the loops over neurons are not
// unrolled): the network runs on a few strong-data interfaces only, and 64
// activations in registers would raise the register count of every flux
// kernel that contains this path.
GRP_HD inline float mlp_eval(const float* __restrict__ w, const float x[6])
{
  const float* W1 = w;
  const float* b1 = W1 + MLP_NIN * MLP_NH;
  const float* W2 = b1 + MLP_NH;
  const float* b2 = W2 + MLP_NH * MLP_NH;
  const float* w3 = b2 + MLP_NH;
  const float b3 = w3[MLP_NH];
  float h1[MLP_NH];
#pragma unroll 1
  for (int j = 0; j < MLP_NH; ++j) {
    float z = b1[j];
#pragma unroll
    for (int i = 0; i < MLP_NIN; ++i) z = fmaf(x[i], W1[i * MLP_NH + j], z);
    h1[j] = fast_tanh(z);
  }
  // the second layer eight outputs at a time: eight independent accumulation
  // chains (each in the order j = 0..63, as a one-output loop would add) keep
  // the chain's latency, not its length, on the critical path
  float y = b3;
#pragma unroll 1
  for (int k0 = 0; k0 < MLP_NH; k0 += 8) {
    float z[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) z[q] = b2[k0 + q];
#pragma unroll 2
    for (int j = 0; j < MLP_NH; ++j) {
      const float h = h1[j];
      const float* Wr = W2 + j * MLP_NH + k0;
#pragma unroll
      for (int q = 0; q < 8; ++q) z[q] = fmaf(h, Wr[q], z[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) y = fmaf(fast_tanh(z[q]), w3[k0 + q], y);
  }
  return y;
}

// The network for one input x (the same in every lane of the warp), evaluated
// by the whole warp: each lane computes hidden units lane and lane + 32 of
// both layers, the output is a warp sum.  hs: 64 floats of shared memory of
// this warp.  Called by all 32 lanes, converged.
__device__ __forceinline__ float mlp_eval_warp(const float* __restrict__ w, const float x[6], float* hs)
{
  const float* W1 = w;
  const float* b1 = W1 + MLP_NIN * MLP_NH;
  const float* W2 = b1 + MLP_NH;
  const float* b2 = W2 + MLP_NH * MLP_NH;
  const float* w3 = b2 + MLP_NH;
  const int l = threadIdx.x & 31;
  float z0 = b1[l], z1 = b1[l + 32];
#pragma unroll
  for (int i = 0; i < MLP_NIN; ++i) {
    z0 = fmaf(x[i], W1[i * MLP_NH + l], z0);
    z1 = fmaf(x[i], W1[i * MLP_NH + l + 32], z1);
  }
  hs[l] = fast_tanh(z0);
  hs[l + 32] = fast_tanh(z1);
  __syncwarp();
  float y0 = b2[l], y1 = b2[l + 32];
#pragma unroll 8
  for (int j = 0; j < MLP_NH; ++j) {
    const float h = hs[j];
    y0 = fmaf(h, W2[j * MLP_NH + l], y0);
    y1 = fmaf(h, W2[j * MLP_NH + l + 32], y1);
  }
  float y = fmaf(fast_tanh(y0), w3[l], fast_tanh(y1) * w3[l + 32]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) y += __shfl_xor_sync(0xffffffffu, y, off);
  __syncwarp();                                  // hs is reused by the next call
  return y + w3[MLP_NH];
}

struct RSInfo {
  double ps = 0.0;               // star pressure
  double base = 0.0;             // two-rarefaction estimate (the base of the learned correction)
  double s3 = 0.0;               // cube of the shock strength ln(p_TR / min(pL, pR))
  float x[6];                    // features (valid when has_x)
  bool has_x = false;            // strong data with a shock of strength >= MLP_S_MIN
  int guess = 0;                 // 0 not tried, 1 network start used, 2 rejected, 3 p_TR start (two rarefactions)
};

// The inference form's decisions for strong data, in FP32 (features x, the
// two-rarefaction base, the cube of the shock strength): whether the start
// comes from the network (the returned value) and the input-box test.
struct LearnedPrep {
  float base, s3;
  bool ok, has_x, inbox;
};

// The decisions and features of strong data worked out before the solve (the
// second flux pass), with the network's output v (valid when the network was
// wanted), so that the solve does not repeat them.
struct LearnedPre {
  LearnedPrep q;
  float x[6];
  float v;
};

GRP_HD __forceinline__ bool learned_prep_f32(const Phys& ph, const Side& L, const Side& R, float x[6],
                                             LearnedPrep& q)
{
  mlp_features(ph, L, R, x);
  q.base = trrs_f32(ph, L, R);
  q.ok = q.base > 0.0f && isfinite(q.base);
  const float sh = q.ok ? logf(q.base / fminf((float)L.p, (float)R.p)) : 0.0f;
  q.s3 = sh * sh * sh;
  q.has_x = q.ok && sh >= (float)MLP_S_MIN;
  q.inbox = true;
  if (ph.guess == 2 && ph.mlp_w && q.has_x) {
#pragma unroll
    for (int i = 0; i < 6; ++i) q.inbox = q.inbox && x[i] >= ph.mlp_box[i] && x[i] <= ph.mlp_box[6 + i];
  }
  return ph.guess == 2 && ph.mlp_w && q.has_x && q.inbox;
}

// The learned-guess path of riemann_state for strong data: features, the
// two-rarefaction base and, for data with a shock, the network; Newton from
// that start.  Returns
// the solver status, or -1 when no learned start was tried.  Kept out of line
// so that its registers do not count against the flux kernels, which take
// this path on a few strong-data interfaces only.
template <bool G75>
#ifdef __CUDA_ARCH__
__device__ __noinline__
#else
inline
#endif
int learned_start(const Phys& ph, const Side& L, const Side& R, RSInfo& info, double& ps, double& us, int& iters,
                  const LearnedPre* pre)
{
  int st = -1;
  double p0 = 0.0;
  bool ok, go = true;
  float v = 0.0f;
  if (ph.features == 2) {
    mlp_features(ph, L, R, info.x);
    // harvest: the record's target ln(p*/p_TR) / (MLP_T_SCALE s^3) needs p_TR
    // and the strength in FP64 (for weak shocks the correction is ~1e-12)
    const double base = trrs<G75>(ph, L, R);
    ok = base > 0.0 && isfinite(base);
    // shock strength s = ln(p_TR / min(pL, pR)); s <= 0: two rarefactions, and
    // p_TR is p* up to rounding; s < MLP_S_MIN: |ln(p*/p_TR)| < 1e-11
    const double sh = ok ? log(base / fmin(L.p, R.p)) : 0.0;
    info.base = base;
    info.s3 = sh * sh * sh;
    info.has_x = ok && sh >= MLP_S_MIN;
    p0 = base;
    if (ph.guess == 2 && ph.mlp_w && ok && info.has_x) {
      bool inbox = true;
#pragma unroll
      for (int i = 0; i < 6; ++i) inbox = inbox && info.x[i] >= ph.mlp_box[i] && info.x[i] <= ph.mlp_box[6 + i];
      v = inbox ? mlp_eval(ph.mlp_w, info.x) : 0.0f;
      const double y = MLP_T_SCALE * info.s3 * (double)v;
      go = inbox && v == v && fabsf(v) <= MLP_VMAX && fabs(y) <= MLP_YMAX;
      p0 = base * exp(y);
    }
  } else {
    // inference: the start in FP32 (the same decisions and correction; Newton
    // converges from it to the same p*).  pre: the decisions, features and
    // network output worked out beforehand (the network by the whole warp)
    LearnedPrep q;
    if (pre) {
      q = pre->q;
#pragma unroll
      for (int i = 0; i < 6; ++i) info.x[i] = pre->x[i];
    } else {
      learned_prep_f32(ph, L, R, info.x, q);
    }
    ok = q.ok;
    info.base = q.base;
    info.s3 = q.s3;
    info.has_x = q.has_x;
    p0 = q.base;
    if (ph.guess == 2 && ph.mlp_w && ok && info.has_x) {
      v = q.inbox ? (pre ? pre->v : mlp_eval(ph.mlp_w, info.x)) : 0.0f;
      const float y = (float)MLP_T_SCALE * q.s3 * v;
      go = q.inbox && v == v && fabsf(v) <= MLP_VMAX && fabsf(y) <= (float)MLP_YMAX;
      p0 = (double)(q.base * expf(y));
    }
  }
  if (ph.guess == 2 && ph.mlp_w && ok) {
    info.guess = 2;
    if (go) {
      Phys pg = ph;
      pg.max_iter = ph.max_iter < MLP_GUESS_MAX_ITER ? ph.max_iter : MLP_GUESS_MAX_ITER;
      st = star_pressure<G75>(pg, L, R, p0, ps, us, iters);
      if (st == ST_OK) info.guess = info.has_x ? 1 : 3;   // 3: p_TR start, not a network start
    }
  }
  return st;
}

// Godunov state at x/t = 0 of conserved data QL | QR, as conserved Q and
// primitive W.  allow_vacuum: vacuum data are sampled and ST_VACUUM returned
// with Q valid.  With a learned model (ph.guess == 2) strong data start Newton
// from the network's prediction (or from p_TR for two rarefactions); an input
// outside the training box, a prediction out of range or not finite, or no
// convergence within MLP_GUESS_MAX_ITER iterations falls back to PVRS
// (iterations add up).  pre: strong data whose learned-start decisions are
// worked out already; strong: 0 data known not to be strong, -1 not known
// (tested here).
template <bool G75>
static GRP_HD int riemann_sides(const Phys& ph, const Side& L, const Side& R, bool allow_vacuum, double Q[3],
                                Prim& W, int& iters, RSInfo* info, const LearnedPre* pre = nullptr,
                                int strong = -1)
{
  double ps = 0.0, us = 0.0;
  int st = -1;
  iters = 0;
  // the learned-guess path (out of line) only for strong data
  if (ph.features && info && (pre || (strong < 0 && strong_data(ph, L, R))))
    st = learned_start<G75>(ph, L, R, *info, ps, us, iters, pre);
  if (st != ST_OK && st != ST_VACUUM) {
    int it2 = 0;
    Phys pv = ph;
    pv.guess = ph.guess == 2 ? 0 : ph.guess;       // classical guess (PVRS) as the fallback
    st = star_pressure<G75>(pv, L, R, 0.0, ps, us, it2);
    iters += it2;
  }
  if (info) info->ps = ps;
  if (st == ST_VACUUM && allow_vacuum) {
    W = sample_vacuum_zero<G75>(ph, L, R);
    to_cons(ph, W, Q);
    return ST_VACUUM;
  }
  if (st != ST_OK) return st;
  W = sample_zero<G75>(ph, L, R, ps, us);
  to_cons(ph, W, Q);
  return ST_OK;
}

template <bool G75>
static GRP_HD int riemann_state(const Phys& ph, const double QL[3], const double QR[3], bool allow_vacuum,
                                double Q[3], Prim& W, int& iters, RSInfo* info = nullptr)
{
  const Side L = make_side(ph, QL);
  const Side R = make_side(ph, QR);
  return riemann_sides<G75>(ph, L, R, allow_vacuum, Q, W, iters, info);
}

// A leading Riemann problem solved before its GRP (the second flux pass solves
// them with the network's starts evaluated by whole warps).
struct Lead {
  int st, iters;
  double Q0[3];
  Prim W0;
  RSInfo info;
};

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
  double k;                // u^2 / 2
  double lam[3];
};

GRP_HD __forceinline__ Eig make_eig(const Phys& ph, const double Q0[3], Prim w, double ir)
{
  Eig e;
  e.u = w.u;
  const double c2 = ph.gamma * w.p * ir;
  e.ic = rsqrt(c2);
  e.c = c2 * e.ic;
  e.H = (Q0[2] + w.p) * ir;
  e.b1 = ph.gm1 * e.ic * e.ic;
  e.k = 0.5 * e.u * e.u;
  e.b2 = e.k * e.b1;
  e.lam[0] = e.u - e.c; e.lam[1] = e.u; e.lam[2] = e.u + e.c;
  e.tie = TIE * (fabs(e.u) + e.c);
  return e;
}

GRP_HD __forceinline__ Eig make_eig(const Phys& ph, const double Q0[3], Prim w)
{
  return make_eig(ph, Q0, w, rcp64(w.r));
}

GRP_HD __forceinline__ void char_proj(const Eig& e, const double D[3], double w[3])
{
  // rows of R^{-1}
  const double uc = e.u * e.ic;
  w[0] = 0.5 * ((e.b2 + uc) * D[0] - (e.b1 * e.u + e.ic) * D[1] + e.b1 * D[2]);
  w[1] = (1.0 - e.b2) * D[0] + e.b1 * e.u * D[1] - e.b1 * D[2];
  w[2] = 0.5 * ((e.b2 - uc) * D[0] - (e.b1 * e.u - e.ic) * D[1] + e.b1 * D[2]);
}

// characteristic amplitudes w back to conserved variables: D = sum_j w_j r_j
GRP_HD __forceinline__ void char_back(const Eig& e, const double w[3], double D[3])
{
  D[0] = w[0] + w[1] + w[2];
  D[1] = (e.u - e.c) * w[0] + e.u * w[1] + (e.u + e.c) * w[2];
  D[2] = (e.H - e.u * e.c) * w[0] + e.k * w[1] + (e.H + e.u * e.c) * w[2];
}

// Upwind weight theta of a field of speed lam in a derivative Riemann problem:
// 0 when lam > tie (left data), 1 when lam < -tie (right data), 1/2 between (a
// sonic field averages the two sides); tie >= 0.  On the GPU both tests are
// integer compares of the bit patterns (exact for non-NaN values: -lam > tie
// with the sign bit flipped), off the FP64 pipe.
// As twice the weight (0, 1 or 2), so that the test for a field that takes
// right data is an integer one too.
GRP_HD __forceinline__ int upwind_weight2(double lam, double tie)
{
#ifdef __CUDA_ARCH__
  const long long b = __double_as_longlong(lam), t = __double_as_longlong(tie);
  if (b > t) return 0;
  if ((b ^ (long long)0x8000000000000000ull) > t) return 2;
  return 1;
#else
  return lam > tie ? 0 : (lam < -tie ? 2 : 1);
#endif
}

// All M derivative Riemann problems of one interface at once:
// D_k = DL_k - sum_j theta_j (l_j . J_k) r_j with J_k = DL_k - DR_k.  theta_j
// depends on the field only, so a field that takes right data (theta_j != 0)
// is applied to every order k in one branch, and its left eigenvector l_j
// (row of R^{-1}) and right eigenvector r_j = (1, r1, r2) are formed only
// there; in smooth subsonic flow that is one field of the three.
// t[c][k]: Taylor coefficients of the traces; D[k][c] for k = 1..M.
template <int M>
GRP_HD __forceinline__ void deriv_rps(const Eig& e, const double tL[][M + 1], const double tR[][M + 1],
                                      double D[M + 1][3])
{
  double J[M + 1][3];
#pragma unroll
  for (int k = 1; k <= M; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      J[k][c] = tL[c][k] - tR[c][k];
      D[k][c] = tL[c][k];
    }
  const double bu = e.b1 * e.u;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int th2 = upwind_weight2(e.lam[j], e.tie);
    if (th2 != 0) {
      // theta_j l_j: theta is 1 or 1/2, a power of two, so folding it into
      // the row changes no bit of the products
      double l0, l1, l2, r1, r2;
      if (j == 1) {
        l0 = 1.0 - e.b2; l1 = bu; l2 = -e.b1;
        if (th2 == 1) { l0 *= 0.5; l1 *= 0.5; l2 *= 0.5; }
        r1 = e.u; r2 = e.k;
      } else {
        const double sg = j == 0 ? 1.0 : -1.0;          // field u - c (j = 0) or u + c (j = 2)
        const double h = th2 == 2 ? 0.5 : 0.25;         // theta / 2
        const double uc = e.u * e.ic;
        l0 = h * (e.b2 + sg * uc); l1 = -h * (bu + sg * e.ic); l2 = h * e.b1;
        r1 = e.lam[j]; r2 = e.H - sg * (e.u * e.c);
      }
#pragma unroll
      for (int k = 1; k <= M; ++k) {
        const double w = l0 * J[k][0] + l1 * J[k][1] + l2 * J[k][2];
        D[k][0] -= w;
        D[k][1] -= w * r1;
        D[k][2] -= w * r2;
      }
    }
  }
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
// gm1: gamma - 1.
// irho, u0, p0: 1/rho, velocity and pressure of the leading state (known to
// the caller), the series' constant terms.
// SRC: with the constant-acceleration source S = (0, -g rho, -g m), in scaled
// variables d_T Q + d_X F = dx S: q[a][b+1] gets hs/(b+1) (0, rho[a][b],
// m[a][b]) added, hs = -g dx.
template <int M, bool SRC = false>
GRP_HD __forceinline__ void ck_euler(double gm1, double rho[Tri<M>::N], double m[Tri<M>::N],
                                         double E[Tri<M>::N], double s[3][M + 1], double irho, double u0, double p0,
                                         double hs = 0.0)
{
  using T = Tri<M>;
  double u[T::N], mu[T::N], Ep[T::N], F1[T::N], F2[T::N];
#pragma unroll
  for (int b = 0; b < M; ++b) {
#pragma unroll
    for (int a = 0; a + b <= M; ++a) {
      const int k = T::idx(a, b);
      if (k == 0) {
        u[0] = u0;
        Ep[0] = E[0] + p0;
        continue;
      }
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
      const int src = T::idx(a + 1, b), dst = T::idx(a, b + 1), here = T::idx(a, b);
      rho[dst] = f * m[src];
      if (SRC) {
        const double h = hs / double(b + 1);
        m[dst] = fma(h, rho[here], f * F1[src]);
        E[dst] = fma(h, m[here], f * F2[src]);
      } else {
        m[dst] = f * F1[src];
        E[dst] = f * F2[src];
      }
    }
  }
#pragma unroll
  for (int b = 0; b <= M; ++b) {
    s[0][b] = rho[T::idx(0, b)];
    s[1][b] = m[T::idx(0, b)];
    s[2][b] = E[T::idx(0, b)];
  }
}

// Node a of the G-point Gauss-Legendre rule on [0, 1].
GRP_HD __forceinline__ double gauss_node(int G, int a)
{
  if (G == 1) return 0.5;
  if (G == 2) return a == 0 ? 0.5 - 0.28867513459481288225 : 0.5 + 0.28867513459481288225;
  return a == 0 ? 0.5 - 0.38729833462074168852 : (a == 1 ? 0.5 : 0.5 + 0.38729833462074168852);
}

// Gauss-Legendre rule with G = ceil((M+1)/2) points on [0, 1]: nodes
// (1 + s)/2 and weights summing to 1.
template <int M>
struct Gauss {
  static constexpr int G = (M + 2) / 2;
  GRP_HD static __forceinline__ double node(int a) { return gauss_node(G, a); }
  GRP_HD static __forceinline__ double weight(int a)
  {
    if (G == 1) return 1.0;
    if (G == 2) return 0.5;
    return a == 1 ? 8.0 / 18.0 : 5.0 / 18.0;
  }
};

// Riemann data that agree to within rounding (each conserved component to
// 2^-48 of the sum of its two values; the momentum on the scale
// sqrt(rho E)) are equal data: the exact solution is the constant state and
// no wave forms.  The interpolating reconstructions (degrees 2 and 4) put the
// interface datum itself on both sides of every interface whose two cells
// kept their polynomials, so there the traces are bitwise equal.
constexpr double EQ_TOL = 3.552713678800501e-15;   // 2^-48

GRP_HD __forceinline__ bool equal_data(const double QL[3], const double QR[3])
{
#ifdef __CUDA_ARCH__
  // identical bits first (integer compares; the interpolating degrees give
  // exactly this at every interface whose cells kept their polynomials)
  if (__double_as_longlong(QL[0]) == __double_as_longlong(QR[0]) &&
      __double_as_longlong(QL[1]) == __double_as_longlong(QR[1]) &&
      __double_as_longlong(QL[2]) == __double_as_longlong(QR[2]))
    return true;
#endif
  const double sr = QL[0] + QR[0], sE = QL[2] + QR[2], dm = QR[1] - QL[1];
  return fabs(QR[0] - QL[0]) <= EQ_TOL * sr && fabs(QR[2] - QL[2]) <= EQ_TOL * sE &&
         dm * dm <= (EQ_TOL * EQ_TOL) * (sr * sE);
}

// ---------------------------------------------------------------------------
// One GRP_M at an interface (Toro-Titarev structure, Section 2) and its flux
// time integral over [0, dt] (numerical flux, Section 2), in scaled
// variables: t[c][k] are the Taylor coefficients p^{(k)}/k! of the
// reconstructions at the interface, nu = dt/dx.  The interface datum for the
// next step is the series at tau = dt.
// ---------------------------------------------------------------------------
// Advection with the source S = k q (SRC), scaled: d_T q + lam d_X q = hk q
// with hk = k dx, so q[a][b+1] = (-lam (a+1) q[a+1][b] + hk q[a][b]) / (b+1).
template <int M>
GRP_HD __forceinline__ void ck_adv_src(double lam, double hk, double q[Tri<M>::N])
{
  using T = Tri<M>;
#pragma unroll
  for (int b = 0; b < M; ++b)
#pragma unroll
    for (int a = 0; a + b + 1 <= M; ++a)
      q[T::idx(a, b + 1)] = (-lam * double(a + 1) * q[T::idx(a + 1, b)] + hk * q[T::idx(a, b)]) / double(b + 1);
}

template <int M, bool SRC = false>
GRP_HD __forceinline__ void grp_adv(double lam, double nu, const double tL[M + 1], const double tR[M + 1],
                                    double& F, double& gnew, double hk = 0.0)
{
  double s[M + 1];
#pragma unroll
  for (int k = 0; k <= M; ++k) s[k] = lam > 0.0 ? tL[k] : (lam < 0.0 ? tR[k] : 0.5 * (tL[k] + tR[k]));
  if (SRC) {
    using T = Tri<M>;
    double q[T::N];
#pragma unroll
    for (int k = 0; k <= M; ++k) q[T::idx(k, 0)] = s[k];
    ck_adv_src<M>(lam, hk, q);
#pragma unroll
    for (int b = 0; b <= M; ++b) s[b] = q[T::idx(0, b)];
  } else {
    // CK for q_t + lam q_x = 0: q[0][b] = (-lam)^b q[b][0]
    double sc = 1.0;
#pragma unroll
    for (int k = 0; k <= M; ++k) { s[k] *= sc; sc *= -lam; }
  }
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
template <int M, bool G75, bool SRC = false>
GRP_HD __forceinline__ int grp_euler(const Phys& ph, double nu, const double tL[3][M + 1],
                                     const double tR[3][M + 1], double F[3], double gnew[3], int& iters,
                                     bool& truncated, RSInfo* info = nullptr, double hs = 0.0,
                                     const Lead* lead = nullptr, const double* tg = nullptr)
{
  const double g = ph.gamma;
  const double QL[3] = {tL[0][0], tL[1][0], tL[2][0]}, QR[3] = {tR[0][0], tR[1][0], tR[2][0]};
  double Q0[3];
  Prim W0;
  double ir0;
  truncated = false;
  if (lead) {
    // the leading Riemann problem solved by the caller
    iters = lead->iters;
    if (info) *info = lead->info;
    if (lead->st != ST_OK) return lead->st;
    Q0[0] = lead->Q0[0]; Q0[1] = lead->Q0[1]; Q0[2] = lead->Q0[2];
    W0 = lead->W0;
    ir0 = rcp64(W0.r);
  } else if (equal_data(QL, QR)) {
    // equal data: the exact solution is the constant state, no Newton (the
    // traces are admissible: an inadmissible one sends its cell to degree 0)
    Q0[0] = QL[0]; Q0[1] = QL[1]; Q0[2] = QL[2];
    ir0 = rcp64(Q0[0]);
    W0.r = Q0[0];
    W0.u = Q0[1] * ir0;
    W0.p = ph.gm1 * (Q0[2] - 0.5 * Q0[1] * W0.u);
    iters = 0;
    if (info) info->ps = W0.p;
  } else {
    const int st = riemann_state<G75>(ph, QL, QR, false, Q0, W0, iters, info);
    if (st != ST_OK) return st;
    ir0 = rcp64(W0.r);
  }
  using T = Tri<M>;
  double rho[T::N], m[T::N], E[T::N];
  rho[0] = Q0[0]; m[0] = Q0[1]; E[0] = Q0[2];
  {
    const Eig e = make_eig(ph, Q0, W0, ir0);
    double D[M + 1][3];
    deriv_rps<M>(e, tL, tR, D);
#pragma unroll
    for (int k = 1; k <= M; ++k) {
      rho[T::idx(k, 0)] = D[k][0]; m[T::idx(k, 0)] = D[k][1]; E[T::idx(k, 0)] = D[k][2];
    }
  }
  double s[3][M + 1];
  ck_euler<M, SRC>(ph.gm1, rho, m, E, s, ir0, W0.u, W0.p, hs);
  // states at the Gauss nodes and at tau = dt; at a node one reciprocal
  // serves both the admissibility test and the flux, at dt (no flux) the
  // test is division-free
  constexpr int G = Gauss<M>::G;
  double Qg[G + 1][3], ug[G], pg[G];
  bool ok = true;
#pragma unroll
  for (int al = 0; al <= G; ++al) {
    // tg: nu x the nodes, formed once per domain (the same products)
    const double Tn = al < G ? (tg ? tg[al] : nu * Gauss<M>::node(al)) : nu;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double v = s[c][M];
#pragma unroll
      for (int k = M - 1; k >= 0; --k) v = v * Tn + s[c][k];
      Qg[al][c] = v;
    }
  }
#pragma unroll
  for (int al = 0; al <= G; ++al) {
    if (al < G) {
      ug[al] = Qg[al][1] * rcp64(Qg[al][0]);        // a non-positive density fails the test below
      pg[al] = ph.gm1 * (Qg[al][2] - 0.5 * Qg[al][1] * ug[al]);
      ok = ok && positive(Qg[al][0]) && positive(pg[al]);
    } else {
      ok = ok && admissible(g, Qg[al][0], Qg[al][1], Qg[al][2]);
    }
  }
  if (!ok) {
    truncated = true;
#pragma unroll
    for (int al = 0; al <= G; ++al) {
      Qg[al][0] = Q0[0]; Qg[al][1] = Q0[1]; Qg[al][2] = Q0[2];
      if (al < G) { ug[al] = W0.u; pg[al] = W0.p; }
    }
  }
  F[0] = F[1] = F[2] = 0.0;
#pragma unroll
  for (int al = 0; al < G; ++al) {
    const double w = Gauss<M>::weight(al);
    F[0] += w * Qg[al][1];
    F[1] += w * (Qg[al][1] * ug[al] + pg[al]);
    F[2] += w * (ug[al] * (Qg[al][2] + pg[al]));
  }
  gnew[0] = Qg[G][0]; gnew[1] = Qg[G][1]; gnew[2] = Qg[G][2];
  return ST_OK;
}

// ---------------------------------------------------------------------------
// Numerical source of a cell (eq. eq:source, Section 2): the space-time
// average of S(Q) over the cell and [0, dt], with Q the cell's own evolution,
// the Cauchy-Kovalevskaya series with the source at the cell centre from its
// reconstruction.  S is linear here, so the average of S(Q) is S of the
// average of the series, taken exactly from its moments: over xi in
// [-1/2, 1/2] the average of xi^a is 2^-a / (a+1) for even a (0 for odd),
// over T in [0, nu] that of T^b is nu^b / (b+1).  b: the zero-mean-basis
// coefficients of the reconstruction (degree 0 after a fallback).
// ---------------------------------------------------------------------------
template <int M>
GRP_HD __forceinline__ void centre_taylor(const double b[5], double t[M + 1])
{
  t[0] = b[0] - b[2] * (1.0 / 12.0) - b[4] * (1.0 / 80.0);
#pragma unroll
  for (int k = 1; k <= M; ++k) t[k] = b[k];
}

template <int M>
GRP_HD __forceinline__ double series_average(const double q[Tri<M>::N], double nu)
{
  using T = Tri<M>;
  double acc = 0.0;
#pragma unroll
  for (int a = 0; a <= M; a += 2) {
    const double mx = a == 0 ? 1.0 : (a == 2 ? 1.0 / 12.0 : 1.0 / 80.0);
    double v = q[T::idx(a, M - a)] * (1.0 / double(M - a + 1));
#pragma unroll
    for (int b = M - a - 1; b >= 0; --b) v = fma(v, nu, q[T::idx(a, b)] * (1.0 / double(b + 1)));
    acc = fma(mx, v, acc);
  }
  return acc;
}

// advection, S = k q: returns S_i
template <int M>
GRP_HD __forceinline__ double cell_source_adv(const double b[5], double lam, double nu, double k, double dx)
{
  using T = Tri<M>;
  double t[M + 1], q[T::N];
  centre_taylor<M>(b, t);
#pragma unroll
  for (int a = 0; a <= M; ++a) q[T::idx(a, 0)] = t[a];
  ck_adv_src<M>(lam, k * dx, q);
  return k * series_average<M>(q, nu);
}

// Euler, S = (0, -g rho, -g m).  A centre state that is not admissible is
// replaced by the cell average, held constant before the evolution.
template <int M>
GRP_HD __forceinline__ void cell_source_euler(const Phys& ph, const double b[3][5], double nu, double dx,
                                              double S[3])
{
  using T = Tri<M>;
  double t[3][M + 1];
#pragma unroll
  for (int c = 0; c < 3; ++c) centre_taylor<M>(b[c], t[c]);
  if (!admissible(ph.gamma, t[0][0], t[1][0], t[2][0])) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      t[c][0] = b[c][0];
#pragma unroll
      for (int k = 1; k <= M; ++k) t[c][k] = 0.0;
    }
  }
  double rho[T::N], m[T::N], E[T::N], s[3][M + 1];
#pragma unroll
  for (int a = 0; a <= M; ++a) { rho[T::idx(a, 0)] = t[0][a]; m[T::idx(a, 0)] = t[1][a]; E[T::idx(a, 0)] = t[2][a]; }
  const double ir = 1.0 / rho[0];
  const double u0 = m[0] * ir, p0 = ph.gm1 * (E[0] - 0.5 * m[0] * u0);
  ck_euler<M, true>(ph.gm1, rho, m, E, s, ir, u0, p0, -ph.src_k * dx);
  S[0] = 0.0;
  S[1] = -ph.src_k * series_average<M>(rho, nu);
  S[2] = -ph.src_k * series_average<M>(m, nu);
}

}  // namespace grp
