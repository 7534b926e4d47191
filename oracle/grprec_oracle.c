/*
 * ORACLE — test infrastructure only; see grprec_oracle.h.
 *
 * Plain FP64, no blocking, no fusion: every function follows one passage of
 * the paper (arXiv 2602.21911) or a textbook definition, cited beside it, in
 * the order the method states it.  Readings of points the paper leaves open
 * are marked READING and listed in the design notes of the repository.
 *
 * Built with -O2 -ffp-contract=off so that x86 and Arm hosts give the same
 * bits.  The file is valid C99 and C++ (an op-counting build includes it with
 * `real` defined as a counting type).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "grprec_oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef OR_REAL_DEFINED
typedef double real;
#define OR_DATA(x) (x)        /* marks a value read from the state (op counting) */
#endif
#ifndef OR_PHASE
#define OR_PHASE(k)           /* op counting: 0 CFL, 1 reconstruction + GRP, 2 update + repair */
#endif
#ifndef OR_LEADING_RP
#define OR_LEADING_RP(L, R, k) /* op counting: brackets the leading Riemann problem (k = 0 before, 1 after) */
#endif

#define MAXM 4
#define MAXC 3
/* READING: signs decided in the Riemann solvers (the contact side, the upwind
 * side of a derivative Riemann problem) treat |speed| <= OR_TIE x (wave-speed
 * scale) as zero, so a stationary contact is not decided by rounding noise. */
#define OR_TIE 1e-10
#ifndef OR_DMP_REL
#define OR_DMP_REL 1e-2
#endif
#ifndef OR_MAX_REPAIR
#define OR_MAX_REPAIR 4
#endif

/* ------------------------------------------------------------------------- */
/* Small dense linear algebra: Gaussian elimination with partial pivoting.   */
/* (data-independent systems only, so plain double)                          */
/* ------------------------------------------------------------------------- */
static int solve_dense_d(int n, double *A /* n*n row-major, destroyed */, double *x /* rhs in, sol out */)
{
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = fabs(A[k * n + k]);
    for (int r = k + 1; r < n; ++r) {
      double v = fabs(A[r * n + k]);
      if (v > best) { best = v; piv = r; }
    }
    if (!(best > 0)) return -1;
    if (piv != k) {
      for (int c = 0; c < n; ++c) { double tmp = A[k * n + c]; A[k * n + c] = A[piv * n + c]; A[piv * n + c] = tmp; }
      double tmp = x[k]; x[k] = x[piv]; x[piv] = tmp;
    }
    for (int r = k + 1; r < n; ++r) {
      double f = A[r * n + k] / A[k * n + k];
      for (int c = k; c < n; ++c) A[r * n + c] = A[r * n + c] - f * A[k * n + c];
      x[r] = x[r] - f * x[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = x[k];
    for (int c = k + 1; c < n; ++c) s = s - A[k * n + c] * x[c];
    x[k] = s / A[k * n + k];
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Section 3.1, GRPrec.  Polynomial p(xi) = sum_k coef[k] xi^k on cell i,     */
/* xi = (x - x_i)/dx in [-1/2, 1/2].  Every condition of the paper is a row:  */
/*   point value  p(xi0)                    -> [xi0^k]                        */
/*   cell average (1/dx) int p dx over [a,b] -> [(b^{k+1}-a^{k+1})/(k+1)]      */
/* ------------------------------------------------------------------------- */
static void row_point_d(int M, double xi0, double *row)
{
  double v = 1;
  for (int k = 0; k <= M; ++k) { row[k] = v; v = v * xi0; }
}

static void row_average_d(int M, double a, double b, double *row)
{
  double pa = a, pb = b;
  for (int k = 0; k <= M; ++k) { row[k] = (pb - pa) / (k + 1); pa = pa * a; pb = pb * b; }
}

/*
 * Degree 1 (first-degree paragraph of Section 3.1): least squares on the two
 *   interface values, cell-i conservation held by a Lagrange multiplier.
 * Degree 2: both interface values and cell-i conservation imposed exactly.
 * Degree 3: least squares on the two interface values and the averages of
 *   cells i-1 and i+1, cell-i conservation by a Lagrange multiplier.
 * Degree 4: both interface values and conservation in cells i-1, i, i+1.
 * READING: the least-squares terms are unweighted, exactly as the functionals
 * are printed.  The minimiser of |A c - b|^2 subject to C c = d solves the
 * KKT system [2 A^T A, -C^T; C, 0] [c; mu] = [2 A^T b; d].
 */
static int recon_kkt(int M, const double *qbar, const double *g, double *coef)
{
  double Arows[4][MAXM + 1], b[4];
  double Crows[5][MAXM + 1], d[5];
  int nA = 0, nC = 0;
  const double half = 0.5, three_half = 1.5;
  if (M < 1 || M > MAXM) return -1;

  if (M == 1 || M == 3) {
    row_point_d(M, -half, Arows[nA]); b[nA++] = g[0];
    row_point_d(M, half, Arows[nA]); b[nA++] = g[1];
    if (M == 3) {
      row_average_d(M, half, three_half, Arows[nA]); b[nA++] = qbar[2];
      row_average_d(M, -three_half, -half, Arows[nA]); b[nA++] = qbar[0];
    }
    row_average_d(M, -half, half, Crows[nC]); d[nC++] = qbar[1];
  } else {
    row_point_d(M, -half, Crows[nC]); d[nC++] = g[0];
    row_point_d(M, half, Crows[nC]); d[nC++] = g[1];
    row_average_d(M, -half, half, Crows[nC]); d[nC++] = qbar[1];
    if (M == 4) {
      row_average_d(M, -three_half, -half, Crows[nC]); d[nC++] = qbar[0];
      row_average_d(M, half, three_half, Crows[nC]); d[nC++] = qbar[2];
    }
  }

  int nu = M + 1, n = nu + nC;
  double K[(MAXM + 1 + 5) * (MAXM + 1 + 5)], rhs[MAXM + 1 + 5];
  for (int i = 0; i < n * n; ++i) K[i] = 0;
  for (int i = 0; i < n; ++i) rhs[i] = 0;
  for (int r = 0; r < nu; ++r) {
    for (int c = 0; c < nu; ++c) {
      double s = 0;
      for (int k = 0; k < nA; ++k) s = s + Arows[k][r] * Arows[k][c];
      K[r * n + c] = 2 * s;
    }
    double s = 0;
    for (int k = 0; k < nA; ++k) s = s + Arows[k][r] * b[k];
    rhs[r] = 2 * s;
    for (int j = 0; j < nC; ++j) K[r * n + nu + j] = -Crows[j][r];
  }
  for (int j = 0; j < nC; ++j) {
    for (int c = 0; c < nu; ++c) K[(nu + j) * n + c] = Crows[j][c];
    rhs[nu + j] = d[j];
  }
  if (solve_dense_d(n, K, rhs) != 0) return -1;
  for (int k = 0; k <= M; ++k) coef[k] = rhs[k];
  for (int k = M + 1; k <= MAXM; ++k) coef[k] = 0;
  return 0;
}

/* The minimiser is linear in the data (q_{i-1}, q_i, q_{i+1}, g_{i-1/2},
 * g_{i+1/2}); column j of the operator is the KKT solution for unit datum j.
 * The operator depends on M only and is built once. */
static double recon_op[MAXM + 1][MAXM + 1][5];
static int recon_op_ready[MAXM + 1];

static const double (*recon_operator(int M))[5]
{
  if (!recon_op_ready[M]) {
    for (int j = 0; j < 5; ++j) {
      double unit[5] = { 0, 0, 0, 0, 0 }, cf[MAXM + 1];
      unit[j] = 1;
      recon_kkt(M, unit, unit + 3, cf);
      for (int k = 0; k <= MAXM; ++k) recon_op[M][k][j] = cf[k];
    }
    recon_op_ready[M] = 1;
  }
  return (const double (*)[5])recon_op[M];
}

/* coefficients of cell i from data = {q_{i-1}, q_i, q_{i+1}, g_{i-1/2}, g_{i+1/2}} */
static void recon_apply(int M, const real *data, real *coef)
{
  const double (*op)[5] = recon_operator(M);
  for (int k = 0; k <= MAXM; ++k) {
    real s = 0;
    for (int j = 0; j < 5; ++j)
      if (op[k][j] != 0) s = s + op[k][j] * data[j];
    coef[k] = k <= M ? s : (real)0;
  }
}

int or_recon(int M, const double *qbar, const double *g, double *coef)
{
  if (M < 1 || M > MAXM) return -1;
  real data[5] = { qbar[0], qbar[1], qbar[2], g[0], g[1] }, cf[MAXM + 1];
  recon_apply(M, data, cf);
  for (int k = 0; k <= MAXM; ++k) coef[k] = (double)cf[k];
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Sections 3.3-3.4, GRPrecNL: p_i = beta_L p_L + beta_C p_C + beta_R p_R,    */
/* beta_k = omega_k / sum omega, omega_k = lambda_k / (eps + OI_k)^r with     */
/* r = 4, eps = 1e-14, lambda_L = lambda_R = 1, lambda_C = 1e9; p_C is the    */
/* linear GRPrec polynomial, p_L and p_R the one-sided polynomials of the     */
/* paragraphs for each degree (every one conserves cell i):                  */
/*   degree 1: p_L interpolates g_{i-1/2}; p_R interpolates g_{i+1/2}         */
/*   degree 2: p_L conserves cell i-1, interpolates g_{i+1/2};               */
/*             p_R conserves cell i+1, interpolates g_{i-1/2}                */
/*   degree 3: both conserve cells i-1, i+1; p_L interpolates g_{i-1/2},     */
/*             p_R interpolates g_{i+1/2}                                     */
/*   degree 4: both conserve cells i-1, i+1; p_L interpolates g_{i-1/2} and  */
/*             g_{i-3/2}, p_R interpolates g_{i+1/2} and g_{i+3/2}           */
/* OI_k = sum_{l=1..M} int_cell (d^l p_k/dx^l)^2 dx^{2l} dx, which in xi is   */
/* dx * sum_l int_{-1/2}^{1/2} (d^l p_k/dxi^l)^2 dxi (READING: the printed     */
/* weight dx^{2l} with the measure dx, taken literally).                      */
/* Data order: d7 = {q_{i-1}, q_i, q_{i+1}, g_{i-3/2}, g_{i-1/2}, g_{i+1/2},  */
/* g_{i+3/2}}.                                                                */
/* ------------------------------------------------------------------------- */
#define OR_NL_R 4
#define OR_NL_EPS 1e-14
#define OR_NL_LAMBDA_C 1e9

static int side_system(int M, int side, const double *d7, double *coef)
{
  double A[(MAXM + 1) * (MAXM + 1)], x[MAXM + 1];
  int n = 0;
  const double h = 0.5, h3 = 1.5;
#define ROW_AVG(a, b, v) do { row_average_d(M, a, b, A + n * (M + 1)); x[n++] = (v); } while (0)
#define ROW_PT(z, v) do { row_point_d(M, z, A + n * (M + 1)); x[n++] = (v); } while (0)
  ROW_AVG(-h, h, d7[1]);                                   /* cell i */
  if (M == 1) {
    if (side == 0) ROW_PT(-h, d7[4]); else ROW_PT(h, d7[5]);
  } else if (M == 2) {
    if (side == 0) { ROW_AVG(-h3, -h, d7[0]); ROW_PT(h, d7[5]); }
    else { ROW_AVG(h, h3, d7[2]); ROW_PT(-h, d7[4]); }
  } else {
    ROW_AVG(-h3, -h, d7[0]);
    ROW_AVG(h, h3, d7[2]);
    if (side == 0) { ROW_PT(-h, d7[4]); if (M == 4) ROW_PT(-h3, d7[3]); }
    else { ROW_PT(h, d7[5]); if (M == 4) ROW_PT(h3, d7[6]); }
  }
#undef ROW_AVG
#undef ROW_PT
  if (n != M + 1) return -1;
  if (solve_dense_d(n, A, x) != 0) return -1;
  for (int k = 0; k <= MAXM; ++k) coef[k] = k <= M ? x[k] : 0;
  return 0;
}

/* p_L, p_R are linear in the 7 data: operator columns from unit data, per M */
static double side_op[2][MAXM + 1][MAXM + 1][7];
static int side_op_ready[MAXM + 1];

static void nl_side_apply(int M, int side, const real *d7, real *coef)
{
  if (!side_op_ready[M]) {
    for (int sd = 0; sd < 2; ++sd)
      for (int j = 0; j < 7; ++j) {
        double unit[7] = { 0, 0, 0, 0, 0, 0, 0 }, cf[MAXM + 1];
        unit[j] = 1;
        side_system(M, sd, unit, cf);
        for (int k = 0; k <= MAXM; ++k) side_op[sd][M][k][j] = cf[k];
      }
    side_op_ready[M] = 1;
  }
  for (int k = 0; k <= MAXM; ++k) {
    real s = 0;
    for (int j = 0; j < 7; ++j)
      if (side_op[side][M][k][j] != 0) s = s + side_op[side][M][k][j] * d7[j];
    coef[k] = k <= M ? s : (real)0;
  }
}

/* dx * sum_{l=1..M} int_{-1/2}^{1/2} (p^{(l)}(xi))^2 dxi, by exact monomial integration */
static real oscillation_indicator(int M, const real *coef, real dx)
{
  real total = 0;
  for (int l = 1; l <= M; ++l) {
    real d[MAXM + 1];                          /* d^l/dxi^l in monomials */
    int nd = M - l;
    for (int k = 0; k <= nd; ++k) {
      real fall = 1;
      for (int r = 0; r < l; ++r) fall = fall * (k + l - r);
      d[k] = coef[k + l] * fall;
    }
    for (int a = 0; a <= nd; ++a)
      for (int b = 0; b <= nd; ++b) {
        int e = a + b;
        if (e % 2) continue;                   /* odd powers integrate to zero */
        double mono = 2.0 * pow(0.5, e + 1) / (e + 1);
        total = total + d[a] * d[b] * mono;
      }
  }
  return dx * total;
}

/* GRPrecNL polynomial of one scalar component; beta (may be NULL) gets the weights L, C, R */
static void recon_nl(int M, const real *d7, real dx, real *coef, real *beta)
{
  real pk[3][MAXM + 1];
  real d5[5] = { d7[0], d7[1], d7[2], d7[4], d7[5] };
  nl_side_apply(M, 0, d7, pk[0]);
  recon_apply(M, d5, pk[1]);
  nl_side_apply(M, 1, d7, pk[2]);
  const double lam[3] = { 1.0, OR_NL_LAMBDA_C, 1.0 };
  real om[3], sum = 0;
  for (int k = 0; k < 3; ++k) {
    real b = OR_NL_EPS + oscillation_indicator(M, pk[k], dx);
    real b2 = b * b;
    om[k] = lam[k] / (b2 * b2);                /* r = 4 */
    sum = sum + om[k];
  }
  for (int q = 0; q <= MAXM; ++q) coef[q] = 0;
  for (int k = 0; k < 3; ++k) {
    real w = om[k] / sum;
    if (beta) beta[k] = w;
    for (int q = 0; q <= M; ++q) coef[q] = coef[q] + w * pk[k][q];
  }
}

int or_recon_nl(int M, const double *d7, double dx, double *coef, double *beta)
{
  if (M < 1 || M > MAXM) return -1;
  real d[7], cf[MAXM + 1], bt[3];
  for (int j = 0; j < 7; ++j) d[j] = d7[j];
  recon_nl(M, d, dx, cf, bt);
  for (int k = 0; k <= MAXM; ++k) coef[k] = (double)cf[k];
  if (beta) for (int k = 0; k < 3; ++k) beta[k] = (double)bt[k];
  return 0;
}

/* k-th xi-derivative of the polynomial at xi0 */
static real poly_deriv(int M, const real *coef, int k, real xi0)
{
  real s = 0;
  for (int j = M; j >= k; --j) {
    real fall = 1;
    for (int r = 0; r < k; ++r) fall = fall * (j - r);
    s = s * xi0 + coef[j] * fall;
  }
  return s;
}

/* ------------------------------------------------------------------------- */
/* Euler equations, ideal gas (Section 4.3): Q = (rho, rho u, E),            */
/* F = (rho u, rho u^2 + p, u (E + p)), E = rho (u^2/2 + e), e = p/((g-1) rho) */
/* ------------------------------------------------------------------------- */
static void cons_to_prim(real gamma, const real *Q, real *W)
{
  real rho = Q[0];
  real u = Q[1] / rho;
  real p = (gamma - 1) * (Q[2] - 0.5 * Q[1] * u);
  W[0] = rho; W[1] = u; W[2] = p;
}

static void prim_to_cons(real gamma, const real *W, real *Q)
{
  Q[0] = W[0];
  Q[1] = W[0] * W[1];
  Q[2] = W[2] / (gamma - 1) + 0.5 * W[0] * W[1] * W[1];
}

static void euler_flux(real gamma, const real *Q, real *F)
{
  real W[3];
  cons_to_prim(gamma, Q, W);
  F[0] = Q[1];
  F[1] = Q[1] * W[1] + W[2];
  F[2] = W[1] * (Q[2] + W[2]);
}

static int euler_admissible(real gamma, const real *Q)
{
  real W[3];
  if (!(Q[0] > 0)) return 0;
  cons_to_prim(gamma, Q, W);
  return W[2] > 0;
}

/* Characteristic variables of the Euler equations at state Q (Section 3.1:
 * systems are reconstructed in characteristic variables): right eigenvectors
 * of the flux Jacobian as the columns of R (textbook form, eigenvalues u - c,
 * u, u + c), and L = R^{-1} by the adjugate. */
static void char_basis(real gamma, const real *Q, real R[3][3], real L[3][3])
{
  real W[3];
  cons_to_prim(gamma, Q, W);
  real u = W[1], c = sqrt(gamma * W[2] / W[0]), H = (Q[2] + W[2]) / W[0];
  R[0][0] = 1;         R[0][1] = 1;             R[0][2] = 1;
  R[1][0] = u - c;     R[1][1] = u;             R[1][2] = u + c;
  R[2][0] = H - u * c; R[2][1] = 0.5 * u * u;   R[2][2] = H + u * c;
  real cof[3][3];
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) {
      int r1 = (r + 1) % 3, r2 = (r + 2) % 3, k1 = (k + 1) % 3, k2 = (k + 2) % 3;
      cof[r][k] = R[r1][k1] * R[r2][k2] - R[r1][k2] * R[r2][k1];
    }
  real det = R[0][0] * cof[0][0] + R[0][1] * cof[0][1] + R[0][2] * cof[0][2];
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) L[r][k] = cof[k][r] / det;
}

int or_char_basis(double gamma, const double *Q, double *R, double *L)
{
  real q[3] = { Q[0], Q[1], Q[2] }, r[3][3], l[3][3];
  char_basis(gamma, q, r, l);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) { R[a * 3 + b] = (double)r[a][b]; L[a * 3 + b] = (double)l[a][b]; }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Exact Riemann solver for the ideal gas (textbook solver; Section 4.1 takes */
/* its interface data from classical Riemann solutions).                     */
/* ------------------------------------------------------------------------- */
/* pressure function f_K(p) and its derivative */
static void pressure_function(real gamma, real p, const real *W, real c, real *f, real *df)
{
  real rhoK = W[0], pK = W[2];
  if (p > pK) { /* shock */
    real A = 2 / ((gamma + 1) * rhoK);
    real B = (gamma - 1) / (gamma + 1) * pK;
    real s = sqrt(A / (p + B));
    *f = (p - pK) * s;
    *df = s * (1 - (p - pK) / (2 * (B + p)));
  } else { /* rarefaction */
    real ratio = p / pK;
    *f = 2 * c / (gamma - 1) * (pow(ratio, (gamma - 1) / (2 * gamma)) - 1);
    *df = 1 / (rhoK * c) * pow(ratio, -(gamma + 1) / (2 * gamma));
  }
}

/*
 * Newton on f(p) = f_L(p) + f_R(p) + u_R - u_L.
 * READING (the paper is silent): start from PVRS floored at 1e-14 max(pL,pR)
 * (or from the two-rarefaction value, or from a given guess); stop when
 * 2|p_{k+1}-p_k|/(p_{k+1}+p_k) < rtol and then take one more iteration; a
 * non-positive iterate halves the step towards the previous iterate.
 */
static int star_pressure(real gamma, const real *WL, const real *WR, int guess_kind, real guess,
                         real rtol, int max_iter, real *pstar, real *ustar, int *iters)
{
  real cL = sqrt(gamma * WL[2] / WL[0]);
  real cR = sqrt(gamma * WR[2] / WR[0]);
  real du = WR[1] - WL[1];
  *iters = 0;
  if (2 * (cL + cR) / (gamma - 1) <= du) return OR_VACUUM;

  real p;
  real pfloor = 1e-14 * (WL[2] > WR[2] ? WL[2] : WR[2]);
  if (guess_kind == OR_GUESS_GIVEN && guess > 0 && isfinite((double)guess)) {
    p = guess;
  } else if (guess_kind == OR_GUESS_TRRS) {
    real z = (gamma - 1) / (2 * gamma);
    real num = cL + cR - 0.5 * (gamma - 1) * du;
    real den = cL * pow(WL[2], -z) + cR * pow(WR[2], -z);
    p = pow(num / den, 1 / z);
  } else {
    real ppv = 0.5 * (WL[2] + WR[2]) - 0.125 * du * (WL[0] + WR[0]) * (cL + cR);
    p = ppv > pfloor ? ppv : pfloor;
  }
  if (!(p > pfloor)) p = pfloor;

  int converged = 0, it = 0;
  while (it < max_iter) {
    real fL, dfL, fR, dfR;
    pressure_function(gamma, p, WL, cL, &fL, &dfL);
    pressure_function(gamma, p, WR, cR, &fR, &dfR);
    real step = -(fL + fR + du) / (dfL + dfR);
    real pn = p + step;
    for (int h = 0; h < 64 && !(pn > 0); ++h) { step = 0.5 * step; pn = p + step; }
    ++it;
    real change = 2 * fabs(pn - p) / (pn + p);
    p = pn;
    if (converged) break;          /* the one extra iteration is done */
    if (change < rtol) converged = 1;
  }
  *iters = it;
  if (!converged) return OR_NEWTON_NO_CONV;
  real fL, dfL, fR, dfR;
  pressure_function(gamma, p, WL, cL, &fL, &dfL);
  pressure_function(gamma, p, WR, cR, &fR, &dfR);
  *pstar = p;
  *ustar = 0.5 * (WL[1] + WR[1]) + 0.5 * (fR - fL);
  return OR_OK;
}

/* Self-similar solution sampled at x/t = 0.  READING: a contact speed u* with
 * |u*| <= OR_TIE (c_L + c_R) counts as stationary and takes the left side. */
static void sample_at_zero(real gamma, const real *WL, const real *WR, real pstar, real ustar, real *W)
{
  real g1 = (gamma - 1) / (2 * gamma), g6 = (gamma - 1) / (gamma + 1);
  real tie = OR_TIE * (sqrt(gamma * WL[2] / WL[0]) + sqrt(gamma * WR[2] / WR[0]));
  if (ustar >= -tie) {
    real c = sqrt(gamma * WL[2] / WL[0]);
    real ratio = pstar / WL[2];
    if (pstar > WL[2]) {
      real S = WL[1] - c * sqrt((gamma + 1) / (2 * gamma) * ratio + g1);
      if (S >= 0) { W[0] = WL[0]; W[1] = WL[1]; W[2] = WL[2]; return; }
      W[0] = WL[0] * (ratio + g6) / (g6 * ratio + 1); W[1] = ustar; W[2] = pstar; return;
    }
    real head = WL[1] - c;
    if (head >= 0) { W[0] = WL[0]; W[1] = WL[1]; W[2] = WL[2]; return; }
    real cstar = c * pow(ratio, g1);
    real tail = ustar - cstar;
    if (tail < 0) { W[0] = WL[0] * pow(ratio, 1 / gamma); W[1] = ustar; W[2] = pstar; return; }
    /* inside the left fan, at the sonic ray */
    real cs = 2 / (gamma + 1) * (c + (gamma - 1) / 2 * WL[1]);
    W[0] = WL[0] * pow(cs / c, 2 / (gamma - 1));
    W[1] = cs;
    W[2] = WL[2] * pow(cs / c, 2 * gamma / (gamma - 1));
    return;
  }
  real c = sqrt(gamma * WR[2] / WR[0]);
  real ratio = pstar / WR[2];
  if (pstar > WR[2]) {
    real S = WR[1] + c * sqrt((gamma + 1) / (2 * gamma) * ratio + g1);
    if (S <= 0) { W[0] = WR[0]; W[1] = WR[1]; W[2] = WR[2]; return; }
    W[0] = WR[0] * (ratio + g6) / (g6 * ratio + 1); W[1] = ustar; W[2] = pstar; return;
  }
  real head = WR[1] + c;
  if (head <= 0) { W[0] = WR[0]; W[1] = WR[1]; W[2] = WR[2]; return; }
  real cstar = c * pow(ratio, g1);
  real tail = ustar + cstar;
  if (tail > 0) { W[0] = WR[0] * pow(ratio, 1 / gamma); W[1] = ustar; W[2] = pstar; return; }
  real cs = 2 / (gamma + 1) * (c - (gamma - 1) / 2 * WR[1]);
  W[0] = WR[0] * pow(cs / c, 2 / (gamma - 1));
  W[1] = -cs;
  W[2] = WR[2] * pow(cs / c, 2 * gamma / (gamma - 1));
}

/* Two rarefactions separated by vacuum (the data generate vacuum), sampled at
 * x/t = 0 (textbook vacuum-generation solution). */
static void sample_vacuum_at_zero(real gamma, const real *WL, const real *WR, real *W)
{
  real cL = sqrt(gamma * WL[2] / WL[0]), cR = sqrt(gamma * WR[2] / WR[0]);
  real tailL = WL[1] + 2 * cL / (gamma - 1), tailR = WR[1] - 2 * cR / (gamma - 1);
  if (WL[1] - cL >= 0) { W[0] = WL[0]; W[1] = WL[1]; W[2] = WL[2]; return; }
  if (tailL > 0) {                  /* inside the left fan */
    real cs = 2 / (gamma + 1) * (cL + (gamma - 1) / 2 * WL[1]);
    W[0] = WL[0] * pow(cs / cL, 2 / (gamma - 1));
    W[1] = cs;
    W[2] = WL[2] * pow(cs / cL, 2 * gamma / (gamma - 1));
    return;
  }
  if (WR[1] + cR <= 0) { W[0] = WR[0]; W[1] = WR[1]; W[2] = WR[2]; return; }
  if (tailR < 0) {                  /* inside the right fan */
    real cs = 2 / (gamma + 1) * (cR - (gamma - 1) / 2 * WR[1]);
    W[0] = WR[0] * pow(cs / cR, 2 / (gamma - 1));
    W[1] = -cs;
    W[2] = WR[2] * pow(cs / cR, 2 * gamma / (gamma - 1));
    return;
  }
  W[0] = 0; W[1] = 0; W[2] = 0;      /* vacuum */
}

/* Conserved state at x/t = 0.  With allow_vacuum, vacuum-generating data are
 * sampled (status OR_VACUUM, Q valid); otherwise OR_VACUUM is a failure. */
static int riemann_state(real gamma, const real *QL, const real *QR, int guess_kind, real guess,
                         real rtol, int max_iter, int allow_vacuum, real *Q, int *iters)
{
  real WL[3], WR[3], W[3], ps, us;
  cons_to_prim(gamma, QL, WL);
  cons_to_prim(gamma, QR, WR);
  int st = star_pressure(gamma, WL, WR, guess_kind, guess, rtol, max_iter, &ps, &us, iters);
  if (st == OR_VACUUM && allow_vacuum) {
    sample_vacuum_at_zero(gamma, WL, WR, W);
    prim_to_cons(gamma, W, Q);
    return OR_VACUUM;
  }
  if (st != OR_OK) return st;
  sample_at_zero(gamma, WL, WR, ps, us, W);
  prim_to_cons(gamma, W, Q);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Derivative Riemann problems (Toro-Titarev solver, Section 2): linear RP    */
/* d_t D + A(Q0) d_x D = 0, Godunov state at x/t = 0 in the eigenbasis.      */
/* READING: a zero eigenvalue averages the two sides.                        */
/* ------------------------------------------------------------------------- */
static void deriv_rp(real gamma, const real *Q0, const real *DL, const real *DR, real *D)
{
  real W[3];
  cons_to_prim(gamma, Q0, W);
  real u = W[1], c = sqrt(gamma * W[2] / W[0]);
  real H = (Q0[2] + W[2]) / W[0];
  /* right eigenvectors of the Jacobian, as columns */
  real R[9] = { 1, 1, 1,
                u - c, u, u + c,
                H - u * c, 0.5 * u * u, H + u * c };
  real lam[3] = { u - c, u, u + c };
  real tie = OR_TIE * (fabs(u) + c);   /* READING: |lambda| within this counts as zero */
  /* left eigenvectors (rows of R^{-1}, textbook closed form), with
   * b1 = (gamma-1)/c^2 and b2 = b1 u^2 / 2 */
  real b1 = (gamma - 1) / (c * c), b2 = 0.5 * b1 * u * u;
  real Linv[9] = { 0.5 * (b2 + u / c), -0.5 * (b1 * u + 1 / c), 0.5 * b1,
                   1 - b2, b1 * u, -b1,
                   0.5 * (b2 - u / c), -0.5 * (b1 * u - 1 / c), 0.5 * b1 };
  for (int c0 = 0; c0 < 3; ++c0) D[c0] = 0;
  for (int j = 0; j < 3; ++j) {
    real wl = 0, wr = 0;
    for (int k = 0; k < 3; ++k) { wl = wl + Linv[j * 3 + k] * DL[k]; wr = wr + Linv[j * 3 + k] * DR[k]; }
    real w = lam[j] > tie ? wl : (lam[j] < -tie ? wr : 0.5 * (wl + wr));
    for (int k = 0; k < 3; ++k) D[k] = D[k] + R[k * 3 + j] * w;
  }
}

/* ------------------------------------------------------------------------- */
/* Cauchy-Kovalevskaya by truncated bivariate power series.                  */
/* Q(x,tau) = sum_{a+b<=M} q[a][b] x^a tau^b; the PDE d_tau Q = -d_x F(Q)     */
/* gives q[a][b+1] = -(a+1)/(b+1) f[a+1][b], the series of F built from the   */
/* known q[.][<=b] by series products and the series quotient u = m/rho.     */
/* ------------------------------------------------------------------------- */
#define SIDX(a, b) ((a) * (MAXM + 1) + (b))

/* Source term S(Q) of eq. eq_hyperbolic_system (Section 2).  Both sources
 * built here are linear in Q, so the series of S(Q(x, tau)) is S applied to
 * each coefficient:
 *   OR_SOURCE_LINEAR (advection):  S(q) = k q
 *   OR_SOURCE_GRAVITY (Euler):     S(rho, m, E) = (0, -g rho, -g m), a constant
 *                                  acceleration -g along x
 * A NULL descriptor or OR_SOURCE_NONE is S = 0. */
typedef struct { int kind; real coef; } srcspec;

static void source_apply(const srcspec *S, const real *Q, real *out)
{
  out[0] = out[1] = out[2] = 0;
  if (!S || S->kind == OR_SOURCE_NONE) return;
  if (S->kind == OR_SOURCE_LINEAR) { out[0] = S->coef * Q[0]; return; }
  out[1] = -S->coef * Q[0];
  out[2] = -S->coef * Q[1];
}

static real series_product(const real *x, const real *y, int a, int b)
{
  real s = 0;
  for (int i = 0; i <= a; ++i)
    for (int j = 0; j <= b; ++j) s = s + x[SIDX(i, j)] * y[SIDX(a - i, b - j)];
  return s;
}

/* With a source, d_tau Q = -d_x F(Q) + S(Q) (the PDE of the GRP, eq. eq:GRP):
 * q[a][b+1] = (-(a+1) f[a+1][b] + s[a][b]) / (b+1), s the series of S(Q). */
static void ck_series(int system, real lambda, real gamma, int M, real q[][MAXC], const srcspec *S)
{
  if (system == OR_ADVECTION) {
    for (int b = 0; b < M; ++b)
      for (int a = 0; a + b + 1 <= M; ++a) {
        real sq[3];
        source_apply(S, q[SIDX(a, b)], sq);
        q[SIDX(a, b + 1)][0] = -(real)(a + 1) / (b + 1) * lambda * q[SIDX(a + 1, b)][0];
        if (S && S->kind != OR_SOURCE_NONE) q[SIDX(a, b + 1)][0] = q[SIDX(a, b + 1)][0] + sq[0] / (b + 1);
      }
    return;
  }
  real rho[(MAXM + 1) * (MAXM + 1)], m[(MAXM + 1) * (MAXM + 1)], E[(MAXM + 1) * (MAXM + 1)];
  real u[(MAXM + 1) * (MAXM + 1)], mu[(MAXM + 1) * (MAXM + 1)], p[(MAXM + 1) * (MAXM + 1)];
  real Ep[(MAXM + 1) * (MAXM + 1)], F[3][(MAXM + 1) * (MAXM + 1)];
  for (int i = 0; i < (MAXM + 1) * (MAXM + 1); ++i) {
    rho[i] = m[i] = E[i] = u[i] = mu[i] = p[i] = Ep[i] = 0;
    F[0][i] = F[1][i] = F[2][i] = 0;
  }
  for (int b = 0; b < M; ++b) {
    for (int a = 0; a + b <= M; ++a) {
      rho[SIDX(a, b)] = q[SIDX(a, b)][0];
      m[SIDX(a, b)] = q[SIDX(a, b)][1];
      E[SIDX(a, b)] = q[SIDX(a, b)][2];
    }
    for (int a = 0; a + b <= M; ++a) {
      /* series quotient: rho * u = m */
      real s = m[SIDX(a, b)];
      for (int i = 0; i <= a; ++i)
        for (int j = 0; j <= b; ++j)
          if (i || j) s = s - rho[SIDX(i, j)] * u[SIDX(a - i, b - j)];
      u[SIDX(a, b)] = s / rho[SIDX(0, 0)];
      mu[SIDX(a, b)] = series_product(m, u, a, b);
      p[SIDX(a, b)] = (gamma - 1) * (E[SIDX(a, b)] - 0.5 * mu[SIDX(a, b)]);
      Ep[SIDX(a, b)] = E[SIDX(a, b)] + p[SIDX(a, b)];
      F[0][SIDX(a, b)] = m[SIDX(a, b)];
      F[1][SIDX(a, b)] = mu[SIDX(a, b)] + p[SIDX(a, b)];
      F[2][SIDX(a, b)] = series_product(u, Ep, a, b);
    }
    for (int a = 0; a + b + 1 <= M; ++a) {
      real sq[3];
      source_apply(S, q[SIDX(a, b)], sq);
      for (int c = 0; c < 3; ++c) {
        q[SIDX(a, b + 1)][c] = -(real)(a + 1) / (b + 1) * F[c][SIDX(a + 1, b)];
        if (S && S->kind != OR_SOURCE_NONE) q[SIDX(a, b + 1)][c] = q[SIDX(a, b + 1)][c] + sq[c] / (b + 1);
      }
    }
  }
}

void or_ck_series(int system, double lambda, double gamma, int M, const double *qa0, double *qout)
{
  int C = system == OR_EULER ? 3 : 1;
  real q[(MAXM + 1) * (MAXM + 1)][MAXC];
  for (int i = 0; i < (MAXM + 1) * (MAXM + 1); ++i) q[i][0] = q[i][1] = q[i][2] = 0;
  for (int a = 0; a <= M; ++a)
    for (int c = 0; c < C; ++c) q[SIDX(a, 0)][c] = qa0[a * C + c];
  ck_series(system, lambda, gamma, M, q, 0);
  for (int a = 0; a <= M; ++a)
    for (int b = 0; b <= M; ++b)
      for (int c = 0; c < C; ++c) qout[(a * (M + 1) + b) * C + c] = q[SIDX(a, b)][c];
}

void or_ck_series_src(int system, double lambda, double gamma, int M, int source, double coef,
                      const double *qa0, double *qout)
{
  int C = system == OR_EULER ? 3 : 1;
  srcspec S = { source, coef };
  real q[(MAXM + 1) * (MAXM + 1)][MAXC];
  for (int i = 0; i < (MAXM + 1) * (MAXM + 1); ++i) q[i][0] = q[i][1] = q[i][2] = 0;
  for (int a = 0; a <= M; ++a)
    for (int c = 0; c < C; ++c) q[SIDX(a, 0)][c] = qa0[a * C + c];
  ck_series(system, lambda, gamma, M, q, &S);
  for (int a = 0; a <= M; ++a)
    for (int b = 0; b <= M; ++b)
      for (int c = 0; c < C; ++c) qout[(a * (M + 1) + b) * C + c] = q[SIDX(a, b)][c];
}

/* ------------------------------------------------------------------------- */
/* One GRP_m at an interface (Toro-Titarev structure, Section 2) and its flux */
/* time integral (numerical flux definition, Section 2).                     */
/* READING: G = ceil((M+1)/2) Gauss-Legendre points on [0, dt]; the interface */
/* datum written back is the Taylor value at tau = dt.                       */
/* ------------------------------------------------------------------------- */
static int gauss_rule(int M, real *s, real *w)
{
  int G = (M + 2) / 2;
  if (G == 1) { s[0] = 0; w[0] = 1; }
  else if (G == 2) { s[0] = -1 / sqrt((real)3); s[1] = 1 / sqrt((real)3); w[0] = w[1] = 0.5; }
  else { s[0] = -sqrt((real)0.6); s[1] = 0; s[2] = sqrt((real)0.6); w[0] = 5.0 / 18; w[1] = 8.0 / 18; w[2] = 5.0 / 18; }
  return G;
}

static int grp_interface(int system, real lambda, real gamma, int M, real dt,
                         const real *trL, const real *trR, real rtol, int max_iter, int guess_kind,
                         real *flux, real *gnew, int *iters, int *truncated, const srcspec *S)
{
  int C = system == OR_EULER ? 3 : 1;
  real q[(MAXM + 1) * (MAXM + 1)][MAXC];
  for (int i = 0; i < (MAXM + 1) * (MAXM + 1); ++i) q[i][0] = q[i][1] = q[i][2] = 0;
  *iters = 0;
  *truncated = 0;
  /* leading term: classical Riemann problem of the traces */
  if (system == OR_ADVECTION) {
    for (int k = 0; k <= M; ++k) {
      real D = lambda > 0 ? trL[k] : (lambda < 0 ? trR[k] : 0.5 * (trL[k] + trR[k]));
      real fact = 1;
      for (int r = 2; r <= k; ++r) fact = fact * r;
      q[SIDX(k, 0)][0] = D / fact;
    }
  } else {
    real Q0[3];
    OR_LEADING_RP(trL, trR, 0);
    int st = riemann_state(gamma, trL, trR, guess_kind, 0, rtol, max_iter, 0, Q0, iters);
    OR_LEADING_RP(trL, trR, 1);
    if (st != OR_OK) return st;
    for (int c = 0; c < 3; ++c) q[SIDX(0, 0)][c] = Q0[c];
    for (int k = 1; k <= M; ++k) {
      real D[3];
      deriv_rp(gamma, Q0, trL + k * 3, trR + k * 3, D);
      real fact = 1;
      for (int r = 2; r <= k; ++r) fact = fact * r;
      for (int c = 0; c < 3; ++c) q[SIDX(k, 0)][c] = D[c] / fact;
    }
  }
  ck_series(system, lambda, gamma, M, q, S);

  real s[3], w[3], Qt[MAXC][4];
  int G = gauss_rule(M, s, w);
  for (int al = 0; al <= G; ++al) {     /* G Gauss points, then tau = dt */
    real tau = al < G ? dt * (1 + s[al]) / 2 : dt;
    for (int c = 0; c < C; ++c) {
      real v = 0;
      for (int b = M; b >= 0; --b) v = v * tau + q[SIDX(0, b)][c];
      Qt[c][al] = v;
    }
  }
  if (system == OR_EULER) {
    int ok = 1;
    for (int al = 0; al <= G; ++al) {
      real Qa[3] = { Qt[0][al], Qt[1][al], Qt[2][al] };
      if (!euler_admissible(gamma, Qa)) ok = 0;
    }
    if (!ok) {       /* READING: truncate this interface's series to its leading term */
      *truncated = 1;
      for (int al = 0; al <= G; ++al)
        for (int c = 0; c < 3; ++c) Qt[c][al] = q[SIDX(0, 0)][c];
    }
  }
  for (int c = 0; c < C; ++c) flux[c] = 0;
  for (int al = 0; al < G; ++al) {
    real F[3];
    if (system == OR_EULER) {
      real Qa[3] = { Qt[0][al], Qt[1][al], Qt[2][al] };
      euler_flux(gamma, Qa, F);
    } else {
      F[0] = lambda * Qt[0][al];
    }
    for (int c = 0; c < C; ++c) flux[c] = flux[c] + w[al] * F[c];
  }
  for (int c = 0; c < C; ++c) gnew[c] = Qt[c][G];
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Exported unit entry points                                                */
/* ------------------------------------------------------------------------- */
int or_star_pressure(double gamma, const double *WL, const double *WR, int guess_kind,
                     double guess, double rtol, int max_iter, double *out)
{
  real wl[3] = { WL[0], WL[1], WL[2] }, wr[3] = { WR[0], WR[1], WR[2] }, ps = 0, us = 0;
  int it = 0;
  int st = star_pressure(gamma, wl, wr, guess_kind, guess, rtol, max_iter, &ps, &us, &it);
  out[0] = ps; out[1] = us; out[2] = it;
  return st;
}

int or_riemann_state(double gamma, const double *QL, const double *QR, double rtol, int max_iter,
                     double *Q, int *iters)
{
  real ql[3] = { QL[0], QL[1], QL[2] }, qr[3] = { QR[0], QR[1], QR[2] }, q[3];
  int st = riemann_state(gamma, ql, qr, OR_GUESS_PVRS, 0, rtol, max_iter, 1, q, iters);
  Q[0] = q[0]; Q[1] = q[1]; Q[2] = q[2];
  return st;
}

void or_deriv_rp(double gamma, const double *Q0, const double *DL, const double *DR, double *D)
{
  real q0[3] = { Q0[0], Q0[1], Q0[2] }, dl[3] = { DL[0], DL[1], DL[2] }, dr[3] = { DR[0], DR[1], DR[2] }, d[3];
  deriv_rp(gamma, q0, dl, dr, d);
  D[0] = d[0]; D[1] = d[1]; D[2] = d[2];
}

int or_grp_interface(int system, double lambda, double gamma, int M, double dt,
                     const double *trL, const double *trR, double rtol, int max_iter,
                     int guess_kind, double *flux, double *gnew, int *iters, int *truncated)
{
  int C = system == OR_EULER ? 3 : 1;
  real tl[(MAXM + 1) * MAXC], tr[(MAXM + 1) * MAXC], f[MAXC], g[MAXC];
  for (int i = 0; i < (M + 1) * C; ++i) { tl[i] = trL[i]; tr[i] = trR[i]; }
  int st = grp_interface(system, lambda, gamma, M, dt, tl, tr, rtol, max_iter, guess_kind, f, g,
                         iters, truncated, 0);
  for (int c = 0; c < C; ++c) { flux[c] = f[c]; gnew[c] = g[c]; }
  return st;
}

int or_init_iface(int system, double lambda, double gamma, int n_ifaces,
                  const double *lim_minus, const double *lim_plus, double *iface)
{
  int worst = OR_OK;
  if (system == OR_ADVECTION) {
    for (int j = 0; j < n_ifaces; ++j)
      iface[j] = lambda > 0 ? lim_minus[j] : (lambda < 0 ? lim_plus[j] : 0.5 * (lim_minus[j] + lim_plus[j]));
    return OR_OK;
  }
  for (int j = 0; j < n_ifaces; ++j) {
    real ql[3], qr[3], q[3];
    int it;
    for (int c = 0; c < 3; ++c) { ql[c] = lim_minus[c * n_ifaces + j]; qr[c] = lim_plus[c * n_ifaces + j]; }
    int st = riemann_state(gamma, ql, qr, OR_GUESS_PVRS, 0, 1e-12, 50, 1, q, &it);
    if (st != OR_OK && st != OR_VACUUM) { worst = st; q[0] = ql[0]; q[1] = ql[1]; q[2] = ql[2]; }
    for (int c = 0; c < 3; ++c) iface[c * n_ifaces + j] = q[c];
  }
  return worst;
}

/* ------------------------------------------------------------------------- */
/* The DET GRP solver (the solver of the paper's computations; Section 2 and  */
/* Section 4.1): in each cell a local space-time Galerkin predictor evolves   */
/* the reconstruction over [t^n, t^n + dt]; at each interface classical       */
/* Riemann problems of the two evolved edge values at the time integration   */
/* points give the flux, and the one at the end of the step the interface    */
/* datum.  READING: the predictor is the standard locally implicit one: a     */
/* tensor-product nodal basis of degree M in space and time on M+1 Gauss-     */
/* Legendre points, the time derivative integrated by parts with upwinding   */
/* from the reconstruction at t^n, nodal quadrature, solved by Picard        */
/* iteration until the largest update is below 1e-13 of the largest nodal    */
/* value (at most 64 iterations).  The Riemann problems are solved exactly   */
/* (this build's solver) for the flux and for the interface datum; the        */
/* paper's two-rarefaction estimate for the Euler interface data is not       */
/* taken.  Time points: the M+1 predictor nodes.                              */
/* ------------------------------------------------------------------------- */
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#define DET_N (MAXM + 1)
typedef struct {
  int n;
  double x[DET_N], w[DET_N];            /* Gauss-Legendre nodes and weights on [0, 1] */
  double D[DET_N][DET_N];               /* D[k][a] = phi_a'(x_k) */
  double e0[DET_N], e1[DET_N];          /* phi_a(0), phi_a(1) */
  double Tinv[DET_N][DET_N];            /* inverse of T_lb = phi_l(1) phi_b(1) - w_b phi_l'(x_b) */
} det_basis;

static det_basis det_tab[MAXM + 1];
static int det_ready[MAXM + 1];

static void gauss_legendre01(int n, double *x, double *w)
{
  for (int k = 0; k < n; ++k) {
    double z = cos(M_PI * (k + 0.75) / (n + 0.5)), pp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1, p1 = z;
      for (int j = 2; j <= n; ++j) { double p2 = ((2 * j - 1) * z * p1 - (j - 1) * p0) / j; p0 = p1; p1 = p2; }
      if (n == 1) { p1 = z; p0 = 1; }
      pp = n * (z * p1 - p0) / (z * z - 1);
      double dz = p1 / pp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[n - 1 - k] = 0.5 * (z + 1);
    w[n - 1 - k] = 1.0 / ((1 - z * z) * pp * pp);       /* 2/((1-z^2)P'^2) on [-1,1], halved */
  }
}

static double lagrange(int n, const double *x, int a, double s)
{
  double v = 1;
  for (int j = 0; j < n; ++j) if (j != a) v *= (s - x[j]) / (x[a] - x[j]);
  return v;
}

static double lagrange_d(int n, const double *x, int a, double s)
{
  double tot = 0;
  for (int m = 0; m < n; ++m) {
    if (m == a) continue;
    double v = 1 / (x[a] - x[m]);
    for (int j = 0; j < n; ++j) if (j != a && j != m) v *= (s - x[j]) / (x[a] - x[j]);
    tot += v;
  }
  return tot;
}

static const det_basis *det_basis_for(int M)
{
  if (!det_ready[M]) {
    det_basis *B = &det_tab[M];
    int n = M + 1;
    B->n = n;
    gauss_legendre01(n, B->x, B->w);
    for (int a = 0; a < n; ++a) {
      B->e0[a] = lagrange(n, B->x, a, 0.0);
      B->e1[a] = lagrange(n, B->x, a, 1.0);
      for (int k = 0; k < n; ++k) B->D[k][a] = lagrange_d(n, B->x, a, B->x[k]);
    }
    for (int col = 0; col < n; ++col) {
      double T[DET_N * DET_N], e[DET_N];
      for (int l = 0; l < n; ++l) {
        for (int b = 0; b < n; ++b) T[l * n + b] = B->e1[l] * B->e1[b] - B->w[b] * B->D[b][l];
        e[l] = l == col ? 1 : 0;
      }
      solve_dense_d(n, T, e);
      for (int l = 0; l < n; ++l) B->Tinv[l][col] = e[l];
    }
    det_ready[M] = 1;
  }
  return &det_tab[M];
}

static void phys_flux(int system, real lambda, real gamma, const real *Q, real *F)
{
  if (system == OR_ADVECTION) F[0] = lambda * Q[0];
  else euler_flux(gamma, Q, F);
}

/* Predictor of one cell from its reconstruction (monomial coefficients in
 * xi = s - 1/2 per component); nu = dt/dx.  Out: edge values at the time
 * nodes and at the end of the step, ed[side][g][c] for g = 0..M (nodes) and
 * g = M+1 (tau = 1), side 0 the left edge (s = 0), 1 the right edge.
 * Returns 0, or -1 when a nodal state is inadmissible (Euler). */
static int det_predict(int system, real lambda, real gamma, int M, real nu, const real *coef /* [C][MAXM+1] */,
                       real ed[2][DET_N + 1][MAXC])
{
  const det_basis *B = det_basis_for(M);
  const int n = B->n, C = system == OR_EULER ? 3 : 1;
  real w[DET_N][MAXC], q[DET_N][DET_N][MAXC], f[DET_N][DET_N][MAXC];
  for (int k = 0; k < n; ++k)
    for (int c = 0; c < C; ++c) {
      real xi = B->x[k] - 0.5, v = 0;
      for (int j = M; j >= 0; --j) v = v * xi + coef[c * (MAXM + 1) + j];
      w[k][c] = v;
      for (int l = 0; l < n; ++l) q[k][l][c] = v;
    }
  for (int it = 0; it < 64; ++it) {
    for (int k = 0; k < n; ++k)
      for (int l = 0; l < n; ++l) {
        if (system == OR_EULER && !euler_admissible(gamma, q[k][l])) return -1;
        phys_flux(system, lambda, gamma, q[k][l], f[k][l]);
      }
    real diff = 0, scale = 0;
    real qn[DET_N][DET_N][MAXC];
    for (int k = 0; k < n; ++k)
      for (int c = 0; c < C; ++c) {
        real rhs[DET_N];
        for (int l = 0; l < n; ++l) {
          real df = 0;
          for (int a = 0; a < n; ++a) df = df + B->D[k][a] * f[a][l][c];
          rhs[l] = B->e0[l] * w[k][c] - nu * B->w[l] * df;
        }
        for (int l = 0; l < n; ++l) {
          real v = 0;
          for (int b = 0; b < n; ++b) v = v + B->Tinv[l][b] * rhs[b];
          qn[k][l][c] = v;
          real dv = fabs(v - q[k][l][c]);
          if (dv > diff) diff = dv;
          if (fabs(v) > scale) scale = fabs(v);
        }
      }
    memcpy(q, qn, sizeof(q));
    if (diff <= 1e-13 * scale) break;
  }
  if (system == OR_EULER)
    for (int k = 0; k < n; ++k)
      for (int l = 0; l < n; ++l)
        if (!euler_admissible(gamma, q[k][l])) return -1;
  for (int side = 0; side < 2; ++side) {
    const double *ex = side ? B->e1 : B->e0;
    for (int c = 0; c < C; ++c) {
      for (int g = 0; g < n; ++g) {
        real v = 0;
        for (int a = 0; a < n; ++a) v = v + ex[a] * q[a][g][c];
        ed[side][g][c] = v;
      }
      real v = 0;
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) v = v + ex[a] * B->e1[b] * q[a][b][c];
      ed[side][n][c] = v;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* One step of one domain: FV update (eq. eq_finite_volume, Section 2).      */
/* ------------------------------------------------------------------------- */
typedef struct {
  int system; real lambda, gamma; int M; real cfl;
  real rtol; int max_iter; int guess_kind; int dt_hold;
  int recon;                  /* OR_RECON_GRPREC or OR_RECON_GRPRECNL */
  int solver;                 /* OR_SOLVER_TT or OR_SOLVER_DET */
  srcspec src;                /* source term S(Q) (Section 2), kind OR_SOURCE_* */
} params;

/* Time-step rule (Section 4.1): dt = C dx / S_max, S_max over the cell averages.
 * READING: the last step is clipped to t_end; dt is recomputed every dt_hold steps. */
static real domain_smax(const params *P, int N, const real *avg, long stride)
{
  if (P->system == OR_ADVECTION) return fabs(P->lambda);
  real smax = 0;
  for (int i = 0; i < N; ++i) {
    real Q[3] = { avg[i], avg[stride + i], avg[2 * stride + i] }, W[3];
    cons_to_prim(P->gamma, Q, W);
    real s = fabs(W[1]) + sqrt(P->gamma * W[2] / W[0]);
    if (s > smax) smax = s;
  }
  return smax;
}

/* Relaxed discrete maximum principle on density and pressure: the candidate
 * must lie within [min - d, max + d] of the old averages of cells i-1, i,
 * i+1 (boundary rule for the neighbours), d = OR_DMP_REL * max(|min|, |max|). */
static int dmp_ok(real gamma, int N, int bc, int i, const real *avg, long cstride, const real *Qc)
{
  int nb[3] = { i - 1, i, i + 1 };
  if (bc == OR_BC_PERIODIC) { nb[0] = (i - 1 + N) % N; nb[2] = (i + 1) % N; }
  else { if (nb[0] < 0) nb[0] = 0; if (nb[2] > N - 1) nb[2] = N - 1; }
  real W[3], lo[2], hi[2];
  for (int k = 0; k < 3; ++k) {
    real Q[3] = { avg[nb[k]], avg[cstride + nb[k]], avg[2 * cstride + nb[k]] };
    cons_to_prim(gamma, Q, W);
    if (k == 0 || W[0] < lo[0]) lo[0] = W[0];
    if (k == 0 || W[0] > hi[0]) hi[0] = W[0];
    if (k == 0 || W[2] < lo[1]) lo[1] = W[2];
    if (k == 0 || W[2] > hi[1]) hi[1] = W[2];
  }
  real Wc[3];
  cons_to_prim(gamma, Qc, Wc);
  real v[2] = { Wc[0], Wc[2] };
  for (int q = 0; q < 2; ++q) {
    real d = OR_DMP_REL * (fabs(lo[q]) > fabs(hi[q]) ? fabs(lo[q]) : fabs(hi[q]));
    if (!(v[q] >= lo[q] - d && v[q] <= hi[q] + d)) return 0;
  }
  return 1;
}

/* First-order Godunov flux at interface j: exact Riemann problem of the two
 * adjacent cell averages (a transmissive end uses the boundary cell twice). */
static int first_order_interface(const params *P, int N, int bc, int j, const real *avg, long cstride,
                                 real *flux, real *gnew, long long *st)
{
  int cl = bc == OR_BC_PERIODIC ? (j - 1 + N) % N : (j - 1 < 0 ? 0 : j - 1);
  int cr = bc == OR_BC_PERIODIC ? j : (j > N - 1 ? N - 1 : j);
  real QL[3], QR[3], Q0[3];
  for (int c = 0; c < 3; ++c) { QL[c] = avg[c * cstride + cl]; QR[c] = avg[c * cstride + cr]; }
  int it = 0;
  int s = riemann_state(P->gamma, QL, QR, P->guess_kind, 0, P->rtol, P->max_iter, 1, Q0, &it);
  st[OR_ST_RS_CALLS] += 1;
  st[OR_ST_NEWTON_SUM] += it;
  if (it > st[OR_ST_NEWTON_MAX]) st[OR_ST_NEWTON_MAX] = it;
  st[OR_ST_LOW_ORDER] += 1;
  if (s != OR_OK && s != OR_VACUUM) return s;
  if (Q0[0] > 0) euler_flux(P->gamma, Q0, flux);
  else flux[0] = flux[1] = flux[2] = 0;            /* vacuum carries no flux */
  for (int c = 0; c < 3; ++c) gnew[c] = Q0[c];
  return OR_OK;
}

/*
 * Numerical source of cell i, eq. eq:source: the space-time average of S(Q)
 * over the cell and [t^n, t^n + dt] (Section 2: "a similar but simpler
 * approach" than the flux).  READING: Q(x, tau) is the cell's own evolution,
 * the Cauchy-Kovalevskaya series (with the source) at the cell centre from
 * the Taylor coefficients of its reconstruction polynomial (no Riemann
 * problem inside a cell), integrated by the G-point Gauss-Legendre rule in
 * space and in time (exact: the series has total degree M and S is linear).
 * A centre state that is not admissible (Euler) is replaced by the cell
 * average, held constant before the evolution.  coef: monomial coefficients in
 * xi = (x - x_i)/dx; avg: the cell average.  out[C].
 */
static void cell_source(const params *P, real dx, real dt, const real *coef, const real *avg, real *out)
{
  const int M = P->M, C = P->system == OR_EULER ? 3 : 1;
  real q[(MAXM + 1) * (MAXM + 1)][MAXC];
  for (int i = 0; i < (MAXM + 1) * (MAXM + 1); ++i) q[i][0] = q[i][1] = q[i][2] = 0;
  real scale = 1;
  for (int a = 0; a <= M; ++a) {
    for (int c = 0; c < C; ++c) q[SIDX(a, 0)][c] = coef[c * (MAXM + 1) + a] / scale;
    scale = scale * dx;
  }
  if (P->system == OR_EULER && !euler_admissible(P->gamma, q[SIDX(0, 0)])) {
    for (int a = 0; a <= M; ++a)
      for (int c = 0; c < 3; ++c) q[SIDX(a, 0)][c] = a == 0 ? avg[c] : (real)0;
  }
  ck_series(P->system, P->lambda, P->gamma, M, q, &P->src);
  real s[3], w[3];
  const int G = gauss_rule(M, s, w);
  for (int c = 0; c < 3; ++c) out[c] = 0;
  for (int al = 0; al < G; ++al)
    for (int be = 0; be < G; ++be) {
      const real x = 0.5 * dx * s[al], tau = 0.5 * dt * (1 + s[be]);
      real Q[3] = { 0, 0, 0 }, S[3];
      for (int c = 0; c < C; ++c)
        for (int a = M; a >= 0; --a) {          /* Horner in x over the tau-polynomials of each power */
          real v = 0;
          for (int b = M - a; b >= 0; --b) v = v * tau + q[SIDX(a, b)][c];
          Q[c] = Q[c] * x + v;
        }
      source_apply(&P->src, Q, S);
      for (int c = 0; c < C; ++c) out[c] = out[c] + w[al] * w[be] * S[c];
    }
}

/*
 * Conservative update, eq. eq_finite_volume (Section 2), from the fluxes
 * flux[j * C + c] of the nif interfaces and the numerical sources
 * src[i * C + c] of the cells (NULL: S = 0), into cand[c * N + i], with
 * the a-posteriori repair (READING, MOOD-like; not in the paper): a candidate
 * average that is inadmissible, or whose density or pressure leaves the range
 * of the old averages of cells i-1, i, i+1 by more than OR_DMP_REL of the
 * range's magnitude (dmp_ok), marks its cell troubled; both of its interfaces
 * not yet recomputed (low[j] == 0) take the first-order Godunov flux of the
 * cell averages and its state as interface datum (gnew), and low[j] is set.
 * The candidates are then formed again from the current fluxes.  Passes
 * 0 .. OR_MAX_REPAIR - 1 repair; pass OR_MAX_REPAIR only checks.  A cell
 * still inadmissible when no further interface can change gives
 * OR_NONPHYSICAL (the candidates are kept: the domain freezes on them).
 */
static int update_repair(const params *P, int N, int bc, real dx, real dt, const real *avg, long cstride,
                         real *flux, real *gnew, char *low, real *cand, const real *src, long long *st)
{
  const int C = P->system == OR_EULER ? 3 : 1;
  int status = OR_OK;
  for (int pass = 0; ; ++pass) {
    int bad = 0, changed = 0;
    for (int i = 0; i < N; ++i) {
      int jl = i, jr = (bc == OR_BC_PERIODIC) ? (i + 1) % N : i + 1;
      for (int c = 0; c < C; ++c)
        cand[c * N + i] = src ? avg[c * cstride + i] - dt / dx * (flux[jr * C + c] - flux[jl * C + c])
                                    + dt * src[i * C + c]
                              : avg[c * cstride + i] - dt / dx * (flux[jr * C + c] - flux[jl * C + c]);
    }
    if (P->system != OR_EULER) break;
    for (int i = 0; i < N && status == OR_OK; ++i) {
      real Q[3] = { cand[i], cand[N + i], cand[2 * N + i] };
      int adm = euler_admissible(P->gamma, Q);
      if (adm && dmp_ok(P->gamma, N, bc, i, avg, cstride, Q)) continue;
      if (!adm) bad = 1;
      if (pass >= OR_MAX_REPAIR) continue;
      int js[2] = { i, (bc == OR_BC_PERIODIC) ? (i + 1) % N : i + 1 };
      for (int e = 0; e < 2; ++e) {
        int j = js[e];
        if (low[j]) continue;
        int s = first_order_interface(P, N, bc, j, avg, cstride, flux + j * C, gnew + j * C, st);
        if (s != OR_OK) { status = s; break; }
        low[j] = 1;
        changed = 1;
      }
    }
    if (status != OR_OK) break;
    if (!changed) { if (bad) status = OR_NONPHYSICAL; break; }
  }
  return status;
}

/*
 * avg, iface point at this domain's first cell / interface; strides are the
 * plane lengths.  Returns a status; on success the domain holds step n+1.
 */
static int step_domain(const params *P, int N, int bc, real dx, real dt, real *avg, long cstride,
                       real *iface, long istride, long long *st)
{
  const int M = P->M, C = P->system == OR_EULER ? 3 : 1;
  const int nif = bc == OR_BC_PERIODIC ? N : N + 1;
  real *coef = (real *)malloc(sizeof(real) * N * C * (MAXM + 1));
  real *flux = (real *)malloc(sizeof(real) * nif * C);
  real *gnew = (real *)malloc(sizeof(real) * nif * C);
  char *low = (char *)calloc(nif, 1);
  int status = OR_OK;

  OR_PHASE(1);
  /* reconstruction, cell by cell, component by component (READING: conserved
   * variables; linear GRPrec commutes with a per-cell characteristic projection) */
  for (int i = 0; i < N; ++i) {
    int im = i - 1, ip = i + 1;
    if (bc == OR_BC_PERIODIC) { im = (im + N) % N; ip = ip % N; }
    else { if (im < 0) im = 0; if (ip > N - 1) ip = N - 1; }  /* ghost = copy */
    int jl = i, jr = (bc == OR_BC_PERIODIC) ? (i + 1) % N : i + 1;
    if (P->recon == OR_RECON_GRPRECNL) {
      /* the two further interfaces of degree 4 (READING: outside a
       * transmissive end the ghost state is the boundary cell's average,
       * on its interfaces too) */
      int jll = i - 1, jrr = i + 2;
      if (bc == OR_BC_PERIODIC) { jll = (jll + N) % N; jrr = jrr % N; }
      real d7[MAXC][7];
      for (int c = 0; c < C; ++c) {
        d7[c][0] = avg[c * cstride + im];
        d7[c][1] = avg[c * cstride + i];
        d7[c][2] = avg[c * cstride + ip];
        d7[c][3] = jll < 0 ? avg[c * cstride + 0] : iface[c * istride + jll];
        d7[c][4] = iface[c * istride + jl];
        d7[c][5] = iface[c * istride + jr];
        d7[c][6] = (bc != OR_BC_PERIODIC && jrr > N) ? avg[c * cstride + N - 1] : iface[c * istride + jrr];
      }
      if (P->system == OR_EULER) {
        /* characteristic variables of the cell average (Section 3.1) */
        real Qi[3] = { avg[i], avg[cstride + i], avg[2 * cstride + i] }, Rm[3][3], Lm[3][3];
        char_basis(P->gamma, Qi, Rm, Lm);
        real w7[3][7], cw[3][MAXM + 1];
        for (int k = 0; k < 3; ++k)
          for (int j = 0; j < 7; ++j) w7[k][j] = Lm[k][0] * d7[0][j] + Lm[k][1] * d7[1][j] + Lm[k][2] * d7[2][j];
        for (int k = 0; k < 3; ++k) recon_nl(M, w7[k], dx, cw[k], 0);
        for (int c = 0; c < 3; ++c)
          for (int q = 0; q <= MAXM; ++q)
            coef[(i * C + c) * (MAXM + 1) + q] = Rm[c][0] * cw[0][q] + Rm[c][1] * cw[1][q] + Rm[c][2] * cw[2][q];
      } else {
        recon_nl(M, d7[0], dx, coef + i * (MAXM + 1), 0);
      }
    } else {
      for (int c = 0; c < C; ++c) {
        real data[5] = { avg[c * cstride + im], avg[c * cstride + i], avg[c * cstride + ip],
                         iface[c * istride + jl], iface[c * istride + jr] };
        recon_apply(M, data, coef + (i * C + c) * (MAXM + 1));
      }
    }
    if (P->system == OR_EULER) {   /* READING: inadmissible trace -> degree 0 */
      int ok = 1;
      for (int side = 0; side < 2; ++side) {
        real Q[3];
        for (int c = 0; c < 3; ++c)
          Q[c] = poly_deriv(M, coef + (i * C + c) * (MAXM + 1), 0, side ? (real)0.5 : (real)-0.5);
        if (!euler_admissible(P->gamma, Q)) ok = 0;
      }
      if (!ok) {
        for (int c = 0; c < 3; ++c)
          for (int k = 0; k <= MAXM; ++k)
            coef[(i * C + c) * (MAXM + 1) + k] = k == 0 ? avg[c * cstride + i] : (real)0;
        st[OR_ST_RECON_FB] += 1;
      }
    }
  }

  if (P->solver == OR_SOLVER_DET) {
    /* predictor in every cell; a cell whose predictor meets an inadmissible
     * state keeps its cell average, unevolved (READING, counted with the
     * reconstruction fallbacks) */
    const int n = M + 1;
    real (*ed)[2][DET_N + 1][MAXC] = (real (*)[2][DET_N + 1][MAXC])malloc(sizeof(*ed) * N);
    real nu = dt / dx;
    for (int i = 0; i < N; ++i) {
      if (det_predict(P->system, P->lambda, P->gamma, M, nu, coef + i * C * (MAXM + 1), ed[i]) != 0) {
        for (int side = 0; side < 2; ++side)
          for (int g = 0; g <= n; ++g)
            for (int c = 0; c < C; ++c) ed[i][side][g][c] = avg[c * cstride + i];
        st[OR_ST_RECON_FB] += 1;
      }
    }
    const det_basis *B = det_basis_for(M);
    for (int j = 0; j < nif && status == OR_OK; ++j) {
      int cl, cr;
      if (bc == OR_BC_PERIODIC) { cl = (j - 1 + N) % N; cr = j; }
      else { cl = j - 1; cr = j; }               /* -1 or N: the constant ghost */
      int fo = 0;
      real Fsum[3] = { 0, 0, 0 };
      for (int g = 0; g <= n && !fo; ++g) {
        real QL[3], QR[3], Q0[3], F[3];
        for (int c = 0; c < C; ++c) {
          QL[c] = cl < 0 ? avg[c * cstride + 0] : ed[cl][1][g][c];
          QR[c] = cr > N - 1 ? avg[c * cstride + N - 1] : ed[cr][0][g][c];
        }
        if (P->system == OR_ADVECTION) {
          Q0[0] = P->lambda > 0 ? QL[0] : (P->lambda < 0 ? QR[0] : 0.5 * (QL[0] + QR[0]));
        } else {
          int it = 0;
          if (!euler_admissible(P->gamma, QL) || !euler_admissible(P->gamma, QR)) { fo = 1; break; }
          int rs = riemann_state(P->gamma, QL, QR, P->guess_kind, 0, P->rtol, P->max_iter, 0, Q0, &it);
          st[OR_ST_RS_CALLS] += 1;
          st[OR_ST_NEWTON_SUM] += it;
          if (it > st[OR_ST_NEWTON_MAX]) st[OR_ST_NEWTON_MAX] = it;
          if (rs != OR_OK) { fo = 1; break; }
        }
        if (g < n) {
          phys_flux(P->system, P->lambda, P->gamma, Q0, F);
          for (int c = 0; c < C; ++c) Fsum[c] = Fsum[c] + B->w[g] * F[c];
        } else {
          for (int c = 0; c < C; ++c) gnew[j * C + c] = Q0[c];
        }
      }
      if (fo) {
        /* READING: an inadmissible evolved edge value or a Riemann problem
         * without solution sends the interface to the first-order flux */
        int s2 = first_order_interface(P, N, bc, j, avg, cstride, flux + j * C, gnew + j * C, st);
        low[j] = 1;
        if (s2 != OR_OK) status = s2;
      } else {
        for (int c = 0; c < C; ++c) flux[j * C + c] = Fsum[c];
      }
    }
    free(ed);
  }

  /* one GRP per interface.  READING (transmissive ends): the outside cell is a
   * ghost holding the boundary cell's average as a constant polynomial. */
  for (int j = 0; j < nif && status == OR_OK && P->solver != OR_SOLVER_DET; ++j) {
    int cl, cr;
    if (bc == OR_BC_PERIODIC) { cl = (j - 1 + N) % N; cr = j; }
    else { cl = j - 1; cr = j; }                  /* -1 or N: the ghost */
    real trL[(MAXM + 1) * MAXC], trR[(MAXM + 1) * MAXC];
    real scale = 1;
    for (int k = 0; k <= M; ++k) {
      for (int c = 0; c < C; ++c) {
        if (cl < 0) trL[k * C + c] = k == 0 ? avg[c * cstride + 0] : (real)0;
        else trL[k * C + c] = poly_deriv(M, coef + (cl * C + c) * (MAXM + 1), k, (real)0.5) / scale;
        if (cr > N - 1) trR[k * C + c] = k == 0 ? avg[c * cstride + N - 1] : (real)0;
        else trR[k * C + c] = poly_deriv(M, coef + (cr * C + c) * (MAXM + 1), k, (real)-0.5) / scale;
      }
      scale = scale * dx;
    }
    int it = 0, tr = 0;
    int s = grp_interface(P->system, P->lambda, P->gamma, M, dt, trL, trR, P->rtol, P->max_iter,
                          P->guess_kind, flux + j * C, gnew + j * C, &it, &tr, &P->src);
    if (P->system == OR_EULER) {
      st[OR_ST_RS_CALLS] += 1;
      st[OR_ST_NEWTON_SUM] += it;
      if (it > st[OR_ST_NEWTON_MAX]) st[OR_ST_NEWTON_MAX] = it;
      st[OR_ST_FLUX_FB] += tr;
      /* READING: a Riemann problem of the traces with no solution (vacuum,
       * no convergence) sends this interface to the first-order flux */
      if (s != OR_OK) {
        s = first_order_interface(P, N, bc, j, avg, cstride, flux + j * C, gnew + j * C, st);
        low[j] = 1;
      }
    }
    if (s != OR_OK) status = s;
  }

  /* numerical sources of the cells (eq. eq:source), from the reconstructions
   * as used for the traces (degree-0 fallback included) */
  real *src = 0;
  if (status == OR_OK && P->src.kind != OR_SOURCE_NONE) {
    src = (real *)malloc(sizeof(real) * N * C);
    for (int i = 0; i < N; ++i) {
      real cf[MAXC * (MAXM + 1)], av[MAXC], out[3];
      for (int c = 0; c < C; ++c) {
        for (int k = 0; k <= MAXM; ++k) cf[c * (MAXM + 1) + k] = coef[(i * C + c) * (MAXM + 1) + k];
        av[c] = avg[c * cstride + i];
      }
      cell_source(P, dx, dt, cf, av, out);
      for (int c = 0; c < C; ++c) src[i * C + c] = out[c];
    }
  }

  OR_PHASE(2);
  real *cand = (real *)malloc(sizeof(real) * N * C);
  if (status == OR_OK) status = update_repair(P, N, bc, dx, dt, avg, cstride, flux, gnew, low, cand, src, st);
  free(src);
  if (status == OR_OK || status == OR_NONPHYSICAL) {
    for (int i = 0; i < N; ++i)
      for (int c = 0; c < C; ++c) avg[c * cstride + i] = cand[c * N + i];
    for (int j = 0; j < nif; ++j)
      for (int c = 0; c < C; ++c) iface[c * istride + j] = gnew[j * C + c];
  }
  free(cand); free(low);
  free(coef); free(flux); free(gnew);
  return status;
}

int or_run(int system, double lambda, double gamma, int M, double cfl,
           int n_domains, const int *n_cells, const double *x_left, const double *x_right,
           const int *bc, double newton_rtol, int newton_max_iter, int guess_kind, int dt_hold,
           double *avg, double *iface, double *t, int *nstep, double *dt_prev, int *status,
           int n_steps, double t_end, long long *stats, const double *dt_fixed, int n_threads)
{
  return or_run_ex(system, lambda, gamma, M, OR_RECON_GRPREC, cfl, n_domains, n_cells, x_left, x_right, bc,
                   newton_rtol, newton_max_iter, guess_kind, dt_hold, avg, iface, t, nstep, dt_prev, status,
                   n_steps, t_end, stats, dt_fixed, n_threads);
}

int or_run_ex(int system, double lambda, double gamma, int M, int recon, double cfl,
              int n_domains, const int *n_cells, const double *x_left, const double *x_right,
              const int *bc, double newton_rtol, int newton_max_iter, int guess_kind, int dt_hold,
              double *avg, double *iface, double *t, int *nstep, double *dt_prev, int *status,
              int n_steps, double t_end, long long *stats, const double *dt_fixed, int n_threads)
{
  return or_run_solver(system, lambda, gamma, M, recon, OR_SOLVER_TT, cfl, n_domains, n_cells, x_left, x_right,
                       bc, newton_rtol, newton_max_iter, guess_kind, dt_hold, avg, iface, t, nstep, dt_prev,
                       status, n_steps, t_end, stats, dt_fixed, n_threads);
}

int or_run_solver(int system, double lambda, double gamma, int M, int recon, int solver, double cfl,
                  int n_domains, const int *n_cells, const double *x_left, const double *x_right,
                  const int *bc, double newton_rtol, int newton_max_iter, int guess_kind, int dt_hold,
                  double *avg, double *iface, double *t, int *nstep, double *dt_prev, int *status,
                  int n_steps, double t_end, long long *stats, const double *dt_fixed, int n_threads)
{
  return or_run_full(system, lambda, gamma, M, recon, solver, OR_SOURCE_NONE, 0.0, cfl, n_domains, n_cells,
                     x_left, x_right, bc, newton_rtol, newton_max_iter, guess_kind, dt_hold, avg, iface, t,
                     nstep, dt_prev, status, n_steps, t_end, stats, dt_fixed, n_threads);
}

int or_run_full(int system, double lambda, double gamma, int M, int recon, int solver, int source,
                double source_coef, double cfl, int n_domains, const int *n_cells, const double *x_left,
                const double *x_right, const int *bc, double newton_rtol, int newton_max_iter, int guess_kind,
                int dt_hold, double *avg, double *iface, double *t, int *nstep, double *dt_prev, int *status,
                int n_steps, double t_end, long long *stats, const double *dt_fixed, int n_threads)
{
  params P;
  P.solver = solver;
  P.src.kind = source;
  P.src.coef = source_coef;
  if (source != OR_SOURCE_NONE && source != OR_SOURCE_LINEAR && source != OR_SOURCE_GRAVITY) return -1;
  if (source == OR_SOURCE_LINEAR && system != OR_ADVECTION) return -1;
  if (source == OR_SOURCE_GRAVITY && system != OR_EULER) return -1;
  if (source != OR_SOURCE_NONE && solver != OR_SOLVER_TT) return -1;   /* the source enters the TT series */
  P.system = system; P.lambda = lambda; P.gamma = gamma; P.M = M; P.cfl = cfl;
  P.rtol = newton_rtol; P.max_iter = newton_max_iter; P.guess_kind = guess_kind;
  P.dt_hold = dt_hold < 1 ? 1 : dt_hold;
  P.recon = recon;
  if (M < 1 || M > MAXM) return -1;
  const int C = system == OR_EULER ? 3 : 1;
  long *coff = (long *)malloc(sizeof(long) * (n_domains + 1));
  long *ioff = (long *)malloc(sizeof(long) * (n_domains + 1));
  coff[0] = ioff[0] = 0;
  for (int d = 0; d < n_domains; ++d) {
    coff[d + 1] = coff[d] + n_cells[d];
    ioff[d + 1] = ioff[d] + n_cells[d] + (bc[d] == OR_BC_TRANSMISSIVE ? 1 : 0);
  }
  const long ctot = coff[n_domains], itot = ioff[n_domains];
  (void)n_threads;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int d = 0; d < n_domains; ++d) {
    const int N = n_cells[d];
    const real dx = (x_right[d] - x_left[d]) / N;
    /* this domain's planes, copied to contiguous real arrays */
    real *a = (real *)malloc(sizeof(real) * N * C);
    real *g = (real *)malloc(sizeof(real) * (N + 1) * C);
    const int nif = (int)(ioff[d + 1] - ioff[d]);
    for (int c = 0; c < C; ++c) {
      for (int i = 0; i < N; ++i) a[c * N + i] = OR_DATA(avg[c * ctot + coff[d] + i]);
      for (int j = 0; j < nif; ++j) g[c * nif + j] = OR_DATA(iface[c * itot + ioff[d] + j]);
    }
    long long *st = stats + (long)d * OR_NSTATS;
    for (int s = 0; s < n_steps; ++s) {
      if (status[d] != OR_OK) break;
      real td = t[d];
      if (!(td < t_end)) break;
      real dt_cfl;
      if (dt_fixed) dt_cfl = dt_fixed[s];
      else if (nstep[d] % P.dt_hold == 0 || !(dt_prev[d] > 0)) {
        OR_PHASE(0);
        dt_cfl = P.cfl * dx / domain_smax(&P, N, a, N);
      }
      else dt_cfl = dt_prev[d];
      real dt = dt_cfl;
      int last = 0;
      if (td + dt >= t_end) { dt = t_end - td; last = 1; }
      int rc = step_domain(&P, N, bc[d], dx, dt, a, N, g, nif, st);
      if (rc != OR_OK && rc != OR_NONPHYSICAL) { status[d] = rc; break; }
      t[d] = last ? t_end : (double)(td + dt);
      nstep[d] += 1;
      dt_prev[d] = dt_cfl;
      st[OR_ST_STEPS] += 1;
      if (rc == OR_NONPHYSICAL) { status[d] = rc; break; }
    }
    for (int c = 0; c < C; ++c) {
      for (int i = 0; i < N; ++i) avg[c * ctot + coff[d] + i] = a[c * N + i];
      for (int j = 0; j < nif; ++j) iface[c * itot + ioff[d] + j] = g[c * nif + j];
    }
    free(a); free(g);
  }
  free(coff); free(ioff);
  return 0;
}

/* The update and repair phase of one Euler step on given fluxes (see
 * update_repair): avg [3][N] old averages, flux and gnew [nif][3] the
 * high-order fluxes and interface data (in: as the GRP produced them; out:
 * after the repair), low [nif] (in/out; 1 = already first order), cand [3][N]
 * the new averages, stats [OR_NSTATS] counters (added to).  Returns the status. */
int or_update_repair(double gamma, int N, int bc, double dx, double dt, const double *avg, double *flux,
                     double *gnew, char *low, double *cand, long long *stats)
{
  params P;
  memset(&P, 0, sizeof(P));
  P.system = OR_EULER; P.gamma = gamma; P.M = 1; P.cfl = 1;
  P.rtol = 1e-12; P.max_iter = 50; P.guess_kind = OR_GUESS_PVRS; P.dt_hold = 1;
  const int nif = bc == OR_BC_PERIODIC ? N : N + 1;
  real *a = (real *)malloc(sizeof(real) * 3 * N), *f = (real *)malloc(sizeof(real) * 3 * nif);
  real *g = (real *)malloc(sizeof(real) * 3 * nif), *cd = (real *)malloc(sizeof(real) * 3 * N);
  for (int k = 0; k < 3 * N; ++k) a[k] = avg[k];
  for (int k = 0; k < 3 * nif; ++k) { f[k] = flux[k]; g[k] = gnew[k]; }
  int st = update_repair(&P, N, bc, dx, dt, a, N, f, g, low, cd, 0, stats);
  for (int k = 0; k < 3 * N; ++k) cand[k] = (double)cd[k];
  for (int k = 0; k < 3 * nif; ++k) { flux[k] = (double)f[k]; gnew[k] = (double)g[k]; }
  free(a); free(f); free(g); free(cd);
  return st;
}
