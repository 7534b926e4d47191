/*
 * ORACLE — test infrastructure only.
 *
 * A plain, slow, FP64 CPU implementation of one time step of the FV+GRPrec
 * ADER scheme (Montecinos, Toro, Mueller, arXiv 2602.21911) for 1D linear
 * advection and the ideal-gas Euler equations.  It shares no code, header or
 * constant with the CUDA library; only the test suite, the smoke check and the
 * bench's CPU-baseline / reference leg may load it.
 *
 * Layout conventions (the same *conventions* as the library, written again):
 *   - domains are concatenated; cell planes are component-major (SoA):
 *       avg[c * n_cells_total + cell_off[d] + i]
 *   - interface index j of a domain is the interface at the LEFT of cell j,
 *     x_{j-1/2}.  A periodic domain has N interfaces (the right edge of cell
 *     N-1 is interface 0); a transmissive domain has N+1.
 *       iface[c * n_ifaces_total + if_off[d] + j]
 */
#ifndef GRPREC_ORACLE_H
#define GRPREC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_ADVECTION = 0, OR_EULER = 1 };
enum { OR_BC_PERIODIC = 0, OR_BC_TRANSMISSIVE = 1 };
enum { OR_GUESS_PVRS = 0, OR_GUESS_TRRS = 1, OR_GUESS_GIVEN = 2 };
enum { OR_RECON_GRPREC = 0, OR_RECON_GRPRECNL = 1 };
enum { OR_SOLVER_TT = 0, OR_SOLVER_DET = 1 };
/* source term S(Q) (Section 2): none; advection S(q) = k q; Euler S = (0, -g rho, -g m) */
enum { OR_SOURCE_NONE = 0, OR_SOURCE_LINEAR = 1, OR_SOURCE_GRAVITY = 2 };
enum {
  OR_OK = 0,
  OR_NEWTON_NO_CONV = 1,
  OR_VACUUM = 2,
  OR_NONPHYSICAL = 3
};
/* per-domain statistics counters */
enum {
  OR_ST_STEPS = 0,        /* steps taken */
  OR_ST_NEWTON_SUM = 1,   /* Newton iterations summed over interfaces */
  OR_ST_NEWTON_MAX = 2,   /* max Newton iterations at one interface */
  OR_ST_RECON_FB = 3,     /* cells reconstructed at degree 0 (admissibility) */
  OR_ST_FLUX_FB = 4,      /* interfaces whose time series was truncated */
  OR_ST_RS_CALLS = 5,     /* exact Riemann solves */
  OR_ST_LOW_ORDER = 6,    /* interfaces recomputed at first order (a posteriori) */
  OR_NSTATS = 7
};

/* Section 3.1: GRPrec polynomial of degree M on cell i, monomial coefficients
 * in xi = (x - x_i)/dx.  qbar = {q_{i-1}, q_i, q_{i+1}}, g = {g_{i-1/2}, g_{i+1/2}}. */
int or_recon(int M, const double *qbar, const double *g, double *coef);

/* Sections 3.3-3.4: GRPrecNL polynomial of degree M (monomial coefficients in
 * xi) from d7 = {q_{i-1}, q_i, q_{i+1}, g_{i-3/2}, g_{i-1/2}, g_{i+1/2},
 * g_{i+3/2}} and the cell width dx; beta (3 values, may be NULL) receives the
 * nonlinear weights of the left, central and right polynomials. */
int or_recon_nl(int M, const double *d7, double dx, double *coef, double *beta);

/* Characteristic variables of the Euler equations at conserved state Q:
 * R (row-major 3x3, right eigenvectors as columns, eigenvalues u-c, u, u+c)
 * and L = R^{-1}. */
int or_char_basis(double gamma, const double *Q, double *R, double *L);

/* Exact Riemann solver for the ideal-gas Euler equations (primitive states). */
int or_star_pressure(double gamma, const double *WL, const double *WR, int guess_kind,
                     double guess, double rtol, int max_iter, double *out /* p*,u*,iters */);
int or_riemann_state(double gamma, const double *QL, const double *QR, double rtol,
                     int max_iter, double *Q /* conserved state at x/t=0 */, int *iters);

/* Derivative Riemann problem: linear RP with the Jacobian frozen at Q0. */
void or_deriv_rp(double gamma, const double *Q0, const double *DL, const double *DR, double *D);

/* Cauchy-Kovalevskaya: series q[a][b][c] (a+b<=M) from q[a][0][c]. */
void or_ck_series(int system, double lambda, double gamma, int M, const double *qa0, double *q);

/* One interface: traces tr{L,R}[k*C + c] = d^k/dx^k of the conserved traces. */
int or_grp_interface(int system, double lambda, double gamma, int M, double dt,
                     const double *trL, const double *trR, double rtol, int max_iter,
                     int guess_kind, double *flux, double *gnew, int *iters, int *truncated);

/* Initial interface data: the leading Riemann state of the one-sided limits. */
int or_init_iface(int system, double lambda, double gamma, int n_ifaces,
                  const double *lim_minus, const double *lim_plus, double *iface);

/* Advance every domain n_steps steps or to t_end, whichever comes first. */
/* The update and repair phase of one Euler step (eq. eq_finite_volume with the
 * a-posteriori first-order repair, a reading: not in the paper) on given
 * high-order fluxes: avg [3][N]; flux, gnew [nif][3] in/out; low [nif] in/out;
 * cand [3][N] out; stats [OR_NSTATS] added to.  Returns OR_OK, OR_NONPHYSICAL
 * or the status of a failed first-order Riemann problem. */
int or_update_repair(double gamma, int N, int bc, double dx, double dt, const double *avg, double *flux,
                     double *gnew, char *low, double *cand, long long *stats);

int or_run(int system, double lambda, double gamma, int M, double cfl,
           int n_domains, const int *n_cells, const double *x_left, const double *x_right,
           const int *bc, double newton_rtol, int newton_max_iter, int guess_kind, int dt_hold,
           double *avg, double *iface, double *t, int *nstep, double *dt_prev, int *status,
           int n_steps, double t_end, long long *stats, const double *dt_fixed, int n_threads);

/* or_run with the reconstruction chosen: OR_RECON_GRPREC (Section 3.1, conserved
 * variables) or OR_RECON_GRPRECNL (Sections 3.3-3.4, characteristic variables
 * for the Euler equations). */
int or_run_ex(int system, double lambda, double gamma, int M, int recon, double cfl,
              int n_domains, const int *n_cells, const double *x_left, const double *x_right,
              const int *bc, double newton_rtol, int newton_max_iter, int guess_kind, int dt_hold,
              double *avg, double *iface, double *t, int *nstep, double *dt_prev, int *status,
              int n_steps, double t_end, long long *stats, const double *dt_fixed, int n_threads);

/* or_run_ex with the GRP solver chosen: OR_SOLVER_TT (Toro-Titarev: exact
 * leading Riemann problem, derivative Riemann problems, Cauchy-Kovalevskaya)
 * or OR_SOLVER_DET (space-time Galerkin predictor per cell, Riemann problems
 * of the evolved edge values at the time integration points). */
int or_run_solver(int system, double lambda, double gamma, int M, int recon, int solver, double cfl,
                  int n_domains, const int *n_cells, const double *x_left, const double *x_right,
                  const int *bc, double newton_rtol, int newton_max_iter, int guess_kind, int dt_hold,
                  double *avg, double *iface, double *t, int *nstep, double *dt_prev, int *status,
                  int n_steps, double t_end, long long *stats, const double *dt_fixed, int n_threads);

/* or_run_solver with a source term (eq. eq_finite_volume with S, Section 2):
 * source = OR_SOURCE_LINEAR (advection, S = source_coef q) or
 * OR_SOURCE_GRAVITY (Euler, S = (0, -g rho, -g m), g = source_coef), with the
 * Toro-Titarev solver only.  Returns -1 for a combination it does not take. */
int or_run_full(int system, double lambda, double gamma, int M, int recon, int solver, int source,
                double source_coef, double cfl, int n_domains, const int *n_cells, const double *x_left,
                const double *x_right, const int *bc, double newton_rtol, int newton_max_iter, int guess_kind,
                int dt_hold, double *avg, double *iface, double *t, int *nstep, double *dt_prev, int *status,
                int n_steps, double t_end, long long *stats, const double *dt_fixed, int n_threads);

/* The Cauchy-Kovalevskaya series with a source term: qa0[a][c] = q_{a,0};
 * qout[a][b][c] (M+1 x M+1 x C) for a + b <= M. */
void or_ck_series_src(int system, double lambda, double gamma, int M, int source, double coef,
                      const double *qa0, double *qout);

#ifdef __cplusplus
}
#endif
#endif
