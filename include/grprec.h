/*
 * grprec.h — C ABI of the GB300 (sm_103a) FV+GRPrec ADER library.
 *
 * One time step of the finite volume scheme of Montecinos, Toro and Mueller,
 * "A generalized Riemann problem-based compact reconstruction method for
 * finite volume schemes" (arXiv 2602.21911), for 1D linear advection and the
 * ideal-gas Euler equations, over many independent 1D domains at once:
 *
 *   Q_i^{n+1} = Q_i^n - dt/dx (F_{i+1/2} - F_{i-1/2}) + dt S_i   (Section 2, eq. eq_finite_volume)
 *
 *   - GRPrec reconstruction of degree M = 1..4 from the cell averages and the
 *     interface data kept from the previous step                (Section 3.1)
 *   - a generalized Riemann problem GRP_M per interface: exact leading-term
 *     Riemann problem by Newton on the star pressure, derivative Riemann
 *     problems, Cauchy-Kovalevskaya time series (Toro-Titarev structure,
 *     Section 2), Gauss time integral of the flux (numerical flux, Section 2)
 *   - write-back of the interface data = the series at tau = dt
 *   - dt = C dx / S_max with S_max over the cell averages          (Section 4.1)
 *
 * Conventions for every entry point:
 *   - Return 0 on success, a negative GRP_E_* code otherwise; grp_status_string
 *     names it.  Nothing is thrown, nothing aborts.
 *   - The library owns all device memory it allocates in grp_create and frees it
 *     in grp_destroy.  The caller owns every buffer it passes; the library never
 *     keeps a caller pointer after a call returns.
 *   - Work is ordered on the stream given in grp_problem (NULL = legacy default
 *     stream).  grp_get_* synchronise that stream before returning.
 *   - State layout (also of caller buffers): component-major planes concatenated
 *     over domains.  Cell planes hold sum(n_cells) doubles each; interface planes
 *     hold sum(n_cells[d] + (bc[d] == TRANSMISSIVE)) doubles each.  Interface j
 *     of a domain is the left edge of its cell j (periodic: the right edge of the
 *     last cell is interface 0).  Components: advection (q); Euler (rho, rho u, E).
 *   - There is no CPU fallback: without a usable CUDA device grp_create fails with
 *     GRP_E_CUDA.
 */
#ifndef GRPREC_H
#define GRPREC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct grp_ctx grp_ctx;   /* opaque, library-owned */

enum { GRP_ADVECTION = 0, GRP_EULER_IDEAL = 1 };                 /* system (Sections 4.2, 4.3) */
enum { GRP_BC_PERIODIC = 0, GRP_BC_TRANSMISSIVE = 1 };            /* per-domain boundary */
enum { GRP_GUESS_PVRS = 0, GRP_GUESS_TRRS = 1, GRP_GUESS_MLP = 2 };/* Newton initial guess for p* */
enum { GRP_LAUNCH_AUTO = 0, GRP_LAUNCH_FLAT = 1, GRP_LAUNCH_FUSED = 2, GRP_LAUNCH_SPLIT = 3,
       GRP_LAUNCH_TILED = 4 };                                                              /* grp_set_launch */
enum { GRP_RECON_GRPREC = 0, GRP_RECON_GRPRECNL = 1 };            /* reconstruction (Sections 3.1, 3.3-3.4) */
enum { GRP_SOLVER_TT = 0, GRP_SOLVER_DET = 1 };                   /* GRP solver (Section 2, Section 4.1) */
enum { GRP_SOURCE_NONE = 0, GRP_SOURCE_LINEAR = 1, GRP_SOURCE_GRAVITY = 2 };  /* source term S(Q) (Section 2) */

/* return codes */
enum {
  GRP_OK = 0,
  GRP_E_INVALID_ARG = -1,
  GRP_E_CUDA = -2,
  GRP_E_NOT_INITIALIZED = -3,
  GRP_E_NO_MODEL = -4,
  GRP_E_MAX_STEPS = -5
};

/* per-domain status (grp_get_stats); a domain with a non-zero status is frozen */
enum {
  GRP_ST_OK = 0,
  GRP_ST_NEWTON_NO_CONV = 1,   /* the star-pressure Newton iteration hit newton_max_iter */
  GRP_ST_VACUUM = 2,           /* reserved: vacuum data are sampled, never fatal */
  GRP_ST_NONPHYSICAL = 3       /* an average stayed inadmissible after the first-order repair */
};

/* per-domain counters (grp_get_stats), each an unsigned 64-bit integer */
enum {
  GRP_STAT_STEPS = 0,          /* steps taken */
  GRP_STAT_NEWTON_SUM = 1,     /* star-pressure Newton iterations, summed (a leading Riemann problem
                                  whose two states agree to 2^-48 has equal data: its exact solution
                                  is that state, and it counts no iteration) */
  GRP_STAT_NEWTON_MAX = 2,     /* max iterations at one interface */
  GRP_STAT_RECON_FB = 3,       /* cells reconstructed at degree 0 (inadmissible trace) */
  GRP_STAT_FLUX_FB = 4,        /* interfaces whose time series was cut to its leading term */
  GRP_STAT_RS_CALLS = 5,       /* exact Riemann solves, equal data included */
  GRP_STAT_LOW_ORDER = 6,      /* interfaces recomputed with the first-order Godunov flux */
  GRP_STAT_GUESS_USED = 7,     /* Newton solves started from the network's prediction */
  GRP_STAT_GUESS_REJECTED = 8, /* learned guesses rejected (range / non-finite / stall) */
  GRP_NSTATS = 9
};

typedef struct {
  int system;            /* GRP_ADVECTION or GRP_EULER_IDEAL */
  double lambda;         /* advection speed (advection only), != 0 */
  double gamma;          /* ratio of specific heats (Euler only), > 1 */
  int M;                 /* GRPrec degree, 1..4: a scheme of order M+1 (Section 3.1) */
  double cfl;            /* Courant coefficient C in (0, 1] (Section 4.1) */
  int n_domains;         /* >= 1 */
  const int *n_cells;    /* host [n_domains], each >= 1 */
  const double *x_left;  /* host [n_domains]; uniform grid on [x_left, x_right] */
  const double *x_right; /* host [n_domains], x_right > x_left */
  const int *bc;         /* host [n_domains], GRP_BC_* */
  double newton_rtol;    /* relative stopping change of the star pressure, e.g. 1e-12 */
  int newton_max_iter;   /* Newton iteration cap, e.g. 50 */
  int guess;             /* GRP_GUESS_*; GRP_GUESS_MLP needs grp_set_guess_model */
  int dt_hold;           /* recompute dt every dt_hold steps; 1 = the paper's rule */
  int device;            /* CUDA device ordinal */
  void *stream;          /* cudaStream_t to order work on (NULL = default stream) */
  int recon;             /* GRP_RECON_GRPREC: linear GRPrec, component-wise in conserved variables
                            (Section 3.1); GRP_RECON_GRPRECNL: the nonlinear convex combination
                            of Sections 3.3-3.4 (weights r = 4, eps = 1e-14, lambda_C = 1e9), in
                            characteristic variables of the cell average for the Euler equations
                            (Section 3.1).  grp_step_noalloc always uses GRPrec. */
  int solver;            /* GRP_SOLVER_TT: Toro-Titarev (exact leading Riemann problem, derivative
                            Riemann problems, Cauchy-Kovalevskaya series, Gauss quadrature);
                            GRP_SOLVER_DET: the solver of the paper's computations (Section 4.1), a
                            space-time Galerkin predictor per cell (degree M in space and time, M+1
                            Gauss-Legendre nodes, Picard iteration to 1e-13) and exact Riemann
                            problems of the evolved edge values at the M+1 time nodes (flux) and at
                            the end of the step (interface datum).  DET runs the FLAT launch form
                            whatever grp_set_launch asks; grp_step_noalloc always uses TT. */
  int source;            /* source term S(Q) of the balance law d_t Q + d_x F(Q) = S(Q) (Section 2):
                            GRP_SOURCE_NONE; GRP_SOURCE_LINEAR, advection only, S(q) = source_coef q;
                            GRP_SOURCE_GRAVITY, Euler only, S = (0, -g rho, -g m) with
                            g = source_coef (a constant acceleration -g along x).  The source enters
                            the GRP's Cauchy-Kovalevskaya series, and the update adds dt S_i, S_i the
                            space-time average of S over the cell's own evolution (eq. eq:source).
                            Needs GRP_SOLVER_TT and GRP_RECON_GRPREC; runs the FLAT launch form;
                            grp_step_noalloc has no source.  Reconstructions of degree <= 2 keep a
                            steady state that is a polynomial of degree <= 2 (Section 3.5). */
  double source_coef;    /* k or g above (finite) */
} grp_problem;

/*
 * Create a context for the problem *p (copied; the arrays are read during the
 * call only).  Allocates the device state.  *out receives the context.
 * Euler equations with GRPrec of degree 2 or 4, the TT solver and no source:
 * the flux phase solves the Riemann problems that are not equal data in a
 * second kernel, from a list of n_if / 4 + 1024 interfaces (n_if = the total
 * interface count) held by the context, (6 (M + 1) + 1) x 8 bytes each;
 * interfaces beyond it are solved in the first kernel.
 * Errors: GRP_E_INVALID_ARG for any field outside its range, GRP_E_CUDA.
 */
int grp_create(grp_ctx **out, const grp_problem *p);

/*
 * Set the initial cell averages and interface data; resets time, steps,
 * statistics and status of every domain.
 *   averages:  C planes of sum(n_cells) doubles (required)
 *   lim_minus: C interface planes, the initial condition's left limits
 *   lim_plus:  C interface planes, right limits, or NULL
 * With lim_plus == NULL the interface data are lim_minus as given.  Otherwise
 * they are the classical Riemann solution of (lim_minus, lim_plus) at x/t = 0
 * (advection: the upwind value): the GRP at t = 0 of the initial data, which
 * equals the point value wherever the initial condition is continuous.
 * ptr_is_device: 0 = host pointers, 1 = device pointers on the context's device.
 */
int grp_set_initial(grp_ctx *ctx, const double *averages, const double *lim_minus,
                    const double *lim_plus, int ptr_is_device);

/*
 * Advance every active domain by n_steps steps (n_steps >= 0).  A domain stops
 * early when it reaches t_end (the last step is clipped to land on t_end; pass
 * INFINITY for no end) or when its status becomes non-zero.  Asynchronous when
 * t_end is infinite or n_steps <= 64; with a finite t_end a longer request
 * synchronises every 64 steps and returns once every domain is done.
 */
int grp_step(grp_ctx *ctx, int n_steps, double t_end);

/*
 * Advance every domain to t_end; returns GRP_E_MAX_STEPS if some active domain
 * has not reached it after max_steps steps.  Steps are enqueued in blocks; the
 * stream is synchronised once per block to test whether every domain is done.
 */
int grp_advance_to(grp_ctx *ctx, double t_end, int max_steps);

/*
 * Copy the state out (any pointer may be NULL to skip it): averages (C cell
 * planes), interface data (C interface planes), t (n_domains doubles).
 * Synchronises the context's stream.
 */
int grp_get_state(grp_ctx *ctx, double *averages, double *iface, double *t, int ptr_is_device);

/*
 * Host copies of the per-domain counters, stats[n_domains][GRP_NSTATS] (may be
 * NULL), and statuses, status[n_domains] (may be NULL).  Synchronises.
 */
int grp_get_stats(grp_ctx *ctx, unsigned long long *stats, int *status);

/*
 * Per-domain error norms of the first component (density / q) against exact
 * cell averages given in the cell layout (ptr_is_device as above):
 *   l1[d] = sum |Q - Q_exact| dx, l2[d] = sqrt(sum |Q - Q_exact|^2 dx),
 *   linf[d] = max |Q - Q_exact|                         (Section 4, table columns)
 * Output arrays are host [n_domains]; any may be NULL.  Synchronises.
 */
int grp_error_norms(grp_ctx *ctx, const double *exact_averages, int ptr_is_device,
                    double *l1, double *l2, double *linf);

/*
 * Launch configuration of grp_step (the results do not depend on it).
 *   GRP_LAUNCH_FLAT:  one sequence of grid-wide kernels per step (S_max,
 *                     fluxes, update, repair rounds, bookkeeping); any domain size.
 *   GRP_LAUNCH_FUSED: one persistent kernel in which each block owns whole
 *                     consecutive domains (about cells_per_block cells) and
 *                     advances them steps_per_launch steps per launch, all
 *                     phases of a step separated by block barriers.
 *   GRP_LAUNCH_SPLIT: two launches per step: the grid-wide flux kernel, then a
 *                     per-domain-group kernel for update, repair, bookkeeping
 *                     and the next step's S_max.
 *   GRP_LAUNCH_TILED: temporal blocking: tiles of cells_per_block cells held in
 *                     shared memory with a halo of steps_per_launch x
 *                     (reach + 4) + 1 cells (reach 1 for GRPrec of degree
 *                     <= 2, else 2; 4 repair rounds), each block advancing its
 *                     tile steps_per_launch steps with dt held over them.  Runs
 *                     only when dt_hold == steps_per_launch, for grp_step with
 *                     an infinite t_end, from a step count that is a multiple
 *                     of steps_per_launch; other steps take the FLAT form.
 *                     Results equal the FLAT form's; a domain that fails inside
 *                     a launch is frozen at the end of that launch.  Not with
 *                     DET or a source term.  A domain that fits one region is
 *                     one tile.  Rejected when a region does not fit 227 KB of
 *                     shared memory.
 *   GRP_LAUNCH_AUTO:  FLAT (DET solver and source terms: always FLAT).
 * threads: 128 or 256 per block (FUSED, SPLIT); cells_per_block in [64, 2^20];
 * steps_per_launch in [1, 1024] (FUSED).  Synchronises the stream.  Defaults:
 * AUTO, 256, 2048, 8.  grp_get_launch reports the form grp_step will take
 * (*batched = GRP_LAUNCH_*) and the number of blocks of the per-group kernels
 * (any pointer may be NULL).
 */
int grp_set_launch(grp_ctx *ctx, int mode, int threads, int cells_per_block, int steps_per_launch);
int grp_get_launch(const grp_ctx *ctx, int *batched, int *threads, int *cells_per_block,
                   int *steps_per_launch, int *blocks);

/*
 * CUDA graphs.  grp_step captures the launch sequence of steps_per_graph
 * consecutive steps (whole launches of the current form) into a CUDA graph
 * once and replays it for every further run of that many steps; shorter
 * remainders are launched directly.  A graph is kept per start buffer, t_end
 * and launch state, and dropped by grp_set_launch, grp_set_graph,
 * grp_set_guess_model, grp_set_harvest and a change of grp_set_kernel_timing.
 * steps_per_graph in [0, 1024]; 0 launches every kernel directly; a value that
 * is not a multiple of steps_per_launch in the FUSED form also launches
 * directly.  Default 16.  Synchronises the stream.
 */
int grp_set_graph(grp_ctx *ctx, int steps_per_graph);

/*
 * Learned Newton initial guess for the star pressure (not in the paper: an
 * FP32 network that replaces the PVRS start of the exact Riemann solver on
 * strong data; the converged p* is unchanged).
 *
 * Network: 6 -> 64 -> 64 -> 1 with tanh hidden layers.  Inputs, for primitive
 * states (rho,u,p)_L,R with rbar = sqrt(rhoL rhoR), pbar = sqrt(pL pR),
 * cbar = sqrt(gamma pbar / rbar), ubar = (uL+uR)/2:
 *   ln(rhoL/rbar), ln(rhoR/rbar), ln(pL/pbar), ln(pR/pbar), (uL-ubar)/cbar, (uR-ubar)/cbar
 * Output: v, the normalised correction of the two-rarefaction estimate p_TR:
 * with the shock strength s = ln(p_TR / min(pL, pR)) the Newton start is
 * p_TR exp(-0.005 s^3 v) (the correction vanishes like s^3; v is of order
 * one).  Strong data, |ln(pL/pR)| > 0.5 or |uR-uL|/cbar > 0.5, with
 * s >= 1e-3 start from the network; strong data with s < 1e-3 (two
 * rarefactions, where p_TR is p*, or weaker shocks) start at p_TR; PVRS starts
 * the rest.
 * Parameters (GRP_MLP_NPARAM floats): W1[6][64],
 * b1[64], W2[64][64], b2[64], w3[64], b3.
 *
 * grp_set_guess_model: load the weights and the input box (12 floats: lo[6],
 * hi[6]); used when grp_problem.guess == GRP_GUESS_MLP.  An input outside the
 * box, an output that is not finite or outside |v| <= 50, or no
 * convergence within 8 Newton iterations falls back to PVRS; the counters
 * GRP_STAT_GUESS_USED / GRP_STAT_GUESS_REJECTED record both.  Pointers host or
 * device (ptr_is_device); copied, not kept.  Synchronises.
 *
 * grp_set_harvest: record (6 inputs, the target v = ln(p* / p_TR) /
 * (-0.005 s^3), Newton iterations) of one strong-data Riemann problem with a
 * shock (those the network serves) in 2^log2_stride, by a hash of
 * (interface, step), from the flux kernel and from the repair rounds of the
 * flat form (whose first-order problems start from the classical estimate),
 * into the caller's device buffer records[capacity][8] during later steps;
 * *count (device, caller-zeroed) counts the offered records and may exceed
 * capacity (the excess is dropped).  records = NULL stops harvesting.
 *
 * Training kernels (device pointers, FP32, ordered on `stream`):
 *   grp_mlp_forward:   y[n] = network(x[n][6])
 *   grp_mlp_loss_grad: *loss = mean (network(x) - t)^2 over n samples (device
 *                      float), grad[GRP_MLP_NPARAM] its gradient; work holds
 *                      GRP_MLP_WORK_FLOATS(n) floats of scratch
 *   grp_mlp_adam:      one Adam step (Kingma & Ba) of the weights with moments
 *                      m, v (GRP_MLP_NPARAM each, zero before step 1)
 */
#define GRP_MLP_NPARAM 4673
#define GRP_MLP_WORK_FLOATS(n) ((long long)(n) * 257)
int grp_set_guess_model(grp_ctx *ctx, const float *weights, int n_weights, const float *box,
                        int ptr_is_device);
int grp_set_harvest(grp_ctx *ctx, float *records, unsigned long long *count, long long capacity,
                    int log2_stride);
int grp_mlp_forward(const float *weights, const float *x, long long n, float *y, void *stream);
int grp_mlp_loss_grad(const float *weights, const float *x, const float *target, long long n,
                      float *grad, float *loss, float *work, void *stream);
int grp_mlp_adam(float *weights, const float *grad, float *m, float *v, int step, float lr,
                 float beta1, float beta2, float eps, void *stream);

/*
 * Leading-term Riemann problems in bulk: the exact ideal-gas solver of the
 * flux kernel (Toro-Titarev GRP, Section 2: Newton on the star pressure to a
 * relative change below newton_rtol, then one more iteration) applied to n
 * independent pairs of conserved states, from the start `guess` (GRP_GUESS_*;
 * GRP_GUESS_MLP needs `weights` and `box` as for grp_set_guess_model, device
 * pointers, and serves strong data only, the rest starting from PVRS).
 * QL, QR: device, 3 planes of n doubles (rho, m, E).  p_start: NULL, or
 * device [n] explicit Newton starts (then `guess` only picks the fallback,
 * which is PVRS).  Out (device): ps[n] the
 * star pressure (0 unless status is 0), iters[n] the Newton iterations of all
 * attempts, status[n] 0 ok / 1 no convergence within newton_max_iter /
 * 2 vacuum data, used[n] (may be NULL) 1 where the learned guess started the
 * converged run.  Ordered on `stream`.  Errors: GRP_E_INVALID_ARG,
 * GRP_E_NO_MODEL, GRP_E_CUDA.
 */
int grp_riemann_batch(double gamma, int guess, double newton_rtol, int newton_max_iter,
                      const float *weights, const float *box, long long n, const double *QL,
                      const double *QR, const double *p_start, double *ps, int *iters, int *status,
                      unsigned char *used, void *stream);

/* Number of kernel launches this context has enqueued since grp_create. */
long long grp_launch_count(const grp_ctx *ctx);

/*
 * Kernel timing for roofline reports.  With timing enabled, every flux-kernel
 * launch of grp_step is bracketed by CUDA events on the context's stream.
 * grp_get_kernel_timing waits for the recorded events, returns the summed
 * milliseconds and the number of timed launches since the last call, and
 * clears the record.  Timing adds two event records per step and nothing else.
 */
int grp_set_kernel_timing(grp_ctx *ctx, int enable);
int grp_get_kernel_timing(grp_ctx *ctx, double *flux_ms, long long *flux_launches);

/*
 * FP64 throughput probe: runs a grid of independent fused multiply-add chains
 * on `device` (one launch, about 0.2 s) and returns the measured FP64 rate in
 * FLOP/s (an FMA counts 2).  The denominator of FP64 roofline fractions.
 */
int grp_probe_fp64_peak(int device, double *flops_per_s);

/*
 * One time step of one domain without any device allocation.  (The paper has
 * no counterpart: this is an integration entry point of this library.)
 *
 * For callers that cannot call cudaMalloc -- code running inside another
 * framework's memory pool or allocator hooks, plug-ins whose host process owns
 * all device memory, loops that must not allocate after start-up.  It runs the
 * same kernels as grp_step (flat form, dt = C dx / S_max of the input averages,
 * clipped to t_end, newton_rtol 1e-12, newton_max_iter 50, PVRS guess) on
 * buffers the caller owns, and keeps its scratch (interface fluxes, repair
 * flags, per-domain words, index tables) in a file-scope __device__ array of
 * the library sized for GRP_NOALLOC_MAX_CELLS cells; every GPU that loads the
 * library holds that array (about 3.5 MB) until the process exits.
 *   avg_in, iface_in:   device, C planes of n_cells / n_ifaces doubles (read)
 *   avg_out, iface_out: device, same sizes (written); must not alias the inputs
 *   t, t_end:           time of the input state, end time (INFINITY: none)
 *   *t_out, *status_out: host; the new time and the GRP_ST_* status
 *   stream:             cudaStream_t of the work (NULL = default stream)
 * n_ifaces = n_cells + (bc == GRP_BC_TRANSMISSIVE).  Allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.  The first call on a
 * device (with that device current) looks up the device address of the scratch
 * array and keeps it for that device; make that first call before any stream
 * capture.  A reset of the device's primary context (cudaDeviceReset)
 * invalidates the kept address: do not call this entry point on a device after
 * resetting it in the same process.  A launch error pending from earlier,
 * unrelated work on the calling thread is cleared on entry, not reported.  Every call shares the
 * scratch and it keeps the last call's contents; the call clears what must
 * start at zero.  Calls that overlap on the GPU (other streams, other host
 * threads) race on the scratch: serialise them.  Synchronises `stream` before
 * returning.  Errors: GRP_E_INVALID_ARG (including n_cells >
 * GRP_NOALLOC_MAX_CELLS), GRP_E_CUDA.
 */
#define GRP_NOALLOC_MAX_CELLS 65536
int grp_step_noalloc(int system, double lambda, double gamma, int M, double cfl, int n_cells,
                     double x_left, double x_right, int bc, const double *avg_in,
                     const double *iface_in, double *avg_out, double *iface_out, double t,
                     double t_end, double *t_out, int *status_out, void *stream);

/* Release every device allocation of the context; ctx may be NULL. */
void grp_destroy(grp_ctx *ctx);

/* Static text for a return code (negative) or a domain status (non-negative). */
const char *grp_status_string(int code);

#ifdef __cplusplus
}
#endif
#endif
