// Kernels of one FV+GRPrec time step over a flat batch of 1D domains.
//
// One step is a short fixed sequence of launches on the context's stream:
//   k_smax         per cell   S_max of every domain (warp max + atomicMax)
//   k_flux<M>      per iface  GRPrec traces -> GRP -> flux, new interface data
//   k_update       per cell   candidate averages, detection flags, list of troubled cells
//   k_repair_list  per listed troubled cell: first-order fluxes on its interfaces
//   k_update_list  per listed repaired interface: candidates of its cells again
//                  (the last two MAX_REPAIR times, on fixed grids)
//   k_finish       per domain time, step count, status, buffer bookkeeping
// Every kernel derives dt from the same per-domain words with the same
// expression, so no extra launch is needed to publish it.
#pragma once
#include "grp_device.cuh"

namespace grp {

constexpr int NSTATS = 9;
enum { S_STEPS = 0, S_NEWTON_SUM, S_NEWTON_MAX, S_RECON_FB, S_FLUX_FB, S_RS_CALLS, S_LOW, S_GUESS_USED,
       S_GUESS_REJ };
constexpr int MAX_REPAIR = 4;   // rounds of the a-posteriori first-order repair
constexpr double DMP_REL = 1e-2; // relaxation of the discrete maximum principle

// This step's time step of one domain, computed once per step after S_max.
struct DomStep {
  double dt, nu, dt_cfl;             // dt (clipped at t_end), dt / dx, the CFL dt kept for dt_hold
  int active, last;                  // the domain steps; this step reaches t_end
  double tg[3];                      // nu x the Gauss nodes of the flux time integral (degree M: (M+2)/2 nodes)
};

struct StepArgs {
  int sys, M, C;
  int recon;                         // 0 GRPrec (Section 3.1), 1 GRPrecNL (Sections 3.3-3.4)
  Phys ph;
  double cfl, t_end;
  int dt_hold;
  int n_domains;
  long long ncell, nif;              // plane lengths
  const long long* cell_off;         // [D+1]
  const long long* if_off;           // [D+1]
  const int* cell_dom;               // [ncell]
  const int* if_dom;                 // [nif]
  const double* dx;                  // [D]
  const unsigned char* bc;           // [D]
  // state
  const double* avg;                 // current averages  [C][ncell]
  double* avg_new;                   // next averages     [C][ncell]
  const double* ifc;                 // current interface data [C][nif]
  double* ifc_new;                   // next interface data    [C][nif]
  double* flux;                      // scratch [C][nif]
  double* srcv = nullptr;            // [C][ncell] numerical source of every cell this step, or null (S = 0)
  double* pold;                      // [ncell] pressure of the current averages, written with S_max
  DomStep* ds;                       // [D] this step's time step of every domain (k_dt or in-block)
  unsigned char* low;                // [nif] 0 high order; 1 first order (flux kernel); 2+r repaired in round r
  unsigned char* troubled;           // [ncell] 0 ok; 1 outside the relaxed DMP; 2 inadmissible
  // per-domain words
  double* t;                         // [D]
  double* dt_prev;                   // [D]
  int* nstep;                        // [D]
  int* status;                       // [D]
  unsigned long long* smax_bits;     // [D] S_max as the bits of a non-negative double
  int* bad;                          // [(MAX_REPAIR+1) * D] newly troubled cells (repair wanted) after pass p
  int* inad;                         // [D] number of inadmissible candidate averages
  int* fail;                         // [D] non-zero: solver failure code this step
  int* any_bad;                      // [MAX_REPAIR+1] any domain troubled after pass p
  // repair work lists of the flat form (compacted: the rounds touch only the
  // troubled cells and their interfaces)
  int* tlist[2];                     // [ncell] troubled cells after pass p-1, in tlist[p & 1]
  int* ilist;                        // [nif] interfaces repaired in the current round
  int* lcount;                       // [2 (MAX_REPAIR+1)]: troubled cells after pass p-1 at [p];
                                     //   interfaces repaired in round r at [MAX_REPAIR + 1 + r]
  unsigned long long* stats;         // [D][NSTATS]
  // interfaces of the flux kernel deferred to k_flux_hard (Riemann data that
  // are not equal data, at the interpolating degrees): their traces and index,
  // solved in a second pass with dense warps; hard_cap = 0 defers nothing
  double* hard_tr = nullptr;         // [2 C (M+1)][hard_cap]: tL then tR, coefficient-major
  long long* hard_idx = nullptr;     // [hard_cap] interface
  // admissibility of the interface data (Euler, flat form at degrees 2 and 4):
  // adm_in[j] = 1 when the current datum at j is admissible (null: test the
  // data), adm_out[j] written with every new datum (null: not kept).  Each
  // datum is tested once, where it is written, instead of twice, as the edge
  // value of the two cells it bounds.
  const unsigned char* adm_in = nullptr;   // [nif]
  unsigned char* adm_out = nullptr;        // [nif]
  unsigned* hard_count = nullptr;    // [3]: interfaces offered this step, blocks of k_flux_hard done,
                                     //   interfaces taken by k_flux_hard
  int hard_cap = 0;
  // harvest of (features, ln(p*/pbar), iterations) records, may be null
  float* harvest;                    // [harvest_cap][8]
  unsigned long long* harvest_count; // records offered (may exceed the capacity)
  long long harvest_cap;
  int harvest_log2_stride;           // keep one offered interface in 2^k
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Warp-aggregated statistics.  Called by all 32 lanes of a warp, converged
// (the kernels that use it never return early); d < 0 marks a lane without a
// domain.  One atomic per group of lanes that share a domain.
__device__ __forceinline__ void warp_stat_add(unsigned long long* stats, int d, int which, unsigned v)
{
  const unsigned grp = __match_any_sync(0xffffffffu, d);
  const unsigned s = __reduce_add_sync(grp, v);
  if (d >= 0 && lane_id() == __ffs(grp) - 1 && s) atomicAdd(stats + (long long)d * NSTATS + which, (unsigned long long)s);
}

__device__ __forceinline__ void warp_stat_max(unsigned long long* stats, int d, int which, unsigned v)
{
  const unsigned grp = __match_any_sync(0xffffffffu, d);
  const unsigned s = __reduce_max_sync(grp, v);
  if (d >= 0 && lane_id() == __ffs(grp) - 1 && s) atomicMax(stats + (long long)d * NSTATS + which, (unsigned long long)s);
}

// The eight per-interface counters of the flux kernels, aggregated per warp
// and domain with one match and four reductions: the Newton sum and maximum,
// and two words packing the small counters (RS calls 0..2 in 7 bits; the 0/1
// flags in 6 bits each: at most 64 and 32 per warp).  st: newton sum, newton
// max, RS calls, truncated, first order, recon fallback, learned guess used,
// learned guess rejected.
__device__ __forceinline__ void warp_flux_stats(unsigned long long* stats, int d, const unsigned st[8], bool guess)
{
  const unsigned grp = __match_any_sync(0xffffffffu, d);
  const unsigned nsum = __reduce_add_sync(grp, st[0]);
  const unsigned nmax = __reduce_max_sync(grp, st[1]);
  const unsigned wa = __reduce_add_sync(grp, st[2] | (st[3] << 7) | (st[4] << 14) | (st[5] << 21));
  const unsigned wb = guess ? __reduce_add_sync(grp, st[6] | (st[7] << 6)) : 0u;
  if (d >= 0 && lane_id() == __ffs(grp) - 1) {
    unsigned long long* S = stats + (long long)d * NSTATS;
    if (nsum) atomicAdd(S + S_NEWTON_SUM, (unsigned long long)nsum);
    if (nmax) atomicMax(S + S_NEWTON_MAX, (unsigned long long)nmax);
    const unsigned rs = wa & 127u, tr = (wa >> 7) & 127u, lo = (wa >> 14) & 127u, fb = (wa >> 21) & 127u;
    if (rs) atomicAdd(S + S_RS_CALLS, (unsigned long long)rs);
    if (tr) atomicAdd(S + S_FLUX_FB, (unsigned long long)tr);
    if (lo) atomicAdd(S + S_LOW, (unsigned long long)lo);
    if (fb) atomicAdd(S + S_RECON_FB, (unsigned long long)fb);
    const unsigned gu = wb & 63u, gr = (wb >> 6) & 63u;
    if (gu) atomicAdd(S + S_GUESS_USED, (unsigned long long)gu);
    if (gr) atomicAdd(S + S_GUESS_REJ, (unsigned long long)gr);
  }
}

// Time-step rule (Section 4.1): dt = C dx / S_max, recomputed every dt_hold
// steps, the last step clipped to t_end.  false: the domain does not move.
// Time step of domain d from its words (S_max complete): one division.
__device__ __forceinline__ void compute_domain_step(const StepArgs& a, int d)
{
  DomStep r{0.0, 0.0, 0.0, 0, 0, {0.0, 0.0, 0.0}};
  const double t = a.t[d];
  if (a.status[d] == ST_OK && t < a.t_end) {
    const double dtp = a.dt_prev[d];
    double dt_cfl;
    if (a.nstep[d] % a.dt_hold == 0 || !(dtp > 0.0)) {
      const double smax = a.sys == SYS_ADV ? fabs(a.ph.lambda) : __longlong_as_double((long long)a.smax_bits[d]);
      dt_cfl = __ddiv_rn(__dmul_rn(a.cfl, a.dx[d]), smax);
    } else {
      dt_cfl = dtp;
    }
    double dt = dt_cfl;
    if (__dadd_rn(t, dt) >= a.t_end) { dt = __dadd_rn(a.t_end, -t); r.last = 1; }
    r.dt = dt;
    r.dt_cfl = dt_cfl;
    r.nu = __ddiv_rn(dt, a.dx[d]);
    // the GRP's Gauss times, formed once per domain instead of per interface
    const int G = (a.M + 2) / 2;
    for (int al = 0; al < G; ++al) r.tg[al] = __dmul_rn(r.nu, gauss_node(G, al));
    r.active = 1;
  }
  a.ds[d] = r;
}

// The step's time step of domain d; false when the domain does not step.
__device__ __forceinline__ bool domain_dt(const StepArgs& a, int d, double& dt, double& dt_cfl, bool& last)
{
  const DomStep& r = a.ds[d];
  dt = r.dt;
  dt_cfl = r.dt_cfl;
  last = r.last != 0;
  return r.active != 0;
}

// Per-domain words of the step: repair flags and failure code cleared (every
// system; the S_max pass clears them too for the Euler equations), then the
// time step.
static __global__ void k_dt(StepArgs a)
{
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d < a.n_domains) {
    for (int p = 0; p <= MAX_REPAIR; ++p) a.bad[p * a.n_domains + d] = 0;
    a.inad[d] = 0;
    a.fail[d] = 0;
    compute_domain_step(a, d);
  }
}

// Neighbour cells of cell i (domain-local) under the domain's boundary rule:
// periodic wrap, or a ghost that copies the boundary cell.
__device__ __forceinline__ void nbr(int i, int N, int bc, int& im, int& ip)
{
  if (bc == 0) { im = i == 0 ? N - 1 : i - 1; ip = i == N - 1 ? 0 : i + 1; }
  else { im = i == 0 ? 0 : i - 1; ip = i == N - 1 ? N - 1 : i + 1; }
}

__device__ __forceinline__ void reset_domain_words(const StepArgs& a, int d)
{
  for (int p = 0; p <= MAX_REPAIR; ++p) a.bad[p * a.n_domains + d] = 0;
  a.inad[d] = 0;
  a.fail[d] = 0;
}

// S_max contribution of cell gi (all 32 lanes call; valid = false lanes add nothing)
__device__ __forceinline__ void smax_cell(const StepArgs& a, long long gi, bool valid)
{
  unsigned long long bits = 0ull;
  int d = -1;
  if (valid) {
    d = a.cell_dom[gi];
    const double g = a.ph.gamma;
    const double r = a.avg[gi], m = a.avg[a.ncell + gi], E = a.avg[2 * a.ncell + gi];
    // |u| + c with one refined reciprocal and one reciprocal square root (an
    // ulp or two from the correctly rounded divisions and root)
    const double ir = rcp64(r);
    const double u = m * ir;
    const double p = a.ph.gm1 * (E - 0.5 * m * u);
    a.pold[gi] = p;                                // for the discrete maximum principle of the update
    const double c2 = g * p * ir;
    // c2 <= 0 or not a number: no sound speed; |u| + c not a number: 0
    // (both tests on the bits, off the FP64 pipe)
    const double sp = fabs(u) + (positive(c2) ? c2 * rsqrt(c2) : 0.0);
    const long long sb = __double_as_longlong(sp);
    bits = sb >= 0ll && sb <= 0x7ff0000000000000ll ? (unsigned long long)sb : 0ull;
  }
  const int d0 = __shfl_sync(0xffffffffu, d, 0);
  if (__all_sync(0xffffffffu, d == d0 && d >= 0)) {
    unsigned long long mx = bits;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
      mx = o > mx ? o : mx;
    }
    if (lane_id() == 0) atomicMax(a.smax_bits + d, mx);
  } else if (valid) {
    atomicMax(a.smax_bits + d, bits);
  }
}

// ------------------------------------------------------------------ k_smax
static __global__ void k_smax(StepArgs a)
{
  const long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && threadIdx.x <= MAX_REPAIR) a.any_bad[threadIdx.x] = 0;
  if (blockIdx.x == 0 && threadIdx.x < 2 * (MAX_REPAIR + 1) && a.lcount) a.lcount[threadIdx.x] = 0;
  const bool valid = gi < a.ncell;
  if (valid && gi == a.cell_off[a.cell_dom[gi]]) reset_domain_words(a, a.cell_dom[gi]);
  if (a.sys != SYS_EULER) return;                  // uniform
  smax_cell(a, gi, valid);
}

// ------------------------------------------------------------------ traces
// Taylor coefficients (scaled) of cell `cell`'s reconstruction at its right
// (side = +1) or left (side = -1) edge, component c; with the degree-0
// fallback when the cell's traces are inadmissible (Euler).
// NL: GRPrecNL, in characteristic variables of the cell average for the
// Euler equations (Section 3.1: systems are reconstructed in characteristic
// variables; linear GRPrec commutes with that projection and runs on the
// conserved variables directly).
template <int SYS, int M, bool NL>
__device__ __forceinline__ void cell_coeffs(const StepArgs& a, long long c0, long long i0, int N, int bc, int i,
                                            double b[3][5], bool& fallback)
{
  int im, ip;
  nbr(i, N, bc, im, ip);
  const int jl = i, jr = (bc == 0) ? (i == N - 1 ? 0 : i + 1) : i + 1;
  constexpr int C = SYS == SYS_EULER ? 3 : 1;
  if (!NL) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const double* A = a.avg + c * a.ncell + c0;
      const double* G = a.ifc + c * a.nif + i0;
      const double qm = (M >= 3) ? A[im] : 0.0, qp = (M >= 3) ? A[ip] : 0.0;
      grprec_coeffs<M>(qm, A[i], qp, G[jl], G[jr], b[c]);
    }
  } else {
    // the further interfaces i-3/2, i+3/2; outside a transmissive end the
    // ghost state (the boundary cell's average) holds on its interfaces too
    const int jll = bc == 0 ? (i == 0 ? N - 1 : i - 1) : i - 1;
    const int jrr = bc == 0 ? (jr == N - 1 ? 0 : jr + 1) : i + 2;
    double d[C][7];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const double* A = a.avg + c * a.ncell + c0;
      const double* G = a.ifc + c * a.nif + i0;
      d[c][0] = A[im]; d[c][1] = A[i]; d[c][2] = A[ip];
      d[c][3] = jll < 0 ? A[0] : G[jll];
      d[c][4] = G[jl]; d[c][5] = G[jr];
      d[c][6] = (bc != 0 && jrr > N) ? A[N - 1] : G[jrr];
    }
    const double dx = a.dx[(int)a.cell_dom[c0 + i]];
    if (SYS == SYS_EULER) {
      const double Qi[3] = {d[0][1], d[1][1], d[2][1]};
      const double iri = rcp64(Qi[0]);
      Prim wi;
      wi.r = Qi[0];
      wi.u = Qi[1] * iri;
      wi.p = a.ph.gm1 * (Qi[2] - 0.5 * Qi[1] * wi.u);
      const Eig e = make_eig(a.ph, Qi, wi, iri);
      double w[3][7];
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        const double D[3] = {d[0][j], d[1][j], d[2][j]};
        double v[3];
        char_proj(e, D, v);
        w[0][j] = v[0]; w[1][j] = v[1]; w[2][j] = v[2];
      }
      double bw[3][5];
#pragma unroll
      for (int k = 0; k < 3; ++k) grprec_nl_coeffs<M>(w[k], dx, bw[k]);
#pragma unroll
      for (int c = 0; c < 3; ++c) b[c][0] = d[c][1];
#pragma unroll
      for (int q = 1; q <= 4; ++q) {
        const double v[3] = {bw[0][q], bw[1][q], bw[2][q]};
        double D[3];
        char_back(e, v, D);
        b[0][q] = D[0]; b[1][q] = D[1]; b[2][q] = D[2];
      }
    } else {
      grprec_nl_coeffs<M>(d[0], dx, b[0]);
    }
  }
  fallback = false;
  if (SYS == SYS_EULER) {
    double tm[3], tp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double t[M + 1];
      edge_taylor<M>(b[c], -1.0, t); tm[c] = t[0];
      edge_taylor<M>(b[c], 1.0, t); tp[c] = t[0];
    }
    const double g = a.ph.gamma;
    if (!admissible(g, tm[0], tm[1], tm[2]) || !admissible(g, tp[0], tp[1], tp[2])) {
      fallback = true;
#pragma unroll
      for (int c = 0; c < 3; ++c) { b[c][1] = b[c][2] = b[c][3] = b[c][4] = 0.0; }
    }
  }
}

// First-order Godunov flux and state at interface j from cell averages.
// Newton starts from the adaptive classical estimate (these data are strong;
// p* does not depend on the start).  The learned guess is not used here: the
// network's evaluation is a chain of thousands of dependent FP32 operations,
// longer than the Newton iterations it saves, and the repair kernels are
// bound by that latency.
template <bool G75>
// info (harvest): the network features and the two-rarefaction base of
// strong data are recorded on the way (the start stays the classical one).
static __device__ int first_order(const StepArgs& a, long long c0, int N, int bc, int j, double F[3], double Q0[3], int& iters,
                                  RSInfo* info = nullptr)
{
  int cl, cr;
  if (bc == 0) { cl = j == 0 ? N - 1 : j - 1; cr = j; }
  else { cl = j == 0 ? 0 : j - 1; cr = j == N ? N - 1 : j; }
  double QL[3], QR[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) { QL[c] = a.avg[c * a.ncell + c0 + cl]; QR[c] = a.avg[c * a.ncell + c0 + cr]; }
  Prim W;
  Phys ph = a.ph;
  ph.guess = GUESS_ADAPTIVE;
  ph.features = info ? 2 : 0;
  const int st = riemann_state<G75>(ph, QL, QR, true, Q0, W, iters, info);
  if (st != ST_OK && st != ST_VACUUM) return st;
  if (positive(Q0[0])) euler_flux(a.ph.gamma, Q0[0], Q0[1], Q0[2], F);
  else F[0] = F[1] = F[2] = 0.0;
  return ST_OK;
}

// The admissibility of one or two conserved states as a flag, out of line:
// the flux kernels call these only where no flag was kept (the first step
// after new data, a truncated series, a first-order datum), and a call is a
// branch the compiler cannot turn into predicated FP64 instructions that every
// lane would issue.
static __device__ __noinline__ unsigned char adm_flag(double g, double r, double m, double E)
{
  return admissible(g, r, m, E) ? 1 : 0;
}
static __device__ __noinline__ bool adm_pair(double g, double r0, double m0, double E0, double r1, double m1, double E1)
{
  return admissible(g, r0, m0, E0) && admissible(g, r1, m1, E1);
}

// ------------------------------------------------------------------ k_flux
// Taylor coefficients of cell `cell`'s reconstruction at its left (em) and
// right (ep) edge, all components; fb: the degree-0 fallback was taken.
// FLAGS: the kernel keeps admissibility flags of the interface data (read
// when a.adm_in is set, else the data are tested out of line).
template <int SYS, int M, bool NL, bool FLAGS = false>
__device__ __forceinline__ void cell_edges(const StepArgs& a, long long c0, long long i0, int N, int bc, int cell,
                                           double em[][M + 1], double ep[][M + 1], bool& fb)
{
  constexpr int C = SYS == SYS_EULER ? 3 : 1;
  double b[3][5];
  if (!NL && (M == 2 || M == 4)) {
    // Degrees 2 and 4 interpolate the cell's interface data (Section 3.1):
    // the polynomial's values at the edges are g_{i-1/2} and g_{i+1/2}
    // themselves, so they are taken as loaded and only the derivative
    // coefficients are evaluated.  The degree-0 fallback tests those values.
    int im, ip;
    nbr(cell, N, bc, im, ip);
    const int jl = cell, jr = (bc == 0) ? (cell == N - 1 ? 0 : cell + 1) : cell + 1;
    double gl[3], gr[3], q0[3];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const double* A = a.avg + c * a.ncell + c0;
      const double* G = a.ifc + c * a.nif + i0;
      const double qm = (M >= 3) ? A[im] : 0.0, qp = (M >= 3) ? A[ip] : 0.0;
      q0[c] = A[cell];
      gl[c] = G[jl];
      gr[c] = G[jr];
      grprec_coeffs<M>(qm, q0[c], qp, gl[c], gr[c], b[c]);
    }
    fb = false;
    if (SYS == SYS_EULER) {
      if (!FLAGS)
        fb = !admissible(a.ph.gamma, gl[0], gl[1], gl[2]) || !admissible(a.ph.gamma, gr[0], gr[1], gr[2]);
      else if (a.adm_in)
        fb = !(a.adm_in[i0 + jl] & a.adm_in[i0 + jr]);
      else
        fb = !adm_pair(a.ph.gamma, gl[0], gl[1], gl[2], gr[0], gr[1], gr[2]);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      double tm[M + 1], tp[M + 1];
      edge_taylor<M>(b[c], -1.0, tm);
      edge_taylor<M>(b[c], 1.0, tp);
      em[c][0] = fb ? q0[c] : gl[c];
      ep[c][0] = fb ? q0[c] : gr[c];
#pragma unroll
      for (int k = 1; k <= M; ++k) {
        em[c][k] = fb ? 0.0 : tm[k];
        ep[c][k] = fb ? 0.0 : tp[k];
      }
    }
    return;
  }
  cell_coeffs<SYS, M, NL>(a, c0, i0, N, bc, cell, b, fb);
#pragma unroll
  for (int c = 0; c < C; ++c) {
    edge_taylor<M>(b[c], -1.0, em[c]);
    edge_taylor<M>(b[c], 1.0, ep[c]);
  }
}

// The ghost beyond a transmissive end: the constant state of boundary cell `cell`.
template <int SYS, int M>
__device__ __forceinline__ void ghost_edge(const StepArgs& a, long long c0, int cell, double t[][M + 1])
{
  constexpr int C = SYS == SYS_EULER ? 3 : 1;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    t[c][0] = a.avg[c * a.ncell + c0 + cell];
#pragma unroll
    for (int k = 1; k <= M; ++k) t[c][k] = 0.0;
  }
}

// Harvest of a solve the network served (strong data with a shock): keep one
// in 2^k, by a hash of (interface, step).
__device__ __forceinline__ void harvest_record(const StepArgs& a, long long gj, int d, const RSInfo& info, int iters)
{
  unsigned h = (unsigned)gj * 2654435761u ^ ((unsigned)a.nstep[d] * 2246822519u);
  h ^= h >> 15; h *= 2654435761u; h ^= h >> 13;
  if ((h & ((1u << a.harvest_log2_stride) - 1u)) == 0u) {
    const unsigned long long k = atomicAdd(a.harvest_count, 1ull);
    if ((long long)k < a.harvest_cap) {
      float* r = a.harvest + 8 * k;
#pragma unroll
      for (int i = 0; i < 6; ++i) r[i] = info.x[i];
      r[6] = (float)(log(info.ps / info.base) / (MLP_T_SCALE * info.s3));
      r[7] = (float)iters;
    }
  }
}

// The GRP at interface gj of an active domain d from the Taylor coefficients
// of the two one-sided reconstructions (tL: left cell at its right edge, tR:
// right cell at its left edge): flux, new interface datum, statistics.
// SRC: the GRP with the source term (eq. eq:GRP): its series carries dx S.
// lead: the leading Riemann problem, solved by the caller (or null).
template <int SYS, int M, bool G75, bool SRC = false>
__device__ __forceinline__ void grp_at(const StepArgs& a, long long gj, int d, long long c0, int N, int bc, int j,
                                       const double tL[][M + 1], const double tR[][M + 1], unsigned st[8],
                                       const Lead* lead = nullptr)
{
  constexpr int C = SYS == SYS_EULER ? 3 : 1;
  a.low[gj] = 0;
  const double nu = a.ds[d].nu;
  const double hsrc = SRC ? (SYS == SYS_ADV ? a.ph.src_k : -a.ph.src_k) * a.dx[d] : 0.0;
  double F[3] = {0.0, 0.0, 0.0}, gnew[3] = {0.0, 0.0, 0.0};
  if (SYS == SYS_ADV) {
    grp_adv<M, SRC>(a.ph.lambda, nu, tL[0], tR[0], F[0], gnew[0], hsrc);
  } else {
    int iters = 0;
    bool trunc = false;
    RSInfo info;
    int rs_st = grp_euler<M, G75, SRC>(a.ph, nu, tL, tR, F, gnew, iters, trunc, &info, hsrc, lead, a.ds[d].tg);
    // an untruncated series passed the admissibility test at tau = dt: its
    // datum is admissible without a second test
    const bool adm_known = rs_st == ST_OK && !trunc;
    st[2] = 1;
    st[3] = trunc ? 1u : 0u;
    st[6] = info.guess == 1 ? 1u : 0u;
    st[7] = info.guess == 2 ? 1u : 0u;
    if (a.harvest && info.has_x && rs_st == ST_OK) harvest_record(a, gj, d, info, iters);
    if (rs_st != ST_OK) {
      // no solution of the traces' Riemann problem: first-order flux here
      int it2 = 0;
      rs_st = first_order<G75>(a, c0, N, bc, j, F, gnew, it2);
      iters += it2;
      st[2] = 2;
      st[4] = 1;
      a.low[gj] = 1;
      if (rs_st != ST_OK) atomicExch(a.fail + d, rs_st);
    }
    st[0] = (unsigned)iters;
    st[1] = (unsigned)iters;
    if (a.adm_out) {
      unsigned char f = 1;
      if (!adm_known) f = adm_flag(a.ph.gamma, gnew[0], gnew[1], gnew[2]);
      a.adm_out[gj] = f;
    }
  }
#pragma unroll
  for (int c = 0; c < C; ++c) {
    a.flux[c * a.nif + gj] = F[c];
    a.ifc_new[c * a.nif + gj] = gnew[c];
  }
}

// Warps overlap by one interface: warp w owns interfaces 31 w .. 31 w + 30.
// Every lane reconstructs the left cell of its interface; the right cell of
// an interface is the left cell of the next one, so its left-edge expansion
// comes from the next lane by a shuffle, and lane 31 (the first interface of
// the next warp) only supplies that cell to lane 30.  32 reconstructions serve
// 31 interfaces, instead of two per interface.
__host__ __device__ constexpr long long flux_threads(long long nif) { return (nif + 30) / 31 * 32; }

// Every thread of the grid reaches the shuffles and the statistics (no early
// return), so the warp-synchronous operations see a full warp.  At least
// GRP_FLUX_MIN_BLOCKS (default 3) blocks of 128 per SM: that lets the compiler
// keep about 130-140 registers per thread, which measured 11 % faster on the
// batched workload than the ~108 it picks for 128-thread blocks without the
// bound.
#ifndef GRP_FLUX_MIN_BLOCKS
#define GRP_FLUX_MIN_BLOCKS 3
#endif
#ifndef GRP_FLUX_TPB
#define GRP_FLUX_TPB 128
#endif
// The numerical source of cell `cell` (SRC kernels): its reconstruction
// coefficients again (linear GRPrec; degree 0 when its traces were
// inadmissible), then the source average of its own evolution.
template <int SYS, int M>
__device__ __forceinline__ void cell_source(const StepArgs& a, long long c0, long long i0, int N, int bc, int cell,
                                            bool fb, int d)
{
  constexpr int C = SYS == SYS_EULER ? 3 : 1;
  int im, ip;
  nbr(cell, N, bc, im, ip);
  const int jl = cell, jr = (bc == 0) ? (cell == N - 1 ? 0 : cell + 1) : cell + 1;
  double b[3][5];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const double* A = a.avg + c * a.ncell + c0;
    const double* G = a.ifc + c * a.nif + i0;
    const double qm = (M >= 3) ? A[im] : 0.0, qp = (M >= 3) ? A[ip] : 0.0;
    grprec_coeffs<M>(qm, A[cell], qp, G[jl], G[jr], b[c]);
    if (fb) b[c][1] = b[c][2] = b[c][3] = b[c][4] = 0.0;
  }
  const double nu = a.ds[d].nu, dx = a.dx[d];
  if (SYS == SYS_ADV) {
    a.srcv[c0 + cell] = cell_source_adv<M>(b[0], a.ph.lambda, nu, a.ph.src_k, dx);
  } else {
    double S[3];
    cell_source_euler<M>(a.ph, b, nu, dx, S);
#pragma unroll
    for (int c = 0; c < 3; ++c) a.srcv[c * a.ncell + c0 + cell] = S[c];
  }
}

// The flux phase of one warp: the interfaces gbase .. gbase + 30 (lanes
// 0..30), lane 31 supplying the reconstruction of the cell left of
// gbase + 31; interfaces at or beyond gend are not this call's.  All 32 lanes
// of the warp call it (shuffles and warp statistics).
// own0 <= gj < own1: the interfaces whose statistics count (a tile's halo
// interfaces are computed but counted by the tile that owns them).
// DEFER: an interface whose two traces are not equal data (a Newton solve,
// in one or two lanes of a warp while the others wait) is written to the
// hard list instead, when a slot is left, and solved by k_flux_hard.
template <int SYS, int M, bool G75, bool NL, bool SRC, bool DEFER = false>
__device__ __forceinline__ void flux_warp(const StepArgs& a, long long gbase, long long gend, long long own0 = 0,
                                          long long own1 = 0x7fffffffffffffffll)
{
  constexpr int C = SYS == SYS_EULER ? 3 : 1;
  const int lane = lane_id();
  const long long gj = gbase + lane;
  // st: newton sum, newton max, RS calls, truncated, first order, recon fallback,
  //     learned guess used, learned guess rejected
  unsigned st[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  int d = -1, j = 0, N = 0, bc = 0, cl = -1;
  long long c0 = 0, i0 = 0;
  bool active = false, fb = false;
  double em[C][M + 1], ep[C][M + 1];           // the left cell at its left and right edge
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int k = 0; k <= M; ++k) em[c][k] = ep[c][k] = 0.0;
  if (gj < gend) {
    d = a.if_dom[gj];
    i0 = a.if_off[d];
    c0 = a.cell_off[d];
    j = (int)(gj - i0);
    N = (int)(a.cell_off[d + 1] - c0);
    bc = a.bc[d];
    active = a.ds[d].active != 0;
    cl = bc == 0 ? (j == 0 ? N - 1 : j - 1) : j - 1;
    if (active && cl >= 0) cell_edges<SYS, M, NL, DEFER>(a, c0, i0, N, bc, cl, em, ep, fb);
    // each cell is the left cell of exactly one interface (lane 31 supplies a
    // reconstruction only; its interface is the next warp's lane 0)
    if (SRC && active && cl >= 0 && lane < 31) cell_source<SYS, M>(a, c0, i0, N, bc, cl, fb, d);
  }
  // the next lane's left cell at its left edge: this interface's right trace
  double rm[C][M + 1];
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int k = 0; k <= M; ++k) rm[c][k] = __shfl_down_sync(0xffffffffu, em[c][k], 1);
  double tL[C][M + 1], tR[C][M + 1];
  bool solve = false, hard = false;
  if (lane < 31 && gj < gend) {
    if (!active) {
#pragma unroll
      for (int c = 0; c < C; ++c) a.ifc_new[c * a.nif + gj] = a.ifc[c * a.nif + gj];
      if (SYS == SYS_EULER && a.adm_out)
        a.adm_out[gj] = a.adm_in ? a.adm_in[gj] : adm_flag(a.ph.gamma, a.ifc[gj], a.ifc[a.nif + gj], a.ifc[2 * a.nif + gj]);
    } else {
      // both traces by register moves (ghost states at transmissive ends), so
      // that the lanes of a warp reach the one GRP below together
      if (cl >= 0) st[5] = fb ? 1u : 0u;       // counted once per cell: at its right interface
      const double* gl = a.avg + c0;                 // the ghost left of cell 0
      const double* gr = a.avg + c0 + N - 1;         // the ghost right of cell N - 1
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const double glc = gl[c * a.ncell];
        tL[c][0] = cl >= 0 ? ep[c][0] : glc;
#pragma unroll
        for (int k = 1; k <= M; ++k) tL[c][k] = cl >= 0 ? ep[c][k] : 0.0;
      }
      // the next interface of this domain sits in the next lane (j below the
      // domain's last interface), and its left cell is this interface's right cell
      const int jlast = bc == 0 ? N - 1 : N;
      if (j >= jlast && bc == 0) {
        // last interface of a periodic domain: its right cell is cell N - 1
        double tx[C][M + 1];
        bool fb2;
        cell_edges<SYS, M, NL, DEFER>(a, c0, i0, N, bc, N - 1, rm, tx, fb2);
      }
      const bool ghost_r = j >= jlast && bc != 0;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const double grc = ghost_r ? gr[c * a.ncell] : 0.0;
        tR[c][0] = ghost_r ? grc : rm[c][0];
#pragma unroll
        for (int k = 1; k <= M; ++k) tR[c][k] = ghost_r ? 0.0 : rm[c][k];
      }
      solve = true;
      if (DEFER && a.hard_cap > 0) {
        const double QL[3] = {tL[0][0], tL[1][0], tL[2][0]}, QR[3] = {tR[0][0], tR[1][0], tR[2][0]};
        hard = !equal_data(QL, QR);
      }
    }
  } else {
    d = -1;
  }
  if (DEFER) {
    // warp-aggregated slots of the hard list (consecutive per warp)
    const unsigned bal = __ballot_sync(0xffffffffu, hard);
    if (bal) {
      const int lead = __ffs(bal) - 1;
      unsigned base = 0;
      if (lane == lead) base = atomicAdd(a.hard_count, (unsigned)__popc(bal));
      base = __shfl_sync(0xffffffffu, base, lead);
      const unsigned slot = base + (unsigned)__popc(bal & ((1u << lane) - 1u));
      if (hard && slot < (unsigned)a.hard_cap) {
        double* R = a.hard_tr + slot;
        const long long cap = a.hard_cap;
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
          for (int k = 0; k <= M; ++k) {
            R[(c * (M + 1) + k) * cap] = tL[c][k];
            R[(C * (M + 1) + c * (M + 1) + k) * cap] = tR[c][k];
          }
        a.hard_idx[slot] = gj;
        solve = false;
      }
    }
  }
  if (solve) grp_at<SYS, M, G75, SRC>(a, gj, d, c0, N, bc, j, tL, tR, st);
  __syncwarp();
  if (SYS == SYS_EULER) {
    warp_flux_stats(a.stats, gj >= own0 && gj < own1 ? d : -1, st, a.ph.guess == 2);
  }
}

// Interfaces are deferred at the interpolating degrees (2 and 4) of the
// linear reconstruction, where all but a few interfaces have equal data.
template <int SYS, int M, bool NL, bool SRC>
__host__ __device__ constexpr bool flux_defers_at()
{
  return SYS == SYS_EULER && !NL && !SRC && (M == 2 || M == 4);
}

template <int SYS, int M, bool G75, bool NL, bool SRC = false>
__global__ void __launch_bounds__(GRP_FLUX_TPB, GRP_FLUX_MIN_BLOCKS) k_flux(StepArgs a)
{
  flux_warp<SYS, M, G75, NL, SRC, flux_defers_at<SYS, M, NL, SRC>()>(
      a, (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 31, a.nif);
}

// Capacity of the hard list and whether a step's flux phase is two launches.
// The list holds a quarter of the interfaces (plus 1024): the interfaces left
// over when it is full are solved in the first pass.
inline long long hard_list_cap(long long nif) { return nif / 4 + 1024; }
inline size_t hard_doubles_per_slot(int M) { return (size_t)2 * 3 * (M + 1); }
inline bool flux_hard_net(const StepArgs& a) { return a.ph.features == 1 && a.ph.guess == 2 && a.ph.mlp_w; }
inline bool flux_defers(const StepArgs& a)
{
  return a.sys == SYS_EULER && a.recon == 0 && !a.srcv && (a.M == 2 || a.M == 4) && a.hard_cap > 0;
}

// The second pass runs one warp per block, so that a warp that finishes frees
// its slot at once (the pass is bound by the latency of its longest Newton
// chains, not by the FP64 pipe), and the warps take chunks of 32 interfaces
// from a counter until the list is done.
#ifndef GRP_HARD_TPB
#define GRP_HARD_TPB 32
#endif
#ifndef GRP_HARD_MIN_BLOCKS
#define GRP_HARD_MIN_BLOCKS 12
#endif
inline unsigned hard_blocks(long long cap, int sms)
{
  const long long need = (cap + GRP_HARD_TPB - 1) / GRP_HARD_TPB;
  const long long fill = 2ll * sms * GRP_HARD_MIN_BLOCKS;
  return (unsigned)(need < fill ? need : fill);
}

// The second pass of the flux kernel: the deferred interfaces, one per lane
// (a warp takes its chunk together, so the warp statistics see full warps).
// The last block to finish resets the list for the next step; every block
// has read the count before it counts itself done.
// NET: the learned start's network is evaluated by the whole warp for each
// lane that wants it (inference with a model; harvest and the classical starts
// take the plain instantiation).
template <int M, bool G75, bool NET>
__global__ void __launch_bounds__(GRP_HARD_TPB, GRP_HARD_MIN_BLOCKS) k_flux_hard(StepArgs a)
{
  constexpr int C = 3;
  const unsigned offered = a.hard_count[0];
  const long long n = offered < (unsigned)a.hard_cap ? offered : a.hard_cap;
  const int lane = lane_id();
  __shared__ float hs[NET ? GRP_HARD_TPB / 32 : 1][MLP_NH];
  for (;;) {
    unsigned b = 0;
    if (lane == 0) b = atomicAdd(a.hard_count + 2, 32u);
    b = __shfl_sync(0xffffffffu, b, 0);
    if ((long long)b >= n) break;
    const long long i = (long long)b + lane;
    unsigned st[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    int d = -1;
    long long gj = 0;
    double tL[C][M + 1], tR[C][M + 1];
    if (i < n) {
      gj = a.hard_idx[i];
      d = a.if_dom[gj];
      const double* R = a.hard_tr + i;
      const long long cap = a.hard_cap;
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int k = 0; k <= M; ++k) {
          tL[c][k] = R[(c * (M + 1) + k) * cap];
          tR[c][k] = R[(C * (M + 1) + c * (M + 1) + k) * cap];
        }
    }
    if (NET) {
      Side L, R;
      LearnedPre pre;
      pre.v = 0.0f;
      bool strong = false, want = false;
      if (d >= 0) {
        const double QL[3] = {tL[0][0], tL[1][0], tL[2][0]}, QR[3] = {tR[0][0], tR[1][0], tR[2][0]};
        L = make_side(a.ph, QL);
        R = make_side(a.ph, QR);
        strong = strong_data(a.ph, L, R);
        if (strong) want = learned_prep_f32(a.ph, L, R, pre.x, pre.q);
      }
      unsigned m = __ballot_sync(0xffffffffu, want);
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1u;
        float xs[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) xs[k] = __shfl_sync(0xffffffffu, pre.x[k], src);
        const float y = mlp_eval_warp(a.ph.mlp_w, xs, hs[threadIdx.x >> 5]);
        if (lane == src) pre.v = y;
      }
      if (d >= 0) {
        Lead ld;
        ld.st = riemann_sides<G75>(a.ph, L, R, false, ld.Q0, ld.W0, ld.iters, &ld.info, strong ? &pre : nullptr,
                                   strong ? 1 : 0);
        const long long i0 = a.if_off[d], c0 = a.cell_off[d];
        const int N = (int)(a.cell_off[d + 1] - c0);
        grp_at<SYS_EULER, M, G75, false>(a, gj, d, c0, N, a.bc[d], (int)(gj - i0), tL, tR, st, &ld);
      }
    } else if (d >= 0) {
      const long long i0 = a.if_off[d], c0 = a.cell_off[d];
      const int N = (int)(a.cell_off[d + 1] - c0);
      grp_at<SYS_EULER, M, G75, false>(a, gj, d, c0, N, a.bc[d], (int)(gj - i0), tL, tR, st);
    }
    __syncwarp();
    warp_flux_stats(a.stats, d, st, a.ph.guess == 2);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.hard_count + 1, 1u) == gridDim.x - 1) {
      a.hard_count[0] = 0u;
      a.hard_count[1] = 0u;
      a.hard_count[2] = 0u;
    }
  }
}

// ------------------------------------------------------------------ update
// Candidate average of cell gi from the flux array, with the a-posteriori
// detection: inadmissible, or outside the relaxed discrete maximum principle
// on density and pressure against the old averages of cells i-1, i, i+1.
// pass < 0: first update of the step; else the re-update after repair round
// `pass`, which recomputes only the cells next to an interface repaired in
// that round (every other candidate depends on unchanged fluxes).
// Returns bit 0: troubled, bit 1: inadmissible.
template <int SYS>
__device__ __forceinline__ int update_one(const StepArgs& a, long long gi, int d, int pass)
{
  constexpr int C = SYS == SYS_EULER ? 3 : 1;
  const long long c0 = a.cell_off[d], i0 = a.if_off[d];
  const int N = (int)(a.cell_off[d + 1] - c0);
  const int i = (int)(gi - c0);
  const int jl = i, jr = (a.bc[d] == 0) ? (i == N - 1 ? 0 : i + 1) : i + 1;
  if (pass >= 0) {
    // a re-update only concerns cells next to an interface repaired in this round
    const unsigned char mark = (unsigned char)(2 + pass);
    if (a.low[i0 + jl] != mark && a.low[i0 + jr] != mark) return 0;
  }
  double dt, dt_cfl;
  bool last;
  const bool active = domain_dt(a, d, dt, dt_cfl, last);
  if (!active) {
    if (pass < 0) {
#pragma unroll
      for (int c = 0; c < C; ++c) a.avg_new[c * a.ncell + gi] = a.avg[c * a.ncell + gi];
    }
    return 0;
  }
  const double r = a.ds[d].nu;
  double Q[3];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    Q[c] = a.avg[c * a.ncell + gi] - r * (a.flux[c * a.nif + i0 + jr] - a.flux[c * a.nif + i0 + jl]);
    if (a.srcv) Q[c] = fma(dt, a.srcv[c * a.ncell + gi], Q[c]);    // + dt S_i (eq. eq_finite_volume)
    a.avg_new[c * a.ncell + gi] = Q[c];
  }
  if (SYS != SYS_EULER) return 0;
  // admissible: rho > 0 and 2 E rho - m^2 = 2 rho p / (g - 1) > 0 (the
  // latter also gives the candidate's rho p below)
  const double a2 = fma(Q[2] + Q[2], Q[0], -(Q[1] * Q[1]));
  const bool adm = positive(Q[0]) && positive(a2);
  bool ok = adm;
  if (adm) {
    int im, ip;
    nbr(i, N, a.bc[d], im, ip);
    const int nb[3] = {im, i, ip};
    // old density and pressure (the pressure as reduced with S_max) of cells
    // i-1, i, i+1.  Both are positive (the old averages are admissible), and
    // positive doubles order as their bit patterns do, so the bounds come from
    // integer min / max (exactly fmin / fmax, off the FP64 pipe), and
    // max(|lo|, |hi|) is hi.
    long long lo0, hi0, lo1, hi1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const long long q = c0 + nb[k];
      const long long r = __double_as_longlong(a.avg[q]), pr = __double_as_longlong(a.pold[q]);
      lo0 = k == 0 ? r : min(lo0, r); hi0 = k == 0 ? r : max(hi0, r);
      lo1 = k == 0 ? pr : min(lo1, pr); hi1 = k == 0 ? pr : max(hi1, pr);
    }
    const double rlo = __longlong_as_double(lo0), rhi = __longlong_as_double(hi0);
    const double plo = __longlong_as_double(lo1), phi = __longlong_as_double(hi1);
    // the candidate pressure p = (g-1)(E - m^2/(2 rho)) against its bounds,
    // multiplied through by rho > 0 (admissible): no division
    const double rp = a.ph.h_gm1 * a2;
    // the band [lo - DMP_REL hi, hi + DMP_REL hi], each end one fma.  Q[0] and
    // rp are positive here, so each bound test is a signed-integer compare of
    // the bits (exact: a negative bound has a negative pattern)
    const long long q0 = __double_as_longlong(Q[0]), rq = __double_as_longlong(rp);
    ok = q0 >= __double_as_longlong(fma(-DMP_REL, rhi, rlo)) && q0 <= __double_as_longlong(fma(DMP_REL, rhi, rhi)) &&
         rq >= __double_as_longlong(fma(-DMP_REL, phi, plo) * Q[0]) &&
         rq <= __double_as_longlong(fma(DMP_REL, phi, phi) * Q[0]);
  }
  const unsigned char flag = adm ? (ok ? 0 : 1) : 2;
  const unsigned char before = pass < 0 ? 0 : a.troubled[gi];
  a.troubled[gi] = flag;
  if (flag) a.bad[(pass + 1) * a.n_domains + d] = 1;
  if (flag == 2 && before != 2) atomicAdd(a.inad + d, 1);
  if (flag != 2 && before == 2) atomicSub(a.inad + d, 1);
  return (ok ? 0 : 1) | (adm ? 0 : 2);
}

template <int SYS>
__global__ void k_update(StepArgs a, int pass)
{
  const long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pass >= 0 && a.any_bad[pass] == 0) return;
  if (gi >= a.ncell) return;
  const int d = a.cell_dom[gi];
  const bool bad = update_one<SYS>(a, gi, d, pass) & 1;
  if (bad) a.any_bad[pass + 1] = 1;
  if (pass < 0 && a.lcount) {
    // warp-aggregated append of the troubled cells to the first work list
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, bad);
    if (m) {
      const int leader = __ffs(m) - 1;
      int base = 0;
      if (lane_id() == leader) base = atomicAdd(a.lcount, __popc(m));
      base = __shfl_sync(act, base, leader);
      if (bad) a.tlist[0][base + __popc(m & ((1u << lane_id()) - 1u))] = (int)gi;
    }
  }
}

// Grid-stride helpers of the work-list kernels (their grids are fixed, so a
// captured graph serves every step).
constexpr int LIST_BLOCKS = 4 * 152, LIST_THREADS = 128;

// First-order Godunov flux at interface gj (round `pass`); appends it to the
// round's interface list.
template <bool G75>
__device__ __forceinline__ void repair_iface(const StepArgs& a, int pass, long long gj)
{
  const int d = a.if_dom[gj];
  const long long c0 = a.cell_off[d], i0 = a.if_off[d];
  const int N = (int)(a.cell_off[d + 1] - c0);
  double F[3], Q0[3];
  int iters = 0;
  RSInfo info;
  const int rs = first_order<G75>(a, c0, N, a.bc[d], (int)(gj - i0), F, Q0, iters, a.harvest ? &info : nullptr);
  // harvest: the strong data with a shock of the repair rounds (the network's
  // domain) are recorded as the flux kernel records its own
  if (a.harvest && rs == ST_OK && info.has_x) harvest_record(a, gj, d, info, iters);
  unsigned long long* S = a.stats + (long long)d * NSTATS;
  atomicAdd(S + S_NEWTON_SUM, (unsigned long long)iters);
  atomicMax(S + S_NEWTON_MAX, (unsigned long long)iters);
  atomicAdd(S + S_RS_CALLS, 1ull);
  atomicAdd(S + S_LOW, 1ull);
  if (rs != ST_OK) { atomicExch(a.fail + d, rs); return; }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a.flux[c * a.nif + gj] = F[c];
    a.ifc_new[c * a.nif + gj] = Q0[c];
  }
  if (a.adm_out) a.adm_out[gj] = admissible(a.ph.gamma, Q0[0], Q0[1], Q0[2]) ? 1 : 0;
  a.low[gj] = (unsigned char)(2 + pass);
  a.ilist[atomicAdd(a.lcount + MAX_REPAIR + 1 + pass, 1)] = (int)gj;
}

// Round `pass` of the repair from the list of troubled cells: each troubled
// cell names its right interface, and its left one unless the left cell is
// troubled too (that cell names it as its right interface, or repaired it in
// an earlier round); interfaces repaired before are skipped.  A block first
// gathers the named interfaces of its slice of the list in shared memory and
// then solves them one per thread, so the warps running Riemann problems are
// full (on this GPU a divergent FP64 instruction costs as much as a full one).
template <bool G75>
__global__ void __launch_bounds__(LIST_THREADS) k_repair_list(StepArgs a, int pass)
{
  __shared__ long long q[2 * LIST_THREADS];
  __shared__ int qn;
  const int n = a.lcount[pass];
  const int* L = a.tlist[pass & 1];
  // the list spread evenly over the whole grid: a short list gives every
  // block a few cells, so each thread solves at most one Riemann problem per
  // pass (the solves are long dependent chains; parallel ones hide latency)
  const int per = (n + (int)gridDim.x - 1) / (int)gridDim.x;
  const int chunk = per < (int)blockDim.x ? per : (int)blockDim.x;
  for (int base = blockIdx.x * chunk; base < n; base += gridDim.x * chunk) {   // uniform per block
    if (threadIdx.x == 0) qn = 0;
    __syncthreads();
    const int k = base + threadIdx.x;
    if ((int)threadIdx.x < chunk && k < n) {
      const long long gi = L[k];
      const int d = a.cell_dom[gi];
      const long long c0 = a.cell_off[d], i0 = a.if_off[d];
      const int N = (int)(a.cell_off[d + 1] - c0);
      const int bc = a.bc[d];
      const int i = (int)(gi - c0);
      const int jr = bc == 0 ? (i == N - 1 ? 0 : i + 1) : i + 1;
      const int il = bc == 0 ? (i == 0 ? N - 1 : i - 1) : i - 1;      // -1: the ghost
      if (!a.low[i0 + jr]) q[atomicAdd(&qn, 1)] = i0 + jr;
      if ((il < 0 || !a.troubled[c0 + il]) && !a.low[i0 + i] && i != jr) q[atomicAdd(&qn, 1)] = i0 + i;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < qn; e += blockDim.x) repair_iface<G75>(a, pass, q[e]);
    __syncthreads();
  }
}

// Re-update after round `pass` from the list of repaired interfaces.  The
// cells next to interface j are its right cell (whose left interface is j)
// and its left cell; the left cell is left to its own left interface when
// that was repaired in this round too, so every cell is updated once.
// Troubled results go to the next round's cell list.
template <int SYS>
__global__ void __launch_bounds__(LIST_THREADS) k_update_list(StepArgs a, int pass)
{
  const int n = a.lcount[MAX_REPAIR + 1 + pass];
  const unsigned char mark = (unsigned char)(2 + pass);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const long long gj = a.ilist[k];
    const int d = a.if_dom[gj];
    const long long c0 = a.cell_off[d], i0 = a.if_off[d];
    const int N = (int)(a.cell_off[d + 1] - c0);
    const int bc = a.bc[d];
    const int j = (int)(gj - i0);
    int cl, cr;
    if (bc == 0) { cl = j == 0 ? N - 1 : j - 1; cr = j; }
    else { cl = j - 1; cr = j == N ? -1 : j; }
    int cells[2], nc = 0;
    if (cr >= 0) cells[nc++] = cr;
    if (cl >= 0 && a.low[i0 + cl] != mark) cells[nc++] = cl;
    for (int q = 0; q < nc; ++q) {
      const long long gi = c0 + cells[q];
      if (update_one<SYS>(a, gi, d, pass) & 1) {
        a.any_bad[pass + 1] = 1;
        if (pass + 1 <= MAX_REPAIR) a.tlist[(pass + 1) & 1][atomicAdd(a.lcount + pass + 1, 1)] = (int)gi;
      }
    }
  }
}

// ------------------------------------------------------------------ repair
// Interfaces of troubled cells (inadmissible, or outside the relaxed discrete
// maximum principle) take the first-order Godunov flux (a-posteriori,
// MOOD-like, bounded to MAX_REPAIR rounds).  repair_one is the sweep form of
// the block-local kernels (k_batch, k_post); the flat form runs the rounds
// from work lists (k_repair_list, k_update_list).
template <bool G75>
static __device__ __forceinline__ void repair_one(const StepArgs& a, int pass, long long gj, int d, unsigned st[3])
{
  if (!a.bad[pass * a.n_domains + d]) return;         // only domains with new troubled cells (all active)
  if (a.low[gj]) return;
  const long long i0 = a.if_off[d], c0 = a.cell_off[d];
  const int j = (int)(gj - i0);
  const int N = (int)(a.cell_off[d + 1] - c0);
  const int bc = a.bc[d];
  int cl, cr;
  if (bc == 0) { cl = j == 0 ? N - 1 : j - 1; cr = j; }
  else { cl = j - 1; cr = j == N ? -1 : j; }
  const bool t = (cl >= 0 && a.troubled[c0 + cl]) || (cr >= 0 && a.troubled[c0 + cr]);
  if (!t) return;
  double F[3], Q0[3];
  int iters = 0;
  const int rs = first_order<G75>(a, c0, N, bc, j, F, Q0, iters);
  st[0] = (unsigned)iters;
  st[1] = 1u;
  if (rs != ST_OK) { atomicExch(a.fail + d, rs); return; }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a.flux[c * a.nif + gj] = F[c];
    a.ifc_new[c * a.nif + gj] = Q0[c];
  }
  a.low[gj] = (unsigned char)(2 + pass);
}

// ------------------------------------------------------------------ finish
// Per-domain bookkeeping at the end of a step: time, step count, the dt kept
// for dt_hold, status; clears S_max for the next step's reduction.
__device__ __forceinline__ void finish_one(const StepArgs& a, int d)
{
  double dt, dt_cfl;
  bool last;
  const bool active = domain_dt(a, d, dt, dt_cfl, last);
  a.smax_bits[d] = 0ull;
  if (!active) return;
  if (a.fail[d]) { a.status[d] = a.fail[d]; return; }
  a.t[d] = last ? a.t_end : a.t[d] + dt;
  a.nstep[d] += 1;
  a.dt_prev[d] = dt_cfl;
  a.stats[(long long)d * NSTATS + S_STEPS] += 1;
  if (a.sys == SYS_EULER && a.inad[d] > 0) a.status[d] = ST_NONPHYS;
}

static __global__ void k_finish(StepArgs a)
{
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d < a.n_domains) finish_one(a, d);
}

// ------------------------------------------------------------------ batched
// Persistent form for batches of short domains: block b owns the contiguous
// domains [grp[b], grp[b+1]) and advances them nsteps steps.  Every phase of a
// step (reset, S_max, GRP fluxes, update, repair rounds, bookkeeping) is local
// to the block, separated by __syncthreads, so one launch covers nsteps steps.
// Buffers alternate per step starting from `parity` (0: A0/I0 current).
template <int SYS, int M, bool G75, bool NL>
__global__ void __launch_bounds__(256, 2) k_batch(StepArgs a, const int* __restrict__ grp, int nsteps, int parity,
                                               double* A0, double* A1, double* I0, double* I1)
{
  __shared__ int s_any[MAX_REPAIR + 1];
  const int b = blockIdx.x, tid = threadIdx.x, bt = blockDim.x;
  const int d0 = grp[b], d1 = grp[b + 1];
  const long long cb = a.cell_off[d0], ce = a.cell_off[d1];
  const long long ib = a.if_off[d0], ie = a.if_off[d1];
  for (int s = 0; s < nsteps; ++s) {
    StepArgs w = a;
    const int par = (parity + s) & 1;
    w.avg = par ? A1 : A0;
    w.avg_new = par ? A0 : A1;
    w.ifc = par ? I1 : I0;
    w.ifc_new = par ? I0 : I1;
    for (int d = d0 + tid; d < d1; d += bt) reset_domain_words(w, d);
    if (tid <= MAX_REPAIR) s_any[tid] = 0;
    __syncthreads();
    if (SYS == SYS_EULER)
      for (long long base = cb; base < ce; base += bt) smax_cell(w, base + tid, base + tid < ce);
    __syncthreads();
    for (int d = d0 + tid; d < d1; d += bt) compute_domain_step(w, d);
    __syncthreads();
    // the flux kernel's warp form: warps overlapping by one interface, each
    // cell reconstructed once per warp
    for (long long base = ib + 31ll * (tid >> 5); base < ie; base += 31ll * (bt >> 5))
      flux_warp<SYS, M, G75, NL, false>(w, base, ie);
    __syncthreads();
    for (long long gi = cb + tid; gi < ce; gi += bt)
      if (update_one<SYS>(w, gi, a.cell_dom[gi], -1) & 1) s_any[0] = 1;
    __syncthreads();
    if (SYS == SYS_EULER) {
      for (int r = 0; r < MAX_REPAIR; ++r) {
        if (s_any[r] == 0) break;                       // uniform: read after a barrier
        for (long long base = ib; base < ie; base += bt) {
          const long long gj = base + tid;
          unsigned st[3] = {0u, 0u, 0u};
          int d = -1;
          if (gj < ie) {
            d = a.if_dom[gj];
            repair_one<G75>(w, r, gj, d, st);
          }
          __syncwarp();
          warp_stat_add(w.stats, d, S_NEWTON_SUM, st[0]);
          warp_stat_max(w.stats, d, S_NEWTON_MAX, st[0]);
          warp_stat_add(w.stats, d, S_RS_CALLS, st[1]);
          warp_stat_add(w.stats, d, S_LOW, st[1]);
        }
        __syncthreads();
        for (long long gi = cb + tid; gi < ce; gi += bt)
          if (update_one<SYS>(w, gi, a.cell_dom[gi], r) & 1) s_any[r + 1] = 1;
        __syncthreads();
      }
    }
    for (int d = d0 + tid; d < d1; d += bt) finish_one(w, d);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ split
// Second half of a step in the split form: block b owns the consecutive
// domains [grp[b], grp[b+1]) whose fluxes k_flux has just computed; it updates
// them, runs the repair rounds locally, does the bookkeeping, and then already
// resets the per-domain words and reduces S_max of the new state for the next
// step's k_flux.
template <int SYS, bool G75>
__global__ void __launch_bounds__(256) k_post(StepArgs a, const int* __restrict__ grp)
{
  __shared__ int s_any[MAX_REPAIR + 1];
  const int b = blockIdx.x, tid = threadIdx.x, bt = blockDim.x;
  const int d0 = grp[b], d1 = grp[b + 1];
  const long long cb = a.cell_off[d0], ce = a.cell_off[d1];
  const long long ib = a.if_off[d0], ie = a.if_off[d1];
  if (tid <= MAX_REPAIR) s_any[tid] = 0;
  __syncthreads();
  for (long long gi = cb + tid; gi < ce; gi += bt)
    if (update_one<SYS>(a, gi, a.cell_dom[gi], -1) & 1) s_any[0] = 1;
  __syncthreads();
  if (SYS == SYS_EULER) {
    for (int r = 0; r < MAX_REPAIR; ++r) {
      if (s_any[r] == 0) break;                       // uniform: read after a barrier
      for (long long base = ib; base < ie; base += bt) {
        const long long gj = base + tid;
        unsigned st[3] = {0u, 0u, 0u};
        int d = -1;
        if (gj < ie) {
          d = a.if_dom[gj];
          repair_one<G75>(a, r, gj, d, st);
        }
        __syncwarp();
        warp_stat_add(a.stats, d, S_NEWTON_SUM, st[0]);
        warp_stat_max(a.stats, d, S_NEWTON_MAX, st[0]);
        warp_stat_add(a.stats, d, S_RS_CALLS, st[1]);
        warp_stat_add(a.stats, d, S_LOW, st[1]);
      }
      __syncthreads();
      for (long long gi = cb + tid; gi < ce; gi += bt)
        if (update_one<SYS>(a, gi, a.cell_dom[gi], r) & 1) s_any[r + 1] = 1;
      __syncthreads();
    }
  }
  for (int d = d0 + tid; d < d1; d += bt) {
    finish_one(a, d);
    reset_domain_words(a, d);
  }
  __syncthreads();
  StepArgs n = a;                                     // the state just written
  n.avg = a.avg_new;
  if (SYS == SYS_EULER)
    for (long long base = cb; base < ce; base += bt) smax_cell(n, base + tid, base + tid < ce);
  __syncthreads();
  for (int d = d0 + tid; d < d1; d += bt) compute_domain_step(n, d);   // next step's dt
}

// ------------------------------------------------------------------ init
// Initial interface data: classical Riemann state of the one-sided limits.
static __global__ void k_init_iface(int sys, Phys ph, long long nif, const double* lm, const double* lp, double* ifc)
{
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nif) return;
  if (sys == SYS_ADV) {
    const double l = ph.lambda;
    ifc[j] = l > 0.0 ? lm[j] : (l < 0.0 ? lp[j] : 0.5 * (lm[j] + lp[j]));
    return;
  }
  double QL[3] = {lm[j], lm[nif + j], lm[2 * nif + j]}, QR[3] = {lp[j], lp[nif + j], lp[2 * nif + j]}, Q[3];
  int it;
  Phys p2 = ph;
  p2.guess = 0;
  Prim W;
  const int st = ph.gamma == 1.4 ? riemann_state<true>(p2, QL, QR, true, Q, W, it)
                                 : riemann_state<false>(p2, QL, QR, true, Q, W, it);
  if (st != ST_OK && st != ST_VACUUM) { Q[0] = QL[0]; Q[1] = QL[1]; Q[2] = QL[2]; }
  ifc[j] = Q[0]; ifc[nif + j] = Q[1]; ifc[2 * nif + j] = Q[2];
}

// Per-domain norms of component 0 against exact averages: out[d] = {L1, L2^2, Linf}.
static __global__ void k_norms(int n_domains, const long long* cell_off, const double* dx, const double* avg,
                        const double* exact, double* out)
{
  const int d = blockIdx.x;
  if (d >= n_domains) return;
  double s1 = 0.0, s2 = 0.0, mx = 0.0;
  for (long long i = cell_off[d] + threadIdx.x; i < cell_off[d + 1]; i += blockDim.x) {
    const double e = fabs(avg[i] - exact[i]);
    s1 += e; s2 += e * e; mx = fmax(mx, e);
  }
  __shared__ double sh[3][256];
  sh[0][threadIdx.x] = s1; sh[1][threadIdx.x] = s2; sh[2][threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
      sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[3 * d] = sh[0][0] * dx[d];
    out[3 * d + 1] = sh[1][0] * dx[d];
    out[3 * d + 2] = sh[2][0];
  }
}

}  // namespace grp
