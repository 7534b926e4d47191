// Temporal blocking of long domains: each block holds a tile of cells in
// shared memory, with a halo on both sides, and advances it several steps
// per launch.  The time step of a domain is held over those steps (dt
// recomputed every dt_hold steps, dt_hold = steps per launch), so the tiles
// of a domain need no exchange inside a launch: the halo is wide enough that
// what its outer cells get wrong (the tile's edge acts as a transmissive end)
// cannot reach the owned cells in that many steps.  Per step a cell's new
// average depends on cells one away (degrees 1-2, linear GRPrec) or two away
// (degrees 3-4, GRPrecNL), and each of the MAX_REPAIR repair rounds can reach
// one cell further, so the halo is steps x (reach + MAX_REPAIR) + 1 cells.
// Every step runs the device functions of the flat form on the tile
// (reconstruction, GRP, update, repair rounds); statistics count the owned
// interfaces only, and each tile writes its owned cells and interfaces.
#pragma once
#include "grp_kernels.cuh"

namespace grp {

struct TileInfo {
  int d;          // domain
  int o0, o1;     // owned cells [o0, o1), domain-local
  int r0, r1;     // region [r0, r1): o0 - H .. o1 + H, clipped at transmissive ends, modulo N when periodic
  int whole;      // the region is the whole domain (its own boundary rule applies at both ends)
};

struct TileArgs {
  const TileInfo* tiles;
  int nsteps;
  int rmax;                   // cells of the largest region
  const double* A;            // averages at the start of the launch [C][ncell]
  double* An;                 // averages after nsteps (the other buffer)
  const double* I;            // interface data at the start [C][nif]
  double* In;                 // interface data after nsteps
  const int* zeros;           // [rmax + 1] zeros: the tile view's cell and interface domain maps
  int* dflag;                 // [D] bit 0: an owned cell inadmissible after a step; failure code << 4
};

constexpr int TILE_THREADS = 128;

// The small per-tile words the flat form's device functions address per domain.
struct TileWords {
  long long cell_off[2], if_off[2];
  double dx;
  DomStep ds;
  unsigned long long stats[NSTATS];
  int bad[MAX_REPAIR + 1], inad, fail, any_bad[MAX_REPAIR + 1];
  int s_any[MAX_REPAIR + 1];
  int flag;
  unsigned char bc;
};

__host__ __device__ inline size_t tile_align(size_t x) { return (x + 15) & ~size_t(15); }

// shared-memory bytes of a tile of rmax cells, C components
__host__ __device__ inline size_t tile_smem_bytes(int C, int rmax)
{
  size_t b = tile_align(sizeof(TileWords));
  b += tile_align(sizeof(double) * 2 * C * rmax);          // averages, two buffers
  b += tile_align(sizeof(double) * 2 * C * (rmax + 1));    // interface data, two buffers
  b += tile_align(sizeof(double) * C * (rmax + 1));        // fluxes
  b += tile_align(sizeof(double) * rmax);                  // old pressures
  b += tile_align(rmax + 1) + tile_align(rmax);            // low, troubled
  return b;
}

template <int SYS, int M, bool G75, bool NL>
__global__ void __launch_bounds__(TILE_THREADS, 3) k_tile(StepArgs a, TileArgs T)
{
  extern __shared__ __align__(16) unsigned char tsm[];
  constexpr int C = SYS == SYS_EULER ? 3 : 1;
  const int tid = threadIdx.x, bt = blockDim.x;
  const TileInfo ti = T.tiles[blockIdx.x];
  const int d = ti.d;
  const long long c0 = a.cell_off[d], i0 = a.if_off[d];
  const int N = (int)(a.cell_off[d + 1] - c0);
  const bool per = a.bc[d] == 0;
  const bool last_if = !per && ti.o1 == N;         // the domain's last interface (transmissive) is owned here
  const int R = ti.r1 - ti.r0;
  const int vbc = ti.whole ? a.bc[d] : 1;
  const int vnif = R + (vbc == 1 ? 1 : 0);
  const int oc0 = ti.o0 - ti.r0, oc1 = ti.o1 - ti.r0;
  const int oif1 = oc1 + (last_if ? 1 : 0);
  auto cell_of = [&](int v) -> long long { long long g = (long long)ti.r0 + v; if (per) g = ((g % N) + N) % N; return g; };
  auto iface_of = [&](int v) -> long long { long long g = (long long)ti.r0 + v; if (per) g = ((g % N) + N) % N; return g; };

  const DomStep step = a.ds[d];
  if (!step.active) {
    // a frozen or finished domain keeps its state
    for (int v = oc0 + tid; v < oc1; v += bt)
      for (int c = 0; c < C; ++c) T.An[c * a.ncell + c0 + cell_of(v)] = T.A[c * a.ncell + c0 + cell_of(v)];
    for (int v = oc0 + tid; v < oif1; v += bt)
      for (int c = 0; c < C; ++c) T.In[c * a.nif + i0 + iface_of(v)] = T.I[c * a.nif + i0 + iface_of(v)];
    return;
  }

  // shared layout
  const int rm = T.rmax;
  unsigned char* p = tsm;
  TileWords* W = (TileWords*)p;                    p += tile_align(sizeof(TileWords));
  double* avs = (double*)p;                        p += tile_align(sizeof(double) * 2 * C * rm);
  double* ifs = (double*)p;                        p += tile_align(sizeof(double) * 2 * C * (rm + 1));
  double* fls = (double*)p;                        p += tile_align(sizeof(double) * C * (rm + 1));
  double* pos = (double*)p;                        p += tile_align(sizeof(double) * rm);
  unsigned char* lows = p;                         p += tile_align(rm + 1);
  unsigned char* trs = p;

  if (tid == 0) {
    W->cell_off[0] = 0; W->cell_off[1] = R;
    W->if_off[0] = 0; W->if_off[1] = vnif;
    W->dx = a.dx[d];
    W->ds = step;
    for (int k = 0; k < NSTATS; ++k) W->stats[k] = 0ull;
    W->flag = 0;
    W->bc = (unsigned char)vbc;
  }
  for (int v = tid; v < R; v += bt)
    for (int c = 0; c < C; ++c) avs[c * rm + v] = T.A[c * a.ncell + c0 + cell_of(v)];
  for (int v = tid; v < vnif; v += bt)
    for (int c = 0; c < C; ++c) ifs[c * (rm + 1) + v] = T.I[c * a.nif + i0 + iface_of(v)];

  // the tile as a one-domain StepArgs of the flat form's device functions
  StepArgs w = a;
  w.n_domains = 1;
  w.ncell = rm;
  w.nif = rm + 1;
  w.cell_off = W->cell_off;
  w.if_off = W->if_off;
  w.cell_dom = T.zeros;
  w.if_dom = T.zeros;
  w.dx = &W->dx;
  w.bc = &W->bc;
  w.ds = &W->ds;
  w.flux = fls;
  w.pold = pos;
  w.low = lows;
  w.troubled = trs;
  w.t = nullptr; w.dt_prev = nullptr; w.nstep = nullptr; w.status = nullptr; w.smax_bits = nullptr;
  w.bad = W->bad; w.inad = &W->inad; w.fail = &W->fail; w.any_bad = W->any_bad;
  w.tlist[0] = w.tlist[1] = nullptr; w.ilist = nullptr; w.lcount = nullptr;
  w.stats = W->stats;
  w.harvest = nullptr; w.harvest_count = nullptr; w.harvest_cap = 0;
  w.srcv = nullptr;

  for (int s = 0; s < T.nsteps; ++s) {
    const int par = s & 1;
    w.avg = avs + par * C * rm;
    w.avg_new = avs + (par ^ 1) * C * rm;
    w.ifc = ifs + par * C * (rm + 1);
    w.ifc_new = ifs + (par ^ 1) * C * (rm + 1);
    if (tid <= MAX_REPAIR) { W->bad[tid] = 0; W->any_bad[tid] = 0; W->s_any[tid] = 0; }
    if (tid == 0) { W->inad = 0; W->fail = 0; }
    __syncthreads();
    if (SYS == SYS_EULER) {
      // pressures of the old averages for the discrete maximum principle (as
      // the S_max pass of the flat form computes them)
      const double g = a.ph.gamma;
      for (int v = tid; v < R; v += bt) {
        const double r = w.avg[v], m = w.avg[rm + v], E = w.avg[2 * rm + v];
        const double u = m * rcp64(r);
        pos[v] = (g - 1.0) * (E - 0.5 * m * u);
      }
    }
    // fluxes of every interface of the region, the flux kernel's warp form
    for (long long base = 31ll * (tid >> 5); base < vnif; base += 31ll * (bt >> 5))
      flux_warp<SYS, M, G75, NL, false>(w, base, vnif, oc0, oif1);
    __syncthreads();
    for (int v = tid; v < R; v += bt)
      if (update_one<SYS>(w, v, 0, -1) & 1) W->s_any[0] = 1;
    __syncthreads();
    if (SYS == SYS_EULER) {
      for (int r = 0; r < MAX_REPAIR; ++r) {
        if (W->s_any[r] == 0) break;                   // uniform: read after a barrier
        for (int base = 0; base < vnif; base += bt) {
          const int v = base + tid;
          unsigned st[3] = {0u, 0u, 0u};
          if (v < vnif) repair_one<G75>(w, r, v, 0, st);
          __syncwarp();
          const int dd = v < vnif && v >= oc0 && v < oif1 ? 0 : -1;
          warp_stat_add(w.stats, dd, S_NEWTON_SUM, st[0]);
          warp_stat_max(w.stats, dd, S_NEWTON_MAX, st[0]);
          warp_stat_add(w.stats, dd, S_RS_CALLS, st[1]);
          warp_stat_add(w.stats, dd, S_LOW, st[1]);
        }
        __syncthreads();
        for (int v = tid; v < R; v += bt)
          if (update_one<SYS>(w, v, 0, r) & 1) W->s_any[r + 1] = 1;
        __syncthreads();
      }
      // the first failure of the tile, as the flat form would have frozen the
      // domain on it: a failed Riemann problem, else an owned cell still
      // inadmissible after the repair
      if (tid == 0 && W->fail) atomicCAS(&W->flag, 0, W->fail << 4);
      __syncthreads();
      for (int v = oc0 + tid; v < oc1; v += bt)
        if (trs[v] == 2) atomicCAS(&W->flag, 0, 1);
    }
    __syncthreads();
  }
  // the owned cells and interfaces of the final buffer
  const int par = T.nsteps & 1;
  const double* fa = avs + par * C * rm;
  const double* fi = ifs + par * C * (rm + 1);
  for (int v = oc0 + tid; v < oc1; v += bt)
    for (int c = 0; c < C; ++c) T.An[c * a.ncell + c0 + cell_of(v)] = fa[c * rm + v];
  for (int v = oc0 + tid; v < oif1; v += bt)
    for (int c = 0; c < C; ++c) T.In[c * a.nif + i0 + iface_of(v)] = fi[c * (rm + 1) + v];
  if (tid < NSTATS && tid != S_STEPS && W->stats[tid]) {
    unsigned long long* S = a.stats + (long long)d * NSTATS;
    if (tid == S_NEWTON_MAX) atomicMax(S + tid, W->stats[tid]);
    else atomicAdd(S + tid, W->stats[tid]);
  }
  if (tid == 0 && W->flag) atomicCAS(T.dflag + d, 0, W->flag);   // a domain's tiles: the first to report
}

// Bookkeeping of nsteps tiled steps per domain: time (added step by step, as
// the flat form does), step counts, the held dt, status.  A domain whose
// owned cell stayed inadmissible, or whose Riemann problem failed, inside the
// launch is frozen at the end of the launch, with the first failure a tile
// reported (the flat form freezes it at the failing step).
static __global__ void k_tile_finish(StepArgs a, int* dflag, int nsteps)
{
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= a.n_domains) return;
  const DomStep r = a.ds[d];
  a.smax_bits[d] = 0ull;
  const int f = dflag[d];
  dflag[d] = 0;
  if (!r.active) return;
  double t = a.t[d];
  for (int s = 0; s < nsteps; ++s) t = t + r.dt;
  a.t[d] = t;
  a.nstep[d] += nsteps;
  a.dt_prev[d] = r.dt_cfl;
  a.stats[(long long)d * NSTATS + S_STEPS] += nsteps;
  if (f >> 4) a.status[d] = f >> 4;
  else if (f & 1) a.status[d] = ST_NONPHYS;
}

}  // namespace grp
