// C ABI of the FV+GRPrec library (declared in include/grprec.h): context
// management, argument checks, device state and the launch sequence of a step.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "grp_kernels.cuh"
#include "grp_launch.h"
#include "grp_tile.cuh"
#include "grprec.h"

using namespace grp;

struct grp_ctx {
  grp_problem p;
  int D = 0, C = 1;
  long long ncell = 0, nif = 0;
  cudaStream_t stream = nullptr;
  bool initialized = false;
  int cur = 0;
  long long launches = 0;
  std::vector<long long> h_cell_off, h_if_off;
  std::vector<double> h_dx;
  std::vector<unsigned char> h_bc;
  // device
  long long *cell_off = nullptr, *if_off = nullptr;
  int *cell_dom = nullptr, *if_dom = nullptr;
  double* dx = nullptr;
  unsigned char* bc = nullptr;
  double* avg[2] = {nullptr, nullptr};
  double* ifc[2] = {nullptr, nullptr};
  double* flux = nullptr;
  double* pold = nullptr;        // pressure of the current averages (S_max pass)
  DomStep* ds = nullptr;         // per-domain time step of the current step
  double* det_ed = nullptr;      // DET: evolved edge values of every cell
  double* srcv = nullptr;        // numerical source of every cell (source terms only)
  double* hard_tr = nullptr;     // flux kernel's deferred interfaces: traces, index, counters
  long long* hard_idx = nullptr;
  unsigned* hard_count = nullptr;
  long long hard_cap = 0;
  // admissibility flags of the interface data, one buffer per state buffer;
  // adm_valid: the flags of the current buffer were written by the last step
  unsigned char* gadm[2] = {nullptr, nullptr};
  bool adm_valid = false;
  unsigned char *low = nullptr, *troubled = nullptr;
  double *t = nullptr, *dt_prev = nullptr;
  int *nstep = nullptr, *status = nullptr;
  unsigned long long* smax_bits = nullptr;
  int *bad = nullptr, *inad = nullptr, *fail = nullptr, *any_bad = nullptr;
  int *tlist0 = nullptr, *tlist1 = nullptr, *ilist = nullptr, *lcount = nullptr;   // repair work lists
  unsigned long long* stats = nullptr;
  double* scratch_norm = nullptr;
  float *mlp = nullptr, *mlp_norm = nullptr;     // learned guess: weights, input box (library-owned)
  float* harvest = nullptr;                        // caller-owned harvest buffer and counter
  unsigned long long* harvest_count = nullptr;
  long long harvest_cap = 0;
  int harvest_log2_stride = 0;
  // launch configuration (grp_set_launch)
  int mode = GRP_LAUNCH_AUTO, threads = 256, cells_per_block = 2048, steps_per_launch = 8;
  int max_cells = 0;
  int* grp = nullptr;            // device [n_blocks + 1] first domain of each block
  int n_blocks = 0;
  // tiled form: tiles, the tile view's zero domain map, per-domain flags
  TileInfo* tiles = nullptr;
  int n_tiles = 0, tile_rmax = 0;
  int* tile_zeros = nullptr;
  int* tile_flag = nullptr;
  long long host_steps = 0;      // steps since grp_set_initial (every active domain takes them with t_end = inf)
  bool smax_ready = false;       // S_max of the current state already reduced (split form)
  // optional CUDA-event timing of the flux kernel launches
  bool timing = false;
  std::vector<cudaEvent_t> ev_free, ev_pending;   // pending: start/stop pairs
  // CUDA graphs of graph_steps steps, replayed by grp_step (grp_set_graph)
  struct Graph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    int start_cur = 0;
    bool smax_ready = false;
    bool adm_valid = false, adm_end = false;   // flags valid at the graph's start and end
    unsigned long long t_end_bits = 0;
    int steps = 0;
    int cur_end = 0;                 // buffer parity after the graph
    long long launches = 0;
    std::vector<cudaGraphNode_t> ev_nodes;   // event-record nodes of the flux timing, in pair order
  };
  int graph_steps = 16;
  bool capturing = false;
  std::vector<Graph> graphs;
  cudaStream_t cap_stream = nullptr;
};

namespace {

thread_local char g_err[256];

int cuda_fail(cudaError_t e, const char* what)
{
  snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
  return GRP_E_CUDA;
}

#define CK(call)                                           \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t n)
{
  return cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
}

void drop_graphs(grp_ctx* c)
{
  for (auto& g : c->graphs) {
    if (g.x) cudaGraphExecDestroy(g.x);
    if (g.g) cudaGraphDestroy(g.g);
  }
  c->graphs.clear();
}

void free_all(grp_ctx* c)
{
  drop_graphs(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->cap_stream = nullptr;
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_pending) cudaEventDestroy(e);
  c->ev_free.clear();
  c->ev_pending.clear();
  void* ptrs[] = {c->cell_off, c->if_off, c->cell_dom, c->if_dom, c->dx, c->bc, c->avg[0], c->avg[1],
                  c->ifc[0], c->ifc[1], c->flux, c->pold, c->ds, c->det_ed, c->srcv, c->low, c->troubled, c->t, c->dt_prev, c->nstep,
                  c->status, c->smax_bits, c->bad, c->inad, c->fail, c->any_bad, c->tlist0, c->tlist1,
                  c->ilist, c->lcount, c->stats,
                  c->scratch_norm, c->mlp, c->mlp_norm, c->grp, c->tiles, c->tile_zeros, c->tile_flag,
                  c->hard_tr, c->hard_idx, c->hard_count, c->gadm[0], c->gadm[1]};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

StepArgs make_args(const grp_ctx* c, double t_end)
{
  StepArgs a;
  a.sys = c->p.system;
  a.M = c->p.M;
  a.recon = c->p.recon;
  a.C = c->C;
  a.ph = make_phys(c->p.lambda, c->p.gamma, c->p.newton_rtol, c->p.newton_max_iter, c->p.guess);
  a.cfl = c->p.cfl;
  a.t_end = t_end;
  a.dt_hold = c->p.dt_hold;
  a.n_domains = c->D;
  a.ncell = c->ncell;
  a.nif = c->nif;
  a.cell_off = c->cell_off;
  a.if_off = c->if_off;
  a.cell_dom = c->cell_dom;
  a.if_dom = c->if_dom;
  a.dx = c->dx;
  a.bc = c->bc;
  a.avg = c->avg[c->cur];
  a.avg_new = c->avg[c->cur ^ 1];
  a.ifc = c->ifc[c->cur];
  a.ifc_new = c->ifc[c->cur ^ 1];
  a.flux = c->flux;
  a.pold = c->pold;
  a.ds = c->ds;
  a.low = c->low;
  a.troubled = c->troubled;
  a.t = c->t;
  a.dt_prev = c->dt_prev;
  a.nstep = c->nstep;
  a.status = c->status;
  a.smax_bits = c->smax_bits;
  a.bad = c->bad;
  a.inad = c->inad;
  a.fail = c->fail;
  a.any_bad = c->any_bad;
  a.tlist[0] = c->tlist0;
  a.tlist[1] = c->tlist1;
  a.ilist = c->ilist;
  a.lcount = c->lcount;
  a.stats = c->stats;
  a.ph.mlp_w = c->mlp;
  a.ph.mlp_box = c->mlp_norm;
  // 2: harvest (the records' targets in FP64); 1: the learned start alone
  a.ph.features = c->harvest ? 2 : (c->p.guess == GRP_GUESS_MLP && c->mlp ? 1 : 0);
  a.harvest = c->harvest;
  a.harvest_count = c->harvest_count;
  a.harvest_cap = c->harvest_cap;
  a.harvest_log2_stride = c->harvest_log2_stride;
  a.srcv = c->srcv;
  a.hard_tr = c->hard_tr;
  a.hard_idx = c->hard_idx;
  a.hard_count = c->hard_count;
  a.hard_cap = (int)c->hard_cap;
  a.ph.src = c->p.source;
  a.ph.src_k = c->p.source_coef;
  return a;
}

unsigned blocks(long long n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

// Timing event on the context's stream; under graph capture an event-record
// node of the graph (an ordinary record would only mark a capture dependency).
cudaError_t record(const grp_ctx* c, cudaEvent_t e)
{
  return c->capturing ? cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal)
                      : cudaEventRecord(e, c->stream);
}

cudaError_t launch_flux(const StepArgs& a, cudaStream_t s)
{
  const bool nl = a.recon == GRP_RECON_GRPRECNL;
  if (a.sys == SYS_ADV) return nl ? launch_flux_adv_nl(a, s) : launch_flux_adv(a, s);
  switch (a.M) {
    case 1: return nl ? launch_flux_euler_m1_nl(a, s) : launch_flux_euler_m1(a, s);
    case 2: return nl ? launch_flux_euler_m2_nl(a, s) : launch_flux_euler_m2(a, s);
    case 3: return nl ? launch_flux_euler_m3_nl(a, s) : launch_flux_euler_m3(a, s);
    case 4: return nl ? launch_flux_euler_m4_nl(a, s) : launch_flux_euler_m4(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch(const BatchLaunch& L, cudaStream_t s)
{
  const bool nl = L.a.recon == GRP_RECON_GRPRECNL;
  if (L.a.sys == SYS_ADV) return nl ? launch_batch_adv_nl(L, s) : launch_batch_adv(L, s);
  switch (L.a.M) {
    case 1: return nl ? launch_batch_euler_m1_nl(L, s) : launch_batch_euler_m1(L, s);
    case 2: return nl ? launch_batch_euler_m2_nl(L, s) : launch_batch_euler_m2(L, s);
    case 3: return nl ? launch_batch_euler_m3_nl(L, s) : launch_batch_euler_m3(L, s);
    case 4: return nl ? launch_batch_euler_m4_nl(L, s) : launch_batch_euler_m4(L, s);
    default: return cudaErrorInvalidValue;
  }
}

// the launch form grp_step takes: FLAT, FUSED or SPLIT
int launch_form(const grp_ctx* c)
{
  if (c->p.solver == GRP_SOLVER_DET) return GRP_LAUNCH_FLAT;     // DET has the flat form only
  if (c->p.source != GRP_SOURCE_NONE) return GRP_LAUNCH_FLAT;     // so do source terms
  // the tiled form holds dt over its steps: dt_hold must equal the steps per launch
  if (c->mode == GRP_LAUNCH_TILED) return c->p.dt_hold == c->steps_per_launch ? GRP_LAUNCH_TILED : GRP_LAUNCH_FLAT;
  if (c->mode != GRP_LAUNCH_AUTO) return c->mode;
  // auto: the flat form (on the batched workload it measured fastest of the
  // four: its grid-wide kernels and compacted lists keep warps full)
  return GRP_LAUNCH_FLAT;
}

bool use_batch(const grp_ctx* c) { return launch_form(c) != GRP_LAUNCH_FLAT; }

// Greedy grouping of consecutive domains into blocks of about
// cells_per_block cells (a longer domain gets a block of its own).
int build_groups(grp_ctx* c)
{
  std::vector<int> g(1, 0);
  long long acc = 0;
  for (int d = 0; d < c->D; ++d) {
    const long long n = c->h_cell_off[d + 1] - c->h_cell_off[d];
    if (acc > 0 && acc + n > c->cells_per_block) { g.push_back(d); acc = 0; }
    acc += n;
  }
  g.push_back(c->D);
  if (c->grp) cudaFree(c->grp);
  c->grp = nullptr;
  CK(cudaMalloc((void**)&c->grp, sizeof(int) * g.size()));
  CK(cudaMemcpy(c->grp, g.data(), sizeof(int) * g.size(), cudaMemcpyHostToDevice));
  c->n_blocks = (int)g.size() - 1;
  return GRP_OK;
}

// nsteps steps of the persistent batched kernel in one launch
int enqueue_batch(grp_ctx* c, int nsteps, double t_end)
{
  c->adm_valid = false;               // this form keeps no admissibility flags
  if (!c->grp) { const int rc = build_groups(c); if (rc) return rc; }
  c->smax_ready = false;
  const StepArgs a = make_args(c, t_end);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->timing) {
    for (cudaEvent_t* e : {&e0, &e1}) {
      if (!c->ev_free.empty()) { *e = c->ev_free.back(); c->ev_free.pop_back(); }
      else CK(cudaEventCreate(e));
    }
    CK(record(c, e0));
  }
  const BatchLaunch L{a, c->grp, (unsigned)c->n_blocks, (unsigned)c->threads, nsteps, c->cur,
                      c->avg[0], c->avg[1], c->ifc[0], c->ifc[1]};
  CK(launch_batch(L, c->stream));
  c->launches++;
  if (c->timing) {
    CK(record(c, e1));
    c->ev_pending.push_back(e0);
    c->ev_pending.push_back(e1);
  }
  c->cur ^= (nsteps & 1);
  c->host_steps += nsteps;
  return GRP_OK;
}

// one step in the split form: grid-wide k_flux, then k_post per domain group
int enqueue_split(grp_ctx* c, double t_end)
{
  c->adm_valid = false;               // this form keeps no admissibility flags
  if (!c->grp) { const int rc = build_groups(c); if (rc) return rc; }
  const StepArgs a = make_args(c, t_end);
  cudaStream_t s = c->stream;
  if (!c->smax_ready) {
    k_smax<<<blocks(c->ncell, 256), 256, 0, s>>>(a);
    k_dt<<<blocks(c->D, 128), 128, 0, s>>>(a);
    c->launches += 2;
    c->smax_ready = true;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->timing) {
    for (cudaEvent_t* e : {&e0, &e1}) {
      if (!c->ev_free.empty()) { *e = c->ev_free.back(); c->ev_free.pop_back(); }
      else CK(cudaEventCreate(e));
    }
    CK(record(c, e0));
  }
  CK(launch_flux(a, s));
  c->launches += flux_defers(a) ? 2 : 1;
  if (c->timing) {
    CK(record(c, e1));
    c->ev_pending.push_back(e0);
    c->ev_pending.push_back(e1);
  }
  const BatchLaunch L{a, c->grp, (unsigned)c->n_blocks, (unsigned)c->threads, 1, c->cur,
                      c->avg[0], c->avg[1], c->ifc[0], c->ifc[1]};
  CK(c->p.system == GRP_ADVECTION ? launch_post_adv(L, s) : launch_post_euler(L, s));
  c->launches++;
  c->cur ^= 1;
  c->host_steps += 1;
  return GRP_OK;
}

// Tiles of cells_per_block owned cells with a halo of
// steps_per_launch x (reach + MAX_REPAIR) + 1 cells; a domain that fits in one
// region is one tile holding the whole domain.
int tile_halo(const grp_ctx* c)
{
  const int reach = (c->p.recon == GRP_RECON_GRPRECNL || c->p.M >= 3) ? 2 : 1;
  return c->steps_per_launch * (reach + MAX_REPAIR) + 1;
}

int build_tiles(grp_ctx* c)
{
  const int T = c->cells_per_block, H = tile_halo(c);
  std::vector<TileInfo> v;
  int rmax = 0;
  for (int d = 0; d < c->D; ++d) {
    const int N = (int)(c->h_cell_off[d + 1] - c->h_cell_off[d]);
    if (N <= T + 2 * H) {
      v.push_back(TileInfo{d, 0, N, 0, N, 1});
      rmax = N > rmax ? N : rmax;
      continue;
    }
    for (int o0 = 0; o0 < N; o0 += T) {
      const int o1 = o0 + T < N ? o0 + T : N;
      int r0 = o0 - H, r1 = o1 + H;
      if (c->h_bc[d] != GRP_BC_PERIODIC) { r0 = r0 < 0 ? 0 : r0; r1 = r1 > N ? N : r1; }
      v.push_back(TileInfo{d, o0, o1, r0, r1, 0});
      rmax = r1 - r0 > rmax ? r1 - r0 : rmax;
    }
  }
  if (c->tiles) cudaFree(c->tiles);
  if (c->tile_zeros) cudaFree(c->tile_zeros);
  if (c->tile_flag) cudaFree(c->tile_flag);
  c->tiles = nullptr; c->tile_zeros = nullptr; c->tile_flag = nullptr;
  CK(cudaMalloc((void**)&c->tiles, sizeof(TileInfo) * v.size()));
  CK(cudaMemcpy(c->tiles, v.data(), sizeof(TileInfo) * v.size(), cudaMemcpyHostToDevice));
  CK(cudaMalloc((void**)&c->tile_zeros, sizeof(int) * (rmax + 1)));
  CK(cudaMemset(c->tile_zeros, 0, sizeof(int) * (rmax + 1)));
  CK(cudaMalloc((void**)&c->tile_flag, sizeof(int) * c->D));
  CK(cudaMemset(c->tile_flag, 0, sizeof(int) * c->D));
  c->n_tiles = (int)v.size();
  c->tile_rmax = rmax;
  // the tile kernel's shared-memory limit, raised here, outside any capture
  TileArgs T0{};
  CK(launch_tile(make_args(c, INFINITY), T0, 0u, tile_smem_bytes(c->C, rmax), c->stream));
  return GRP_OK;
}

// steps_per_launch steps of every domain in one tile launch (t_end = inf)
int enqueue_tiled(grp_ctx* c)
{
  c->adm_valid = false;               // this form keeps no admissibility flags
  if (!c->tiles) { const int rc = build_tiles(c); if (rc) return rc; }
  c->smax_ready = false;
  const StepArgs a = make_args(c, INFINITY);
  cudaStream_t s = c->stream;
  if (c->p.system == GRP_EULER_IDEAL) {
    k_smax<<<blocks(c->ncell, 256), 256, 0, s>>>(a);
    c->launches++;
  }
  k_dt<<<blocks(c->D, 128), 128, 0, s>>>(a);
  c->launches++;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->timing) {
    for (cudaEvent_t* e : {&e0, &e1}) {
      if (!c->ev_free.empty()) { *e = c->ev_free.back(); c->ev_free.pop_back(); }
      else CK(cudaEventCreate(e));
    }
    CK(record(c, e0));
  }
  TileArgs T;
  T.tiles = c->tiles;
  T.nsteps = c->steps_per_launch;
  T.rmax = c->tile_rmax;
  T.A = c->avg[c->cur];
  T.An = c->avg[c->cur ^ 1];
  T.I = c->ifc[c->cur];
  T.In = c->ifc[c->cur ^ 1];
  T.zeros = c->tile_zeros;
  T.dflag = c->tile_flag;
  CK(launch_tile(a, T, (unsigned)c->n_tiles, tile_smem_bytes(c->C, c->tile_rmax), s));   // (attribute set by build_tiles)
  c->launches++;
  if (c->timing) {
    CK(record(c, e1));
    c->ev_pending.push_back(e0);
    c->ev_pending.push_back(e1);
  }
  CK(launch_tile_finish(a, c->tile_flag, c->steps_per_launch, s));
  c->launches++;
  c->cur ^= 1;
  c->host_steps += c->steps_per_launch;
  return GRP_OK;
}

int enqueue_step(grp_ctx* c, double t_end)
{
  c->smax_ready = false;
  StepArgs a = make_args(c, t_end);
  // the flat flux kernel at degrees 2 and 4 keeps the interface data's
  // admissibility flags; the first step after new data tests the data
  const bool flags = c->gadm[0] && flux_defers(a);
  if (flags) {
    a.adm_in = c->adm_valid ? c->gadm[c->cur] : nullptr;
    a.adm_out = c->gadm[c->cur ^ 1];
  }
  cudaStream_t s = c->stream;
  const bool euler = c->p.system == GRP_EULER_IDEAL;
  if (euler) {
    k_smax<<<blocks(c->ncell, 256), 256, 0, s>>>(a);
    c->launches++;
  }
  k_dt<<<blocks(c->D, 128), 128, 0, s>>>(a);
  c->launches++;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->timing) {
    for (cudaEvent_t* e : {&e0, &e1}) {
      if (!c->ev_free.empty()) { *e = c->ev_free.back(); c->ev_free.pop_back(); }
      else CK(cudaEventCreate(e));
    }
    CK(record(c, e0));
  }
  if (c->p.solver == GRP_SOLVER_DET) {
    CK(launch_det_step(a, c->det_ed, s));            // predictor (two phases), then the interface Riemann problems
    c->launches += 3;
  } else {
    CK(c->p.source != GRP_SOURCE_NONE ? launch_flux_src(a, s) : launch_flux(a, s));
    c->launches += flux_defers(a) ? 2 : 1;
  }
  if (c->timing) {
    CK(record(c, e1));
    c->ev_pending.push_back(e0);
    c->ev_pending.push_back(e1);
  }
  if (euler) {
    k_update<SYS_EULER><<<blocks(c->ncell, 256), 256, 0, s>>>(a, -1);
    c->launches++;
    // repair rounds over the compacted lists of troubled cells and repaired interfaces
    for (int r = 0; r < MAX_REPAIR; ++r) {
      if (c->p.gamma == 1.4) k_repair_list<true><<<LIST_BLOCKS, LIST_THREADS, 0, s>>>(a, r);
      else k_repair_list<false><<<LIST_BLOCKS, LIST_THREADS, 0, s>>>(a, r);
      k_update_list<SYS_EULER><<<LIST_BLOCKS, LIST_THREADS, 0, s>>>(a, r);
      c->launches += 2;
    }
  } else {
    k_update<SYS_ADV><<<blocks(c->ncell, 256), 256, 0, s>>>(a, -1);
    c->launches++;
  }
  k_finish<<<blocks(c->D, 128), 128, 0, s>>>(a);
  c->launches++;
  CK(cudaGetLastError());
  c->adm_valid = flags;
  c->cur ^= 1;
  c->host_steps += 1;
  return GRP_OK;
}

int step_n(grp_ctx* c, int n_steps, double t_end);

// true when every domain has reached t_end or is frozen (synchronises the stream)
int all_done(grp_ctx* c, double t_end, bool& done)
{
  std::vector<double> ht(c->D);
  std::vector<int> hs(c->D);
  CK(cudaMemcpyAsync(ht.data(), c->t, sizeof(double) * c->D, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(hs.data(), c->status, sizeof(int) * c->D, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  done = true;
  for (int d = 0; d < c->D; ++d)
    if (hs[d] == GRP_ST_OK && ht[d] < t_end) { done = false; break; }
  return GRP_OK;
}

}  // namespace

extern "C" {

const char* grp_status_string(int code)
{
  switch (code) {
    case GRP_OK: return "ok";
    case GRP_E_INVALID_ARG: return "invalid argument";
    case GRP_E_CUDA: return g_err[0] ? g_err : "CUDA error";
    case GRP_E_NOT_INITIALIZED: return "initial data not set";
    case GRP_E_NO_MODEL: return "no learned guess model loaded";
    case GRP_E_MAX_STEPS: return "max_steps reached before t_end";
    case GRP_ST_NEWTON_NO_CONV: return "domain frozen: star-pressure Newton did not converge";
    case GRP_ST_VACUUM: return "vacuum";
    case GRP_ST_NONPHYSICAL: return "domain frozen: inadmissible state after repair";
    default: return "unknown code";
  }
}

int grp_create(grp_ctx** out, const grp_problem* p)
{
  if (!out || !p) return GRP_E_INVALID_ARG;
  *out = nullptr;
  if (p->system != GRP_ADVECTION && p->system != GRP_EULER_IDEAL) return GRP_E_INVALID_ARG;
  if (p->M < 1 || p->M > 4) return GRP_E_INVALID_ARG;
  if (!(p->cfl > 0.0 && p->cfl <= 1.0)) return GRP_E_INVALID_ARG;
  if (p->n_domains < 1 || !p->n_cells || !p->x_left || !p->x_right || !p->bc) return GRP_E_INVALID_ARG;
  if (p->system == GRP_ADVECTION && !(p->lambda != 0.0 && isfinite(p->lambda))) return GRP_E_INVALID_ARG;
  if (p->system == GRP_EULER_IDEAL && !(p->gamma > 1.0 && isfinite(p->gamma))) return GRP_E_INVALID_ARG;
  if (!(p->newton_rtol > 0.0) || p->newton_max_iter < 2) return GRP_E_INVALID_ARG;
  if (p->guess < GRP_GUESS_PVRS || p->guess > GRP_GUESS_MLP) return GRP_E_INVALID_ARG;
  if (p->dt_hold < 1) return GRP_E_INVALID_ARG;
  if (p->recon != GRP_RECON_GRPREC && p->recon != GRP_RECON_GRPRECNL) return GRP_E_INVALID_ARG;
  if (p->solver != GRP_SOLVER_TT && p->solver != GRP_SOLVER_DET) return GRP_E_INVALID_ARG;
  if (p->source != GRP_SOURCE_NONE) {
    // a source term: S = k q for advection, the constant acceleration for the
    // Euler equations; it enters the Toro-Titarev series, with linear GRPrec
    const bool kind_ok = (p->source == GRP_SOURCE_LINEAR && p->system == GRP_ADVECTION) ||
                         (p->source == GRP_SOURCE_GRAVITY && p->system == GRP_EULER_IDEAL);
    if (!kind_ok || !isfinite(p->source_coef) || p->solver != GRP_SOLVER_TT || p->recon != GRP_RECON_GRPREC)
      return GRP_E_INVALID_ARG;
  }
  grp_ctx* c = new grp_ctx();
  c->p = *p;
  c->p.n_cells = nullptr; c->p.x_left = nullptr; c->p.x_right = nullptr; c->p.bc = nullptr;
  c->D = p->n_domains;
  c->C = p->system == GRP_EULER_IDEAL ? 3 : 1;
  c->stream = (cudaStream_t)p->stream;
  c->h_cell_off.assign(c->D + 1, 0);
  c->h_if_off.assign(c->D + 1, 0);
  c->h_dx.assign(c->D, 0.0);
  std::vector<unsigned char> hbc(c->D);
  c->h_bc.assign(c->D, 0);
  for (int d = 0; d < c->D; ++d) {
    const int N = p->n_cells[d];
    if (N < 1 || (p->bc[d] != GRP_BC_PERIODIC && p->bc[d] != GRP_BC_TRANSMISSIVE) ||
        !(p->x_right[d] > p->x_left[d]) || !isfinite(p->x_left[d]) || !isfinite(p->x_right[d])) {
      delete c;
      return GRP_E_INVALID_ARG;
    }
    c->h_cell_off[d + 1] = c->h_cell_off[d] + N;
    c->h_if_off[d + 1] = c->h_if_off[d] + N + (p->bc[d] == GRP_BC_TRANSMISSIVE ? 1 : 0);
    c->h_dx[d] = (p->x_right[d] - p->x_left[d]) / N;
    hbc[d] = (unsigned char)p->bc[d];
    c->h_bc[d] = hbc[d];
    if (N > c->max_cells) c->max_cells = N;
  }
  c->ncell = c->h_cell_off[c->D];
  c->nif = c->h_if_off[c->D];
  if (c->ncell >= (1ll << 31) || c->nif >= (1ll << 31)) { delete c; return GRP_E_INVALID_ARG; }
  std::vector<int> cdom(c->ncell), idom(c->nif);
  for (int d = 0; d < c->D; ++d) {
    for (long long i = c->h_cell_off[d]; i < c->h_cell_off[d + 1]; ++i) cdom[i] = d;
    for (long long j = c->h_if_off[d]; j < c->h_if_off[d + 1]; ++j) idom[j] = d;
  }
  cudaError_t e = cudaSetDevice(p->device);
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaSetDevice"); }
  const int D = c->D, C = c->C;
#define AL(ptr, n)                                                    \
  if ((e = dalloc(&c->ptr, (n))) != cudaSuccess) {                    \
    free_all(c); delete c; return cuda_fail(e, "cudaMalloc " #ptr); \
  }
  AL(cell_off, D + 1) AL(if_off, D + 1) AL(cell_dom, c->ncell) AL(if_dom, c->nif) AL(dx, D) AL(bc, D)
  AL(avg[0], C * c->ncell) AL(avg[1], C * c->ncell) AL(ifc[0], C * c->nif) AL(ifc[1], C * c->nif)
  AL(flux, C * c->nif) AL(pold, c->ncell) AL(ds, D) AL(low, c->nif) AL(troubled, c->ncell) AL(t, D) AL(dt_prev, D) AL(nstep, D)
  AL(status, D) AL(smax_bits, D) AL(bad, (MAX_REPAIR + 1) * D) AL(inad, D) AL(fail, D)
  AL(any_bad, MAX_REPAIR + 1) AL(stats, (long long)NSTATS * D) AL(scratch_norm, 3 * D)
  AL(tlist0, c->ncell) AL(tlist1, c->ncell) AL(ilist, c->nif) AL(lcount, 2 * (MAX_REPAIR + 1))
  if (p->source != GRP_SOURCE_NONE) AL(srcv, (long long)C * c->ncell)
  if (p->system == GRP_EULER_IDEAL && p->recon == GRP_RECON_GRPREC && p->solver != GRP_SOLVER_DET &&
      p->source == GRP_SOURCE_NONE && (p->M == 2 || p->M == 4)) {
    c->hard_cap = hard_list_cap(c->nif);
    AL(hard_tr, (long long)hard_doubles_per_slot(p->M) * c->hard_cap) AL(hard_idx, c->hard_cap) AL(hard_count, 3)
    AL(gadm[0], c->nif) AL(gadm[1], c->nif)
    if ((e = cudaMemset(c->hard_count, 0, 3 * sizeof(unsigned))) != cudaSuccess) {
      free_all(c); delete c; return cuda_fail(e, "cudaMemset hard_count");
    }
  }
  if (p->solver == GRP_SOLVER_DET) {
    AL(det_ed, (long long)det_doubles(p->M, C, c->ncell))
    if (det_prepare(p->device) != 0) { free_all(c); delete c; return cuda_fail(cudaErrorUnknown, "DET tables"); }
  }
#undef AL
  struct Cp { void* dst; const void* src; size_t n; } cps[] = {
      {c->cell_off, c->h_cell_off.data(), sizeof(long long) * (D + 1)},
      {c->if_off, c->h_if_off.data(), sizeof(long long) * (D + 1)},
      {c->cell_dom, cdom.data(), sizeof(int) * c->ncell},
      {c->if_dom, idom.data(), sizeof(int) * c->nif},
      {c->dx, c->h_dx.data(), sizeof(double) * D},
      {c->bc, hbc.data(), (size_t)D}};
  for (auto& cp : cps) {
    if ((e = cudaMemcpy(cp.dst, cp.src, cp.n, cudaMemcpyHostToDevice)) != cudaSuccess) {
      free_all(c); delete c; return cuda_fail(e, "cudaMemcpy metadata");
    }
  }
  *out = c;
  return GRP_OK;
}

void grp_destroy(grp_ctx* c)
{
  if (!c) return;
  cudaSetDevice(c->p.device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_all(c);
  delete c;
}

int grp_set_initial(grp_ctx* c, const double* averages, const double* lim_minus, const double* lim_plus,
                    int ptr_is_device)
{
  if (!c || !averages || !lim_minus) return GRP_E_INVALID_ARG;
  CK(cudaSetDevice(c->p.device));
  const cudaMemcpyKind k = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaStream_t s = c->stream;
  c->adm_valid = false;
  c->cur = 0;
  CK(cudaMemcpyAsync(c->avg[0], averages, sizeof(double) * c->C * c->ncell, k, s));
  if (!lim_plus) {
    CK(cudaMemcpyAsync(c->ifc[0], lim_minus, sizeof(double) * c->C * c->nif, k, s));
  } else {
    // both limits staged in the two halves of the flux scratch and the spare plane set
    double* lm = c->flux;
    double* lp = c->ifc[1];
    CK(cudaMemcpyAsync(lm, lim_minus, sizeof(double) * c->C * c->nif, k, s));
    CK(cudaMemcpyAsync(lp, lim_plus, sizeof(double) * c->C * c->nif, k, s));
    const Phys ph = make_phys(c->p.lambda, c->p.gamma, c->p.newton_rtol, c->p.newton_max_iter, 0);
    k_init_iface<<<blocks(c->nif, 128), 128, 0, s>>>(c->p.system, ph, c->nif, lm, lp, c->ifc[0]);
    c->launches++;
    CK(cudaGetLastError());
  }
  const int D = c->D;
  CK(cudaMemsetAsync(c->t, 0, sizeof(double) * D, s));
  CK(cudaMemsetAsync(c->dt_prev, 0, sizeof(double) * D, s));
  CK(cudaMemsetAsync(c->nstep, 0, sizeof(int) * D, s));
  CK(cudaMemsetAsync(c->status, 0, sizeof(int) * D, s));
  CK(cudaMemsetAsync(c->smax_bits, 0, sizeof(unsigned long long) * D, s));
  CK(cudaMemsetAsync(c->stats, 0, sizeof(unsigned long long) * NSTATS * D, s));
  CK(cudaMemsetAsync(c->low, 0, c->nif, s));
  CK(cudaMemsetAsync(c->troubled, 0, c->ncell, s));
  // per-domain repair and failure words: the flat form clears them every
  // step, the block-local forms at the start of their first step
  CK(cudaMemsetAsync(c->bad, 0, sizeof(int) * (MAX_REPAIR + 1) * D, s));
  CK(cudaMemsetAsync(c->inad, 0, sizeof(int) * D, s));
  CK(cudaMemsetAsync(c->fail, 0, sizeof(int) * D, s));
  c->initialized = true;
  c->host_steps = 0;
  c->smax_ready = false;
  return GRP_OK;
}

int grp_step(grp_ctx* c, int n_steps, double t_end)
{
  if (!c || n_steps < 0 || isnan(t_end)) return GRP_E_INVALID_ARG;
  if (!c->initialized) return GRP_E_NOT_INITIALIZED;
  if (c->p.guess == GRP_GUESS_MLP && !c->mlp) return GRP_E_NO_MODEL;
  CK(cudaSetDevice(c->p.device));
  return step_n(c, n_steps, t_end);
}

int grp_set_launch(grp_ctx* c, int mode, int threads, int cells_per_block, int steps_per_launch)
{
  if (!c || mode < GRP_LAUNCH_AUTO || mode > GRP_LAUNCH_TILED) return GRP_E_INVALID_ARG;
  if (threads != 128 && threads != 256) return GRP_E_INVALID_ARG;
  if (cells_per_block < 64 || cells_per_block > (1 << 20) || steps_per_launch < 1 || steps_per_launch > 1024)
    return GRP_E_INVALID_ARG;
  if (mode == GRP_LAUNCH_TILED) {
    // the largest region of a tile must fit the shared memory of a block
    grp_ctx probe = grp_ctx();
    probe.p = c->p;
    probe.steps_per_launch = steps_per_launch;
    const long long rmax = (long long)cells_per_block + 2ll * tile_halo(&probe);
    if (rmax > (1 << 20) || tile_smem_bytes(c->C, (int)rmax) > 227u * 1024u) return GRP_E_INVALID_ARG;
  }
  CK(cudaSetDevice(c->p.device));
  CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
  drop_graphs(c);
  const bool regroup = cells_per_block != c->cells_per_block;
  c->mode = mode;
  c->threads = threads;
  c->cells_per_block = cells_per_block;
  c->steps_per_launch = steps_per_launch;
  if (regroup && c->grp) { cudaFree(c->grp); c->grp = nullptr; }
  if (c->tiles) { cudaFree(c->tiles); c->tiles = nullptr; }       // rebuilt for the new tile and depth
  return GRP_OK;
}

int grp_get_launch(const grp_ctx* c, int* batched, int* threads, int* cells_per_block, int* steps_per_launch,
                   int* blocks)
{
  if (!c) return GRP_E_INVALID_ARG;
  if (batched) *batched = launch_form(c);
  if (threads) *threads = c->threads;
  if (cells_per_block) *cells_per_block = c->cells_per_block;
  if (steps_per_launch) *steps_per_launch = c->steps_per_launch;
  if (blocks) {
    long long nb = 0, acc = 0;
    for (int d = 0; d < c->D; ++d) {
      const long long n = c->h_cell_off[d + 1] - c->h_cell_off[d];
      if (acc > 0 && acc + n > c->cells_per_block) { ++nb; acc = 0; }
      acc += n;
    }
    *blocks = (int)(nb + 1);
  }
  return GRP_OK;
}

}  // extern "C"

namespace {
// steps one launch unit of the current form advances
// the tiled form serves steps without an end time, in whole units that start
// where dt is recomputed (every steps_per_launch steps)
bool tiled_now(const grp_ctx* c, double t_end)
{
  return launch_form(c) == GRP_LAUNCH_TILED && isinf(t_end) && t_end > 0 &&
         c->host_steps % c->steps_per_launch == 0;
}

int unit_steps(const grp_ctx* c, double t_end)
{
  const int form = launch_form(c);
  if (form == GRP_LAUNCH_FUSED) return c->steps_per_launch;
  if (form == GRP_LAUNCH_TILED && tiled_now(c, t_end)) return c->steps_per_launch;
  return 1;
}

int enqueue_unit(grp_ctx* c, int k, double t_end)
{
  const int form = launch_form(c);
  if (form == GRP_LAUNCH_FUSED) return enqueue_batch(c, k, t_end);
  if (form == GRP_LAUNCH_SPLIT) return enqueue_split(c, t_end);
  if (form == GRP_LAUNCH_TILED && k == c->steps_per_launch && tiled_now(c, t_end)) return enqueue_tiled(c);
  for (int i = 0; i < k; ++i) {
    const int rc = enqueue_step(c, t_end);
    if (rc) return rc;
  }
  return GRP_OK;
}

unsigned long long bits_of(double x)
{
  unsigned long long b;
  memcpy(&b, &x, sizeof b);
  return b;
}

// Captures `steps` steps (whole launch units) starting from the context's
// current buffer parity into a CUDA graph.  The kernels' arguments (buffer
// pointers, t_end) are fixed in the graph, so a graph serves one start parity,
// one split-form S_max state and one t_end.
int capture_graph(grp_ctx* c, int steps, double t_end, grp_ctx::Graph& out)
{
  if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  // the domain groups are built (allocation, copy) before capture begins
  if ((launch_form(c) == GRP_LAUNCH_FUSED || launch_form(c) == GRP_LAUNCH_SPLIT) && !c->grp) {
    const int rc = build_groups(c);
    if (rc) return rc;
  }
  if (launch_form(c) == GRP_LAUNCH_TILED && !c->tiles) {
    const int rc = build_tiles(c);
    if (rc) return rc;
  }
  // timing events are created before capture begins
  if (c->timing)
    while (c->ev_free.size() < (size_t)(2 * steps)) {
      cudaEvent_t e = nullptr;
      CK(cudaEventCreate(&e));
      c->ev_free.push_back(e);
    }
  out = grp_ctx::Graph();
  out.start_cur = c->cur;
  out.smax_ready = c->smax_ready;
  out.adm_valid = c->adm_valid;
  out.t_end_bits = bits_of(t_end);
  out.steps = steps;
  const int cur0 = c->cur;
  const long long launches0 = c->launches;
  const size_t ev0 = c->ev_pending.size();
  const bool smax0 = c->smax_ready;
  const bool adm0 = c->adm_valid;
  cudaStream_t user = c->stream;
  CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  c->stream = c->cap_stream;
  c->capturing = true;
  int rc = GRP_OK;
  const long long hs0 = c->host_steps;
  const int k = unit_steps(c, t_end);
  for (int i = 0; i < steps && rc == GRP_OK; i += k) rc = enqueue_unit(c, k, t_end);
  cudaGraph_t g = nullptr;
  const cudaError_t e_end = cudaStreamEndCapture(c->cap_stream, &g);
  c->stream = user;
  c->capturing = false;
  out.launches = c->launches - launches0;
  out.adm_end = c->adm_valid;
  c->adm_valid = adm0;
  out.cur_end = c->cur;
  c->host_steps = hs0;
  // the timing events recorded during capture become nodes of the graph
  std::vector<cudaEvent_t> evs(c->ev_pending.begin() + ev0, c->ev_pending.end());
  c->ev_pending.resize(ev0);
  for (cudaEvent_t e : evs) c->ev_free.push_back(e);
  c->cur = cur0;
  c->launches = launches0;
  c->smax_ready = smax0;
  if (rc != GRP_OK) { if (g) cudaGraphDestroy(g); return rc; }
  if (e_end != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e_end, "cudaStreamEndCapture"); }
  out.g = g;
  if (!evs.empty()) {
    size_t nn = 0;
    CK(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    CK(cudaGraphGetNodes(g, nodes.data(), &nn));
    out.ev_nodes.assign(evs.size(), nullptr);
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType ty;
      CK(cudaGraphNodeGetType(nd, &ty));
      if (ty != cudaGraphNodeTypeEventRecord) continue;
      cudaEvent_t ev = nullptr;
      CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
      for (size_t j = 0; j < evs.size(); ++j)
        if (evs[j] == ev && !out.ev_nodes[j]) { out.ev_nodes[j] = nd; break; }
    }
    for (cudaGraphNode_t nd : out.ev_nodes)
      if (!nd) { cudaGraphDestroy(g); out.g = nullptr; snprintf(g_err, sizeof(g_err), "graph event nodes"); return GRP_E_CUDA; }
  }
  const cudaError_t e_inst = cudaGraphInstantiate(&out.x, g, 0);
  if (e_inst != cudaSuccess) { cudaGraphDestroy(g); out.g = nullptr; return cuda_fail(e_inst, "cudaGraphInstantiate"); }
  return GRP_OK;
}

// Replays (capturing first if needed) the graph of c->graph_steps steps.
int replay_graph(grp_ctx* c, double t_end)
{
  const unsigned long long tb = bits_of(t_end);
  grp_ctx::Graph* G = nullptr;
  for (auto& g : c->graphs)
    if (g.start_cur == c->cur && g.smax_ready == c->smax_ready && g.adm_valid == c->adm_valid &&
        g.t_end_bits == tb && g.steps == c->graph_steps)
      G = &g;
  if (!G) {
    if (c->graphs.size() >= 8) drop_graphs(c);      // t_end changed repeatedly: start over
    grp_ctx::Graph g;
    const int rc = capture_graph(c, c->graph_steps, t_end, g);
    if (rc) return rc;
    c->graphs.push_back(g);
    G = &c->graphs.back();
  }
  if (c->timing) {
    for (size_t j = 0; j < G->ev_nodes.size(); ++j) {
      cudaEvent_t e = nullptr;
      if (!c->ev_free.empty()) { e = c->ev_free.back(); c->ev_free.pop_back(); }
      else CK(cudaEventCreate(&e));
      CK(cudaGraphExecEventRecordNodeSetEvent(G->x, G->ev_nodes[j], e));
      c->ev_pending.push_back(e);
    }
  }
  CK(cudaGraphLaunch(G->x, c->stream));
  c->launches += G->launches;
  c->cur = G->cur_end;
  c->adm_valid = G->adm_end;
  c->host_steps += G->steps;
  if (launch_form(c) == GRP_LAUNCH_SPLIT) c->smax_ready = true;
  else c->smax_ready = false;
  return GRP_OK;
}

int step_n(grp_ctx* c, int n_steps, double t_end)
{
  // With a finite t_end, long requests test completion every DONE_CHECK steps
  // so that the steps left after every domain has arrived are not enqueued.
  const int DONE_CHECK = 64;
  int since_check = 0;
  for (int i = 0; i < n_steps;) {
    if (isfinite(t_end) && i > 0 && since_check >= DONE_CHECK) {
      bool done = false;
      const int rc = all_done(c, t_end, done);
      if (rc) return rc;
      if (done) break;
      since_check = 0;
    }
    int k = unit_steps(c, t_end);
    if (c->graph_steps > 0 && n_steps - i >= c->graph_steps && c->graph_steps % k == 0 &&
        (launch_form(c) != GRP_LAUNCH_TILED || tiled_now(c, t_end) || !isinf(t_end))) {
      const int rc = replay_graph(c, t_end);
      if (rc) return rc;
      k = c->graph_steps;
    } else {
      if (k > n_steps - i) k = n_steps - i;
      const int rc = enqueue_unit(c, k, t_end);
      if (rc) return rc;
    }
    i += k;
    since_check += k;
  }
  return GRP_OK;
}
}  // namespace

extern "C" {

int grp_advance_to(grp_ctx* c, double t_end, int max_steps)
{
  if (!c || !isfinite(t_end) || max_steps < 0) return GRP_E_INVALID_ARG;
  if (!c->initialized) return GRP_E_NOT_INITIALIZED;
  CK(cudaSetDevice(c->p.device));
  int done_steps = 0;
  const int block = 32;
  while (true) {
    bool all = false;
    const int rc0 = all_done(c, t_end, all);
    if (rc0) return rc0;
    if (all) return GRP_OK;
    if (done_steps >= max_steps) return GRP_E_MAX_STEPS;
    const int n = max_steps - done_steps < block ? max_steps - done_steps : block;
    const int rc = step_n(c, n, t_end);
    if (rc) return rc;
    done_steps += n;
  }
}

int grp_get_state(grp_ctx* c, double* averages, double* iface, double* t, int ptr_is_device)
{
  if (!c) return GRP_E_INVALID_ARG;
  if (!c->initialized) return GRP_E_NOT_INITIALIZED;
  CK(cudaSetDevice(c->p.device));
  const cudaMemcpyKind k = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (averages) CK(cudaMemcpyAsync(averages, c->avg[c->cur], sizeof(double) * c->C * c->ncell, k, c->stream));
  if (iface) CK(cudaMemcpyAsync(iface, c->ifc[c->cur], sizeof(double) * c->C * c->nif, k, c->stream));
  if (t) CK(cudaMemcpyAsync(t, c->t, sizeof(double) * c->D, k, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return GRP_OK;
}

int grp_get_stats(grp_ctx* c, unsigned long long* stats, int* status)
{
  if (!c) return GRP_E_INVALID_ARG;
  CK(cudaSetDevice(c->p.device));
  if (stats)
    CK(cudaMemcpyAsync(stats, c->stats, sizeof(unsigned long long) * NSTATS * c->D, cudaMemcpyDeviceToHost,
                       c->stream));
  if (status) CK(cudaMemcpyAsync(status, c->status, sizeof(int) * c->D, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return GRP_OK;
}

int grp_error_norms(grp_ctx* c, const double* exact, int ptr_is_device, double* l1, double* l2, double* linf)
{
  if (!c || !exact) return GRP_E_INVALID_ARG;
  if (!c->initialized) return GRP_E_NOT_INITIALIZED;
  CK(cudaSetDevice(c->p.device));
  const double* dex = exact;
  if (!ptr_is_device) {
    // staged in the flux scratch (C * nif >= ncell doubles), free between steps
    CK(cudaMemcpyAsync(c->flux, exact, sizeof(double) * c->ncell, cudaMemcpyHostToDevice, c->stream));
    dex = c->flux;
  }
  k_norms<<<c->D, 256, 0, c->stream>>>(c->D, c->cell_off, c->dx, c->avg[c->cur], dex, c->scratch_norm);
  c->launches++;
  CK(cudaGetLastError());
  std::vector<double> h(3 * c->D);
  CK(cudaMemcpyAsync(h.data(), c->scratch_norm, sizeof(double) * 3 * c->D, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int d = 0; d < c->D; ++d) {
    if (l1) l1[d] = h[3 * d];
    if (l2) l2[d] = sqrt(h[3 * d + 1]);
    if (linf) linf[d] = h[3 * d + 2];
  }
  return GRP_OK;
}

long long grp_launch_count(const grp_ctx* c) { return c ? c->launches : 0; }

int grp_set_guess_model(grp_ctx* c, const float* weights, int n_weights, const float* box, int ptr_is_device)
{
  if (!c || !weights || !box || n_weights != MLP_NPARAM) return GRP_E_INVALID_ARG;
  CK(cudaSetDevice(c->p.device));
  CK(cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  if (!c->mlp) CK(cudaMalloc((void**)&c->mlp, sizeof(float) * MLP_NPARAM));
  if (!c->mlp_norm) CK(cudaMalloc((void**)&c->mlp_norm, sizeof(float) * 12));
  const cudaMemcpyKind k = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(c->mlp, weights, sizeof(float) * MLP_NPARAM, k, c->stream));
  CK(cudaMemcpyAsync(c->mlp_norm, box, sizeof(float) * 12, k, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return GRP_OK;
}

int grp_set_harvest(grp_ctx* c, float* records, unsigned long long* count, long long capacity, int log2_stride)
{
  if (!c || log2_stride < 0 || log2_stride > 30) return GRP_E_INVALID_ARG;
  if (records && (!count || capacity < 1)) return GRP_E_INVALID_ARG;
  CK(cudaSetDevice(c->p.device));
  CK(cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  c->harvest = records;
  c->harvest_count = records ? count : nullptr;
  c->harvest_cap = records ? capacity : 0;
  c->harvest_log2_stride = log2_stride;
  return GRP_OK;
}

int grp_set_kernel_timing(grp_ctx* c, int enable)
{
  if (!c) return GRP_E_INVALID_ARG;
  if (c->timing != (enable != 0)) {
    CK(cudaSetDevice(c->p.device));
    CK(cudaStreamSynchronize(c->stream));
    drop_graphs(c);
  }
  c->timing = enable != 0;
  return GRP_OK;
}

int grp_set_graph(grp_ctx* c, int steps_per_graph)
{
  if (!c || steps_per_graph < 0 || steps_per_graph > 1024) return GRP_E_INVALID_ARG;
  CK(cudaSetDevice(c->p.device));
  CK(cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  c->graph_steps = steps_per_graph;
  return GRP_OK;
}

int grp_get_kernel_timing(grp_ctx* c, double* flux_ms, long long* flux_launches)
{
  if (!c) return GRP_E_INVALID_ARG;
  CK(cudaSetDevice(c->p.device));
  double total = 0.0;
  long long n = 0;
  for (size_t k = 0; k + 1 < c->ev_pending.size(); k += 2) {
    CK(cudaEventSynchronize(c->ev_pending[k + 1]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev_pending[k], c->ev_pending[k + 1]));
    total += ms;
    ++n;
  }
  for (cudaEvent_t e : c->ev_pending) c->ev_free.push_back(e);
  c->ev_pending.clear();
  if (flux_ms) *flux_ms = total;
  if (flux_launches) *flux_launches = n;
  return GRP_OK;
}

}  // extern "C"
