// grp_step_noalloc: one time step of one domain without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator hooks, plug-ins loaded into a process
// whose device memory is owned by a host application, or real-time loops that
// must not allocate after start-up.  This entry point lets them advance one
// domain with buffers they already own.  The kernels are the same as those of
// grp_step (flat form); the scratch they need -- the interface-flux array, the
// repair flags, the per-domain words and the index tables -- lives in one
// file-scope __device__ array, sized for GRP_NOALLOC_MAX_CELLS cells, that every
// GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "grp_kernels.cuh"
#include "grp_launch.h"
#include "grprec.h"

using namespace grp;

namespace {

constexpr long long NA_CELLS = GRP_NOALLOC_MAX_CELLS;
constexpr long long NA_IFACES = NA_CELLS + 1;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// byte offsets of each scratch array
constexpr size_t OFF_FLUX = 0;
constexpr size_t OFF_LOW = align256(OFF_FLUX + sizeof(double) * 3 * NA_IFACES);
constexpr size_t OFF_TROUBLED = align256(OFF_LOW + NA_IFACES);
constexpr size_t OFF_CELL_DOM = align256(OFF_TROUBLED + NA_CELLS);
constexpr size_t OFF_IF_DOM = align256(OFF_CELL_DOM + sizeof(int) * NA_CELLS);
constexpr size_t OFF_TLIST0 = align256(OFF_IF_DOM + sizeof(int) * NA_IFACES);
constexpr size_t OFF_TLIST1 = align256(OFF_TLIST0 + sizeof(int) * NA_CELLS);
constexpr size_t OFF_ILIST = align256(OFF_TLIST1 + sizeof(int) * NA_CELLS);
constexpr size_t OFF_POLD = align256(OFF_ILIST + sizeof(int) * NA_IFACES);
constexpr size_t OFF_DS = align256(OFF_POLD + sizeof(double) * NA_CELLS);
constexpr size_t OFF_WORDS = align256(OFF_DS + sizeof(DomStep));

// per-domain words of the single domain, in one struct
struct Words {
  long long cell_off[2], if_off[2];
  double dx, t, dt_prev;
  unsigned long long smax_bits;
  unsigned long long stats[NSTATS];
  int nstep, status, fail;
  int bad[MAX_REPAIR + 1], inad, any_bad[MAX_REPAIR + 1];
  int lcount[2 * (MAX_REPAIR + 1)];
  unsigned char bc;
};
constexpr size_t SCRATCH_BYTES = align256(OFF_WORDS + sizeof(Words));
// the public header states the size as about 3.5 MB
static_assert(SCRATCH_BYTES > 3400000 && SCRATCH_BYTES < 3600000, "update the scratch size in grprec.h");

// The scratch.  Every call shares it and it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
// Device address of g_scratch per device, looked up once per device with that
// device current.  The lock makes concurrent first calls from several host
// threads safe.  A reset of a device's primary context (cudaDeviceReset)
// invalidates the address kept for it (the header says so).
std::mutex g_scratch_lock;
unsigned char* g_scratch_addr[MAX_DEVICES];

// Zeroes what must start at zero and writes the index tables and words.
__global__ void k_noalloc_setup(unsigned char* base, int N, int nif, double dx, int bc, double t)
{
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int* cell_dom = (int*)(base + OFF_CELL_DOM);
  int* if_dom = (int*)(base + OFF_IF_DOM);
  if (i < N) { cell_dom[i] = 0; base[OFF_TROUBLED + i] = 0; }
  if (i < nif) { if_dom[i] = 0; base[OFF_LOW + i] = 0; }
  if (i == 0) {
    Words* w = (Words*)(base + OFF_WORDS);
    w->cell_off[0] = 0; w->cell_off[1] = N;
    w->if_off[0] = 0; w->if_off[1] = nif;
    w->dx = dx; w->t = t; w->dt_prev = 0.0;
    w->smax_bits = 0ull;
    for (int k = 0; k < NSTATS; ++k) w->stats[k] = 0ull;
    w->nstep = 0; w->status = 0; w->fail = 0;
    for (int p = 0; p <= MAX_REPAIR; ++p) { w->bad[p] = 0; w->any_bad[p] = 0; }
    for (int p = 0; p < 2 * (MAX_REPAIR + 1); ++p) w->lcount[p] = 0;
    w->inad = 0;
    w->bc = (unsigned char)bc;
  }
}

cudaError_t flux_dispatch(const StepArgs& a, cudaStream_t s)
{
  if (a.sys == SYS_ADV) return launch_flux_adv(a, s);
  switch (a.M) {
    case 1: return launch_flux_euler_m1(a, s);
    case 2: return launch_flux_euler_m2(a, s);
    case 3: return launch_flux_euler_m3(a, s);
    case 4: return launch_flux_euler_m4(a, s);
    default: return cudaErrorInvalidValue;
  }
}

unsigned nblk(long long n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

}  // namespace

extern "C" int grp_step_noalloc(int system, double lambda, double gamma, int M, double cfl, int n_cells,
                                double x_left, double x_right, int bc, const double* avg_in,
                                const double* iface_in, double* avg_out, double* iface_out, double t,
                                double t_end, double* t_out, int* status_out, void* stream)
{
  if (system != GRP_ADVECTION && system != GRP_EULER_IDEAL) return GRP_E_INVALID_ARG;
  if (M < 1 || M > 4 || !(cfl > 0.0 && cfl <= 1.0)) return GRP_E_INVALID_ARG;
  if (n_cells < 1 || n_cells > GRP_NOALLOC_MAX_CELLS) return GRP_E_INVALID_ARG;
  if (!(x_right > x_left) || (bc != GRP_BC_PERIODIC && bc != GRP_BC_TRANSMISSIVE)) return GRP_E_INVALID_ARG;
  if (system == GRP_ADVECTION && !(lambda != 0.0 && isfinite(lambda))) return GRP_E_INVALID_ARG;
  if (system == GRP_EULER_IDEAL && !(gamma > 1.0 && isfinite(gamma))) return GRP_E_INVALID_ARG;
  if (!avg_in || !iface_in || !avg_out || !iface_out || !t_out || !status_out) return GRP_E_INVALID_ARG;
  if ((const double*)avg_out == avg_in || (const double*)iface_out == iface_in) return GRP_E_INVALID_ARG;
  if (isnan(t) || isnan(t_end)) return GRP_E_INVALID_ARG;

  // a pending launch error of earlier, unrelated work on this thread is
  // cleared here so that it is not reported as this call's failure
  (void)cudaGetLastError();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return GRP_E_CUDA;
  {
    std::lock_guard<std::mutex> lock(g_scratch_lock);
    if (!g_scratch_addr[dev]) {
      // once per device, with that device current: the device address of the
      // scratch (in host code the symbol itself is only a host-side stand-in)
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return GRP_E_CUDA;
      g_scratch_addr[dev] = (unsigned char*)p;
    }
  }
  unsigned char* base = g_scratch_addr[dev];
  cudaStream_t s = (cudaStream_t)stream;
  const int N = n_cells, nif = N + (bc == GRP_BC_TRANSMISSIVE ? 1 : 0);
  const double dx = (x_right - x_left) / N;
  Words* w = (Words*)(base + OFF_WORDS);

  k_noalloc_setup<<<nblk(nif, 256), 256, 0, s>>>(base, N, nif, dx, bc, t);

  StepArgs a;
  a.sys = system; a.M = M; a.C = system == GRP_EULER_IDEAL ? 3 : 1;
  a.recon = GRP_RECON_GRPREC;
  a.ph = make_phys(lambda, gamma, 1e-12, 50, 0);
  a.cfl = cfl; a.t_end = t_end; a.dt_hold = 1;
  a.n_domains = 1; a.ncell = N; a.nif = nif;
  a.cell_off = w->cell_off; a.if_off = w->if_off;
  a.cell_dom = (const int*)(base + OFF_CELL_DOM); a.if_dom = (const int*)(base + OFF_IF_DOM);
  a.dx = &w->dx; a.bc = &w->bc;
  a.avg = avg_in; a.avg_new = avg_out; a.ifc = iface_in; a.ifc_new = iface_out;
  a.flux = (double*)(base + OFF_FLUX);
  a.pold = (double*)(base + OFF_POLD);
  a.ds = (DomStep*)(base + OFF_DS);
  a.low = base + OFF_LOW; a.troubled = base + OFF_TROUBLED;
  a.t = &w->t; a.dt_prev = &w->dt_prev; a.nstep = &w->nstep; a.status = &w->status;
  a.smax_bits = &w->smax_bits;
  a.bad = w->bad; a.inad = &w->inad; a.fail = &w->fail; a.any_bad = w->any_bad;
  a.tlist[0] = (int*)(base + OFF_TLIST0); a.tlist[1] = (int*)(base + OFF_TLIST1);
  a.ilist = (int*)(base + OFF_ILIST); a.lcount = w->lcount;
  a.stats = w->stats;
  a.harvest = nullptr; a.harvest_count = nullptr; a.harvest_cap = 0; a.harvest_log2_stride = 0;

  // the flat step sequence of grp_step
  const bool euler = system == GRP_EULER_IDEAL;
  if (euler) k_smax<<<nblk(N, 256), 256, 0, s>>>(a);
  k_dt<<<1, 32, 0, s>>>(a);
  if (flux_dispatch(a, s) != cudaSuccess) return GRP_E_CUDA;
  if (euler) {
    k_update<SYS_EULER><<<nblk(N, 256), 256, 0, s>>>(a, -1);
    for (int r = 0; r < MAX_REPAIR; ++r) {
      if (gamma == 1.4) k_repair_list<true><<<LIST_BLOCKS, LIST_THREADS, 0, s>>>(a, r);
      else k_repair_list<false><<<LIST_BLOCKS, LIST_THREADS, 0, s>>>(a, r);
      k_update_list<SYS_EULER><<<LIST_BLOCKS, LIST_THREADS, 0, s>>>(a, r);
    }
  } else {
    k_update<SYS_ADV><<<nblk(N, 256), 256, 0, s>>>(a, -1);
  }
  k_finish<<<1, 32, 0, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return GRP_E_CUDA;
  if (cudaMemcpyAsync(t_out, &w->t, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GRP_E_CUDA;
  if (cudaMemcpyAsync(status_out, &w->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return GRP_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GRP_E_CUDA;
  return GRP_OK;
}
