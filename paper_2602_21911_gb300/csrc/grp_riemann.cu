// grp_riemann_batch: independent leading-term Riemann problems of the ideal
// gas solved in bulk with the solver of the flux kernel (exact solver of
// Section 2: Newton on the star pressure, relative change below rtol plus
// one more iteration), from a chosen Newton start.  It serves users who need
// the exact solver alone, and measures what each start costs in iterations.
#include <cuda_runtime.h>
#include <math.h>

#include "grp_device.cuh"
#include "grprec.h"

using namespace grp;

namespace {

template <bool G75>
__global__ void k_riemann_batch(Phys ph, long long n, const double* __restrict__ QL, const double* __restrict__ QR,
                                const double* __restrict__ p_start, double* __restrict__ ps,
                                int* __restrict__ iters, int* __restrict__ status, unsigned char* __restrict__ used)
{
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double l[3] = {QL[i], QL[n + i], QL[2 * n + i]};
  const double r[3] = {QR[i], QR[n + i], QR[2 * n + i]};
  int st, it = 0;
  double p = 0.0;
  bool by_net = false;
  if (p_start) {
    // explicit start; PVRS when it fails
    const Side L = make_side(ph, l), R = make_side(ph, r);
    double us;
    st = star_pressure<G75>(ph, L, R, p_start[i], p, us, it);
    if (st == ST_NO_CONV) {
      int it2 = 0;
      Phys pv = ph;
      pv.guess = 0;
      st = star_pressure<G75>(pv, L, R, 0.0, p, us, it2);
      it += it2;
    }
  } else {
    RSInfo info;
    double Q[3];
    Prim W;
    st = riemann_state<G75>(ph, l, r, true, Q, W, it, &info);
    p = info.ps;
    by_net = info.guess == 1;
  }
  ps[i] = st == ST_OK ? p : 0.0;
  iters[i] = it;
  status[i] = st;
  if (used) used[i] = by_net ? 1 : 0;
}

}  // namespace

extern "C" int grp_riemann_batch(double gamma, int guess, double newton_rtol, int newton_max_iter,
                                 const float* weights, const float* box, long long n, const double* QL,
                                 const double* QR, const double* p_start, double* ps, int* iters, int* status,
                                 unsigned char* used, void* stream)
{
  if (!(gamma > 1.0 && isfinite(gamma)) || guess < GRP_GUESS_PVRS || guess > GRP_GUESS_MLP) return GRP_E_INVALID_ARG;
  if (!(newton_rtol > 0.0) || newton_max_iter < 2 || n < 0) return GRP_E_INVALID_ARG;
  if (guess == GRP_GUESS_MLP && (!weights || !box)) return GRP_E_NO_MODEL;
  if (n == 0) return GRP_OK;
  if (!QL || !QR || !ps || !iters || !status) return GRP_E_INVALID_ARG;
  Phys ph = make_phys(0.0, gamma, newton_rtol, newton_max_iter, guess);
  ph.mlp_w = guess == GRP_GUESS_MLP ? weights : nullptr;
  ph.mlp_box = guess == GRP_GUESS_MLP ? box : nullptr;
  ph.features = guess == GRP_GUESS_MLP ? 1 : 0;
  const unsigned nb = (unsigned)((n + 127) / 128);
  if (gamma == 1.4)
    k_riemann_batch<true><<<nb, 128, 0, (cudaStream_t)stream>>>(ph, n, QL, QR, p_start, ps, iters, status, used);
  else
    k_riemann_batch<false><<<nb, 128, 0, (cudaStream_t)stream>>>(ph, n, QL, QR, p_start, ps, iters, status, used);
  return cudaGetLastError() == cudaSuccess ? GRP_OK : GRP_E_CUDA;
}
