// Reductions over the cell averages (FP64): the CFL wave speeds and the
// conservation totals.  Warp shuffles inside a block, one partial per block,
// then a single-block pass in a fixed order (deterministic for a given grid).
#include <math.h>

#include <algorithm>

#include "hweno_internal.h"

namespace hw {
namespace {

constexpr int RT = 256;       // threads per block
constexpr int MAXB = 1024;    // blocks of the first pass (partials per quantity)

template <int K>
__device__ __forceinline__ void block_reduce(double (&v)[K], bool is_max, double (*sm)[RT / 32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v[k], o);
      v[k] = is_max ? fmax(v[k], w) : v[k] + w;
    }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sm[k][wid] = v[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double x = lane < RT / 32 ? sm[k][lane] : 0.0;   // 0 is neutral for sums and for max of speeds
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_down_sync(0xffffffffu, x, o);
        x = is_max ? fmax(x, w) : x + w;
      }
      v[k] = x;
    }
  }
}

// Largest |f'| (scalars) or |velocity| + sound speed (Euler) per direction,
// from cell averages.  A non-physical average yields +inf (dt = 0).  With the
// positivity check off the sound speed uses max(p, 0).
__global__ void __launch_bounds__(RT) wavespeed_kernel(Prob P, const double* __restrict__ U, double* __restrict__ part) {
  __shared__ double sm[2][RT / 32];
  double v[2] = {0.0, 0.0};
  const long long n = (long long)P.nx * (P.jhi - P.jlo);   // owned rows
  for (long long t = (long long)blockIdx.x * RT + threadIdx.x; t < n; t += (long long)gridDim.x * RT) {
    const int i = (int)(t % P.nx), j = P.jlo + (int)(t / P.nx);
    if (P.sol_j > 0 && is_solid(P, i, j)) continue;    // the step's block takes no part
    double sx, sy;
    if (P.eq == EQ_ADV) { sx = fabs(P.adv_a); sy = fabs(P.adv_b); }
    else if (P.eq == EQ_BURGERS) { sx = sy = fabs(U[sidx(P, 0, 0, i, j)]); }
    else {
      const double rho = U[sidx(P, 0, 0, i, j)];
      const double mu = U[sidx(P, 1, 0, i, j)] / rho;
      const double nu = P.nvar == 4 ? U[sidx(P, 2, 0, i, j)] / rho : 0.0;
      const double E = U[sidx(P, P.nvar - 1, 0, i, j)];
      const double p = (P.gamma - 1.0) * (E - 0.5 * rho * (mu * mu + nu * nu));
      cell_speeds(P, rho, mu, nu, p, sx, sy);
    }
    v[0] = fmax(v[0], sx);
    v[1] = fmax(v[1], sy);
  }
  block_reduce<2>(v, true, sm);
  if (threadIdx.x == 0) { part[blockIdx.x] = v[0]; part[MAXB + blockIdx.x] = v[1]; }
}

__global__ void __launch_bounds__(RT) totals_kernel(Prob P, const double* __restrict__ U, double* __restrict__ part) {
  __shared__ double sm[4][RT / 32];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const long long n = (long long)P.nx * (P.jhi - P.jlo);   // owned rows
  for (long long t = (long long)blockIdx.x * RT + threadIdx.x; t < n; t += (long long)gridDim.x * RT) {
    const int i = (int)(t % P.nx), j = P.jlo + (int)(t / P.nx);
    if (P.sol_j > 0 && is_solid(P, i, j)) continue;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < P.nvar) v[k] += U[sidx(P, k, 0, i, j)];
  }
  block_reduce<4>(v, false, sm);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) part[k * MAXB + blockIdx.x] = v[k];
}

// Single block: reduce K rows of nb partials each into out[K].
template <int K>
__global__ void __launch_bounds__(RT) finish_kernel(const double* __restrict__ part, int nb, bool is_max,
                                                    double* __restrict__ out) {
  __shared__ double sm[K][RT / 32];
  double v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    v[k] = 0.0;
    for (int b = threadIdx.x; b < nb; b += RT) v[k] = is_max ? fmax(v[k], part[k * MAXB + b]) : v[k] + part[k * MAXB + b];
  }
  block_reduce<K>(v, is_max, sm);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = v[k];
}

int first_pass_blocks(const Prob& P) {
  const long long n = (long long)P.nx * (P.jhi - P.jlo);
  return (int)std::min<long long>(MAXB, (n + RT - 1) / RT);
}

// The step length of hweno_advance on the device, from the wave-speed maxima in
// sp[0..1]: the CFL rule of the host's hweno_max_dt (same expressions), clipped
// to the remaining time; st[0] = t, st[1] = dt, st[2] = steps taken,
// st[3] = the time at the start of the step, par = {T, cfl, max_steps}.  dt = -1 marks a step to skip (done, step budget
// spent, or a non-physical average, which also sets ST_NONPOSITIVE and
// ST_NODT; the latter fails the call whatever the positivity switch).
__global__ void advance_dt_kernel(Prob P, const double* __restrict__ sp, const double* __restrict__ par,
                                  double* __restrict__ st, unsigned* __restrict__ status) {
  const double ax = sp[0], ay = sp[1];
  const double T = par[0], cfl = par[1], maxs = par[2];
  double dtc;
  if (P.nmom == 2) dtc = ax > 0.0 ? cfl * P.dx / ax : INFINITY;
  else {
    const double r = ax / P.dx + ay / P.dy;
    dtc = r > 0.0 ? cfl / r : INFINITY;
  }
  const double t = st[0], rem = T - t;
  st[3] = t;
  double dt = -1.0;
  if (!(dtc > 0.0) || isnan(dtc)) {
    atomicOr(status, ST_NONPOSITIVE | ST_NODT);
  } else if (st[2] < maxs && rem > 1e-14 * fmax(1.0, fabs(T))) {
    dt = fmin(dtc, rem);
    st[0] = dtc >= rem ? T : t + dt;
    st[2] += 1.0;
  }
  st[1] = dt;
}

// Fixed-state ghost table for the stage at time t (or, with dtp set, at
// *tn + c * *dtp read on the device; a skipped step, *dtp < 0, leaves it).
// Products and sums are rounded separately (no fused multiply-add), as the
// host computes the same positions and times.
__global__ void fixfill_kernel(FixSpec F, double* __restrict__ tab, double t, const double* __restrict__ tn,
                               const double* __restrict__ dtp, double c) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 4 * F.fixlen) return;
  if (dtp) {
    const double dt = *dtp;
    if (dt < 0.0) return;
    t = __dadd_rn(*tn, __dmul_rn(c, dt));
  }
  const int side = q / F.fixlen, pos = q % F.fixlen - 1;
  const double at = __dmul_rn((double)pos + 0.5, side < 2 ? F.dy : F.dx);
  const double pc = __dadd_rn(side < 2 ? F.y0 : F.x0, at);
  const double* src = nullptr;
  if (pos <= F.n[side]) {
    if (F.seg[side] && pc < __dadd_rn(F.c0[side], __dmul_rn(F.speed[side], t))) src = F.a[side];
    else if (F.inflow[side]) src = F.b[side];
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) tab[4 * (long long)q + v] = src ? src[v] : 0.0;
}

// The float copy of rows [j0, j0 + nrows) of every moment plane (FP32 form):
// each state value rounded to nearest by integer work, as the update kernel
// rounds the values it writes.
__global__ void shadow32_kernel(Prob P, const double* __restrict__ U, float* __restrict__ U32, int j0, int nrows) {
  const long long per = (long long)nrows * P.nx, n = (long long)P.nvar * P.nmom * per;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long q = t / per, r = t % per;
    const long long si = q * P.plane + (long long)(j0 + r / P.nx) * P.pitch + r % P.nx;
    U32[si] = f32_rn(U[si]);
  }
}

}  // namespace

void run_shadow32(const Prob& P, const double* U, float* U32, int j0, int nrows, cudaStream_t st) {
  const long long n = (long long)P.nvar * P.nmom * nrows * P.nx;
  if (n <= 0) return;
  const int nb = (int)std::min<long long>((n + RT - 1) / RT, (long long)P.nsm * 16);
  shadow32_kernel<<<nb, RT, 0, st>>>(P, U, U32, j0, nrows);
}

void run_fixfill(const FixSpec& F, double* tab, double t, const double* tn, const double* dtp, double c,
                 cudaStream_t st) {
  const int n = 4 * F.fixlen;
  fixfill_kernel<<<(n + 127) / 128, 128, 0, st>>>(F, tab, t, tn, dtp, c);
}

void run_advance_dt(const Prob& P, const double* speeds, const double* par, double* st, unsigned* status,
                    cudaStream_t s) {
  advance_dt_kernel<<<1, 1, 0, s>>>(P, speeds, par, st, status);
}

int reduce_partials_len(const Prob&) { return 4 * MAXB; }

void run_wavespeed(const Prob& P, const double* U, double* partials, double* out, cudaStream_t st) {
  const int nb = first_pass_blocks(P);
  wavespeed_kernel<<<nb, RT, 0, st>>>(P, U, partials);
  finish_kernel<2><<<1, RT, 0, st>>>(partials, nb, true, out);
}

void run_totals(const Prob& P, const double* U, double* partials, double* out, cudaStream_t st) {
  const int nb = first_pass_blocks(P);
  totals_kernel<<<nb, RT, 0, st>>>(P, U, partials);
  finish_kernel<4><<<1, RT, 0, st>>>(partials, nb, false, out);
}

}  // namespace hw
