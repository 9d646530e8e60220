// Allocation-free variant of the CFL wave-speed reduction (hweno_max_dt_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs while a memory budget is
// frozen, that must not trigger the implicit device synchronisation an
// allocation can cause, or that has no way to keep a handle (which allocates
// its buffers at creation) alive.  This entry point needs no handle: the
// caller passes the state and the result buffer, and the per-block partial
// maxima live in the file-scope array below, which every GPU that loads the
// library holds until the process exits.
//
// Limits: one partial per 256 cells, NOALLOC_MAX_BLOCKS of them, so at most
// NOALLOC_MAX_CELLS = 4,194,304 cells (2048 x 2048); larger grids are rejected.
// The partial array is shared by every call on a device: calls whose work
// overlaps on the GPU (different streams, no ordering between them) race.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "hweno.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NOALLOC_MAX_BLOCKS = 16384;
constexpr long long NOALLOC_MAX_CELLS = (long long)NOALLOC_MAX_BLOCKS * NA_THREADS;
constexpr int NA_MAX_DEVICES = 64;

// Partial maxima: [0, NOALLOC_MAX_BLOCKS) for x, [NOALLOC_MAX_BLOCKS, 2*...) for y (256 KiB).
static __device__ __align__(256) double g_noalloc_partials[2 * NOALLOC_MAX_BLOCKS];

// Device address of g_noalloc_partials per device, taken once per device.
double* g_partials_addr[NA_MAX_DEVICES] = {nullptr};
std::mutex g_setup_mutex;

struct NaProb {
  int nx, ny, nvar, nmom, eq;
  double gamma, adv_a, adv_b;
};

// Largest |f'| (scalar laws) or |velocity| + sound speed (Euler) per direction
// over the cells of block b (cell averages; a non-physical average gives +inf).
__global__ void __launch_bounds__(NA_THREADS) noalloc_speed_kernel(NaProb P, const double* __restrict__ m,
                                                                  double* __restrict__ part) {
  __shared__ double sm[2][NA_THREADS / 32];
  const long long n = (long long)P.nx * P.ny;
  const long long t = (long long)blockIdx.x * NA_THREADS + threadIdx.x;
  double sx = 0.0, sy = 0.0;
  if (t < n) {
    const int nmom = P.nmom;
    const long long plane = n;
    if (P.eq == HWENO_ADVECTION) { sx = fabs(P.adv_a); sy = fabs(P.adv_b); }
    else if (P.eq == HWENO_BURGERS) { sx = sy = fabs(m[t]); }
    else {
      const double rho = m[t];
      const double mu = m[(long long)1 * nmom * plane + t] / rho;
      const double nu = P.nvar == 4 ? m[(long long)2 * nmom * plane + t] / rho : 0.0;
      const double E = m[(long long)(P.nvar - 1) * nmom * plane + t];
      const double p = (P.gamma - 1.0) * (E - 0.5 * rho * (mu * mu + nu * nu));
      const double c = sqrt(P.gamma * p / rho);
      sx = fabs(mu) + c;
      sy = fabs(nu) + c;
      if (!(rho > 0.0) || !(p > 0.0) || !isfinite(sx + sy)) sx = sy = INFINITY;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sx = fmax(sx, __shfl_down_sync(0xffffffffu, sx, o));
    sy = fmax(sy, __shfl_down_sync(0xffffffffu, sy, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sm[0][wid] = sx; sm[1][wid] = sy; }
  __syncthreads();
  if (wid == 0) {
    sx = lane < NA_THREADS / 32 ? sm[0][lane] : 0.0;
    sy = lane < NA_THREADS / 32 ? sm[1][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      sx = fmax(sx, __shfl_down_sync(0xffffffffu, sx, o));
      sy = fmax(sy, __shfl_down_sync(0xffffffffu, sy, o));
    }
    if (lane == 0) { part[blockIdx.x] = sx; part[NOALLOC_MAX_BLOCKS + blockIdx.x] = sy; }
  }
}

// One block: the maxima over the nb partials of this call, then dt.
__global__ void __launch_bounds__(NA_THREADS) noalloc_finish_kernel(const double* __restrict__ part, int nb, int dim,
                                                                   double dx, double dy, double cfl,
                                                                   double* __restrict__ out) {
  __shared__ double sm[2][NA_THREADS / 32];
  double sx = 0.0, sy = 0.0;
  for (int b = threadIdx.x; b < nb; b += NA_THREADS) {
    sx = fmax(sx, part[b]);
    sy = fmax(sy, part[NOALLOC_MAX_BLOCKS + b]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    sx = fmax(sx, __shfl_down_sync(0xffffffffu, sx, o));
    sy = fmax(sy, __shfl_down_sync(0xffffffffu, sy, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sm[0][wid] = sx; sm[1][wid] = sy; }
  __syncthreads();
  if (threadIdx.x == 0) {
    sx = 0.0;
    sy = 0.0;
    for (int w = 0; w < NA_THREADS / 32; ++w) { sx = fmax(sx, sm[0][w]); sy = fmax(sy, sm[1][w]); }
    double dt;
    if (dim == 1) dt = sx > 0.0 ? cfl * dx / sx : INFINITY;
    else {
      const double r = sx / dx + sy / dy;
      dt = r > 0.0 ? cfl / r : INFINITY;
    }
    out[0] = sx;
    out[1] = sy;
    out[2] = (isfinite(sx) && isfinite(sy)) ? dt : 0.0;
  }
}

}  // namespace

extern "C" hweno_status hweno_max_dt_noalloc(const hweno_grid* g, double gamma, const double* m, double cfl,
                                             double* out, void* cuda_stream) {
  if (!g || !m || !out) {
    fprintf(stderr, "hweno_max_dt_noalloc: grid, m and out must not be NULL\n");
    return HWENO_EINVAL;
  }
  if ((g->dim != 1 && g->dim != 2) || g->nx < 1 || (g->dim == 2 && g->ny < 1) || !(g->x1 > g->x0) ||
      (g->dim == 2 && !(g->y1 > g->y0)) || g->eq < 0 || g->eq > 2 || !(cfl > 0.0) ||
      (g->eq == HWENO_EULER && !(gamma > 1.0))) {
    fprintf(stderr, "hweno_max_dt_noalloc: invalid grid, equation, gamma or cfl\n");
    return HWENO_EINVAL;
  }
  const long long ncell = (long long)g->nx * (g->dim == 2 ? g->ny : 1);
  if (ncell > NOALLOC_MAX_CELLS) {
    fprintf(stderr, "hweno_max_dt_noalloc: %lld cells exceed the maximum of %lld (static scratch of %d partials)\n",
            ncell, NOALLOC_MAX_CELLS, NOALLOC_MAX_BLOCKS);
    return HWENO_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return HWENO_ECUDA;
  double* part;
  {
    // first call on this device (with the device current): host code needs the
    // device address of the array; its name is only a host-side stand-in.
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
      if (e != cudaSuccess || !p) {
        fprintf(stderr, "hweno_max_dt_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
        return HWENO_ECUDA;
      }
      g_partials_addr[dev] = (double*)p;
    }
    part = g_partials_addr[dev];
  }
  NaProb P;
  P.nx = g->nx;
  P.ny = g->dim == 2 ? g->ny : 1;
  P.nvar = g->eq == HWENO_EULER ? (g->dim == 1 ? 3 : 4) : 1;
  P.nmom = g->dim == 1 ? 2 : 3;
  P.eq = g->eq;
  P.gamma = gamma;
  P.adv_a = g->adv_a;
  P.adv_b = g->adv_b;
  const double dx = (g->x1 - g->x0) / g->nx;
  const double dy = g->dim == 2 ? (g->y1 - g->y0) / g->ny : 1.0;
  const int nb = (int)((ncell + NA_THREADS - 1) / NA_THREADS);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  noalloc_speed_kernel<<<nb, NA_THREADS, 0, st>>>(P, m, part);
  noalloc_finish_kernel<<<1, NA_THREADS, 0, st>>>(part, nb, g->dim, dx, dy, cfl, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "hweno_max_dt_noalloc: launch failed: %s\n", cudaGetErrorString(e));
    return HWENO_ECUDA;
  }
  return HWENO_OK;
}
