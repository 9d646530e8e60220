// Two-dimensional stage pipeline of the moment-based multi-resolution HWENO
// scheme (Sec. 2.2 of Li, Shu & Qiu, arXiv 2201.12193) on sm_103a.
//
// One Runge-Kutta stage is four launches on the caller's stream:
//   rec2d   (Step 1)    every cell: 3x3 moments -> 16 Gauss-Lobatto values per
//                       variable (eq. (2D-re-u)) + KXRCF face-velocity partials;
//   flag2d  (Step 2)    KXRCF (eq. (KXRCF_), (line-integral-average_)), the
//                       dimension-by-dimension first-moment modification of
//                       troubled cells (eq. (vi)) and a compacted list of them;
//   rec2d*  (Step 2.3)  the troubled cells again, from the modified moments;
//   update2d (Step 3)   HLLC/LLF fluxes at the Gauss-Lobatto points of every
//                       face (eq. (integral2), (integral3)), the cell quadrature
//                       (eq. (integral1)), L(U) of eq. (2D-equ-int-approximation)
//                       and the SSP-RK3 combination (eq. (Runge-Kutta)).
// Each cell is reconstructed once per stage (plus once more if troubled):
// FP64 arithmetic is the scarce resource on this GPU, so the pipeline keeps
// the point values in HBM rather than recomputing a halo.
#include <algorithm>

#include "hweno_internal.h"

namespace hw {
namespace {

constexpr int TX = 32, TY = 4;   // update tile (one warp per row)
constexpr int RB = 128;          // threads per block of the per-cell kernels

__device__ __forceinline__ int mpt(const Img& m, int k, int l) {
  if (m.sx < 0) k = 3 - k;
  if (m.sy < 0) l = 3 - l;
  return k * 4 + l;
}

__device__ __forceinline__ long long goff(const Prob& P, int i, int j) { return (long long)j * P.gpitch + i; }

// Images of the 3x3 block around (i,j); the boundary map is separable, so
// three x-images and three y-images describe all nine cells.
struct Nbr {
  int xi[3], xs[3];     // image column and sign of the x first moment, for ox = -1, 0, 1
  int yj[3], ys[3];     // image row and sign of the y first moment, for oy = -1, 0, 1
};

__device__ __forceinline__ Nbr neighbours(const Prob& P, int i, int j) {
  Nbr n;
#pragma unroll
  for (int o = -1; o <= 1; ++o) {
    const Img a = image(P, i + o, j), b = image(P, i, j + o);
    n.xi[o + 1] = a.i; n.xs[o + 1] = a.sx;
    n.yj[o + 1] = b.j; n.ys[o + 1] = b.sy;
  }
  return n;
}

// Moment of kind 0 (average), 1 (x first moment) or 2 (y first moment) of
// the stencil cell (ox, oy); first moments of troubled cells come from the
// modified copy in the FLAGGED pass (eq. (vi) applied before Step 2.3).
template <bool FLAGGED>
__device__ __forceinline__ double load_mom(const Prob& P, const double* __restrict__ U, const uint8_t* __restrict__ mask,
                                           const double* __restrict__ Mod, const Nbr& n, int var, int kind, int ox,
                                           int oy) {
  const int ci = n.xi[ox + 1], cj = n.yj[oy + 1];
  const long long so = (long long)cj * P.pitch + ci;
  if (kind == 0) return U[(long long)(var * 3) * P.plane + so];
  double v;
  if (FLAGGED && mask[(long long)cj * P.nx + ci]) v = Mod[(long long)(var * 2 + kind - 1) * P.plane + so];
  else v = U[(long long)(var * 3 + kind) * P.plane + so];
  return (kind == 1 ? n.xs[ox + 1] : n.ys[oy + 1]) < 0 ? -v : v;
}

template <typename T, int NV, bool FLAGGED>
__device__ __forceinline__ void rec2d_cell(const Prob& P, const Weights<T>& W, const Beta2<T>& B,
                                           const double* __restrict__ U, const uint8_t* __restrict__ mask,
                                           const double* __restrict__ Mod, int i, int j, T* __restrict__ G,
                                           T* __restrict__ aux) {
  const Nbr nb = neighbours(P, i, j);
  const long long o = goff(P, i, j);
  T rinv[16];
  T pxl = T(0), pxr = T(0), pyb = T(0), pyt = T(0), nrm = T(0);
#pragma unroll 1
  for (int v = 0; v < NV; ++v) {
    T d[23];
#pragma unroll
    for (int c = 0; c < 23; ++c) {
      int kind, ox, oy;
      d4_slot(c, kind, ox, oy);
      d[c] = T(load_mom<FLAGGED>(P, U, mask, Mod, nb, v, kind, ox, oy));
    }
    T out[16];
    recon2d<T>(W, B, d, out);
#pragma unroll
    for (int p = 0; p < 16; ++p) G[(long long)(v * 16 + p) * P.gplane + o] = out[p];
    if (!FLAGGED) {
      if (v == 0) {
#pragma unroll
        for (int p = 0; p < 16; ++p) nrm = tmax(nrm, tabs(out[p]));
        if (P.eq == EQ_EULER) {
          // 1/rho at the 12 boundary points (the face velocities need only those)
          constexpr int bp[12] = {0, 1, 2, 3, 4, 7, 8, 11, 12, 13, 14, 15};
          if constexpr (sizeof(T) == 8) {
            T x[12], r[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) x[q] = out[bp[q]];
            batch_inverse<12, T>(x, r);
#pragma unroll
            for (int q = 0; q < 12; ++q) rinv[bp[q]] = r[q];
          } else {
#pragma unroll
            for (int q = 0; q < 12; ++q) rinv[bp[q]] = T(1) / out[bp[q]];
          }
        } else if (P.eq == EQ_BURGERS) {
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            pxl += gl_w<T>(l) * out[l];
            pxr += gl_w<T>(l) * out[12 + l];
            pyb += gl_w<T>(l) * out[l * 4];
            pyt += gl_w<T>(l) * out[l * 4 + 3];
          }
        } else {
          pxl = pxr = T(P.adv_a);
          pyb = pyt = T(P.adv_b);
        }
      } else if (P.eq == EQ_EULER && v == 1) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          pxl += gl_w<T>(l) * (out[l] * rinv[l]);
          pxr += gl_w<T>(l) * (out[12 + l] * rinv[12 + l]);
        }
      } else if (P.eq == EQ_EULER && v == 2) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          pyb += gl_w<T>(k) * (out[k * 4] * rinv[k * 4]);
          pyt += gl_w<T>(k) * (out[k * 4 + 3] * rinv[k * 4 + 3]);
        }
      }
    }
  }
  if (!FLAGGED) {
    aux[0 * P.gplane + o] = pxl;
    aux[1 * P.gplane + o] = pxr;
    aux[2 * P.gplane + o] = pyb;
    aux[3 * P.gplane + o] = pyt;
    aux[4 * P.gplane + o] = nrm;
  }
}

template <typename T, int NV, bool FLAGGED>
__global__ void __launch_bounds__(RB) rec2d_kernel(Prob P, Weights<T> W, Beta2<T> B, const double* __restrict__ U,
                                                  const uint8_t* __restrict__ mask, const double* __restrict__ Mod,
                                                  const int* __restrict__ list, const int* __restrict__ count,
                                                  T* __restrict__ G, T* __restrict__ aux) {
  const long long ncell = (long long)P.nx * P.ny;
  const long long n = FLAGGED ? (long long)*count : ncell;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int cell = FLAGGED ? list[t] : (int)t;
    rec2d_cell<T, NV, FLAGGED>(P, W, B, U, mask, Mod, cell % P.nx, cell / P.nx, G, aux);
  }
}

// KXRCF value of eq. (KXRCF_) with eq. (line-integral-average_): inflow faces by
// the sign of the GL-weighted face velocity (average of both sides), jumps of
// the indicator variable (variable 0) weighted by dy w_l or dx w_k.
template <typename T>
__device__ __forceinline__ T kxrcf2d(const Prob& P, const Weights<T>& W, const T* __restrict__ G,
                                     const T* __restrict__ aux, int i, int j) {
  const long long o = goff(P, i, j);
  const Img L = image(P, i - 1, j), R = image(P, i + 1, j), Bo = image(P, i, j - 1), Tp = image(P, i, j + 1);
  const long long oL = goff(P, L.i, L.j), oR = goff(P, R.i, R.j), oB = goff(P, Bo.i, Bo.j), oT = goff(P, Tp.i, Tp.j);
  const T vxl = T(0.5) * (aux[(L.sx < 0 ? 0 : 1) * P.gplane + oL] + aux[0 * P.gplane + o]);
  const T vxr = T(0.5) * (aux[1 * P.gplane + o] + aux[(R.sx < 0 ? 1 : 0) * P.gplane + oR]);
  const T vyb = T(0.5) * (aux[(Bo.sy < 0 ? 2 : 3) * P.gplane + oB] + aux[2 * P.gplane + o]);
  const T vyt = T(0.5) * (aux[3 * P.gplane + o] + aux[(Tp.sy < 0 ? 3 : 2) * P.gplane + oT]);
  const T dx = T(P.dx), dy = T(P.dy);
  T s = T(0), len = T(0);
  if (vxl > T(KX_VDEAD)) {
#pragma unroll
    for (int l = 0; l < 4; ++l) s += dy * gl_w<T>(l) * (G[(long long)(l)*P.gplane + o] - G[(long long)mpt(L, 3, l) * P.gplane + oL]);
    len += dy;
  }
  if (-vxr > T(KX_VDEAD)) {
#pragma unroll
    for (int l = 0; l < 4; ++l) s += dy * gl_w<T>(l) * (G[(long long)(12 + l) * P.gplane + o] - G[(long long)mpt(R, 0, l) * P.gplane + oR]);
    len += dy;
  }
  if (vyb > T(KX_VDEAD)) {
#pragma unroll
    for (int k = 0; k < 4; ++k) s += dx * gl_w<T>(k) * (G[(long long)(k * 4) * P.gplane + o] - G[(long long)mpt(Bo, k, 3) * P.gplane + oB]);
    len += dx;
  }
  if (-vyt > T(KX_VDEAD)) {
#pragma unroll
    for (int k = 0; k < 4; ++k) s += dx * gl_w<T>(k) * (G[(long long)(k * 4 + 3) * P.gplane + o] - G[(long long)mpt(Tp, k, 0) * P.gplane + oT]);
    len += dx;
  }
  const T nrm = aux[4 * P.gplane + o];
  if (len == T(0) || nrm == T(0)) return T(0);
  return tabs(s) / len / (W.h2 * nrm);
}

template <typename T, int NV>
__global__ void __launch_bounds__(TX * TY) flag2d_kernel(Prob P, Weights<T> W, const double* __restrict__ U,
                                                        const T* __restrict__ G, const T* __restrict__ aux,
                                                        uint8_t* __restrict__ mask, double* __restrict__ Mod,
                                                        int* __restrict__ list, int* __restrict__ count,
                                                        double* __restrict__ aleph) {
  const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
  const bool valid = i < P.nx && j < P.ny;
  bool flag = false;
  if (valid) {
    if (P.indicator == IND_ALL) {
      flag = true;
    } else if (P.indicator == IND_KXRCF) {
      const T a = kxrcf2d<T>(P, W, G, aux, i, j);
      if (aleph) aleph[(long long)j * P.nx + i] = double(a);
      flag = a > T(1);
    }
  }
  // warp-aggregated append to the troubled-cell list (a warp is one tile row)
  const unsigned act = __ballot_sync(0xffffffffu, flag);
  if (act) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(act));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (flag) list[base + __popc(act & ((1u << lane) - 1u))] = j * P.nx + i;
  }
  if (!valid) return;
  mask[(long long)j * P.nx + i] = flag ? 1 : 0;
  if (!flag) return;
  // Step 2.2 (dimension by dimension): modified first moments from the
  // pre-modification moments of the x and y neighbours.
  const Img L = image(P, i - 1, j), R = image(P, i + 1, j), Bo = image(P, i, j - 1), Tp = image(P, i, j + 1);
  const long long o = (long long)j * P.pitch + i;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double uL = U[sidx(P, v, 0, L.i, L.j)], uR = U[sidx(P, v, 0, R.i, R.j)];
    const double vL = L.sx * U[sidx(P, v, 1, L.i, L.j)], vR = R.sx * U[sidx(P, v, 1, R.i, R.j)];
    const double uB = U[sidx(P, v, 0, Bo.i, Bo.j)], uT = U[sidx(P, v, 0, Tp.i, Tp.j)];
    const double wB = Bo.sy * U[sidx(P, v, 2, Bo.i, Bo.j)], wT = Tp.sy * U[sidx(P, v, 2, Tp.i, Tp.j)];
    Mod[(long long)(v * 2 + 0) * P.plane + o] = MOD_WU * (uR - uL) + MOD_WV * (vL + vR);
    Mod[(long long)(v * 2 + 1) * P.plane + o] = MOD_WU * (uT - uB) + MOD_WV * (wB + wT);
  }
}

template <typename T, int NV>
__device__ __forceinline__ void gl_state(const Prob& P, const T* __restrict__ G, const Img& m, int k, int l, T (&u)[NV]) {
  const long long o = goff(P, m.i, m.j);
  const int p = mpt(m, k, l);
#pragma unroll
  for (int v = 0; v < NV; ++v) u[v] = G[(long long)(v * 16 + p) * P.gplane + o];
}

struct Rk {
  const double* Uin; const double* Un; double* Uout;
  const uint8_t* mask; const double* Mod; const uint8_t* maskN; const double* ModN;
  double dt, cA, cB;
  double* Lout; double* Umod;
  unsigned* status;
};

template <typename T, int NV>
__global__ void __launch_bounds__(TX * TY) update2d_kernel(Prob P, const T* __restrict__ G, Rk S) {
  __shared__ T xf[TY][TX + 1][4][NV];
  __shared__ T yf[TY + 1][TX][4][NV];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int i = i0 + tx, j = j0 + ty;
  const bool live = i < P.nx && j < P.ny;
  const Img self{i, j, 1, 1};
  // Every face flux of the tile at one Gauss-Lobatto point per iteration, by one
  // call site, so that a face shared by two tiles gets bitwise the same flux
  // from both (the flux differences then telescope exactly in FP64).
  // xf[r][c] is the face left of cell (i0 + c, j0 + r); yf[r][c] the face below it.
  constexpr int NXP = (TX + 1) * TY * 4, NYP = TX * (TY + 1) * 4;
  for (int f = ty * TX + tx; f < NXP + NYP; f += TX * TY) {
    T uL[NV], uR[NV];
    if (f < NXP) {
      const int l = f & 3, face = f >> 2, c = face % (TX + 1), r = face / (TX + 1);
      const int il = i0 + c - 1, jj = j0 + r;
      if (jj >= P.ny || il >= P.nx) continue;
      gl_state<T, NV>(P, G, image(P, il, jj), 3, l, uL);
      gl_state<T, NV>(P, G, image(P, il + 1, jj), 0, l, uR);
      num_flux<T, NV>(P, uL, uR, 0, xf[r][c][l]);
    } else {
      const int g = f - NXP, k = g & 3, face = g >> 2, c = face % TX, r = face / TX;
      const int ii = i0 + c, jb = j0 + r - 1;
      if (ii >= P.nx || jb >= P.ny) continue;
      gl_state<T, NV>(P, G, image(P, ii, jb), k, 3, uL);
      gl_state<T, NV>(P, G, image(P, ii, jb + 1), k, 0, uR);
      num_flux<T, NV>(P, uL, uR, 1, yf[r][c][k]);
    }
  }
  __syncthreads();
  if (!live) return;
  // face integrals (eq. (integral2), (integral3)) and the cell quadrature (eq. (integral1))
  T Fp[NV], Fm[NV], Fpe[NV], Fme[NV], Gp[NV], Gm[NV], Gpx[NV], Gmx[NV], Fc[NV], Gc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Fp[v] = Fm[v] = Fpe[v] = Fme[v] = Gp[v] = Gm[v] = Gpx[v] = Gmx[v] = Fc[v] = Gc[v] = T(0);
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const T w = gl_w<T>(l), we = gl_w<T>(l) * gl_x<T>(l);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Fp[v] += w * xf[ty][tx + 1][l][v];
      Fpe[v] += we * xf[ty][tx + 1][l][v];
      Fm[v] += w * xf[ty][tx][l][v];
      Fme[v] += we * xf[ty][tx][l][v];
      Gp[v] += w * yf[ty + 1][tx][l][v];
      Gpx[v] += we * yf[ty + 1][tx][l][v];
      Gm[v] += w * yf[ty][tx][l][v];
      Gmx[v] += we * yf[ty][tx][l][v];
    }
  }
  if constexpr (NV == 4 && sizeof(T) == 8) {
    // Euler, FP64: the 16 reciprocal densities with one division
    T rho[16], inv[16];
#pragma unroll
    for (int p = 0; p < 16; ++p) rho[p] = G[(long long)p * P.gplane + goff(P, i, j)];
    batch_inverse<16, T>(rho, inv);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        T u[NV], fx[NV], gy[NV];
        gl_state<T, NV>(P, G, self, k, l, u);
        euler_flux_inv<T, NV>(P, u, inv[k * 4 + l], 0, fx);
        euler_flux_inv<T, NV>(P, u, inv[k * 4 + l], 1, gy);
        const T w = gl_w<T>(k) * gl_w<T>(l);
#pragma unroll
        for (int v = 0; v < NV; ++v) { Fc[v] += w * fx[v]; Gc[v] += w * gy[v]; }
      }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        T u[NV], fx[NV], gy[NV];
        gl_state<T, NV>(P, G, self, k, l, u);
        phys_flux<T, NV>(P, u, 0, fx);
        phys_flux<T, NV>(P, u, 1, gy);
        const T w = gl_w<T>(k) * gl_w<T>(l);
#pragma unroll
        for (int v = 0; v < NV; ++v) { Fc[v] += w * fx[v]; Gc[v] += w * gy[v]; }
      }
  }
  // eq. (2D-equ-int-approximation); the average equation in FP64 from the
  // face integrals so that the flux differences telescope in every precision
  const double idx = 1.0 / P.dx, idy = 1.0 / P.dy;
  const T tidx = T(idx), tidy = T(idy);
  const long long so = (long long)j * P.pitch + i;
  const long long cell = (long long)j * P.nx + i;
  const bool fk = S.mask[cell] != 0;
  const bool fn = S.maskN && S.maskN[cell] != 0;
  double newavg[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double L[3];
    L[0] = -((double)Fp[v] - (double)Fm[v]) * idx - ((double)Gp[v] - (double)Gm[v]) * idy;
    L[1] = (double)(-(Fp[v] + Fm[v]) * T(0.5) * tidx + Fc[v] * tidx - (Gpx[v] - Gmx[v]) * tidy);
    L[2] = (double)(-(Fpe[v] - Fme[v]) * tidx - (Gp[v] + Gm[v]) * T(0.5) * tidy + Gc[v] * tidy);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const long long si = (long long)(v * 3 + m) * P.plane + so;
      const double uin = (m > 0 && fk) ? S.Mod[(long long)(v * 2 + m - 1) * P.plane + so] : S.Uin[si];
      if (S.Lout) {
        S.Lout[si] = L[m];
        if (S.Umod) S.Umod[si] = uin;
        continue;
      }
      const double un = (m > 0 && fn) ? S.ModN[(long long)(v * 2 + m - 1) * P.plane + so] : S.Un[si];
      const double r = S.cA * un + S.cB * (uin + S.dt * L[m]);
      S.Uout[si] = r;
      if (m == 0) newavg[v] = r;
      if (!isfinite(r)) atomicOr(S.status, ST_NONFINITE);
    }
  }
  if (!S.Lout && P.eq == EQ_EULER && NV == 4) {
    const double rho = newavg[0];
    const double p = (P.gamma - 1.0) * (newavg[NV - 1] - 0.5 * (newavg[1] * newavg[1] + newavg[2] * newavg[2]) / rho);
    if (!(rho > 0.0) || !(p > 0.0)) atomicOr(S.status, ST_NONPOSITIVE);
  }
}

template <typename T, int NV>
void stage_t(const Prob& P, const Weights<T>& W, const Beta2<T>& Bt, const Bufs& B, const StageCall& S, cudaStream_t st) {
  const long long ncell = (long long)P.nx * P.ny;
  int* cnt = B.count + S.stage;
  cudaMemsetAsync(cnt, 0, sizeof(int), st);
  const int rblocks = (int)((ncell + RB - 1) / RB);
  if (B.prof) B.prof->begin(0, st);
  rec2d_kernel<T, NV, false><<<rblocks, RB, 0, st>>>(P, W, Bt, S.Uin, nullptr, nullptr, nullptr, nullptr,
                                                     (T*)B.G, (T*)B.aux);
  if (B.prof) B.prof->end(st);
  const dim3 blk(TX, TY), grd((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
  if (B.prof) B.prof->begin(1, st);
  flag2d_kernel<T, NV><<<grd, blk, 0, st>>>(P, W, S.Uin, (const T*)B.G, (const T*)B.aux, S.mask, S.Mod, B.list,
                                            cnt, S.aleph);
  if (B.prof) B.prof->end(st);
  if (P.indicator != IND_NONE) {
    const int fblocks = (int)std::min<long long>(rblocks, (long long)P.nsm * 8);
    if (B.prof) B.prof->begin(2, st);
    rec2d_kernel<T, NV, true><<<fblocks, RB, 0, st>>>(P, W, Bt, S.Uin, S.mask, S.Mod, B.list, cnt, (T*)B.G, nullptr);
    if (B.prof) B.prof->end(st);
  }
  Rk r{S.Uin, S.Un, S.Uout, S.mask, S.Mod, S.maskN, S.ModN, S.dt, S.cA, S.cB, S.Lout, S.Umod, B.status};
  if (B.prof) B.prof->begin(3, st);
  update2d_kernel<T, NV><<<grd, blk, 0, st>>>(P, (const T*)B.G, r);
  if (B.prof) B.prof->end(st);
}

}  // namespace

void run_stage_2d(const Prob& P, const HostTabs& T, int fp32, const Bufs& B, const StageCall& S, cudaStream_t st) {
  if (P.nvar == 4) {
    if (fp32) stage_t<float, 4>(P, T.wf, T.b2f, B, S, st);
    else stage_t<double, 4>(P, T.wd, T.b2d, B, S, st);
  } else {
    if (fp32) stage_t<float, 1>(P, T.wf, T.b2f, B, S, st);
    else stage_t<double, 1>(P, T.wd, T.b2d, B, S, st);
  }
}

}  // namespace hw
