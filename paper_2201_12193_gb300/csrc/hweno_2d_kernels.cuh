// Kernels of the two-dimensional stage pipeline and of the batched persistent
// stage (shared by the per-precision translation units; internal linkage).
#pragma once
#include <algorithm>
#include <type_traits>

#include "hweno_internal.h"

namespace hw {
namespace {


constexpr int TX = 32, TY = 4;   // update tile (one warp per row)
constexpr int RB = 128;          // threads per block of the per-cell kernels

// Images of the 3x3 block around (i,j); the boundary map is separable, so
// three x-images and three y-images describe all nine cells.
struct Nbr {
  int xi[3], xs[3];     // image column and sign of the x first moment, for ox = -1, 0, 1
  int yj[3], ys[3];     // image row and sign of the y first moment, for oy = -1, 0, 1
  int neg[3][3];        // variables negated by reflective walls, [oy + 1][ox + 1]
  int fs[3][3];         // fixed-state ghost entry (-1: none), set when FIX
  int ci[3][3], cj[3][3], csx[3][3], csy[3][3];   // FIX: the full image of each cell
};

template <bool FIX>
__device__ __forceinline__ Nbr neighbours(const Prob& P, int i, int j) {
  Nbr n;
  int nx[3], ny[3];
#pragma unroll
  for (int o = -1; o <= 1; ++o) {
    // by the kinds alone: a fixed ghost in the separable x or y image does
    // not make its row or column fixed for the diagonal cells
    const Img a = image_kind(P, i + o, j), b = image_kind(P, i, j + o);
    n.xi[o + 1] = a.i; n.xs[o + 1] = a.sx; nx[o + 1] = a.neg;
    n.yj[o + 1] = b.j; n.ys[o + 1] = b.sy; ny[o + 1] = b.neg;
  }
#pragma unroll
  for (int oy = 0; oy < 3; ++oy)
#pragma unroll
    for (int ox = 0; ox < 3; ++ox) n.neg[oy][ox] = nx[ox] | ny[oy];
  if constexpr (FIX) {
    // fixed-state ghosts and the solid block break the separable form: the full
    // image of each cell (equal to the separable one wherever neither applies)
#pragma unroll
    for (int oy = 0; oy < 3; ++oy)
#pragma unroll
      for (int ox = 0; ox < 3; ++ox) {
        const Img m = image(P, i + ox - 1, j + oy - 1, i, j);
        n.fs[oy][ox] = m.fs;
        n.neg[oy][ox] = m.fs >= 0 ? m.neg : (P.sol_j > 0 ? m.neg : n.neg[oy][ox]);
        n.ci[oy][ox] = m.fs >= 0 ? n.xi[ox] : m.i;
        n.cj[oy][ox] = m.fs >= 0 ? n.yj[oy] : m.j;
        n.csx[oy][ox] = m.fs >= 0 ? n.xs[ox] : m.sx;
        n.csy[oy][ox] = m.fs >= 0 ? n.ys[oy] : m.sy;
      }
  }
  return n;
}

// Reconstruction passes: every cell from the stage input (PLAIN); the listed
// troubled cells from the modified moments (FLAGGED, Step 2.3); or every cell,
// those already flagged (mask 1) from the modified moments (MIXED: the learned
// indicator decides before Step 1).
enum RecMode { REC_PLAIN = 0, REC_FLAGGED = 1, REC_MIXED = 2 };

// Moment of kind 0 (average), 1 (x first moment) or 2 (y first moment) of
// the stencil cell (ox, oy); when usemod, first moments of flagged stencil
// cells come from the modified copy (eq. (vi) applied before Step 2.3).
template <int MODE, bool SIGNBIT, bool FIX>
__device__ __forceinline__ double load_mom(const Prob& P, const double* __restrict__ U, const uint8_t* __restrict__ mask,
                                           const double* __restrict__ Mod, const Nbr& n, int var, int kind, int ox,
                                           int oy, bool usemod) {
  if constexpr (FIX) {
    const int fs = n.fs[oy + 1][ox + 1];
    if (fs >= 0) return kind == 0 ? ((n.neg[oy + 1][ox + 1] >> var) & 1 ? -1.0 : 1.0) * P.fixtab[4 * fs + var] : 0.0;
  }
  const int ci = FIX ? n.ci[oy + 1][ox + 1] : n.xi[ox + 1], cj = FIX ? n.cj[oy + 1][ox + 1] : n.yj[oy + 1];
  const int sxm = FIX ? n.csx[oy + 1][ox + 1] : n.xs[ox + 1], sym = FIX ? n.csy[oy + 1][ox + 1] : n.ys[oy + 1];
  const long long so = (long long)cj * P.pitch + ci;
  if constexpr (SIGNBIT) {
    // FP64 / FP32 paths: the sign bit flipped by integer work (no FP64
    // instruction; bitwise the same as negation), measured 6 % faster in FP64
    unsigned long long flip = ((n.neg[oy + 1][ox + 1] >> var) & 1) ? 1ull : 0ull;
    double v;
    if (kind == 0) {
      v = U[(long long)(var * 3) * P.plane + so];
    } else {
      if (MODE != REC_PLAIN && usemod && mask[(long long)cj * P.nx + ci] == 1)
        v = Mod[(long long)(var * 2 + kind - 1) * P.plane + so];
      else
        v = U[(long long)(var * 3 + kind) * P.plane + so];
      if (kind == 1 && sxm < 0) flip ^= 1ull;
      if (kind == 2 && sym < 0) flip ^= 1ull;
    }
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)(flip << 63));
  } else {
    // double-float path: plain negation (fewer registers there, measured faster)
    if (kind == 0) {
      const double u = U[(long long)(var * 3) * P.plane + so];
      return (n.neg[oy + 1][ox + 1] >> var) & 1 ? -u : u;
    }
    double v;
    if (MODE != REC_PLAIN && usemod && mask[(long long)cj * P.nx + ci] == 1)
      v = Mod[(long long)(var * 2 + kind - 1) * P.plane + so];
    else
      v = U[(long long)(var * 3 + kind) * P.plane + so];
    if (kind == 1 && sxm < 0) v = -v;
    if (kind == 2 && sym < 0) v = -v;
    return (n.neg[oy + 1][ox + 1] >> var) & 1 ? -v : v;
  }
}

// FP32 form: the moment from the float copy of the state the update kernel
// writes beside it (the state rounded to nearest), signs flipped by integer
// work; modified first moments of flagged cells still come from the FP64 copy.
template <int MODE>
__device__ __forceinline__ float load_mom32(const Prob& P, const float* __restrict__ U32,
                                            const uint8_t* __restrict__ mask, const double* __restrict__ Mod,
                                            const Nbr& n, int var, int kind, int ox, int oy, bool usemod) {
  const int ci = n.xi[ox + 1], cj = n.yj[oy + 1];
  const long long so = (long long)cj * P.pitch + ci;
  unsigned flip = (n.neg[oy + 1][ox + 1] >> var) & 1u;
  float v;
  if (kind == 0) {
    v = U32[(long long)(var * 3) * P.plane + so];
  } else {
    if (MODE != REC_PLAIN && usemod && mask[(long long)cj * P.nx + ci] == 1)
      v = float(Mod[(long long)(var * 2 + kind - 1) * P.plane + so]);
    else
      v = U32[(long long)(var * 3 + kind) * P.plane + so];
    if (kind == 1 && n.xs[ox + 1] < 0) flip ^= 1u;
    if (kind == 2 && n.ys[oy + 1] < 0) flip ^= 1u;
  }
  return __uint_as_float(__float_as_uint(v) ^ (flip << 31));
}

template <typename T, int NV, int MODE, bool FIX = false, bool S32 = false>
__device__ __forceinline__ void rec2d_cell(const Prob& P, const Weights<T>& W, const Beta2<T>& B,
                                           const double* __restrict__ U, const uint8_t* __restrict__ mask,
                                           const double* __restrict__ Mod, int i, int j, T* __restrict__ G,
                                           T* __restrict__ aux, const float* __restrict__ U32 = nullptr) {
  constexpr bool FLAGGED = MODE == REC_FLAGGED;
  const bool usemod = MODE == REC_FLAGGED || (MODE == REC_MIXED && mask[(long long)j * P.nx + i] == 1);
  const Nbr nb = neighbours<FIX>(P, i, j);
  const long long o = goff(P, i, j);
  // float copy, plain pass, all 3 x 3 cells inside the grid: no image to apply,
  // the moments are read at fixed offsets from the cell's own
  const bool inner = S32 && MODE == REC_PLAIN && i > 0 && i < P.nx - 1 && j > 0 && j < P.ny - 1;
  const float* __restrict__ Uc = S32 ? U32 + ((long long)j * P.pitch + i) : nullptr;
  T rinv[16];
  T pxl = T(0), pxr = T(0), pyb = T(0), pyt = T(0), nrm = T(0);
#pragma unroll 1
  for (int v = 0; v < NV; ++v) {
    T d[23];
    if (inner) {
#pragma unroll
      for (int c = 0; c < 23; ++c) {
        int kind, ox, oy;
        d4_slot(c, kind, ox, oy);
        d[c] = T(Uc[(long long)(v * 3 + kind) * P.plane + (long long)oy * P.pitch + ox]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 23; ++c) {
        int kind, ox, oy;
        d4_slot(c, kind, ox, oy);
        if constexpr (S32)
          d[c] = load_mom32<MODE>(P, U32, mask, Mod, nb, v, kind, ox, oy, usemod);
        else
          d[c] = from_double<T>(load_mom<MODE, !is_df64<T>::value, FIX>(P, U, mask, Mod, nb, v, kind, ox, oy, usemod));
      }
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
            batch_inverse_ranged<12, T>(x, r);
#pragma unroll
            for (int q = 0; q < 12; ++q) rinv[bp[q]] = r[q];
          } else {
#pragma unroll
            for (int q = 0; q < 12; ++q) rinv[bp[q]] = rcp(out[bp[q]]);
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

// rerec (REC_FLAGGED only, may be null) accumulates the number of cells
// reconstructed a second time.
// Double-float: 4 resident blocks per SM (at most 128 registers, a few spills)
// beat 3 (168 registers, none): 7.0 vs 8.3 ms per launch at 2048^2.  FP32 with
// the float copy: 8 blocks (64 registers, 164 B of spills) measured 0.545 ms per
// 2048^2 launch against 0.685 at 4 blocks (119 registers).  FP64 is pipe-bound:
// 2, 3 or 4 blocks run alike.
template <typename T, int NV, int MODE, bool FIX = false, bool S32 = false>
__global__ void __launch_bounds__(RB, (is_df64<T>::value ? 4 : (std::is_same<T, float>::value ? 8 : 1))) rec2d_kernel(Prob P, Weights<T> W, Beta2<T> B, const double* __restrict__ U,
                                                  const uint8_t* __restrict__ mask, const double* __restrict__ Mod,
                                                  const int* __restrict__ list, const int* __restrict__ count,
                                                  T* __restrict__ G, T* __restrict__ aux,
                                                  unsigned long long* __restrict__ rerec,
                                                  const float* __restrict__ U32 = nullptr) {
  constexpr bool FLAGGED = MODE == REC_FLAGGED;
  const long long ncell = (long long)P.nx * P.ny;
  const long long n = FLAGGED ? (long long)*count : ncell;
  if (FLAGGED && rerec && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(rerec, (unsigned long long)n);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int cell = FLAGGED ? list[t] : (int)t;
    if (FIX && is_solid(P, cell % P.nx, cell / P.nx)) continue;   // solid cells are images, never read
    rec2d_cell<T, NV, MODE, FIX, S32>(P, W, B, U, mask, Mod, cell % P.nx, cell / P.nx, G, aux, U32);
  }
}

// Step 2.1 for one cell: the troubled-cell decision of the configured indicator.
template <typename T>
__device__ __forceinline__ bool flag2d_cell(const Prob& P, const Weights<T>& W, const double* __restrict__ U,
                                            const T* __restrict__ G, const T* __restrict__ aux, int i, int j,
                                            double* __restrict__ aleph) {
  if (P.sol_j > 0 && is_solid(P, i, j)) {
    if (aleph) aleph[(long long)j * P.nx + i] = 0.0;
    return false;
  }
  if (P.indicator == IND_ALL) return true;
  if (P.indicator == IND_TVB) return tvb_cell(P, U, i, j);
  if (P.indicator != IND_KXRCF) return false;
  const T a = kxrcf2d<T>(P, W, G, aux, i, j);
  if (aleph) aleph[(long long)j * P.nx + i] = double(a);
  return a > T(1);
}

// Step 2.2 for one troubled cell (dimension by dimension): modified first
// moments from the pre-modification moments of the x and y neighbours.
template <int NV>
__device__ __forceinline__ void modify2d_cell(const Prob& P, const double* __restrict__ U, double* __restrict__ Mod,
                                              int i, int j) {
  const Img L = image(P, i - 1, j, i, j), R = image(P, i + 1, j, i, j), Bo = image(P, i, j - 1, i, j),
            Tp = image(P, i, j + 1, i, j);
  const long long o = (long long)j * P.pitch + i;
  // moment (kind 1: x, 2: y first moment) of an edge neighbour; a fixed-state
  // ghost has its state as average and zero first moments
  auto mom = [&](const Img& m, int v, int kind) -> double {
    if (m.fs >= 0) return kind == 0 ? fixed_val(P, m, v) : 0.0;
    const int g = vsign(m, v) * (kind == 1 ? m.sx : kind == 2 ? m.sy : 1);
    return g * U[sidx(P, v, kind, m.i, m.j)];
  };
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double uL = mom(L, v, 0), uR = mom(R, v, 0), vL = mom(L, v, 1), vR = mom(R, v, 1);
    const double uB = mom(Bo, v, 0), uT = mom(Tp, v, 0), wB = mom(Bo, v, 2), wT = mom(Tp, v, 2);
    Mod[(long long)(v * 2 + 0) * P.plane + o] = MOD_WU * (uR - uL) + MOD_WV * (vL + vR);
    Mod[(long long)(v * 2 + 1) * P.plane + o] = MOD_WU * (uT - uB) + MOD_WV * (wB + wT);
  }
}

// Warp-aggregated append of flagged entries to a list (all 32 lanes take part).
template <typename E>
__device__ __forceinline__ void warp_append(bool flag, E entry, E* __restrict__ list, int* __restrict__ count) {
  const unsigned act = __ballot_sync(0xffffffffu, flag);
  if (!act) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(act) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(act));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (flag) list[base + __popc(act & ((1u << lane) - 1u))] = entry;
}

template <typename T, int NV>
__global__ void __launch_bounds__(TX * TY) flag2d_kernel(Prob P, Weights<T> W, const double* __restrict__ U,
                                                        const T* __restrict__ G, const T* __restrict__ aux,
                                                        uint8_t* __restrict__ mask, double* __restrict__ Mod,
                                                        int* __restrict__ list, int* __restrict__ count,
                                                        double* __restrict__ aleph) {
  const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
  const bool valid = i < P.nx && j < P.ny;
  const bool flag = valid && flag2d_cell<T>(P, W, U, G, aux, i, j, aleph);
  warp_append<int>(flag, j * P.nx + i, list, count);   // a warp is one tile row
  if (!valid) return;
  mask[(long long)j * P.nx + i] = flag ? 1 : 0;
  if (flag) modify2d_cell<NV>(P, U, Mod, i, j);
}

// KXRCF for the cells the learned indicator left undecided (mask 2): the
// decision, eq. (vi) for the troubled ones and their list for Step 2.3.
template <typename T, int NV>
__global__ void __launch_bounds__(RB) fallback2d_kernel(Prob P, Weights<T> W, const double* __restrict__ U,
                                                       const T* __restrict__ G, const T* __restrict__ aux,
                                                       const int* __restrict__ und, const int* __restrict__ und_count,
                                                       uint8_t* __restrict__ mask, double* __restrict__ Mod,
                                                       int* __restrict__ list, int* __restrict__ count,
                                                       double* __restrict__ aleph) {
  const long long n = *und_count;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // warp-uniform trip count: every lane of a warp takes part in the append
  for (long long b = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < n; b += stride) {
    const long long t = b + (threadIdx.x & 31);
    bool flag = false;
    int cell = 0;
    if (t < n) {
      cell = und[t];
      const int i = cell % P.nx, j = cell / P.nx;
      const T a = kxrcf2d<T>(P, W, G, aux, i, j);
      if (aleph) aleph[cell] = double(a);
      flag = a > T(1);
      mask[cell] = flag ? 1 : 0;
      if (flag) modify2d_cell<NV>(P, U, Mod, i, j);
    }
    warp_append<int>(flag, cell, list, count);
  }
}

template <typename T, int NV>
__device__ __forceinline__ void gl_state(const Prob& P, const T* __restrict__ G, const Img& m, int k, int l, T (&u)[NV]) {
  if (m.fs >= 0) {   // fixed-state ghost: its state at every point
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = from_double<T>(fixed_val(P, m, v));
    return;
  }
  const long long o = goff(P, m.i, m.j);
  const int p = mpt(m, k, l);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const T x = G[(long long)(v * 16 + p) * P.gplane + o];
    u[v] = (m.neg >> v) & 1 ? -x : x;
  }
}

// The numerical flux of one face point, one inlined solver for both
// directions: a y face is an x face with the two momentum components
// exchanged (the HLLC expressions are the same, term for term); at a wall
// face the star branch is taken.
template <typename T, int NV>
__device__ __forceinline__ void face_flux(const Prob& P, T (&uL)[NV], T (&uR)[NV], bool xd, bool wall, T* out) {
  if constexpr (NV == 4) {
    if (!xd) {
      const T a = uL[1], b = uR[1];
      uL[1] = uL[2]; uL[2] = a;
      uR[1] = uR[2]; uR[2] = b;
    }
    T F[4];
    hllc<T, 4>(P, uL, uR, 0, F, wall);
    out[0] = F[0];
    out[1] = xd ? F[1] : F[2];
    out[2] = xd ? F[2] : F[1];
    out[3] = F[3];
  } else {
    num_flux<T, NV>(P, uL, uR, xd ? 0 : 1, out);
  }
}

struct Rk {
  const double* Uin; const double* Un; double* Uout;
  const uint8_t* mask; const double* Mod; const uint8_t* maskN; const double* ModN;
  double dt, cA, cB;
  double* Lout; double* Umod;
  unsigned* status;
  const double* dtp;     // dt on the device (overrides dt); < 0: skip, Uout = Uin
  float* U32out = nullptr;   // FP32 form: the float copy of Uout (the next stage's reconstruction input)
};

// Where update2d_tile reads point values and stage states: global memory (any
// tile) or, for an interior tile of the FP32 TMA kernel, the boxes staged in
// shared memory.  The arithmetic is the same template either way, so both give
// bitwise the same results.
template <typename T>
struct GlobalSrc {
  static constexpr bool staged = false;
  const T* __restrict__ G;
  __device__ __forceinline__ T g(const Prob& P, int v, int p, int i, int j) const {
    return G[(long long)(v * 16 + p) * P.gplane + goff(P, i, j)];
  }
  __device__ __forceinline__ double uin(const Prob& P, const Rk& S, int q, int i, int j) const {
    return S.Uin[(long long)q * P.plane + (long long)j * P.pitch + i];
  }
  __device__ __forceinline__ double un(const Prob& P, const Rk& S, int q, int i, int j) const {
    return S.Un[(long long)q * P.plane + (long long)j * P.pitch + i];
  }
};

// The TMA kernel's shared-memory box (FP32): the tile's own point values,
// [64 planes][4 rows][32 columns] from cell (i0, j0); the one-cell halo the face
// fluxes need and the stage states come from global memory.
constexpr int GBX = 32, GBY = 4;
struct StagedSrc {
  static constexpr bool staged = true;
  const float* gs;
  const float* __restrict__ G;
  int i0, j0;
  __device__ __forceinline__ float g(const Prob& P, int v, int p, int i, int j) const {
    const int x = i - i0, y = j - j0;
    if ((unsigned)x < (unsigned)GBX && (unsigned)y < (unsigned)GBY) return gs[((v * 16 + p) * GBY + y) * GBX + x];
    return G[(long long)(v * 16 + p) * P.gplane + goff(P, i, j)];
  }
  __device__ __forceinline__ double uin(const Prob& P, const Rk& S, int q, int i, int j) const {
    return S.Uin[(long long)q * P.plane + (long long)j * P.pitch + i];
  }
  __device__ __forceinline__ double un(const Prob& P, const Rk& S, int q, int i, int j) const {
    return S.Un[(long long)q * P.plane + (long long)j * P.pitch + i];
  }
};

// Step 3 for the TXV x TYV tile at (i0, j0): face fluxes into shared memory, then
// quadrature, L(U) and the Runge-Kutta combination per cell.  tid = ty*TXV + tx.
// SOLID: the handle may have a solid block (FP64 2D Euler only); without it the
// wall-face code is not compiled in (the batched kernel runs at the register limit).
template <typename T, int NV, int TXV, int TYV, bool SOLID = false, typename Src = GlobalSrc<T>>
__device__ __forceinline__ void update2d_tile(const Prob& P, const Src& src, const Rk& S, int i0, int j0,
                                              int tid, T (&xf)[TYV][TXV + 1][4][NV], T (&yf)[TYV + 1][TXV][4][NV]) {
  const int tx = tid % TXV, ty = tid / TXV;
  const int i = i0 + tx, j = j0 + ty;
  const bool live = i < P.nx && j < P.ny;
  // Every face flux of the tile at one Gauss-Lobatto point per iteration, by one
  // call site, so that a face shared by two tiles gets bitwise the same flux
  // from both (the flux differences then telescope exactly in FP64).
  // xf[r][c] is the face left of cell (i0 + c, j0 + r); yf[r][c] the face below it.
  constexpr int NXP = (TXV + 1) * TYV * 4, NYP = TXV * (TYV + 1) * 4;
  // a tile whose faces all join cells inside the grid (no image, no solid cell):
  // the point values at fixed offsets
  const bool tin = Src::staged || ((!SOLID || P.sol_j == 0) && i0 >= 1 && i0 + TXV < P.nx && j0 >= 1 && j0 + TYV < P.ny);
  __syncthreads();   // the shared arrays may still be read for a previous tile
  for (int f = tid; f < NXP + NYP; f += TXV * TYV) {
    // the face's GL point q, its slot (c, r) in the tile, its two cells a
    // (left / below) and b (right / above) and their point indices
    const bool xd = f < NXP;
    const int g = xd ? f : f - NXP, q = g & 3, face = g >> 2;
    const int c = xd ? face % (TXV + 1) : face % TXV, r = xd ? face / (TXV + 1) : face / TXV;
    const int aI = xd ? i0 + c - 1 : i0 + c, aJ = xd ? j0 + r : j0 + r - 1;
    const int bI = xd ? aI + 1 : aI, bJ = xd ? aJ : aJ + 1;
    const int ka = xd ? 3 : q, la = xd ? q : 3, kb = xd ? 0 : q, lb = xd ? q : 0;
    T uL[NV], uR[NV];
    bool wall = false;
    if (tin) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        uL[v] = src.g(P, v, ka * 4 + la, aI, aJ);
        uR[v] = src.g(P, v, kb * 4 + lb, bI, bJ);
      }
    } else if constexpr (!Src::staged) {
      const T* __restrict__ G = src.G;
      if (aJ >= P.ny || aI >= P.nx) continue;
      const bool sa = SOLID && P.sol_j > 0 && is_solid(P, aI, aJ), sb = SOLID && P.sol_j > 0 && is_solid(P, bI, bJ);
      // a face no fluid cell uses (solid on one side, solid or outside on the
      // other) is skipped: only solid cells would read it, and they are not updated
      if (SOLID && P.sol_j > 0 && (sa || aI < 0 || aJ < 0) && (sb || bI >= P.nx || bJ >= P.ny)) continue;
      if (!sa) gl_state<T, NV>(P, G, image(P, aI, aJ), ka, la, uL);
      if (!sb) gl_state<T, NV>(P, G, image(P, bI, bJ), kb, lb, uR);
      // a face shared with a solid cell: the outer state is the reflection of
      // the fluid side's own (the wall-normal momentum negated)
      const int wn = xd ? 1 : 2;
      if (sb && !sa) {
#pragma unroll
        for (int v = 0; v < NV; ++v) uR[v] = v == wn ? -uL[v] : uL[v];
      }
      if (sa && !sb) {
#pragma unroll
        for (int v = 0; v < NV; ++v) uL[v] = v == wn ? -uR[v] : uR[v];
      }
      wall = sa || sb;
    }
    face_flux<T, NV>(P, uL, uR, xd, wall, xd ? xf[r][c][q] : yf[r][c][q]);
  }
  __syncthreads();
  if (!live) return;
  if (SOLID && P.sol_j > 0 && is_solid(P, i, j)) {   // solid cells are not updated: the state passes through
    if (!S.Lout) {
#pragma unroll 1
      for (int q = 0; q < NV * 3; ++q) {
        const long long si = (long long)q * P.plane + (long long)j * P.pitch + i;
        S.Uout[si] = S.Uin[si];
        if (S.U32out) S.U32out[si] = f32_rn(S.Uin[si]);
      }
    } else {
#pragma unroll 1
      for (int q = 0; q < NV * 3; ++q) {
        const long long si = (long long)q * P.plane + (long long)j * P.pitch + i;
        S.Lout[si] = 0.0;
        if (S.Umod) S.Umod[si] = S.Uin[si];
      }
    }
    return;
  }
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
    for (int p = 0; p < 16; ++p) rho[p] = src.g(P, 0, p, i, j);
    batch_inverse_ranged<16, T>(rho, inv);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        T u[NV], fx[NV], gy[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = src.g(P, v, k * 4 + l, i, j);
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
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = src.g(P, v, k * 4 + l, i, j);
        phys_flux<T, NV>(P, u, 0, fx);
        phys_flux<T, NV>(P, u, 1, gy);
        const T w = gl_w<T>(k) * gl_w<T>(l);
#pragma unroll
        for (int v = 0; v < NV; ++v) { Fc[v] += w * fx[v]; Gc[v] += w * gy[v]; }
      }
  }
  // eq. (2D-equ-int-approximation); the average equation in FP64 from the
  // face integrals so that the flux differences telescope in every precision
  // (FP32 values widened by integer work: the FP64 pipe keeps only the sums)
  const double idx = P.crdx.d, idy = P.crdy.d;
  const T tidx = pc<T>(P.crdx), tidy = pc<T>(P.crdy);
  const long long so = (long long)j * P.pitch + i;
  const long long cell = (long long)j * P.nx + i;
  // modified first moments in the combination (persist), and always in the Umod output of Lout
  const bool fk = S.mask[cell] != 0 && (P.persist || S.Lout);
  const bool fn = P.persist && S.maskN && S.maskN[cell] != 0;
  // the first stage has no U^n term (cA = 0, cB = 1): U^(1) = U' + dt L
  const bool first = S.cA == 0.0;
  const bool owned = j >= P.jlo && j < P.jhi;
  double newavg[NV];
  bool finite = true;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double L[3];
    L[0] = -(to_f64(Fp[v]) - to_f64(Fm[v])) * idx - (to_f64(Gp[v]) - to_f64(Gm[v])) * idy;
    L[1] = to_f64(-(Fp[v] + Fm[v]) * T(0.5) * tidx + Fc[v] * tidx - (Gpx[v] - Gmx[v]) * tidy);
    L[2] = to_f64(-(Fpe[v] - Fme[v]) * tidx - (Gp[v] + Gm[v]) * T(0.5) * tidy + Gc[v] * tidy);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const long long si = (long long)(v * 3 + m) * P.plane + so;
      const double uin = (m > 0 && fk) ? S.Mod[(long long)(v * 2 + m - 1) * P.plane + so] : src.uin(P, S, v * 3 + m, i, j);
      if (S.Lout) {
        S.Lout[si] = L[m];
        if (S.Umod) S.Umod[si] = uin;
        continue;
      }
      double r;
      if (first) {
        r = fma(S.dt, L[m], uin);
      } else {
        const double un = (m > 0 && fn) ? S.ModN[(long long)(v * 2 + m - 1) * P.plane + so] : src.un(P, S, v * 3 + m, i, j);
        r = S.cA * un + S.cB * (uin + S.dt * L[m]);
      }
      S.Uout[si] = r;
      if (S.U32out) S.U32out[si] = f32_rn(r);
      if (m == 0) newavg[v] = r;
      // non-finite by the exponent field (integer work, no FP64 compare)
      finite = finite && ((__double_as_longlong(r) >> 52) & 0x7FF) != 0x7FF;
    }
  }
  if (!S.Lout && !finite && owned) atomicOr(S.status, ST_NONFINITE);
  if (!S.Lout && P.eq == EQ_EULER && NV == 4 && owned) {
    // rho > 0 and p = (gamma - 1)(E - |m|^2 / (2 rho)) > 0, the latter as 2 E rho > |m|^2 (no division)
    const double rho = newavg[0];
    const double m2 = newavg[1] * newavg[1] + newavg[2] * newavg[2];
    if (!(rho > 0.0) || !(2.0 * newavg[NV - 1] * rho > m2)) atomicOr(S.status, ST_NONPOSITIVE);
  }
}

template <typename T, int NV, bool SOLID = false>
__global__ void __launch_bounds__(TX * TY, (std::is_same<T, float>::value ? 8 : 3)) update2d_kernel(Prob P, const T* __restrict__ G, Rk S) {
  __shared__ T xf[TY][TX + 1][4][NV];
  __shared__ T yf[TY + 1][TX][4][NV];
  if (S.dtp) {
    S.dt = *S.dtp;
    if (S.dt < 0.0) {   // a skipped step (block-uniform): the state passes through unchanged
      const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
      if (i < P.nx && j < P.ny && !S.Lout)
        for (int q = 0; q < NV * 3; ++q) {
          const long long si = (long long)q * P.plane + (long long)j * P.pitch + i;
          S.Uout[si] = S.Uin[si];
          if (S.U32out) S.U32out[si] = f32_rn(S.Uin[si]);
        }
      return;
    }
  }
  update2d_tile<T, NV, TX, TY, SOLID>(P, GlobalSrc<T>{G}, S, blockIdx.x * TX, blockIdx.y * TY,
                                      threadIdx.y * TX + threadIdx.x, xf, yf);
}

// ---------------------------------------------------------------- TMA-staged update (FP32 form)
// An interior tile loads its own point values (a 32 x 4 x 64-plane box from
// cell (i0, j0), 32 KB) with one cp.async.bulk.tensor into shared memory,
// completing on an mbarrier; the halo points and the stage states come from
// global memory, and tiles at the grid's edges take the global-memory path
// (boundary images).  An option (hweno_set_tma): with 52 KB of shared memory a
// block, 4 blocks fit an SM against the global kernel's 8, and the global
// kernel measured faster (1.07 against 1.46 ms per 2048^2 launch; a 40 x 6 box
// with the halo and both stage states in shared memory, 2 blocks per SM: 1.63).
constexpr unsigned GBOX_BYTES = GBX * GBY * 64 * 4;
constexpr unsigned TMA_SMEM = GBOX_BYTES + 128;
constexpr unsigned long long MBAR_POLL_LIMIT = 1ull << 22;
static_assert(GBX == TX && GBY == TY, "the box covers one update tile");

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_load3d(void* dst, const CUtensorMap* map, int x, int y, int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      :: "r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(bar) : "memory");
}

// Phase `parity` of the mbarrier at `bar` completed; at most `limit` polls, false if the wait gave up.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, unsigned long long limit) {
  for (unsigned long long k = 0; k < limit; ++k) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(TX * TY, 4) update2d_tma_kernel(Prob P, const float* __restrict__ G, Rk S,
                                                                  const __grid_constant__ CUtensorMap tmG) {
  __shared__ float xf[TY][TX + 1][4][4];
  __shared__ float yf[TY + 1][TX][4][4];
  extern __shared__ __align__(128) unsigned char dsm[];
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  if (S.dtp) {
    S.dt = *S.dtp;
    if (S.dt < 0.0) {   // a skipped step (block-uniform): the state passes through unchanged
      const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
      if (i < P.nx && j < P.ny)
        for (int q = 0; q < 12; ++q) {
          const long long si = (long long)q * P.plane + (long long)j * P.pitch + i;
          S.Uout[si] = S.Uin[si];
          if (S.U32out) S.U32out[si] = f32_rn(S.Uin[si]);
        }
      return;
    }
  }
  if (!(i0 >= 1 && i0 + TX < P.nx && j0 >= 1 && j0 + TY < P.ny)) {
    update2d_tile<float, 4, TX, TY>(P, GlobalSrc<float>{G}, S, i0, j0, tid, xf, yf);
    return;
  }
  float* gs = reinterpret_cast<float*>(dsm);
  const unsigned bar = smem_u32(dsm + GBOX_BYTES);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(GBOX_BYTES) : "memory");
    tma_load3d(gs, &tmG, i0, j0, 0, bar);   // i0 is a multiple of 32 floats (16-byte aligned)
  }
  if (!mbar_wait(bar, 0, MBAR_POLL_LIMIT)) {
    // gave up: report, wait (bounded) for the copies still in flight, skip the tile
    if (tid == 0) atomicOr(S.status, ST_TIMEOUT);
    mbar_wait(bar, 0, MBAR_POLL_LIMIT);
    return;
  }
  update2d_tile<float, 4, TX, TY, false, StagedSrc>(P, StagedSrc{gs, G, i0, j0}, S, i0, j0, tid, xf, yf);
}

// The TMA update kernel needs more than 48 KB of dynamic shared memory.
[[maybe_unused]] bool set_update_tma_attribute() {
  return cudaFuncSetAttribute(update2d_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TMA_SMEM) ==
         cudaSuccess;
}

}  // namespace
}  // namespace hw

#include "hweno_fused.cuh"

namespace hw {
namespace {

// Fixed-state ghosts are supported for 2D Euler in FP64 (the library rejects
// other combinations), so only that instantiation carries the FIX variant.
template <typename T, int NV, int MODE>
void launch_rec2d(int blocks, cudaStream_t st, const Prob& P, const Weights<T>& W, const Beta2<T>& Bt,
                  const double* U, const uint8_t* mask, const double* Mod, const int* list, const int* count, T* G,
                  T* aux, unsigned long long* rerec, const float* U32 = nullptr) {
  if constexpr (std::is_same<T, float>::value) {
    if (U32) {   // FP32 form with the float copy of the state: no per-moment conversion
      rec2d_kernel<T, NV, MODE, false, true><<<blocks, RB, 0, st>>>(P, W, Bt, U, mask, Mod, list, count, G, aux,
                                                                    rerec, U32);
      return;
    }
  }
  if constexpr (NV == 4 && std::is_same<T, double>::value) {
    if (P.fixtab || P.sol_j > 0) {
      rec2d_kernel<T, NV, MODE, true><<<blocks, RB, 0, st>>>(P, W, Bt, U, mask, Mod, list, count, G, aux, rerec);
      return;
    }
  }
  rec2d_kernel<T, NV, MODE><<<blocks, RB, 0, st>>>(P, W, Bt, U, mask, Mod, list, count, G, aux, rerec);
}

template <typename T, int NV>
void stage_t(const Prob& P, const HostTabs& HT, const Weights<T>& W, const Beta2<T>& Bt, const Bufs& B,
             const StageCall& S, cudaStream_t st) {
  if constexpr (NV == 4) {
    if (fused_applies(P, NV)) {   // the whole stage in one launch
      Rk r{S.Uin, S.Un, S.Uout, S.mask, S.Mod, S.maskN, S.ModN, S.dt, S.cA, S.cB, S.Lout, S.Umod, B.status, S.dtp};
      FzOut o{S.mask, S.Mod, S.aleph, B.rerec};
      if (B.prof) B.prof->begin(5, st);
      launch_fused2d<T>(P, W, Bt, r, o, st);
      if (B.prof) B.prof->end(st);
      return;
    }
  }
  const long long ncell = (long long)P.nx * P.ny;
  int* cnt = B.count + S.stage;
  cudaMemsetAsync(cnt, 0, sizeof(int), st);
  const int rblocks = (int)((ncell + RB - 1) / RB);
  const int fblocks = (int)std::min<long long>(rblocks, (long long)P.nsm * 8);
  const dim3 blk(TX, TY), grd((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
  if (NV == 4 && P.indicator == IND_MLP) {
    // Learned indicator first (moments only): confident cells are decided and
    // modified before Step 1, which then reconstructs them from the modified
    // moments; KXRCF decides the rest from the Step-1 point values, and only
    // the cells it flags are reconstructed again.
    int* ucnt = B.und_count + S.stage;
    cudaMemsetAsync(ucnt, 0, sizeof(int), st);
    if (B.prof) B.prof->begin(4, st);
    run_mlpre2d(P, B.mlp, B.mlp_conf, S.Uin, S.mask, S.Mod, B.und, ucnt, B.mlp_stats, B.mlp_prob, st);
    if (B.prof) B.prof->end(st);
    if (B.prof) B.prof->begin(0, st);
    rec2d_kernel<T, NV, REC_MIXED><<<rblocks, RB, 0, st>>>(P, W, Bt, S.Uin, S.mask, S.Mod, nullptr, nullptr,
                                                           (T*)B.G, (T*)B.aux, nullptr);
    if (B.prof) B.prof->end(st);
    if (B.prof) B.prof->begin(1, st);
    fallback2d_kernel<T, NV><<<fblocks, RB, 0, st>>>(P, W, S.Uin, (const T*)B.G, (const T*)B.aux, B.und, ucnt,
                                                     S.mask, S.Mod, B.list, cnt, S.aleph);
    if (B.prof) B.prof->end(st);
  } else {
    if (B.prof) B.prof->begin(0, st);
    launch_rec2d<T, NV, REC_PLAIN>(rblocks, st, P, W, Bt, S.Uin, nullptr, nullptr, nullptr, nullptr, (T*)B.G,
                                   (T*)B.aux, nullptr, S.U32in);
    if (B.prof) B.prof->end(st);
    if (B.prof) B.prof->begin(1, st);
    flag2d_kernel<T, NV><<<grd, blk, 0, st>>>(P, W, S.Uin, (const T*)B.G, (const T*)B.aux, S.mask, S.Mod, B.list,
                                              cnt, S.aleph);
    if (B.prof) B.prof->end(st);
  }
  if (P.indicator != IND_NONE) {
    if (B.prof) B.prof->begin(2, st);
    launch_rec2d<T, NV, REC_FLAGGED>(fblocks, st, P, W, Bt, S.Uin, S.mask, S.Mod, B.list, cnt, (T*)B.G, nullptr,
                                     B.rerec, S.U32in);
    if (B.prof) B.prof->end(st);
  }
  Rk r{S.Uin, S.Un, S.Uout, S.mask, S.Mod, S.maskN, S.ModN, S.dt, S.cA, S.cB, S.Lout, S.Umod, B.status, S.dtp,
       std::is_same<T, float>::value ? S.U32out : nullptr};
  if (B.prof) B.prof->begin(3, st);
  if constexpr (NV == 4 && std::is_same<T, double>::value) {
    if (P.sol_j > 0) update2d_kernel<T, NV, true><<<grd, blk, 0, st>>>(P, (const T*)B.G, r);
    else update2d_kernel<T, NV><<<grd, blk, 0, st>>>(P, (const T*)B.G, r);
  } else if constexpr (NV == 4 && std::is_same<T, float>::value) {
    if (B.tmG && !S.Lout)
      update2d_tma_kernel<<<grd, blk, TMA_SMEM, st>>>(P, (const float*)B.G, r, *B.tmG);
    else
      update2d_kernel<T, NV><<<grd, blk, 0, st>>>(P, (const T*)B.G, r);
  } else {
    update2d_kernel<T, NV><<<grd, blk, 0, st>>>(P, (const T*)B.G, r);
  }
  if (B.prof) B.prof->end(st);
}

// ---------------------------------------------------------------- batched problems
//
// One persistent cooperative launch per Runge-Kutta stage advances every problem
// of a batch.  Work items of all problems form one list per phase (128-cell rows
// for the per-cell phases, update tiles for the flux phase); the resident blocks
// stride over it.  Phases are separated by a grid barrier whose wait is bounded:
// past the limit the block records ST_TIMEOUT and continues (the host reports
// HWENO_ETIMEOUT), so no wait can hang the GPU.

// nblocks: arrivals that release the barrier; limit: polls before the wait gives up.
__device__ __forceinline__ void grid_barrier(unsigned* bar, unsigned nblocks, unsigned* status,
                                             unsigned long long limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long spins = 0;
      while (*vgen == gen) {
        if (++spins > limit) {
          atomicOr(status, ST_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// problem owning work item it (first[] ascending)
template <int FIELD>
__device__ __forceinline__ int owner(const BProb* __restrict__ probs, int n, int it) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int f = FIELD == 0 ? probs[mid].rec_first : probs[mid].upd_first;
    if (f <= it) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T, int TXV, int TYV>
__global__ void __launch_bounds__(TXV * TYV) batch_stage_kernel(BatchStage A, Weights<T> W, Beta2<T> B) {
  static_assert(TXV * TYV == RB, "tiles and rows use the same block");
  __shared__ T xf[TYV][TXV + 1][4][4];
  __shared__ T yf[TYV + 1][TXV][4][4];
  const int tid = threadIdx.x;
  const unsigned nb = gridDim.x;
  T* G = (T*)A.G;
  T* aux = (T*)A.aux;
  // CFL wave speeds of U^n (first stage, when the caller gives no dt)
  if (A.stage == 0 && !A.dt_in) {
    for (int it = blockIdx.x; it < A.n_rec; it += nb) {
      const int p = owner<0>(A.probs, A.nprob, it);
      const Prob P = A.probs[p].P;
      const double* U = A.Uin + A.probs[p].uoff;
      const int cell = (it - A.probs[p].rec_first) * RB + tid;
      double sx = 0.0, sy = 0.0;
      if (cell < P.nx * P.ny) {
        const int i = cell % P.nx, j = cell / P.nx;
        const double rho = U[sidx(P, 0, 0, i, j)];
        const double mu = U[sidx(P, 1, 0, i, j)] / rho, nu = U[sidx(P, 2, 0, i, j)] / rho;
        const double pr = (P.gamma - 1.0) * (U[sidx(P, 3, 0, i, j)] - 0.5 * rho * (mu * mu + nu * nu));
        cell_speeds(P, rho, mu, nu, pr, sx, sy);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sx = fmax(sx, __shfl_down_sync(0xffffffffu, sx, o));
        sy = fmax(sy, __shfl_down_sync(0xffffffffu, sy, o));
      }
      if ((tid & 31) == 0) {   // non-negative doubles order like their bit patterns
        atomicMax(A.speeds + 2 * p, (unsigned long long)__double_as_longlong(sx));
        atomicMax(A.speeds + 2 * p + 1, (unsigned long long)__double_as_longlong(sy));
      }
    }
    grid_barrier(A.bar, nb + A.bar_extra, A.status, A.spin_limit);
  }
  // Step 1: every cell
  for (int it = blockIdx.x; it < A.n_rec; it += nb) {
    const int p = owner<0>(A.probs, A.nprob, it);
    const BProb& Q = A.probs[p];
    const int cell = (it - Q.rec_first) * RB + tid;
    if (cell < Q.P.nx * Q.P.ny)
      rec2d_cell<T, 4, REC_PLAIN>(Q.P, W, B, A.Uin + Q.uoff, nullptr, nullptr, cell % Q.P.nx, cell / Q.P.nx, G + Q.goff,
                              aux + Q.aoff);
  }
  grid_barrier(A.bar, nb + A.bar_extra, A.status, A.spin_limit);
  // Steps 2.1-2.2
  for (int it = blockIdx.x; it < A.n_rec; it += nb) {
    const int p = owner<0>(A.probs, A.nprob, it);
    const BProb& Q = A.probs[p];
    const int cell = (it - Q.rec_first) * RB + tid;
    const bool valid = cell < Q.P.nx * Q.P.ny;
    const int i = cell % Q.P.nx, j = cell / Q.P.nx;
    const bool flag = valid && flag2d_cell<T>(Q.P, W, A.Uin + Q.uoff, G + Q.goff, aux + Q.aoff, i, j, nullptr);
    warp_append<unsigned long long>(flag, ((unsigned long long)p << 32) | (unsigned)cell, A.list, A.count);
    if (valid) {
      A.mask[Q.coff + cell] = flag ? 1 : 0;
      if (flag) modify2d_cell<4>(Q.P, A.Uin + Q.uoff, A.Mod + Q.moff, i, j);
    }
  }
  grid_barrier(A.bar, nb + A.bar_extra, A.status, A.spin_limit);
  // Step 2.3: troubled cells
  {
    const int n = *(volatile int*)A.count;
    for (int t = blockIdx.x * RB + tid; t < n; t += nb * RB) {
      const unsigned long long e = A.list[t];
      const int p = (int)(e >> 32), cell = (int)(e & 0xffffffffu);
      // after a barrier wait that gave up, an entry may not be written yet
      if (p < 0 || p >= A.nprob || cell < 0 || cell >= A.probs[p].P.nx * A.probs[p].P.ny) continue;
      const BProb& Q = A.probs[p];
      rec2d_cell<T, 4, REC_FLAGGED>(Q.P, W, B, A.Uin + Q.uoff, A.mask + Q.coff, A.Mod + Q.moff, cell % Q.P.nx,
                             cell / Q.P.nx, G + Q.goff, nullptr);
    }
  }
  grid_barrier(A.bar, nb + A.bar_extra, A.status, A.spin_limit);
  // Step 3: fluxes, quadrature, L, Runge-Kutta
  for (int it = blockIdx.x; it < A.n_upd; it += nb) {
    const int p = owner<1>(A.probs, A.nprob, it);
    const BProb& Q = A.probs[p];
    double dt;
    if (A.dt_in) {
      dt = A.dt_in[p];
    } else {
      const double ax = __longlong_as_double((long long)A.speeds[2 * p]);
      const double ay = __longlong_as_double((long long)A.speeds[2 * p + 1]);
      const double r = ax / Q.P.dx + ay / Q.P.dy;
      dt = (r > 0.0 && isfinite(r)) ? A.cfl / r : 0.0;
    }
    const int t = it - Q.upd_first;
    if (A.stage == 0 && t == 0 && tid == 0) A.dt_out[p] = dt;
    Rk S{A.Uin + Q.uoff, A.Un + Q.uoff, A.Uout + Q.uoff, A.mask + Q.coff, A.Mod + Q.moff,
         A.maskN ? A.maskN + Q.coff : nullptr, A.ModN ? A.ModN + Q.moff : nullptr, dt, A.cA, A.cB,
         nullptr, nullptr, A.pstatus + p};
    update2d_tile<T, 4, TXV, TYV>(Q.P, GlobalSrc<T>{G + Q.goff}, S, (t % Q.tiles_x) * TXV, (t / Q.tiles_x) * TYV, tid,
                                  xf, yf);
  }
}

template <typename T, int TXV, int TYV>
cudaError_t launch_batch(const Weights<T>& W, const Beta2<T>& Bt, const BatchStage& S, int nsm, cudaStream_t st) {
  auto kern = batch_stage_kernel<T, TXV, TYV>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RB, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nsm * per_sm);
  cfg.blockDim = dim3(RB);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, S, W, Bt);
}

}  // namespace
}  // namespace hw
