// Device-side building blocks of the HWENO stage kernels (sm_103a).
//
// Scheme: moment-based multi-resolution HWENO, Li, Shu & Qiu (arXiv 2201.12193).
// Section and equation names below are the paper's.
//
// Precision: T = double (FP64 path), float (FP32-bulk path) or df64 (double-float
// path, df64.cuh).  The state, the Runge-Kutta combination and the conservation
// sums stay FP64 in all three.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "hweno_parity.h"
#include "df64.cuh"

namespace hw {

constexpr int EQ_ADV = 0, EQ_BURGERS = 1, EQ_EULER = 2;
constexpr int BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2;
constexpr int IND_NONE = 0, IND_KXRCF = 1, IND_ALL = 2, IND_MLP = 3, IND_TVB = 4;

// device status word bits
constexpr unsigned ST_NONFINITE = 1u;     // a non-finite value in the new state
constexpr unsigned ST_NONPOSITIVE = 2u;   // rho <= 0 or p <= 0 in a new cell average (Euler)
constexpr unsigned ST_NODT = 8u;          // no CFL step length (rho <= 0 or a non-finite wave speed)

// A problem constant in the three compute precisions, converted once on the
// host (the same roundings as the device conversions: float by round to
// nearest, double-float as the nearest float plus the nearest float of the
// rest), so kernels do not spend FP64 instructions converting it per use.
struct PConst {
  double d;
  float f;
  df64 x;
};
template <typename T> __device__ __forceinline__ T pc(const PConst& c);
template <> __device__ __forceinline__ double pc<double>(const PConst& c) { return c.d; }
template <> __device__ __forceinline__ float pc<float>(const PConst& c) { return c.f; }
template <> __device__ __forceinline__ df64 pc<df64>(const PConst& c) { return c.x; }

// Problem description passed by value to every kernel.
struct Prob {
  int nx, ny;             // cells (ny = 1 in 1D)
  int pitch;              // row stride of the state arrays (doubles)
  long long plane;        // stride of one (variable, moment) plane = ny * pitch
  int gpitch;             // row stride of the point-value / aux arrays (elements of T)
  long long gplane;       // ny * gpitch
  int nvar, nmom;         // conserved variables; moments per variable (2 in 1D, 3 in 2D)
  int eq, indicator;
  int bc[4];              // x-lo, x-hi, y-lo, y-hi
  double dx, dy;
  double gamma;           // ratio of specific heats
  double adv_a, adv_b;    // linear advection speeds
  int nsm;                // multiprocessors of the device (grid sizing)
  double tvb_m;           // TVB constant M (indicator IND_TVB)
  int charwise;           // 1D Euler: reconstruction in local characteristic variables
  int positivity;         // 1: rho <= 0 or p <= 0 averages are non-physical; 0: p is
                          //    clamped at 0 in the sound speed (only rho <= 0 / non-finite fail)
  const double* fixtab;   // fixed-state ghost cells (inflow; 2D Euler): [side][pos + 1][4] conserved
                          //    states for ghost positions pos in [-1, n] along each side, rho = 0
                          //    where the side's kind applies instead; null: no fixed-state side
  int fixlen;             // entries per side of fixtab
  int persist;            // 1: the first moments modified in troubled cells (eq. (vi)) replace the
                          //    stage input and enter the Runge-Kutta combination; 0: they serve
                          //    L only and the combination takes the stage states as they entered
  int fused;              // one fused kernel per stage (1D default; 2D Euler option) instead of the pipeline
  PConst cgamma, cdx, cdy, crdx, crdy, cdx2;   // gamma, dx, dy, 1/dx, 1/dy, dx^2
  PConst cgm1, chk;   // gamma - 1 and (gamma + 1) / (2 gamma) of eq. (COEF)
  int sol_i, sol_j;       // solid block (2D Euler, the forward step): cells i >= sol_i, j < sol_j;
                          //    sol_j = 0: none
  int jlo, jhi;           // owned rows [jlo, jhi): the rows a row-slab of a decomposed grid owns (the
                          //    others are halo rows refilled from the neighbours before each stage);
                          //    only they enter the status checks, the CFL reduction and the totals
};

// Sound speed of a cell average for the CFL rule; +inf marks a non-physical
// average (dt = 0, the host reports it).
__device__ __forceinline__ void cell_speeds(const Prob& P, double rho, double mu, double nu, double p, double& sx,
                                            double& sy) {
  const double c = sqrt(P.gamma * (P.positivity ? p : fmax(p, 0.0)) / rho);
  sx = fabs(mu) + c;
  sy = fabs(nu) + c;
  if (!(rho > 0.0) || (P.positivity && !(p > 0.0)) || !isfinite(sx + sy)) sx = sy = INFINITY;
}

// Linear-weight data of eq. (linear-weight) and eq. (p) for positive gbar[4]:
// gamma_{l,4} = g_l / S_4 and p_l = (S_l q_l - S_{l-1} q_{l-1}) / g_l.
template <typename T>
struct Weights {
  T gam[4];      // gamma_{l,4}
  T sg[4];       // S_l / g_l
  T s1g[4];      // S_{l-1} / g_l  (0 for l = 1)
  T eps;         // 1e-10 of eqs. (w1_-LR), (non-linear-weight)
};

// Rows of the smoothness indicators beta_2..beta_4 for the run-time weights,
// in the flat parity-basis order of hweno_parity.h: beta_l = sum_rows (row . s)^2
// with row = (S_l/g_l) R C_l - (S_{l-1}/g_l) R C_{l-1}  (eq. (beta), (2D-beta), (p)).
template <typename T> struct Beta1 { T B2[hwp::D1_NB2]; T B3[hwp::D1_NB3]; T B4[hwp::D1_NB4]; };
template <typename T> struct Beta2 { T B2[hwp::D2_NB2]; T B3[hwp::D2_NB3]; T B4[hwp::D2_NB4]; };

// Gauss-Lobatto nodes and weights of eq. (F)
template <typename T> __device__ __forceinline__ T gl_w(int k) { return (k == 0 || k == 3) ? T(1.0 / 12.0) : T(5.0 / 12.0); }
template <typename T> __device__ __forceinline__ T gl_x(int k) {
  return k == 0 ? T(-0.5) : k == 1 ? T(-0.22360679774997896964) : k == 2 ? T(0.22360679774997896964) : T(0.5);
}

template <typename T> __device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }
template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

// ---------------------------------------------------------------- boundary images
// A ghost cell is the image of an interior cell: periodic wrap, or (transmissive)
// the mirror about the boundary face, under which the mirrored direction's first
// moment changes sign and point values are reversed along that direction.
// A reflective boundary (a solid wall, Euler only) is the transmissive mirror
// with the wall-normal momentum negated as well (all its moments and point
// values): neg has bit v set for each variable v the image negates
// (variable 1 = x momentum, 2 = y momentum in 2D).
// A fixed-state ghost (inflow, the post-shock boundaries of the double Mach
// reflection) holds a constant state, entry fs of Prob::fixtab: that average,
// zero first moments, the same value at every Gauss-Lobatto point, never
// troubled.  Corners take the y rule on the cell the x rule gives (ghost
// columns first, then ghost rows over all columns): a fixed y ghost wins, and
// the y mirror of a fixed x ghost negates its y momentum at a wall.
struct Img { int i, j, sx, sy, neg, fs; };

__device__ __forceinline__ int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

// Solid block of the forward-facing step (Example 3.10): in-domain cells with
// i >= sol_i and j < sol_j.
__device__ __forceinline__ bool is_solid(const Prob& P, int i, int j) {
  return P.sol_j > 0 && i >= P.sol_i && i < P.nx && j >= 0 && j < P.sol_j;
}

// The block's faces are reflective walls: a solid cell in the stencil of the
// fluid cell (vi, vj) is that cell's wall image, mirrored across the vertical
// face when the viewer lies left of it (vi < sol_i), across the horizontal
// face when the viewer lies above it (vj >= sol_j), across both (a point
// reflection through the corner) for the one viewer diagonal to the corner;
// each crossed face negates its wall-normal momentum and its normal first
// moment.  The image depends on the viewer (the corner cell seen from its left
// neighbour is that neighbour's x mirror, from above the y mirror of the cell
// above it).
__device__ __forceinline__ void solid_image(const Prob& P, int vi, int vj, Img& r) {
  if (r.fs >= 0 || !is_solid(P, r.i, r.j)) return;
  if (vi < P.sol_i) { r.i = 2 * P.sol_i - 1 - r.i; r.sx = -r.sx; r.neg ^= 2; }
  if (vj >= P.sol_j) { r.j = 2 * P.sol_j - 1 - r.j; r.sy = -r.sy; r.neg ^= 4; }
}

// The image of cell (i, j) by the boundary sides alone (a cell of the solid
// block maps to itself; callers that can meet one use the viewer form below).
__device__ __forceinline__ Img image(const Prob& P, int i, int j) {
  Img r{i, j, 1, 1, 0, -1};
  if (j < 0 || j >= P.ny) {
    const int side = j < 0 ? 2 : 3;
    if (P.fixtab) {
      const int e = side * P.fixlen + i + 1;
      if (P.fixtab[4 * e] > 0.0) { r.fs = e; return r; }
    }
    const int k = P.bc[side];
    if (k == BC_PERIODIC) r.j = wrap(j, P.ny);
    else { r.j = j < 0 ? -1 - j : 2 * P.ny - 1 - j; r.sy = -1; if (k == BC_REFLECTIVE) r.neg |= 4; }
  }
  if (i < 0 || i >= P.nx) {
    const int side = i < 0 ? 0 : 1;
    if (P.fixtab) {
      const int e = side * P.fixlen + r.j + 1;
      if (P.fixtab[4 * e] > 0.0) { r.fs = e; return r; }
    }
    const int k = P.bc[side];
    if (k == BC_PERIODIC) r.i = wrap(i, P.nx);
    else { r.i = i < 0 ? -1 - i : 2 * P.nx - 1 - i; r.sx = -1; if (k == BC_REFLECTIVE) r.neg |= 2; }
  }
  return r;
}

// The image of cell (i, j) as the stencil of the fluid cell (vi, vj) sees it:
// boundary sides first, then the solid block.
__device__ __forceinline__ Img image(const Prob& P, int i, int j, int vi, int vj) {
  Img r = image(P, i, j);
  if (P.sol_j > 0) solid_image(P, vi, vj, r);
  return r;
}

// The image by the sides' kinds alone (fixed states ignored; an inflow side
// maps like a transmissive one).  Separable in x and y; equal to image() for
// every cell image() does not make a fixed-state ghost.
__device__ __forceinline__ Img image_kind(const Prob& P, int i, int j) {
  Img r{i, j, 1, 1, 0, -1};
  if (i < 0 || i >= P.nx) {
    const int k = P.bc[i < 0 ? 0 : 1];
    if (k == BC_PERIODIC) r.i = wrap(i, P.nx);
    else { r.i = i < 0 ? -1 - i : 2 * P.nx - 1 - i; r.sx = -1; if (k == BC_REFLECTIVE) r.neg |= 2; }
  }
  if (j < 0 || j >= P.ny) {
    const int k = P.bc[j < 0 ? 2 : 3];
    if (k == BC_PERIODIC) r.j = wrap(j, P.ny);
    else { r.j = j < 0 ? -1 - j : 2 * P.ny - 1 - j; r.sy = -1; if (k == BC_REFLECTIVE) r.neg |= 4; }
  }
  return r;
}

// Variable v of a fixed-state ghost (its average and every point value)
__device__ __forceinline__ double fixed_val(const Prob& P, const Img& m, int v) {
  return ((m.neg >> v) & 1 ? -1.0 : 1.0) * P.fixtab[4 * m.fs + v];
}

// Sign of variable v of an image cell (reflective walls)
__device__ __forceinline__ int vsign(const Img& m, int v) { return (m.neg >> v) & 1 ? -1 : 1; }

__device__ __forceinline__ long long sidx(const Prob& P, int var, int mom, int i, int j) {
  return (long long)(var * P.nmom + mom) * P.plane + (long long)j * P.pitch + i;
}

// Cell average of variable v of an image cell, fixed-state ghosts included.
__device__ __forceinline__ double avg_img(const Prob& P, const double* __restrict__ U, const Img& m, int v) {
  if (m.fs >= 0) return fixed_val(P, m, v);
  return vsign(m, v) * U[sidx(P, v, 0, m.i, m.j)];
}

// ---------------------------------------------------------------- physics
// Physical flux of eq. (1D-Euler) / (2D-Euler) or of the scalar laws in
// direction dir (0 = x, 1 = y); NV = 1 (scalar), 3 (1D Euler), 4 (2D Euler).
// 1/x correctly rounded (the same value as the IEEE division 1/x) by the
// reciprocal intrinsics of the two hardware precisions; double-float divides.
template <typename T> __device__ __forceinline__ T rcp(T x) { return T(1) / x; }
template <> __device__ __forceinline__ float rcp<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ double rcp<double>(double x) { return __drcp_rn(x); }

template <typename T, int NV>
__device__ __forceinline__ void phys_flux(const Prob& P, const T* u, int dir, T* f) {
  if constexpr (NV == 1) {
    if (P.eq == EQ_ADV) f[0] = T(dir == 0 ? P.adv_a : P.adv_b) * u[0];
    else f[0] = T(0.5) * u[0] * u[0];
  } else if constexpr (NV == 3) {
    const T g = pc<T>(P.cgamma);
    const T inv = rcp(u[0]), mu = u[1] * inv, E = u[2];
    const T p = (g - T(1)) * (E - T(0.5) * u[1] * mu);
    f[0] = u[1]; f[1] = u[1] * mu + p; f[2] = mu * (E + p);
  } else {
    const T g = pc<T>(P.cgamma);
    const T inv = rcp(u[0]), mu = u[1] * inv, nu = u[2] * inv, E = u[3];
    const T p = (g - T(1)) * (E - T(0.5) * (u[1] * mu + u[2] * nu));
    if (dir == 0) { f[0] = u[1]; f[1] = u[1] * mu + p; f[2] = u[1] * nu; f[3] = mu * (E + p); }
    else          { f[0] = u[2]; f[1] = u[2] * mu; f[2] = u[2] * nu + p; f[3] = nu * (E + p); }
  }
}

// Euler flux with the reciprocal of the density supplied by the caller.
template <typename T, int NV>
__device__ __forceinline__ void euler_flux_inv(const Prob& P, const T* u, T inv, int dir, T* f) {
  const T g = pc<T>(P.cgamma);
  if constexpr (NV == 3) {
    const T mu = u[1] * inv, E = u[2];
    const T p = (g - T(1)) * (E - T(0.5) * u[1] * mu);
    f[0] = u[1]; f[1] = u[1] * mu + p; f[2] = mu * (E + p);
  } else {
    const T mu = u[1] * inv, nu = u[2] * inv, E = u[3];
    const T p = (g - T(1)) * (E - T(0.5) * (u[1] * mu + u[2] * nu));
    if (dir == 0) { f[0] = u[1]; f[1] = u[1] * mu + p; f[2] = u[1] * nu; f[3] = mu * (E + p); }
    else          { f[0] = u[2]; f[1] = u[2] * mu; f[2] = u[2] * nu + p; f[3] = nu * (E + p); }
  }
}

// Reciprocals of N values with a single division (prefix products, one inverse,
// back substitution); used by the FP64 path, where a division costs about as
// much as a dozen fused multiply-adds.
template <int N, typename T>
__device__ __forceinline__ void batch_inverse(const T (&x)[N], T (&inv)[N]) {
  T pre[N];
  pre[0] = x[0];
#pragma unroll
  for (int i = 1; i < N; ++i) pre[i] = pre[i - 1] * x[i];
  T r = rcp(pre[N - 1]);
#pragma unroll
  for (int i = N - 1; i > 0; --i) {
    inv[i] = r * pre[i - 1];
    r = r * x[i];
  }
  inv[0] = r;
}

// Reciprocals for the FP64-class types.  FP64: one division for all N.
// Double-float carries FP32's exponent range, where a product of 12 or 16
// densities can underflow, so it inverts groups of 4.
template <int N, typename T>
__device__ __forceinline__ void batch_inverse_ranged(const T (&x)[N], T (&inv)[N]) {
  if constexpr (is_df64<T>::value) {
    static_assert(N % 4 == 0, "groups of four");
#pragma unroll
    for (int g = 0; g < N; g += 4) {
      const T xs[4] = {x[g], x[g + 1], x[g + 2], x[g + 3]};
      T r[4];
      batch_inverse<4, T>(xs, r);
#pragma unroll
      for (int k = 0; k < 4; ++k) inv[g + k] = r[k];
    }
  } else {
    batch_inverse<N, T>(x, inv);
  }
}

// One common denominator for the nonlinear weights is safe in FP64 only: it
// multiplies four (beta + eps) factors (eps^4 = 1e-40 is below FP32's range,
// which double-float shares).
template <typename T> struct one_division { static constexpr bool value = sizeof(T) == 8 && !is_df64<T>::value; };

// Velocity seen by the KXRCF indicator for scalar laws (Remarks 2, 3): f'(u), g'(u).
template <typename T>
__device__ __forceinline__ T scalar_velocity(const Prob& P, T u, int dir) {
  if (P.eq == EQ_ADV) return T(dir == 0 ? P.adv_a : P.adv_b);
  return u;
}

// HLLC flux, eqs. (f_HLLC), (COEF), (uLR_), as a rotated 1D solver in direction
// dir (the tangential velocity is carried through the star state).
// Branch order: 0 <= sL -> fL; 0 <= s* -> f*L; 0 <= sR -> f*R; else fR.
// wall: the face of the forward step's solid block (one side the reflection of
// the other): the star branch is taken whatever the sign of the wave-speed
// estimate, so the flux carries no mass or energy (s* = 0) and the normal
// momentum flux is the star pressure -- the estimate of eq. (COEF) gives
// s_L > 0 for flow running into a wall faster than about its sound speed,
// where the first branch of eq. (f_HLLC) would let the gas through the wall.
template <typename T, int NV>
__device__ __forceinline__ void hllc(const Prob& P, const T* uL, const T* uR, int dir, T* F, bool wall = false) {
  constexpr bool two = NV == 4;
  const T g = pc<T>(P.cgamma);
  const int in = 1 + dir, it = 2 - dir;
  constexpr int iE = NV - 1;
  const T rL = uL[0], rR = uR[0];
  // one reciprocal for both densities' reciprocals
  const T q = rcp(rL * rR);
  const T iL = rR * q, iR = rL * q;
  const T mL = uL[in] * iL, mR = uR[in] * iR;
  const T tL = two ? uL[it] * iL : T(0), tR = two ? uR[it] * iR : T(0);
  const T EL = uL[iE], ER = uR[iE];
  const T gm1 = pc<T>(P.cgm1);
  const T pL = gm1 * (EL - T(0.5) * rL * (mL * mL + tL * tL));
  const T pR = gm1 * (ER - T(0.5) * rR * (mR * mR + tR * tR));
  const T gL = g * iL, gR = g * iR;
  const T cL = sqrt(gL * pL), cR = sqrt(gR * pR);
  const T rs = T(0.5) * (rL + rR), cs = T(0.5) * (cL + cR);
  const T crs = cs * rs;
  const T ps = T(0.5) * (pL + pR + (mL - mR) * crs);
  const T ss = T(0.5) * (mL + mR + (pL - pR) / crs);
  // eq. (COEF): c_K coef_K = sqrt(gamma p_K / rho_K) sqrt(1 + k (p* / p_K - 1)) with
  // k = (gamma + 1) / (2 gamma) when p* > p_K, else c_K.  FP64 keeps the two roots
  // (the second only where p* > p_K); FP32 and double-float take one root,
  // sqrt(gamma / rho_K (p_K + k max(p* - p_K, 0))), without the divisions by p_K
  // (measured 5 % faster in the double-float update, 1 % slower in FP64).  A
  // non-finite p* stays non-finite either way (the comparison is written so), and
  // the branches below then fall through to f_R.
  const T k = pc<T>(P.chk);
  T sL, sR;
  if constexpr (std::is_same<T, double>::value) {
    const T coefL = ps <= pL ? T(1) : sqrt(T(1) + k * (ps / pL - T(1)));
    const T coefR = ps <= pR ? T(1) : sqrt(T(1) + k * (ps / pR - T(1)));
    sL = mL - cL * coefL;
    sR = mR + cR * coefR;
  } else {
    const T dL = ps - pL, dR = ps - pR;
    sL = mL - sqrt(gL * (pL + k * (dL <= T(0) ? T(0) : dL)));
    sR = mR + sqrt(gR * (pR + k * (dR <= T(0) ? T(0) : dR)));
  }
  const bool useL = (!wall && T(0) <= sL) || T(0) <= ss;     // left physical or left star flux
  const T rK = useL ? rL : rR, mK = useL ? mL : mR, tK = useL ? tL : tR;
  const T EK = useL ? EL : ER, pK = useL ? pL : pR, sK = useL ? sL : sR;
  // physical normal flux of the chosen side
  T fK[NV], uK[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) uK[v] = useL ? uL[v] : uR[v];
  fK[0] = rK * mK;
  fK[1] = dir == 0 ? rK * mK * mK + pK : rK * mK * tK;
  if constexpr (two) fK[2] = dir == 0 ? rK * mK * tK : rK * mK * mK + pK;
  fK[iE] = mK * (EK + pK);
  if (!wall && (T(0) <= sL || !(T(0) <= sR || T(0) <= ss))) {   // supersonic: fL or fR
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = fK[v];
    return;
  }
  const T a = sK - mK, b = sK - ss;
  // D = 1/(a b) gives 1/a and 1/b with one reciprocal
  const T iK = useL ? iL : iR;
  const T D = rcp(a * b);
  const T fac = rK * a * (a * D);
  const T ek = EK * iK;
  const T pk = pK * iK * (b * D);
  T us[NV];
  us[0] = fac;
  us[in] = fac * ss;
  if constexpr (two) us[it] = fac * tK;
  us[iE] = fac * (ek + (ss - mK) * (ss + pk));
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = fK[v] + sK * (us[v] - uK[v]);
}

// Scalar laws: local Lax-Friedrichs flux with alpha = max(|f'(uL)|, |f'(uR)|).
template <typename T>
__device__ __forceinline__ T llf(const Prob& P, T uL, T uR, int dir) {
  T fl, fr;
  phys_flux<T, 1>(P, &uL, dir, &fl);
  phys_flux<T, 1>(P, &uR, dir, &fr);
  const T aL = tabs(scalar_velocity(P, uL, dir)), aR = tabs(scalar_velocity(P, uR, dir));
  return T(0.5) * (fl + fr) - T(0.5) * tmax(aL, aR) * (uR - uL);
}

template <typename T, int NV>
__device__ __forceinline__ void num_flux(const Prob& P, const T* uL, const T* uR, int dir, T* F) {
  if constexpr (NV == 1) F[0] = llf(P, uL[0], uR[0], dir);
  else hllc<T, NV>(P, uL, uR, dir, F);
}

// ---------------------------------------------------------------- nonlinear weights
// WENO-Z weights of eqs. (tau4), (non-linear-weight) and the combination of
// eq. (re-p) rewritten on q_1..q_4:  u = sum_k c_k q_k with
// c_k = omega_k S_k/g_k - omega_{k+1} S_k/g_{k+1},  c_4 = omega_4 S_4/g_4.
template <typename T>
__device__ __forceinline__ void combine_weights(const Weights<T>& W, const T beta[4], T c[4]) {
  const T tau4s = tabs(beta[3] - beta[0]) + tabs(beta[3] - beta[1]) + tabs(beta[3] - beta[2]);
  const T tau4 = (tau4s * T(1.0 / 3.0)) * (tau4s * T(1.0 / 3.0));
  T om[4];
  if constexpr (one_division<T>::value) {
    // FP64: one division.  With x_l = beta_l + eps, wbar_l = gamma_l (x_l + tau)/x_l;
    // scaling every wbar_l by prod_m x_m gives N_l = gamma_l (x_l + tau) prod_{m!=l} x_m
    // and omega_l = N_l / sum_m N_m.
    const T x0 = beta[0] + W.eps, x1 = beta[1] + W.eps, x2 = beta[2] + W.eps, x3 = beta[3] + W.eps;
    const T p01 = x0 * x1, p23 = x2 * x3;
    const T n0 = W.gam[0] * (x0 + tau4) * (x1 * p23);
    const T n1 = W.gam[1] * (x1 + tau4) * (x0 * p23);
    const T n2 = W.gam[2] * (x2 + tau4) * (p01 * x3);
    const T n3 = W.gam[3] * (x3 + tau4) * (p01 * x2);
    const T inv = rcp((n0 + n1) + (n2 + n3));
    om[0] = n0 * inv; om[1] = n1 * inv; om[2] = n2 * inv; om[3] = n3 * inv;
  } else {
    T wb[4], ws = T(0);
#pragma unroll
    for (int l = 0; l < 4; ++l) { wb[l] = W.gam[l] * (T(1) + tau4 / (beta[l] + W.eps)); ws += wb[l]; }
    const T inv = rcp(ws);
#pragma unroll
    for (int l = 0; l < 4; ++l) om[l] = wb[l] * inv;
  }
  c[0] = om[0] * W.sg[0] - om[1] * W.s1g[1];
  c[1] = om[1] * W.sg[1] - om[2] * W.s1g[2];
  c[2] = om[2] * W.sg[2] - om[3] * W.s1g[3];
  c[3] = om[3] * W.sg[3];
}

// ---------------------------------------------------------------- 1D reconstruction
// d = (u_{i-1}, u_i, u_{i+1}, v_{i-1}, v_i, v_{i+1}) of one variable; out = the
// four Gauss-Lobatto values of eq. (re-u).  Steps 1.1-1.3 of the 1D algorithm.
template <typename T>
__device__ __forceinline__ void recon1d(const Weights<T>& W, const Beta1<T>& B, const T (&d)[6], T (&out)[4]) {
  T s[6];
  hwp::split1d<T>(d, s);
  T beta[4];
  hwp::beta1d<T>(B.B2, B.B3, B.B4, s, beta[1], beta[2], beta[3]);
  // beta_1: eqs. (beta1-LR), (tau1), (w1_-LR), (w1-LR), (beta1)
  {
    const T dl = d[1] - d[0], dr = d[2] - d[1];
    const T bl = dl * dl, br = dr * dr;
    const T t1 = tabs(br - bl) * tabs(br - bl);
    T gg;
    if constexpr (sizeof(T) == 8) {   // common denominator: one division
      const T xl = bl + W.eps, xr = br + W.eps;
      const T nl = (xl + t1) * xr, nr = (xr + t1) * xl;
      gg = (nl * dl + nr * dr) / (nl + nr);
    } else {
      const T wl = T(0.5) * (T(1) + t1 / (bl + W.eps));
      const T wr = T(0.5) * (T(1) + t1 / (br + W.eps));
      const T inv = rcp(wl + wr);
      gg = (wl * inv) * dl + (wr * inv) * dr;
    }
    beta[0] = gg * gg;
  }
  T c[4];
  combine_weights(W, beta, c);
  hwp::values1d<T>(s, d[1], c, out);
}

// ---------------------------------------------------------------- 2D reconstruction
// d = the 23 data of q_4 (u at labels 1..9, v at 1,3,4,5,6,7,9, w at
// 1,2,3,5,7,8,9; labels of the paper's 3x3 stencil table), out[k*4+l] =
// u_{i,j}(xi_k, eta_l) of eq. (2D-re-u).  Steps 1.1-1.3 of the 2D algorithm.
// Square cells: beta_1 of eq. (2D-beta1) is (sum w_1k Dx_k)^2 + (sum w_1k Dy_k)^2.
template <typename T>
__device__ __forceinline__ void recon2d(const Weights<T>& W, const Beta2<T>& B, const T (&d)[23], T (&out)[16]) {
  T s[23];
  hwp::split2d<T>(d, s);
  T beta[4];
  hwp::beta2d<T>(B.B2, B.B3, B.B4, s, beta[1], beta[2], beta[3]);
  // beta_1: eqs. (2D-q1-1234) .. (2D-beta1); tau_1 over the 6 unordered pairs
  {
    const T u2 = d[1], u4 = d[3], u5 = d[4], u6 = d[5], u8 = d[7];
    const T bx[4] = {u5 - u4, u6 - u5, u6 - u5, u5 - u4};
    const T by[4] = {u8 - u5, u8 - u5, u5 - u2, u5 - u2};
    T b1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) b1[k] = bx[k] * bx[k] + by[k] * by[k];
    T ts = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int l = k + 1; l < 4; ++l) ts += tabs(b1[k] - b1[l]);
    const T t1 = (ts * T(1.0 / 6.0)) * (ts * T(1.0 / 6.0));
    T gx = T(0), gy = T(0);
    if constexpr (one_division<T>::value) {   // common denominator: one division
      const T y0 = b1[0] + W.eps, y1 = b1[1] + W.eps, y2 = b1[2] + W.eps, y3 = b1[3] + W.eps;
      const T p01 = y0 * y1, p23 = y2 * y3;
      const T n[4] = {(y0 + t1) * (y1 * p23), (y1 + t1) * (y0 * p23), (y2 + t1) * (p01 * y3), (y3 + t1) * (p01 * y2)};
      const T inv = rcp((n[0] + n[1]) + (n[2] + n[3]));
#pragma unroll
      for (int k = 0; k < 4; ++k) { gx = fma(n[k], bx[k], gx); gy = fma(n[k], by[k], gy); }
      gx *= inv;
      gy *= inv;
    } else {
      T w[4], wsum = T(0);
#pragma unroll
      for (int k = 0; k < 4; ++k) { w[k] = T(0.25) * (T(1) + t1 / (b1[k] + W.eps)); wsum += w[k]; }
      const T inv = rcp(wsum);
#pragma unroll
      for (int k = 0; k < 4; ++k) { gx = fma(w[k] * inv, bx[k], gx); gy = fma(w[k] * inv, by[k], gy); }
    }
    beta[0] = gx * gx + gy * gy;
  }
  T c[4];
  combine_weights(W, beta, c);
  hwp::values2d<T>(s, d[4], c, out);
}

// Positions (ox, oy, kind) of the 23 data of q_4 in gather order.
__device__ __forceinline__ void d4_slot(int c, int& kind, int& ox, int& oy) {
  // u at labels 1..9 (bottom row first), v at 1,3,4,5,6,7,9, w at 1,2,3,5,7,8,9
  const int vl[7] = {1, 3, 4, 5, 6, 7, 9};
  const int wl[7] = {1, 2, 3, 5, 7, 8, 9};
  int lbl;
  if (c < 9) { kind = 0; lbl = c + 1; }
  else if (c < 16) { kind = 1; lbl = vl[c - 9]; }
  else { kind = 2; lbl = wl[c - 16]; }
  ox = (lbl - 1) % 3 - 1;
  oy = (lbl - 1) / 3 - 1;
}

// A face counts as inflow in KXRCF when its velocity exceeds this (absolute,
// in the problem's velocity units): rounding noise around a fluid exactly at
// rest must not decide the indicator.
constexpr double KX_VDEAD = 1e-12;

// Modification weights of eq. (vi) (quartic p_0 of eq. (p0)):
// vbar_i <- -5/76 u_{i-1} + 5/76 u_{i+1} - 11/38 v_{i-1} - 11/38 v_{i+1}.
constexpr double MOD_WU = 5.0 / 76.0;
constexpr double MOD_WV = -11.0 / 38.0;

// ---------------------------------------------------------------- 2D point values and KXRCF
// Point-value arrays G[var][16][j][gpitch]; point (k, l) of a possibly mirrored image cell.
__device__ __forceinline__ int mpt(const Img& m, int k, int l) {
  if (m.sx < 0) k = 3 - k;
  if (m.sy < 0) l = 3 - l;
  return k * 4 + l;
}

__device__ __forceinline__ long long goff(const Prob& P, int i, int j) { return (long long)j * P.gpitch + i; }

// KXRCF value of eq. (KXRCF_) with eq. (line-integral-average_): inflow faces by
// the sign of the GL-weighted face velocity (average of both sides), jumps of
// the indicator variable (variable 0) weighted by dy w_l or dx w_k.
template <typename T>
__device__ __forceinline__ T kxrcf2d(const Prob& P, const Weights<T>& W, const T* __restrict__ G,
                                     const T* __restrict__ aux, int i, int j) {
  const long long o = goff(P, i, j);
  const Img L = image(P, i - 1, j, i, j), R = image(P, i + 1, j, i, j), Bo = image(P, i, j - 1, i, j),
            Tp = image(P, i, j + 1, i, j);
  const long long oL = goff(P, L.i, L.j), oR = goff(P, R.i, R.j), oB = goff(P, Bo.i, Bo.j), oT = goff(P, Tp.i, Tp.j);
  // the neighbours' face velocities (the x ones negated through an x wall, the y
  // ones through a y wall); a fixed-state ghost's is its own state's velocity
  const T axl = L.fs >= 0 ? from_double<T>(P.fixtab[4 * L.fs + 1] / P.fixtab[4 * L.fs]) : aux[(L.sx < 0 ? 0 : 1) * P.gplane + oL];
  const T axr = R.fs >= 0 ? from_double<T>(P.fixtab[4 * R.fs + 1] / P.fixtab[4 * R.fs]) : aux[(R.sx < 0 ? 1 : 0) * P.gplane + oR];
  const T ayb = Bo.fs >= 0 ? from_double<T>(P.fixtab[4 * Bo.fs + 2] / P.fixtab[4 * Bo.fs]) : aux[(Bo.sy < 0 ? 2 : 3) * P.gplane + oB];
  const T ayt = Tp.fs >= 0 ? from_double<T>(P.fixtab[4 * Tp.fs + 2] / P.fixtab[4 * Tp.fs]) : aux[(Tp.sy < 0 ? 3 : 2) * P.gplane + oT];
  const T vxl = T(0.5) * ((L.neg & 2 ? -axl : axl) + aux[0 * P.gplane + o]);
  const T vxr = T(0.5) * (aux[1 * P.gplane + o] + (R.neg & 2 ? -axr : axr));
  const T vyb = T(0.5) * ((Bo.neg & 4 ? -ayb : ayb) + aux[2 * P.gplane + o]);
  const T vyt = T(0.5) * (aux[3 * P.gplane + o] + (Tp.neg & 4 ? -ayt : ayt));
  // the indicator variable (density) of a neighbour at its point (k, l)
  auto rho_at = [&](const Img& m, long long om, int k, int l) -> T {
    return m.fs >= 0 ? from_double<T>(P.fixtab[4 * m.fs]) : G[(long long)mpt(m, k, l) * P.gplane + om];
  };
  const T dx = pc<T>(P.cdx), dy = pc<T>(P.cdy);
  T s = T(0), len = T(0);
  // a face shared with a solid cell (the forward step's block) is a wall, never an inflow face
  const bool wl = P.sol_j > 0 && is_solid(P, i - 1, j), wr = P.sol_j > 0 && is_solid(P, i + 1, j);
  const bool wb = P.sol_j > 0 && is_solid(P, i, j - 1), wt = P.sol_j > 0 && is_solid(P, i, j + 1);
  if (vxl > T(KX_VDEAD) && !wl) {
#pragma unroll
    for (int l = 0; l < 4; ++l) s += dy * gl_w<T>(l) * (G[(long long)(l)*P.gplane + o] - rho_at(L, oL, 3, l));
    len += dy;
  }
  if (-vxr > T(KX_VDEAD) && !wr) {
#pragma unroll
    for (int l = 0; l < 4; ++l) s += dy * gl_w<T>(l) * (G[(long long)(12 + l) * P.gplane + o] - rho_at(R, oR, 0, l));
    len += dy;
  }
  if (vyb > T(KX_VDEAD) && !wb) {
#pragma unroll
    for (int k = 0; k < 4; ++k) s += dx * gl_w<T>(k) * (G[(long long)(k * 4) * P.gplane + o] - rho_at(Bo, oB, k, 3));
    len += dx;
  }
  if (-vyt > T(KX_VDEAD) && !wt) {
#pragma unroll
    for (int k = 0; k < 4; ++k) s += dx * gl_w<T>(k) * (G[(long long)(k * 4 + 3) * P.gplane + o] - rho_at(Tp, oT, k, 0));
    len += dx;
  }
  const T nrm = aux[4 * P.gplane + o];
  if (len == T(0) || nrm == T(0)) return T(0);
  return tabs(s) / len / (pc<T>(P.cdx2) * nrm);   // h^{(l+1)/3}, l = 5, h = dx
}

// ---------------------------------------------------------------- TVB indicator
// The minmod-based TVB indicator named in Remark 2 (Cockburn & Shu's TVB
// limiter used as a troubled-cell indicator) on the indicator variable
// (variable 0), acting on the cell's linear polynomial fixed by its moments:
// its face deviations are +-6 vbar (x) and +-6 wbar (y).  The cell is troubled
// when the modified minmod m(a, b, c) = a if |a| <= M h^2, else minmod(a, b, c)
// changes a = 6 vbar (6 wbar) against the forward and backward differences of
// the averages in that direction.  FP64: it reads only the FP64 state.
__device__ __forceinline__ bool tvb_changes(double a, double b, double c, double bound) {
  if (!(fabs(a) > bound)) return false;
  double mm = 0.0;
  if (a > 0.0 && b > 0.0 && c > 0.0) mm = fmin(a, fmin(b, c));
  else if (a < 0.0 && b < 0.0 && c < 0.0) mm = fmax(a, fmax(b, c));
  return mm != a;
}

__device__ __forceinline__ bool tvb_cell(const Prob& P, const double* __restrict__ U, int i, int j) {
  const double bound = P.tvb_m * P.dx * P.dx;
  const double u0 = U[sidx(P, 0, 0, i, j)];
  const Img L = image(P, i - 1, j, i, j), R = image(P, i + 1, j, i, j);
  const double ax = 6.0 * U[sidx(P, 0, 1, i, j)];
  if (tvb_changes(ax, avg_img(P, U, R, 0) - u0, u0 - avg_img(P, U, L, 0), bound)) return true;
  if (P.nmom == 2) return false;
  const Img Bo = image(P, i, j - 1, i, j), Tp = image(P, i, j + 1, i, j);
  const double ay = 6.0 * U[sidx(P, 0, 2, i, j)];
  return tvb_changes(ay, avg_img(P, U, Tp, 0) - u0, u0 - avg_img(P, U, Bo, 0), bound);
}

}  // namespace hw
