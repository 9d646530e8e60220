// One-dimensional stage pipeline of the moment-based multi-resolution HWENO
// scheme (Sec. 2.1 of Li, Shu & Qiu, arXiv 2201.12193) on sm_103a.
//
// Same four steps per Runge-Kutta stage as the 2D pipeline:
//   rec1d    Step 1: 3-cell moments -> 4 Gauss-Lobatto values (eq. (re-u))
//   flag1d   Step 2.1/2.2: KXRCF (eq. (KXRCF), (line-integral-average)) and
//            the modified first moment of eq. (vi) in troubled cells
//   rec1d*   Step 2.3: troubled cells again from the modified moments
//   update1d Step 3: HLLC/LLF fluxes, quadrature of eq. (F), L(U) of
//            eq. (1D-equ-int-approximation), SSP-RK3 (eq. (Runge-Kutta)).
#include <algorithm>

#include "hweno_internal.h"

namespace hw {
namespace {

constexpr int RB = 128;
constexpr int UB = RB + 32;   // update threads: one per face (RB + 1) then one per cell (RB)

__device__ __forceinline__ int mpt1(const Img& m, int k) { return m.sx < 0 ? 3 - k : k; }

template <bool FLAGGED>
__device__ __forceinline__ double load_mom1(const Prob& P, const double* __restrict__ U, const uint8_t* __restrict__ mask,
                                            const double* __restrict__ Mod, int var, int kind, const Img& m) {
  const int g = vsign(m, var);      // reflective wall: the normal momentum negated
  if (kind == 0) return g * U[sidx(P, var, 0, m.i, 0)];
  double v;
  if (FLAGGED && mask[m.i]) v = Mod[(long long)var * P.plane + m.i];
  else v = U[sidx(P, var, 1, m.i, 0)];
  return m.sx < 0 ? -g * v : g * v;
}

// One thread per (cell, variable): the variables of a cell are independent in
// Step 1, and the 1D problems are small, so spreading them over threads cuts
// the latency of the pass (the KXRCF face velocities and norm are formed from
// the point values in the indicator pass).
template <typename T, int NV, bool FLAGGED>
__global__ void __launch_bounds__(RB) rec1d_kernel(Prob P, Weights<T> W, Beta1<T> B, const double* __restrict__ U,
                                                  const uint8_t* __restrict__ mask, const double* __restrict__ Mod,
                                                  const int* __restrict__ list, const int* __restrict__ count,
                                                  T* __restrict__ G, unsigned long long* __restrict__ rerec) {
  const int n = FLAGGED ? *count : P.nx;
  if (FLAGGED && rerec && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(rerec, (unsigned long long)n);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * NV; t += gridDim.x * blockDim.x) {
    const int v = t / n, e = t - v * n;
    const int i = FLAGGED ? list[e] : e;
    const Img nb[3] = {image(P, i - 1, 0), image(P, i, 0), image(P, i + 1, 0)};
    T d[6];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      d[c] = from_double<T>(load_mom1<FLAGGED>(P, U, mask, Mod, v, 0, nb[c]));
      d[3 + c] = from_double<T>(load_mom1<FLAGGED>(P, U, mask, Mod, v, 1, nb[c]));
    }
    T out[4];
    recon1d<T>(W, B, d, out);
#pragma unroll
    for (int p = 0; p < 4; ++p) G[(long long)(v * 4 + p) * P.gplane + i] = out[p];
  }
}

// Eigenvectors of the 1D Euler flux Jacobian at the state (rho, rho u, E):
// right R (columns: u - c, u, u + c) and left L (rows), L R = I (Toro, Riemann
// Solvers and Numerical Methods for Fluid Dynamics, Sec. 3.1).
__device__ __forceinline__ void euler1d_eigvec(double gam, double r, double m, double E, double (&R)[3][3],
                                               double (&L)[3][3]) {
  const double mu = m / r, p = (gam - 1.0) * (E - 0.5 * r * mu * mu);
  const double cs = sqrt(gam * p / r), H = (E + p) / r;
  const double b1 = (gam - 1.0) / (cs * cs), b2 = 0.5 * b1 * mu * mu;
  R[0][0] = 1.0; R[0][1] = 1.0; R[0][2] = 1.0;
  R[1][0] = mu - cs; R[1][1] = mu; R[1][2] = mu + cs;
  R[2][0] = H - mu * cs; R[2][1] = 0.5 * mu * mu; R[2][2] = H + mu * cs;
  L[0][0] = 0.5 * (b2 + mu / cs); L[0][1] = -0.5 * (b1 * mu + 1.0 / cs); L[0][2] = 0.5 * b1;
  L[1][0] = 1.0 - b2; L[1][1] = b1 * mu; L[1][2] = -b1;
  L[2][0] = 0.5 * (b2 - mu / cs); L[2][1] = -0.5 * (b1 * mu - 1.0 / cs); L[2][2] = 0.5 * b1;
}

// Step 1 (and 2.3 when FLAGGED) in local characteristic variables (1D Euler,
// Prob::charwise): the moments of the 3-cell stencil are projected on the
// characteristic fields of the target cell's average state, each field is
// reconstructed by the scalar procedure (its own smoothness indicators and
// weights), and the point values are mapped back.  One thread per cell.
template <typename T, bool FLAGGED>
__global__ void __launch_bounds__(RB) rec1d_char_kernel(Prob P, Weights<T> W, Beta1<T> B,
                                                       const double* __restrict__ U, const uint8_t* __restrict__ mask,
                                                       const double* __restrict__ Mod, const int* __restrict__ list,
                                                       const int* __restrict__ count, T* __restrict__ G,
                                                       unsigned long long* __restrict__ rerec) {
  const int n = FLAGGED ? *count : P.nx;
  if (FLAGGED && rerec && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(rerec, (unsigned long long)n);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int i = FLAGGED ? list[t] : t;
    const Img nb[3] = {image(P, i - 1, 0), image(P, i, 0), image(P, i + 1, 0)};
    double Rd[3][3], Ld[3][3];
    euler1d_eigvec(P.gamma, U[sidx(P, 0, 0, i, 0)], U[sidx(P, 1, 0, i, 0)], U[sidx(P, 2, 0, i, 0)], Rd, Ld);
    T dv[3][6];
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dv[v][c] = from_double<T>(load_mom1<FLAGGED>(P, U, mask, Mod, v, 0, nb[c]));
        dv[v][3 + c] = from_double<T>(load_mom1<FLAGGED>(P, U, mask, Mod, v, 1, nb[c]));
      }
    T w[3][4];
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
      const T l0 = from_double<T>(Ld[f][0]), l1 = from_double<T>(Ld[f][1]), l2 = from_double<T>(Ld[f][2]);
      T d[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) d[q] = l0 * dv[0][q] + l1 * dv[1][q] + l2 * dv[2][q];
      recon1d<T>(W, B, d, w[f]);
    }
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      const T r0 = from_double<T>(Rd[v][0]), r1 = from_double<T>(Rd[v][1]), r2 = from_double<T>(Rd[v][2]);
#pragma unroll
      for (int p = 0; p < 4; ++p) G[(long long)(v * 4 + p) * P.gplane + i] = r0 * w[0][p] + r1 * w[1][p] + r2 * w[2][p];
    }
  }
}

// KXRCF face velocity of a cell at its left (side 0) or right (side 1) face,
// from its own point values: u at the face (scalars, f'(u)) or (rho u)/rho (Euler).
// KXRCF value of a cell (eq. (KXRCF) with the line integral of
// eq. (line-integral-average) reduced to the two end points in 1D): the jumps
// jl, jr of the density at the inflow faces (face velocities vl, vr), over
// h^{(l+1)/3} (l = 5) times the cell's largest density point value nrm.  The
// pipeline and the fused stage both call this, so their flags agree bit for bit.
template <typename T>
__device__ __forceinline__ T kxrcf1(const Prob& P, T jl, T jr, T vl, T vr, T nrm) {
  const T s = jl * (vl > T(KX_VDEAD) ? T(1) : T(0)) + jr * (-vr > T(KX_VDEAD) ? T(1) : T(0));
  return nrm == T(0) ? T(0) : tabs(s) / (T(P.dx * P.dx) * nrm);
}

// Modified first moment of a troubled cell, eq. (vi): from the neighbours'
// averages uL, uR and first moments vL, vR (image signs applied).
__device__ __forceinline__ double mod1(double uL, double uR, double vL, double vR) {
  return MOD_WU * (uR - uL) + MOD_WV * (vL + vR);
}

template <typename T, int NV>
__device__ __forceinline__ T face_vel1(const Prob& P, const T* __restrict__ G, int c, int side) {
  const int p = side ? 3 : 0;
  if constexpr (NV == 1) return scalar_velocity(P, G[(long long)p * P.gplane + c], 0);
  else return G[(long long)(4 + p) * P.gplane + c] / G[(long long)p * P.gplane + c];
}

template <typename T, int NV>
__global__ void __launch_bounds__(RB) flag1d_kernel(Prob P, Weights<T> W, const double* __restrict__ U,
                                                   const T* __restrict__ G,
                                                   uint8_t* __restrict__ mask, double* __restrict__ Mod,
                                                   int* __restrict__ list, int* __restrict__ count,
                                                   double* __restrict__ aleph) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < P.nx;
  bool flag = false;
  Img L{0, 0, 1, 1, 0, -1}, R{0, 0, 1, 1, 0, -1};
  if (valid) {
    L = image(P, i - 1, 0);
    R = image(P, i + 1, 0);
    if (P.indicator == IND_ALL) {
      flag = true;
    } else if (P.indicator == IND_TVB) {
      flag = tvb_cell(P, U, i, 0);
    } else if (P.indicator == IND_KXRCF) {
      // face velocities: average of both sides' velocities at the face
      const T al = face_vel1<T, NV>(P, G, L.i, L.sx < 0 ? 0 : 1), ar = face_vel1<T, NV>(P, G, R.i, R.sx < 0 ? 1 : 0);
      const T vl = T(0.5) * ((L.neg & 2 ? -al : al) + face_vel1<T, NV>(P, G, i, 0));
      const T vr = T(0.5) * (face_vel1<T, NV>(P, G, i, 1) + (R.neg & 2 ? -ar : ar));
      const T jl = G[0 * P.gplane + i] - G[(long long)mpt1(L, 3) * P.gplane + L.i];
      const T jr = G[3 * P.gplane + i] - G[(long long)mpt1(R, 0) * P.gplane + R.i];
      T nrm = T(0);
#pragma unroll
      for (int p = 0; p < 4; ++p) nrm = tmax(nrm, tabs(G[(long long)p * P.gplane + i]));
      const T a = kxrcf1<T>(P, jl, jr, vl, vr, nrm);
      if (aleph) aleph[i] = double(a);
      flag = a > T(1);
    }
  }
  const unsigned act = __ballot_sync(0xffffffffu, flag);
  if (act) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(act));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (flag) list[base + __popc(act & ((1u << lane) - 1u))] = i;
  }
  if (!valid) return;
  mask[i] = flag ? 1 : 0;
  if (!flag) return;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int gL = vsign(L, v), gR = vsign(R, v);
    const double uL = gL * U[sidx(P, v, 0, L.i, 0)], uR = gR * U[sidx(P, v, 0, R.i, 0)];
    const double vL = gL * L.sx * U[sidx(P, v, 1, L.i, 0)], vR = gR * R.sx * U[sidx(P, v, 1, R.i, 0)];
    Mod[(long long)v * P.plane + i] = mod1(uL, uR, vL, vR);
  }
}

struct Rk1 {
  const double* Uin; const double* Un; double* Uout;
  const uint8_t* mask; const double* Mod; const uint8_t* maskN; const double* ModN;
  double dt, cA, cB;
  double* Lout; double* Umod;
  unsigned* status;
  const double* dtp;     // dt on the device (overrides dt); < 0: skip, Uout = Uin
};

template <typename T, int NV>
__device__ __forceinline__ void gl1(const Prob& P, const T* __restrict__ G, const Img& m, int k, T (&u)[NV]) {
  const int p = mpt1(m, k);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const T x = G[(long long)(v * 4 + p) * P.gplane + m.i];
    u[v] = (m.neg >> v) & 1 ? -x : x;
  }
}

// Quadrature of eq. (F): the weighted physical flux at the cell's 4
// Gauss-Lobatto points u[k] (FP64 Euler: the four reciprocal densities with
// one division).
template <typename T, int NV>
__device__ __forceinline__ void quad1(const Prob& P, const T (&u)[4][NV], T (&F)[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = T(0);
  if constexpr (NV == 3 && one_division<T>::value) {
    T rho[4], inv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) rho[k] = u[k][0];
    batch_inverse<4, T>(rho, inv);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T f[NV];
      euler_flux_inv<T, NV>(P, u[k], inv[k], 0, f);
#pragma unroll
      for (int v = 0; v < NV; ++v) F[v] += gl_w<T>(k) * f[v];
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T f[NV];
      phys_flux<T, NV>(P, u[k], 0, f);
#pragma unroll
      for (int v = 0; v < NV; ++v) F[v] += gl_w<T>(k) * f[v];
    }
  }
}

// L(U) of eq. (1D-equ-int-approximation) of cell i from its face fluxes fp
// (right), fm (left) and quadrature F, and the SSP-RK3 combination of
// eq. (Runge-Kutta) (or L and the stage input into Lout / Umod).  The average
// equation is formed in FP64 from the widened face fluxes so that the flux
// differences telescope in every precision; FP32 values are widened by integer
// work and the first stage (cA = 0, cB = 1: U^(1) = U + dt L) is one FMA
// without U^n, so the FP64 pipe carries only the sums.  uin: the cell's stage
// input, its first moments replaced by those of eq. (vi) when it is flagged
// and they persist (or Lout asks for them).  Both 1D stage forms call this.
template <typename T, int NV>
__device__ __forceinline__ void rk1_cell(const Prob& P, const Rk1& S, int i, const T* fp, const T* fm,
                                         const T (&F)[NV], const double (&uinc)[2 * NV]) {
  const double idx = P.crdx.d;
  const T tidx = pc<T>(P.crdx);
  const bool fn = P.persist && S.maskN && S.maskN[i] != 0;
  const bool first = S.cA == 0.0;
  double newavg[NV];
  bool finite = true;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double L[2];
    L[0] = -(to_f64(fp[v]) - to_f64(fm[v])) * idx;
    L[1] = to_f64(-(fp[v] + fm[v]) * T(0.5) * tidx + F[v] * tidx);
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const long long si = (long long)(v * 2 + m) * P.plane + i;
      const double uin = uinc[v * 2 + m];
      if (S.Lout) {
        S.Lout[si] = L[m];
        if (S.Umod) S.Umod[si] = uin;
        continue;
      }
      double r;
      if (first) {
        r = fma(S.dt, L[m], uin);
      } else {
        const double un = (m == 1 && fn) ? S.ModN[(long long)v * P.plane + i] : S.Un[si];
        r = S.cA * un + S.cB * (uin + S.dt * L[m]);
      }
      S.Uout[si] = r;
      if (m == 0) newavg[v] = r;
      // non-finite by the exponent field (integer work, no FP64 compare)
      finite = finite && ((__double_as_longlong(r) >> 52) & 0x7FF) != 0x7FF;
    }
  }
  if (S.Lout) return;
  if (!finite) atomicOr(S.status, ST_NONFINITE);
  if (NV == 3) {
    // rho > 0 and p = (gamma - 1)(E - m^2 / (2 rho)) > 0, the latter as 2 E rho > m^2 (no division)
    const double rho = newavg[0];
    if (!(rho > 0.0) || !(2.0 * newavg[NV - 1] * rho > newavg[1] * newavg[1])) atomicOr(S.status, ST_NONPOSITIVE);
  }
}

template <typename T, int NV>
__global__ void __launch_bounds__(UB) update1d_kernel(Prob P, const T* __restrict__ G, Rk1 S) {
  __shared__ T fx[RB + 1][NV];
  const int t = threadIdx.x;
  const int i0 = blockIdx.x * RB;
  const int i = i0 + t;
  const bool live = t < RB && i < P.nx;
  if (S.dtp) {
    S.dt = *S.dtp;
    if (S.dt < 0.0) {   // a skipped step (block-uniform): the state passes through unchanged
      if (live && !S.Lout)
        for (int q = 0; q < NV * 2; ++q) S.Uout[(long long)q * P.plane + i] = S.Uin[(long long)q * P.plane + i];
      return;
    }
  }
  const Img self{i, 0, 1, 1, 0, -1};
  // fx[c] is the face left of cell i0 + c; one call site computes every face so
  // that faces shared by two blocks get bitwise the same flux.
  for (int c = t; c <= RB; c += UB) {     // UB > RB: at most one face per thread
    const int il = i0 + c - 1;
    if (il >= P.nx) continue;
    T uL[NV], uR[NV];
    gl1<T, NV>(P, G, image(P, il, 0), 3, uL);
    gl1<T, NV>(P, G, image(P, il + 1, 0), 0, uR);
    num_flux<T, NV>(P, uL, uR, 0, fx[c]);
  }
  __syncthreads();
  if (!live) return;
  T u[4][NV], F[NV];
#pragma unroll
  for (int k = 0; k < 4; ++k) gl1<T, NV>(P, G, self, k, u[k]);
  quad1<T, NV>(P, u, F);
  // modified first moments in the combination (persist), and always in the Umod output of Lout
  const bool fk = S.mask[i] != 0 && (P.persist || S.Lout);
  double uin[2 * NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    uin[2 * v] = S.Uin[(long long)(2 * v) * P.plane + i];
    uin[2 * v + 1] = fk ? S.Mod[(long long)v * P.plane + i] : S.Uin[(long long)(2 * v + 1) * P.plane + i];
  }
  rk1_cell<T, NV>(P, S, i, fx[t + 1], fx[t], F, uin);
}

}  // namespace
}  // namespace hw

#include "hweno_fused1d.cuh"

namespace hw {
namespace {

template <typename T, int NV, int SEG, int NT>
void fused1d_launch(const Prob& P, const Weights<T>& W, const Beta1<T>& Bt, const Rk1& r, const Bufs& B,
                    const StageCall& S, cudaStream_t st) {
  constexpr int smem = (int)sizeof(Fused1dSmem<T, NV, SEG>);
  static const bool attr = smem <= 48 * 1024 ||
      cudaFuncSetAttribute(fused1d_kernel<T, NV, SEG, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
          cudaSuccess;
  (void)attr;
  fused1d_kernel<T, NV, SEG, NT><<<(P.nx + SEG - 1) / SEG, NT, smem, st>>>(P, W, Bt, r, S.mask, S.Mod, S.aleph,
                                                                             B.rerec);
}

template <typename T, int NV>
void stage_t(const Prob& P, const Weights<T>& W, const Beta1<T>& Bt, const Bufs& B, const StageCall& S, cudaStream_t st) {
  Rk1 r{S.Uin, S.Un, S.Uout, S.mask, S.Mod, S.maskN, S.ModN, S.dt, S.cA, S.cB, S.Lout, S.Umod, B.status, S.dtp};
  if (P.fused) {   // the whole stage in one launch (hweno_set_fused)
    if (B.prof) B.prof->begin(5, st);
    if (P.nx >= 2 * P.nsm * 250) fused1d_launch<T, NV, 250, 256>(P, W, Bt, r, B, S, st);
    else fused1d_launch<T, NV, 32, 128>(P, W, Bt, r, B, S, st);
    if (B.prof) B.prof->end(st);
    return;
  }
  int* cnt = B.count + S.stage;
  cudaMemsetAsync(cnt, 0, sizeof(int), st);
  const int blocks = (P.nx + RB - 1) / RB, rblocks = (P.nx * NV + RB - 1) / RB;
  bool charwise = false;
  if constexpr (NV == 3) charwise = P.charwise != 0;
  if (B.prof) B.prof->begin(0, st);
  if (charwise)
    rec1d_char_kernel<T, false><<<blocks, RB, 0, st>>>(P, W, Bt, S.Uin, nullptr, nullptr, nullptr, nullptr, (T*)B.G,
                                                       nullptr);
  else
    rec1d_kernel<T, NV, false><<<rblocks, RB, 0, st>>>(P, W, Bt, S.Uin, nullptr, nullptr, nullptr, nullptr, (T*)B.G,
                                                       nullptr);
  if (B.prof) B.prof->end(st);
  if (B.prof) B.prof->begin(1, st);
  flag1d_kernel<T, NV><<<blocks, RB, 0, st>>>(P, W, S.Uin, (const T*)B.G, S.mask, S.Mod, B.list, cnt,
                                              S.aleph);
  if (B.prof) B.prof->end(st);
  if (P.indicator != IND_NONE) {
    if (B.prof) B.prof->begin(2, st);
    if (charwise)
      rec1d_char_kernel<T, true><<<blocks, RB, 0, st>>>(P, W, Bt, S.Uin, S.mask, S.Mod, B.list, cnt, (T*)B.G, B.rerec);
    else
      rec1d_kernel<T, NV, true><<<rblocks, RB, 0, st>>>(P, W, Bt, S.Uin, S.mask, S.Mod, B.list, cnt, (T*)B.G, B.rerec);
    if (B.prof) B.prof->end(st);
  }
  if (B.prof) B.prof->begin(3, st);
  update1d_kernel<T, NV><<<blocks, UB, 0, st>>>(P, (const T*)B.G, r);
  if (B.prof) B.prof->end(st);
}

}  // namespace

void run_stage_1d(const Prob& P, const HostTabs& T, int prec, const Bufs& B, const StageCall& S, cudaStream_t st) {
  if (P.nvar == 3) {
    if (prec == PREC_FP32) stage_t<float, 3>(P, T.wf, T.b1f, B, S, st);
    else if (prec == PREC_DF64) stage_t<df64, 3>(P, T.wx, T.b1x, B, S, st);
    else stage_t<double, 3>(P, T.wd, T.b1d, B, S, st);
  } else {
    if (prec == PREC_FP32) stage_t<float, 1>(P, T.wf, T.b1f, B, S, st);
    else if (prec == PREC_DF64) stage_t<df64, 1>(P, T.wx, T.b1x, B, S, st);
    else stage_t<double, 1>(P, T.wd, T.b1d, B, S, st);
  }
}

}  // namespace hw
