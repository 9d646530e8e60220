// One fused kernel per Runge-Kutta stage in 1D (Sec. 2.1, Steps 1-3): the
// moments of a segment of S cells and a halo of 4 on each side enter shared
// memory once; the point values of Step 1, the KXRCF flags and eq. (vi) of
// Step 2, the troubled re-reconstruction of Step 2.3, the face fluxes, the
// quadrature of eq. (F), L(U) and the Runge-Kutta combination then run on
// shared memory, and only the stage input, U^n and the outputs touch HBM.
//
// The halo follows the dependencies: the fluxes of the owned cells' faces need
// point values of cells -1 .. S; their re-reconstruction needs flags and
// modified moments of -2 .. S + 1; those need point values of -3 .. S + 2,
// which need moments of -4 .. S + 3.
//
// Ghost positions beyond a non-periodic side are not reconstructed: they take
// their image's point values, flag and modified moments with the image's signs,
// exactly as the multi-launch pipeline reads them through image(); beyond a
// periodic side the window holds the real cells of the other end, computed like
// any other.  Every step uses the pipeline's own device functions and
// arithmetic, so the two give bitwise the same states.
//
// Two shapes: segments of 250 cells on 256 threads for long grids (the 256
// positions of Step 1 fill the block NV times over, the flags, faces and cells
// one pass each), and segments of 32 cells on 128 threads for short ones, so
// that a grid of a few thousand cells still spreads over the SMs.
#pragma once

namespace hw {
namespace {

template <typename T, int NV, int S>
struct Fused1dSmem {
  static constexpr int W = S + 8;   // window: owned + 4 each side
  double U[2 * NV][W];   // moments with the image signs applied (FP64: eq. (vi) and the state)
  T UT[2 * NV][W];       // the same in the compute precision (the reconstruction's input)
  T G[4 * NV][W];        // point values
  T V[2][W];             // KXRCF velocities at the left and right end points
  double Mod[NV][W];     // modified first moments of flagged positions
  T FX[S + 1][NV];       // face fluxes, FX[c] left of owned cell c
  uint8_t F[W];          // troubled flags
  short list[W];         // flagged positions to re-reconstruct
  int nlist;
  int nown;              // owned troubled cells (the re-reconstruction count)
};

// A double in the compute precision by integer work where that matters (FP32:
// the same rounding as the FP64 conversion); double-float by its split.
template <typename T> __device__ __forceinline__ T f1_conv(double x) { return from_double<T>(x); }
template <> __device__ __forceinline__ float f1_conv<float>(double x) { return f32_rn(x); }

// Window position p holds cell i0 - 4 + p.  A ghost beyond a non-periodic side
// mirrors a real cell of the window; in the last (ragged) segment the positions
// more than 4 cells past the right side feed no owned cell and stay unused
// (their images could lie outside the grid).
__device__ __forceinline__ bool f1_mirror(const Prob& P, int i) {
  return (i < 0 && P.bc[0] != BC_PERIODIC) || (i >= P.nx && i < P.nx + 4 && P.bc[1] != BC_PERIODIC);
}
__device__ __forceinline__ bool f1_dead(const Prob& P, int i) { return i >= P.nx + 4 && P.bc[1] != BC_PERIODIC; }

// x with its sign flipped when neg (the image sign of a ghost): integer work,
// equal to the pipeline's multiplication by -1 for every non-NaN x
__device__ __forceinline__ double f1_flip(double x, bool neg) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)neg << 63));
}

template <typename T, int NV, int S, int NT>
__global__ void __launch_bounds__(NT) fused1d_kernel(Prob P, Weights<T> W, Beta1<T> B, Rk1 R,
                                                     uint8_t* __restrict__ mask, double* __restrict__ ModOut,
                                                     double* __restrict__ aleph,
                                                     unsigned long long* __restrict__ rerec) {
  constexpr int WN = S + 8;
  extern __shared__ __align__(16) unsigned char f1_smem[];
  Fused1dSmem<T, NV, S>& sm = *reinterpret_cast<Fused1dSmem<T, NV, S>*>(f1_smem);
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * S;
  if (R.dtp) {
    R.dt = *R.dtp;
    if (R.dt < 0.0) {   // a skipped step (block-uniform): the state passes through unchanged
      for (int c = tid; c < S; c += NT) {
        const int i = i0 + c;
        if (i < P.nx && !R.Lout)
          for (int q = 0; q < NV * 2; ++q) R.Uout[(long long)q * P.plane + i] = R.Uin[(long long)q * P.plane + i];
      }
      return;
    }
  }
  if (tid == 0) { sm.nlist = 0; sm.nown = 0; }
  // ---- moments of the window, image signs applied (load_mom1 of the pipeline)
  for (int p = tid; p < WN; p += NT) {
    sm.F[p] = 0;
    if (f1_dead(P, i0 - 4 + p)) {
#pragma unroll
      for (int q = 0; q < 2 * NV; ++q) { sm.U[q][p] = 0.0; sm.UT[q][p] = T(0); }
      continue;
    }
    const Img m = image(P, i0 - 4 + p, 0);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const bool ng = (m.neg >> v) & 1;
      const double u = f1_flip(R.Uin[sidx(P, v, 0, m.i, 0)], ng);
      const double vv = f1_flip(R.Uin[sidx(P, v, 1, m.i, 0)], ng != (m.sx < 0));
      sm.U[2 * v][p] = u;
      sm.U[2 * v + 1][p] = vv;
      sm.UT[2 * v][p] = f1_conv<T>(u);
      sm.UT[2 * v + 1][p] = f1_conv<T>(vv);
    }
  }
  __syncthreads();
  // ---- Step 1: point values of positions 1 .. WN - 2 (cells -3 .. S + 2)
  for (int t = tid; t < (WN - 2) * NV; t += NT) {
    const int v = t / (WN - 2), p = 1 + t % (WN - 2);
    if (f1_mirror(P, i0 - 4 + p) || f1_dead(P, i0 - 4 + p)) continue;
    T d[6];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      d[c] = sm.UT[2 * v][p - 1 + c];
      d[3 + c] = sm.UT[2 * v + 1][p - 1 + c];
    }
    T out[4];
    recon1d<T>(W, B, d, out);
#pragma unroll
    for (int k = 0; k < 4; ++k) sm.G[v * 4 + k][p] = out[k];
  }
  __syncthreads();
  // mirrored ghosts: the image's point values (gl1 of the pipeline)
  auto mirror_G = [&](int plo, int phi) {
    for (int p = plo + tid; p < phi; p += NT) {
      const int i = i0 - 4 + p;
      if (!f1_mirror(P, i)) continue;
      const Img m = image(P, i, 0);
      const int q = m.i - (i0 - 4);
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const T x = sm.G[v * 4 + (m.sx < 0 ? 3 - k : k)][q];
          sm.G[v * 4 + k][p] = (m.neg >> v) & 1 ? -x : x;
        }
    }
  };
  mirror_G(1, WN - 1);
  __syncthreads();
  // ---- Step 2.1 / 2.2: flags and eq. (vi) of positions 2 .. WN - 3 (cells -2 .. S + 1)
  if (P.indicator == IND_KXRCF) {
    // the velocities at both end points of positions 1 .. WN - 2 (a ghost's
    // carry the image's signs, as the pipeline applies them)
    for (int p = 1 + tid; p < WN - 1; p += NT) {
      if (f1_dead(P, i0 - 4 + p)) continue;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int k = s ? 3 : 0;
        if constexpr (NV == 1) sm.V[s][p] = scalar_velocity(P, sm.G[k][p], 0);
        else sm.V[s][p] = sm.G[4 + k][p] / sm.G[k][p];
      }
    }
    __syncthreads();
  }
  for (int p = 2 + tid; p < WN - 2; p += NT) {
    const int i = i0 - 4 + p;
    if (f1_mirror(P, i) || f1_dead(P, i)) continue;
    bool flag = false;
    if (P.indicator == IND_ALL) {
      flag = true;
    } else if (P.indicator == IND_KXRCF) {
      const T vl = T(0.5) * (sm.V[1][p - 1] + sm.V[0][p]);
      const T vr = T(0.5) * (sm.V[1][p] + sm.V[0][p + 1]);
      const T jl = sm.G[0][p] - sm.G[3][p - 1];
      const T jr = sm.G[3][p] - sm.G[0][p + 1];
      T nrm = T(0);
#pragma unroll
      for (int k = 0; k < 4; ++k) nrm = tmax(nrm, tabs(sm.G[k][p]));
      const T a = kxrcf1<T>(P, jl, jr, vl, vr, nrm);
      if (aleph && p >= 4 && p < 4 + S && i < P.nx) aleph[i] = double(a);
      flag = a > T(1);
    }
    sm.F[p] = flag ? 1 : 0;
    if (flag) {
#pragma unroll
      for (int v = 0; v < NV; ++v)
        sm.Mod[v][p] = mod1(sm.U[2 * v][p - 1], sm.U[2 * v][p + 1], sm.U[2 * v + 1][p - 1], sm.U[2 * v + 1][p + 1]);
    }
  }
  __syncthreads();
  if (P.indicator != IND_NONE) {
    // mirrored ghosts take their image's flag and modified moments (load_mom1<true> of the pipeline)
    for (int p = 2 + tid; p < WN - 2; p += NT) {
      const int i = i0 - 4 + p;
      if (!f1_mirror(P, i)) continue;
      const Img m = image(P, i, 0);
      const int q = m.i - (i0 - 4);
      sm.F[p] = sm.F[q];
      if (sm.F[q]) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int g = vsign(m, v);
          sm.Mod[v][p] = m.sx < 0 ? -g * sm.Mod[v][q] : g * sm.Mod[v][q];
        }
      }
    }
    __syncthreads();
    // ---- Step 2.3: flagged positions 3 .. WN - 4 (cells -1 .. S) again, from the modified moments
    for (int p = 3 + tid; p < WN - 3; p += NT) {
      const int i = i0 - 4 + p;
      if (!sm.F[p] || f1_mirror(P, i)) continue;
      sm.list[atomicAdd(&sm.nlist, 1)] = (short)p;
      if (p >= 4 && p < 4 + S && i < P.nx) atomicAdd(&sm.nown, 1);
    }
    __syncthreads();
    const int nl = sm.nlist;
    for (int t = tid; t < nl * NV; t += NT) {
      const int v = t / nl, p = sm.list[t % nl];
      T d[6];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int q = p - 1 + c;
        d[c] = sm.UT[2 * v][q];
        d[3 + c] = sm.F[q] ? f1_conv<T>(sm.Mod[v][q]) : sm.UT[2 * v + 1][q];
      }
      T out[4];
      recon1d<T>(W, B, d, out);
#pragma unroll
      for (int k = 0; k < 4; ++k) sm.G[v * 4 + k][p] = out[k];
    }
    __syncthreads();
    if (nl) {   // block-uniform
      mirror_G(3, WN - 3);
      __syncthreads();
    }
    if (tid == 0 && rerec && sm.nown) atomicAdd(rerec, (unsigned long long)sm.nown);
  }
  // ---- Step 3: the face fluxes (face c left of owned cell c; one call site as in the pipeline)
  for (int c = tid; c <= S; c += NT) {
    if (i0 + c - 1 >= P.nx) continue;
    T uL[NV], uR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      uL[v] = sm.G[v * 4 + 3][3 + c];
      uR[v] = sm.G[v * 4][4 + c];
    }
    num_flux<T, NV>(P, uL, uR, 0, sm.FX[c]);
  }
  __syncthreads();
  for (int c = tid; c < S; c += NT) {
    const int i = i0 + c, p = 4 + c;
    if (i >= P.nx) return;
    T u[4][NV], Fq[NV];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int v = 0; v < NV; ++v) u[k][v] = sm.G[v * 4 + k][p];
    quad1<T, NV>(P, u, Fq);
    const bool flagged = sm.F[p] != 0;
    mask[i] = flagged ? 1 : 0;
    double uin[2 * NV];   // the stage input (an owned cell's moments carry no sign)
#pragma unroll
    for (int q = 0; q < 2 * NV; ++q) uin[q] = sm.U[q][p];
    if (flagged) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double mv = sm.Mod[v][p];
        if (R.Lout || P.persist) uin[2 * v + 1] = mv;
        if (ModOut) ModOut[(long long)v * P.plane + i] = mv;
      }
    }
    rk1_cell<T, NV>(P, R, i, sm.FX[c + 1], sm.FX[c], Fq, uin);
  }
}

}  // namespace
}  // namespace hw
