// One fused kernel per Runge-Kutta stage for 2D Euler (Sec. 2.2, Steps 1-3):
// reconstruction, KXRCF and the first-moment modification, troubled-cell
// re-reconstruction, HLLC fluxes, Gauss-Lobatto quadratures, L(U) and the
// Runge-Kutta combination, with the point values kept in shared memory.
//
// Each block owns a strip segment of FZ_W columns x H rows and sweeps it from
// bottom to top.  A row of moments (FZ_W + 8 columns: the halo of 4 the
// stage needs) enters a 5-row ring in shared memory per iteration, and every
// later step of the stage runs one row behind the step it depends on:
//   moments row j+4 -> point values row j+3 -> KXRCF and eq. (vi) row j+2 ->
//   troubled re-reconstruction row j+1 -> fluxes, quadrature, update row j.
// Rows are therefore reconstructed once per segment (plus 6 halo rows per
// segment) and columns FZ_WC / FZ_W times.  Nothing but the stage input, the
// Runge-Kutta operands and the outputs touches global memory.
//
// Boundary images (periodic, transmissive, reflective) are applied when the
// moments enter shared memory: ghost cells become ordinary window cells (their
// averages, signed first moments and wall-negated momenta), so every later
// step reads plain neighbours.  A ghost cell's point values, flag and modified
// moments are then those of its image up to rounding (the reconstruction and
// the indicator are mirror-equivariant), where the multi-launch pipeline maps
// them exactly.
#pragma once

namespace hw {
namespace {

constexpr int FZ_WC = 32;              // window columns of point values: owned + 3 each side
constexpr int FZ_W = FZ_WC - 6;        // owned columns per block
constexpr int FZ_MC = FZ_WC + 2;       // window columns of moments: owned + 4 each side
constexpr int FZ_NT = 4 * FZ_WC;       // threads: one per (column, variable) in the reconstruction
constexpr int FZ_H = 64;               // owned rows per block

template <typename T>
struct FusedSmem {
  T G[4][4][16][FZ_WC];      // point values of 4 rows (ring by row): pass 1, then final
  T M[5][12][FZ_MC];         // moments of 5 rows (ring) in the compute precision, plane var*3 + moment
  double Mod[3][8][FZ_WC];   // modified first moments (FP64), plane var*2 + (moment-1), 3 rows (ring)
  T A[3][5][FZ_WC];          // KXRCF partials: face velocities x-, x+, y-, y+ and the density norm
  T XF[FZ_W + 1][4][4];      // x-face fluxes of the row being updated [face][point][var]
  T YF[2][FZ_W][4][4];       // y-face fluxes below rows (ring of 2) [face][point][var]
  uint8_t F[3][FZ_WC];       // troubled flags of 3 rows (ring)
  int list[FZ_WC];           // flagged columns of the row being re-reconstructed
  int nlist;
  unsigned nrerec;           // owned cells re-reconstructed by this block
};

__device__ __forceinline__ int ring5(int r) { return (r + 20) % 5; }   // rows >= -4
__device__ __forceinline__ int ring4(int r) { return (r + 20) & 3; }
// Butterfly shuffle of a value of the compute precision (all 32 lanes take part).
template <typename T> __device__ __forceinline__ T shfl_xor_t(T x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }
template <> __device__ __forceinline__ df64 shfl_xor_t<df64>(df64 x, int o) {
  return df64(__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o));
}
__device__ __forceinline__ int ring3(int r) { return (r + 21) % 3; }
__device__ __forceinline__ int iclamp(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Modified first moments of eq. (vi), dimension by dimension (Step 2.2), of the
// window cell at (i, j) (a ghost position allowed: its value in the ghost's own
// frame), from the FP64 stage input through the boundary images.
template <int NV>
__device__ __forceinline__ void fz_modify(const Prob& P, const double* __restrict__ U, int i, int j,
                                          double (&mod)[8]) {
  i = iclamp(i, -3, P.nx + 2);
  j = iclamp(j, -3, P.ny + 2);
  const Img L = image_kind(P, i - 1, j), R = image_kind(P, i + 1, j), Bo = image_kind(P, i, j - 1),
            Tp = image_kind(P, i, j + 1);
  auto mom = [&](const Img& m, int v, int kind) -> double {
    const int g = vsign(m, v) * (kind == 1 ? m.sx : kind == 2 ? m.sy : 1);
    return g * U[sidx(P, v, kind, m.i, m.j)];
  };
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double uL = mom(L, v, 0), uR = mom(R, v, 0), vL = mom(L, v, 1), vR = mom(R, v, 1);
    const double uB = mom(Bo, v, 0), uT = mom(Tp, v, 0), wB = mom(Bo, v, 2), wT = mom(Tp, v, 2);
    mod[v * 2 + 0] = MOD_WU * (uR - uL) + MOD_WV * (vL + vR);
    mod[v * 2 + 1] = MOD_WU * (uT - uB) + MOD_WV * (wB + wT);
  }
}

// KXRCF value (eq. (KXRCF_), (line-integral-average_)) of window column c of
// the row in ring slots (g: point values of rows below / at / above; a: partials).
template <typename T>
__device__ __forceinline__ T fz_kxrcf(const Prob& P, const FusedSmem<T>& sm, int gb, int gc, int gt, int ab, int ac,
                                      int at, int c) {
  const T vxl = T(0.5) * (sm.A[ac][1][c - 1] + sm.A[ac][0][c]);
  const T vxr = T(0.5) * (sm.A[ac][1][c] + sm.A[ac][0][c + 1]);
  const T vyb = T(0.5) * (sm.A[ab][3][c] + sm.A[ac][2][c]);
  const T vyt = T(0.5) * (sm.A[ac][3][c] + sm.A[at][2][c]);
  const T dx = pc<T>(P.cdx), dy = pc<T>(P.cdy);
  T s = T(0), len = T(0);
  if (vxl > T(KX_VDEAD)) {
#pragma unroll
    for (int l = 0; l < 4; ++l) s += dy * gl_w<T>(l) * (sm.G[gc][0][l][c] - sm.G[gc][0][12 + l][c - 1]);
    len += dy;
  }
  if (-vxr > T(KX_VDEAD)) {
#pragma unroll
    for (int l = 0; l < 4; ++l) s += dy * gl_w<T>(l) * (sm.G[gc][0][12 + l][c] - sm.G[gc][0][l][c + 1]);
    len += dy;
  }
  if (vyb > T(KX_VDEAD)) {
#pragma unroll
    for (int k = 0; k < 4; ++k) s += dx * gl_w<T>(k) * (sm.G[gc][0][k * 4][c] - sm.G[gb][0][k * 4 + 3][c]);
    len += dx;
  }
  if (-vyt > T(KX_VDEAD)) {
#pragma unroll
    for (int k = 0; k < 4; ++k) s += dx * gl_w<T>(k) * (sm.G[gc][0][k * 4 + 3][c] - sm.G[gt][0][k * 4][c]);
    len += dx;
  }
  const T nrm = sm.A[ac][4][c];
  if (len == T(0) || nrm == T(0)) return T(0);
  return tabs(s) / len / (pc<T>(P.cdx2) * nrm);
}

struct FzOut {
  uint8_t* mask;                 // this stage's flags [ny][nx]
  double* Mod;                   // modified first moments of owned troubled cells (state planes)
  double* aleph;                 // optional KXRCF values [ny][nx]
  unsigned long long* rerec;     // cells reconstructed a second time (accumulates)
};

template <typename T>
__global__ void __launch_bounds__(FZ_NT, sizeof(T) == 4 ? 4 : 2)
    fused2d_kernel(Prob P, Weights<T> W, Beta2<T> B, Rk S, FzOut O) {
  static_assert(FZ_WC == 32, "one warp spans the window's columns");
  extern __shared__ __align__(16) unsigned char fz_raw[];
  FusedSmem<T>& sm = *reinterpret_cast<FusedSmem<T>*>(fz_raw);
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * FZ_W, j0 = blockIdx.y * FZ_H;
  const int hown = min(FZ_H, P.ny - j0);
  if (tid == 0) sm.nrerec = 0;
  double dt = S.dt;
  if (S.dtp) {
    dt = *S.dtp;
    if (dt < 0.0) {   // a skipped step (hweno_advance): the owned cells pass through unchanged
      if (!S.Lout)
        for (int t = tid; t < 12 * FZ_W * hown; t += FZ_NT) {
          const int q = t / (FZ_W * hown), r = t % (FZ_W * hown);
          const int i = i0 + r % FZ_W, j = j0 + r / FZ_W;
          if (i < P.nx) {
            const long long si = (long long)q * P.plane + (long long)j * P.pitch + i;
            S.Uout[si] = S.Uin[si];
          }
        }
      return;
    }
  }
  const bool kx = P.indicator == IND_KXRCF;
  // A moment row is loaded one iteration ahead (registers) and stored into the
  // ring at the start of the next, so its memory latency overlaps a whole
  // iteration of arithmetic; likewise the Runge-Kutta operands of the row
  // being updated are loaded at the start of its iteration.
  constexpr int NPRE = (12 * FZ_MC + FZ_NT - 1) / FZ_NT;
  double pre[NPRE];
  unsigned preneg = 0;
  auto prefetch = [&](int jrow) {
    const int jc = iclamp(jrow, -4, P.ny + 3);
    preneg = 0;
#pragma unroll
    for (int u = 0; u < NPRE; ++u) {
      const int t = tid + u * FZ_NT;
      pre[u] = 0.0;
      if (t < 12 * FZ_MC) {
        const int pl = t / FZ_MC, cm = t - pl * FZ_MC;
        const int var = pl / 3, mom = pl - var * 3;
        const Img m = image_kind(P, iclamp(i0 - 4 + cm, -4, P.nx + 3), jc);
        pre[u] = S.Uin[sidx(P, var, mom, m.i, m.j)];
        unsigned neg = (m.neg >> var) & 1;
        if (mom == 1 && m.sx < 0) neg ^= 1u;
        if (mom == 2 && m.sy < 0) neg ^= 1u;
        preneg |= neg << u;
      }
    }
  };
  prefetch(j0 - 4);
  // Ghost cells at non-periodic sides: a ghost's flag is its image's (the
  // indicator's inflow faces are not mirror-symmetric at a transmissive side,
  // where the normal velocity keeps its sign), and the point values of the
  // ghost next to the side are the mirrored final values of its image, as the
  // pipeline reads them.  Image column (window) / row of a position, or the
  // position itself where the side is periodic or the cell is inside.
  auto img_col = [&](int c) -> int {
    const int i = i0 - 3 + c;
    if (i < 0 && P.bc[0] != BC_PERIODIC) return -1 - i - i0 + 3;
    if (i >= P.nx && P.bc[1] != BC_PERIODIC) return 2 * P.nx - 1 - i - i0 + 3;
    return c;
  };
  auto img_row = [&](int r) -> int {
    if (r < 0 && P.bc[2] != BC_PERIODIC) return -1 - r;
    if (r >= P.ny && P.bc[3] != BC_PERIODIC) return 2 * P.ny - 1 - r;
    return r;
  };
  for (int q = 0; q < hown + 8; ++q) {
    const int jm = j0 - 4 + q;   // moments enter; rows jm-1, jm-2, jm-3, jm-4 follow
    // ---- Step 0: the prefetched row of moments into the ring, boundary images applied
    {
      const int s5 = ring5(jm);
#pragma unroll
      for (int u = 0; u < NPRE; ++u) {
        const int t = tid + u * FZ_NT;
        if (t < 12 * FZ_MC) {
          const int pl = t / FZ_MC, cm = t - pl * FZ_MC;
          const double x = ((preneg >> u) & 1u) ? -pre[u] : pre[u];
          // FP32 bulk: round with integer operations (no FP64 instruction per moment)
          if constexpr (std::is_same<T, float>::value) sm.M[s5][pl][cm] = f32_rn(x);
          else sm.M[s5][pl][cm] = from_double<T>(x);
        }
      }
    }
    if (q + 1 < hown + 8) prefetch(jm + 1);
    // the Runge-Kutta operands of row jm - 4 (updated at the end of this iteration)
    double rin[3] = {0.0, 0.0, 0.0}, rn[3] = {0.0, 0.0, 0.0};
    bool rfn = false;
    if (q >= 8 && tid < 4 * FZ_W && i0 + (tid >> 2) < P.nx) {
      const int ju = jm - 4, i = i0 + (tid >> 2), v = tid & 3;
      const long long so = (long long)ju * P.pitch + i;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const long long si = (long long)(v * 3 + m) * P.plane + so;
        rin[m] = S.Uin[si];
        if (!S.Lout && S.cA != 0.0) rn[m] = S.Un[si];
      }
      rfn = P.persist && S.maskN && S.maskN[(long long)ju * P.nx + i] != 0;
    }
    __syncthreads();
    // ---- Step 1: point values of row jg, every window column, one variable per thread
    const int jg = jm - 1;
    if (q >= 2) {
      const int c = tid % FZ_WC, v = tid / FZ_WC;
      T d[23];
#pragma unroll
      for (int e = 0; e < 23; ++e) {
        int kind, ox, oy;
        d4_slot(e, kind, ox, oy);
        d[e] = sm.M[ring5(jg + oy)][v * 3 + kind][c + 1 + ox];
      }
      T out[16];
      recon2d<T>(W, B, d, out);
      const int s4 = ring4(jg);
#pragma unroll
      for (int p = 0; p < 16; ++p) sm.G[s4][v][p][c] = out[p];
    }
    __syncthreads();
    // KXRCF partials of row jg: GL-weighted face velocities and the density norm
    if (q >= 2 && tid < FZ_WC) {
      const int c = tid, s5 = ring4(jg), s3 = ring3(jg);
      T nrm = T(0);
#pragma unroll
      for (int p = 0; p < 16; ++p) nrm = tmax(nrm, tabs(sm.G[s5][0][p][c]));
      constexpr int bp[12] = {0, 1, 2, 3, 4, 7, 8, 11, 12, 13, 14, 15};
      T rinv[16];
      if constexpr (sizeof(T) == 8) {
        T x[12], r[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) x[k] = sm.G[s5][0][bp[k]][c];
        batch_inverse_ranged<12, T>(x, r);
#pragma unroll
        for (int k = 0; k < 12; ++k) rinv[bp[k]] = r[k];
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) rinv[bp[k]] = rcp(sm.G[s5][0][bp[k]][c]);
      }
      T pxl = T(0), pxr = T(0), pyb = T(0), pyt = T(0);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        pxl += gl_w<T>(l) * (sm.G[s5][1][l][c] * rinv[l]);
        pxr += gl_w<T>(l) * (sm.G[s5][1][12 + l][c] * rinv[12 + l]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        pyb += gl_w<T>(k) * (sm.G[s5][2][k * 4][c] * rinv[k * 4]);
        pyt += gl_w<T>(k) * (sm.G[s5][2][k * 4 + 3][c] * rinv[k * 4 + 3]);
      }
      sm.A[s3][0][c] = pxl;
      sm.A[s3][1][c] = pxr;
      sm.A[s3][2][c] = pyb;
      sm.A[s3][3][c] = pyt;
      sm.A[s3][4][c] = nrm;
    }
    __syncthreads();
    // ---- Steps 2.1-2.2: flags and modified first moments of row jf
    const int jf = jm - 2;
    if (q >= 4 && tid < FZ_WC) {
      const int c = tid, s3 = ring3(jf);
      bool flag = false;
      T a = T(0);
      if (c >= 1 && c <= FZ_WC - 2) {
        if (P.indicator == IND_ALL) flag = true;
        else if (kx) {
          a = fz_kxrcf<T>(P, sm, ring4(jf - 1), ring4(jf), ring4(jf + 1), ring3(jf - 1), s3, ring3(jf + 1), c);
          flag = a > T(1);
        }
      }
      sm.F[s3][c] = flag ? 1 : 0;
      const int i = i0 - 3 + c;
      double mod[8];
      // a ghost's modified moments are needed wherever its image is troubled
      if (flag || img_col(c) != c || img_row(jf) != jf) {
        fz_modify<4>(P, S.Uin, i, jf, mod);
#pragma unroll
        for (int k = 0; k < 8; ++k) sm.Mod[s3][k][c] = mod[k];
      }
      if (c >= 3 && c < 3 + FZ_W && i < P.nx && jf >= j0 && jf < j0 + hown) {
        const long long cell = (long long)jf * P.nx + i;
        O.mask[cell] = flag ? 1 : 0;
        if (O.aleph && kx) O.aleph[cell] = double(a);
        if (flag) {
          const long long so = (long long)jf * P.pitch + i;
#pragma unroll
          for (int k = 0; k < 8; ++k) O.Mod[(long long)k * P.plane + so] = mod[k];
          atomicAdd(&sm.nrerec, 1u);
        }
      }
    }
    __syncthreads();
    // ---- Step 2.3: re-reconstruct the troubled cells of row jr from the modified moments
    const int jr = jm - 3;
    if (q >= 6 && P.indicator != IND_NONE) {
      if (tid < 32) {
        const bool f = tid >= 2 && tid <= FZ_WC - 3 && sm.F[ring3(jr)][tid];
        const unsigned b = __ballot_sync(0xffffffffu, f);
        if (f) sm.list[__popc(b & ((1u << tid) - 1u))] = tid;
        if (tid == 0) sm.nlist = __popc(b);
      }
      __syncthreads();
      const int n = sm.nlist;
      for (int it = tid; it < 4 * n; it += FZ_NT) {
        const int c = sm.list[it % n], v = it / n;
        T d[23];
#pragma unroll
        for (int e = 0; e < 23; ++e) {
          int kind, ox, oy;
          d4_slot(e, kind, ox, oy);
          const int r3 = ring3(jr + oy);
          // the stencil cell's flag, a ghost's taken from its image (when the
          // image's row is in the ring; else the ghost itself is being
          // re-reconstructed, and its values are replaced by the mirror below)
          int fr = img_row(jr + oy), fc = img_col(c + ox);
          if (fr < jr - 1 || fr > jr + 1) fr = jr + oy;
          if (fc < 0 || fc >= FZ_WC) fc = c + ox;
          if (kind > 0 && sm.F[ring3(fr)][fc])
            d[e] = from_double<T>(sm.Mod[r3][v * 2 + kind - 1][c + ox]);
          else
            d[e] = sm.M[ring5(jr + oy)][v * 3 + kind][c + 1 + ox];
        }
        T out[16];
        recon2d<T>(W, B, d, out);
        const int s4 = ring4(jr);
#pragma unroll
        for (int p = 0; p < 16; ++p) sm.G[s4][v][p][c] = out[p];
      }
    }
    __syncthreads();
    // ---- ghosts next to non-periodic sides: mirrored final point values of their images
    // (x: the ghost columns of row ju; y: the ghost row below the first row of the
    // grid, one iteration early, and the one above the last row)
    const int ju = jm - 4;
    if (q >= 7) {
      const int cl = 2 - i0, cr = P.nx - i0 + 3;          // window columns of x ghosts i = -1, i = nx
      const bool gl = q >= 8 && cl >= 2 && P.bc[0] != BC_PERIODIC;
      const bool gr = q >= 8 && cr <= FZ_WC - 3 && P.bc[1] != BC_PERIODIC;
      const bool gb = q == 7 && ju + 1 == 0 && P.bc[2] != BC_PERIODIC;
      const bool gt = q >= 8 && ju == P.ny - 1 && P.bc[3] != BC_PERIODIC;
      if (gl || gr || gb || gt) {
        const int s = ring4(ju);
        for (int t = tid; t < 64; t += FZ_NT) {     // x: row ju, (var, point)
          const int v = t >> 4, pt = t & 15, k = pt >> 2, l = pt & 3;
          if (gl) sm.G[s][v][pt][cl] = (v == 1 && P.bc[0] == BC_REFLECTIVE ? T(-1) : T(1)) * sm.G[s][v][(3 - k) * 4 + l][cl + 1];
          if (gr) sm.G[s][v][pt][cr] = (v == 1 && P.bc[1] == BC_REFLECTIVE ? T(-1) : T(1)) * sm.G[s][v][(3 - k) * 4 + l][cr - 1];
        }
        if (gb || gt) {                              // y: ghost row -1 from row 0, or row ny from row ny - 1
          const int sg = gb ? ring4(-1) : ring4(ju + 1), si = gb ? ring4(0) : s;
          const T sgn = P.bc[gb ? 2 : 3] == BC_REFLECTIVE ? T(-1) : T(1);
          for (int t = tid; t < 64 * FZ_WC; t += FZ_NT) {
            const int c = t % FZ_WC, vp = t / FZ_WC, v = vp >> 4, pt = vp & 15, k = pt >> 2, l = pt & 3;
            sm.G[sg][v][pt][c] = (v == 2 ? sgn : T(1)) * sm.G[si][v][k * 4 + 3 - l][c];
          }
        }
      }
      __syncthreads();
    }
    // ---- Step 3: fluxes.  q == 7: the y faces below the segment's first row;
    // q >= 8: the x faces of row ju and the y faces above it
    if (q >= 7) {
      const int s = ring4(ju), st = ring4(ju + 1);
      constexpr int NX = 4 * (FZ_W + 1), NY = 4 * FZ_W;
      const int nx_items = q >= 8 ? NX : 0;
      const int total = nx_items + NY;
      for (int it = tid; it < total; it += FZ_NT) {
        T uL[4], uR[4];
        if (it < nx_items) {
          const int f = it >> 2, l = it & 3;
#pragma unroll
          for (int v = 0; v < 4; ++v) { uL[v] = sm.G[s][v][12 + l][2 + f]; uR[v] = sm.G[s][v][l][3 + f]; }
          num_flux<T, 4>(P, uL, uR, 0, sm.XF[f][l]);
        } else {
          const int g = it - nx_items, f = g >> 2, k = g & 3;
#pragma unroll
          for (int v = 0; v < 4; ++v) { uL[v] = sm.G[s][v][k * 4 + 3][3 + f]; uR[v] = sm.G[st][v][k * 4][3 + f]; }
          num_flux<T, 4>(P, uL, uR, 1, sm.YF[(ju + 1) & 1][f][k]);
        }
      }
    }
    __syncthreads();
    // quadrature, L(U) and the Runge-Kutta combination of row ju: four threads per
    // cell, each the interior quadrature of one Gauss-Lobatto row (k), then one
    // variable's face integrals and moments
    if (q >= 8) {
      // every lane of a warp takes part in the shuffles; lanes past the owned
      // cells (act false) compute on cell 0 and write nothing
      const bool act = tid < 4 * FZ_W;
      const int f = act ? tid >> 2 : 0, g = tid & 3, c = 3 + f, i = i0 + f, s = ring4(ju);
      T Fc[4], Gc[4];
      {
        T rho[4], inv[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) rho[l] = sm.G[s][0][g * 4 + l][c];
        if constexpr (sizeof(T) == 8) batch_inverse<4, T>(rho, inv);
        else {
#pragma unroll
          for (int l = 0; l < 4; ++l) inv[l] = rcp(rho[l]);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) Fc[v] = Gc[v] = T(0);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          T u[4], fx[4], gy[4];
#pragma unroll
          for (int v = 0; v < 4; ++v) u[v] = sm.G[s][v][g * 4 + l][c];
          euler_flux_inv<T, 4>(P, u, inv[l], 0, fx);
          euler_flux_inv<T, 4>(P, u, inv[l], 1, gy);
          const T w = gl_w<T>(g) * gl_w<T>(l);
#pragma unroll
          for (int v = 0; v < 4; ++v) { Fc[v] += w * fx[v]; Gc[v] += w * gy[v]; }
        }
      }
      // sum the four Gauss-Lobatto rows (lanes 4f .. 4f+3 of one warp)
#pragma unroll
      for (int o = 1; o <= 2; o <<= 1)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          Fc[v] += shfl_xor_t(Fc[v], o);
          Gc[v] += shfl_xor_t(Gc[v], o);
        }
      const int v = g;
      T Fp = T(0), Fm = T(0), Fpe = T(0), Fme = T(0), Gp = T(0), Gm = T(0), Gpx = T(0), Gmx = T(0);
      const int yt = (ju + 1) & 1, yb = ju & 1;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const T w = gl_w<T>(l), we = gl_w<T>(l) * gl_x<T>(l);
        Fp += w * sm.XF[f + 1][l][v];
        Fpe += we * sm.XF[f + 1][l][v];
        Fm += w * sm.XF[f][l][v];
        Fme += we * sm.XF[f][l][v];
        Gp += w * sm.YF[yt][f][l][v];
        Gpx += we * sm.YF[yt][f][l][v];
        Gm += w * sm.YF[yb][f][l][v];
        Gmx += we * sm.YF[yb][f][l][v];
      }
      T Fcv = Fc[0], Gcv = Gc[0];
#pragma unroll
      for (int k = 1; k < 4; ++k)
        if (v == k) { Fcv = Fc[k]; Gcv = Gc[k]; }
      // eq. (2D-equ-int-approximation); the average equation in FP64 from the
      // face integrals so that the flux differences telescope in every precision
      const double idx = P.crdx.d, idy = P.crdy.d;
      const T tidx = pc<T>(P.crdx), tidy = pc<T>(P.crdy);
      double L[3];
      L[0] = -(to_f64(Fp) - to_f64(Fm)) * idx - (to_f64(Gp) - to_f64(Gm)) * idy;
      L[1] = to_f64(-(Fp + Fm) * T(0.5) * tidx + Fcv * tidx - (Gpx - Gmx) * tidy);
      L[2] = to_f64(-(Fpe - Fme) * tidx - (Gp + Gm) * T(0.5) * tidy + Gcv * tidy);
      const bool live = act && i < P.nx;
      const bool first = S.cA == 0.0;   // the first stage has no U^n term
      bool finite = true;
      double newavg = 0.0;
      if (live) {
        const long long so = (long long)ju * P.pitch + i;
        const bool fk = sm.F[ring3(ju)][c] != 0 && (P.persist || S.Lout);
        const bool fn = rfn;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          const long long si = (long long)(v * 3 + m) * P.plane + so;
          const double uin = (m > 0 && fk) ? sm.Mod[ring3(ju)][v * 2 + m - 1][c] : rin[m];
          if (S.Lout) {
            S.Lout[si] = L[m];
            if (S.Umod) S.Umod[si] = uin;
            continue;
          }
          double r;
          if (first) {   // U^(1) = U' + dt L
            r = fma(dt, L[m], uin);
          } else {
            const double un = (m > 0 && fn) ? S.ModN[(long long)(v * 2 + m - 1) * P.plane + so] : rn[m];
            r = S.cA * un + S.cB * (uin + dt * L[m]);
          }
          S.Uout[si] = r;
          if (m == 0) newavg = r;
          finite = finite && ((__double_as_longlong(r) >> 52) & 0x7FF) != 0x7FF;
        }
        if (!finite && ju >= P.jlo && ju < P.jhi) atomicOr(S.status, ST_NONFINITE);
      }
      // positivity of the new cell average (lane v = 0 gathers the cell's four variables)
      const int base = (tid & 31) & ~3;
      const double a1 = __shfl_sync(0xffffffffu, newavg, base + 1);
      const double a2 = __shfl_sync(0xffffffffu, newavg, base + 2);
      const double a3 = __shfl_sync(0xffffffffu, newavg, base + 3);
      if (live && v == 0 && !S.Lout && ju >= P.jlo && ju < P.jhi) {
        // p = (gamma - 1)(E - |rho v|^2 / (2 rho)) > 0 with rho > 0, without a division
        const double rho = newavg;
        if (!(rho > 0.0) || !(2.0 * a3 * rho > a1 * a1 + a2 * a2)) atomicOr(S.status, ST_NONPOSITIVE);
      }
    }
    // the next iteration's first writes (moment ring, then after a barrier the
    // point values) touch rows no thread reads any more in this iteration
  }
  __syncthreads();
  if (tid == 0 && O.rerec && P.indicator != IND_NONE && sm.nrerec) atomicAdd(O.rerec, (unsigned long long)sm.nrerec);
}

// Shared memory of the fused kernel for the compute precision T (bytes).
template <typename T>
constexpr size_t fused_smem_bytes() { return sizeof(FusedSmem<T>); }

// The fused stage applies to 2D Euler with KXRCF, every cell or no cell
// troubled, and periodic / transmissive / reflective sides.
inline bool fused_applies(const Prob& P, int nv) {
  return P.fused && nv == 4 && !P.fixtab && P.sol_j == 0 &&
         (P.indicator == IND_NONE || P.indicator == IND_KXRCF || P.indicator == IND_ALL);
}

template <typename T>
cudaError_t launch_fused2d(const Prob& P, const Weights<T>& W, const Beta2<T>& Bt, const Rk& r, const FzOut& O,
                           cudaStream_t st) {
  const size_t smem = fused_smem_bytes<T>();
  cudaError_t e = cudaFuncSetAttribute(fused2d_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((P.nx + FZ_W - 1) / FZ_W, (P.ny + FZ_H - 1) / FZ_H);
  fused2d_kernel<T><<<grid, FZ_NT, smem, st>>>(P, W, Bt, r, O);
  return cudaGetLastError();
}

}  // namespace
}  // namespace hw
