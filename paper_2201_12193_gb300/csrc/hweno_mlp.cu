// Learned troubled-cell indicator: a 108 -> 64 -> 64 -> 1 MLP (GELU hidden units,
// sigmoid output) over each cell's 3x3 neighbourhood of moments, on BF16 tensor
// cores (mma.sync m16n8k16, FP32 accumulation).  Features, inference, the fused
// forward+backward training kernel, Adam, and the stage kernel that flags cells
// by the network ahead of reconstruction and leaves the cells below the
// confidence threshold to KXRCF.
// No counterpart in the paper: the paper's indicator (KXRCF) stays the label
// source, the fallback and the judge.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "hweno_internal.h"

namespace hw {
namespace {

constexpr int NIN = 108, NINP = 112, NH = 64;
constexpr int S1 = 114;   // row stride (bf16) of 112-wide rows: 57 words (odd), so per-row stores by
                          // 32 threads and the fragment loads hit distinct banks
constexpr int S2 = 72;    // padded row stride of 64-wide rows
constexpr float CLIPF = 8.0f;

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// erf by the rational approximation of Abramowitz & Stegun, Handbook of
// Mathematical Functions, formula 7.1.26 (Hastings): for z >= 0,
// erf z = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-z^2), t = 1 / (1 + p z),
// with |error| <= 1.5e-7, odd extension for z < 0.  About a dozen instructions
// (one reciprocal, one exponential), against the far longer erff: the hidden
// activations are BF16-rounded (2^-9 relative) after this.
__device__ __forceinline__ float erf_as(float z) {
  const float a = fabsf(z);
  const float t = __frcp_rn(fmaf(0.3275911f, a, 1.0f));
  const float poly =
      t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
  return copysignf(1.0f - poly * __expf(-a * a), z);
}

// GELU x Phi(x) = x (1 + erf(x / sqrt 2)) / 2 and its derivative Phi(x) + x phi(x).
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erf_as(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erf_as(x * 0.70710678118654752f)) + x * __expf(-0.5f * x * x) * 0.39894228040143268f;
}

// ---------------------------------------------------------------- features
// Double -> float by the IEEE-754 bit layout (sign, exponent rebias 1023 -> 127,
// mantissa truncated to 23 bits): integer ALU only, no FP64 pipe.  Magnitudes
// below 2^-126 become 0 (the features are normalised and BF16-rounded after
// this, so the truncation's 2^-23 relative error is far below their rounding).
__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7FFu) - (1023 - 127);
  if (e <= 0) return 0.0f;
  if (e >= 255) return __uint_as_float((hi & 0x80000000u) | 0x7F800000u);
  return __uint_as_float((hi & 0x80000000u) | ((unsigned)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

__device__ __forceinline__ float clipf(float x) { return fminf(CLIPF, fmaxf(-CLIPF, x)); }

// 108 normalised features of cell (i, j): per variable and 3x3 cell k (paper
// label order), (ubar_k - ubar_c, vbar_k, wbar_k) / D with
// D = max |ubar_k - ubar_c| + h^2 max |ubar_k| + 1e-12 (h^2 |u| is the scale
// KXRCF compares jumps against), the centre's own average slot holding
// ubar_c / (max |ubar_k| + 1e-12); clipped to [-8, 8]; boundary images as in
// the scheme.  The differences ubar_k - ubar_c are taken in FP64 (they cancel),
// everything after in FP32.  emit(q, value) receives feature q.
template <typename Emit>
__device__ __forceinline__ void cell_features(const Prob& P, const double* __restrict__ U, int i, int j, Emit emit) {
  int xi[3], xs[3], yj[3], ys[3], xn[3], yn[3];
#pragma unroll
  for (int o = -1; o <= 1; ++o) {
    const Img a = image(P, i + o, j), b = image(P, i, j + o);
    xi[o + 1] = a.i; xs[o + 1] = a.sx; yj[o + 1] = b.j; ys[o + 1] = b.sy; xn[o + 1] = a.neg; yn[o + 1] = b.neg;
  }
  const float h2 = (float)(P.dx * P.dx);
#pragma unroll 1
  for (int v = 0; v < 4; ++v) {
    const double* U0 = U + (long long)(v * 3) * P.plane;
    const double* U1 = U0 + P.plane;
    const double* U2 = U1 + P.plane;
    const long long oc = (long long)yj[1] * P.pitch + xi[1];
    const double uc = U0[oc];
    float du[9], vb[9], wb[9];
    float D = 0.f, umax = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int ox = k % 3, oy = k / 3;
      const long long so = (long long)yj[oy] * P.pitch + xi[ox];
      const bool wall = ((xn[ox] | yn[oy]) >> v) & 1;     // reflective image: normal momentum negated
      const double uk = wall ? -U0[so] : U0[so];
      du[k] = d2f_trunc(uk - uc);
      umax = fmaxf(umax, fabsf(d2f_trunc(uk)));
      D = fmaxf(D, fabsf(du[k]));
      float a = d2f_trunc(U1[so]), b = d2f_trunc(U2[so]);
      if (wall) { a = -a; b = -b; }
      vb[k] = xs[ox] < 0 ? -a : a;
      wb[k] = ys[oy] < 0 ? -b : b;
    }
    const float inv = 1.0f / (D + h2 * umax + 1e-12f);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      emit(v * 27 + k, k == 4 ? clipf(d2f_trunc(uc) / (umax + 1e-12f)) : clipf(du[k] * inv));
      emit(v * 27 + 9 + k, clipf(vb[k] * inv));
      emit(v * 27 + 18 + k, clipf(wb[k] * inv));
    }
  }
}

__global__ void features_kernel(Prob P, const double* __restrict__ U, const int* __restrict__ cells, int n,
                                float* __restrict__ X) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int c = cells[t];
  float* row = X + (long long)t * NIN;
  cell_features(P, U, c % P.nx, c / P.nx, [&](int q, float x) { row[q] = x; });
}

// ---------------------------------------------------------------- parameters
// Flat FP32 parameters: W1[64][108], b1[64], W2[64][64], b2[64], W3[64], b3[1].
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH, NPARAM = OFF_B3 + 1;

// Forward weights staged in shared memory: BF16 W1 [64][S1] (K padded to 112)
// and W2 [64][S2]; FP32 b1, b2, W3, b3.  (Training adds W2^T.)
struct WSmem {
  __nv_bfloat16 w1[NH * S1];
  __nv_bfloat16 w2[NH * S2];
  float b1[NH], b2[NH], w3[NH], b3;
};

__device__ void load_weights(const float* __restrict__ th, WSmem& S) {
  for (int q = threadIdx.x; q < NH * S1; q += blockDim.x) {
    const int o = q / S1, k = q % S1;
    S.w1[q] = __float2bfloat16_rn(k < NIN ? th[OFF_W1 + o * NIN + k] : 0.0f);
  }
  for (int q = threadIdx.x; q < NH * S2; q += blockDim.x) {
    const int o = q / S2, k = q % S2;
    S.w2[q] = __float2bfloat16_rn(k < NH ? th[OFF_W2 + o * NH + k] : 0.0f);
  }
  for (int q = threadIdx.x; q < NH; q += blockDim.x) {
    S.b1[q] = th[OFF_B1 + q];
    S.b2[q] = th[OFF_B2 + q];
    S.w3[q] = th[OFF_W3 + q];
  }
  if (threadIdx.x == 0) S.b3 = th[OFF_B3];
}

// Forward of one 16-row tile (rows r0.. of Xs, stride S1) by one warp.
// Leaves a1, a2 (FP32, C-fragment layout), the BF16 A-fragments of h1, and
// the logits of rows g and g+8 (g = lane/4) in z[0], z[1] (all 4 lanes of a group).
struct Frag {
  float a1[8][4];
  float a2[8][4];
  unsigned h1[4][4];
};

__device__ __forceinline__ void tile_forward(const __nv_bfloat16* __restrict__ Xs, int r0, const WSmem& S, Frag& F,
                                             float (&z)[2]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int n = 0; n < 8; ++n) F.a1[n][0] = F.a1[n][1] = F.a1[n][2] = F.a1[n][3] = 0.f;
#pragma unroll
  for (int kb = 0; kb < NINP / 16; ++kb) {
    unsigned a[4];
    const __nv_bfloat16* x0 = Xs + (r0 + g) * S1 + kb * 16 + 2 * t;
    const __nv_bfloat16* x1 = Xs + (r0 + g + 8) * S1 + kb * 16 + 2 * t;
    a[0] = *reinterpret_cast<const unsigned*>(x0);
    a[1] = *reinterpret_cast<const unsigned*>(x1);
    a[2] = *reinterpret_cast<const unsigned*>(x0 + 8);
    a[3] = *reinterpret_cast<const unsigned*>(x1 + 8);
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const __nv_bfloat16* w = S.w1 + (n * 8 + g) * S1 + kb * 16 + 2 * t;
      mma16816(F.a1[n], a, *reinterpret_cast<const unsigned*>(w), *reinterpret_cast<const unsigned*>(w + 8));
    }
  }
  // bias, GELU, BF16 A-fragments of layer 2
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const int c = n * 8 + 2 * t;
    F.a1[n][0] += S.b1[c]; F.a1[n][1] += S.b1[c + 1]; F.a1[n][2] += S.b1[c]; F.a1[n][3] += S.b1[c + 1];
  }
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    F.h1[kb][0] = pack_bf16(gelu(F.a1[2 * kb][0]), gelu(F.a1[2 * kb][1]));
    F.h1[kb][1] = pack_bf16(gelu(F.a1[2 * kb][2]), gelu(F.a1[2 * kb][3]));
    F.h1[kb][2] = pack_bf16(gelu(F.a1[2 * kb + 1][0]), gelu(F.a1[2 * kb + 1][1]));
    F.h1[kb][3] = pack_bf16(gelu(F.a1[2 * kb + 1][2]), gelu(F.a1[2 * kb + 1][3]));
  }
#pragma unroll
  for (int n = 0; n < 8; ++n) F.a2[n][0] = F.a2[n][1] = F.a2[n][2] = F.a2[n][3] = 0.f;
#pragma unroll
  for (int kb = 0; kb < 4; ++kb)
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const __nv_bfloat16* w = S.w2 + (n * 8 + g) * S2 + kb * 16 + 2 * t;
      mma16816(F.a2[n], F.h1[kb], *reinterpret_cast<const unsigned*>(w), *reinterpret_cast<const unsigned*>(w + 8));
    }
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const int c = n * 8 + 2 * t;
    F.a2[n][0] += S.b2[c]; F.a2[n][1] += S.b2[c + 1]; F.a2[n][2] += S.b2[c]; F.a2[n][3] += S.b2[c + 1];
    s0 += gelu(F.a2[n][0]) * S.w3[c] + gelu(F.a2[n][1]) * S.w3[c + 1];
    s1 += gelu(F.a2[n][2]) * S.w3[c] + gelu(F.a2[n][3]) * S.w3[c + 1];
  }
  s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
  s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
  z[0] = s0 + S.b3;
  z[1] = s1 + S.b3;
}

// ---------------------------------------------------------------- dataset inference
constexpr int FT = 128;   // threads (4 warps) and rows per block tile (2 m-tiles per warp)

__global__ void __launch_bounds__(FT) mlp_forward_kernel(const float* __restrict__ th, const float* __restrict__ X,
                                                         int n, float* __restrict__ prob) {
  extern __shared__ __align__(16) unsigned char smem[];
  WSmem& S = *reinterpret_cast<WSmem*>(smem);
  __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(smem + sizeof(WSmem));
  load_weights(th, S);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int base = blockIdx.x * FT; base < n; base += gridDim.x * FT) {
    __syncthreads();
    for (int q = threadIdx.x; q < FT * S1; q += FT) {
      const int r = q / S1, k = q % S1;
      const int row = base + r;
      Xs[q] = __float2bfloat16_rn((row < n && k < NIN) ? X[(long long)row * NIN + k] : 0.0f);
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int r0 = warp * 32 + m * 16;
      Frag F;
      float z[2];
      tile_forward(Xs, r0, S, F, z);
      if (t == 0) {
        const int ra = base + r0 + g, rb = ra + 8;
        if (ra < n) prob[ra] = 1.0f / (1.0f + expf(-z[0]));
        if (rb < n) prob[rb] = 1.0f / (1.0f + expf(-z[1]));
      }
    }
  }
}

// ---------------------------------------------------------------- training
// Fused forward + backward of the weighted mean BCE over tiles of 64 samples
// (one 16-row tile per warp); weight gradients by tensor-core GEMMs over the
// tile's rows from transposed BF16 copies in shared memory; block gradients in
// shared memory, added to the global FP32 gradient once per block.
constexpr int TT = 128, TR = 64;

struct TSmem {
  WSmem W;
  __nv_bfloat16 w2t[NH * S2];     // W2^T
  __nv_bfloat16 xs[TR * S1];      // X tile [row][feature]
  __nv_bfloat16 xt[NINP * S2];    // X^T [feature][row]
  __nv_bfloat16 h1t[NH * S2];     // h1^T
  __nv_bfloat16 da2t[NH * S2];    // (dL/da2)^T
  __nv_bfloat16 da1t[NH * S2];    // (dL/da1)^T
  float gw1[NH * NINP];
  float gw2[NH * NH];
  // per-warp sums (one writer each), combined in warp order at the end
  float gb1[TT / 32][NH], gb2[TT / 32][NH], gw3[TT / 32][NH], gb3[TT / 32], loss[TT / 32];
};

// Sum over the 8 lanes of a warp that share lane & 3, in a fixed tree order.
__device__ __forceinline__ float sum_over_g(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

__global__ void __launch_bounds__(TT) mlp_train_kernel(const float* __restrict__ th, const float* __restrict__ X,
                                                       const float* __restrict__ y, const float* __restrict__ wt,
                                                       int n, float inv_n, float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem[];
  TSmem& S = *reinterpret_cast<TSmem*>(smem);
  load_weights(th, S.W);
  for (int q = threadIdx.x; q < NH * S2; q += TT) {
    const int o = q / S2, k = q % S2;
    S.w2t[q] = __float2bfloat16_rn(k < NH ? th[OFF_W2 + k * NH + o] : 0.0f);
  }
  for (int q = threadIdx.x; q < NH * NINP; q += TT) S.gw1[q] = 0.f;
  for (int q = threadIdx.x; q < NH * NH; q += TT) S.gw2[q] = 0.f;
  for (int q = threadIdx.x; q < (TT / 32) * NH; q += TT) {
    (&S.gb1[0][0])[q] = 0.f; (&S.gb2[0][0])[q] = 0.f; (&S.gw3[0][0])[q] = 0.f;
  }
  if (threadIdx.x < TT / 32) { S.gb3[threadIdx.x] = 0.f; S.loss[threadIdx.x] = 0.f; }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int base = blockIdx.x * TR; base < n; base += gridDim.x * TR) {
    __syncthreads();
    for (int q = threadIdx.x; q < TR * NINP; q += TT) {
      const int r = q / NINP, k = q % NINP;
      const int row = base + r;
      const __nv_bfloat16 v = __float2bfloat16_rn((row < n && k < NIN) ? X[(long long)row * NIN + k] : 0.0f);
      S.xs[r * S1 + k] = v;
      S.xt[k * S2 + r] = v;
    }
    __syncthreads();
    // ---- per warp: rows r0 .. r0+15 of the tile
    const int r0 = warp * 16;
    Frag F;
    float z[2];
    tile_forward(S.xs, r0, S.W, F, z);
    float dz[2], ls = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = base + r0 + g + 8 * h;
      float d = 0.f;
      if (row < n) {
        const float p = 1.0f / (1.0f + expf(-z[h]));
        const float w = wt ? wt[row] : 1.0f;
        const float yy = y[row];
        d = w * (p - yy) * inv_n;
        ls += -w * (yy * logf(p + 1e-12f) + (1.f - yy) * logf(1.f - p + 1e-12f)) * inv_n;
      }
      dz[h] = d;
    }
    {   // the four lanes of a row hold the same dz: lanes t == 0 count it
      const float lw = sum_over_g(t == 0 ? ls : 0.f), gw = sum_over_g(t == 0 ? dz[0] + dz[1] : 0.f);
      if (lane == 0) { S.loss[warp] += lw; S.gb3[warp] += gw; }
    }
    // layer 3 and layer 2 gradients (C-fragment positions of this thread)
    float da2[8][4];
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) {
      const int c = nb * 8 + 2 * t;
      float gw3a = 0.f, gw3b = 0.f, gb2a = 0.f, gb2b = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float a = F.a2[nb][e];
        const float dzr = dz[e >> 1];
        const float w3 = S.W.w3[c + (e & 1)];
        if (e & 1) gw3b += dzr * gelu(a); else gw3a += dzr * gelu(a);
        da2[nb][e] = dzr * w3 * gelu_grad(a);
        if (e & 1) gb2b += da2[nb][e]; else gb2a += da2[nb][e];
      }
      gw3a = sum_over_g(gw3a); gw3b = sum_over_g(gw3b);
      gb2a = sum_over_g(gb2a); gb2b = sum_over_g(gb2b);
      if (g == 0) {
        S.gw3[warp][c] += gw3a; S.gw3[warp][c + 1] += gw3b;
        S.gb2[warp][c] += gb2a; S.gb2[warp][c + 1] += gb2b;
      }
      // transposed BF16 copies for the weight-gradient GEMMs
      S.da2t[c * S2 + r0 + g] = __float2bfloat16_rn(da2[nb][0]);
      S.da2t[(c + 1) * S2 + r0 + g] = __float2bfloat16_rn(da2[nb][1]);
      S.da2t[c * S2 + r0 + g + 8] = __float2bfloat16_rn(da2[nb][2]);
      S.da2t[(c + 1) * S2 + r0 + g + 8] = __float2bfloat16_rn(da2[nb][3]);
    }
    // h1^T (the BF16 values layer 2 consumed)
#pragma unroll
    for (int kb = 0; kb < 4; ++kb)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&F.h1[kb][e]);
        const int c = kb * 16 + (e >> 1) * 8 + 2 * t, row = r0 + g + (e & 1) * 8;
        S.h1t[c * S2 + row] = v.x;
        S.h1t[(c + 1) * S2 + row] = v.y;
      }
    // dh1 = da2 W2 (B from W2^T), then da1 = dh1 * gelu'(a1)
    unsigned da2f[4][4];
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
      da2f[kb][0] = pack_bf16(da2[2 * kb][0], da2[2 * kb][1]);
      da2f[kb][1] = pack_bf16(da2[2 * kb][2], da2[2 * kb][3]);
      da2f[kb][2] = pack_bf16(da2[2 * kb + 1][0], da2[2 * kb + 1][1]);
      da2f[kb][3] = pack_bf16(da2[2 * kb + 1][2], da2[2 * kb + 1][3]);
    }
    float dh1[8][4];
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) dh1[nb][0] = dh1[nb][1] = dh1[nb][2] = dh1[nb][3] = 0.f;
#pragma unroll
    for (int kb = 0; kb < 4; ++kb)
#pragma unroll
      for (int nb = 0; nb < 8; ++nb) {
        const __nv_bfloat16* w = S.w2t + (nb * 8 + g) * S2 + kb * 16 + 2 * t;
        mma16816(dh1[nb], da2f[kb], *reinterpret_cast<const unsigned*>(w), *reinterpret_cast<const unsigned*>(w + 8));
      }
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) {
      const int c = nb * 8 + 2 * t;
      float gb1a = 0.f, gb1b = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float d = dh1[nb][e] * gelu_grad(F.a1[nb][e]);
        if (e & 1) gb1b += d; else gb1a += d;
        S.da1t[(c + (e & 1)) * S2 + r0 + g + (e >> 1) * 8] = __float2bfloat16_rn(d);
      }
      gb1a = sum_over_g(gb1a); gb1b = sum_over_g(gb1b);
      if (g == 0) { S.gb1[warp][c] += gb1a; S.gb1[warp][c + 1] += gb1b; }
    }
    __syncthreads();
    // weight gradients over the 64 rows of the tile: warp w owns output rows 16w..16w+15
    {
      const int o0 = warp * 16;
      float acc[8][4];
#pragma unroll
      for (int nb = 0; nb < 8; ++nb) acc[nb][0] = acc[nb][1] = acc[nb][2] = acc[nb][3] = 0.f;
#pragma unroll
      for (int kb = 0; kb < TR / 16; ++kb) {
        unsigned a[4];
        const __nv_bfloat16* p0 = S.da2t + (o0 + g) * S2 + kb * 16 + 2 * t;
        const __nv_bfloat16* p1 = S.da2t + (o0 + g + 8) * S2 + kb * 16 + 2 * t;
        a[0] = *reinterpret_cast<const unsigned*>(p0); a[1] = *reinterpret_cast<const unsigned*>(p1);
        a[2] = *reinterpret_cast<const unsigned*>(p0 + 8); a[3] = *reinterpret_cast<const unsigned*>(p1 + 8);
#pragma unroll
        for (int nb = 0; nb < 8; ++nb) {
          const __nv_bfloat16* b = S.h1t + (nb * 8 + g) * S2 + kb * 16 + 2 * t;
          mma16816(acc[nb], a, *reinterpret_cast<const unsigned*>(b), *reinterpret_cast<const unsigned*>(b + 8));
        }
      }
#pragma unroll
      for (int nb = 0; nb < 8; ++nb) {
        const int c = nb * 8 + 2 * t;
        S.gw2[(o0 + g) * NH + c] += acc[nb][0];
        S.gw2[(o0 + g) * NH + c + 1] += acc[nb][1];
        S.gw2[(o0 + g + 8) * NH + c] += acc[nb][2];
        S.gw2[(o0 + g + 8) * NH + c + 1] += acc[nb][3];
      }
      float acc1[14][4];
#pragma unroll
      for (int nb = 0; nb < 14; ++nb) acc1[nb][0] = acc1[nb][1] = acc1[nb][2] = acc1[nb][3] = 0.f;
#pragma unroll
      for (int kb = 0; kb < TR / 16; ++kb) {
        unsigned a[4];
        const __nv_bfloat16* p0 = S.da1t + (o0 + g) * S2 + kb * 16 + 2 * t;
        const __nv_bfloat16* p1 = S.da1t + (o0 + g + 8) * S2 + kb * 16 + 2 * t;
        a[0] = *reinterpret_cast<const unsigned*>(p0); a[1] = *reinterpret_cast<const unsigned*>(p1);
        a[2] = *reinterpret_cast<const unsigned*>(p0 + 8); a[3] = *reinterpret_cast<const unsigned*>(p1 + 8);
#pragma unroll
        for (int nb = 0; nb < 14; ++nb) {
          const __nv_bfloat16* b = S.xt + (nb * 8 + g) * S2 + kb * 16 + 2 * t;
          mma16816(acc1[nb], a, *reinterpret_cast<const unsigned*>(b), *reinterpret_cast<const unsigned*>(b + 8));
        }
      }
#pragma unroll
      for (int nb = 0; nb < 14; ++nb) {
        const int c = nb * 8 + 2 * t;
        S.gw1[(o0 + g) * NINP + c] += acc1[nb][0];
        S.gw1[(o0 + g) * NINP + c + 1] += acc1[nb][1];
        S.gw1[(o0 + g + 8) * NINP + c] += acc1[nb][2];
        S.gw1[(o0 + g + 8) * NINP + c + 1] += acc1[nb][3];
      }
    }
  }
  __syncthreads();
  // this block's gradient and loss into its own row of part (NPARAM + 1 floats);
  // train_sum_kernel adds the rows in block order
  float* row = part + (long long)blockIdx.x * (NPARAM + 1);
  for (int q = threadIdx.x; q < NH * NIN; q += TT) row[OFF_W1 + q] = S.gw1[(q / NIN) * NINP + q % NIN];
  for (int q = threadIdx.x; q < NH * NH; q += TT) row[OFF_W2 + q] = S.gw2[q];
  for (int q = threadIdx.x; q < NH; q += TT) {
    float b1 = 0.f, b2 = 0.f, w3 = 0.f;
#pragma unroll
    for (int w = 0; w < TT / 32; ++w) { b1 += S.gb1[w][q]; b2 += S.gb2[w][q]; w3 += S.gw3[w][q]; }
    row[OFF_B1 + q] = b1;
    row[OFF_B2 + q] = b2;
    row[OFF_W3 + q] = w3;
  }
  if (threadIdx.x == 0) {
    float b3 = 0.f, ls = 0.f;
#pragma unroll
    for (int w = 0; w < TT / 32; ++w) { b3 += S.gb3[w]; ls += S.loss[w]; }
    row[OFF_B3] = b3;
    row[NPARAM] = ls;
  }
}

// grad[q] += sum over blocks b (in order) of part[b][q]; *loss likewise from slot NPARAM.
__global__ void train_sum_kernel(const float* __restrict__ part, int nblocks, float* __restrict__ grad,
                                 float* __restrict__ loss) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > NPARAM) return;
  float s = 0.f;
  for (int b = 0; b < nblocks; ++b) s += part[(long long)b * (NPARAM + 1) + q];
  if (q < NPARAM) grad[q] += s;
  else *loss += s;
}

__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ grad, float* __restrict__ m1,
                            float* __restrict__ m2, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float g = grad[q];
  const float a = b1 * m1[q] + (1.f - b1) * g;
  const float b = b2 * m2[q] + (1.f - b2) * g * g;
  m1[q] = a;
  m2[q] = b;
  th[q] -= lr * (a * c1) / (sqrtf(b * c2) + eps);
}

// ---------------------------------------------------------------- stage kernel
// Learned indicator ahead of Step 1: for every cell the network's probability
// s from the stage input's moments; where the confidence max(s, 1-s) reaches
// conf the network decides (mask 0/1, eq. (vi) for flagged cells), otherwise
// the cell is marked undecided (mask 2) and listed for KXRCF after Step 1.
// Tile 32 x 4 cells, one warp per row; persistent blocks load the weights once.
constexpr int MTX = 32, MTY = 4, MTN = MTX * MTY;

__global__ void __launch_bounds__(MTN) mlpre2d_kernel(Prob P, const float* __restrict__ th, float conf,
                                                      const double* __restrict__ U, uint8_t* __restrict__ mask,
                                                      double* __restrict__ Mod, int* __restrict__ und,
                                                      int* __restrict__ und_count, int* __restrict__ stats,
                                                      float* __restrict__ prob) {
  extern __shared__ __align__(16) unsigned char smem[];
  WSmem& S = *reinterpret_cast<WSmem*>(smem);
  __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(smem + sizeof(WSmem));
  float* zs = reinterpret_cast<float*>(smem + sizeof(WSmem) + MTN * S1 * sizeof(__nv_bfloat16));
  load_weights(th, S);
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int tiles_x = (P.nx + MTX - 1) / MTX, ntiles = tiles_x * ((P.ny + MTY - 1) / MTY);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i = (tile % tiles_x) * MTX + (tid % MTX), j = (tile / tiles_x) * MTY + (tid / MTX);
    const bool valid = i < P.nx && j < P.ny;
    __syncthreads();   // the weights are staged; Xs / zs of the previous tile are free
    {
      __nv_bfloat16* row = Xs + tid * S1;
      if (valid) {
        cell_features(P, U, i, j, [&](int q, float x) { row[q] = __float2bfloat16_rn(x); });
      } else {
        for (int q = 0; q < NIN; q += 2) *reinterpret_cast<unsigned*>(row + q) = 0u;
      }
#pragma unroll
      for (int q = NIN; q < NINP; q += 2) *reinterpret_cast<unsigned*>(row + q) = 0u;   // K padding
    }
    __syncthreads();
    {
      // warp w owns rows 32w .. 32w+31 of the tile (= its own cells)
#pragma unroll 1
      for (int m = 0; m < 2; ++m) {
        const int r0 = warp * 32 + m * 16;
        Frag F;
        float z[2];
        tile_forward(Xs, r0, S, F, z);
        if (t == 0) { zs[r0 + g] = z[0]; zs[r0 + g + 8] = z[1]; }
      }
    }
    __syncwarp();
    bool flag = false, undecided = false;
    if (valid) {
      const float s = 1.0f / (1.0f + expf(-zs[tid]));
      if (prob) prob[(long long)j * P.nx + i] = s;
      if (fmaxf(s, 1.f - s) >= conf) flag = s > 0.5f;
      else undecided = true;
    }
    // warp-aggregated append of the undecided cells (a warp is one tile row)
    const unsigned act = __ballot_sync(0xffffffffu, undecided);
    if (act) {
      const int leader = __ffs(act) - 1;
      int b = 0;
      if (lane == leader) {
        b = atomicAdd(und_count, __popc(act));
        atomicAdd(stats, __popc(act));
      }
      b = __shfl_sync(0xffffffffu, b, leader);
      if (undecided) und[b + __popc(act & ((1u << lane) - 1u))] = j * P.nx + i;
    }
    if (valid) {
      mask[(long long)j * P.nx + i] = undecided ? 2 : (flag ? 1 : 0);
      if (flag) {
        const Img L = image(P, i - 1, j), R = image(P, i + 1, j), Bo = image(P, i, j - 1), Tp = image(P, i, j + 1);
        const long long o = (long long)j * P.pitch + i;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int gL = vsign(L, v), gR = vsign(R, v), gB = vsign(Bo, v), gT = vsign(Tp, v);
          const double uL = gL * U[sidx(P, v, 0, L.i, L.j)], uR = gR * U[sidx(P, v, 0, R.i, R.j)];
          const double vL = gL * L.sx * U[sidx(P, v, 1, L.i, L.j)], vR = gR * R.sx * U[sidx(P, v, 1, R.i, R.j)];
          const double uB = gB * U[sidx(P, v, 0, Bo.i, Bo.j)], uT = gT * U[sidx(P, v, 0, Tp.i, Tp.j)];
          const double wB = gB * Bo.sy * U[sidx(P, v, 2, Bo.i, Bo.j)], wT = gT * Tp.sy * U[sidx(P, v, 2, Tp.i, Tp.j)];
          Mod[(long long)(v * 2 + 0) * P.plane + o] = MOD_WU * (uR - uL) + MOD_WV * (vL + vR);
          Mod[(long long)(v * 2 + 1) * P.plane + o] = MOD_WU * (uT - uB) + MOD_WV * (wB + wT);
        }
      }
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- host launchers

int mlp_nparam() { return NPARAM; }

cudaError_t run_features(const Prob& P, const double* U, const int* cells, int n, float* X, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  features_kernel<<<(n + 127) / 128, 128, 0, st>>>(P, U, cells, n, X);
  return cudaGetLastError();
}

cudaError_t run_mlp_forward(const float* th, const float* X, int n, float* prob, int nsm, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const size_t sm = sizeof(WSmem) + FT * S1 * sizeof(__nv_bfloat16);
  cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int blocks = (int)std::min<long long>((n + FT - 1) / FT, (long long)nsm * 4);
  mlp_forward_kernel<<<blocks, FT, sm, st>>>(th, X, n, prob);
  return cudaGetLastError();
}

cudaError_t run_mlp_train(const float* th, const float* X, const float* y, const float* w, int n, float* grad,
                          float* loss, int nsm, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const size_t sm = sizeof(TSmem);
  cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int blocks = (int)std::min<long long>((n + TR - 1) / TR, (long long)nsm);
  // per-block partial sums, added in block order: the gradient does not depend
  // on the order in which blocks finish (training runs are reproducible)
  static float* part = nullptr;
  static size_t cap = 0;
  const size_t need = (size_t)blocks * (NPARAM + 1);
  if (need > cap) {
    if (part) cudaFree(part);
    part = nullptr;
    cap = 0;
    if ((e = cudaMalloc(&part, need * sizeof(float))) != cudaSuccess) return e;
    cap = need;
  }
  mlp_train_kernel<<<blocks, TT, sm, st>>>(th, X, y, w, n, 1.0f / (float)n, part);
  train_sum_kernel<<<(NPARAM + 1 + 255) / 256, 256, 0, st>>>(part, blocks, grad, loss);
  return cudaGetLastError();
}

cudaError_t run_adam(float* th, const float* grad, float* m1, float* m2, int step, float lr, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f / (1.0f - powf(b1, (float)step)), c2 = 1.0f / (1.0f - powf(b2, (float)step));
  adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(th, grad, m1, m2, NPARAM, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

cudaError_t run_mlpre2d(const Prob& P, const float* th, float conf, const double* U, uint8_t* mask, double* Mod,
                        int* und, int* und_count, int* stats, float* prob, cudaStream_t st) {
  const size_t sm = sizeof(WSmem) + MTN * S1 * sizeof(__nv_bfloat16) + MTN * sizeof(float);
  const long long ntiles = (long long)((P.nx + MTX - 1) / MTX) * ((P.ny + MTY - 1) / MTY);
  const unsigned grd = (unsigned)std::min<long long>(ntiles, (long long)P.nsm * 4);   // 4 blocks fit an SM
  cudaError_t e = cudaFuncSetAttribute(mlpre2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  mlpre2d_kernel<<<grd, MTN, sm, st>>>(P, th, conf, U, mask, Mod, und, und_count, stats, prob);
  return cudaGetLastError();
}

}  // namespace hw
