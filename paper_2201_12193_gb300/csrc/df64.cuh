// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers, giving a 48-bit significand with FP32's exponent range.  On this
// GPU FP32 runs ~60x faster than FP64, so a df64 operation of 6-20 FP32
// instructions is still several times cheaper than an FP64 one.
//
// The operations are the classical error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly;
//   FastTwoSum (Dekker 1971): the same when |a| >= |b|;
//   TwoProd with a fused multiply-add: p + e = a * b exactly;
// combined as in the double-double arithmetic of Dekker (1971) and Hida, Li &
// Bailey (QD library, 2001), in their "sloppy" (cheaper) addition, whose error
// is bounded by about 2^-47 (|a| + |b|).  Every FP32 step uses the _rn
// intrinsics, which the compiler never contracts into FMAs (contraction would
// break the exactness of the transformations).
#pragma once

#include <cuda_runtime.h>

namespace hw {

// the df64 overloads below must not hide the float / double ones
using ::fma;
using ::sqrt;

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // From a double: folded at compile time for literals; at run time it costs
  // FP64 conversions, so state loads use df_split() instead.
  __host__ __device__ constexpr df64(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr df64(int x) : hi((float)x), lo(0.0f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df64(s, e);
}

__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// A double split into hi + lo with integer operations only (no FP64 pipe):
// hi = the double with its significand truncated to 24 bits (exact in FP32),
// lo = the remaining 29 significand bits rounded to FP32; |x - (hi + lo)| <=
// 2^-47 |x|.  Magnitudes outside [2^-74, 2^127] (zeros, tiny values,
// non-finite) take the FP64 conversion instead.
__device__ __forceinline__ df64 df_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const int e = (int)((h32 >> 20) & 0x7FFu);
  if (e < 949 || e > 1150) return df64((float)x, (float)(x - (double)(float)x));
  const unsigned sign = h32 & 0x80000000u;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29));
  const float scale = __uint_as_float((unsigned)(e - 948) << 23);            // 2^(e - 1075)
  const float lo = __fmul_rn(__uint2float_rn(l32 & 0x1FFFFFFFu), scale);
  return df64(hi, __uint_as_float(__float_as_uint(lo) | sign));
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const df64 s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// a * b + c with one renormalisation
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df64 s = df_two_sum(p, c.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

// Quotient: an FP32 estimate refined twice by the df64 residual a - q b.
__device__ __forceinline__ df64 operator/(df64 a, df64 b) {
  const float inv = __frcp_rn(b.hi);
  const float q1 = __fmul_rn(a.hi, inv);
  df64 r = a - b * df64(q1, 0.0f);
  const float q2 = __fmul_rn(r.hi, inv);
  df64 q = df_fast_two_sum(q1, q2);
  r = a - b * q;
  const float q3 = __fmul_rn(r.hi, inv);
  return q + df64(q3, 0.0f);
}

// Square root: the FP32 root s refined by one Newton step in df64,
// sqrt(a) ~ s + (a - s^2) / (2 s).
__device__ __forceinline__ df64 sqrt(df64 a) {
  if (!(a.hi > 0.0f)) return df64(sqrtf(a.hi), 0.0f);     // 0, or NaN for a < 0
  const float s = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(s, s);
  const float e = __fmaf_rn(s, s, -p);                     // s^2 = p + e exactly
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), a.lo);
  return df_fast_two_sum(s, __fmul_rn(r, __fdividef(0.5f, s)));
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

__device__ __forceinline__ bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(b < a) && a.hi == a.hi && b.hi == b.hi; }
__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return b <= a; }
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }

template <typename T> struct is_df64 { static constexpr bool value = false; };
template <> struct is_df64<df64> { static constexpr bool value = true; };

// A double rounded to the nearest float (ties to even) with integer operations
// only, so the conversion takes no FP64-pipe instruction (GB300 issues FP64 at a
// small fraction of the FP32 rate).  IEEE 754 binary64 -> binary32: keep the
// sign, rebias the exponent (1023 -> 127), keep the top 23 of the 52 fraction
// bits and round on the 29 dropped bits (above half up; exactly half up when
// the kept fraction is odd); a carry out of the fraction raises the exponent,
// and out of the largest finite float gives infinity, as rounding must.
// Results that are not normal floats (zero, subnormal, non-finite inputs)
// take the FP64 conversion.
__device__ __forceinline__ float f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
  const int e = (int)((h >> 20) & 0x7FFu);
  if (e < 897 || e > 1150) return __double2float_rn(x);
  const unsigned keep = ((h & 0xFFFFFu) << 3) | (l >> 29);
  const unsigned rest = l & 0x1FFFFFFFu;
  unsigned f = (h & 0x80000000u) | ((unsigned)(e - 896) << 23) | keep;
  if (rest > 0x10000000u || (rest == 0x10000000u && (keep & 1u))) f += 1u;
  return __uint_as_float(f);
}

// A float widened to double with integer operations only (exact: every float is
// a double): the sign kept, the exponent rebiased (127 -> 1023), the 23 fraction
// bits placed at the top of the 52; zeros keep their sign; subnormal and
// non-finite floats take the FP64 conversion.
__device__ __forceinline__ double f64_of_f32(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) {
    if ((b & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    return (double)x;
  }
  const unsigned h = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)h, (int)((b & 0x7u) << 29));
}

// A compute-type value as a double (float by the integer widening above).
template <typename T> __device__ __forceinline__ double to_f64(T x) { return (double)x; }
template <> __device__ __forceinline__ double to_f64<float>(float x) { return f64_of_f32(x); }

// A run-time double in the compute type (df64 by the integer split; float by
// the FP64 conversion, which measured faster than f32_rn in the gathers of the
// multi-launch reconstruction, where the FP64 pipe is not the bound).
template <typename T> __device__ __forceinline__ T from_double(double x) { return T(x); }
template <> __device__ __forceinline__ df64 from_double<df64>(double x) { return df_split(x); }

}  // namespace hw
