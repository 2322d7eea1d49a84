// Double-float arithmetic on the FP32 units, for the FP64-vector stencil
// kernels of the MIXED_DF mode (scatter W^T / dW^T and gather W / dW of
// Sec. 3.1).
//
// A value is the unevaluated sum hi + lo of two floats.  Products and sums
// use the classical error-free transformations: the exact product
// a b = p + e with p = fl(a b), e = fma(a, b, -p) (one FMA), and Knuth's
// TwoSum a + b = s + t (six additions, no branch).  A product of two
// double-floats drops the lo*lo term and rounds the cross terms once,
// so its relative error is ~2^-46; a running sum keeps its rounding errors
// in the lo word.  This gives ~2^-44 of the sum of the terms' magnitudes,
// against 2^-24 for FP32 and 2^-53 for FP64, at a cost of ~10 FP32
// operations per multiply-add -- GB300 issues FP32 at ~64x its FP64 rate.
//
// Conversions to and from FP64 use integer operations on the bit patterns
// (GB300's FP64 units are the scarce resource these kernels avoid):
// df_split keeps the top 24 significand bits of a double as hi and rounds
// the remaining 29 to float as lo (exact for |x| in [2^-74, 2^127], hi
// alone below; zero and subnormal inputs give zero); df_to_double rounds
// hi + lo to the nearest double.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dski {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_zero() { return {0.f, 0.f}; }

// hi + lo == x (up to lo's rounding to 24 bits) by integer operations.
__device__ __forceinline__ dfl df_split(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t s = (uint32_t)(u >> 63) << 31;
  const int E = (int)((u >> 52) & 0x7FF);
  const unsigned long long M = u & ((1ULL << 52) - 1);
  const int ef = E - 1023 + 127;   // float exponent field of hi
  if (E == 0 || ef <= 0) return df_zero();   // zero, subnormal, or below FP32's normal range
  if (ef >= 255) return {__uint_as_float(s | 0x7F800000u), 0.f};   // beyond FP32: inf
  const float hi = __uint_as_float(s | ((uint32_t)ef << 23) | (uint32_t)(M >> 29));
  // the low 29 bits, worth r 2^(E - 1075)
  const uint32_t r = (uint32_t)(M & ((1u << 29) - 1));
  const int el = E - 1075 + 127;   // exponent field of 2^(E - 1075)
  float lo = 0.f;
  if (r != 0 && el > 0) {
    const float rf = __uint2float_rn(r);   // < 2^29, rounded to 24 bits
    lo = rf * __uint_as_float((uint32_t)el << 23);
    if (s) lo = -lo;
  }
  return {hi, lo};
}

// Float to double by its bit pattern (exact; subnormal floats give zero).
__device__ __forceinline__ unsigned long long df_bits_of_float(float f, int* e2,
                                                               unsigned long long* mant,
                                                               uint32_t* sgn) {
  const uint32_t b = __float_as_uint(f);
  *sgn = b >> 31;
  const int E = (int)((b >> 23) & 0xFF);
  if (E == 0) {
    *mant = 0;
    *e2 = 0;
    return 0;
  }
  *mant = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);   // value = mant 2^(E - 150)
  *e2 = E - 150;
  return 1;
}

// The double nearest to hi + lo (ties away from zero), by integer operations.
// Both words are put on the scale 2^(e - 38) of the larger one (each
// significand < 2^24, so each term < 2^62 and their sum fits in an int64);
// the smaller word is rounded there when it lies more than 38 bits below.
__device__ __forceinline__ double df_to_double(dfl a) {
  int eh, el;
  unsigned long long mh, ml;
  uint32_t sh, sl;
  const bool nh = df_bits_of_float(a.hi, &eh, &mh, &sh);
  const bool nl = df_bits_of_float(a.lo, &el, &ml, &sl);
  if (!nh && !nl) return 0.0;
  const int top = !nl ? eh : (!nh ? el : (eh > el ? eh : el));
  const int ex = top - 38;
  auto scaled = [ex](bool nz, int e, unsigned long long m, uint32_t sg) -> long long {
    if (!nz) return 0;
    const int d = e - ex;   // <= 38
    long long v;
    if (d >= 0) v = (long long)(m << d);
    else if (d > -40) v = (long long)((m + (1ULL << (-d - 1))) >> (-d));
    else v = 0;
    return sg ? -v : v;
  };
  const long long V = scaled(nh, eh, mh, sh) + scaled(nl, el, ml, sl);
  if (V == 0) return 0.0;
  const unsigned long long sgn = V < 0 ? (1ULL << 63) : 0ULL;
  unsigned long long A = V < 0 ? (unsigned long long)(-V) : (unsigned long long)V;
  const int nb = 64 - __clzll((long long)A);
  int e2 = ex;
  unsigned long long mant;
  if (nb > 53) {
    const int k = nb - 53;
    A = (A + (1ULL << (k - 1))) >> k;
    e2 += k;
    if (A >> 53) {
      A >>= 1;
      ++e2;
    }
    mant = A;
  } else {
    mant = A << (53 - nb);
    e2 -= 53 - nb;
  }
  const long long be = (long long)e2 + 52 + 1023;
  if (be <= 0) return 0.0;
  if (be >= 2047) return __longlong_as_double((long long)(sgn | (0x7FFULL << 52)));
  return __longlong_as_double(
      (long long)(sgn | ((unsigned long long)be << 52) | (mant & ((1ULL << 52) - 1))));
}

// Knuth's TwoSum: s + t == a + b exactly (s = fl(a + b)).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a b as a double-float (lo*lo dropped, cross terms rounded once).
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return {p, e};   // unnormalised: |e| may reach a few ulps of p
}

// acc += x (x possibly unnormalised): TwoSum on the high words, the low
// words and the rounding error collected in lo.
__device__ __forceinline__ void df_acc(dfl& acc, dfl x) {
  float s, t;
  two_sum(acc.hi, x.hi, s, t);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, x.lo));
}

// acc += a b.
__device__ __forceinline__ void df_fma_acc(dfl& acc, dfl a, dfl b) { df_acc(acc, df_mul(a, b)); }

// Renormalise so that |lo| <= ulp(hi) / 2 (Fast2Sum; |hi| >= |lo| holds
// after accumulation unless the sum cancelled, where TwoSum is used).
__device__ __forceinline__ dfl df_norm(dfl a) {
  float s, t;
  two_sum(a.hi, a.lo, s, t);
  return {s, t};
}

}  // namespace dski
