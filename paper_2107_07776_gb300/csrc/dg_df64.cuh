// Float-float ("double-float") arithmetic for the FP64-accurate operator
// kernels on GB300, whose FP32 pipes issue about 61 times the FP64 rate.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, a 48-bit significand within FP32's exponent range.  The
// operations are the error-free transformations of Knuth (TwoSum, The Art of
// Computer Programming vol. 2, 4.2.2) and Dekker (FastTwoSum; "A
// floating-point technique for extending the available precision", Numer.
// Math. 18, 1971), with the exact product error from one fused multiply-add.
// Every step uses explicitly rounded intrinsics so the compiler cannot
// contract or reorder them.  Error of one operation: a few units of 2^-48
// of the operands' magnitude; the kernels that use it keep FP64 storage and
// convert at loads and stores.
#pragma once

#include <cuda_runtime.h>

namespace dg {

struct df64 {
  float hi, lo;
};

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// requires |a| >= |b| or a == 0
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// Sum of two pairs: TwoSum of the leading parts, the trailing parts added
// into the error, one FastTwoSum (Dekker's add2).  The error is a few units
// of 2^-48 of |a| + |b| -- the order of the error the operands already
// carry from their own rounding, which is what a sum of rounded terms can
// resolve -- at 11 FP32 operations instead of 20 for the variant that also
// bounds the error by |a + b|.
__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
  const df64 s = df_two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df64 df_neg(df64 a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// a * b + c in one pass: the exact product error (one FMA) and the cross
// terms go straight into the error of the sum, so the product needs no
// renormalisation of its own (15 FP32 operations instead of 18).
__device__ __forceinline__ df64 df_fma(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df64 s = df_two_sum(p, c.hi);
  const float t = __fadd_rn(s.lo, __fadd_rn(e, c.lo));
  return df_fast_two_sum(s.hi, t);
}

// Compensated accumulation of float-float products (the Dot2 scheme of
// Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci.
// Comput. 26, 2005, carried to float-float operands): the leading parts of
// the products are summed with TwoSum, and every rounding error -- the exact
// product errors (one FMA), the cross terms hi*lo and the TwoSum errors --
// goes into one FP32 error word; one FastTwoSum at the end.  12 FP32
// operations per product instead of 15 for a chain of df_fma, with an error
// of a few units of 2^-48 of the sum of the terms' magnitudes (the order of
// the error the chain has).
struct DfAcc {
  float s, e;
};

__device__ __forceinline__ DfAcc acc_of(df64 c) { return {c.hi, c.lo}; }

// first product of an empty sum (no TwoSum needed)
__device__ __forceinline__ DfAcc acc_prod(df64 x, df64 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return {p, e};
}

__device__ __forceinline__ void acc_fma(DfAcc& a, df64 x, df64 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  const df64 t = df_two_sum(a.s, p);
  a.s = t.hi;
  a.e = __fadd_rn(a.e, __fadd_rn(t.lo, e));
}

__device__ __forceinline__ void acc_add(DfAcc& a, df64 x) {
  const df64 t = df_two_sum(a.s, x.hi);
  a.s = t.hi;
  a.e = __fadd_rn(a.e, __fadd_rn(t.lo, x.lo));
}

__device__ __forceinline__ df64 acc_value(const DfAcc& a) { return df_fast_two_sum(a.s, a.e); }

// a += b for two partial sums (independent accumulators shorten the
// dependency chain of a long sum; they are merged at the end)
__device__ __forceinline__ void acc_merge(DfAcc& a, const DfAcc& b) {
  const df64 t = df_two_sum(a.s, b.s);
  a.s = t.hi;
  a.e = __fadd_rn(a.e, __fadd_rn(t.lo, b.e));
}

// A float-float value stored in 8 bytes of a double-typed array (the
// pre-split copies the FP64 operator kernels read): the bits are the pair.
__device__ __forceinline__ df64 df_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return {__uint_as_float((unsigned int)(b & 0xffffffffull)), __uint_as_float((unsigned int)(b >> 32))};
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) { return df_add(a, b); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df64 operator-(df64 a) { return df_neg(a); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) { return df_mul(a, b); }
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = df_add(a, b); }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = df_add(a, df_neg(b)); }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = df_mul(a, b); }

__device__ __forceinline__ df64 df_abs(df64 a) { return a.hi < 0.0f ? df_neg(a) : a; }
__device__ __forceinline__ bool df_less(df64 a, df64 b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ df64 df_max(df64 a, df64 b) { return df_less(a, b) ? b : a; }

__device__ __forceinline__ df64 df_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

// Split of a constant: plain casts (round to nearest, like the intrinsics
// above) that the compiler folds for literal arguments, so constants cost no
// conversion instruction at run time.
__device__ __forceinline__ df64 df_const(double x) {
  const float h = static_cast<float>(x);
  return {h, static_cast<float>(x - static_cast<double>(h))};
}

// Exact widening of a float to double with integer operations only (no
// FP64-pipe conversion, not even a predicated one): the sign is kept, the
// exponent rebiased (127 -> 1023) and the 23 fraction bits moved to the top
// of the 52.  Zeros, subnormals (normalised by their leading one),
// infinities and NaNs are built the same way.
__device__ __forceinline__ double df_widen(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu;
  const unsigned int m = u & 0x7FFFFFu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  unsigned long long bits;
  if (e == 0u) {
    if (m == 0u) {
      bits = sgn;
    } else {  // m 2^-149 = 1.f 2^(p-149), p the position of m's leading one
      const int p = 31 - __clz((int)m);
      const unsigned long long frac = ((unsigned long long)m << (52 - p)) & 0xFFFFFFFFFFFFFull;
      bits = sgn | ((unsigned long long)(p - 149 + 1023) << 52) | frac;
    }
  } else if (e == 0xFFu) {
    bits = sgn | (0x7FFull << 52) | ((unsigned long long)m << 29);
  } else {
    bits = sgn | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
  }
  return __longlong_as_double((long long)bits);
}

// A double narrowed to float with integer operations only (no FP64-pipe
// conversion): the leading 24 significant bits, truncated (relative error
// below 2^-23); magnitudes below FP32's normal range give a signed zero,
// above it (and infinities) a signed infinity, NaN stays NaN.  For FP32
// preconditioner arithmetic on FP64 data.
__device__ __forceinline__ float df_narrow(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int top = (unsigned int)(b >> 32);
  const unsigned int sign = top & 0x80000000u;
  const int e = (int)((top >> 20) & 0x7FFu);
  const int ef = e - 1023 + 127;
  if (ef <= 0) return __int_as_float((int)sign);
  if (ef >= 255) {
    const bool nan = e == 0x7FF && (b & 0xFFFFFFFFFFFFFull) != 0ull;
    return __int_as_float((int)(sign | 0x7F800000u | (nan ? 0x00400000u : 0u)));
  }
  return __int_as_float((int)(sign | ((unsigned int)ef << 23) | (unsigned int)((b >> 29) & 0x7FFFFFull)));
}

// hi + lo rounded once to double (a single FP64 addition)
__device__ __forceinline__ double df_to(df64 a) { return df_widen(a.hi) + df_widen(a.lo); }

// Split of a double into a float pair with integer operations only (no FP64
// instruction -- also none that a predicated fallback would issue): hi keeps
// the sign, exponent and leading 23 fraction bits; the remaining 29 fraction
// bits become lo (truncated to 24 significant bits, a relative error below
// 2^-47 of x), and one FastTwoSum renormalises the pair.  The float-float
// format's exponent range applies: lo is dropped once it would fall below
// FP32's normal range (|x| < 2^-102: relative error up to 2^-23), the pair
// is (+-0, 0) below 2^-126 and (+-inf or NaN, 0) from 2^128 on.
__device__ __forceinline__ df64 df_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int top = (unsigned int)(b >> 32);
  const unsigned int sign = top & 0x80000000u;
  const int e = (int)((top >> 20) & 0x7FFu);
  const int ef = e - 1023 + 127;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (ef <= 0) return {__int_as_float((int)sign), 0.0f};
  if (ef >= 255) {
    const unsigned int nan = (e == 0x7FF && m != 0ull) ? 0x00400000u : 0u;
    return {__int_as_float((int)(sign | 0x7F800000u | nan)), 0.0f};
  }
  const float hi = __int_as_float((int)(sign | ((unsigned int)ef << 23) | (unsigned int)(m >> 29)));
  const unsigned int r = (unsigned int)(m & 0x1FFFFFFFull);
  if (r == 0u) return {hi, 0.0f};
  const int p = 31 - __clz((int)r);  // position of the remainder's leading one
  const int el = ef - 52 + p;        // its biased FP32 exponent
  if (el <= 0) return {hi, 0.0f};
  const unsigned int mant = p >= 23 ? (r >> (p - 23)) : (r << (23 - p));
  const float lo = __int_as_float((int)(sign | ((unsigned int)el << 23) | (mant & 0x7FFFFFu)));
  return df_fast_two_sum(hi, lo);
}

// Sum of products in the arithmetic type A: a plain FMA chain for float and
// double, the compensated accumulator for float-float.
template <typename A>
struct SumOf {
  A v;
  __device__ __forceinline__ void start(A x, A y) { v = x * y; }
  __device__ __forceinline__ void fma(A x, A y) { v = __fma_any(x, y, v); }
  __device__ __forceinline__ A value() const { return v; }
  __device__ __forceinline__ void merge(const SumOf& o) { v = v + o.v; }
  __device__ __forceinline__ static A __fma_any(A x, A y, A c) {
    if constexpr (sizeof(A) == 4) return __fmaf_rn(x, y, c);
    else return __fma_rn(x, y, c);
  }
};

template <>
struct SumOf<df64> {
  DfAcc a;
  __device__ __forceinline__ void start(df64 x, df64 y) { a = acc_prod(x, y); }
  __device__ __forceinline__ void fma(df64 x, df64 y) { acc_fma(a, x, y); }
  __device__ __forceinline__ df64 value() const { return acc_value(a); }
  __device__ __forceinline__ void merge(const SumOf& o) { acc_merge(a, o.a); }
};

// Arithmetic-type adapters for kernels templated on the arithmetic type A
// (float, double or df64) and the storage type T (float or double).
template <typename A>
struct Arith;

template <>
struct Arith<float> {
  __device__ static float from(double x) { return (float)x; }
  __device__ static float from(float x) { return x; }
  __device__ static float c(double x) { return (float)x; }
  __device__ static float abs(float x) { return fabsf(x); }
  __device__ static float max(float a, float b) { return fmaxf(a, b); }
  __device__ static float to_f(float x) { return x; }
  __device__ static double to_d(float x) { return (double)x; }
  __device__ static float fma(float a, float b, float c) { return fmaf(a, b, c); }
};

template <>
struct Arith<double> {
  __device__ static double from(double x) { return x; }
  __device__ static double from(float x) { return (double)x; }
  __device__ static double c(double x) { return x; }
  __device__ static double abs(double x) { return fabs(x); }
  __device__ static double max(double a, double b) { return fmax(a, b); }
  __device__ static float to_f(double x) { return (float)x; }
  __device__ static double to_d(double x) { return x; }
  __device__ static double fma(double a, double b, double c) { return ::fma(a, b, c); }
};

template <>
struct Arith<df64> {
  __device__ static df64 from(double x) { return df_split(x); }
  __device__ static df64 from(float x) { return {x, 0.0f}; }
  __device__ static df64 c(double x) { return df_const(x); }
  __device__ static df64 abs(df64 x) { return df_abs(x); }
  __device__ static df64 max(df64 a, df64 b) { return df_max(a, b); }
  __device__ static float to_f(df64 x) { return x.hi; }
  __device__ static double to_d(df64 x) { return df_to(x); }
  __device__ static df64 fma(df64 a, df64 b, df64 c) { return df_fma(a, b, c); }
};

}  // namespace dg
