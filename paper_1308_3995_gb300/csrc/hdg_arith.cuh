// Scalar arithmetic the element kernels are written against, in two flavours:
//
//   Ar<double>: IEEE binary64 on the FP64 pipe.
//   Ar<ff>:     "float-float" (double-word) numbers, value = hi + lo with two
//               binary32 words, i.e. a ~48-bit significand, computed entirely
//               on the FP32 pipe, which on GB300 is ~58x wider than the FP64
//               one.  Built from the classical error-free transformations:
//               TwoSum (Knuth), FastTwoSum (Dekker, |a| >= |b|) and the
//               FMA-based exact product error a*b - fl(a*b).  Products follow
//               the usual double-word scheme (exact hi*hi product plus the two
//               cross terms, renormalised); sums of double-words add the two
//               high and the two low words with TwoSum and renormalise twice
//               (the "accurate" double-word addition).  Accumulations in the
//               kernels (dot products, LU updates) use a compensated
//               multiply-add that keeps the running error in the low word
//               unnormalised; values are renormalised before they are used as
//               factors.
//
// Both flavours expose the same static functions, so one kernel template
// serves the FP64 path and the float-float path.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace hdg {

struct __align__(8) ff {
  float hi, lo;
};

// ------------------------------------------------------------------ error-free transformations
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // requires |a| >= |b| (or a == 0)
  const float s = a + b;
  return {s, b - (s - a)};
}

// double -> float-float (hi = nearest float, lo = nearest float of the remainder)
__device__ __forceinline__ ff ff_from_double(double d) {
  const float h = __double2float_rn(d);
  return {h, __double2float_rn(d - (double)h)};
}

// float-float -> double without the FP64 pipe: hi's exact binary64 pattern is
// assembled from its bits and lo (|lo| <= half an ulp of hi when normalised)
// is added to that pattern's significand in integer arithmetic, in units of
// hi's binary64 ulp (bits of lo below that unit are truncated: < 1 ulp).  A
// subtraction from a power-of-two hi borrows into the binade below, where the
// ulp is half as large, so there the integer difference is doubled.
__device__ __forceinline__ double ff_to_double(ff v) {
  const unsigned int hb = __float_as_uint(v.hi), lb = __float_as_uint(v.lo);
  const unsigned int he = (hb >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(hb & 0x80000000u) << 32;
  if (he == 0u) return __longlong_as_double((long long)sign);  // zero (subnormal hi flushes to zero)
  if (he == 0xffu)                                               // inf / nan
    return __longlong_as_double((long long)(sign | (0x7ffull << 52) | ((unsigned long long)(hb & 0x7fffffu) << 29)));
  unsigned long long d = sign | ((unsigned long long)(he + 896u) << 52) | ((unsigned long long)(hb & 0x7fffffu) << 29);
  const unsigned int le = (lb >> 23) & 0xffu;
  const int sh = (int)le - (int)he + 29;  // lo's significand LSB relative to hi's binary64 ulp
  const unsigned long long m = 0x800000ull | (unsigned long long)(lb & 0x7fffffu);
  unsigned long long add = (sh >= 0) ? (m << sh) : (sh > -24 ? (m >> (-sh)) : 0ull);
  add = (le == 0u) ? 0ull : add;
  const bool same = ((hb ^ lb) & 0x80000000u) == 0u;
  const bool pow2 = (hb & 0x7fffffu) == 0u;
  d = same ? d + add : d - (pow2 ? 2ull * add : add);
  return __longlong_as_double((long long)d);
}

// binary64 -> float-float without the FP64 pipe: hi = the leading 24
// significand bits of d, lo = the next 23 (both truncated, so |lo| < ulp(hi)
// and |hi + lo - d| < 2^-46 |d|), from the two 32-bit halves of the bit
// pattern: hi by re-basing the exponent, lo as the integer of the next 23 bits
// (made a float exactly by the 2^23 magic-number subtraction) times 2^(e - 46).
// |d| < 2^-126 flushes to zero; for 2^-126 <= |d| < 2^-80 lo is dropped (24
// bits kept); |d| >= 2^128 becomes +-inf; NaN stays NaN.
__device__ __forceinline__ ff ff_split_double(double d) {
  const unsigned int hw = (unsigned int)__double2hiint(d), lw = (unsigned int)__double2loint(d);
  const unsigned int sign = hw & 0x80000000u;
  const unsigned int ex = (hw >> 20) & 0x7ffu;
  if (ex <= 896u) return {__uint_as_float(sign), 0.0f};
  if (ex >= 1151u)
    return {__uint_as_float(sign | 0x7f800000u | ((ex == 2047u && ((hw & 0xfffffu) | lw)) ? 0x400000u : 0u)), 0.0f};
  const float hi = __uint_as_float(sign | ((ex - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  const float r = __uint_as_float(0x4b000000u | ((lw & 0x1fffffffu) >> 6)) - 8388608.0f;  // exact, < 2^23
  const float lo = (ex >= 943u) ? r * __uint_as_float((ex - 942u) << 23) : 0.0f;       // r * 2^(e - 46)
  return {hi, __uint_as_float(__float_as_uint(lo) | sign)};
}

template <class T>
struct Ar;

// ------------------------------------------------------------------ binary64
template <>
struct Ar<double> {
  using T = double;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T from_d(double d) { return d; }
  static __device__ __forceinline__ double to_d(T a) { return a; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T neg(T a) { return -a; }
  static __device__ __forceinline__ T abs(T a) { return fabs(a); }
  // acc += a*b and acc -= a*b (one rounding each)
  static __device__ __forceinline__ void madd(T& acc, T a, T b) { acc = fma(a, b, acc); }
  static __device__ __forceinline__ void msub(T& acc, T a, T b) { acc = fma(-a, b, acc); }
  static __device__ __forceinline__ T norm(T a) { return a; }
  static __device__ __forceinline__ T rcp(T a) { return __drcp_rn(a); }
  // |a| as an ordered integer key (for pivot search off the FP pipe) and a non-finite test
  static __device__ __forceinline__ unsigned long long key(T a) {
    return (unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull;
  }
  static __device__ __forceinline__ int bad(T a) { return (__double2hiint(a) & 0x7ff00000) == 0x7ff00000; }
};

// ------------------------------------------------------------------ float-float
template <>
struct Ar<ff> {
  using T = ff;
  static __device__ __forceinline__ T zero() { return {0.0f, 0.0f}; }
  static __device__ __forceinline__ T from_d(double d) { return ff_from_double(d); }
  static __device__ __forceinline__ double to_d(T a) { return ff_to_double(a); }
  static __device__ __forceinline__ T add(T a, T b) {
    ff s = two_sum(a.hi, b.hi);
    const ff t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
  }
  static __device__ __forceinline__ T neg(T a) { return {-a.hi, -a.lo}; }
  // |a| of a normalised value (the sign is the high word's)
  static __device__ __forceinline__ T abs(T a) { return a.hi < 0.0f ? neg(a) : a; }
  static __device__ __forceinline__ T sub(T a, T b) { return add(a, neg(b)); }
  static __device__ __forceinline__ T mul(T a, T b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
  }
  // compensated acc += a*b: the exact error of the leading product and of the
  // running high-word sum go to the (unnormalised) low word
  static __device__ __forceinline__ void madd(T& acc, T a, T b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const ff s = two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo += s.lo + e;
  }
  static __device__ __forceinline__ void msub(T& acc, T a, T b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const ff s = two_sum(acc.hi, -p);
    acc.hi = s.hi;
    acc.lo += s.lo - e;
  }
  static __device__ __forceinline__ T norm(T a) { return two_sum(a.hi, a.lo); }
  // 1/a: binary32 reciprocal refined by one Newton step in double-word arithmetic
  static __device__ __forceinline__ T rcp(T a) {
    const float r = __frcp_rn(a.hi);
    // e = 1 - a*r exactly enough: a*r = 1 + small, computed with the product error
    const float p = a.hi * r;
    float e = fmaf(a.hi, r, -p);      // a.hi*r = p + e exactly
    e = fmaf(a.lo, r, e);
    const float res = (1.0f - p) - e; // 1 - a*r, |.| ~ 2^-24
    const ff rr = fast_two_sum(r, r * res);
    return rr;
  }
  static __device__ __forceinline__ unsigned long long key(T a) {
    return (unsigned long long)(__float_as_uint(a.hi) & 0x7fffffffu);
  }
  static __device__ __forceinline__ int bad(T a) { return (__float_as_uint(a.hi) & 0x7f800000u) == 0x7f800000u; }
};

// square roots (used only by the viscous flux: T^{3/2} in Sutherland's law)
__device__ __forceinline__ double ar_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ ff ar_sqrt(ff a) {
  // binary32 root refined by one Newton step in double-word arithmetic: r + (a - r^2) / (2 r)
  const float r = sqrtf(a.hi);
  const float p = r * r;
  const float e = fmaf(r, r, -p);                      // r^2 = p + e exactly
  const float res = ((a.hi - p) - e) + a.lo;           // a - r^2
  return fast_two_sum(r, res * (0.5f / r));
}

// Forward-mode dual number with ND tangent directions, over the arithmetic T.
template <class T, int ND>
struct Dual {
  T v;
  T d[ND];
};
template <class T, int ND>
__device__ __forceinline__ Dual<T, ND> dconst(T c) {
  Dual<T, ND> r;
  r.v = c;
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = Ar<T>::zero();
  return r;
}
template <class T, int ND>
__device__ __forceinline__ Dual<T, ND> dadd(const Dual<T, ND>& a, const Dual<T, ND>& b) {
  Dual<T, ND> r;
  r.v = Ar<T>::add(a.v, b.v);
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = Ar<T>::add(a.d[i], b.d[i]);
  return r;
}
template <class T, int ND>
__device__ __forceinline__ Dual<T, ND> dsub(const Dual<T, ND>& a, const Dual<T, ND>& b) {
  Dual<T, ND> r;
  r.v = Ar<T>::sub(a.v, b.v);
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = Ar<T>::sub(a.d[i], b.d[i]);
  return r;
}
template <class T, int ND>
__device__ __forceinline__ Dual<T, ND> dmul(const Dual<T, ND>& a, const Dual<T, ND>& b) {
  Dual<T, ND> r;
  r.v = Ar<T>::mul(a.v, b.v);
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = Ar<T>::add(Ar<T>::mul(a.v, b.d[i]), Ar<T>::mul(a.d[i], b.v));
  return r;
}
template <class T, int ND>
__device__ __forceinline__ Dual<T, ND> dscale(const Dual<T, ND>& a, T s) {
  Dual<T, ND> r;
  r.v = Ar<T>::mul(a.v, s);
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = Ar<T>::mul(a.d[i], s);
  return r;
}
template <class T, int ND>
__device__ __forceinline__ Dual<T, ND> drcp(const Dual<T, ND>& a) {  // 1/a, d(1/a) = -da / a^2
  Dual<T, ND> r;
  r.v = Ar<T>::rcp(a.v);
  const T m = Ar<T>::neg(Ar<T>::mul(r.v, r.v));
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = Ar<T>::mul(a.d[i], m);
  return r;
}
template <class T, int ND>
__device__ __forceinline__ Dual<T, ND> dsqrt(const Dual<T, ND>& a) {  // d sqrt(a) = da / (2 sqrt(a))
  Dual<T, ND> r;
  r.v = ar_sqrt(a.v);
  const T h = Ar<T>::mul(Ar<T>::from_d(0.5), Ar<T>::rcp(r.v));
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = Ar<T>::mul(a.d[i], h);
  return r;
}

}  // namespace hdg
