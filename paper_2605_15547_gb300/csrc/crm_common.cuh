// crm_common.cuh -- arithmetic building blocks shared by every evaluator.
//
// Three tiers evaluate each function (the paper's Sec. II.A design, with the rounding
// test of Sec. II.B applied to every tier):
//   plain  : FP64 internal arithmetic (the paper's single-precision design, Sec. II.A),
//   df     : FP32 double-float fast path (the paper's future-work direction, Sec. IV),
//   dd     : double-double slow path for the rare lanes whose rounding test failed.
// Every tier returns an approximation with a proven relative error bound eps; the
// rounding test below accepts it only if no rounding boundary (midpoint) lies within
// eps of it, so that the accepted result equals RN(f(x)).
//
// The library is compiled with -fmad=false: no multiply-add is fused unless written as
// an explicit fma, so every rounding below happens exactly where the code says.
#pragma once
#include <stdint.h>

#define CRM_DEV __device__ __forceinline__
#define CRM_NOINL __device__ __noinline__

namespace crm {

// 1.5 * 2^23: adding it rounds a float of magnitude < 2^22 to an integer in its low bits
#define CRM_SHIFTER_F 0x1.8p23f

// ------------------------------------------------------------------ bit helpers
CRM_DEV uint32_t fbits(float x) { return __float_as_uint(x); }
CRM_DEV float bitsf(uint32_t b) { return __uint_as_float(b); }
CRM_DEV uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }
CRM_DEV double bitsd(uint64_t b) { return __longlong_as_double((long long)b); }

// ------------------------------------------------------------------ error-free transforms
template <class T> struct Pair { T hi, lo; };
template <class T> CRM_DEV Pair<T> operator-(Pair<T> a) { return {-a.hi, -a.lo}; }

CRM_DEV float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
CRM_DEV double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

// s + e == a + b exactly (Knuth TwoSum, 6 operations, no ordering requirement)
template <class T> CRM_DEV Pair<T> two_sum(T a, T b) {
  T s = a + b;
  T bb = s - a;
  T e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
// s + e == a + b exactly when exponent(a) >= exponent(b) or a == 0 (Dekker Fast2Sum)
template <class T> CRM_DEV Pair<T> fast_two_sum(T a, T b) {
  T s = a + b;
  T e = b - (s - a);
  return {s, e};
}
// p + e == a * b exactly (barring underflow)
template <class T> CRM_DEV Pair<T> two_prod(T a, T b) {
  T p = a * b;
  return {p, fma_(a, b, -p)};
}

// ------------------------------------------------------------------ double-double
// Accurate sum of two double-double numbers (relative error <= 3u^2 + O(u^3)).
CRM_DEV Pair<double> dd_add(Pair<double> a, Pair<double> b) {
  Pair<double> s = two_sum(a.hi, b.hi);
  Pair<double> t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
CRM_DEV Pair<double> dd_add_d(Pair<double> a, double b) {
  Pair<double> s = two_sum(a.hi, b);
  s.lo += a.lo;
  return fast_two_sum(s.hi, s.lo);
}
// Product of double-double numbers (relative error <= 5u^2 + O(u^3)).
CRM_DEV Pair<double> dd_mul(Pair<double> a, Pair<double> b) {
  Pair<double> p = two_prod(a.hi, b.hi);
  double t = fma_(a.hi, b.lo, a.lo * b.hi);
  p.lo += t;
  return fast_two_sum(p.hi, p.lo);
}
CRM_DEV Pair<double> dd_mul_d(Pair<double> a, double b) {
  Pair<double> p = two_prod(a.hi, b);
  p.lo = fma_(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
CRM_DEV Pair<double> dd_sqr(Pair<double> a) {
  Pair<double> p = two_prod(a.hi, a.hi);
  p.lo = fma_(2.0 * a.hi, a.lo, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
// a / b for double-double (relative error below 2^-100 for normal operands): a quotient
// from the rounded reciprocal of b.hi (relative error 2^-52), corrected twice from exact
// residuals.  One FP64 division instead of three: the slow tiers are latency-bound.
CRM_DEV Pair<double> dd_div(Pair<double> a, Pair<double> b) {
  const double rb = 1.0 / b.hi;
  double q1 = a.hi * rb;
  Pair<double> r = dd_add(a, dd_mul_d(b, -q1));
  double q2 = r.hi * rb;
  r = dd_add(r, dd_mul_d(b, -q2));
  double q3 = r.hi * rb;
  Pair<double> q = fast_two_sum(q1, q2);
  return dd_add_d(q, q3);
}
CRM_DEV Pair<double> dd_neg(Pair<double> a) { return {-a.hi, -a.lo}; }
CRM_DEV Pair<double> dd(double h, double l) { return {h, l}; }

// ------------------------------------------------------------------ double-float helpers
// Quotient of float pairs: q1 from the hardware reciprocal (relative error ~2^-22), the
// residual a - q1 b with an exact product split, one correction: relative error < 2^-43.
// df_div_raw leaves the quotient unnormalised (q1 + q2, |q2| < 2^-20 |q1|).
CRM_DEV Pair<float> df_div_raw(Pair<float> a, Pair<float> b) {
  float r = __fdividef(1.0f, b.hi);
  float q1 = a.hi * r;
  float p = q1 * b.hi;
  float pl = fma_(q1, b.hi, -p);
  float rr = (a.hi - p) - pl;
  rr = rr + fma_(-q1, b.lo, a.lo);
  float q2 = rr * r;
  return {q1, q2};
}
CRM_DEV Pair<float> df_div(Pair<float> a, Pair<float> b) {
  Pair<float> q = df_div_raw(a, b);
  return fast_two_sum(q.hi, q.lo);
}
// Product of float pairs (relative error < 2^-45)
CRM_DEV Pair<float> df_mul(Pair<float> a, Pair<float> b) {
  float p = a.hi * b.hi;
  float pl = fma_(a.hi, b.hi, -p);
  pl = fma_(a.hi, b.lo, pl);
  pl = fma_(a.lo, b.hi, pl);
  return fast_two_sum(p, pl);
}
// The same product left unnormalised (p + pl, |pl| below 2^-22 |p|), for a sum that
// renormalises anyway (df_add)
CRM_DEV Pair<float> df_mul_raw(Pair<float> a, Pair<float> b) {
  float p = a.hi * b.hi;
  float pl = fma_(a.hi, b.hi, -p);
  pl = fma_(a.hi, b.lo, pl);
  pl = fma_(a.lo, b.hi, pl);
  return {p, pl};
}
// Sum of float pairs when |a.hi| >= |b.hi| (or a.hi = 0): Fast2Sum on the leading words;
// the _raw form leaves the sum unnormalised (for round_df)
CRM_DEV Pair<float> df_add_ordered_raw(Pair<float> a, Pair<float> b) {
  Pair<float> s = fast_two_sum(a.hi, b.hi);
  s.lo = s.lo + (a.lo + b.lo);
  return s;
}
CRM_DEV Pair<float> df_add_ordered(Pair<float> a, Pair<float> b) {
  Pair<float> s = df_add_ordered_raw(a, b);
  return fast_two_sum(s.hi, s.lo);
}
// Sum of float pairs without ordering assumption
CRM_DEV Pair<float> df_add(Pair<float> a, Pair<float> b) {
  Pair<float> s = two_sum(a.hi, b.hi);
  s.lo = s.lo + (a.lo + b.lo);
  return fast_two_sum(s.hi, s.lo);
}

// ------------------------------------------------------------------ rounding tests
// Plain tier: y (a double, finite, |y| >= 2^-1000) approximates the exact value v with
// |v - y| <= D units in the last place of y.  Returns true ("hard") unless RN_f32(v) is
// certainly RN_f32(y).  Binary32 rounding boundaries, seen in y's significand, are the
// patterns t == 2^(s-1) modulo 2^s where s = 29 for normal float results and grows by
// one per binade below 2^-126 (subnormal results); they are tested with integer ops.
CRM_DEV bool hard_d_to_f(double y, uint32_t D) {
  uint64_t u = dbits(y) & 0x7FFFFFFFFFFFFFFFull;
  int E = (int)(u >> 52) - 1023;
  int s = -97 - E;
  s = s < 29 ? 29 : (s > 55 ? 55 : s);
  uint64_t m = (u & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  uint64_t t = m & ((1ull << s) - 1);
  uint64_t h = 1ull << (s - 1);
  return (t - h + D) <= 2ull * D;
}

// Double-float tier: y = s + r (s normal, |r| <= 2^-14 |s|, the pair need not be
// normalised) approximates v with |v - y| <= eps_true |y|, eps_true <= 2^-37.  With
// e = 2^-36 |s| (exact), a+ = RN(r + e) and a- = RN(r - e) lie outside
// [r - eps_true |y|, r + eps_true |y|]: their roundings cost at most 2^-24 (|r| + e)
// < 2^-37.9 |s|, and eps_true |y| <= 2^-37 (1 + 2^-14) |s|, together below e.  So
// s + a- <= v <= s + a+, and as round-to-nearest is monotone, RN(s + a-) == RN(s + a+)
// implies that both equal RN(v): the paper's comparison of the roundings of y - e and
// y + e (Sec. II.B), with the two ends formed from the unnormalised pair.  Otherwise
// the lane is hard.  An easy lane's result is RN(s + r), the value a normalised pair
// would give; a NaN in s makes the lane hard.  Six operations; renormalising the pair
// and testing the distance to the nearest midpoint would take eight.
CRM_DEV float round_df(float s, float r, bool &hard) {
  const float e = fabsf(s) * 0x1p-36f;
  const float hi = s + (r + e), lo = s + (r - e);
  hard = hi != lo;
  return hi;
}

// Slow tier: y = s + t (double-double, |t| <= ulp(s)/2) approximates v with
// |v - y| <= e.  Returns RN_f32(v) and sets hard when a binary32 midpoint (or the
// overflow threshold) lies within reach.  Uses directed conversions to find the two
// binary32 neighbours of s; their midpoint is exact in binary64.
CRM_DEV float round_dd_to_f(double s, double t, double e, bool &hard) {
  float dn = __double2float_rd(s), up = __double2float_ru(s);
  hard = false;
  if (dn == up) return dn;  // s is a binary32 value; v lies within e + |t| << ulp of it
  double mid;
  if (isinf(up))
    mid = 0x1.ffffffp+127;  // RN overflow threshold 2^128 - 2^103
  else if (isinf(dn))
    mid = -0x1.ffffffp+127;
  else
    mid = 0.5 * ((double)dn + (double)up);
  double dist = (s - mid) + t;  // exact enough: s - mid is exact (Sterbenz) and small
  if (fabs(dist) <= e) {
    hard = true;
    return __double2float_rn(s);
  }
  return dist > 0 ? up : dn;
}

// ------------------------------------------------------------------ misc
// Block-cooperative copy of a table into shared memory (bytes a multiple of 4).
CRM_DEV void copy_tab(void *dst, const void *src, int bytes) {
  const uint32_t *s = (const uint32_t *)src;
  uint32_t *d = (uint32_t *)dst;
  for (int i = threadIdx.x; i < bytes / 4; i += blockDim.x) d[i] = s[i];
}

CRM_DEV float qnan_of(float x) { return bitsf(fbits(x) | 0x00400000u); }
CRM_DEV double qnan_of(double x) { return bitsd(dbits(x) | 0x0008000000000000ull); }
#define CRM_QNAN_F (__uint_as_float(0x7FC00000u))
#define CRM_QNAN_D (__longlong_as_double(0x7FF8000000000000ll))
#define CRM_INF_F (__uint_as_float(0x7F800000u))
#define CRM_INF_D (__longlong_as_double(0x7FF0000000000000ll))

// 2^k as a double for k in [-1022, 1023]
CRM_DEV double pow2d(int k) { return bitsd((uint64_t)(k + 1023) << 52); }
// y * 2^k for a normal double y whose scaled value stays normal
CRM_DEV double scale_d(double y, int k) { return bitsd(dbits(y) + ((uint64_t)(int64_t)k << 52)); }

}  // namespace crm
