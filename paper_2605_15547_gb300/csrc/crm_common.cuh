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
// e = 2^-36 |s|, a+ = RN(r + e) and a- = RN(r - e) (each one FMA on s, whose sign only
// swaps the two) lie outside [r - eps_true |y|, r + eps_true |y|]: their roundings cost
// at most 2^-24 (|r| + e) < 2^-37.9 |s|, and eps_true |y| <= 2^-37 (1 + 2^-14) |s|,
// together below e.  So s + a- <= v <= s + a+, and as round-to-nearest is monotone,
// RN(s + a-) == RN(s + a+) implies that both equal RN(v): the paper's comparison of the
// roundings of y - e and y + e (Sec. II.B), with the two ends formed from the
// unnormalised pair.  Otherwise the lane is hard.  An easy lane's result is RN(s + r),
// the value a normalised pair would give; a NaN or an infinity in s makes the lane hard.
// Five operations; renormalising the pair and testing the distance to the nearest
// midpoint would take eight.
//
// With sg (the directed-rounding and 16-bit kernels) the test changes: the lane returns
// c = RN(s + r) and *sg = the sign of v - c, which is all a rounding direction needs
// (RD(v) = c or the float below it, and so on, see the finishers below).  s - c is exact
// (c lies within 2^-13 of s), d = (s - c) + r has one rounding, and RN is monotone, so
// |d| > e implies |y - c| > e and sign(v - c) = sign(d); otherwise v is too close to c
// (or equal to it: an exact result) and the lane is hard.
CRM_DEV float round_df(float s, float r, bool &hard, int *sg = nullptr) {
  if (sg) {
    const float e = fabsf(s) * 0x1p-36f;
    const float c = s + r;
    const float d = (s - c) + r;
    hard = !(fabsf(d) > e);  // NaN: hard
    *sg = d > 0.0f ? 1 : -1;
    return c;
  }
  const float hi = s + fma_(s, 0x1p-36f, r), lo = s + fma_(s, -0x1p-36f, r);
  hard = hi != lo;
  return hi;
}

// The sign of a float as -1, 0 or 1 (the sign of v - c for shortcuts whose error has the
// sign of x, 0 for x = 0).
CRM_DEV int sgnf(float x) { return x > 0.0f ? 1 : (x < 0.0f ? -1 : 0); }
// Store v in *sg when sg is set (RN kernels pass none: the code folds away).
CRM_DEV void put_sg(int *sg, int v) {
  if (sg) *sg = v;
}

// Slow tier: y = s + t (double-double, |t| <= ulp(s)/2) approximates v with
// |v - y| <= e.  Returns RN_f32(v) and sets hard when a binary32 midpoint (or the
// overflow threshold) lies within reach.  Uses directed conversions to find the two
// binary32 neighbours of s; their midpoint is exact in binary64.
CRM_DEV float round_dd_to_f(double s, double t, double e, bool &hard, int *sg = nullptr) {
  if (sg) {  // c = RN32(s) and the sign of v - c, decided unless |(s - c) + t| <= e
    const float c = __double2float_rn(s);
    if (isinf(c)) {  // beyond the binary32 range: the finite value lies inside the infinity
      hard = false;
      *sg = c > 0.0f ? -1 : 1;
      return c;
    }
    const double d = (s - (double)c) + t;  // s - c exact
    hard = !(fabs(d) > e);
    *sg = d > 0.0 ? 1 : -1;
    return c;
  }
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

// ------------------------------------------------------------------ directed rounding and 16-bit formats
// An evaluator run with sg returns a binary32 c within a fraction of an ulp of v = f(x) and
// sg = sign(v - c) (0 when v = c exactly).  That pair fixes RD32(v) and RU32(v), and from
// them every rounding of v to binary32, IEEE binary16 or bfloat16 in every direction
// (IEEE 754 Sec. 4.3; the paper's final step rounds toward zero with a sticky bit and then
// converts in the caller's mode, Sec. II.A):
//   RD32(v) = c if sg >= 0, else the float below c;  RU32(v) = c if sg <= 0, else above;
//   RZ = RD for v > 0, RU for v < 0;
//   for a 16-bit format F: RD_F(v) = RD_F(RD32(v)) and RU_F(v) = RU_F(RU32(v)) (every
//   number of F is a binary32 number, so none lies strictly between RD32(v) and RU32(v));
//   RN_F(v) = RN_F(a) when a = RD32(v) and b = RU32(v) round alike; otherwise a midpoint of
//   F (a binary32 number with at most 12 significant bits) lies in [a, b], so it is a or
//   b: v lies above it (take RU_F(a)) when it is a, below it (RD_F(b)) when it is b;
//   a = b (v exact) gives RN_F(a), ties to even.
enum { CRM_RM_RN = 0, CRM_RM_RD = 1, CRM_RM_RU = 2, CRM_RM_RZ = 3 };

// Neighbours of a binary32 number by its bit pattern (c not NaN; next_up(+inf) and
// next_down(-inf) are not used)
CRM_DEV float next_up_f(float c) {
  const uint32_t b = fbits(c);
  if ((b & 0x7FFFFFFFu) == 0) return bitsf(1u);  // +-0 -> smallest subnormal
  return bitsf((b >> 31) ? b - 1u : b + 1u);
}
CRM_DEV float next_down_f(float c) {
  const uint32_t b = fbits(c);
  if ((b & 0x7FFFFFFFu) == 0) return bitsf(0x80000001u);
  return bitsf((b >> 31) ? b + 1u : b - 1u);
}
CRM_DEV float rd32(float c, int sg) { return sg < 0 ? next_down_f(c) : c; }
CRM_DEV float ru32(float c, int sg) { return sg > 0 ? next_up_f(c) : c; }
// The sign of v: c's when c != 0, else sg's (v = 0 exactly when both are 0)
CRM_DEV bool v_negative(float c, int sg) { return c != 0.0f ? c < 0.0f : (sg != 0 ? sg < 0 : fbits(c) >> 31); }

// binary32 result in mode rm (NaN passes through)
CRM_DEV float finish_f32(float c, int sg, int rm) {
  if (c != c) return c;
  if (rm == CRM_RM_RD || (rm == CRM_RM_RZ && !v_negative(c, sg))) return rd32(c, sg);
  if (rm == CRM_RM_RU || rm == CRM_RM_RZ) return ru32(c, sg);
  return c;
}

// Rounding of a binary32 number a to a 16-bit format, in one direction (dir: -1 down, +1
// up, 0 toward zero, 2 to nearest with ties to even), as a 16-bit pattern.  bfloat16 is the
// top half of the binary32 pattern (same exponent range); binary16 rebiases the exponent
// (emin -14, quantum 2^-24 below 2^-14, overflow beyond 65504).
CRM_DEV uint16_t round_to_bf16(float a, int dir) {
  const uint32_t b = fbits(a);
  if (a != a) return (uint16_t)((b >> 16) | 0x0040u);  // quiet NaN, sign and payload top
  const uint32_t mag = b & 0x7FFFFFFFu, sgn = b >> 31;
  const uint32_t q = mag >> 16, rem = mag & 0xFFFFu;
  uint32_t r = q;
  const bool away = dir == 2 ? (rem > 0x8000u || (rem == 0x8000u && (q & 1u))) : (rem != 0 && dir == (sgn ? -1 : 1));
  if (away) r = q + 1u;  // carries into the exponent, up to the infinity pattern
  return (uint16_t)((sgn << 15) | r);
}
CRM_DEV uint16_t round_to_f16(float a, int dir) {
  const uint32_t b = fbits(a);
  const uint32_t sgn = (b >> 31) << 15;
  if (a != a) return (uint16_t)(sgn | 0x7E00u | ((b >> 13) & 0x03FFu));
  const uint32_t mag = b & 0x7FFFFFFFu;
  const int E = (int)(mag >> 23) - 127;  // a = 1.m 2^E for normal a
  if (mag == 0x7F800000u) return (uint16_t)(sgn | 0x7C00u);
  // the value as an integer multiple of the quantum: q = |a| / 2^(max(E, -14) - 10),
  // with the discarded bits rem (out of unit)
  uint32_t q, rem, unit;
  if (E > 15) {  // beyond binary16's range: the largest finite or infinity
    const bool up = dir == 2 || dir == (sgn ? -1 : 1);
    return (uint16_t)(sgn | (up ? 0x7C00u : 0x7BFFu));
  }
  const uint32_t M = mag >= 0x00800000u ? ((mag & 0x007FFFFFu) | 0x00800000u) : (mag & 0x007FFFFFu);
  const int e2 = mag >= 0x00800000u ? E : -126;  // |a| = M 2^(e2 - 23)
  const int drop = (e2 > -14 ? e2 : -14) - 10 - (e2 - 23);  // bits of M below the quantum: 13..
  if (drop >= 32) {
    q = 0;
    rem = M;  // nonzero for a != 0
    unit = 0;  // rem compared with half below
  } else {
    q = M >> drop;
    rem = M & ((1u << drop) - 1u);
    unit = 1u << drop;
  }
  bool away;
  if (dir == 2) {
    if (drop >= 32) away = false;  // |a| < 2^-25 * 2: below half the smallest subnormal
    else away = rem > (unit >> 1) || (rem == (unit >> 1) && (q & 1u));
  } else {
    away = rem != 0 && dir == (sgn ? -1 : 1);
  }
  q += away ? 1u : 0u;
  // q counts quanta of 2^((e2 > -14 ? e2 : -14) - 10): for normal results the pattern is
  // (biased exponent << 10) + (q - 2^10); a carry to 2^11 moves to the next binade
  uint32_t bits;
  if (e2 > -14 || q >= 0x400u) {
    const int ee = (e2 > -14 ? e2 : -14);
    bits = ((uint32_t)(ee + 15) << 10) + (q - 0x400u);  // q in [2^10, 2^11]: carry ok
    if (bits >= 0x7C00u) {  // overflow: infinity, or the largest finite toward zero
      const bool up = dir == 2 || dir == (sgn ? -1 : 1);
      bits = up ? 0x7C00u : 0x7BFFu;
    }
  } else {
    bits = q;  // subnormal (or zero)
  }
  return (uint16_t)(sgn | bits);
}
// Is the binary32 number a exactly halfway between two consecutive numbers of the 16-bit
// format (the overflow threshold included)?
template <bool BF> CRM_DEV bool is_mid16(float a) {
  const uint32_t mag = fbits(a) & 0x7FFFFFFFu;
  if (mag >= 0x7F800000u) return false;
  if (BF) return (mag & 0xFFFFu) == 0x8000u;
  const int E = (int)(mag >> 23) - 127;
  if (mag < 0x00800000u || E > 15) return false;  // far below 2^-25 or beyond the range
  const int drop = (E > -14 ? E : -14) - 10 - (E - 23);
  if (drop >= 25) return false;
  const uint32_t M = (mag & 0x007FFFFFu) | 0x00800000u;
  return (M & ((1u << drop) - 1u)) == (1u << (drop - 1));
}
template <bool BF> CRM_DEV uint16_t round_to16(float a, int dir) {
  return BF ? round_to_bf16(a, dir) : round_to_f16(a, dir);
}
// 16-bit result in mode rm from (c, sg), c within one binary32 ulp of v = f(x).  Directed:
// round RD32(v) down or RU32(v) up.  To nearest: the format's midpoints are binary32
// numbers, so none lies strictly between v and c; RN16(v) = RN16(c) unless c is a
// midpoint, where sg says on which side v lies (sg = 0: v = c, ties to even).
template <bool BF> CRM_DEV uint16_t finish_16(float c, int sg, int rm) {
  if (c != c) return round_to16<BF>(c, 2);
  const bool neg = v_negative(c, sg);
  if (rm == CRM_RM_RD || (rm == CRM_RM_RZ && !neg)) return round_to16<BF>(rd32(c, sg), -1);
  if (rm == CRM_RM_RU || rm == CRM_RM_RZ) return round_to16<BF>(ru32(c, sg), 1);
  return round_to16<BF>(c, (sg != 0 && is_mid16<BF>(c)) ? sg : 2);
}
// 16-bit input to binary32 (exact)
template <bool BF> CRM_DEV float from16(uint16_t h) {
  if (BF) return bitsf((uint32_t)h << 16);
  const uint32_t sgn = (uint32_t)(h & 0x8000u) << 16, e = (h >> 10) & 0x1Fu, m = h & 0x3FFu;
  if (e == 0x1Fu) return bitsf(sgn | 0x7F800000u | (m << 13));  // inf, NaN (payload kept)
  if (e != 0) return bitsf(sgn | ((e + 112u) << 23) | (m << 13));
  return bitsf(sgn | fbits((float)m * 0x1p-24f));  // subnormal or zero: exact
}

// binary64 neighbours and result in mode rm
CRM_DEV double next_up_d(double c) {
  const uint64_t b = dbits(c);
  if ((b & 0x7FFFFFFFFFFFFFFFull) == 0) return bitsd(1ull);
  return bitsd((b >> 63) ? b - 1ull : b + 1ull);
}
CRM_DEV double next_down_d(double c) {
  const uint64_t b = dbits(c);
  if ((b & 0x7FFFFFFFFFFFFFFFull) == 0) return bitsd(0x8000000000000001ull);
  return bitsd((b >> 63) ? b + 1ull : b - 1ull);
}
CRM_DEV double finish_f64(double c, int sg, int rm) {
  if (c != c) return c;
  const bool neg = c != 0.0 ? c < 0.0 : (sg != 0 ? sg < 0 : (dbits(c) >> 63) != 0);
  if (rm == CRM_RM_RD || (rm == CRM_RM_RZ && !neg)) return sg < 0 ? next_down_d(c) : c;
  if (rm == CRM_RM_RU || rm == CRM_RM_RZ) return sg > 0 ? next_up_d(c) : c;
  return c;
}

// ------------------------------------------------------------------ misc
// Block-cooperative copy of a table into shared memory (bytes a multiple of 4).
CRM_DEV void copy_tab(void *dst, const void *src, int bytes) {
  const uint32_t *s = (const uint32_t *)src;
  uint32_t *d = (uint32_t *)dst;
  for (int i = threadIdx.x; i < bytes / 4; i += blockDim.x) d[i] = s[i];
}

CRM_DEV float qnan_of(float x) { return bitsf(fbits(x) | 0x00400000u); }
// The hardware reciprocal square root, rsqrt.approx.ftz.f32: relative error below 2^-22.9
// for a normal argument (a subnormal one is flushed to zero; callers pass normal ones).
CRM_DEV float rsqrt_hw(float a) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
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
